// The device state owned by a geneo handle, and the phase entry points the
// setup orchestration calls.
#pragma once

#include "common.cuh"

struct geneo_handle_s {
  geneo::DevMem mem;        // everything the handle keeps
  cudaStream_t stream = 0;  // stream of the last synchronising call
  cudaStream_t aux = nullptr;       // second stream (coarse solve, concurrent factorisations)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_afac = nullptr;   // end of the A_j factorisation on the aux stream
  geneo::SolveStreams solve_streams;  // lanes of the size-class band solves
  geneo::SolveSet setA;               // the A_j factors in size classes (local solves)
  geneo_options_t opt{};
  bool fp32 = false;

  // global problem (device copies)
  int64_t n = 0, nnz = 0;
  int64_t* rowptr = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;
  uint8_t* dir = nullptr;

  // subdomains
  int N = 0;
  int64_t sumN = 0;                // total rows of all N_j
  std::vector<geneo::SubDesc> hsub;
  geneo::SubDesc* dsub = nullptr;
  int32_t* Nlist = nullptr;        // [sumN] global dof of each N-row
  int32_t* Dlist = nullptr;        // [sumN] D_j stored at offN (first nD entries)
  int32_t* dpos = nullptr;         // [sumN] position in N_j of D entry
  int32_t* nToD = nullptr;         // [sumN] D index of an N-row or -1
  double* pu = nullptr;            // [sumN] X_j on N_j

  // inverse map global dof -> (subdomain, D index), sorted by subdomain
  int64_t* invD_ptr = nullptr;     // [n+1]
  int32_t* invD_sub = nullptr;
  int32_t* invD_loc = nullptr;

  // Dirichlet band factors
  void* bandA = nullptr;           // double or float
  geneo::BandDesc* dbandA = nullptr;
  int maxwA = 0;
  int maxnD = 0;                   // largest Dirichlet dof count
  // FP32 mode: A_j whose FP32 factorisation had a weak pivot, factored in
  // FP64 (their FP32 descriptors get n = 0)
  double* bandA64 = nullptr;
  geneo::BandDesc* dbandA64 = nullptr;
  int nA64 = 0, maxwA64 = 0, maxnA64 = 0;
  std::vector<uint8_t> a64;        // [N] 1: A_j factored in FP64
  int nK64 = 0;                    // the same count for K_j (setup only)
  int factor_classes = 0;          // FP32: factorisation batches (size classes) of K_j and A_j
  int local_stages = 0;            // pipeline depth of the local solve picked by the autotuner

  // coarse space
  int dimH = 0, wH = 0;
  int maxm = 0;
  double* Z = nullptr;             // per subdomain nD x m, column-major
  double* bandH = nullptr;         // band factor of A_H
  geneo::BandDesc* dbandH = nullptr;
  int64_t* xoffH = nullptr;        // {0}
  double* Hinv = nullptr;          // A_H^{-1} (dimH x dimH), or NULL: band solves
  double* yH = nullptr;            // [dimH] coarse solution
  // SELL-32 copy of A for the PCG products: slice s holds rows 32 s .. 32 s
  // + 31, entry t of row 32 s + l at sell_off[s] + 32 t + l (padding: value
  // 0, column of the row itself)
  int64_t* sell_off = nullptr;     // [n/32 + 1]
  int32_t* sell_col = nullptr;
  double* sell_val = nullptr;
  int64_t sell_nnz = 0;
  int spmv_blocks = 1024;          // grid of the SELL product (resident blocks)
  std::vector<double> lambda_host; // [N * s] ascending lambda per subdomain
  int s_block = 0;
  int eig_iters = 0;
  int eig_second_pass = 0;         // subdomains solved again with the full block
  int eig_o64 = 0;                 // FP32 mode: subdomains orthogonalised in FP64
  int eig_unconv = 0;              // subdomains left unconverged at eig_maxit

  // apply / PCG work
  double* u = nullptr;             // [sumD] local solutions
  int64_t* uoff = nullptr;         // [N] offsets into u (= offN)
  double* cH = nullptr;            // [dimH] coarse vector
  double *r = nullptr, *zv = nullptr, *p = nullptr, *q = nullptr, *x = nullptr;
  double* red = nullptr;           // reduction scratch
  double* scal = nullptr;          // device scalars
  double* hpin = nullptr;          // pinned host scalars
  int red_blocks = 0;

  double factor_flops = 0, factor_ms = 0, eig_flops = 0, eig_ms = 0;
  double apply_flops = 0, apply_bytes = 0;
  double local_solve_flops = 0, local_solve_bytes = 0, spmv_flops = 0, spmv_bytes = 0;
  double* hist = nullptr;          // PCG alpha/beta history (2 * hist_cap)
  int hist_cap = 0;
  std::vector<double> pcg_host;    // host work of geneo_pcg_solve_noalloc (sized at setup)
  // several right-hand sides at once (solve_block.cu): n x kBlk blocks and
  // the subdomain vectors of kBlk columns, allocated on first use
  double *blk_r = nullptr, *blk_z = nullptr, *blk_p = nullptr, *blk_q = nullptr, *blk_t = nullptr;
  double *blk_u = nullptr, *blk_c = nullptr, *blk_y = nullptr, *blk_part = nullptr, *blk_scal = nullptr;
  int32_t* blk_mask = nullptr;
  int64_t* blk_uoff = nullptr;
  int device = -1;                 // device the handle was set up on

  geneo::KernelProfiler prof;

  geneo::DevStatus* dstat = nullptr;
  geneo::DevStatus hstat{};
  double setup_ms[8] = {0};
};

namespace geneo {
geneo_status_t check_status(geneo_handle_s* h, cudaStream_t s);

// assembly.cu
struct AssemblyOut {
  // local CSR over N-rows (pattern of A restricted to N_j x N_j)
  int64_t* lrow = nullptr;  // [sumN+1]
  int32_t* lcol = nullptr;
  double* lK = nullptr;     // K = Atilde - sigma B
  double* lB = nullptr;     // B = X A^o X  (or X Atilde X)
  double* lA = nullptr;     // A on the local pattern
  int64_t lnnz = 0;
  int32_t* e_tau = nullptr;    // element multiplicity (number of subdomains)
  int32_t* cnt_all = nullptr;  // elements per dof
  void* bandK = nullptr;
  BandDesc* dbandK = nullptr;
  int maxwK = 0;
  std::vector<BandDesc> hbandK, hbandA;  // host copies of the solve descriptors
  int32_t* weak = nullptr;  // [2N] FP32 factorisations with a weak pivot (K_j, A_j)
  // K_j factored again in FP64
  double* bandK64 = nullptr;
  BandDesc* dbandK64 = nullptr;
  int nK64 = 0, maxwK64 = 0, maxnK64 = 0;
};
geneo_status_t build_structure(geneo_handle_s* h, const geneo_problem_t* p, AssemblyOut& a,
                               DevMem& tmp, cudaStream_t s);
geneo_status_t assemble_local(geneo_handle_s* h, const geneo_problem_t* p, AssemblyOut& out,
                              DevMem& tmp, cudaStream_t s, double* ms_assembly,
                              double* ms_factor);
// FP32 mode, after the A_j factorisation has finished: factor in FP64 the A_j
// flagged weak (adaptive precision per subdomain).
geneo_status_t refactor_weak_A(geneo_handle_s* h, AssemblyOut& a, DevMem& tmp, cudaStream_t s);

// lobpcg.cu
geneo_status_t local_eigensolve(geneo_handle_s* h, AssemblyOut& a, DevMem& tmp, cudaStream_t s,
                                double** X_out, int64_t* ld_unused);

// coarse.cu
geneo_status_t build_coarse(geneo_handle_s* h, const AssemblyOut& a, const double* X,
                            DevMem& tmp, cudaStream_t s, double* ms_basis, double* ms_matrix,
                            double* ms_factor);

// solve.cu
// Condition estimate lambda_max / lambda_min of the Lanczos tridiagonal
// matrix of CG coefficients a[0..m), b[0..m-1) (bisection; work d, e of m).
double condition_estimate_fixed(const double* a, const double* b, int m, double* d, double* e);
geneo_status_t alloc_solver(geneo_handle_s* h);
// time the local solve's pipeline depths on this batch once per shape
geneo_status_t tune_local_solve(geneo_handle_s* h);
geneo_status_t apply_prec(geneo_handle_s* h, const double* r, double* z, cudaStream_t s);
geneo_status_t pcg(geneo_handle_s* h, const double* b, double* x, double tol, int maxit,
                   geneo_solve_info_t* info, cudaStream_t s);
// solve_block.cu: k <= kBlk right-hand sides at once (stride n, device)
constexpr int kBlk = 8;
geneo_status_t pcg_block(geneo_handle_s* h, const double* b, double* x, int k, double tol, int maxit,
                         geneo_solve_info_t* info, cudaStream_t s);
}  // namespace geneo
