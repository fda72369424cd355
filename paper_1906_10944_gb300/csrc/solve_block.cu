// Preconditioned CG for several right-hand sides at once (Section 5, one
// system matrix, k <= kBlk right-hand sides): k independent CG recurrences
// advanced in lockstep, so each iteration streams A and the subdomain
// factors once for all k vectors.  Per iteration: Q = A P (SELL-32 product
// of k columns), alpha_c = rz_c / p_c.q_c, X += P alpha, R -= Q alpha,
// Z = M^{-1} R (restriction of k columns, the banded local solves with k
// right-hand sides, the coarse product A_H^{-1} C with k columns, the
// prolongation), beta_c = rz_c' / rz_c, P = Z + P beta.  Each column has
// its own scalars, its own stopping test (true residual, replacement and
// restart exactly as the one-vector solve in solve.cu) and stops on its
// own; a stopped column keeps its x (alpha = 0) while the others go on.
// All inner products are fixed-order two-stage reductions.
#include <algorithm>
#include <cmath>
#include <vector>

#include "handle.cuh"

namespace geneo {
namespace {

constexpr int kT = 256;
constexpr int kNb = 512;   // blocks of the vector kernels (partials per column)
constexpr int kSl = 16;    // scalar slots per column
// slots: 0 rz, 1 alpha, 2 beta, 3 rr, 4 pq, 5 bb, 6 flag, 7 true rr,
//        8 active (1.0 / 0.0), 9 restart (1.0: beta = 0 at the next update)

// Q = A P for k columns (SELL-32, thread per row, a slice per warp):
// partial p_c.q_c per block
__global__ void __launch_bounds__(kT)
k_spmm_sell_cols(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ scol,
                 const double* __restrict__ sval, const double* __restrict__ P, double* __restrict__ Q, int k,
                 double* __restrict__ part) {
  __shared__ double red[kT / 32];
  const int l = threadIdx.x & 31;
  const int64_t nsl = (n + 31) / 32;
  double dsum[kBlk];
#pragma unroll
  for (int c = 0; c < kBlk; ++c) dsum[c] = 0.0;
  for (int64_t sl = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; sl < nsl;
       sl += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t o = off[sl] + l;
    const int w = (int)((off[sl + 1] - off[sl]) >> 5);
    double acc[kBlk];
#pragma unroll
    for (int c = 0; c < kBlk; ++c) acc[c] = 0.0;
    for (int t = 0; t < w; ++t) {
      const int64_t e = o + 32 * (int64_t)t;
      const double v = sval[e];
      const int64_t cc = scol[e];
#pragma unroll
      for (int c = 0; c < kBlk; ++c)
        if (c < k) acc[c] += v * P[c * n + cc];
    }
    const int64_t r = sl * 32 + l;
    if (r < n) {
#pragma unroll
      for (int c = 0; c < kBlk; ++c)
        if (c < k) {
          Q[c * n + r] = acc[c];
          dsum[c] += acc[c] * P[c * n + r];
        }
    }
  }
  for (int c = 0; c < k; ++c) {
    const double sc = block_sum(dsum[c], red);
    if (threadIdx.x == 0) part[(int64_t)c * kNb + blockIdx.x] = sc;
  }
}

// R_c = B_c - A X_c for k columns; partial r_c.r_c per block
__global__ void __launch_bounds__(kT)
k_resid_sell_cols(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ scol,
                  const double* __restrict__ sval, const double* __restrict__ X, const double* __restrict__ B,
                  double* __restrict__ Rt, int k, double* __restrict__ part) {
  __shared__ double red[kT / 32];
  const int l = threadIdx.x & 31;
  const int64_t nsl = (n + 31) / 32;
  double rs[kBlk];
#pragma unroll
  for (int c = 0; c < kBlk; ++c) rs[c] = 0.0;
  for (int64_t sl = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; sl < nsl;
       sl += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t o = off[sl] + l;
    const int w = (int)((off[sl + 1] - off[sl]) >> 5);
    double acc[kBlk];
#pragma unroll
    for (int c = 0; c < kBlk; ++c) acc[c] = 0.0;
    for (int t = 0; t < w; ++t) {
      const int64_t e = o + 32 * (int64_t)t;
      const double v = sval[e];
      const int64_t cc = scol[e];
#pragma unroll
      for (int c = 0; c < kBlk; ++c)
        if (c < k) acc[c] += v * X[c * n + cc];
    }
    const int64_t r = sl * 32 + l;
    if (r < n) {
#pragma unroll
      for (int c = 0; c < kBlk; ++c)
        if (c < k) {
          const double ri = B[c * n + r] - acc[c];
          Rt[c * n + r] = ri;
          rs[c] += ri * ri;
        }
    }
  }
  for (int c = 0; c < k; ++c) {
    const double sc = block_sum(rs[c], red);
    if (threadIdx.x == 0) part[(int64_t)c * kNb + blockIdx.x] = sc;
  }
}

// partial a_c.b_c per block for k columns
__global__ void __launch_bounds__(kT)
k_dot_cols(int64_t n, const double* __restrict__ A, const double* __restrict__ B, int k, double* __restrict__ part) {
  __shared__ double red[kT / 32];
  for (int c = 0; c < k; ++c) {
    double s = 0.0;
    const double* a = A + (int64_t)c * n;
    const double* b = B + (int64_t)c * n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
      s += a[i] * b[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[(int64_t)c * kNb + blockIdx.x] = s;
  }
}

// per column (block c): the sum of its partials, then the scalar step `what`
// (as k_finish in solve.cu); inactive columns keep alpha = 0
__global__ void k_finish_cols(const double* __restrict__ part, double* __restrict__ scal, int what,
                              double* __restrict__ hist_a, double* __restrict__ hist_b, int hcap, int it) {
  __shared__ double red[kT / 32];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < kNb; i += blockDim.x) s += part[(int64_t)c * kNb + i];
  s = block_sum(s, red);
  if (threadIdx.x != 0) return;
  double* sc = scal + c * kSl;
  const bool act = sc[8] != 0.0;
  if (what == 0) {          // rz of a (re)start
    sc[0] = s;
    if (act && !(s > 0.0)) sc[6] = 1.0;
  } else if (what == 1) {   // alpha = rz / pq
    sc[4] = s;
    if (!act) {
      sc[1] = 0.0;
    } else if (!(s > 0.0)) {
      sc[6] = 1.0;
      sc[1] = 0.0;
    } else {
      sc[1] = sc[0] / s;
    }
    if (act) hist_a[(int64_t)c * hcap + it] = sc[1];
  } else if (what == 2) {   // rr
    sc[3] = s;
  } else if (what == 3) {   // beta = rz_new / rz (0 after a restart)
    if (act && !(s > 0.0)) sc[6] = 1.0;
    const bool rs = sc[9] != 0.0;
    sc[2] = (rs || !(sc[0] > 0.0)) ? 0.0 : s / sc[0];
    sc[0] = s;
    sc[9] = 0.0;
    if (act && !rs) hist_b[(int64_t)c * hcap + it] = sc[2];
  } else if (what == 4) {   // bb
    sc[5] = s;
  } else if (what == 5) {   // true rr
    sc[7] = s;
  }
}

// X_c += alpha_c P_c, R_c -= alpha_c Q_c; partial r_c.r_c per block
__global__ void __launch_bounds__(kT)
k_update_xr_cols(int64_t n, const double* __restrict__ scal, const double* __restrict__ P,
                 const double* __restrict__ Q, double* __restrict__ X, double* __restrict__ R, int k,
                 double* __restrict__ part) {
  __shared__ double red[kT / 32];
  for (int c = 0; c < k; ++c) {
    const double alpha = scal[c * kSl + 1];
    double s = 0.0;
    const int64_t o = (int64_t)c * n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
      X[o + i] += alpha * P[o + i];
      const double ri = R[o + i] - alpha * Q[o + i];
      R[o + i] = ri;
      s += ri * ri;
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[(int64_t)c * kNb + blockIdx.x] = s;
  }
}

// P_c = Z_c + beta_c P_c (active columns)
__global__ void k_update_p_cols(int64_t n, const double* __restrict__ scal, const double* __restrict__ Z,
                                double* __restrict__ P, int k) {
  for (int c = 0; c < k; ++c) {
    if (scal[c * kSl + 8] == 0.0) continue;
    const double beta = scal[c * kSl + 2];
    const int64_t o = (int64_t)c * n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
      P[o + i] = Z[o + i] + beta * P[o + i];
  }
}

// column c of Dst = column c of Src where mask[c] != 0 (replacement)
__global__ void k_copy_masked(int64_t n, const double* __restrict__ Src, double* __restrict__ Dst, int k,
                              const int32_t* __restrict__ mask) {
  for (int c = 0; c < k; ++c) {
    if (!mask[c]) continue;
    const int64_t o = (int64_t)c * n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
      Dst[o + i] = Src[o + i];
  }
}

// restriction of k columns: U_j (nD_j x k at k offN_j) and C (dimH x k)
__global__ void __launch_bounds__(kT)
k_restrict_cols(const SubDesc* __restrict__ sub, const int32_t* __restrict__ Dlist, const double* __restrict__ R,
                int64_t n, const double* __restrict__ Z, double* __restrict__ U, double* __restrict__ C, int dimH,
                int k) {
  const int j = blockIdx.x;
  const SubDesc d = sub[j];
  __shared__ double red[kT / 32];
  const int32_t* Dj = Dlist + d.offN;
  double* uj = U + (int64_t)k * d.offN;
  for (int c = 0; c < k; ++c)
    for (int i = threadIdx.x; i < d.nD; i += blockDim.x) uj[(int64_t)c * d.nD + i] = R[c * n + Dj[i]];
  const double* zj = Z + d.offZ;
  for (int c = 0; c < k; ++c)
    for (int m = 0; m < d.m; ++m) {
      double s = 0.0;
      for (int i = threadIdx.x; i < d.nD; i += blockDim.x) s += zj[(int64_t)m * d.nD + i] * R[c * n + Dj[i]];
      s = block_sum(s, red);
      if (threadIdx.x == 0) C[(int64_t)c * dimH + d.offH + m] = s;
    }
}

// Y = X C with X = A_H^{-1} (row i read as column i): one warp per row
__global__ void __launch_bounds__(kT)
k_coarse_gemm(const double* __restrict__ X, int dim, const double* __restrict__ C, double* __restrict__ Y, int k) {
  const int lane = threadIdx.x & 31;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < dim; i += (gridDim.x * blockDim.x) >> 5) {
    const double* xi = X + (int64_t)i * dim;
    double a[kBlk];
#pragma unroll
    for (int c = 0; c < kBlk; ++c) a[c] = 0.0;
    for (int jj = lane; jj < dim; jj += 32) {
      const double v = xi[jj];
#pragma unroll
      for (int c = 0; c < kBlk; ++c)
        if (c < k) a[c] += v * C[(int64_t)c * dim + jj];
    }
#pragma unroll
    for (int c = 0; c < kBlk; ++c)
      if (c < k) {
        const double t = warp_sum(a[c]);
        if (lane == 0) Y[(int64_t)c * dim + i] = t;
      }
  }
}

// prolongation of k columns (gather form, as k_prolong in solve.cu)
__global__ void __launch_bounds__(kT)
k_prolong_cols(int64_t n, const uint8_t* __restrict__ dir, const double* __restrict__ R,
               const int64_t* __restrict__ invD_ptr, const int32_t* __restrict__ invD_sub,
               const int32_t* __restrict__ invD_loc, const SubDesc* __restrict__ sub, const double* __restrict__ U,
               const double* __restrict__ Z, const double* __restrict__ Y, int dimH, double* __restrict__ Zout,
               int k) {
  for (int64_t kk = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; kk < n; kk += (int64_t)gridDim.x * blockDim.x) {
    if (dir[kk]) {
      for (int c = 0; c < k; ++c) Zout[c * n + kk] = R[c * n + kk];
      continue;
    }
    double acc[kBlk];
#pragma unroll
    for (int c = 0; c < kBlk; ++c) acc[c] = 0.0;
    for (int64_t t = invD_ptr[kk]; t < invD_ptr[kk + 1]; ++t) {
      const int j = invD_sub[t], i = invD_loc[t];
      const SubDesc& d = sub[j];
      const double* uj = U + (int64_t)k * d.offN + i;
      const double* zr = Z + d.offZ + i;
#pragma unroll
      for (int c = 0; c < kBlk; ++c) {
        if (c >= k) break;
        double v = uj[(int64_t)c * d.nD];
        if (Y)
          for (int m = 0; m < d.m; ++m) v += zr[(int64_t)m * d.nD] * Y[(int64_t)c * dimH + d.offH + m];
        acc[c] += v;
      }
    }
#pragma unroll
    for (int c = 0; c < kBlk; ++c)
      if (c < k) Zout[c * n + kk] = acc[c];
  }
}

double cond_est(const double* a, const double* b, int m, std::vector<double>& d, std::vector<double>& e) {
  if (m <= 0) return 1.0;
  d.assign(m, 0.0);
  e.assign(std::max(m, 1), 0.0);
  return condition_estimate_fixed(a, b, m, d.data(), e.data());
}

}  // namespace

// Z = M^{-1} R for k <= kBlk columns (stride n); the block buffers of the
// handle hold the subdomain vectors.
geneo_status_t apply_prec_cols(geneo_handle_s* h, const double* R, double* Zo, int k, cudaStream_t s) {
  const int N = h->N;
  k_restrict_cols<<<N, kT, 0, s>>>(h->dsub, h->Dlist, R, h->n, h->Z, h->blk_u, h->blk_c, std::max(h->dimH, 1), k);
  note_launch();
  GENEO_CUDA(cudaGetLastError());
  const double* Y = nullptr;
  if (h->dimH > 0) {
    if (!h->Hinv) return GENEO_ERR_ARG;  // the block solve needs the dense coarse inverse
    const int g = std::min(ceil_div(h->dimH, kT / 32), 152 * 8);
    k_coarse_gemm<<<g, kT, 0, s>>>(h->Hinv, h->dimH, h->blk_c, h->blk_y, k); note_launch();
    GENEO_CUDA(cudaGetLastError());
    Y = h->blk_y;
  }
  const int pl = h->prof.begin(GENEO_PROF_LOCAL_SOLVE, h->local_solve_flops * k, h->local_solve_bytes, s);
  GENEO_TRY(solve_set_run(h->setA, h->solve_streams, h->blk_u, h->blk_uoff, k, nullptr, nullptr, h->dstat, s));
  h->prof.end(pl, s);
  const int grid = (int)std::min<int64_t>((h->n + kT - 1) / kT, 152 * 8);
  k_prolong_cols<<<grid, kT, 0, s>>>(h->n, h->dir, R, h->invD_ptr, h->invD_sub, h->invD_loc, h->dsub, h->blk_u,
                                     h->Z, Y, std::max(h->dimH, 1), Zo, k);
  note_launch();
  GENEO_CUDA(cudaGetLastError());
  return GENEO_OK;
}

geneo_status_t block_buffers(geneo_handle_s* h) {
  if (h->blk_r) return GENEO_OK;
  DevMem& M = h->mem;
  const size_t nk = (size_t)h->n * kBlk;
  GENEO_TRY(M.get(&h->blk_r, nk));
  GENEO_TRY(M.get(&h->blk_z, nk));
  GENEO_TRY(M.get(&h->blk_p, nk));
  GENEO_TRY(M.get(&h->blk_q, nk));
  GENEO_TRY(M.get(&h->blk_t, nk));
  GENEO_TRY(M.get(&h->blk_u, (size_t)h->sumN * kBlk));
  GENEO_TRY(M.get(&h->blk_c, (size_t)std::max(h->dimH, 1) * kBlk));
  GENEO_TRY(M.get(&h->blk_y, (size_t)std::max(h->dimH, 1) * kBlk));
  GENEO_TRY(M.get(&h->blk_part, (size_t)kNb * kBlk));
  GENEO_TRY(M.get(&h->blk_scal, (size_t)kSl * kBlk));
  GENEO_TRY(M.get(&h->blk_mask, (size_t)kBlk));
  GENEO_TRY(M.get(&h->blk_uoff, (size_t)h->N));
  return GENEO_OK;
}

// k right-hand sides b (stride n) into x (stride n), device arrays.
geneo_status_t pcg_block(geneo_handle_s* h, const double* b, double* x, int k, double tol, int maxit,
                         geneo_solve_info_t* info, cudaStream_t s) {
  if (k < 1 || k > kBlk) return GENEO_ERR_ARG;
  h->mem.stream = s;
  GENEO_TRY(block_buffers(h));
  const int64_t n = h->n;
  {
    // subdomain vector offsets for k columns: subdomain j at k offN_j
    std::vector<int64_t> off(h->N);
    for (int j = 0; j < h->N; ++j) off[j] = (int64_t)k * h->hsub[j].offN;
    GENEO_CUDA(cudaMemcpyAsync(h->blk_uoff, off.data(), sizeof(int64_t) * h->N, cudaMemcpyHostToDevice, s));
  }
  const int cap = std::max(maxit, 1) + 1;
  double *ha_d = nullptr, *hb_d = nullptr;
  DevMem tmp;
  tmp.stream = s;
  GENEO_TRY(tmp.get(&ha_d, (size_t)cap * k));
  GENEO_TRY(tmp.get(&hb_d, (size_t)cap * k));
  double* scal = h->blk_scal;
  double* part = h->blk_part;
  double *R = h->blk_r, *Zv = h->blk_z, *P = h->blk_p, *Q = h->blk_q, *T = h->blk_t;
  std::vector<double> hs((size_t)kSl * k);
  auto read_scal = [&]() -> geneo_status_t {
    GENEO_CUDA(cudaMemcpyAsync(hs.data(), scal, sizeof(double) * kSl * k, cudaMemcpyDeviceToHost, s));
    GENEO_CUDA(cudaStreamSynchronize(s));
    return GENEO_OK;
  };
  auto set_scal = [&]() -> geneo_status_t {
    GENEO_CUDA(cudaMemcpyAsync(scal, hs.data(), sizeof(double) * kSl * k, cudaMemcpyHostToDevice, s));
    return GENEO_OK;
  };
  GENEO_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n * k, s));
  GENEO_CUDA(cudaMemcpyAsync(R, b, sizeof(double) * n * k, cudaMemcpyDeviceToDevice, s));
  std::fill(hs.begin(), hs.end(), 0.0);
  for (int c = 0; c < k; ++c) hs[c * kSl + 8] = 1.0;
  GENEO_TRY(set_scal());
  k_dot_cols<<<kNb, kT, 0, s>>>(n, b, b, k, part); note_launch();
  k_finish_cols<<<k, kT, 0, s>>>(part, scal, 4, ha_d, hb_d, cap, 0); note_launch();
  GENEO_CUDA(cudaGetLastError());
  GENEO_TRY(read_scal());
  std::vector<double> bnorm(k), rel(k, 1.0), rel_true(k, NAN), last_true(k, INFINITY);
  std::vector<int> replaced(k, 0), n_lanczos(k, -1), its(k, 0), state(k, 0);  // state 0 run, 1 done, 2 stop
  std::vector<int32_t> mask(k, 0);
  bool nonfinite = false;
  for (int c = 0; c < k; ++c) {
    bnorm[c] = std::sqrt(hs[c * kSl + 5]);
    if (!std::isfinite(bnorm[c])) nonfinite = true;
    if (bnorm[c] == 0.0 || !std::isfinite(bnorm[c])) {
      state[c] = bnorm[c] == 0.0 ? 1 : 2;
      hs[c * kSl + 8] = 0.0;
      rel[c] = rel_true[c] = 0.0;
    }
  }
  GENEO_TRY(set_scal());
  auto restart_all = [&]() -> geneo_status_t {  // Z = M^{-1} R, P = Z, rz (all columns)
    GENEO_TRY(apply_prec_cols(h, R, Zv, k, s));
    GENEO_CUDA(cudaMemcpyAsync(P, Zv, sizeof(double) * n * k, cudaMemcpyDeviceToDevice, s));
    k_dot_cols<<<kNb, kT, 0, s>>>(n, R, Zv, k, part); note_launch();
    k_finish_cols<<<k, kT, 0, s>>>(part, scal, 0, ha_d, hb_d, cap, 0); note_launch();
    GENEO_CUDA(cudaGetLastError());
    return GENEO_OK;
  };
  GENEO_TRY(restart_all());
  int it = 0;
  auto running = [&]() {
    for (int c = 0; c < k; ++c)
      if (state[c] == 0) return true;
    return false;
  };
  while (it < maxit && it < cap - 1 && running()) {
    {
      const int pv = h->prof.begin(GENEO_PROF_SPMV, h->spmv_flops * k, h->spmv_bytes, s);
      k_spmm_sell_cols<<<kNb, kT, 0, s>>>(n, h->sell_off, h->sell_col, h->sell_val, P, Q, k, part); note_launch();
      h->prof.end(pv, s);
    }
    k_finish_cols<<<k, kT, 0, s>>>(part, scal, 1, ha_d, hb_d, cap, it); note_launch();
    k_update_xr_cols<<<kNb, kT, 0, s>>>(n, scal, P, Q, x, R, k, part); note_launch();
    k_finish_cols<<<k, kT, 0, s>>>(part, scal, 2, ha_d, hb_d, cap, it); note_launch();
    GENEO_CUDA(cudaGetLastError());
    GENEO_TRY(read_scal());
    ++it;
    bool check = false;
    for (int c = 0; c < k; ++c) {
      if (state[c] != 0) continue;
      its[c] = it;
      if (hs[c * kSl + 6] != 0.0) {  // breakdown
        state[c] = 2;
        hs[c * kSl + 8] = 0.0;
        continue;
      }
      rel[c] = std::sqrt(hs[c * kSl + 3]) / bnorm[c];
      if (!std::isfinite(rel[c])) {
        nonfinite = true;
        state[c] = 2;
        hs[c * kSl + 8] = 0.0;
        continue;
      }
      if (rel[c] <= tol) check = true;
    }
    std::fill(mask.begin(), mask.end(), 0);
    if (check) {
      k_resid_sell_cols<<<kNb, kT, 0, s>>>(n, h->sell_off, h->sell_col, h->sell_val, x, b, T, k, part); note_launch();
      k_finish_cols<<<k, kT, 0, s>>>(part, scal, 5, ha_d, hb_d, cap, it); note_launch();
      GENEO_CUDA(cudaGetLastError());
      GENEO_TRY(read_scal());
      for (int c = 0; c < k; ++c) {
        if (state[c] != 0 || !(rel[c] <= tol)) continue;
        rel_true[c] = std::sqrt(hs[c * kSl + 7]) / bnorm[c];
        if (rel_true[c] <= tol) {
          state[c] = 1;
        } else if (replaced[c] >= 5 || !(rel_true[c] <= 0.5 * last_true[c])) {
          state[c] = 2;
        } else {
          last_true[c] = rel_true[c];
          ++replaced[c];
          if (n_lanczos[c] < 0) n_lanczos[c] = it;
          mask[c] = 1;
          hs[c * kSl + 9] = 1.0;  // beta = 0 at this iteration's update
        }
        if (state[c] != 0) hs[c * kSl + 8] = 0.0;
      }
    }
    GENEO_TRY(set_scal());
    if (!running()) break;
    bool any_mask = false;
    for (int c = 0; c < k; ++c) any_mask |= mask[c] != 0;
    if (any_mask) {
      GENEO_CUDA(cudaMemcpyAsync(h->blk_mask, mask.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, s));
      k_copy_masked<<<kNb, kT, 0, s>>>(n, T, R, k, h->blk_mask); note_launch();
    }
    GENEO_TRY(apply_prec_cols(h, R, Zv, k, s));
    k_dot_cols<<<kNb, kT, 0, s>>>(n, R, Zv, k, part); note_launch();
    k_finish_cols<<<k, kT, 0, s>>>(part, scal, 3, ha_d, hb_d, cap, it - 1); note_launch();
    k_update_p_cols<<<kNb, kT, 0, s>>>(n, scal, Zv, P, k); note_launch();
    GENEO_CUDA(cudaGetLastError());
  }
  // columns still running at the cap: their true residual
  bool left = false;
  for (int c = 0; c < k; ++c) left |= state[c] == 0 || !std::isfinite(rel_true[c]);
  if (left) {
    k_resid_sell_cols<<<kNb, kT, 0, s>>>(n, h->sell_off, h->sell_col, h->sell_val, x, b, T, k, part); note_launch();
    k_finish_cols<<<k, kT, 0, s>>>(part, scal, 5, ha_d, hb_d, cap, it); note_launch();
    GENEO_CUDA(cudaGetLastError());
    GENEO_TRY(read_scal());
    for (int c = 0; c < k; ++c)
      if (state[c] == 0 || !std::isfinite(rel_true[c]))
        rel_true[c] = bnorm[c] > 0.0 ? std::sqrt(hs[c * kSl + 7]) / bnorm[c] : 0.0;
  }
  bool all_conv = true, any_break = false;
  for (int c = 0; c < k; ++c) {
    if (!(rel_true[c] <= tol) && bnorm[c] != 0.0) all_conv = false;
    if (hs[c * kSl + 6] != 0.0) any_break = true;
  }
  if (info) {
    const int c = k - 1;  // the last right-hand side, as geneo_pcg_solve reports
    std::vector<double> ha(cap), hb(cap), dd, ee;
    GENEO_CUDA(cudaMemcpyAsync(ha.data(), ha_d + (int64_t)c * cap, sizeof(double) * cap, cudaMemcpyDeviceToHost, s));
    GENEO_CUDA(cudaMemcpyAsync(hb.data(), hb_d + (int64_t)c * cap, sizeof(double) * cap, cudaMemcpyDeviceToHost, s));
    GENEO_CUDA(cudaStreamSynchronize(s));
    const int nal = std::min(n_lanczos[c] >= 0 ? n_lanczos[c] : its[c], cap);
    info->iterations = its[c];
    info->converged = bnorm[c] == 0.0 || rel_true[c] <= tol;
    info->rel_residual = rel[c];
    info->true_residual = rel_true[c];
    info->replacements = replaced[c];
    info->kappa_estimate = bnorm[c] == 0.0 ? 1.0 : cond_est(ha.data(), hb.data(), nal, dd, ee);
    info->resid_hist_len = 0;
  }
  GENEO_CUDA(cudaStreamSynchronize(s));
  tmp.free_all();
  GENEO_TRY(check_status(h, s));
  if (nonfinite) return GENEO_ERR_NONFINITE;
  if (any_break) return GENEO_ERR_BREAKDOWN;
  if (!all_conv) return GENEO_ERR_PCG_NOCONV;
  return GENEO_OK;
}

}  // namespace geneo
