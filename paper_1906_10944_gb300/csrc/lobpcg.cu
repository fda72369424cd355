// Batched shift-and-invert block eigensolver for the GenEO local problems.
//
// Section 3, eq. 5 and Section 4.3: Atilde_j p = lambda X_j A_j^o X_j p.
// Section 4.4: with K_j = Atilde_j - sigma B_j (B_j = X_j A_j^o X_j) the
// transformed problem B_j x = nu K_j x, nu = 1/(lambda - sigma), has the
// same eigenvectors and the wanted (smallest) lambda become the largest nu.
//
// The paper solves each transformed problem with ARPACK.  Here all
// subdomains are solved at once by a locally optimal block preconditioned
// conjugate-gradient iteration (LOBPCG) on the pencil (B_j, K_j), with the
// exact shift-invert operator K_j^{-1} (banded Cholesky factor) as the
// preconditioner.  Per iteration and subdomain:
//   R = B X - K X diag(nu)            residuals, relative norms rn_i
//   W = K^{-1} R[:, active]           active = columns with rn_i > tol
//   Q = [W, P], K-orthogonalised against X and K-orthonormalised, twice
//     (SVQB the first time, Cholesky QR the second, SVQB where it fails)
//   Rayleigh-Ritz on S = [X, Q] (S^T K S = I): eig(S^T B S), top s
//   P = Q U_Q, X = S U
// Stop when every Ritz pair below the threshold tau is converged and the
// first one at or above tau is converged too (or all nev_max in fixed-count
// mode).  Residuals are FP64.  With FP32 factors the first
// orthogonalisation pass runs in FP32 and the second, the block products,
// the Gram matrices and the Rayleigh-Ritz sweeps in double-single arithmetic
// (about 46 bits; the products and Gram matrices of the subdomains whose K_j
// needed FP64 stay FP64); with FP64 factors all of it is FP64.  The K^{-1} solves use the factor's
// precision.
//
// Dense small problems (at most kMaxW = 104 columns) are solved by parallel
// cyclic Jacobi in shared memory, one thread block per subdomain.
#include <algorithm>
#include <chrono>
#include <type_traits>
#include <cstdio>

#include "ds.cuh"
#include "handle.cuh"

namespace geneo {
namespace {

constexpr int kT = 256;
constexpr int kMaxW = 104;      // largest [X, Q] width handled by the dense kernels
constexpr int kRS = 4;          // row splits of the Gram kernel
constexpr int kRB = 32;         // rows per shared-memory chunk in the Gram kernel
constexpr int kMaxSweeps = 40;  // bound of the Jacobi sweep loop
constexpr int kFirstPassNev = 8; // wanted pairs of the narrow first pass
constexpr int kStallIts = 6;     // FP32 first passes: iterations without halving the residual
constexpr int kStallFrom = 12;   // ... counted from this iteration of a pass on
constexpr int kForce64From = 30; // FP32 mode: subdomains still iterating here switch to FP64

// A multivector operand: columns [c0 + c0d[j], + width) of a buffer holding W
// columns per subdomain (rows = nN_j, column-major, ld = nN_j), storage S
// (FP64 buffers, or the FP32 copies used by the first orthogonalisation pass).
template <typename S>
struct ColRefT {
  S* base;
  int W;
  int c0;
  const int32_t* c0d;
  int w;
  const int32_t* wd;
  const int32_t* wd2;  // width = w + wd[j] + wd2[j] (NULL terms are 0)
};
using ColRef = ColRefT<double>;
using ColRef32 = ColRefT<float>;

template <typename S>
__device__ __forceinline__ int cr_c0(const ColRefT<S>& r, int j) { return r.c0 + (r.c0d ? r.c0d[j] : 0); }
template <typename S>
__device__ __forceinline__ int cr_w(const ColRefT<S>& r, int j) {
  return r.w + (r.wd ? r.wd[j] : 0) + (r.wd2 ? r.wd2[j] : 0);
}
template <typename S>
__device__ __forceinline__ S* cr_ptr(const ColRefT<S>& r, const SubDesc& d, int j) {
  return r.base + d.offN * (int64_t)r.W + (int64_t)cr_c0(r, j) * d.nN;
}

template <typename S>
ColRefT<S> cref(S* base, int W, int c0, const int32_t* c0d, int w, const int32_t* wd,
                const int32_t* wd2 = nullptr) {
  return ColRefT<S>{base, W, c0, c0d, w, wd, wd2};
}

// ---------------------------------------------------------------------------
// Multivector kernels (grid: x = row blocks, y = subdomain).
// ---------------------------------------------------------------------------
// S is the storage and arithmetic type: double, or float for the first
// orthogonalisation pass (FP32 copies of the operand and of K's values, so
// nothing is converted in the inner loop).
template <typename S>
__global__ void __launch_bounds__(kT)
k_spmm(const SubDesc* __restrict__ sub, const int64_t* __restrict__ lrow,
       const int32_t* __restrict__ lcol, const S* __restrict__ v1, const S* __restrict__ v2,
       ColRefT<S> X, ColRefT<S> Y1, ColRefT<S> Y2, const int32_t* __restrict__ skip) {
  using C = S;
  const int j = blockIdx.y;
  if (skip && skip[j]) return;
  const SubDesc d = sub[j];
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= d.nN) return;
  const int w = cr_w(X, j);
  const S* x = cr_ptr(X, d, j);
  S* y1 = cr_ptr(Y1, d, j);
  S* y2 = v2 ? cr_ptr(Y2, d, j) : nullptr;
  const int64_t e0 = lrow[d.offN + a], e1 = lrow[d.offN + a + 1];
  const int64_t nn = d.nN;
  // four columns per pass: the row's column indices and values are read once
  // per four vectors
  int c = 0;
  for (; c + 4 <= w; c += 4) {
    const S* xc = x + (int64_t)c * nn;
    C s10 = 0, s11 = 0, s12 = 0, s13 = 0, s20 = 0, s21 = 0, s22 = 0, s23 = 0;
    for (int64_t e = e0; e < e1; ++e) {
      const int col = lcol[e];
      const C x0 = (C)xc[col], x1 = (C)xc[nn + col], x2 = (C)xc[2 * nn + col], x3 = (C)xc[3 * nn + col];
      const C va = (C)v1[e];
      s10 += va * x0; s11 += va * x1; s12 += va * x2; s13 += va * x3;
      if (v2) {
        const C vb = (C)v2[e];
        s20 += vb * x0; s21 += vb * x1; s22 += vb * x2; s23 += vb * x3;
      }
    }
    y1[c * nn + a] = s10; y1[(c + 1) * nn + a] = s11; y1[(c + 2) * nn + a] = s12; y1[(c + 3) * nn + a] = s13;
    if (v2) {
      y2[c * nn + a] = s20; y2[(c + 1) * nn + a] = s21; y2[(c + 2) * nn + a] = s22; y2[(c + 3) * nn + a] = s23;
    }
  }
  for (; c < w; ++c) {
    const S* xc = x + (int64_t)c * nn;
    C s1 = 0, s2 = 0;
    for (int64_t e = e0; e < e1; ++e) {
      const C xv = (C)xc[lcol[e]];
      s1 += (C)v1[e] * xv;
      if (v2) s2 += (C)v2[e] * xv;
    }
    y1[c * nn + a] = s1;
    if (v2) y2[c * nn + a] = s2;
  }
}

// ---------------------------------------------------------------------------
// Double-single SpMM for the FP32 mode (ds.cuh): the FP64 products with K_j
// and B_j are the eigensolver's largest cost at FP64's 1/64 rate on GB300;
// about 46 significant bits relative to sum |a x|, far below the
// eigensolver's residual tolerance.
// ---------------------------------------------------------------------------
// FP64 values rounded to FP32 (the first pass's copy of K)
__global__ void k_to_f32(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

// FP64 column block -> (hi, lo) float pairs (split_bits): X2 has X's layout
// (same W and columns)
__global__ void k_split_cols(const SubDesc* __restrict__ sub, ColRef X, ColRefT<float2> X2,
                             const int32_t* __restrict__ skip) {
  const int j = blockIdx.y;
  if (skip && skip[j]) return;
  const SubDesc d = sub[j];
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= d.nN) return;
  const int w = cr_w(X, j);
  const double* x = cr_ptr(X, d, j);
  float2* x2 = cr_ptr(X2, d, j);
  for (int c = 0; c < w; ++c) x2[(int64_t)c * d.nN + a] = split_bits(x[(int64_t)c * d.nN + a]);
}

// Longest row of the local CSR matrices (all subdomains).
__global__ void k_max_rowlen(const int64_t* __restrict__ lrow, int64_t rows, int32_t* __restrict__ out) {
  int m = 0;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x)
    m = max(m, (int)(lrow[r + 1] - lrow[r]));
  m = max(m, __shfl_xor_sync(0xffffffffu, m, 16));
  m = max(m, __shfl_xor_sync(0xffffffffu, m, 8));
  m = max(m, __shfl_xor_sync(0xffffffffu, m, 4));
  m = max(m, __shfl_xor_sync(0xffffffffu, m, 2));
  m = max(m, __shfl_xor_sync(0xffffffffu, m, 1));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// Local K and B in a padded column-major row layout (ELLPACK) for the
// double-single SpMM: subdomain j's block starts at offN * L, entry t of row
// a at t * nN + a, so a warp's loads of entry t of 32 consecutive rows are
// contiguous.  Short rows are padded with column a and value 0.
__global__ void k_build_ell(const SubDesc* __restrict__ sub, const int64_t* __restrict__ lrow,
                            const int32_t* __restrict__ lcol, const double* __restrict__ vK,
                            const double* __restrict__ vB, int L, int32_t* __restrict__ ecol,
                            float2* __restrict__ eK, float2* __restrict__ eB) {
  const int j = blockIdx.y;
  const SubDesc d = sub[j];
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= d.nN) return;
  const int64_t e0 = lrow[d.offN + a], e1 = lrow[d.offN + a + 1];
  const int64_t base = d.offN * (int64_t)L + a;
  for (int t = 0; t < L; ++t) {
    const int64_t e = e0 + t;
    const int64_t o = base + (int64_t)t * d.nN;
    if (e < e1) {
      ecol[o] = lcol[e];
      const double k = vK[e], b = vB[e];
      const float kh = (float)k, bh = (float)b;
      eK[o] = make_float2(kh, (float)(k - (double)kh));
      eB[o] = make_float2(bh, (float)(b - (double)bh));
    } else {
      ecol[o] = a;
      eK[o] = make_float2(0.f, 0.f);
      eB[o] = make_float2(0.f, 0.f);
    }
  }
}

// Y1 = V1 X (and Y2 = V2 X when v2 is given) in double-single arithmetic from
// the ELLPACK layout, results stored in FP64; one row per thread, four
// columns per pass (more columns per pass cost occupancy, which this
// gather-bound loop needs more), the entry loop unrolled three times so that
// the loads of several entries are in flight before their gathers.  Each
// entry and operand value is one 8-byte (hi, lo) load.
__global__ void __launch_bounds__(kT)
k_spmm_ds(const SubDesc* __restrict__ sub, int L, const int32_t* __restrict__ ecol,
          const float2* __restrict__ v1, const float2* __restrict__ v2, ColRefT<float2> X2, ColRef Y1,
          ColRef Y2, const int32_t* __restrict__ skip) {
  const int j = blockIdx.y;
  if (skip && skip[j]) return;
  const SubDesc d = sub[j];
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= d.nN) return;
  const int w = cr_w(X2, j);
  const float2* x2 = cr_ptr(X2, d, j);
  double* y1 = cr_ptr(Y1, d, j);
  double* y2 = v2 ? cr_ptr(Y2, d, j) : nullptr;
  const int64_t nn = d.nN;
  const int64_t base = d.offN * (int64_t)L + a;
  constexpr int CP = 4;
  for (int c = 0; c < w; c += CP) {
    const int nc = min(CP, w - c);
    DS s1[CP], s2[CP];
#pragma unroll
    for (int z = 0; z < CP; ++z) s1[z] = s2[z] = DS{0.f, 0.f};
    const float2* xc = x2 + (int64_t)c * nn;
#pragma unroll 3
    for (int t = 0; t < L; ++t) {
      const int64_t o = base + (int64_t)t * nn;
      const int col = ecol[o];
      const float2 va = v1[o];
      const float2 vb = v2 ? v2[o] : make_float2(0.f, 0.f);
#pragma unroll
      for (int z = 0; z < CP; ++z) {
        if (z < nc) {
          const float2 xv = xc[z * nn + col];
          ds_fma(s1[z], va.x, va.y, xv.x, xv.y);
          if (v2) ds_fma(s2[z], vb.x, vb.y, xv.x, xv.y);
        }
      }
    }
#pragma unroll
    for (int z = 0; z < CP; ++z) {
      if (z < nc) {
        y1[(c + z) * nn + a] = acc_value(s1[z]);
        if (v2) y2[(c + z) * nn + a] = acc_value(s2[z]);
      }
    }
  }
}

// Y = X columnwise copy (with conversion between storage types)
template <typename SS, typename SD>
__global__ void k_copy_cols(const SubDesc* __restrict__ sub, ColRefT<SS> Src, ColRefT<SD> Dst,
                            const int32_t* __restrict__ skip) {
  const int j = blockIdx.y;
  if (skip && skip[j]) return;
  const SubDesc d = sub[j];
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= d.nN) return;
  const int w = cr_w(Src, j);
  const SS* s = cr_ptr(Src, d, j);
  SD* t = cr_ptr(Dst, d, j);
  for (int c = 0; c < w; ++c) t[(int64_t)c * d.nN + a] = cv<SD>(s[(int64_t)c * d.nN + a]);
}

// Partial Gram matrices G = A^T B over a row split; ld of G is ldg.
// The output is cut into 4x4 register tiles (lower triangle only when sym,
// A == B); when there are fewer tiles than threads, each tile is shared by
// several row groups (thread g of a tile takes rows g, g + groups, ... of
// every staged chunk) and the groups' partials are summed in a fixed order at
// the end, so all warps issue FP64 FMAs.
template <typename S>
__global__ void __launch_bounds__(kT, 2)
k_gram_part(const SubDesc* __restrict__ sub, ColRefT<S> A, ColRefT<S> B, int sym, double* __restrict__ Gp,
            int ldg, int nsub, const int32_t* __restrict__ skip, int only_wide = 0) {
  using C = S;
  const int j = blockIdx.y, rs = blockIdx.x;
  if (skip && skip[j]) return;
  const SubDesc d = sub[j];
  const int p = cr_w(A, j), q = cr_w(B, j);
  if (only_wide) {
    const int tp0 = (p + 3) >> 2, tq0 = (q + 3) >> 2;
    if ((sym ? tp0 * (tp0 + 1) / 2 : tp0 * tq0) <= kT && 4 * (tp0 + tq0) <= 128) return;  // done by k_gram_one
  }
  double* G = Gp + ((int64_t)rs * nsub + j) * ldg * ldg;
  if (p <= 0 || q <= 0) return;
  const S* a = cr_ptr(A, d, j);
  const S* b = cr_ptr(B, d, j);
  extern __shared__ __align__(16) unsigned char gsm_raw[];
  C* As = reinterpret_cast<C*>(gsm_raw);   // [kRB][kMaxW + 1]
  C* Bs = As + kRB * (kMaxW + 1);          // [kRB][kMaxW + 1]
  constexpr int LDS = kMaxW + 1;
  const int tp = (p + 3) >> 2, tq = (q + 3) >> 2;
  // tiles: full tp x tq grid, or its lower triangle (ti >= tj) when sym
  const int ntiles = sym ? tp * (tp + 1) / 2 : tp * tq;
  const int groups = max(1, kT / ntiles);
  const int tpt = (ntiles + kT - 1) / kT;   // tiles per thread when groups == 1 (<= 3)
  const int g = threadIdx.x / ntiles;       // row group (groups > 1)
  int own[3];
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    const int tx = (int)threadIdx.x;
    int t = groups > 1 ? (tx < groups * ntiles ? tx % ntiles : -1) : (u < tpt ? tx + u * kT : -1);
    if (groups > 1 && u > 0) t = -1;
    if (t >= ntiles) t = -1;
    own[u] = t;
  }
  auto tile_rc = [&](int t, int& ti, int& tj) {
    if (sym) {  // row-major enumeration of the lower triangle
      int r = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
      while ((r + 1) * (r + 2) / 2 <= t) ++r;
      while (r * (r + 1) / 2 > t) --r;
      ti = r;
      tj = t - r * (r + 1) / 2;
    } else {
      ti = t % tp;
      tj = t / tp;
    }
  };
  C acc[3][16];
#pragma unroll
  for (int u = 0; u < 3; ++u)
#pragma unroll
    for (int z = 0; z < 16; ++z) acc[u][z] = 0;
  const int r0 = (int)((int64_t)rs * d.nN / kRS), r1 = (int)((int64_t)(rs + 1) * d.nN / kRS);
  for (int rb = r0; rb < r1; rb += kRB) {
    const int nr = min(kRB, r1 - rb);
    __syncthreads();
    for (int idx = threadIdx.x; idx < kRB * p; idx += kT) {
      const int r = idx % kRB, c = idx / kRB;
      As[r * LDS + c] = r < nr ? (C)a[(int64_t)c * d.nN + rb + r] : (C)0;
    }
    for (int idx = threadIdx.x; idx < kRB * q; idx += kT) {
      const int r = idx % kRB, c = idx / kRB;
      Bs[r * LDS + c] = r < nr ? (C)b[(int64_t)c * d.nN + rb + r] : (C)0;
    }
    __syncthreads();
    const int rstart = groups > 1 ? g : 0;
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      if (own[u] < 0) continue;
      int ti, tj;
      tile_rc(own[u], ti, tj);
      for (int r = rstart; r < nr; r += groups) {
        C av[4], bv[4];
#pragma unroll
        for (int z = 0; z < 4; ++z) {
          av[z] = (4 * ti + z < p) ? As[r * LDS + 4 * ti + z] : (C)0;
          bv[z] = (4 * tj + z < q) ? Bs[r * LDS + 4 * tj + z] : (C)0;
        }
#pragma unroll
        for (int z = 0; z < 4; ++z)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[u][z * 4 + y] += av[z] * bv[y];
      }
    }
  }
  if (groups > 1) {
    // sum the row groups' partials: group-major in shared memory
    __syncthreads();
    double* red = reinterpret_cast<double*>(gsm_raw);  // groups * ntiles * 16 <= kT * 16
    if (own[0] >= 0)
#pragma unroll
      for (int z = 0; z < 16; ++z) red[((size_t)g * ntiles + own[0]) * 16 + z] = acc[0][z];
    __syncthreads();
    for (int o = threadIdx.x; o < ntiles * 16; o += kT) {
      const int t = o / 16, z = o % 16;
      double sum = 0.0;
      for (int gg = 0; gg < groups; ++gg) sum += red[((size_t)gg * ntiles + t) * 16 + z];
      int ti, tj;
      tile_rc(t, ti, tj);
      const int r = 4 * ti + z / 4, c = 4 * tj + z % 4;
      if (r < p && c < q) G[(int64_t)c * ldg + r] = sum;
    }
    return;
  }
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    if (own[u] < 0) continue;
    int ti, tj;
    tile_rc(own[u], ti, tj);
#pragma unroll
    for (int z = 0; z < 4; ++z)
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        const int r = 4 * ti + z, c = 4 * tj + y;
        if (r < p && c < q) G[(int64_t)c * ldg + r] = acc[u][z * 4 + y];
      }
  }
}

// Partial Gram matrices for the common case of at most kT 4 x 4 tiles and at
// most 128 padded columns of A and B together: one tile per thread (row groups when there
// are fewer tiles than threads), columns zero-padded to a multiple of four in
// shared memory (no bounds tests in the inner loop), and the next chunk of
// rows prefetched into registers while the current one is multiplied (one
// barrier per chunk).  Subdomains with more tiles are left to k_gram_part
// (mode 1); this kernel skips them, and k_gram_part in mode 1 skips the
// others.  Same partial layout and summation order rules as k_gram_part.
template <typename S, bool DSM = false>
__global__ void __launch_bounds__(kT, 2)
k_gram_one(const SubDesc* __restrict__ sub, ColRefT<S> A, ColRefT<S> B, int sym, double* __restrict__ Gp,
           int ldg, int nsub, const int32_t* __restrict__ skip) {
  using C = S;
  // DSM (S = double): the chunk is staged as (hi, lo) float pairs and the
  // products accumulate in double-single arithmetic (ds_fma)
  using E = std::conditional_t<DSM, float2, C>;   // staged element
  using Acc = std::conditional_t<DSM, DS, C>;
  const int j = blockIdx.y, rs = blockIdx.x;
  if (skip && skip[j]) return;
  const SubDesc d = sub[j];
  const int p = cr_w(A, j), q = cr_w(B, j);
  if (p <= 0 || q <= 0) return;
  const int tp = (p + 3) >> 2, tq = (q + 3) >> 2;
  const int ntiles = sym ? tp * (tp + 1) / 2 : tp * tq;
  if (ntiles > kT || 4 * (tp + tq) > 128) return;  // left to k_gram_part
  double* G = Gp + ((int64_t)rs * nsub + j) * ldg * ldg;
  const S* a = cr_ptr(A, d, j);
  const S* b = cr_ptr(B, d, j);
  const int pp = 4 * tp, qp = 4 * tq;          // padded widths
  extern __shared__ __align__(16) unsigned char gsm_raw[];
  E* buf = reinterpret_cast<E*>(gsm_raw);      // 2 x kRB x (pp + qp)
  const int chunk = kRB * (pp + qp);
  const int groups = kT / ntiles;
  const int tx = (int)threadIdx.x;
  const int g = tx / ntiles;
  const int t = tx < groups * ntiles ? tx % ntiles : -1;
  int ti = 0, tj = 0;
  if (t >= 0) {
    if (sym) {
      int r = (int)((sqrtf(8.f * t + 1.f) - 1.f) * 0.5f);
      while ((r + 1) * (r + 2) / 2 <= t) ++r;
      while (r * (r + 1) / 2 > t) --r;
      ti = r;
      tj = t - r * (r + 1) / 2;
    } else {
      ti = t % tp;
      tj = t / tp;
    }
  }
  Acc acc[16];
#pragma unroll
  for (int z = 0; z < 16; ++z) acc[z] = Acc{};
  const int r0 = (int)((int64_t)rs * d.nN / kRS), r1 = (int)((int64_t)(rs + 1) * d.nN / kRS);
  // thread (lane, warp) handles row `lane` of a chunk and the combined
  // [A | B] columns warp + 8 u (kRB = 32 rows, 8 warps, up to 128 columns);
  // rows beyond the range and padded columns are zero
  static_assert(kRB == 32 && kT == 256, "chunk mapping assumes 32 rows and 8 warps");
  constexpr int kPre = 16;
  const int lane = tx & 31, wq = tx >> 5;
  C pre[kPre];
  auto fetch = [&](int rb) {
    const bool rowok = rb + lane < r1;
#pragma unroll
    for (int u = 0; u < kPre; ++u) {
      const int cc = wq + 8 * u;
      C v = 0;
      if (rowok) {
        if (cc < p) v = (C)a[(int64_t)cc * d.nN + rb + lane];
        else if (cc >= pp && cc - pp < q) v = (C)b[(int64_t)(cc - pp) * d.nN + rb + lane];
      }
      pre[u] = v;
    }
  };
  auto stash = [&](E* dst) {
#pragma unroll
    for (int u = 0; u < kPre; ++u) {
      const int cc = wq + 8 * u;
      if (cc < pp + qp) {
        if constexpr (DSM) {
          dst[lane * (pp + qp) + cc] = split_bits(pre[u]);
        } else {
          dst[lane * (pp + qp) + cc] = pre[u];
        }
      }
    }
  };
  int cur = 0;
  if (r0 < r1) {
    fetch(r0);
    stash(buf);
  }
  __syncthreads();
  for (int rb = r0; rb < r1; rb += kRB) {
    const bool more = rb + kRB < r1;
    if (more) fetch(rb + kRB);
    const E* X = buf + (size_t)cur * chunk;
    if (t >= 0) {
      const int nr = min(kRB, r1 - rb);
      for (int r = g; r < nr; r += groups) {
        const E* row = X + r * (pp + qp);
        E av[4], bv[4];
#pragma unroll
        for (int z = 0; z < 4; ++z) {
          av[z] = row[4 * ti + z];
          bv[z] = row[pp + 4 * tj + z];
        }
#pragma unroll
        for (int z = 0; z < 4; ++z)
#pragma unroll
          for (int y = 0; y < 4; ++y) {
            if constexpr (DSM) ds_fma(acc[z * 4 + y], av[z].x, av[z].y, bv[y].x, bv[y].y);
            else acc[z * 4 + y] += av[z] * bv[y];
          }
      }
    }
    if (more) stash(buf + (size_t)(cur ^ 1) * chunk);
    __syncthreads();
    cur ^= 1;
  }
  if (groups > 1) {
    // sum the row groups' partials: group-major in shared memory
    double* red = reinterpret_cast<double*>(gsm_raw);  // groups * ntiles * 16 <= kT * 16
    if (t >= 0)
#pragma unroll
      for (int z = 0; z < 16; ++z) red[((size_t)g * ntiles + t) * 16 + z] = acc_value(acc[z]);
    __syncthreads();
    for (int o = threadIdx.x; o < ntiles * 16; o += kT) {
      const int tt = o / 16, z = o % 16;
      double sum = 0.0;
      for (int gg = 0; gg < groups; ++gg) sum += red[((size_t)gg * ntiles + tt) * 16 + z];
      int a0, b0;
      if (sym) {
        int r = (int)((sqrtf(8.f * tt + 1.f) - 1.f) * 0.5f);
        while ((r + 1) * (r + 2) / 2 <= tt) ++r;
        while (r * (r + 1) / 2 > tt) --r;
        a0 = r;
        b0 = tt - r * (r + 1) / 2;
      } else {
        a0 = tt % tp;
        b0 = tt / tp;
      }
      const int rr = 4 * a0 + z / 4, cc = 4 * b0 + z % 4;
      if (rr < p && cc < q) G[(int64_t)cc * ldg + rr] = sum;
    }
    return;
  }
  if (t >= 0)
#pragma unroll
    for (int z = 0; z < 4; ++z)
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        const int r = 4 * ti + z, c = 4 * tj + y;
        if (r < p && c < q) G[(int64_t)c * ldg + r] = acc_value(acc[z * 4 + y]);
      }
}

// G = sum of the row-split partials (fixed order); sym mirrors the lower part.
template <typename S>
__global__ void k_gram_reduce(const SubDesc* __restrict__ sub, ColRefT<S> A, ColRefT<S> B, int sym,
                              const double* __restrict__ Gp, double* __restrict__ G, int ldg,
                              int nsub, const int32_t* __restrict__ skip) {
  const int j = blockIdx.x;
  if (skip && skip[j]) return;
  const int p = cr_w(A, j), q = cr_w(B, j);
  for (int idx = threadIdx.x; idx < p * q; idx += blockDim.x) {
    int r = idx % p, c = idx / p;
    int rr = r, cc = c;
    if (sym && c > r) { rr = c; cc = r; }
    double s = 0.0;
    for (int rs = 0; rs < kRS; ++rs) s += Gp[((int64_t)rs * nsub + j) * ldg * ldg + (int64_t)cc * ldg + rr];
    G[(int64_t)j * ldg * ldg + (int64_t)c * ldg + r] = s;
  }
}

// C = beta*C + alpha * A * T, T = rows [t0 + t0d[j], ...) of a per-subdomain
// ldg x ldg matrix (column-major).  p = width(A), q = width(C).
// FP64 kernel: one row per thread, eight output columns at a time.
__global__ void __launch_bounds__(kT)
k_gemm_nn(const SubDesc* __restrict__ sub, ColRef A, const double* __restrict__ Tm, int ldg,
          int t0, const int32_t* __restrict__ t0d, ColRef Cout, double alpha, double beta,
          const int32_t* __restrict__ skip) {
  const int j = blockIdx.y;
  if (skip && skip[j]) return;
  const SubDesc d = sub[j];
  const int p = cr_w(A, j), q = cr_w(Cout, j);
  if (q <= 0) return;
  extern __shared__ __align__(16) unsigned char ts_raw[];
  double* Ts = reinterpret_cast<double*>(ts_raw);  // p x q, Ts[i*q + c]
  const double* T = Tm + (int64_t)j * ldg * ldg + t0 + (t0d ? t0d[j] : 0);
  for (int idx = threadIdx.x; idx < p * q; idx += blockDim.x) {
    const int i = idx % p, c = idx / p;
    Ts[i * q + c] = T[(int64_t)c * ldg + i];
  }
  __syncthreads();
  const int a_row = blockIdx.x * blockDim.x + threadIdx.x;
  if (a_row >= d.nN) return;
  const double* a = cr_ptr(A, d, j);
  double* cm = cr_ptr(Cout, d, j);
  constexpr int CB = 8;
  for (int c0 = 0; c0 < q; c0 += CB) {
    double acc[CB];
#pragma unroll
    for (int z = 0; z < CB; ++z) acc[z] = 0.0;
    for (int i = 0; i < p; ++i) {
      const double av = a[(int64_t)i * d.nN + a_row];
#pragma unroll
      for (int z = 0; z < CB; ++z)
        if (c0 + z < q) acc[z] += av * Ts[i * q + c0 + z];
    }
#pragma unroll
    for (int z = 0; z < CB; ++z) {
      const int c = c0 + z;
      if (c < q) {
        double* o = cm + (int64_t)c * d.nN + a_row;
        *o = (beta == 0.0 ? 0.0 : beta * *o) + alpha * acc[z];
      }
    }
  }
}

// The same product in double-single arithmetic (FP32 mode): T staged as
// (hi, lo) pairs, each A value split once per sixteen output columns, FP64
// epilogue.
__global__ void __launch_bounds__(kT)
k_gemm_ds(const SubDesc* __restrict__ sub, ColRef A, const double* __restrict__ Tm, int ldg,
          int t0, const int32_t* __restrict__ t0d, ColRef Cout, double alpha, double beta,
          const int32_t* __restrict__ skip) {
  const int j = blockIdx.y;
  if (skip && skip[j]) return;
  const SubDesc d = sub[j];
  const int p = cr_w(A, j), q = cr_w(Cout, j);
  if (q <= 0) return;
  extern __shared__ __align__(16) unsigned char ts_raw[];
  float2* Ts = reinterpret_cast<float2*>(ts_raw);  // p x q, Ts[i*q + c]
  const double* T = Tm + (int64_t)j * ldg * ldg + t0 + (t0d ? t0d[j] : 0);
  for (int idx = threadIdx.x; idx < p * q; idx += blockDim.x) {
    const int i = idx % p, c = idx / p;
    Ts[i * q + c] = split_bits(T[(int64_t)c * ldg + i]);
  }
  __syncthreads();
  const int a_row = blockIdx.x * blockDim.x + threadIdx.x;
  if (a_row >= d.nN) return;
  const double* a = cr_ptr(A, d, j);
  double* cm = cr_ptr(Cout, d, j);
  constexpr int CB = 16;
  for (int c0 = 0; c0 < q; c0 += CB) {
    DS acc[CB];
#pragma unroll
    for (int z = 0; z < CB; ++z) acc[z] = DS{0.f, 0.f};
    for (int i = 0; i < p; ++i) {
      const float2 av = split_bits(a[(int64_t)i * d.nN + a_row]);
#pragma unroll
      for (int z = 0; z < CB; ++z)
        if (c0 + z < q) {
          const float2 tv = Ts[i * q + c0 + z];
          ds_fma(acc[z], av.x, av.y, tv.x, tv.y);
        }
    }
    const bool copy = beta == 0.0 && alpha == 1.0, sub1 = beta == 1.0 && alpha == -1.0;
#pragma unroll
    for (int z = 0; z < CB; ++z) {
      const int c = c0 + z;
      if (c < q) {
        double* o = cm + (int64_t)c * d.nN + a_row;
        if (copy) *o = acc_value(acc[z]);
        else if (sub1) *o = *o - acc_value(acc[z]);
        else *o = (beta == 0.0 ? 0.0 : beta * *o) + alpha * acc_value(acc[z]);
      }
    }
  }
}

// FP32-arithmetic GEMM.  A has storage SA, C storage SO; each A value is
// read (and converted) once per 32 output columns; T rows are read as
// four-wide vectors.  Epilogue:
//  corr = 0 and SO = float: everything in FP32 (first orthogonalisation pass);
//  otherwise the FP32 product is added in FP64: C = beta C + alpha (acc +
//  [addI] A[:, c]).  With addI, T - I is used in the product, so A T = A +
//  A (T - I) keeps FP64 accuracy for T near I (the second pass).
// f64 (may be NULL): subdomains with f64[j] == 0 take FP64 arithmetic
// (T not near I there).
template <typename SA, typename SO>
__global__ void __launch_bounds__(kT)
k_gemm32(const SubDesc* __restrict__ sub, ColRefT<SA> A, const double* __restrict__ Tm, int ldg,
         int t0, const int32_t* __restrict__ t0d, ColRefT<SO> Cout, double alpha, double beta,
         const int32_t* __restrict__ skip, int corr, int addI, const int32_t* __restrict__ f64) {
  const int j = blockIdx.y;
  if (skip && skip[j]) return;
  const SubDesc d = sub[j];
  const int p = cr_w(A, j), q = cr_w(Cout, j);
  if (q <= 0) return;
  const bool wide = f64 && f64[j] == 0;
  const int qp = (q + 3) & ~3;
  extern __shared__ __align__(16) unsigned char ts_raw[];
  float* Ts = reinterpret_cast<float*>(ts_raw);        // p x qp, Ts[i*qp + c]
  double* Td = reinterpret_cast<double*>(ts_raw);      // p x q (FP64 override)
  const double* T = Tm + (int64_t)j * ldg * ldg + t0 + (t0d ? t0d[j] : 0);
  for (int idx = threadIdx.x; idx < p * qp; idx += blockDim.x) {
    const int i = idx / qp, c = idx % qp;
    double v = c < q ? T[(int64_t)c * ldg + i] : 0.0;
    if (addI && i == c) v -= 1.0;
    if (wide) {
      if (c < q) Td[i * q + c] = v;
    } else {
      Ts[i * qp + c] = (float)v;
    }
  }
  __syncthreads();
  const int a_row = blockIdx.x * blockDim.x + threadIdx.x;
  if (a_row >= d.nN) return;
  const SA* a = cr_ptr(A, d, j);
  SO* cm = cr_ptr(Cout, d, j);
  if (wide) {
    for (int c = 0; c < q; ++c) {
      double acc = 0.0;
      for (int i = 0; i < p; ++i) acc += cv<double>(a[(int64_t)i * d.nN + a_row]) * Td[i * q + c];
      SO* o = cm + (int64_t)c * d.nN + a_row;
      const double v = acc + (addI ? cv<double>(a[(int64_t)c * d.nN + a_row]) : 0.0);
      *o = cv<SO>((beta == 0.0 ? 0.0 : beta * cv<double>(*o)) + alpha * v);
    }
    return;
  }
  for (int c0 = 0; c0 < q; c0 += 32) {
    const int nc = min(32, q - c0);
    float acc[32];
#pragma unroll
    for (int z = 0; z < 32; ++z) acc[z] = 0.f;
    for (int i = 0; i < p; ++i) {
      const float av = cv<float>(a[(int64_t)i * d.nN + a_row]);
      const float* tr = Ts + i * qp + c0;
#pragma unroll
      for (int z4 = 0; z4 < 8; ++z4) {
        if (4 * z4 < nc) {
          const float4 t4 = *reinterpret_cast<const float4*>(tr + 4 * z4);
          acc[4 * z4] += av * t4.x;
          acc[4 * z4 + 1] += av * t4.y;
          acc[4 * z4 + 2] += av * t4.z;
          acc[4 * z4 + 3] += av * t4.w;
        }
      }
    }
    // FP64 epilogue without the FP64 multiplications for the two forms the
    // eigensolver uses (C = A T and C = C - A T): GB300 issues FP64 at 1/64
    // of the FP32 rate
    const bool copy = beta == 0.0 && alpha == 1.0, sub1 = beta == 1.0 && alpha == -1.0;
#pragma unroll
    for (int z = 0; z < 32; ++z) {
      if (z < nc) {
        const int c = c0 + z;
        SO* o = cm + (int64_t)c * d.nN + a_row;
        if (corr || sizeof(SO) == 8) {
          const double pz = f2d_bits(acc[z]);
          const double v = addI ? pz + cv<double>(a[(int64_t)c * d.nN + a_row]) : pz;
          if (copy) *o = cv<SO>(v);
          else if (sub1) *o = cv<SO>(cv<double>(*o) - v);
          else *o = cv<SO>((beta == 0.0 ? 0.0 : beta * cv<double>(*o)) + alpha * v);
        } else {
          *o = (SO)((beta == 0.0 ? 0.f : (float)beta * (float)*o) + (float)alpha * acc[z]);
        }
      }
    }
  }
}

// Counter-based start block: uniform(-1, 1) from SplitMix64.
__global__ void k_init_random(const SubDesc* __restrict__ sub, ColRef X, uint64_t seed,
                              const int32_t* __restrict__ skip) {
  const int j = blockIdx.y;
  if (skip && skip[j]) return;
  const SubDesc d = sub[j];
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= d.nN) return;
  const int w = cr_w(X, j);
  double* x = cr_ptr(X, d, j);
  for (int c = 0; c < w; ++c) {
    const uint64_t ctr = ((uint64_t)j << 40) ^ ((uint64_t)c << 28) ^ (uint64_t)a;
    const uint64_t u = splitmix64(seed ^ splitmix64(ctr));
    x[(int64_t)c * d.nN + a] = (double)(u >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
}

// ---------------------------------------------------------------------------
// Dense symmetric eigensolver: parallel cyclic Jacobi (round-robin pairs) in
// arithmetic T (float, double, or double-single dsv).  A (m x m, row stride
// lda) is overwritten by its diagonal form, V receives the eigenvectors
// (columns).  Whole block participates.
//
// All M/2 rotations of a round are disjoint, so the round is A <- R A R^T
// with R block diagonal in the pairs: entry block (k, l) of the result (rows
// of pair k, columns of pair l) is R_k A_kl R_l^T.  A stays exactly
// symmetric, so only the blocks k <= l are formed and each is written to
// both of its places; every block is read and written by one thread, in
// place.  One barrier after the rotations, one after the update.
// ---------------------------------------------------------------------------
template <typename T> struct JacobiOps;
template <> struct JacobiOps<float> {
  using R = float;  // norms and pivot tests
  static constexpr float eps_off = 1e-13f, eps_rot = 1e-9f, tiny = 1e-37f;
  __device__ static float mag(float v) { return v; }
};
template <> struct JacobiOps<double> {
  using R = double;
  static constexpr double eps_off = 1e-30, eps_rot = 1e-18, tiny = 1e-300;
  __device__ static double mag(double v) { return v; }
};
// double-single: about 46 bits, so the off-diagonal mass stops near 1e-26 of
// the whole; the sweeps stop at 1e-24 (off-diagonal entries 1e-12 of the
// norm, far below what the Ritz values and vectors need).  Norms from the
// high parts in FP32: the caller scales A to |a_ij| <= 1 (a power of two).
template <> struct JacobiOps<dsv> {
  using R = float;
  static constexpr float eps_off = 1e-24f, eps_rot = 1e-14f, tiny = 1e-37f;
  __device__ static float mag(dsv v) { return v.h; }
};

// Rotation (c, s) that annihilates a_pq; false when a_pq is negligible.
template <typename T>
__device__ __forceinline__ bool jacobi_rot(T app, T aqq, T apq, T& c, T& s) {
  using J = JacobiOps<T>;
  if (!(fabs(apq) > J::tiny && fabs(apq) > J::eps_rot * sqrt(fabs(app * aqq)))) return false;
  const T theta = (aqq - app) / (T(2) * apq);
  const T t = (theta >= T(0) ? T(1) : T(-1)) / (fabs(theta) + sqrt(theta * theta + T(1)));
  c = T(1) / sqrt(t * t + T(1));
  s = t * c;
  return s != T(0);
}
// Double-single: the angle in FP32 from the double-single difference of the
// pivots.  An angle good to FP32 leaves a_pq about 1e-7 of its size instead of
// zero (the next sweep removes the rest, Jacobi converges just as well with
// such angles); what must hold to double-single precision is c^2 + s^2 = 1:
// c = (1 + t^2)^(-1/2) from the correctly rounded FP32 value and one Newton
// step in double-single (error about 3/8 of the square of the FP32 one),
// s = t c.
template <>
__device__ __forceinline__ bool jacobi_rot<dsv>(dsv app, dsv aqq, dsv apq, dsv& c, dsv& s) {
  using J = JacobiOps<dsv>;
  const float a = fabsf(apq.h);
  if (!(a > J::tiny && a > J::eps_rot * sqrtf(fabsf(app.h * aqq.h)))) return false;
  const float theta = (aqq - app).h / (2.f * apq.h);
  const float t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(fmaf(theta, theta, 1.f)));
  if (!(t != 0.f)) return false;
  const dsv x = dsv(1.f, 0.f) + dsv(t, 0.f) * dsv(t, 0.f);
  const float r0 = __frsqrt_rn(x.h);
  const float delta = (dsv(1.f, 0.f) - x * (dsv(r0, 0.f) * dsv(r0, 0.f))).h;
  c = dsv(r0, 0.f) + dsv(0.5f * r0 * delta, 0.f);
  s = dsv(t, 0.f) * c;
  return true;
}

template <typename T>
__device__ void jacobi_eig(T* A, int lda, T* V, int ldv, int m, T* cs, T* sn,
                           typename JacobiOps<T>::R* red) {
  using J = JacobiOps<T>;
  using R = typename J::R;
  __shared__ int jp[kMaxW / 2 + 1], jq[kMaxW / 2 + 1], jact[kMaxW / 2 + 1];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int M = m + (m & 1), H = M / 2;
  for (int idx = tid; idx < m * m; idx += nt) {
    const int r = idx % m, c = idx / m;
    V[r * ldv + c] = (r == c) ? T(1.0) : T(0.0);
  }
  __syncthreads();
  if (m <= 1) return;
  for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
    R off = R(0), all = R(0);
    for (int idx = tid; idx < m * m; idx += nt) {
      const int r = idx % m, c = idx / m;
      const R v = J::mag(A[r * lda + c]);
      all += v * v;
      if (r != c) off += v * v;
    }
    off = block_sum(off, red);
    all = block_sum(all, red);
    if (off <= J::eps_off * all || all == R(0)) break;
    for (int round = 0; round < M - 1; ++round) {
      // pair k: (M-1, round) for k = 0; ((round+k)%(M-1), (round-k+M-1)%(M-1))
      // otherwise; q = M - 1 = m is the padding index of odd m
      for (int k = tid; k < H; k += nt) {
        int pi, qi;
        if (k == 0) { pi = M - 1; qi = round; }
        else { pi = (round + k) % (M - 1); qi = (round - k + M - 1) % (M - 1); }
        if (pi > qi) { const int t = pi; pi = qi; qi = t; }
        T c = T(1.0), sv = T(0.0);
        const bool act = qi < m && jacobi_rot(A[pi * lda + pi], A[qi * lda + qi], A[pi * lda + qi], c, sv);
        jp[k] = pi;
        jq[k] = qi;
        jact[k] = act;
        cs[k] = act ? c : T(1.0);
        sn[k] = act ? sv : T(0.0);
      }
      __syncthreads();
      // A <- R A R^T over the blocks k <= l
      for (int idx = tid; idx < H * H; idx += nt) {
        const int k = idx / H, l = idx % H;
        if (k > l || !(jact[k] | jact[l])) continue;
        const int pk = jp[k], qk = jq[k], pl = jp[l], ql = jq[l];
        const bool hk = qk < m, hl = ql < m;
        const T z = T(0.0);
        const T a00 = A[pk * lda + pl];
        const T a01 = hl ? A[pk * lda + ql] : z;
        const T a10 = hk ? A[qk * lda + pl] : z;
        const T a11 = (hk && hl) ? A[qk * lda + ql] : z;
        T t00 = a00, t01 = a01, t10 = a10, t11 = a11;
        if (jact[l]) {
          const T c = cs[l], s = sn[l];
          t00 = a00 * c - a01 * s;
          t01 = a00 * s + a01 * c;
          t10 = a10 * c - a11 * s;
          t11 = a10 * s + a11 * c;
        }
        T b00 = t00, b01 = t01, b10 = t10, b11 = t11;
        if (jact[k]) {
          const T c = cs[k], s = sn[k];
          b00 = c * t00 - s * t10;
          b10 = s * t00 + c * t10;
          b01 = c * t01 - s * t11;
          b11 = s * t01 + c * t11;
        }
        if (k == l) {
          // the diagonal block: one value for both off-diagonal places
          A[pk * lda + pk] = b00;
          if (hk) {
            A[pk * lda + qk] = b01;
            A[qk * lda + pk] = b01;
            A[qk * lda + qk] = b11;
          }
          continue;
        }
        A[pk * lda + pl] = b00;
        A[pl * lda + pk] = b00;
        if (hl) {
          A[pk * lda + ql] = b01;
          A[ql * lda + pk] = b01;
        }
        if (hk) {
          A[qk * lda + pl] = b10;
          A[pl * lda + qk] = b10;
        }
        if (hk && hl) {
          A[qk * lda + ql] = b11;
          A[ql * lda + qk] = b11;
        }
      }
      // V <- V R^T (columns of the pairs)
      for (int idx = tid; idx < H * m; idx += nt) {
        const int k = idx / m, row = idx % m;
        if (!jact[k]) continue;
        const int pi = jp[k], qi = jq[k];
        const T c = cs[k], s = sn[k];
        const T vp = V[row * ldv + pi], vq = V[row * ldv + qi];
        V[row * ldv + pi] = c * vp - s * vq;
        V[row * ldv + qi] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
}

// Shared memory of the dense kernels for matrices of order <= wmax (row
// stride wmax + 1), arithmetic T.
template <typename T>
size_t dense_smem_bytes(int wmax) {
  return sizeof(T) * ((size_t)2 * wmax * (wmax + 1) + 6 * (size_t)wmax + kT / 32 + 8);
}

// SVQB: columns whose Gram matrix is G (q x q) -> T (q x r) with
// (M T)^T K (M T) = I; directions with eigenvalue below drop * max are
// removed.  Writes T into Tout (ldg) and r into r_out[j].  The Jacobi step
// runs in arithmetic T (FP32 for a Gram formed in FP32 arithmetic).
template <typename T>
__global__ void __launch_bounds__(kT)
k_svqb(const double* __restrict__ Gall, double* __restrict__ Tout, int ldg,
       const int32_t* __restrict__ wq, const int32_t* __restrict__ wq2, int32_t* __restrict__ r_out,
       double drop, const int32_t* __restrict__ skip, int wmax) {
  const int j = blockIdx.x;
  if (skip && skip[j]) return;
  const int q = (wq ? wq[j] : 0) + (wq2 ? wq2[j] : 0);
  extern __shared__ __align__(16) unsigned char dsm_raw[];
  const int LD = wmax + 1;
  T* A = reinterpret_cast<T*>(dsm_raw);
  T* V = A + (size_t)wmax * LD;
  T* dsc = V + (size_t)wmax * LD;
  T* ev = dsc + wmax;
  T* cs = ev + wmax;
  T* sn = cs + wmax;
  T* red = sn + wmax;
  __shared__ int keep[kMaxW];
  __shared__ int nkeep;
  if (q <= 0) {
    if (threadIdx.x == 0) r_out[j] = 0;
    return;
  }
  const double* G = Gall + (int64_t)j * ldg * ldg;
  for (int i = threadIdx.x; i < q; i += blockDim.x) {
    const double g = G[(int64_t)i * ldg + i];
    dsc[i] = g > 0.0 ? (T)(1.0 / sqrt(g)) : T(0);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < q * q; idx += blockDim.x) {
    const int r = idx % q, c = idx / q;
    const double g = 0.5 * (G[(int64_t)c * ldg + r] + G[(int64_t)r * ldg + c]);
    A[r * LD + c] = (T)((double)dsc[r] * g * (double)dsc[c]);
  }
  __syncthreads();
  jacobi_eig<T>(A, LD, V, LD, q, cs, sn, red);
  for (int i = threadIdx.x; i < q; i += blockDim.x) ev[i] = A[i * LD + i];
  __syncthreads();
  if (threadIdx.x == 0) {
    T mx = T(0);
    for (int i = 0; i < q; ++i) mx = fmax(mx, ev[i]);
    int r = 0;
    for (int i = 0; i < q; ++i)
      if (mx > T(0) && (double)ev[i] > drop * (double)mx) keep[r++] = i;
    nkeep = r;
    r_out[j] = r;
  }
  __syncthreads();
  double* Tm = Tout + (int64_t)j * ldg * ldg;
  for (int idx = threadIdx.x; idx < q * nkeep; idx += blockDim.x) {
    const int r = idx % q, k = idx / q;
    const int i = keep[k];
    Tm[(int64_t)k * ldg + r] = (double)dsc[r] * (double)V[r * LD + i] / sqrt((double)ev[i]);
  }
}

// K-orthonormalisation of a nearly orthonormal block (Cholesky QR): with
// D = diag(G)^{-1/2} and D G D = L L^T, T = D L^{-T} gives (M T)^T K (M T) = I
// and keeps all q columns.  A pivot below 1e-8 (D G D has unit diagonal)
// switches this subdomain to the SVQB path above, which drops dependent
// directions.
__global__ void __launch_bounds__(kT)
k_cholqr(const double* __restrict__ Gall, double* __restrict__ Tout, int ldg,
         const int32_t* __restrict__ wq, int32_t* __restrict__ r_out, double drop,
         const int32_t* __restrict__ skip, int wmax) {
  const int j = blockIdx.x;
  if (skip && skip[j]) return;
  const int q = wq[j];
  extern __shared__ __align__(16) unsigned char dsm_raw[];
  const int LD = wmax + 1;
  double* A = reinterpret_cast<double*>(dsm_raw);
  double* V = A + (size_t)wmax * LD;
  double* dsc = V + (size_t)wmax * LD;
  __shared__ int bad;
  if (q <= 0) {
    if (threadIdx.x == 0) r_out[j] = 0;
    return;
  }
  const double* G = Gall + (int64_t)j * ldg * ldg;
  for (int i = threadIdx.x; i < q; i += blockDim.x) {
    const double g = G[(int64_t)i * ldg + i];
    dsc[i] = g > 0.0 ? 1.0 / sqrt(g) : 0.0;
  }
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int idx = threadIdx.x; idx < q * q; idx += blockDim.x) {
    const int r = idx % q, c = idx / q;
    A[r * LD + c] = dsc[r] * 0.5 * (G[(int64_t)c * ldg + r] + G[(int64_t)r * ldg + c]) * dsc[c];
  }
  __syncthreads();
  // right-looking Cholesky, lower triangle of A
  for (int c = 0; c < q; ++c) {
    const double piv = A[c * LD + c];
    if (!(piv > 1e-8)) {
      if (threadIdx.x == 0) bad = 1;
      break;
    }
    const double dl = sqrt(piv);
    __syncthreads();
    for (int r = c + 1 + threadIdx.x; r < q; r += blockDim.x) A[r * LD + c] /= dl;
    if (threadIdx.x == 0) A[c * LD + c] = dl;
    __syncthreads();
    const int rem = q - c - 1;
    for (int idx = threadIdx.x; idx < rem * rem; idx += blockDim.x) {
      const int r = c + 1 + idx % rem, t = c + 1 + idx / rem;
      if (t <= r) A[r * LD + t] -= A[r * LD + c] * A[t * LD + c];
    }
    __syncthreads();
  }
  __syncthreads();
  if (bad) return;  // r_out left for the SVQB fallback (flagged below)
  // V = L^{-T} (upper triangular): column k solves L^T v = e_k by back
  // substitution, one thread per column
  for (int k = threadIdx.x; k < q; k += blockDim.x) {
    for (int r = q - 1; r >= 0; --r) {
      double v = r == k ? 1.0 : 0.0;
      if (r > k) v = 0.0;
      else {
        for (int t = r + 1; t <= k; ++t) v -= A[t * LD + r] * V[t * LD + k];
        v /= A[r * LD + r];
      }
      V[r * LD + k] = v;
    }
  }
  __syncthreads();
  double* Tm = Tout + (int64_t)j * ldg * ldg;
  for (int idx = threadIdx.x; idx < q * q; idx += blockDim.x) {
    const int r = idx % q, k = idx / q;
    Tm[(int64_t)k * ldg + r] = dsc[r] * V[r * LD + k];
  }
  if (threadIdx.x == 0) r_out[j] = q;
}

// Marks the subdomains whose Cholesky QR failed: the kernel above leaves
// r_out[j] = -1 (set here beforehand) so the SVQB pass can run on them only.
__global__ void k_mark_fallback(const int32_t* __restrict__ r_out, const int32_t* __restrict__ skip,
                                int32_t* __restrict__ redo, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) redo[j] = (skip && skip[j]) ? 1 : (r_out[j] < 0 ? 0 : 1);
}

__global__ void k_fill_i32(int32_t* __restrict__ dst, int32_t v, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) dst[j] = v;
}

// Rayleigh-Ritz: eig of G (m x m, m = s_j + q_j), keep the s_j largest in
// descending order: nu[0..s_j), U (m x s_j) into Tout.  Jacobi in arithmetic
// T: FP64, or double-single in the FP32 mode (GB300 issues FP64 at 1/64 of
// the FP32 rate, and the sweeps are most of this kernel).  The double-single
// sweeps run on G scaled by a power of two to |g_ij| < 1 (exact).
template <typename T>
__global__ void __launch_bounds__(kT)
k_rr(const double* __restrict__ Gall, double* __restrict__ Tout, int ldg,
     const int32_t* __restrict__ sj, const int32_t* __restrict__ qj, double* __restrict__ nu_out,
     int ldnu, const int32_t* __restrict__ skip, int wmax) {
  const int j = blockIdx.x;
  if (skip && skip[j]) return;
  const int s = sj[j];
  const int m = s + (qj ? qj[j] : 0);
  extern __shared__ __align__(16) unsigned char dsm_raw[];
  const int LD = wmax + 1;
  static_assert(sizeof(T) == sizeof(double), "layout of dense_smem_bytes<double>");
  T* A = reinterpret_cast<T*>(dsm_raw);
  T* V = A + (size_t)wmax * LD;
  double* ev = reinterpret_cast<double*>(V + (size_t)wmax * LD);
  T* cs = reinterpret_cast<T*>(ev + wmax);
  T* sn = cs + wmax;
  auto* red = reinterpret_cast<typename JacobiOps<T>::R*>(sn + wmax);
  __shared__ int order[kMaxW];
  __shared__ double wmx[kT / 32];
  if (m <= 0) return;
  const double* G = Gall + (int64_t)j * ldg * ldg;
  int ex = 0;
  if constexpr (!std::is_same_v<T, double>) {
    double mx = 0.0;
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
      const int r = idx % m, c = idx / m;
      mx = fmax(mx, fabs(0.5 * (G[(int64_t)c * ldg + r] + G[(int64_t)r * ldg + c])));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) wmx[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, wmx[w]);
    if (mx > 0.0 && isfinite(mx)) frexp(mx, &ex);
  }
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int r = idx % m, c = idx / m;
    const double g = 0.5 * (G[(int64_t)c * ldg + r] + G[(int64_t)r * ldg + c]);
    if constexpr (std::is_same_v<T, double>) A[r * LD + c] = g;
    else A[r * LD + c] = T(ldexp(g, -ex));
  }
  __syncthreads();
  jacobi_eig<T>(A, LD, V, LD, m, cs, sn, red);
  for (int i = threadIdx.x; i < m; i += blockDim.x) ev[i] = ldexp(to_double(A[i * LD + i]), ex);
  __syncthreads();
  // rank in descending order (ties by index)
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    int rk = 0;
    for (int k = 0; k < m; ++k) rk += (ev[k] > ev[i]) || (ev[k] == ev[i] && k < i);
    order[rk] = i;
  }
  __syncthreads();
  double* U = Tout + (int64_t)j * ldg * ldg;
  for (int idx = threadIdx.x; idx < m * s; idx += blockDim.x) {
    const int r = idx % m, k = idx / m;
    U[(int64_t)k * ldg + r] = to_double(V[r * LD + order[k]]);
  }
  for (int k = threadIdx.x; k < s; k += blockDim.x) nu_out[(int64_t)j * ldnu + k] = ev[order[k]];
}

// Residuals, convergence and the next search block.  One block per
// subdomain.  R = BX - KX diag(nu) is written (active columns only,
// compacted) to S after X, then the s_p columns of P follow.
__global__ void __launch_bounds__(kT)
k_resid(const SubDesc* __restrict__ sub, ColRef S, ColRef BX, ColRef KX, ColRef P,
        const double* __restrict__ nu_all, int ldnu, const int32_t* __restrict__ sj,
        const int32_t* __restrict__ spj, int32_t* __restrict__ aj, int32_t* __restrict__ qj,
        int32_t* __restrict__ done, int32_t* __restrict__ iters, int32_t* __restrict__ notdone,
        double* __restrict__ rn_out, double tol, double tau, double sigma, const int32_t* __restrict__ nevj, int fixed,
        int it, double* __restrict__ best, int32_t* __restrict__ stall, int32_t* __restrict__ o64,
        int32_t* __restrict__ ok32, int stall_lim) {
  const int j = blockIdx.x;
  if (done[j]) return;
  const SubDesc d = sub[j];
  const int s = sj[j];
  const int nev = nevj[j];
  const double* nu = nu_all + (int64_t)j * ldnu;
  const double* bx = cr_ptr(BX, d, j);
  const double* kx = cr_ptr(KX, d, j);
  __shared__ double rn[kMaxW];
  __shared__ int act[kMaxW];
  __shared__ int na, fin;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = wid; c < s; c += nw) {
    double r2 = 0.0, b2 = 0.0, k2 = 0.0;
    const double* bc = bx + (int64_t)c * d.nN;
    const double* kc = kx + (int64_t)c * d.nN;
    const double nc = nu[c];
    for (int a = lane; a < d.nN; a += 32) {
      const double bv = bc[a], kv = kc[a];
      const double rv = bv - nc * kv;
      r2 += rv * rv;
      b2 += bv * bv;
      k2 += kv * kv;
    }
    r2 = warp_sum(r2);
    b2 = warp_sum(b2);
    k2 = warp_sum(k2);
    if (lane == 0) {
      const double den = sqrt(b2) + fabs(nc) * sqrt(k2);
      rn[c] = den > 0.0 ? sqrt(r2) / den : 0.0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    bool ok = true;
    if (fixed) {
      for (int i = 0; i < min(nev, s); ++i) ok = ok && rn[i] <= tol;
    } else {
      for (int i = 0; i < min(nev, s); ++i) {
        if (rn[i] > tol) { ok = false; break; }
        const double lam = nu[i] > 0.0 ? sigma + 1.0 / nu[i] : INFINITY;
        if (lam >= tau) break;
      }
    }
    int k = 0;
    for (int i = 0; i < s; ++i)
      if (rn[i] > tol) act[k++] = i;
    na = k;
    fin = ok || k == 0;
    if (fin) {
      done[j] = 1;
    } else {
      atomicAdd(notdone, 1);
    }
    // FP32 first passes: a subdomain whose largest wanted residual has not
    // halved in stall_lim iterations (counted after iteration kStallFrom of
    // the pass), or that is still iterating at iteration kForce64From,
    // switches to FP64 products and orthogonalisation (notdone[1] counts the
    // switches)
    if (best && !fin && !o64[j]) {
      double r = 0.0;
      for (int i = 0; i < min(nev, s); ++i) {
        r = fmax(r, rn[i]);
        const double lam = nu[i] > 0.0 ? sigma + 1.0 / nu[i] : INFINITY;
        if (!fixed && lam >= tau) break;
      }
      bool sw = false;
      if (it >= kForce64From) {  // a straggler: FP64 from here on
        sw = true;
      } else if (it <= kStallFrom || r < 0.5 * best[j]) {
        best[j] = r;
        stall[j] = 0;
      } else if (++stall[j] >= stall_lim) {
        sw = true;
      }
      if (sw) {
        o64[j] = 1;
        ok32[j] = 0;
        atomicAdd(notdone + 1, 1);
      }
    }
    iters[j] = it;
    aj[j] = fin ? 0 : k;
    qj[j] = fin ? 0 : k + spj[j];
    for (int i = 0; i < s; ++i) rn_out[(int64_t)j * ldnu + i] = rn[i];
  }
  __syncthreads();
  if (fin) return;
  double* sbase = cr_ptr(S, d, j);
  double* w0 = sbase + (int64_t)s * d.nN;
  const int k = na;
  // S, BX, KX and P are distinct buffers: the loads of later rows may be
  // issued before the stores of earlier ones
  for (int t = 0; t < k; ++t) {
    const int c = act[t];
    const double nc = nu[c];
    const double* __restrict__ bc = bx + (int64_t)c * d.nN;
    const double* __restrict__ kc = kx + (int64_t)c * d.nN;
    double* __restrict__ o = w0 + (int64_t)t * d.nN;
#pragma unroll 4
    for (int a = threadIdx.x; a < d.nN; a += blockDim.x) o[a] = bc[a] - nc * kc[a];
  }
  const int sp = spj[j];
  const double* pc = cr_ptr(P, d, j);
  for (int t = 0; t < sp; ++t) {
    double* __restrict__ o = w0 + (int64_t)(k + t) * d.nN;
    const double* __restrict__ src = pc + (int64_t)t * d.nN;
#pragma unroll 4
    for (int a = threadIdx.x; a < d.nN; a += blockDim.x) o[a] = src[a];
  }
}


__global__ void k_sub_nnz(const SubDesc* __restrict__ sub, const int64_t* __restrict__ lrow,
                          int64_t* __restrict__ out, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) out[j] = lrow[sub[j].offN + sub[j].nN] - lrow[sub[j].offN];
}

__global__ void k_clear_p(int32_t* __restrict__ spj, const int32_t* __restrict__ skip, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n && !skip[j]) spj[j] = 0;
}

__global__ void k_set_i32(int32_t* __restrict__ dst, const int32_t* __restrict__ src, int n,
                          const int32_t* __restrict__ skip) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n && !(skip && skip[j])) dst[j] = src[j];
}

// Skip flags of the two orthogonalisation flavours with FP32 factors:
// skip32 = done or o64 (FP32 first pass), skip64 = done or not o64 (FP64
// first pass for the subdomains whose K_j needed FP64).
__global__ void k_split_skip(const int32_t* __restrict__ done, const int32_t* __restrict__ o64,
                             int32_t* __restrict__ skip32, int32_t* __restrict__ skip64, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) {
    const int dj = done ? done[j] : 0;  // done may be NULL (nothing skipped)
    skip32[j] = dj || o64[j];
    skip64[j] = dj || !o64[j];
  }
}

// f[j] = f[j] and not o64[j] (FP32-arithmetic flags of k_gemm32)
__global__ void k_and_not(int32_t* __restrict__ f, const int32_t* __restrict__ o64, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n && o64[j]) f[j] = 0;
}

inline double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

geneo_status_t local_eigensolve(geneo_handle_s* h, AssemblyOut& asmb, DevMem& tmp, cudaStream_t st,
                                double** X_out, int64_t* ld_unused) {
  (void)ld_unused;
  const int N = h->N;
  const geneo_options_t& o = h->opt;
  const int nev = o.nev_max;
  const int s = h->s_block;
  const int W3 = 3 * s;
  const int ldg = W3;
  if (W3 > kMaxW) return GENEO_ERR_ARG;
  const int64_t rows = h->sumN;
  double *S, *KS, *BS, *P, *Tmp, *G, *Gp, *Tm, *nu, *rn;
  GENEO_TRY(tmp.get(&S, (size_t)rows * W3));
  GENEO_TRY(tmp.get(&KS, (size_t)rows * W3));
  GENEO_TRY(tmp.get(&BS, (size_t)rows * W3));
  GENEO_TRY(tmp.get(&Tmp, (size_t)rows * W3));
  GENEO_TRY(tmp.get(&P, (size_t)rows * s));
  GENEO_TRY(tmp.get(&G, (size_t)N * ldg * ldg));
  GENEO_TRY(tmp.get(&Gp, (size_t)kRS * N * ldg * ldg));
  GENEO_TRY(tmp.get(&Tm, (size_t)N * ldg * ldg));
  GENEO_TRY(tmp.get(&nu, (size_t)N * s));
  GENEO_TRY(tmp.get(&rn, (size_t)N * s));
  int32_t *sj, *aj, *qj, *rj, *spj, *done, *iters, *notdone, *nevj;
  GENEO_TRY(tmp.get(&nevj, (size_t)N));
  GENEO_TRY(tmp.get(&sj, (size_t)N));
  GENEO_TRY(tmp.get(&aj, (size_t)N));
  GENEO_TRY(tmp.get(&qj, (size_t)N));
  GENEO_TRY(tmp.get(&rj, (size_t)N));
  GENEO_TRY(tmp.get(&spj, (size_t)N));
  GENEO_TRY(tmp.get(&done, (size_t)N));
  GENEO_TRY(tmp.get(&iters, (size_t)N));
  GENEO_TRY(tmp.get(&notdone, 2));
  GENEO_CUDA(cudaMemsetAsync(S, 0, sizeof(double) * rows * W3, st));
  GENEO_CUDA(cudaMemsetAsync(P, 0, sizeof(double) * rows * s, st));
  GENEO_CUDA(cudaMemsetAsync(nu, 0, sizeof(double) * N * s, st));
  GENEO_CUDA(cudaMemsetAsync(spj, 0, sizeof(int32_t) * N, st));
  GENEO_CUDA(cudaMemsetAsync(done, 0, sizeof(int32_t) * N, st));
  GENEO_CUDA(cudaMemsetAsync(iters, 0, sizeof(int32_t) * N, st));
  int maxn = 0;
  for (int j = 0; j < N; ++j) maxn = std::max(maxn, h->hsub[j].nN);
  const dim3 gridR(ceil_div(maxn, kT), N);
  // dense kernels sized by the block width: [X, Q] has at most 3 s columns
  const int wmax = W3;
  const size_t dense_smem = dense_smem_bytes<double>(wmax);
  const size_t dense_smem32 = dense_smem_bytes<float>(wmax);
  // order and shared memory of the dense kernels in the current pass: three
  // times the pass's widest block (the narrow first pass needs far less, so
  // many more blocks share an SM)
  int wcur = wmax;
  size_t dsm = dense_smem, dsm32 = dense_smem32;
  auto set_dense = [&](int w) {
    wcur = std::max(1, std::min(wmax, w));
    dsm = dense_smem_bytes<double>(wcur);
    dsm32 = dense_smem_bytes<float>(wcur);
  };
  GENEO_CUDA(allow_smem(k_svqb<double>));
  GENEO_CUDA(allow_smem(k_svqb<float>));
  GENEO_CUDA(allow_smem(k_cholqr));
  GENEO_CUDA(allow_smem(k_rr<double>));
  GENEO_CUDA(allow_smem(k_rr<dsv>));
  int32_t* redo = nullptr;
  GENEO_TRY(tmp.get(&redo, (size_t)N));
  const size_t nn_smem = sizeof(double) * W3 * W3;
  const size_t gram_smem = sizeof(double) * std::max(2 * kRB * (kMaxW + 1), 16 * kT);
  GENEO_CUDA(allow_smem(k_gram_part<double>));
  // k_gram_one: two chunks of kRB rows x (p + q) padded columns (widths <= 64
  // there, since wider subdomains go to k_gram_part), or the group partials
  const size_t gram1_smem = sizeof(double) * std::max((size_t)2 * kRB * 128, (size_t)16 * kT);
  GENEO_CUDA(allow_smem(k_gram_one<double>));
  GENEO_CUDA(allow_smem(k_gram_one<double, true>));
  GENEO_CUDA(allow_smem(k_gram_one<float>));
  GENEO_CUDA(allow_smem(k_gram_part<float>));
  GENEO_CUDA(allow_smem(k_gemm_nn));
  GENEO_CUDA(allow_smem(k_gemm_ds));
  GENEO_CUDA(allow_smem(k_gemm32<float, float>));
  GENEO_CUDA(allow_smem(k_gemm32<float, double>));
  GENEO_CUDA(allow_smem(k_gemm32<double, double>));

  const bool f32 = h->fp32;
  // Rayleigh-Ritz sweeps in double-single arithmetic in the FP32 mode
  auto rr_launch = [&](const double* Gm, double* Tt, int ld, const int32_t* s_, const int32_t* q_,
                       double* nu_, int ldnu, const int32_t* skip, int wm) {
    if (f32) k_rr<dsv><<<N, kT, dsm, st>>>(Gm, Tt, ld, s_, q_, nu_, ldnu, skip, wm);
    else k_rr<double><<<N, kT, dsm, st>>>(Gm, Tt, ld, s_, q_, nu_, ldnu, skip, wm);
  };
  // Subdomains whose K_j was factored in FP64 (a weak FP32 pivot: coefficient
  // contrast beyond FP32) also orthogonalise in FP64: their K-norms span
  // that contrast, which FP32 Gram matrices and corrections do not resolve.
  // o64 / ok32: per-subdomain flags; n64 of them set.
  int n64 = 0;
  int32_t *o64 = nullptr, *ok32 = nullptr, *skip32 = nullptr, *skip64 = nullptr;
  double* best = nullptr;        // per subdomain: smallest wanted residual so far
  int32_t* stall = nullptr;      // iterations since it last halved
  if (f32) {
    GENEO_TRY(tmp.get(&best, (size_t)N));
    GENEO_TRY(tmp.get(&stall, (size_t)N));
    std::vector<int32_t> ho(N, 0), hk(N, 1);
    for (int j = 0; j < N; ++j)
      if ((int)asmb.hbandK.size() == N && asmb.hbandK[j].n == 0) { ho[j] = 1; hk[j] = 0; ++n64; }
    GENEO_TRY(tmp.get(&o64, (size_t)N));
    GENEO_TRY(tmp.get(&ok32, (size_t)N));
    GENEO_TRY(tmp.get(&skip32, (size_t)N));
    GENEO_TRY(tmp.get(&skip64, (size_t)N));
    GENEO_CUDA(cudaMemcpyAsync(o64, ho.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, st));
    GENEO_CUDA(cudaMemcpyAsync(ok32, hk.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, st));
  }
  // FP32 copies for the first orthogonalisation pass: [X, Q] and [KX, KQ]
  // (same layout as S and KS) and the values of K
  // With FP32 factors the FP64 products with K and B run in double-single
  // arithmetic (k_spmm_ds): K and B as (hi, lo) float pairs in ELLPACK
  // layout, the operand split into pairs in X2, which overlays S32 and KS32
  // (dead at every such product) first.
  // Subdomains orthogonalised in FP64 (o64) keep FP64 products: their
  // contrast makes K x cancel beyond double-single accuracy.
  float *S32 = nullptr, *KS32 = nullptr, *lK32 = nullptr;
  float2 *eK2 = nullptr, *eB2 = nullptr, *X2 = nullptr;
  int32_t *ecol = nullptr, *dsk1 = nullptr, *dsk2 = nullptr;
  int ell = 0;  // ELLPACK row length (longest local row)
  if (f32) {
    const size_t nz = (size_t)std::max<int64_t>(asmb.lnnz, 1);
    // S32 and KS32 adjoin: X2 (rows x W3 pairs) overlays both
    GENEO_TRY(tmp.get(&S32, (size_t)rows * W3 * 2));
    KS32 = S32 + (size_t)rows * W3;
    X2 = reinterpret_cast<float2*>(S32);
    GENEO_TRY(tmp.get(&lK32, nz));
    GENEO_TRY(tmp.get(&dsk1, (size_t)N));
    GENEO_TRY(tmp.get(&dsk2, (size_t)N));
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((asmb.lnnz + kT - 1) / kT, 152 * 16));
    k_to_f32<<<g, kT, 0, st>>>(asmb.lK, lK32, asmb.lnnz); note_launch();
    int32_t* dl = dsk1;
    GENEO_CUDA(cudaMemsetAsync(dl, 0, sizeof(int32_t), st));
    k_max_rowlen<<<152 * 4, kT, 0, st>>>(asmb.lrow, rows, dl); note_launch();
    GENEO_CUDA(cudaMemcpyAsync(&ell, dl, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    GENEO_CUDA(cudaStreamSynchronize(st));
    const size_t ne = (size_t)std::max<int64_t>(rows * (int64_t)ell, 1);
    GENEO_TRY(tmp.get(&ecol, ne));
    GENEO_TRY(tmp.get(&eK2, ne));
    GENEO_TRY(tmp.get(&eB2, ne));
    k_build_ell<<<gridR, kT, 0, st>>>(h->dsub, asmb.lrow, asmb.lcol, asmb.lK, asmb.lB, ell, ecol, eK2, eB2);
    note_launch();
    GENEO_CUDA(cudaGetLastError());
  }
  std::vector<int64_t> hxoff(N);
  for (int j = 0; j < N; ++j) hxoff[j] = h->hsub[j].offN * (int64_t)W3;
  int64_t *xoffX, *xoffQ;
  GENEO_TRY(tmp.get(&xoffX, (size_t)N));
  GENEO_TRY(tmp.get(&xoffQ, (size_t)N));
  GENEO_CUDA(cudaMemcpyAsync(xoffX, hxoff.data(), sizeof(int64_t) * N, cudaMemcpyHostToDevice, st));

  EventTimer evs;
  std::vector<double> kflops(N);
  for (int j = 0; j < N; ++j) kflops[j] = band_solve_flops(h->hsub[j].nN, h->hsub[j].wK);
  h->eig_flops = 0.0;
  // the K_j factors (FP32 and FP64 refactorisations) in size classes
  SolveSet setK;
  GENEO_TRY(make_solve_set(asmb.bandK, !f32, asmb.dbandK, N, f32 ? asmb.bandK64 : nullptr,
                           f32 ? asmb.dbandK64 : nullptr, f32 ? asmb.nK64 : 0, tmp, st, &setK, true));
  auto solveK_raw = [&](int64_t* xoff, const int32_t* ncols, const int32_t* skip, int kmax,
                        int active) -> geneo_status_t {
    return solve_set_run(setK, h->solve_streams, S, xoff, kmax, ncols, skip, h->dstat, st,
                         o.eig_solve_tf32 ? 1 : 3, 0, active);
  };
  // timed with CUDA events; flops from the per-subdomain column counts
  auto solveK = [&](int64_t* xoff, const int32_t* ncols, const int32_t* skip) -> geneo_status_t {
    std::vector<int32_t> hc(N), hk(N, 0);
    GENEO_CUDA(cudaMemcpyAsync(hc.data(), ncols, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, st));
    if (skip) GENEO_CUDA(cudaMemcpyAsync(hk.data(), skip, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, st));
    GENEO_CUDA(cudaStreamSynchronize(st));
    double fl = 0.0, by = 0.0;
    const double esz = f32 ? 4.0 : 8.0;
    // widest block and subdomains left (in the last iterations few remain,
    // and their solves are cut into column parts on the idle SMs)
    int kmax = 0, active = 0;
    for (int j = 0; j < N; ++j)
      if (!hk[j]) {
        kmax = std::max(kmax, (int)hc[j]);
        active += hc[j] > 0;
      }
    for (int j = 0; j < N; ++j)
      if (!hk[j] && hc[j] > 0) {
        fl += kflops[j] * hc[j];
        const bool k64 = f32 && (int)asmb.hbandK.size() == N && asmb.hbandK[j].n == 0;  // factored in FP64
        by += 2.0 * (k64 ? 8.0 : esz) * band_entries(h->hsub[j].nN, h->hsub[j].wK) + 16.0 * h->hsub[j].nN * hc[j];
      }
    h->eig_flops += fl;
    const int pr = h->prof.begin(GENEO_PROF_EIG_SOLVE, fl, by, st);
    evs.start(st);
    geneo_status_t r = kmax > 0 ? solveK_raw(xoff, ncols, skip, kmax, active) : GENEO_OK;
    h->prof.end(pr, st);
    evs.stop();
    h->eig_ms = evs.ms;
    return r;
  };
  // --- profile mode: host copies of the per-subdomain widths of a launch
  const bool prof = h->prof.on;
  std::vector<int64_t> hnnz(N, 0);
  if (prof) {
    int64_t* dnnz = nullptr;
    GENEO_TRY(tmp.get(&dnnz, (size_t)N));
    k_sub_nnz<<<ceil_div(N, 128), 128, 0, st>>>(h->dsub, asmb.lrow, dnnz, N); note_launch();
    GENEO_CUDA(cudaMemcpyAsync(hnnz.data(), dnnz, sizeof(int64_t) * N, cudaMemcpyDeviceToHost, st));
    GENEO_CUDA(cudaStreamSynchronize(st));
  }
  // widths of a column reference per subdomain (0 for skipped subdomains)
  auto host_widths = [&](const auto& R, const int32_t* skip, std::vector<int>& out) -> geneo_status_t {
    out.assign(N, R.w);
    std::vector<int32_t> t(N), sk(N, 0);
    if (skip) GENEO_CUDA(cudaMemcpyAsync(sk.data(), skip, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, st));
    const int32_t* srcs[2] = {R.wd, R.wd2};
    for (const int32_t* src : srcs) {
      if (!src) continue;
      GENEO_CUDA(cudaMemcpyAsync(t.data(), src, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, st));
      GENEO_CUDA(cudaStreamSynchronize(st));
      for (int j = 0; j < N; ++j) out[j] += t[j];
    }
    GENEO_CUDA(cudaStreamSynchronize(st));
    for (int j = 0; j < N; ++j) if (sk[j]) out[j] = 0;
    return GENEO_OK;
  };
  // Launches on FP32 copies are profiled as their own family.
  auto gram = [&](auto A, auto B, int sym, const int32_t* skip) -> geneo_status_t {
    using S = std::remove_pointer_t<decltype(A.base)>;
    double fl = 0.0, by = 0.0;
    if (prof) {
      std::vector<int> wa, wb;
      GENEO_TRY(host_widths(A, skip, wa));
      GENEO_TRY(host_widths(B, skip, wb));
      for (int j = 0; j < N; ++j) {
        const double n = h->hsub[j].nN;
        fl += sym ? n * wa[j] * (wa[j] + 1.0) : 2.0 * n * wa[j] * wb[j];
        by += sizeof(S) * n * (wa[j] + (sym ? 0 : wb[j]));
      }
    }
    const int pr = h->prof.begin(sizeof(S) == 4 ? GENEO_PROF_ORTHO32 : GENEO_PROF_GRAM, fl, by, st);
    // FP32 mode: double-single products (FP64 where the subdomain is o64)
    bool one_done = false;
    if constexpr (sizeof(S) == 8) {
      if (f32 && n64 < N) {
        const int32_t* sds = skip;
        const int32_t* s64 = nullptr;
        if (n64 > 0) {
          k_split_skip<<<ceil_div(N, 128), 128, 0, st>>>(skip, o64, dsk1, dsk2, N); note_launch();
          sds = dsk1;
          s64 = dsk2;
        }
        k_gram_one<double, true><<<dim3(kRS, N), kT, gram1_smem, st>>>(h->dsub, A, B, sym, Gp, ldg, N, sds);
        note_launch();
        if (s64) {
          k_gram_one<double, false><<<dim3(kRS, N), kT, gram1_smem, st>>>(h->dsub, A, B, sym, Gp, ldg, N, s64);
          note_launch();
        }
        one_done = true;
      }
    }
    if (!one_done) {
      k_gram_one<S><<<dim3(kRS, N), kT, gram1_smem, st>>>(h->dsub, A, B, sym, Gp, ldg, N, skip); note_launch();
    }
    if (W3 > 64) {
      k_gram_part<S><<<dim3(kRS, N), kT, gram_smem, st>>>(h->dsub, A, B, sym, Gp, ldg, N, skip, 1);
      note_launch();
    }
    k_gram_reduce<S><<<N, kT, 0, st>>>(h->dsub, A, B, sym, Gp, G, ldg, N, skip); note_launch();
    h->prof.end(pr, st);
    GENEO_CUDA(cudaGetLastError());
    return GENEO_OK;
  };
  auto gemm_cost = [&](const auto& A, const auto& C, double beta, const int32_t* skip, double esz,
                       double& fl, double& by) -> geneo_status_t {
    fl = 0.0;
    by = 0.0;
    if (!prof) return GENEO_OK;
    std::vector<int> wa, wc;
    GENEO_TRY(host_widths(A, skip, wa));
    GENEO_TRY(host_widths(C, skip, wc));
    for (int j = 0; j < N; ++j) {
      const double n = h->hsub[j].nN;
      fl += 2.0 * n * wa[j] * wc[j];
      by += esz * n * (wa[j] + wc[j] * (beta == 0.0 ? 1.0 : 2.0));
    }
    return GENEO_OK;
  };
  // FP64 C = beta C + alpha A T
  auto gemm = [&](ColRef A, const double* Tmat, int t0, const int32_t* t0d, ColRef C, double alpha,
                  double beta, const int32_t* skip) -> geneo_status_t {
    double fl, by;
    GENEO_TRY(gemm_cost(A, C, beta, skip, 8.0, fl, by));
    const int pr = h->prof.begin(GENEO_PROF_GEMM, fl, by, st);
    const int32_t* sk = skip;  // subdomains left for the FP64 kernel
    bool all_ds = false;
    if (f32 && n64 < N) {  // double-single arithmetic except for the o64 subdomains
      const int32_t* sds = skip;
      if (n64 > 0) {
        k_split_skip<<<ceil_div(N, 128), 128, 0, st>>>(skip, o64, dsk1, dsk2, N); note_launch();
        sds = dsk1;
        sk = dsk2;
      }
      k_gemm_ds<<<gridR, kT, nn_smem, st>>>(h->dsub, A, Tmat, ldg, t0, t0d, C, alpha, beta, sds); note_launch();
      all_ds = n64 == 0;
    }
    if (!all_ds) {
      k_gemm_nn<<<gridR, kT, nn_smem, st>>>(h->dsub, A, Tmat, ldg, t0, t0d, C, alpha, beta, sk); note_launch();
    }
    h->prof.end(pr, st);
    GENEO_CUDA(cudaGetLastError());
    return GENEO_OK;
  };
  // FP32-arithmetic C = beta C + alpha A T (epilogue rules at k_gemm32)
  auto gemm32 = [&](auto A, const double* Tmat, int t0, const int32_t* t0d, auto C, double alpha,
                    double beta, const int32_t* skip, int corr, int addI = 0,
                    const int32_t* f64flag = nullptr) -> geneo_status_t {
    using SA = std::remove_pointer_t<decltype(A.base)>;
    using SO = std::remove_pointer_t<decltype(C.base)>;
    double fl, by;
    GENEO_TRY(gemm_cost(A, C, beta, skip, 4.0, fl, by));
    const int pr = h->prof.begin(GENEO_PROF_ORTHO32, fl, by, st);
    k_gemm32<SA, SO><<<gridR, kT, nn_smem, st>>>(h->dsub, A, Tmat, ldg, t0, t0d, C, alpha, beta, skip,
                                                 corr, addI, f64flag);
    note_launch();
    h->prof.end(pr, st);
    GENEO_CUDA(cudaGetLastError());
    return GENEO_OK;
  };
  auto spmm = [&](bool withK, bool withB, auto X, auto YK, auto YB, const int32_t* skip) {
    using S = std::remove_pointer_t<decltype(X.base)>;
    double fl = 0.0, by = 0.0;
    if (prof) {
      std::vector<int> wx;
      if (host_widths(X, skip, wx) != GENEO_OK) wx.assign(N, 0);
      const double nm = (withK && withB) ? 2.0 : 1.0;
      for (int j = 0; j < N; ++j) {
        fl += 2.0 * nm * (double)hnnz[j] * wx[j];
        by += (double)hnnz[j] * (4.0 + sizeof(S) * nm) + sizeof(S) * h->hsub[j].nN * wx[j] * (1.0 + nm);
      }
    }
    const int pr = h->prof.begin(sizeof(S) == 4 ? GENEO_PROF_ORTHO32 : GENEO_PROF_SPMM, fl, by, st);
    const S* vK;
    const S* vB;
    if constexpr (sizeof(S) == 4) {
      vK = lK32;
      vB = nullptr;
    } else {
      vK = asmb.lK;
      vB = asmb.lB;
    }
    const int32_t* sk = skip;  // subdomains left for the plain kernel
    if constexpr (sizeof(S) == 8) {
      if (f32 && X.W == W3 && n64 < N) {
        const int32_t* sds = skip;
        if (n64 > 0) {
          k_split_skip<<<ceil_div(N, 128), 128, 0, st>>>(skip, o64, dsk1, dsk2, N); note_launch();
          sds = dsk1;
          sk = dsk2;
        }
        const ColRefT<float2> Xs{X2, X.W, X.c0, X.c0d, X.w, X.wd, X.wd2};
        k_split_cols<<<gridR, kT, 0, st>>>(h->dsub, X, Xs, sds); note_launch();
        const bool both = withK && withB;
        k_spmm_ds<<<gridR, kT, 0, st>>>(h->dsub, ell, ecol, withK ? eK2 : eB2, both ? eB2 : nullptr, Xs,
                                        withK ? YK : YB, YB, sds);
        note_launch();
        if (n64 == 0) {
          h->prof.end(pr, st);
          return;
        }
      }
    }
    if (withK && withB) {
      k_spmm<S><<<gridR, kT, 0, st>>>(h->dsub, asmb.lrow, asmb.lcol, vK, vB, X, YK, YB, sk);
    } else if (withK) {
      k_spmm<S><<<gridR, kT, 0, st>>>(h->dsub, asmb.lrow, asmb.lcol, vK, nullptr, X, YK, YK, sk);
    } else {
      k_spmm<S><<<gridR, kT, 0, st>>>(h->dsub, asmb.lrow, asmb.lcol, vB, nullptr, X, YB, YB, sk);
    }
    note_launch();
    h->prof.end(pr, st);
  };
  // storage conversion of a column block (FP64 <-> FP32 copies)
  auto cvt = [&](auto Src, auto Dst, const int32_t* skip) {
    using SS = std::remove_pointer_t<decltype(Src.base)>;
    using SD = std::remove_pointer_t<decltype(Dst.base)>;
    const int pr = h->prof.begin(GENEO_PROF_ORTHO32, 0.0, 0.0, st);
    k_copy_cols<SS, SD><<<gridR, kT, 0, st>>>(h->dsub, Src, Dst, skip); note_launch();
    h->prof.end(pr, st);
  };

  // Column references
  const ColRef Xr = cref(S, W3, 0, nullptr, 0, sj);
  const ColRef KXr = cref(KS, W3, 0, nullptr, 0, sj);
  const ColRef BXr = cref(BS, W3, 0, nullptr, 0, sj);
  const ColRef Qr = cref(S, W3, 0, sj, 0, qj);        // Q after X
  const ColRef KQr = cref(KS, W3, 0, sj, 0, qj);
  const ColRef Pr = cref(P, W3 / 3, 0, nullptr, 0, spj);
  const ColRef Sr = cref(S, W3, 0, nullptr, 0, sj, qj);  // [X, Q]
  const ColRef BSr = cref(BS, W3, 0, nullptr, 0, sj, qj);
  const ColRef BQr = cref(BS, W3, 0, sj, 0, qj);
  const ColRef32 Sr32 = cref(S32, W3, 0, nullptr, 0, sj, qj);   // FP32 [X, Q]
  const ColRef32 Xr32 = cref(S32, W3, 0, nullptr, 0, sj);
  const ColRef32 Qr32 = cref(S32, W3, 0, sj, 0, qj);
  const ColRef32 KXr32 = cref(KS32, W3, 0, nullptr, 0, sj);
  const ColRef32 KQr32 = cref(KS32, W3, 0, sj, 0, qj);

  // Start block for the subdomains with skip[j] == 0: X = K^{-1} B R
  // (R counter-based random), K-orthonormalised by SVQB, Rayleigh-Ritz.
  auto init_block = [&](const int32_t* skip, uint64_t seed) -> geneo_status_t {
    k_init_random<<<gridR, kT, 0, st>>>(h->dsub, cref(Tmp, W3, 0, nullptr, 0, sj), seed, skip); note_launch();
    spmm(false, true, cref(Tmp, W3, 0, nullptr, 0, sj), Xr, Xr, skip);   // S[:, 0:s] = B R
    GENEO_CUDA(cudaGetLastError());
    GENEO_TRY(solveK(xoffX, sj, skip));
    spmm(true, false, Xr, KXr, KXr, skip);
    GENEO_TRY(gram(Xr, KXr, 1, skip));
    { const int prs = h->prof.begin(GENEO_PROF_SMALL_EIG, 0.0, 0.0, st); k_svqb<double><<<N, kT, dsm, st>>>(G, Tm, ldg, sj, nullptr, rj, 1e-14, skip, wcur); note_launch(); h->prof.end(prs, st); }
    GENEO_TRY(gemm(Xr, Tm, 0, nullptr, cref(Tmp, W3, 0, nullptr, 0, rj), 1.0, 0.0, skip));
    k_set_i32<<<ceil_div(N, 128), 128, 0, st>>>(sj, rj, N, skip); note_launch();
    k_copy_cols<double, double><<<gridR, kT, 0, st>>>(h->dsub, cref(Tmp, W3, 0, nullptr, 0, sj), Xr, skip); note_launch();
    spmm(false, true, Xr, BXr, BXr, skip);
    GENEO_TRY(gram(Xr, BXr, 1, skip));
    { const int prs = h->prof.begin(GENEO_PROF_SMALL_EIG, 0.0, 0.0, st); rr_launch(G, Tm, ldg, sj, nullptr, nu, s, skip, wcur); note_launch(); h->prof.end(prs, st); }
    GENEO_TRY(gemm(Xr, Tm, 0, nullptr, cref(Tmp, W3, 0, nullptr, 0, sj), 1.0, 0.0, skip));
    k_copy_cols<double, double><<<gridR, kT, 0, st>>>(h->dsub, cref(Tmp, W3, 0, nullptr, 0, sj), Xr, skip); note_launch();
    GENEO_CUDA(cudaGetLastError());
    return GENEO_OK;
  };
  std::vector<int64_t> hq(N);
  int total_it = 0;
  auto iterate = [&]() -> geneo_status_t {
    int remaining = N;
    for (int it = 0; it < o.eig_maxit; ++it, ++total_it) {
      spmm(true, true, Xr, KXr, BXr, done);
      GENEO_CUDA(cudaMemsetAsync(notdone, 0, 2 * sizeof(int32_t), st));
      k_resid<<<N, kT, 0, st>>>(h->dsub, cref(S, W3, 0, nullptr, 0, nullptr), BXr, KXr, Pr, nu, s, sj,
                                spj, aj, qj, done, iters, notdone, rn, o.eig_tol, o.tau, o.sigma, nevj,
                                o.fixed_nev, it, f32 ? best : nullptr, stall, o64, ok32, kStallIts); note_launch();
      GENEO_CUDA(cudaGetLastError());
      int32_t cnt[2] = {0, 0};
      GENEO_CUDA(cudaMemcpyAsync(cnt, notdone, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      GENEO_CUDA(cudaStreamSynchronize(st));
      remaining = cnt[0];
      n64 += cnt[1];
      if (remaining == 0) break;
      // W = K^{-1} R (active columns start at column s_j)
      std::vector<int32_t> hsj(N);
      GENEO_CUDA(cudaMemcpyAsync(hsj.data(), sj, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, st));
      GENEO_CUDA(cudaStreamSynchronize(st));
      for (int j = 0; j < N; ++j) hq[j] = hxoff[j] + (int64_t)hsj[j] * h->hsub[j].nN;
      GENEO_CUDA(cudaMemcpyAsync(xoffQ, hq.data(), sizeof(int64_t) * N, cudaMemcpyHostToDevice, st));
      GENEO_TRY(solveK(xoffQ, aj, done));
      // Q = [W, P]: K-orthogonalise against X and K-orthonormalise by SVQB,
      // twice.  SVQB's rescaling of nearly dependent directions amplifies the
      // residual X-components a single round leaves, and the Rayleigh-Ritz
      // step below assumes a K-orthonormal [X, Q].
      // X^T K Q is formed as (KX)^T Q: KX from the residual step is current.
      // With FP32 factors the first pass runs on FP32 copies of X, Q and KX
      // (it removes the bulk of the X components); the second, FP64 pass sets
      // the final K-orthonormality that Rayleigh-Ritz relies on.
      // with FP32 factors, the FP32 flavour skips s32 and the FP64 one s64
      const int32_t* s32 = done;
      const int32_t* s64 = nullptr;
      if (f32 && n64 > 0) {
        k_split_skip<<<ceil_div(N, 128), 128, 0, st>>>(done, o64, skip32, skip64, N); note_launch();
        s32 = skip32;
        s64 = skip64;
      }
      const bool any32 = f32 && n64 < N;
      for (int pass = 0; pass < 2; ++pass) {
        if (f32 && pass == 0) {
          if (any32) {
            cvt(Sr, Sr32, s32);
            cvt(KXr, KXr32, s32);
            GENEO_TRY(gram(KXr32, Qr32, 0, s32));
            GENEO_TRY(gemm32(Xr32, G, 0, nullptr, Qr32, -1.0, 1.0, s32, 0));
            spmm(true, false, Qr32, KQr32, KQr32, s32);
            GENEO_TRY(gram(Qr32, KQr32, 1, s32));
            {
              const int prs = h->prof.begin(GENEO_PROF_SMALL_EIG, 0.0, 0.0, st);
              k_svqb<float><<<N, kT, dsm32, st>>>(G, Tm, ldg, qj, nullptr, rj, 1e-12, s32, wcur); note_launch();
              h->prof.end(prs, st);
            }
            // Q = Q32 T straight into the FP64 block (no aliasing: T acts on the copy)
            GENEO_TRY(gemm32(Qr32, Tm, 0, nullptr, cref(S, W3, 0, sj, 0, rj), 1.0, 0.0, s32, 1));
            k_set_i32<<<ceil_div(N, 128), 128, 0, st>>>(qj, rj, N, s32); note_launch();
            GENEO_CUDA(cudaGetLastError());
          }
          if (!s64) continue;
        }
        // FP64 pass (the first pass of the o64 subdomains when pass == 0)
        const int32_t* sp = (f32 && pass == 0) ? s64 : done;
        GENEO_TRY(gram(KXr, Qr, 0, sp));
        // after an FP32 first pass X G is a small correction: FP32 product,
        // subtracted in FP64
        if (f32 && pass == 1) {
          if (any32) GENEO_TRY(gemm32(Xr32, G, 0, nullptr, Qr, -1.0, 1.0, s32, 1));
          if (s64) GENEO_TRY(gemm(Xr, G, 0, nullptr, Qr, -1.0, 1.0, s64));
        } else {
          GENEO_TRY(gemm(Xr, G, 0, nullptr, Qr, -1.0, 1.0, sp));
        }
        spmm(true, false, Qr, KQr, KQr, sp);
        GENEO_TRY(gram(Qr, KQr, 1, sp));
        {
          const int prs = h->prof.begin(GENEO_PROF_SMALL_EIG, 0.0, 0.0, st);
          if (pass == 0) {
            k_svqb<double><<<N, kT, dsm, st>>>(G, Tm, ldg, qj, nullptr, rj, 1e-12, sp, wcur);
            note_launch();
          } else {
            // the block is nearly K-orthonormal: Cholesky QR, SVQB where a
            // pivot is too small
            k_fill_i32<<<ceil_div(N, 128), 128, 0, st>>>(rj, -1, N); note_launch();
            k_cholqr<<<N, kT, dsm, st>>>(G, Tm, ldg, qj, rj, 1e-12, done, wcur); note_launch();
            k_mark_fallback<<<ceil_div(N, 128), 128, 0, st>>>(rj, done, redo, N); note_launch();
            k_svqb<double><<<N, kT, dsm, st>>>(G, Tm, ldg, qj, nullptr, rj, 1e-12, redo, wcur); note_launch();
            if (f32 && n64 > 0) { k_and_not<<<ceil_div(N, 128), 128, 0, st>>>(redo, o64, N); note_launch(); }
          }
          h->prof.end(prs, st);
        }
        // second pass with FP32 factors: T = D L^{-T} is near I where
        // Cholesky QR succeeded (redo[j] == 1): Q T = Q + Q (T - I) with an
        // FP32 product; the SVQB fallback and o64 subdomains stay FP64
        if (pass == 1 && f32)
          GENEO_TRY(gemm32(Qr, Tm, 0, nullptr, cref(Tmp, W3, 0, nullptr, 0, rj), 1.0, 0.0, done, 1, 1, redo));
        else
          GENEO_TRY(gemm(Qr, Tm, 0, nullptr, cref(Tmp, W3, 0, nullptr, 0, rj), 1.0, 0.0, sp));
        k_set_i32<<<ceil_div(N, 128), 128, 0, st>>>(qj, rj, N, sp); note_launch();
        k_copy_cols<double, double><<<gridR, kT, 0, st>>>(h->dsub, cref(Tmp, W3, 0, nullptr, 0, qj), Qr, sp); note_launch();
        GENEO_CUDA(cudaGetLastError());
      }
      // Rayleigh-Ritz on S = [X, Q]; BX from the residual step is current,
      // only BQ is new
      spmm(false, true, Qr, BQr, BQr, done);
      GENEO_TRY(gram(Sr, BSr, 1, done));
      { const int prs = h->prof.begin(GENEO_PROF_SMALL_EIG, 0.0, 0.0, st); rr_launch(G, Tm, ldg, sj, qj, nu, s, done, wcur); note_launch(); h->prof.end(prs, st); }
      // P = Q U[s_j:, :], X = S U
      // P only spans the next search block: FP32 arithmetic with FP32 factors
      if (f32) GENEO_TRY(gemm32(Qr, Tm, 0, sj, cref(P, s, 0, nullptr, 0, sj), 1.0, 0.0, done, 0, 0,
                                n64 > 0 ? ok32 : nullptr));
      else GENEO_TRY(gemm(Qr, Tm, 0, sj, cref(P, s, 0, nullptr, 0, sj), 1.0, 0.0, done));
      k_set_i32<<<ceil_div(N, 128), 128, 0, st>>>(spj, sj, N, done); note_launch();
      GENEO_TRY(gemm(Sr, Tm, 0, nullptr, cref(Tmp, W3, 0, nullptr, 0, sj), 1.0, 0.0, done));
      k_copy_cols<double, double><<<gridR, kT, 0, st>>>(h->dsub, cref(Tmp, W3, 0, nullptr, 0, sj), Xr, done); note_launch();
      GENEO_CUDA(cudaGetLastError());
      GENEO_TRY(check_status(h, st));
    }
    return GENEO_OK;
  };

  auto t0 = std::chrono::steady_clock::now();
  // Pass 1 with a narrow block: most subdomains have only a few eigenvalues
  // below tau.  A subdomain whose narrow block fills with converged
  // eigenvalues below tau is solved again with the full width (pass 2).
  const int guard = s - nev;
  const int nev1 = o.fixed_nev ? nev : std::min(nev, o.first_nev > 0 ? o.first_nev : kFirstPassNev);
  {
    std::vector<int32_t> hs1(N), hn1(N, nev1);
    int smax = 1;
    for (int j = 0; j < N; ++j) {
      hs1[j] = std::min(nev1 + guard, h->hsub[j].nN);
      smax = std::max(smax, hs1[j]);
    }
    set_dense(3 * smax);
    GENEO_CUDA(cudaMemcpyAsync(sj, hs1.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, st));
    GENEO_CUDA(cudaMemcpyAsync(nevj, hn1.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, st));
  }
  GENEO_TRY(init_block(nullptr, o.seed));
  GENEO_TRY(iterate());
  // subdomains the first pass left unconverged at eig_maxit
  std::vector<int32_t> hdone1(N), unconv(N, 0);
  GENEO_CUDA(cudaMemcpyAsync(hdone1.data(), done, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, st));
  GENEO_CUDA(cudaStreamSynchronize(st));
  for (int j = 0; j < N; ++j) unconv[j] = hdone1[j] ? 0 : 1;
  if (nev1 < nev) {
    std::vector<double> hnu1((size_t)N * s);
    GENEO_CUDA(cudaMemcpyAsync(hnu1.data(), nu, sizeof(double) * N * s, cudaMemcpyDeviceToHost, st));
    GENEO_CUDA(cudaStreamSynchronize(st));
    std::vector<int32_t> redo(N, 1), hs2(N), hn2(N, nev);
    int nredo = 0;
    for (int j = 0; j < N; ++j) {
      int below = 0;
      for (int i = 0; i < nev1; ++i) {
        const double v = hnu1[(size_t)j * s + i];
        if (v > 0.0 && o.sigma + 1.0 / v < o.tau) ++below;
      }
      hs2[j] = std::min(s, h->hsub[j].nN);
      if (below >= nev1 && hs2[j] > nev1) {
        redo[j] = 0;   // skip flag 0: solve again
        ++nredo;
      }
    }
    h->eig_second_pass = nredo;
    if (nredo > 0) {
      // done[j] = 1 for the others; widen the block of the redone ones
      for (int j = 0; j < N; ++j) if (redo[j]) hs2[j] = -1;
      std::vector<int32_t> hsj_now(N);
      GENEO_CUDA(cudaMemcpyAsync(hsj_now.data(), sj, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, st));
      GENEO_CUDA(cudaStreamSynchronize(st));
      for (int j = 0; j < N; ++j) if (hs2[j] < 0) hs2[j] = hsj_now[j];
      GENEO_CUDA(cudaMemcpyAsync(sj, hs2.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, st));
      GENEO_CUDA(cudaMemcpyAsync(nevj, hn2.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, st));
      GENEO_CUDA(cudaMemcpyAsync(done, redo.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, st));
      k_clear_p<<<ceil_div(N, 128), 128, 0, st>>>(spj, done, N); note_launch();
      set_dense(wmax);
      GENEO_TRY(init_block(done, o.seed ^ 0x9E3779B97F4A7C15ull));
      GENEO_TRY(iterate());
      // a redone subdomain counts by its second pass
      std::vector<int32_t> hdone2(N);
      GENEO_CUDA(cudaMemcpyAsync(hdone2.data(), done, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, st));
      GENEO_CUDA(cudaStreamSynchronize(st));
      for (int j = 0; j < N; ++j)
        if (!redo[j]) unconv[j] = hdone2[j] ? 0 : 1;
    }
  }
  h->eig_unconv = 0;
  for (int j = 0; j < N; ++j) h->eig_unconv += unconv[j];
  const int it = total_it;
  h->eig_iters = it;
  h->eig_o64 = n64;
  h->setup_ms[3] = ms_since(t0);
  // eigenvalues lambda = sigma + 1/nu (ascending in lambda = descending nu)
  std::vector<double> hnu((size_t)N * s);
  std::vector<int32_t> hsj(N);
  GENEO_CUDA(cudaMemcpyAsync(hnu.data(), nu, sizeof(double) * N * s, cudaMemcpyDeviceToHost, st));
  GENEO_CUDA(cudaMemcpyAsync(hsj.data(), sj, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, st));
  GENEO_CUDA(cudaStreamSynchronize(st));
  h->lambda_host.assign((size_t)N * s, INFINITY);
  for (int j = 0; j < N; ++j) {
    h->hsub[j].s = hsj[j];
    for (int i = 0; i < hsj[j]; ++i) {
      const double v = hnu[(size_t)j * s + i];
      h->lambda_host[(size_t)j * s + i] = v > 0.0 ? o.sigma + 1.0 / v : INFINITY;
    }
  }
  *X_out = S;  // X occupies columns [0, s_j) of S (buffer width 3s)
  return check_status(h, st);
}

}  // namespace geneo
