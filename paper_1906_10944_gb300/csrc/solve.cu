// Two-level additive Schwarz application and preconditioned CG.
//
// Section 3, Definition 2:
//   z = sum_j R_j^T A_j^{-1} R_j r + R_H^T A_H^{-1} R_H r,
// Section 4.5: (R_H r)_i = phi_i . r and R_H^T y = sum_i phi_i y_i.
// Steps on the device:
//   1. per subdomain: u_j = r[D_j] (restriction) and c_j = Z_j^T r[D_j]
//   2. batched banded solves L_j L_j^T u_j = u_j
//   3. banded solve of the coarse system A_H y = c
//   4. per global dof k (gather form over the subdomains whose D contains k):
//      z_k = sum_j (u_j[k] + Z_j[k, :] y_j); z_k = r_k on global Dirichlet dofs.
// PCG (Section 5): x0 = 0, stop when ||r||_2 <= tol ||b||_2; all dot
// products are two-stage fixed-order reductions, so iterates are bitwise
// reproducible run to run.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "handle.cuh"

namespace geneo {
namespace {

constexpr int kT = 256;
constexpr int kRedBlocks = 1024;
// allocation-free PCG: largest maxit accepted and scalar slots of its scratch
constexpr int kNoAllocMaxIt = 4095;
constexpr int kNoAllocScalars = 16;

// u_j = R_j r and c_j = Z_j^T r (the restriction to the coarse space) in one
// pass over r: each gathered r value serves u and up to kRm coarse products,
// and the kRm sums share one block reduction (fixed order).
constexpr int kRm = 8;
__global__ void __launch_bounds__(kT)
k_restrict(const SubDesc* __restrict__ sub, const int32_t* __restrict__ Dlist, const double* __restrict__ r,
           const double* __restrict__ Z, double* __restrict__ u, double* __restrict__ c) {
  const int j = blockIdx.x;
  const SubDesc d = sub[j];
  __shared__ double red[kT / 32][kRm];
  const int32_t* Dj = Dlist + d.offN;
  double* uj = u + d.offN;
  const double* zj = Z + d.offZ;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (d.m == 0) {
    for (int i = threadIdx.x; i < d.nD; i += blockDim.x) uj[i] = r[Dj[i]];
    return;
  }
  for (int k0 = 0; k0 < d.m; k0 += kRm) {
    const int km = min(kRm, d.m - k0);
    double acc[kRm];
#pragma unroll
    for (int k = 0; k < kRm; ++k) acc[k] = 0.0;
    for (int i = threadIdx.x; i < d.nD; i += blockDim.x) {
      const double rv = r[Dj[i]];
      if (k0 == 0) uj[i] = rv;
#pragma unroll
      for (int k = 0; k < kRm; ++k)
        if (k < km) acc[k] += zj[(int64_t)(k0 + k) * d.nD + i] * rv;
    }
#pragma unroll
    for (int k = 0; k < kRm; ++k) {
      const double v = warp_sum(acc[k]);
      if (lane == 0) red[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < km) {
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += red[w][threadIdx.x];
      c[d.offH + k0 + threadIdx.x] = t;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kT)
k_prolong(int64_t n, const uint8_t* __restrict__ dir, const double* __restrict__ r,
          const int64_t* __restrict__ invD_ptr, const int32_t* __restrict__ invD_sub,
          const int32_t* __restrict__ invD_loc, const SubDesc* __restrict__ sub,
          const double* __restrict__ u, const double* __restrict__ Z, const double* __restrict__ y,
          double* __restrict__ z) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    if (dir[k]) {
      z[k] = r[k];
      continue;
    }
    double acc = 0.0;
    for (int64_t t = invD_ptr[k]; t < invD_ptr[k + 1]; ++t) {
      const int j = invD_sub[t], i = invD_loc[t];
      const SubDesc& d = sub[j];
      double v = u[d.offN + i];
      const double* zr = Z + d.offZ + i;
      for (int c = 0; c < d.m; ++c) v += zr[(int64_t)c * d.nD] * y[d.offH + c];
      acc += v;
    }
    z[k] = acc;
  }
}

__global__ void __launch_bounds__(kT)
k_dot(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ part) {
  __shared__ double red[kT / 32];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s += a[i] * b[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// ---------------------------------------------------------------------------
// SELL-32 copy of A for the PCG products (one thread per row, the 32 rows of
// a slice in one warp, so every value and column load is one coalesced
// 128- or 256-byte access; the p gathers hit L2).  Built once per handle.
// ---------------------------------------------------------------------------
// slice length: 32 x the longest row of the slice
__global__ void k_sell_len(int64_t n, const int64_t* __restrict__ rowptr, int64_t* __restrict__ len) {
  const int lane = threadIdx.x & 31;
  const int64_t nsl = (n + 31) / 32;
  for (int64_t sl = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; sl < nsl;
       sl += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t r = sl * 32 + lane;
    int l = r < n ? (int)(rowptr[r + 1] - rowptr[r]) : 0;
    for (int o = 16; o > 0; o >>= 1) l = max(l, __shfl_xor_sync(0xffffffffu, l, o));
    if (lane == 0) len[sl] = 32 * (int64_t)l;
  }
}

__global__ void k_sell_fill(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            const double* __restrict__ val, const int64_t* __restrict__ off,
                            int32_t* __restrict__ scol, double* __restrict__ sval) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < ((n + 31) & ~(int64_t)31);
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sl = r >> 5, l = r & 31;
    const int64_t o = off[sl], w = (off[sl + 1] - o) >> 5;
    const int64_t b = r < n ? rowptr[r] : 0, len = r < n ? rowptr[r + 1] - b : 0;
    for (int64_t t = 0; t < w; ++t) {
      const bool in = t < len;
      scol[o + 32 * t + l] = in ? col[b + t] : (int32_t)(r < n ? r : 0);
      sval[o + 32 * t + l] = in ? val[b + t] : 0.0;
    }
  }
}

// y = A x for the rows of two slices at once (lane l: rows 32 sl + l and
// 32 sl2 + l; sl2 < 0: none), four products of each in flight
__device__ __forceinline__ void sell_row2(const int64_t* __restrict__ off, const int32_t* __restrict__ scol,
                                          const double* __restrict__ sval, const double* __restrict__ x,
                                          int64_t sl, int64_t sl2, int l, double* y) {
  const int64_t oa = off[sl] + l;
  const int wa = (int)((off[sl + 1] - off[sl]) >> 5);
  const int64_t ob = sl2 >= 0 ? off[sl2] + l : 0;
  const int wb = sl2 >= 0 ? (int)((off[sl2 + 1] - off[sl2]) >> 5) : 0;
  double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
  const int wm = min(wa, wb);
  int t = 0;
  for (; t + 1 < wm; t += 2) {
    const int64_t ea = oa + 32 * (int64_t)t, eb = ob + 32 * (int64_t)t;
    const double v0 = sval[ea], v1 = sval[ea + 32], u0 = sval[eb], u1 = sval[eb + 32];
    const int32_t c0 = scol[ea], c1 = scol[ea + 32], d0 = scol[eb], d1 = scol[eb + 32];
    a0 += v0 * x[c0];
    a1 += v1 * x[c1];
    b0 += u0 * x[d0];
    b1 += u1 * x[d1];
  }
  for (int ta = t; ta < wa; ++ta) {
    const int64_t e = oa + 32 * (int64_t)ta;
    a0 += sval[e] * x[scol[e]];
  }
  for (int tb = t; tb < wb; ++tb) {
    const int64_t e = ob + 32 * (int64_t)tb;
    b0 += sval[e] * x[scol[e]];
  }
  y[0] = a0 + a1;
  y[1] = b0 + b1;
}

// y = A x for the rows of one slice (lane l: row 32 sl + l), four products in flight
__device__ __forceinline__ double sell_row(const int64_t* __restrict__ off, const int32_t* __restrict__ scol,
                                           const double* __restrict__ sval, const double* __restrict__ x,
                                           int64_t sl, int l) {
  const int64_t o = off[sl] + l;
  const int w = (int)((off[sl + 1] - off[sl]) >> 5);
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int t = 0;
  for (; t + 3 < w; t += 4) {
    const int64_t e = o + 32 * (int64_t)t;
    a0 += sval[e] * x[scol[e]];
    a1 += sval[e + 32] * x[scol[e + 32]];
    a2 += sval[e + 64] * x[scol[e + 64]];
    a3 += sval[e + 96] * x[scol[e + 96]];
  }
  for (; t < w; ++t) {
    const int64_t e = o + 32 * (int64_t)t;
    a0 += sval[e] * x[scol[e]];
  }
  return (a0 + a1) + (a2 + a3);
}

// q = A p; partial sums of p.q per block
__global__ void __launch_bounds__(kT)
k_spmv_sell_dot(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ scol,
                const double* __restrict__ sval, const double* __restrict__ p, double* __restrict__ q,
                double* __restrict__ part) {
  __shared__ double red[kT / 32];
  const int l = threadIdx.x & 31;
  const int64_t nsl = (n + 31) / 32;
  double dsum = 0.0;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t sl = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; sl < nsl; sl += 2 * nw) {
    const int64_t sl2 = sl + nw < nsl ? sl + nw : -1;
    double v[2];
    sell_row2(off, scol, sval, p, sl, sl2, l, v);
    const int64_t r = sl * 32 + l, r2 = (sl + nw) * 32 + l;
    if (r < n) {
      q[r] = v[0];
      dsum += v[0] * p[r];
    }
    if (sl2 >= 0 && r2 < n) {
      q[r2] = v[1];
      dsum += v[1] * p[r2];
    }
  }
  dsum = block_sum(dsum, red);
  if (threadIdx.x == 0) part[blockIdx.x] = dsum;
}

// r = b - A x; partial sums of r.r per block
__global__ void __launch_bounds__(kT)
k_true_resid_sell(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ scol,
                  const double* __restrict__ sval, const double* __restrict__ x, const double* __restrict__ b,
                  double* __restrict__ r, double* __restrict__ part) {
  __shared__ double red[kT / 32];
  const int l = threadIdx.x & 31;
  const int64_t nsl = (n + 31) / 32;
  double rsum = 0.0;
  for (int64_t sl = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; sl < nsl;
       sl += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const double v = sell_row(off, scol, sval, x, sl, l);
    const int64_t i = sl * 32 + l;
    if (i < n) {
      const double ri = b[i] - v;
      r[i] = ri;
      rsum += ri * ri;
    }
  }
  rsum = block_sum(rsum, red);
  if (threadIdx.x == 0) part[blockIdx.x] = rsum;
}

// y = X c with X = A_H^{-1} (symmetric; row i read as column i, contiguous):
// one warp per row
__global__ void __launch_bounds__(kT)
k_coarse_gemv(const double* __restrict__ X, int dim, const double* __restrict__ c, double* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < dim; i += (gridDim.x * blockDim.x) >> 5) {
    const double* xi = X + (int64_t)i * dim;
    double a = 0.0;
    for (int j = lane; j < dim; j += 32) a += xi[j] * c[j];
    a = warp_sum(a);
    if (lane == 0) y[i] = a;
  }
}

// scalars: 0 rz, 1 alpha, 2 beta, 3 rr, 4 pq, 5 bb, 6 flag
__global__ void k_finish(const double* __restrict__ part, int nb, double* __restrict__ scal, int what,
                         double* __restrict__ hist_a, double* __restrict__ hist_b, int it) {
  __shared__ double red[kT / 32];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[i];
  s = block_sum(s, red);
  if (threadIdx.x != 0) return;
  if (what == 0) {            // rz0
    scal[0] = s;
    if (!(s > 0.0)) scal[6] = 1.0;
  } else if (what == 1) {     // alpha = rz / pq
    scal[4] = s;
    if (!(s > 0.0)) { scal[6] = 1.0; scal[1] = 0.0; }
    else scal[1] = scal[0] / s;
    hist_a[it] = scal[1];
  } else if (what == 2) {     // rr
    scal[3] = s;
  } else if (what == 3) {     // beta = rz_new / rz
    if (!(s > 0.0)) scal[6] = 1.0;
    scal[2] = scal[0] > 0.0 ? s / scal[0] : 0.0;
    scal[0] = s;
    hist_b[it] = scal[2];
  } else if (what == 4) {     // bb
    scal[5] = s;
  } else if (what == 5) {     // ||b - A x||^2
    scal[7] = s;
  }
}

__global__ void __launch_bounds__(kT)
k_update_xr(int64_t n, const double* __restrict__ scal, const double* __restrict__ p,
            const double* __restrict__ q, double* __restrict__ x, double* __restrict__ r,
            double* __restrict__ part) {
  __shared__ double red[kT / 32];
  const double alpha = scal[1];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    s += ri * ri;
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_update_p(int64_t n, const double* __restrict__ scal, const double* __restrict__ z,
                           double* __restrict__ p) {
  const double beta = scal[2];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}

// ---------------------------------------------------------------------------
// PCG kernels of the non-deterministic mode (options.deterministic = 0): the
// inner products are accumulated with atomic additions into the scalar
// slots, and the scalar updates are folded into the kernels that use them,
// so an iteration needs four launches besides the preconditioner instead of
// seven.  Slots (parity p = iteration & 1): RZ[p] = 8 + p, PQ[p] = 10 + p,
// RR[p] = 12 + p; flag 6 as in k_finish.
// ---------------------------------------------------------------------------
constexpr int kRZ = 8, kPQ = 10, kRR = 12;

__device__ __forceinline__ void block_atomic_add(double v, double* dst, double* red) {
  v = block_sum(v, red);
  if (threadIdx.x == 0) atomicAdd(dst, v);
}

// q = A p, PQ[par] += p.q; clears the other parity's slots for their next use
__global__ void __launch_bounds__(kT)
k_spmv_atomic(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ scol,
              const double* __restrict__ sval, const double* __restrict__ p, double* __restrict__ q,
              double* __restrict__ scal, int par) {
  __shared__ double red[kT / 32];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    scal[kRZ + (par ^ 1)] = 0.0;
    scal[kPQ + (par ^ 1)] = 0.0;
    scal[kRR + (par ^ 1)] = 0.0;
  }
  const int l = threadIdx.x & 31;
  const int64_t nsl = (n + 31) / 32;
  double dsum = 0.0;
  for (int64_t sl = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; sl < nsl;
       sl += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const double v = sell_row(off, scol, sval, p, sl, l);
    const int64_t r = sl * 32 + l;
    if (r < n) {
      q[r] = v;
      dsum += v * p[r];
    }
  }
  block_atomic_add(dsum, &scal[kPQ + par], red);
}

// alpha = RZ[par] / PQ[par]; x += alpha p, r -= alpha q, RR[par] += r.r
__global__ void __launch_bounds__(kT)
k_update_xr_atomic(int64_t n, double* __restrict__ scal, const double* __restrict__ p,
                   const double* __restrict__ q, double* __restrict__ x, double* __restrict__ r,
                   double* __restrict__ hist_a, int it, int par) {
  __shared__ double red[kT / 32];
  const double pq = scal[kPQ + par];
  const bool bad = !(pq > 0.0);
  const double alpha = bad ? 0.0 : scal[kRZ + par] / pq;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    hist_a[it] = alpha;
    if (bad) scal[6] = 1.0;
  }
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    s += ri * ri;
  }
  block_atomic_add(s, &scal[kRR + par], red);
}

// scal[slot] += a.b
__global__ void __launch_bounds__(kT)
k_dot_atomic(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ scal,
             int slot) {
  __shared__ double red[kT / 32];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s += a[i] * b[i];
  block_atomic_add(s, &scal[slot], red);
}

// beta = RZ[par ^ 1] / RZ[par] (new over old); p = z + beta p
__global__ void k_update_p_atomic(int64_t n, double* __restrict__ scal, const double* __restrict__ z,
                                  double* __restrict__ p, double* __restrict__ hist_b, int it, int par) {
  const double rz_new = scal[kRZ + (par ^ 1)], rz_old = scal[kRZ + par];
  const double beta = rz_old > 0.0 ? rz_new / rz_old : 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    hist_b[it] = beta;
    if (!(rz_new > 0.0)) scal[6] = 1.0;
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}

}  // namespace

// Condition estimate lambda_max / lambda_min of the Lanczos tridiagonal
// matrix of the CG coefficients (alpha a[0..m), beta b[0..m-1)): both
// extreme eigenvalues by bisection on the Sturm sequence count, in caller
// storage d, e of m entries.
double condition_estimate_fixed(const double* a, const double* b, int m, double* d, double* e) {
  if (m <= 0) return 1.0;
  for (int i = 0; i < m; ++i) {
    d[i] = 1.0 / a[i] + (i > 0 ? b[i - 1] / a[i - 1] : 0.0);
    if (i < m - 1) e[i] = std::sqrt(std::max(b[i], 0.0)) / a[i];
  }
  auto count = [&](double x) {
    int c = 0;
    double q = d[0] - x;
    if (q < 0) ++c;
    for (int i = 1; i < m; ++i) {
      q = d[i] - x - e[i - 1] * e[i - 1] / (q == 0.0 ? 1e-300 : q);
      if (q < 0) ++c;
    }
    return c;
  };
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(e[i]) : 0.0);
    lo = std::min(lo, d[i] - r);
    hi = std::max(hi, d[i] + r);
  }
  double ext[2];
  for (int which = 0; which < 2; ++which) {
    const int k = which == 0 ? 0 : m - 1;
    double l = lo, u = hi;
    for (int it = 0; it < 200 && u - l > 1e-15 * std::max(std::fabs(l), std::fabs(u)); ++it) {
      const double mid = 0.5 * (l + u);
      if (count(mid) > k) u = mid; else l = mid;
    }
    ext[which] = 0.5 * (l + u);
  }
  return ext[1] / ext[0];
}

// Autotuner of the preconditioner's local solve (the one-right-hand-side
// band solve with the vector resident in shared memory): each pipeline
// depth (2, 3, 4 stages; deeper stages take more shared memory and so fewer
// blocks per SM) is timed on this batch, on a scratch copy of the subdomain
// vectors, and the fastest is kept for the process, keyed by (precision,
// largest band width, largest order, batch size).  The depths are timed in
// turn, four rounds after a warm-up launch of each, one launch per CUDA-event
// pair, and each depth keeps its fastest launch: a single short window per
// depth is at the mercy of whatever else the GPU does at that moment.  Runs
// once per key at the end of a setup.
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, int> g_tune;
}  // namespace

geneo_status_t tune_local_solve(geneo_handle_s* h) {
  const auto key = std::make_tuple(h->fp32 ? 1 : 0, h->maxwA, h->maxnD, h->N);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      h->local_stages = it->second;
      return GENEO_OK;
    }
  }
  cudaStream_t s = h->mem.stream;
  DevMem tmp;
  tmp.stream = s;
  double* scratch = nullptr;
  GENEO_TRY(tmp.get(&scratch, (size_t)std::max<int64_t>(h->sumN, 1)));
  GENEO_CUDA(cudaMemsetAsync(scratch, 0, sizeof(double) * h->sumN, s));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  GENEO_CUDA(cudaEventCreate(&e0));
  GENEO_CUDA(cudaEventCreate(&e1));
  auto run = [&](int stages) -> geneo_status_t {
    return solve_set_run(h->setA, h->solve_streams, scratch, h->uoff, 1, nullptr, nullptr, h->dstat, s, 3, stages);
  };
  constexpr int kDepths = 3, kRounds = 4;
  float best_ms[kDepths];
  bool ok[kDepths];
  for (int i = 0; i < kDepths; ++i) {
    best_ms[i] = 1e30f;
    ok[i] = run(2 + i) == GENEO_OK;  // warm-up (and the shared-memory attribute)
  }
  for (int r = 0; r < kRounds; ++r)
    for (int i = 0; i < kDepths; ++i) {
      if (!ok[i]) continue;
      GENEO_CUDA(cudaEventRecord(e0, s));
      ok[i] = run(2 + i) == GENEO_OK;
      GENEO_CUDA(cudaEventRecord(e1, s));
      GENEO_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      GENEO_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ok[i]) best_ms[i] = std::min(best_ms[i], ms);
    }
  int best = 0;
  float bms = 1e30f;
  for (int i = 0; i < kDepths; ++i)
    if (ok[i] && best_ms[i] < bms) {
      bms = best_ms[i];
      best = 2 + i;
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  GENEO_CUDA(cudaStreamSynchronize(s));
  tmp.free_all();
  h->local_stages = best;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[key] = best;
  return GENEO_OK;
}

geneo_status_t alloc_solver(geneo_handle_s* h) {
  DevMem& M = h->mem;
  const int64_t n = h->n;
  GENEO_TRY(M.get(&h->u, (size_t)h->sumN));
  GENEO_TRY(M.get(&h->cH, (size_t)std::max(h->dimH, 1)));
  GENEO_TRY(M.get(&h->r, (size_t)n));
  GENEO_TRY(M.get(&h->zv, (size_t)n));
  GENEO_TRY(M.get(&h->p, (size_t)n));
  GENEO_TRY(M.get(&h->q, (size_t)n));
  GENEO_TRY(M.get(&h->red, (size_t)kRedBlocks));
  GENEO_TRY(M.get(&h->scal, 16));
  GENEO_TRY(M.get(&h->uoff, (size_t)h->N));
  std::vector<int64_t> off(h->N);
  for (int j = 0; j < h->N; ++j) off[j] = h->hsub[j].offN;
  GENEO_CUDA(cudaMemcpy(h->uoff, off.data(), sizeof(int64_t) * h->N, cudaMemcpyHostToDevice));
  GENEO_TRY(M.get(&h->xoffH, 1));
  GENEO_CUDA(cudaMemset(h->xoffH, 0, sizeof(int64_t)));
  {
    // SELL-32 copy of A for the PCG products
    const int64_t nsl = (n + 31) / 32;
    DevMem tmp;
    tmp.stream = h->mem.stream;
    int64_t* len = nullptr;
    GENEO_TRY(tmp.get(&len, (size_t)nsl + 1));
    GENEO_TRY(M.get(&h->sell_off, (size_t)nsl + 1));
    const int g = (int)std::min<int64_t>((nsl * 32 + kT - 1) / kT, 152 * 16);
    k_sell_len<<<g, kT, 0, h->mem.stream>>>(n, h->rowptr, len); note_launch();
    GENEO_CUDA(cudaMemsetAsync(len + nsl, 0, sizeof(int64_t), h->mem.stream));
    int64_t tot = 0;
    GENEO_TRY(exclusive_scan_i64(len, h->sell_off, nsl + 1, &tot, tmp, h->mem.stream));
    GENEO_TRY(M.get(&h->sell_col, (size_t)std::max<int64_t>(tot, 1)));
    GENEO_TRY(M.get(&h->sell_val, (size_t)std::max<int64_t>(tot, 1)));
    k_sell_fill<<<g, kT, 0, h->mem.stream>>>(n, h->rowptr, h->col, h->val, h->sell_off, h->sell_col,
                                             h->sell_val); note_launch();
    GENEO_CUDA(cudaGetLastError());
    GENEO_CUDA(cudaStreamSynchronize(h->mem.stream));
    tmp.free_all();
    h->sell_nnz = tot;
    // the product's grid: the blocks that are resident at once (no tail wave)
    int dev = 0, sms = 0, occ = 0;
    GENEO_CUDA(cudaGetDevice(&dev));
    GENEO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    GENEO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_spmv_sell_dot, kT, 0));
    h->spmv_blocks = std::max(1, std::min(kRedBlocks, sms * std::max(occ, 1)));
  }
  if (!h->hpin) GENEO_CUDA(cudaMallocHost(&h->hpin, 16 * sizeof(double)));
  // the A_j factors in size classes for the local solves
  GENEO_TRY(make_solve_set(h->bandA, !h->fp32, h->dbandA, h->N, h->fp32 ? h->bandA64 : nullptr,
                           h->fp32 ? h->dbandA64 : nullptr, h->fp32 ? h->nA64 : 0, M, M.stream, &h->setA));
  // host arrays of the allocation-free solve (Lanczos coefficients and the
  // bisection work), sized once here so that solve never touches the heap
  h->pcg_host.assign(4 * (size_t)(kNoAllocMaxIt + 1), 0.0);
  h->red_blocks = kRedBlocks;
  // algorithmic work of one apply
  // bytes per factor entry: 4 with FP32 factors, 8 for those factored in FP64
  auto esz_of = [&](int j) { return h->fp32 && !(j < (int)h->a64.size() && h->a64[j]) ? 4.0 : 8.0; };
  double fl = 0.0, by = 0.0, sumD = 0.0;
  for (int j = 0; j < h->N; ++j) {
    const SubDesc& d = h->hsub[j];
    fl += band_solve_flops(d.nD, d.wA) + 4.0 * (double)d.nD * d.m;
    by += 2.0 * esz_of(j) * band_entries(d.nD, d.wA) + 2.0 * 8.0 * (double)d.nD * d.m;
    sumD += d.nD;
  }
  fl += band_solve_flops(h->dimH, h->wH);
  by += 2.0 * 8.0 * band_entries(h->dimH, h->wH);
  by += 8.0 * (2.0 * (double)n + 3.0 * sumD);  // r, z, gathered r, u written and read
  h->apply_flops = fl;
  h->apply_bytes = by;
  double lfl = 0.0, lby = 0.0;
  for (int j = 0; j < h->N; ++j) {
    const SubDesc& d = h->hsub[j];
    lfl += band_solve_flops(d.nD, d.wA);
    lby += 2.0 * esz_of(j) * band_entries(d.nD, d.wA) + 8.0 * 2.0 * d.nD;  // factor twice; u in and out once
  }
  h->local_solve_flops = lfl;
  h->local_solve_bytes = lby;
  h->spmv_flops = 2.0 * (double)h->nnz;
  // algorithmic bytes of q = A p with p.q: A once (values and columns), p
  // read once, q written once, the row offsets
  h->spmv_bytes = 12.0 * (double)h->nnz + 8.0 * (double)n + 24.0 * (double)n;
  return GENEO_OK;
}

geneo_status_t apply_prec(geneo_handle_s* h, const double* r, double* z, cudaStream_t s) {
  const int N = h->N;
  k_restrict<<<N, kT, 0, s>>>(h->dsub, h->Dlist, r, h->Z, h->u, h->cH); note_launch();
  GENEO_CUDA(cudaGetLastError());
  // the coarse solve: a dense product with A_H^{-1} on this stream (short),
  // or the band solve on one SM beside the batched local solves
  if (h->dimH > 0 && h->Hinv) {
    const double dm = h->dimH;
    const int pc = h->prof.begin(GENEO_PROF_COARSE_SOLVE, 2.0 * dm * dm, 8.0 * dm * dm + 16.0 * dm, s);
    const int g = std::min(ceil_div(h->dimH, kT / 32), 152 * 8);
    k_coarse_gemv<<<g, kT, 0, s>>>(h->Hinv, h->dimH, h->cH, h->yH); note_launch();
    GENEO_CUDA(cudaGetLastError());
    h->prof.end(pc, s);
  } else if (h->dimH > 0) {
    GENEO_CUDA(cudaEventRecord(h->ev_fork, s));
    GENEO_CUDA(cudaStreamWaitEvent(h->aux, h->ev_fork, 0));
    {
      const int pc = h->prof.begin(GENEO_PROF_COARSE_SOLVE, band_solve_flops(h->dimH, h->wH),
                                   2.0 * 8.0 * band_entries(h->dimH, h->wH) + 16.0 * h->dimH, h->aux);
      GENEO_TRY(band_solve<double>(h->bandH, h->dbandH, 1, h->wH, h->cH, h->xoffH, 1, nullptr, nullptr,
                                   h->dstat, h->aux, h->dimH));
      h->prof.end(pc, h->aux);
    }
    GENEO_CUDA(cudaEventRecord(h->ev_join, h->aux));
  }
  const int pl = h->prof.begin(GENEO_PROF_LOCAL_SOLVE, h->local_solve_flops, h->local_solve_bytes, s);
  // size classes of the A_j (FP32 and FP64 factors) on the solve lanes
  GENEO_TRY(solve_set_run(h->setA, h->solve_streams, h->u, h->uoff, 1, nullptr, nullptr, h->dstat, s, 3,
                          h->local_stages));
  h->prof.end(pl, s);
  if (h->dimH > 0 && !h->Hinv) GENEO_CUDA(cudaStreamWaitEvent(s, h->ev_join, 0));
  const int grid = (int)std::min<int64_t>((h->n + kT - 1) / kT, 152 * 8);
  k_prolong<<<grid, kT, 0, s>>>(h->n, h->dir, r, h->invD_ptr, h->invD_sub, h->invD_loc, h->dsub,
                                h->u, h->Z, h->Hinv ? h->yH : h->cH, z); note_launch();
  GENEO_CUDA(cudaGetLastError());
  return GENEO_OK;
}

// Buffers of one PCG solve: device reduction partials, scalars and the
// alpha/beta history (cap entries each), and host arrays of cap entries for
// the condition estimate.
struct PcgBufs {
  double *red, *scal, *da, *db;
  int cap;
  double *ha, *hb, *hd, *he;
};

// Preconditioned CG (Section 5), x0 = 0.  The recursive residual is tested
// first; when it reaches tol the true residual b - A x is formed, and while
// that is still above tol it replaces the recursive one and CG restarts from
// x (p = M^{-1} r), at most kMaxReplace times and only while each
// replacement at least halves the true residual (below that the rounding of
// x in FP64 bounds what any iteration can reach).  The Lanczos estimate of
// kappa(M^{-1} A) uses the coefficients before the first replacement.
constexpr int kMaxReplace = 5;

geneo_status_t pcg_core(geneo_handle_s* h, const double* b, double* x, double tol, int maxit,
                        geneo_solve_info_t* info, cudaStream_t s, const PcgBufs& B) {
  const int64_t n = h->n;
  const int nb = kRedBlocks;
  double* scal = B.scal;
  double* red = B.red;
  GENEO_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
  GENEO_CUDA(cudaMemcpyAsync(h->r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  GENEO_CUDA(cudaMemsetAsync(scal, 0, sizeof(double) * 16, s));
  k_dot<<<nb, kT, 0, s>>>(n, b, b, red); note_launch();
  k_finish<<<1, kT, 0, s>>>(red, nb, scal, 4, B.da, B.db, 0); note_launch();
  GENEO_CUDA(cudaGetLastError());
  GENEO_CUDA(cudaMemcpyAsync(h->hpin, scal, sizeof(double) * 8, cudaMemcpyDeviceToHost, s));
  GENEO_CUDA(cudaStreamSynchronize(s));
  const double bnorm = std::sqrt(h->hpin[5]);
  int hist_len = 0;
  auto push_hist = [&](double v) {
    if (info && info->resid_hist && hist_len < info->resid_hist_cap) info->resid_hist[hist_len] = v;
    ++hist_len;
  };
  if (info) {
    info->iterations = 0;
    info->converged = 0;
    info->rel_residual = NAN;
    info->true_residual = NAN;
    info->kappa_estimate = NAN;
    info->replacements = 0;
    info->resid_hist_len = 0;
  }
  if (!std::isfinite(bnorm)) return GENEO_ERR_NONFINITE;
  if (bnorm == 0.0) {
    if (info) {
      info->converged = 1;
      info->rel_residual = 0.0;
      info->true_residual = 0.0;
      info->kappa_estimate = 1.0;
    }
    return GENEO_OK;
  }
  push_hist(1.0);
  const bool det = h->opt.deterministic != 0;
  int it = 0;
  auto restart = [&]() -> geneo_status_t {  // p = z = M^{-1} r, rz = r.z
    GENEO_TRY(apply_prec(h, h->r, h->zv, s));
    GENEO_CUDA(cudaMemcpyAsync(h->p, h->zv, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    if (det) {
      k_dot<<<nb, kT, 0, s>>>(n, h->r, h->zv, red); note_launch();
      k_finish<<<1, kT, 0, s>>>(red, nb, scal, 0, B.da, B.db, 0); note_launch();
    } else {
      GENEO_CUDA(cudaMemsetAsync(scal + kRZ, 0, sizeof(double) * 6, s));
      k_dot_atomic<<<nb, kT, 0, s>>>(n, h->r, h->zv, scal, kRZ + (it & 1)); note_launch();
    }
    GENEO_CUDA(cudaGetLastError());
    return GENEO_OK;
  };
  // true residual into zv (free between the update and the next apply)
  auto true_residual = [&](double* out) -> geneo_status_t {
    k_true_resid_sell<<<nb, kT, 0, s>>>(n, h->sell_off, h->sell_col, h->sell_val, x, b, h->zv, red);
    note_launch();
    k_finish<<<1, kT, 0, s>>>(red, nb, scal, 5, B.da, B.db, 0); note_launch();
    GENEO_CUDA(cudaGetLastError());
    GENEO_CUDA(cudaMemcpyAsync(h->hpin, scal, sizeof(double) * 8, cudaMemcpyDeviceToHost, s));
    GENEO_CUDA(cudaStreamSynchronize(s));
    *out = std::sqrt(h->hpin[7]) / bnorm;
    return GENEO_OK;
  };
  GENEO_TRY(restart());
  int replaced = 0, n_lanczos = -1;
  double rel = 1.0, rel_true = NAN, last_true = INFINITY;
  bool breakdown = false, converged = false, have_true = false, nonfinite = false;
  while (it < maxit && it < B.cap - 1) {
    const int par = it & 1;
    {
      const int pv = h->prof.begin(GENEO_PROF_SPMV, h->spmv_flops, h->spmv_bytes, s);
      if (det) {
        k_spmv_sell_dot<<<h->spmv_blocks, kT, 0, s>>>(n, h->sell_off, h->sell_col, h->sell_val, h->p, h->q,
                                                      red);
        note_launch();
      } else {
        k_spmv_atomic<<<nb, kT, 0, s>>>(n, h->sell_off, h->sell_col, h->sell_val, h->p, h->q, scal, par);
        note_launch();
      }
      h->prof.end(pv, s);
    }
    if (det) {
      k_finish<<<1, kT, 0, s>>>(red, h->spmv_blocks, scal, 1, B.da, B.db, it); note_launch();
      k_update_xr<<<nb, kT, 0, s>>>(n, scal, h->p, h->q, x, h->r, red); note_launch();
      k_finish<<<1, kT, 0, s>>>(red, nb, scal, 2, B.da, B.db, it); note_launch();
    } else {
      k_update_xr_atomic<<<nb, kT, 0, s>>>(n, scal, h->p, h->q, x, h->r, B.da, it, par); note_launch();
    }
    GENEO_CUDA(cudaGetLastError());
    GENEO_CUDA(cudaMemcpyAsync(h->hpin, scal, sizeof(double) * 16, cudaMemcpyDeviceToHost, s));
    GENEO_CUDA(cudaStreamSynchronize(s));
    if (!det) h->hpin[3] = h->hpin[kRR + par];
    ++it;
    have_true = false;
    if (h->hpin[6] != 0.0) {
      breakdown = true;
      break;
    }
    rel = std::sqrt(h->hpin[3]) / bnorm;
    push_hist(rel);
    if (!std::isfinite(rel)) {
      nonfinite = true;
      break;
    }
    if (rel <= tol) {
      GENEO_TRY(true_residual(&rel_true));
      have_true = true;
      if (rel_true <= tol) {
        converged = true;
        break;
      }
      if (replaced >= kMaxReplace || !(rel_true <= 0.5 * last_true)) break;
      last_true = rel_true;
      ++replaced;
      if (n_lanczos < 0) n_lanczos = it;
      GENEO_CUDA(cudaMemcpyAsync(h->r, h->zv, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      GENEO_TRY(restart());
      continue;
    }
    GENEO_TRY(apply_prec(h, h->r, h->zv, s));
    if (det) {
      k_dot<<<nb, kT, 0, s>>>(n, h->r, h->zv, red); note_launch();
      k_finish<<<1, kT, 0, s>>>(red, nb, scal, 3, B.da, B.db, it - 1); note_launch();
      k_update_p<<<nb, kT, 0, s>>>(n, scal, h->zv, h->p); note_launch();
    } else {
      k_dot_atomic<<<nb, kT, 0, s>>>(n, h->r, h->zv, scal, kRZ + (par ^ 1)); note_launch();
      k_update_p_atomic<<<nb, kT, 0, s>>>(n, scal, h->zv, h->p, B.db, it - 1, par); note_launch();
    }
    GENEO_CUDA(cudaGetLastError());
  }
  if (!have_true && !breakdown && !nonfinite) GENEO_TRY(true_residual(&rel_true));
  int nalpha = n_lanczos >= 0 ? n_lanczos : (breakdown ? std::max(it - 1, 0) : it);
  nalpha = std::min(nalpha, B.cap);
  if (nalpha > 0) {
    GENEO_CUDA(cudaMemcpyAsync(B.ha, B.da, sizeof(double) * nalpha, cudaMemcpyDeviceToHost, s));
    GENEO_CUDA(cudaMemcpyAsync(B.hb, B.db, sizeof(double) * nalpha, cudaMemcpyDeviceToHost, s));
  }
  GENEO_CUDA(cudaStreamSynchronize(s));
  if (info) {
    info->iterations = it;
    info->converged = converged;
    info->rel_residual = rel;
    info->true_residual = rel_true;
    info->replacements = replaced;
    info->kappa_estimate = condition_estimate_fixed(B.ha, B.hb, nalpha, B.hd, B.he);
    info->resid_hist_len = std::min(hist_len, info->resid_hist ? info->resid_hist_cap : 0);
  }
  GENEO_TRY(check_status(h, s));
  if (nonfinite || !std::isfinite(rel_true) && !breakdown) return GENEO_ERR_NONFINITE;
  if (breakdown) return GENEO_ERR_BREAKDOWN;
  if (!converged) return GENEO_ERR_PCG_NOCONV;
  return GENEO_OK;
}

geneo_status_t pcg(geneo_handle_s* h, const double* b, double* x, double tol, int maxit,
                   geneo_solve_info_t* info, cudaStream_t s) {
  const int cap = std::max(maxit, 1) + 1;
  if (h->hist_cap < cap) {
    h->mem.stream = s;  // the handle's last stream (see geneo_destroy)
    if (h->hist) h->mem.release(h->hist);
    h->hist = nullptr;
    GENEO_TRY(h->mem.get(&h->hist, 2 * (size_t)cap));
    h->hist_cap = cap;
  }
  std::vector<double> host(4 * (size_t)cap);
  const PcgBufs B{h->red, h->scal, h->hist, h->hist + h->hist_cap, cap,
                  host.data(), host.data() + cap, host.data() + 2 * cap, host.data() + 3 * cap};
  geneo_status_t st = pcg_core(h, b, x, tol, maxit, info, s, B);
  h->prof.collect();
  return st;
}

// ---------------------------------------------------------------------------
// PCG that allocates nothing (geneo_pcg_solve_noalloc).
//
// The reduction partials, the PCG scalars and the alpha/beta history live in
// one file-scope device array of fixed size instead of handle or call
// allocations.  Every device that loads the library holds its own copy until
// the process exits.  Host code never uses the array's name as an address:
// the device address is obtained once per device with cudaGetSymbolAddress
// (with that device current) and cached.  All calls share the array, so calls
// whose work overlaps on the GPU race with each other.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNoAllocDoubles = kRedBlocks + kNoAllocScalars + 2 * (kNoAllocMaxIt + 1);
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_pcg_scratch[kNoAllocDoubles];  // 73,856 bytes

std::mutex g_scratch_mu;
double* g_scratch_addr[kMaxDevices] = {};

geneo_status_t pcg_scratch(double** out) {
  int dev = 0;
  GENEO_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return GENEO_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    GENEO_CUDA(cudaGetSymbolAddress(&p, g_pcg_scratch));
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return GENEO_OK;
}


}  // namespace

geneo_status_t pcg_noalloc(geneo_handle_s* h, const double* b, double* x, double tol, int maxit,
                           geneo_solve_info_t* info, cudaStream_t s) {
  if (maxit > kNoAllocMaxIt || h->prof.on) return GENEO_ERR_ARG;
  int dev = -1;
  GENEO_CUDA(cudaGetDevice(&dev));
  if (dev != h->device) return GENEO_ERR_ARG;
  if ((int)h->pcg_host.size() < 4 * (kNoAllocMaxIt + 1)) return GENEO_ERR_ARG;
  h->mem.stream = s;  // the handle's last stream (see geneo_destroy); no allocation
  double* scr = nullptr;
  GENEO_TRY(pcg_scratch(&scr));
  constexpr int cap = kNoAllocMaxIt + 1;
  double* hh = h->pcg_host.data();
  const PcgBufs B{scr, scr + kRedBlocks, scr + kRedBlocks + kNoAllocScalars,
                  scr + kRedBlocks + kNoAllocScalars + cap, cap, hh, hh + cap, hh + 2 * cap, hh + 3 * cap};
  return pcg_core(h, b, x, tol, maxit, info, s, B);
}

}  // namespace geneo

extern "C" geneo_status_t geneo_pcg_solve_noalloc(geneo_handle_t h, const double* b_dev, double* x_dev,
                                                  double tol, int32_t maxit,
                                                  geneo_solve_info_t* info, void* stream) {
  if (!h || !b_dev || !x_dev || !(tol > 0.0) || maxit < 0 || maxit > geneo::kNoAllocMaxIt)
    return GENEO_ERR_ARG;
  return geneo::pcg_noalloc(h, b_dev, x_dev, tol, maxit, info, (cudaStream_t)stream);
}
