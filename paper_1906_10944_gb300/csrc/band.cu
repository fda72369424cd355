// Batched banded Cholesky factorisation and triangular solves.
//
// The local Dirichlet matrices A_j = R_j A R_j^T (Section 3), the shifted
// Neumann matrices K_j = Atilde_j - sigma B_j of the spectral transformation
// (Section 4.4) and the coarse matrix A_H (Section 4.5) are all banded in the
// natural (lexicographic) dof order of a box subdomain, so one banded kernel
// family serves all three.  One thread block owns one matrix; the batch is
// the grid.  Storage: lower band, column-major, entry (r, c) with
// 0 <= r - c <= w at L[c*(w+1) + (r - c)].
//
// Factorisation (right-looking, block width NB): per step the NB x NB
// diagonal block is factored by one warp, the panel rows below are solved
// against it (one thread per row, registers), and the trailing w x w
// triangle receives the rank-NB update in 4x4 register tiles.  Pivots that
// are not positive are reported (GENEO_ERR_NOT_SPD) and replaced by 1 so the
// kernel always finishes.
#include "common.cuh"

namespace geneo {

namespace {

constexpr int kThreads = 256;
constexpr int kSolveKmax = 64;   // right-hand sides handled per launch

template <typename T>
__device__ __forceinline__ bool finite_pos(T v) { return v > T(0) && isfinite(v); }

template <typename T, int NB, bool SMEMP>
__global__ void __launch_bounds__(kThreads)
k_band_potrf(T* __restrict__ base, const BandDesc* __restrict__ descs, int phmax,
             DevStatus* st) {
  const BandDesc d = descs[blockIdx.x];
  const int n = d.n, w = d.w;
  const int64_t ld = (int64_t)w + 1;
  T* L = base + d.off;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Dk = reinterpret_cast<T*>(smem_raw);   // [NB][NB+1]
  T* Ps = Dk + NB * (NB + 1);               // [NB][phmax] (SMEMP only)
  const int tid = threadIdx.x, nt = blockDim.x;
  constexpr int DS = NB + 1;

  for (int kb = 0; kb < n; kb += NB) {
    const int b = min(NB, n - kb);
    const int h = min(w, n - kb - b);
    // 1. diagonal block
    for (int idx = tid; idx < NB * NB; idx += nt) {
      const int r = idx % NB, c = idx / NB;
      T v = T(0);
      if (r < b && c < b && r >= c && r - c <= w) v = L[(int64_t)(kb + c) * ld + (r - c)];
      Dk[r * DS + c] = v;
    }
    __syncthreads();
    // 2. unblocked Cholesky of the diagonal block by warp 0
    if (tid < 32) {
      const int lane = tid;
      for (int t = 0; t < b; ++t) {
        if (lane == t) {
          T dv = Dk[t * DS + t];
          if (!finite_pos(dv)) {
            record_error(st, GENEO_ERR_NOT_SPD, d.id, (int64_t)kb + t);
            dv = T(1);
          }
          Dk[t * DS + t] = sqrt(dv);
        }
        __syncwarp();
        const T piv = Dk[t * DS + t];
        if (lane > t && lane < b) Dk[lane * DS + t] /= piv;
        __syncwarp();
        if (lane > t && lane < b) {
          const T lrt = Dk[lane * DS + t];
          for (int u = t + 1; u <= lane; ++u) Dk[lane * DS + u] -= lrt * Dk[u * DS + t];
        }
        __syncwarp();
      }
    }
    __syncthreads();
    // 3. store the factored diagonal block
    for (int idx = tid; idx < NB * NB; idx += nt) {
      const int r = idx % NB, c = idx / NB;
      if (r < b && c < b && r >= c && r - c <= w) L[(int64_t)(kb + c) * ld + (r - c)] = Dk[r * DS + c];
    }
    // 4. panel: rows kb+b+i solve x L_kk^T = a
    for (int i = tid; i < h; i += nt) {
      const int rr = kb + b + i;
      T x[NB];
#pragma unroll
      for (int t = 0; t < NB; ++t) {
        T v = T(0);
        if (t < b) {
          const int dd = rr - (kb + t);
          if (dd <= w) v = L[(int64_t)(kb + t) * ld + dd];
        }
        x[t] = v;
      }
#pragma unroll
      for (int t = 0; t < NB; ++t) {
        if (t < b) {
          T v = x[t];
#pragma unroll
          for (int u = 0; u < t; ++u) v -= x[u] * Dk[t * DS + u];
          x[t] = v / Dk[t * DS + t];
        }
      }
#pragma unroll
      for (int t = 0; t < NB; ++t) {
        if (t < b) {
          const int dd = rr - (kb + t);
          if (dd <= w) L[(int64_t)(kb + t) * ld + dd] = x[t];
          if (SMEMP) Ps[t * phmax + i] = (dd <= w) ? x[t] : T(0);
        }
      }
    }
    __syncthreads();
    // 5. trailing update of the h x h window, 4x4 register tiles
    const int T4 = (h + 3) >> 2;
    for (int idx = tid; idx < T4 * T4; idx += nt) {
      const int ti = idx % T4, tj = idx / T4;
      if (tj > ti) continue;
      T acc[4][4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int p = 0; p < 4; ++p) acc[q][p] = T(0);
      for (int t = 0; t < b; ++t) {
        T pr[4], pc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int i = 4 * ti + q, j = 4 * tj + q;
          if (SMEMP) {
            pr[q] = (i < h) ? Ps[t * phmax + i] : T(0);
            pc[q] = (j < h) ? Ps[t * phmax + j] : T(0);
          } else {
            const int di = b + i - t, dj = b + j - t;
            pr[q] = (i < h && di <= w) ? L[(int64_t)(kb + t) * ld + di] : T(0);
            pc[q] = (j < h && dj <= w) ? L[(int64_t)(kb + t) * ld + dj] : T(0);
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int p = 0; p < 4; ++p) acc[q][p] += pr[q] * pc[p];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const int j = 4 * tj + p;
        if (j >= h) continue;
        const int64_t colbase = (int64_t)(kb + b + j) * ld;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int i = 4 * ti + q;
          if (i < h && i >= j) L[colbase + (i - j)] -= acc[q][p];
        }
      }
    }
    __syncthreads();
  }
}

// Forward then backward substitution with L and L^T, in place on X.
template <typename T, int NB>
__global__ void __launch_bounds__(kThreads)
k_band_solve(const T* __restrict__ base, const BandDesc* __restrict__ descs,
             double* __restrict__ xbase, const int64_t* __restrict__ xoff, int col0, int kcap,
             const int32_t* __restrict__ nrhs_dev, const int32_t* __restrict__ skip) {
  const int mi = blockIdx.x;
  if (skip && skip[mi]) return;
  int k = kcap;
  if (nrhs_dev) k = min(k, nrhs_dev[mi] - col0);
  if (k <= 0) return;
  const BandDesc d = descs[mi];
  const int n = d.n, w = d.w;
  if (n <= 0) return;
  const int64_t ld = (int64_t)w + 1;
  const T* L = base + d.off;
  double* X = xbase + xoff[mi] + (int64_t)col0 * n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int DS = NB + 1;
  T* Dk = reinterpret_cast<T*>(smem_raw);   // [NB][NB+1]
  T* Yb = Dk + NB * DS;                     // [NB][k]
  T* Red = Yb + NB * kSolveKmax;            // partial sums
  const int tid = threadIdx.x, nt = blockDim.x;

  auto load_diag = [&](int kb, int b) {
    for (int idx = tid; idx < NB * NB; idx += nt) {
      const int r = idx % NB, c = idx / NB;
      T v = T(0);
      if (r < b && c < b && r >= c && r - c <= w) v = L[(int64_t)(kb + c) * ld + (r - c)];
      Dk[r * DS + c] = v;
    }
  };

  // ---- forward: L y = x (right-looking, panel columns are contiguous)
  for (int kb = 0; kb < n; kb += NB) {
    const int b = min(NB, n - kb);
    const int h = min(w, n - kb - b);
    load_diag(kb, b);
    for (int idx = tid; idx < b * k; idx += nt) {
      const int t = idx % b, c = idx / b;
      Yb[t * k + c] = (T)X[(int64_t)c * n + kb + t];
    }
    __syncthreads();
    for (int c = tid; c < k; c += nt) {
      for (int t = 0; t < b; ++t) {
        T v = Yb[t * k + c];
        for (int u = 0; u < t; ++u) v -= Dk[t * DS + u] * Yb[u * k + c];
        Yb[t * k + c] = v / Dk[t * DS + t];
      }
    }
    __syncthreads();
    for (int idx = tid; idx < b * k; idx += nt) {
      const int t = idx % b, c = idx / b;
      X[(int64_t)c * n + kb + t] = (double)Yb[t * k + c];
    }
    constexpr int CB = 4;
    const int ncg = (k + CB - 1) / CB;
    for (int idx = tid; idx < h * ncg; idx += nt) {
      const int i = idx % h, cg = idx / h;
      const int r = kb + b + i;
      T acc[CB];
#pragma unroll
      for (int q = 0; q < CB; ++q) acc[q] = T(0);
      const int t0 = max(0, b + i - w);
      for (int t = t0; t < b; ++t) {
        const T l = L[(int64_t)(kb + t) * ld + (b + i - t)];
#pragma unroll
        for (int q = 0; q < CB; ++q) {
          const int c = cg * CB + q;
          if (c < k) acc[q] += l * Yb[t * k + c];
        }
      }
#pragma unroll
      for (int q = 0; q < CB; ++q) {
        const int c = cg * CB + q;
        if (c < k) X[(int64_t)c * n + r] -= (double)acc[q];
      }
    }
    __syncthreads();
  }

  // ---- backward: L^T x = y (left-looking: dot products with panel columns)
  const int nblk = (n + NB - 1) / NB;
  for (int bi = nblk - 1; bi >= 0; --bi) {
    const int kb = bi * NB;
    const int b = min(NB, n - kb);
    const int h = min(w, n - kb - b);
    load_diag(kb, b);
    for (int idx = tid; idx < b * k; idx += nt) {
      const int t = idx % b, c = idx / b;
      Yb[t * k + c] = (T)X[(int64_t)c * n + kb + t];
    }
    __syncthreads();
    if (h > 0) {
      const int nout = b * k;
      const int S = max(1, min(8, nt / nout));
      for (int o = tid; o < S * nout; o += nt) {
        const int seg = o / nout, rem = o % nout;
        const int t = rem % b, c = rem / b;
        const int i0 = (int)((int64_t)seg * h / S), i1 = (int)((int64_t)(seg + 1) * h / S);
        const int iend = min(i1, w - b + t + 1);   // band limit: b + i - t <= w
        T acc = T(0);
        const T* lc = L + (int64_t)(kb + t) * ld + (b - t);
        const double* xc = X + (int64_t)c * n + kb + b;
        for (int i = i0; i < iend; ++i) acc += lc[i] * (T)xc[i];
        Red[o] = acc;
      }
      __syncthreads();
      for (int rem = tid; rem < nout; rem += nt) {
        T s = T(0);
        for (int seg = 0; seg < S; ++seg) s += Red[seg * nout + rem];
        const int t = rem % b, c = rem / b;
        Yb[t * k + c] -= s;
      }
      __syncthreads();
    }
    for (int c = tid; c < k; c += nt) {
      for (int t = b - 1; t >= 0; --t) {
        T v = Yb[t * k + c];
        for (int u = t + 1; u < b; ++u) v -= Dk[u * DS + t] * Yb[u * k + c];
        Yb[t * k + c] = v / Dk[t * DS + t];
      }
    }
    __syncthreads();
    for (int idx = tid; idx < b * k; idx += nt) {
      const int t = idx % b, c = idx / b;
      X[(int64_t)c * n + kb + t] = (double)Yb[t * k + c];
    }
    __syncthreads();
  }
}

constexpr int kNB = 32;
constexpr size_t kSmemCap = 200 * 1024;

}  // namespace

template <typename T>
geneo_status_t band_potrf(T* base, const BandDesc* d_desc, int count, int max_w, DevStatus* st,
                          cudaStream_t s) {
  if (count <= 0) return GENEO_OK;
  const size_t diag = (size_t)kNB * (kNB + 1) * sizeof(T);
  const size_t panel = (size_t)max_w * kNB * sizeof(T);
  if (diag + panel <= kSmemCap) {
    auto kern = k_band_potrf<T, kNB, true>;
    GENEO_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(diag + panel)));
    kern<<<count, kThreads, diag + panel, s>>>(base, d_desc, max_w, st); note_launch();
  } else {
    auto kern = k_band_potrf<T, kNB, false>;
    kern<<<count, kThreads, diag, s>>>(base, d_desc, 0, st); note_launch();
  }
  GENEO_CUDA(cudaGetLastError());
  return GENEO_OK;
}

template <typename T>
geneo_status_t band_solve(const T* base, const BandDesc* d_desc, int count, int max_w,
                          double* xbase, const int64_t* xoff, int nrhs, const int32_t* nrhs_dev,
                          const int32_t* skip_dev, cudaStream_t s) {
  (void)max_w;
  if (count <= 0 || nrhs <= 0) return GENEO_OK;
  const size_t smem = (size_t)kNB * (kNB + 1) * sizeof(T) + (size_t)kNB * kSolveKmax * sizeof(T) +
                      (size_t)std::max(kThreads, kNB * kSolveKmax) * sizeof(T);
  auto kern = k_band_solve<T, kNB>;
  GENEO_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  for (int c0 = 0; c0 < nrhs; c0 += kSolveKmax) {
    const int kc = std::min(kSolveKmax, nrhs - c0);
    kern<<<count, kThreads, smem, s>>>(base, d_desc, xbase, xoff, c0, kc, nrhs_dev, skip_dev); note_launch();
    GENEO_CUDA(cudaGetLastError());
  }
  return GENEO_OK;
}

template geneo_status_t band_potrf<double>(double*, const BandDesc*, int, int, DevStatus*,
                                           cudaStream_t);
template geneo_status_t band_potrf<float>(float*, const BandDesc*, int, int, DevStatus*,
                                          cudaStream_t);
template geneo_status_t band_solve<double>(const double*, const BandDesc*, int, int, double*,
                                           const int64_t*, int, const int32_t*, const int32_t*,
                                           cudaStream_t);
template geneo_status_t band_solve<float>(const float*, const BandDesc*, int, int, double*,
                                          const int64_t*, int, const int32_t*, const int32_t*,
                                          cudaStream_t);

}  // namespace geneo
