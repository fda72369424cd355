// Batched banded Cholesky factorisation and triangular solves.
//
// The local Dirichlet matrices A_j = R_j A R_j^T (Section 3), the shifted
// Neumann matrices K_j = Atilde_j - sigma B_j of the spectral transformation
// (Section 4.4) and the coarse matrix A_H (Section 4.5) are all banded in the
// natural (lexicographic) dof order of a box subdomain, so one banded kernel
// family serves all three.  One thread block owns one matrix; the batch is
// the grid.  Storage: lower band by rows (BandDesc in common.cuh).
//
// Factorisation (right-looking, block width NB): per step the NB x NB
// diagonal block is factored by one warp, the panel rows below are solved
// against it (one thread per row, registers), and the trailing w x w
// triangle receives the rank-NB update in 4x4 register tiles.  Pivots that
// are not positive are reported (GENEO_ERR_NOT_SPD) and replaced by 1 so the
// kernel always finishes.
//
// Solves (L L^T x = b, in place): the factor is streamed block row by block
// row (SNB rows, one contiguous chunk) into shared memory by bulk copies on
// an mbarrier pipeline.  The forward sweep is left-looking (each new row is
// a dot product with the last w solved rows, kept in a shared ring), the
// backward sweep right-looking (the rows above the current block are
// updated in the shared ring); diagonal blocks are solved by warp shuffles.
// The factor is read once per sweep; b and x once each.
#include "common.cuh"
#include "ds.cuh"
#include "ptx.cuh"

namespace geneo {

namespace {

constexpr int kThreads = 256;

template <typename T>
__device__ __forceinline__ bool finite_pos(T v) { return v > T(0) && isfinite(v); }

// four consecutive values from 16-byte aligned shared memory
__device__ __forceinline__ void load4(const float* p, float* o) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void load4(const double* p, double* o) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 c = *reinterpret_cast<const double2*>(p + 2);
  o[0] = a.x; o[1] = a.y; o[2] = c.x; o[3] = c.y;
}

__device__ __forceinline__ void store4(float* p, const float* o) {
  *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
}
__device__ __forceinline__ void store4(double* p, const double* o) {
  *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
  *reinterpret_cast<double2*>(p + 2) = make_double2(o[2], o[3]);
}

__device__ __forceinline__ void load4(const dsv* p, dsv* o) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  const float4 c = *reinterpret_cast<const float4*>(p + 2);
  o[0] = dsv(a.x, a.y); o[1] = dsv(a.z, a.w); o[2] = dsv(c.x, c.y); o[3] = dsv(c.z, c.w);
}
__device__ __forceinline__ void store4(dsv* p, const dsv* o) {
  *reinterpret_cast<float4*>(p) = make_float4(o[0].h, o[0].l, o[1].h, o[1].l);
  *reinterpret_cast<float4*>(p + 2) = make_float4(o[2].h, o[2].l, o[3].h, o[3].l);
}

__device__ __forceinline__ int64_t bidx(int r, int c, int w, int64_t ld) {
  return (int64_t)r * ld + (c - r + w);
}

template <typename T, int NB, bool SMEMP>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 2 : 1)
k_band_potrf(T* __restrict__ base, const BandDesc* __restrict__ descs, int phmax,
             DevStatus* st, int32_t* __restrict__ weak, float weak_tol) {
  const BandDesc d = descs[blockIdx.x];
  const int n = d.n, w = d.w;
  const int64_t ld = d.ld;
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
      const int r = idx / NB, c = idx % NB;
      T v = T(0);
      if (r < b && c < b && r >= c && r - c <= w) v = L[bidx(kb + r, kb + c, w, ld)];
      Dk[r * DS + c] = v;
    }
    __syncthreads();
    // 2. unblocked Cholesky of the diagonal block by warp 0
    if (tid < 32) {
      const int lane = tid;
      for (int t = 0; t < b; ++t) {
        if (lane == t) {
          T dv = Dk[t * DS + t];
          if (weak) {
            if (!(dv > T(weak_tol))) weak[d.id] = 1;
            if (!finite_pos(dv)) dv = T(1);
          } else if (!finite_pos(dv)) {
            record_error(st, isfinite(dv) ? GENEO_ERR_NOT_SPD : GENEO_ERR_NONFINITE, d.id, (int64_t)kb + t);
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
      const int r = idx / NB, c = idx % NB;
      if (r < b && c < b && r >= c && r - c <= w) L[bidx(kb + r, kb + c, w, ld)] = Dk[r * DS + c];
    }
    // 4. panel: rows kb+b+i solve x L_kk^T = a
    for (int i = tid; i < h; i += nt) {
      const int rr = kb + b + i;
      T x[NB];
#pragma unroll
      for (int t = 0; t < NB; ++t) {
        T v = T(0);
        if (t < b && rr - (kb + t) <= w) v = L[bidx(rr, kb + t, w, ld)];
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
          const bool inb = rr - (kb + t) <= w;
          if (inb) L[bidx(rr, kb + t, w, ld)] = x[t];
          if (SMEMP) Ps[t * phmax + i] = inb ? x[t] : T(0);
        }
      }
    }
    if (SMEMP) {
      const int h4 = (h + 3) & ~3;
      for (int idx = tid; idx < b * (h4 - h); idx += nt) {
        const int t = idx / (h4 - h), i = h + idx % (h4 - h);
        Ps[t * phmax + i] = T(0);
      }
    }
    __syncthreads();
    // 5. trailing update of the h x h window, 4x4 register tiles
    //    (consecutive threads take consecutive column tiles of one row tile)
    const int T4 = (h + 3) >> 2;
    for (int idx = tid; idx < T4 * T4; idx += nt) {
      const int ti = idx / T4, tj = idx % T4;
      if (tj > ti) continue;
      T acc[4][4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int p = 0; p < 4; ++p) acc[q][p] = T(0);
      for (int t = 0; t < b; ++t) {
        T pr[4], pc[4];
        if (SMEMP) {
          // the panel rows beyond h are zero in shared memory (phmax >= h
          // rounded up to 4), so whole 4-vectors can be read: pr is the same
          // address for the warp (broadcast), pc one 16-byte vector per thread
          const T* prow = Ps + (size_t)t * phmax;
#pragma unroll
          for (int q = 0; q < 4; ++q) pr[q] = prow[4 * ti + q];
          load4(prow + 4 * tj, pc);
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int i = 4 * ti + q, j = 4 * tj + q;
            pr[q] = (i < h && b + i - t <= w) ? L[bidx(kb + b + i, kb + t, w, ld)] : T(0);
            pc[q] = (j < h && b + j - t <= w) ? L[bidx(kb + b + j, kb + t, w, ld)] : T(0);
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int p = 0; p < 4; ++p) acc[q][p] += pr[q] * pc[p];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = 4 * ti + q;
        if (i >= h) continue;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const int j = 4 * tj + p;
          if (j < h && i >= j) L[bidx(kb + b + i, kb + b + j, w, ld)] -= acc[q][p];
        }
      }
    }
    __syncthreads();
  }
}

// Right-looking factorisation of one large band over many SMs (the coarse
// matrix A_H, whose FP64 work is too much for one SM).  Per panel of NB
// columns: one warp factors the diagonal block (k_band_panel_diag), a grid
// of one-warp blocks solves the panel rows below it, one row per thread
// (k_band_panel_rows), then a grid of 64 x 64 tiles applies the rank-NB
// update to the trailing window (k_band_trail).  Three launches per panel;
// the stream orders them.  GB300 issues FP64 at 2 fused multiply-adds per
// clock per SM, so the rows' solves (h NB^2 / 2 of them) are spread over
// h / 32 SMs instead of one.
template <typename T, int NB>
__global__ void __launch_bounds__(32)
k_band_panel_diag(T* __restrict__ base, const BandDesc* __restrict__ descs, int kb, DevStatus* st) {
  const BandDesc d = descs[0];
  const int n = d.n, w = d.w;
  const int64_t ld = d.ld;
  T* L = base + d.off;
  __shared__ T Dk[NB * (NB + 1)];
  constexpr int DS = NB + 1;
  const int lane = threadIdx.x;
  const int b = min(NB, n - kb);
  for (int idx = lane; idx < NB * NB; idx += 32) {
    const int r = idx / NB, c = idx % NB;
    T v = T(0);
    if (r < b && c < b && r >= c && r - c <= w) v = L[bidx(kb + r, kb + c, w, ld)];
    Dk[r * DS + c] = v;
  }
  __syncwarp();
  for (int t = 0; t < b; ++t) {
    if (lane == t) {
      T dv = Dk[t * DS + t];
      if (!finite_pos(dv)) {
        record_error(st, isfinite(dv) ? GENEO_ERR_NOT_SPD : GENEO_ERR_NONFINITE, d.id, (int64_t)kb + t);
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
  for (int idx = lane; idx < NB * NB; idx += 32) {
    const int r = idx / NB, c = idx % NB;
    if (r < b && c < b && r >= c && r - c <= w) L[bidx(kb + r, kb + c, w, ld)] = Dk[r * DS + c];
  }
}

// Rows kb + b + 32 blockIdx.x + lane of the panel: x L_kk^T = a (the
// diagonal block already factored), multiplying by the pivots' reciprocals.
template <typename T, int NB>
__global__ void __launch_bounds__(32)
k_band_panel_rows(T* __restrict__ base, const BandDesc* __restrict__ descs, int kb) {
  const BandDesc d = descs[0];
  const int n = d.n, w = d.w;
  const int64_t ld = d.ld;
  T* L = base + d.off;
  __shared__ T Dk[NB * (NB + 1)];
  __shared__ T rp[NB];
  constexpr int DS = NB + 1;
  const int lane = threadIdx.x;
  const int b = min(NB, n - kb);
  const int h = min(w, n - kb - b);
  for (int idx = lane; idx < NB * NB; idx += 32) {
    const int r = idx / NB, c = idx % NB;
    Dk[r * DS + c] = (r < b && c < b && r >= c && r - c <= w) ? L[bidx(kb + r, kb + c, w, ld)] : T(0);
  }
  __syncwarp();
  for (int t = lane; t < NB; t += 32) rp[t] = t < b ? T(1) / Dk[t * DS + t] : T(0);
  __syncwarp();
  const int i = 32 * blockIdx.x + lane;
  if (i >= h) return;
  const int rr = kb + b + i;
  T x[NB];
#pragma unroll
  for (int t = 0; t < NB; ++t) x[t] = (t < b && rr - (kb + t) <= w) ? L[bidx(rr, kb + t, w, ld)] : T(0);
#pragma unroll
  for (int t = 0; t < NB; ++t) {
    if (t < b) {
      T v = x[t];
#pragma unroll
      for (int u = 0; u < t; ++u) v -= x[u] * Dk[t * DS + u];
      x[t] = v * rp[t];
    }
  }
#pragma unroll
  for (int t = 0; t < NB; ++t)
    if (t < b && rr - (kb + t) <= w) L[bidx(rr, kb + t, w, ld)] = x[t];
}

// Trailing update of panel kb: C(i, i') -= sum_t P(i, t) P(i', t) over the
// h x h window below the panel, block (ti, tj) of 64 x 64 (ti >= tj), 4 x 4
// register tiles, panel rows staged in shared memory.
template <typename T, int NB>
__global__ void __launch_bounds__(kThreads)
k_band_trail(T* __restrict__ base, const BandDesc* __restrict__ descs, int kb) {
  const BandDesc d = descs[0];
  const int n = d.n, w = d.w;
  const int64_t ld = d.ld;
  T* L = base + d.off;
  const int b = min(NB, n - kb);
  const int h = min(w, n - kb - b);
  // block index -> (ti, tj) in the lower triangle, row-major
  const int t = blockIdx.x;
  int ti = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
  while (ti * (ti + 1) / 2 > t) --ti;
  const int tj = t - ti * (ti + 1) / 2;
  const int i0 = 64 * ti, j0 = 64 * tj;
  if (i0 >= h) return;
  __shared__ T Pi[NB][64 + 1], Pj[NB][64 + 1];
  for (int idx = threadIdx.x; idx < NB * 64; idx += blockDim.x) {
    const int tt = idx / 64, r = idx % 64;
    const int ii = i0 + r, jj = j0 + r;
    Pi[tt][r] = (tt < b && ii < h && b + ii - tt <= w) ? L[bidx(kb + b + ii, kb + tt, w, ld)] : T(0);
    Pj[tt][r] = (tt < b && jj < h && b + jj - tt <= w) ? L[bidx(kb + b + jj, kb + tt, w, ld)] : T(0);
  }
  __syncthreads();
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;  // 16 x 16 threads, 4 x 4 each
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = T(0);
  for (int tt = 0; tt < b; ++tt) {
    T pr[4], pc[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      pr[a] = Pi[tt][4 * ty + a];
      pc[a] = Pj[tt][4 * tx + a];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][c] += pr[a] * pc[c];
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + 4 * ty + a;
    if (i >= h) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int jj = j0 + 4 * tx + c;
      if (jj < h && jj <= i) L[bidx(kb + b + i, kb + b + jj, w, ld)] -= acc[a][c];
    }
  }
}

// Equilibration of a band before its FP32 factorisation: s_r = a_rr^{-1/2}
// (1 where a_rr is not positive: the factorisation reports it), then every
// entry a_rc *= s_r s_c, so the factor is that of S A S (unit diagonal) and
// A^{-1} = S (S A S)^{-1} S.  Grid: (row blocks, matrices).
template <typename T>
__global__ void k_band_equil_s(T* __restrict__ base, const BandDesc* __restrict__ descs) {
  const BandDesc d = descs[blockIdx.y];
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (d.scl < 0 || r >= d.n) return;
  const T a = base[d.off + (int64_t)r * d.ld + d.w];
  base[d.scl + r] = a > T(0) ? T(1) / sqrt(a) : T(1);
}

template <typename T>
__global__ void __launch_bounds__(256)
k_band_equil_a(T* __restrict__ base, const BandDesc* __restrict__ descs) {
  const BandDesc d = descs[blockIdx.y];
  if (d.scl < 0) return;
  const T* S = base + d.scl;
  for (int i = 0; i < 16; ++i) {
    const int r = blockIdx.x * 16 + i;
    if (r >= d.n) return;
    const T sr = S[r];
    T* row = base + d.off + (int64_t)r * d.ld;
    for (int off = max(0, d.w - r) + (int)threadIdx.x; off <= d.w; off += blockDim.x)
      row[off] *= sr * S[r - d.w + off];
  }
}

// x = s o x on columns [0, k) of the solve vectors (before and after the
// solves that do not apply the scaling themselves)
template <typename T>
__global__ void k_band_scale_x(const T* __restrict__ base, const BandDesc* __restrict__ descs,
                               double* __restrict__ xbase, const int64_t* __restrict__ xoff, int col0,
                               int kcap, const int32_t* __restrict__ nrhs_dev, const int32_t* __restrict__ skip) {
  const BandDesc d = descs[blockIdx.y];
  // vectors, counts and skip flags are indexed by the subdomain id (a
  // batch may hold a subset of the subdomains)
  const int mi = d.id >= 0 ? d.id : (int)blockIdx.y;
  if (skip && skip[mi]) return;
  if (d.scl < 0) return;
  int k = kcap;
  if (nrhs_dev) k = min(k, nrhs_dev[mi] - col0);
  const T* S = base + d.scl;
  double* X = xbase + xoff[mi] + (int64_t)col0 * d.n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)k * d.n;
       idx += (int64_t)gridDim.x * blockDim.x)
    X[idx] *= (double)S[idx % d.n];
}

// Inverses M of the 16 x 16 diagonal blocks of a factored band (FP64
// arithmetic, rounded to T), stored transposed (M(i, t) at 16 t + i): a
// half-warp per block, lane c forms column c by forward substitution.  The solves apply these blocks as small products, so
// no dependent chain of divisions sits on their sequential path.
template <typename T>
__global__ void __launch_bounds__(256)
k_band_dinv(T* __restrict__ base, const BandDesc* __restrict__ descs) {
  const BandDesc d = descs[blockIdx.y];
  const int lane = threadIdx.x & 31, c = lane & 15;
  const int blk = (blockIdx.x * 8 + (threadIdx.x >> 5)) * 2 + (lane >> 4);
  const int nb = (d.n + 15) / 16;
  if (blk >= nb || d.dinv < 0) return;
  const int kb = blk * 16, b = min(16, d.n - kb), w = d.w, ld = d.ld;
  const T* L = base + d.off;
  double x[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    double v = 0.0;
    if (r < b && c < b && r >= c) {
      v = r == c ? 1.0 : 0.0;
#pragma unroll
      for (int t = 0; t < r; ++t)
        if (t >= c && r - t <= w) v -= (double)L[(int64_t)(kb + r) * ld + (t - r + w)] * x[t];
      v /= (double)L[(int64_t)(kb + r) * ld + w];
    }
    x[r] = v;
  }
  T* D = base + d.dinv + (int64_t)blk * 256;
#pragma unroll
  for (int r = 0; r < 16; ++r) D[c * 16 + r] = (T)x[r];
}

// ---------------------------------------------------------------------------
// Left-looking FP32 band Cholesky on the tensor cores.
//
// Panel j (columns j .. j+b-1, b <= 32) of the rows r in [j, j + R),
// R = min(n, j + b + w) - j, is first brought up to date with all finished
// columns k in [j - w, j):
//   U(r, c) = A(r, c) - sum_k L(r, k) L(c, k),
// an (R x w) x (w x 32) product whose operands are whole band rows: the
// panel's own rows (staged once per panel) and the rows r (streamed in
// chunks of 16 by bulk copies, two buffers).  For each chunk's 16 x 32 tile
// every warp takes an eighth of the k range and accumulates it with m16n8k8
// TF32 MMAs in three passes (hi*hi + hi*lo + lo*hi with x = hi + lo, both
// TF32, split_tf32_rn), which keeps close to FP32 accuracy; the eight partial tiles go
// to one of two shared buffers and are summed in a fixed order while the next
// chunk multiplies (one block barrier per chunk).  Then the 32 x 32 diagonal
// block is factored by one warp in registers and the rows below by
// substitution, one row per thread.  Only the panel columns are written; the
// trailing window is never rewritten.
// ---------------------------------------------------------------------------
// x = hi + lo, both TF32 (split_tf32_rn), as the MMA's operand bits
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  float h, l;
  split_tf32_rn(x, h, l);
  hi = __float_as_uint(h);
  lo = __float_as_uint(l);
}
__device__ __forceinline__ void mma_tf32(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

constexpr int kPB = 32;   // panel width of the tensor-core factorisation
constexpr int kMC = 16;   // rows per streamed chunk (one 16-row MMA tile)
constexpr int kUS = kPB + 1;  // row stride of the panel block in shared memory

// Shared memory of the tensor-core factorisation for half-bandwidth w.
inline size_t potrf_tc_smem(int w) {
  const size_t ld = (size_t)band_ld(w);
  return 128 + sizeof(float) * ((kPB + 2 * kMC) * ld + (size_t)(w + kPB) * kUS + kPB + 2 * 8 * 16 * 32);
}

__global__ void __launch_bounds__(kThreads, 1)
k_band_potrf_tc(float* __restrict__ base, const BandDesc* __restrict__ descs, DevStatus* st,
                int32_t* __restrict__ weak, float weak_tol) {
  const BandDesc d = descs[blockIdx.x];
  const int n = d.n, w = d.w;
  const int ld = d.ld;
  float* L = base + d.off;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);                  // 0: panel rows, 1-2: chunks
  float* Cs = reinterpret_cast<float*>(smem_raw + 128);                    // kPB x ld
  float* Rs = Cs + (size_t)kPB * ld;                                       // 2 x kMC x ld
  float* Us = Rs + (size_t)2 * kMC * ld;                                   // (w + kPB) x kUS panel block
  float* Dinv = Us + (size_t)(w + kPB) * kUS;                              // kPB reciprocal pivots
  float* Red = Dinv + kPB;                                                 // 2 x 8 warps x 16 x 32 partials
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int g = lane >> 2, tg = lane & 3;
  if (tid == 0) {
    for (int i = 0; i < 3; ++i) mbar_init(&bars[i], 1);
    fence_barrier_init();
  }
  __syncthreads();
  uint32_t ph[3] = {0, 0, 0};      // next phase to wait for, per barrier
  int issued[3] = {0, 0, 0};       // thread 0: copies issued per barrier
  bool ok = true;                  // warp 0's view (thread 0 issues the copies)
  auto load_rows = [&](int bar, float* dst, int r0, int rows) {
    const uint32_t bytes = (uint32_t)((size_t)rows * ld * sizeof(float));
    mbar_arrive_expect_tx(&bars[bar], bytes);
    bulk_load(dst, L + (int64_t)r0 * ld, bytes, &bars[bar]);
    ++issued[bar];
  };
  // warp 0 waits; the block is released by the barrier that follows
  auto wait_bar = [&](int bar, int64_t where) {
    if (wid == 0 && ok) {
      ok = mbar_wait_bounded(&bars[bar], ph[bar] & 1, st, d.id, where);
    }
    ++ph[bar];
    __syncthreads();
  };

  for (int j = 0; j < n; j += kPB) {
    const int b = min(kPB, n - j);
    const int R = min(n, j + b + w) - j;
    const int kbeg = max(0, j - w);
    const int nch = (R + kMC - 1) / kMC;
    // the previous panel's columns were written by ordinary stores: order
    // them before the bulk copies that read them
    if (tid == 0 && ok) {
      fence_proxy_async_global();
      fence_proxy_async();
      load_rows(0, Cs, j, b);
      load_rows(1, Rs, j, min(kMC, R));
    }
    wait_bar(0, j);
    // One block barrier per chunk: the partial tiles of chunk ch go to
    // Red[ch & 1] and are summed in the next iteration (or after the loop),
    // with the A values each thread needs captured in registers before the
    // chunk's rows are overwritten; the next chunk's copy is issued after the
    // barrier, when no warp still reads the buffer it refills.
    const int nt2 = wid & 3, qh = wid >> 2;   // this thread's two reduce outputs
    float pa[2] = {0.f, 0.f};                 // A values of the pending chunk
    int prow = -1;                            // first row of the pending chunk (-1: none)
    auto reduce_pending = [&]() {
      if (prow < 0) return;
      const float* Rp = Red + (size_t)(((prow - j) / kMC) & 1) * (8 * 16 * 32);
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
        const int q = 2 * qh + h2;
        float sum = 0.f;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) sum += Rp[((size_t)kk * 16 + nt2 * 4 + q) * 32 + lane];
        const int r = prow + g + ((q & 2) ? 8 : 0);  // c0,c1: row g; c2,c3: row g+8
        const int cl = 8 * nt2 + 2 * tg + (q & 1), c = j + cl;
        if (r < j + R) {
          float u = 0.f;
          if (cl < b && c <= r && r - c <= w) u = pa[h2] - sum;
          Us[(size_t)(r - j) * kUS + cl] = u;
        }
      }
    };
    for (int ch = 0; ch < nch; ++ch) {
      const int buf = ch & 1;
      const int r0 = j + ch * kMC;
      wait_bar(1 + buf, (int64_t)j * 1024 + ch);
      if (tid == 0 && ok && ch + 1 < nch)
        load_rows(1 + (buf ^ 1), Rs + (size_t)(buf ^ 1) * kMC * ld, r0 + kMC, min(kMC, R - (ch + 1) * kMC));
      const float* Rb = Rs + (size_t)buf * kMC * ld;
      // warp kq: rows r0 .. r0 + 15, all 32 panel columns, over the kq-th
      // eighth of the k-steps of the tile's range
      const int kq = wid;
      const int ra = r0 + g, rb = r0 + g + 8;
      const bool va = ra < j + R, vb = rb < j + R;
      // element offsets of L(r, 0) in the staged rows (may be negative; an
      // index is formed only for k in the row's band)
      const int ia = g * ld + (w - ra);
      const int ib = (g + 8) * ld + (w - rb);
      const int klo = max(kbeg, r0 - w);          // no row of the tile reaches below klo
      const int kst = kbeg + ((klo - kbeg) & ~7);
      const int nsteps = (j - kst + 7) >> 3;
      const int s0 = kst + 8 * ((nsteps * kq) >> 3), s1 = kst + 8 * ((nsteps * (kq + 1)) >> 3);
      // every row and column is in band from kfull on
      const int kfull = max(r0 + 15, j + b - 1) - w;
      float acc[4][3][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 3; ++v)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[u][v][q] = 0.f;
      for (int k0 = s0; k0 < s1; k0 += 8) {
        const bool masked = k0 < kfull || k0 + 8 > j;
        const int k1 = k0 + tg, k2 = k0 + tg + 4;
        float x[4];
        if (!masked) {
          x[0] = va ? Rb[ia + k1] : 0.f;
          x[1] = vb ? Rb[ib + k1] : 0.f;
          x[2] = va ? Rb[ia + k2] : 0.f;
          x[3] = vb ? Rb[ib + k2] : 0.f;
        } else {
          x[0] = (va && k1 < j && k1 >= ra - w && k1 >= 0) ? Rb[ia + k1] : 0.f;
          x[1] = (vb && k1 < j && k1 >= rb - w && k1 >= 0) ? Rb[ib + k1] : 0.f;
          x[2] = (va && k2 < j && k2 >= ra - w && k2 >= 0) ? Rb[ia + k2] : 0.f;
          x[3] = (vb && k2 < j && k2 >= rb - w && k2 >= 0) ? Rb[ib + k2] : 0.f;
        }
        uint32_t ah[4], al[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) split_tf32(x[q], ah[q], al[q]);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          const int cn = 8 * nt + g, cc = j + cn;
          const int ic = cn * ld + (w - cc);
          float y0, y1;
          if (!masked) {
            y0 = cn < b ? Cs[ic + k1] : 0.f;
            y1 = cn < b ? Cs[ic + k2] : 0.f;
          } else {
            y0 = (cn < b && k1 < j && k1 >= cc - w && k1 >= 0) ? Cs[ic + k1] : 0.f;
            y1 = (cn < b && k2 < j && k2 >= cc - w && k2 >= 0) ? Cs[ic + k2] : 0.f;
          }
          uint32_t bh[2], bl[2];
          split_tf32(y0, bh[0], bl[0]);
          split_tf32(y1, bh[1], bl[1]);
          mma_tf32(acc[nt][0], al, bh);
          mma_tf32(acc[nt][1], ah, bl);
          mma_tf32(acc[nt][2], ah, bh);
        }
      }
      // partial sums of this eighth (small terms first), lane-contiguous
      float* Rw = Red + (size_t)buf * (8 * 16 * 32);
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          Rw[((size_t)kq * 16 + nt * 4 + q) * 32 + lane] = (acc[nt][0][q] + acc[nt][1][q]) + acc[nt][2][q];
      // warp w: n-tile w & 3, outputs q of half w >> 2; U = A - sum into the
      // panel block (zero outside the lower band), for the previous chunk
      reduce_pending();
      // capture this chunk's A values for its reduction in the next iteration
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
        const int q = 2 * qh + h2;
        const int r = r0 + g + ((q & 2) ? 8 : 0);
        const int cl = 8 * nt2 + 2 * tg + (q & 1), c = j + cl;
        pa[h2] = (r < j + R && cl < b && c <= r && r - c <= w) ? Rb[(size_t)(r - r0) * ld + (c - r + w)] : 0.f;
      }
      prow = r0;
    }
    __syncthreads();
    reduce_pending();
    __syncthreads();
    // ---- factor the panel's diagonal block in warp 0: lane r holds row r in
    // registers; step t takes pivot t from lane t (a pivot that is not
    // positive is reported and replaced by 1), scales column t and updates
    // the trailing part with shuffled column-t values (no block barriers).
    if (wid == 0) {
      float a[kPB];
#pragma unroll
      for (int u = 0; u < kPB; ++u) a[u] = (lane < b && u <= lane) ? Us[lane * kUS + u] : 0.f;
#pragma unroll
      for (int t = 0; t < kPB; ++t) {
        if (t < b) {  // uniform over the warp
          float p = __shfl_sync(0xffffffffu, a[t], t);
          if (weak) {
            if (lane == 0 && !(p > weak_tol)) weak[d.id] = 1;
            if (!finite_pos(p)) p = 1.f;
          } else if (!finite_pos(p)) {
            if (lane == 0) record_error(st, isfinite(p) ? GENEO_ERR_NOT_SPD : GENEO_ERR_NONFINITE, d.id, (int64_t)j + t);
            p = 1.f;
          }
          const float inv = rsqrtf(p);
          if (lane == t) {
            a[t] = p * inv;  // sqrt(pivot)
            Dinv[t] = inv;
          } else if (lane > t) {
            a[t] *= inv;
          }
#pragma unroll
          for (int u = t + 1; u < kPB; ++u) {
            const float lut = __shfl_sync(0xffffffffu, a[t], u);
            if (lane >= u) a[u] -= a[t] * lut;
          }
        }
      }
      if (lane < b) {
#pragma unroll
        for (int u = 0; u < kPB; ++u)
          if (u <= lane) Us[lane * kUS + u] = a[u];
      } else {
        Dinv[lane] = 0.f;
      }
    }
    __syncthreads();
    // rows below: x L_jj^T = u, one row per thread (stride kUS: no bank conflicts)
    for (int i = b + tid; i < R; i += kThreads) {
      float* ur = Us + (size_t)i * kUS;
      float x[kPB];
#pragma unroll
      for (int t = 0; t < kPB; ++t) x[t] = ur[t];
#pragma unroll
      for (int t = 0; t < kPB; ++t) {
        if (t < b) {
          float v = x[t];
#pragma unroll
          for (int u = 0; u < t; ++u) v -= x[u] * Us[t * kUS + u];
          x[t] = v * Dinv[t];
        }
      }
#pragma unroll
      for (int t = 0; t < kPB; ++t) ur[t] = x[t];
    }
    __syncthreads();
    // the panel's columns back to the band, one warp per row (coalesced)
    for (int i = wid; i < R; i += kThreads / 32) {
      const int r = j + i, c = j + lane;
      if (lane < b && c <= r && r - c <= w) L[(int64_t)r * ld + (c - r + w)] = Us[(size_t)i * kUS + lane];
    }
    __syncthreads();
  }
  // after a timed-out wait, let the copies still in flight land (bounded)
  if (tid == 0 && !ok)
    for (int bar = 0; bar < 3; ++bar)
      for (uint32_t p = ph[bar]; p < (uint32_t)issued[bar]; ++p)
        mbar_wait_bounded(&bars[bar], p & 1, st, d.id, -1);
}

// rows per streamed block: 16, or 4 for bands too wide for 16-row stages
// pipeline depth of the multi-right-hand-side solve: two stages leave room
// for the right-hand-side ring and two blocks per SM
template <typename T> struct Stages { static constexpr int v = 2; };

// Block v of the visit order 0..nb-1 (forward), nb-1..0 (backward).
__device__ __forceinline__ int visit_block(int v, int nb) { return v < nb ? v : 2 * nb - 1 - v; }

template <typename T, typename A, int kSNB, int kMaxRhsPerWarp, int kStages>
__global__ void __launch_bounds__(kThreads, kMaxRhsPerWarp == 1 ? (sizeof(T) == 4 ? 4 : 2) : 2)
k_band_solve(const T* __restrict__ base, const BandDesc* __restrict__ descs,
             double* __restrict__ xbase, const int64_t* __restrict__ xoff, int col0, int kcap,
             const int32_t* __restrict__ nrhs_dev, const int32_t* __restrict__ skip, int ring,
             DevStatus* st) {
  const BandDesc d = descs[blockIdx.x];
  // vectors, counts and skip flags are indexed by the subdomain id (a
  // batch may hold a subset of the subdomains)
  const int mi = d.id >= 0 ? d.id : (int)blockIdx.x;
  if (skip && skip[mi]) return;
  // column split: block y of gridDim.y takes its share of the kcap columns
  {
    const int cpp = (kcap + (int)gridDim.y - 1) / (int)gridDim.y;
    col0 += (int)blockIdx.y * cpp;
    kcap = min(cpp, kcap - (int)blockIdx.y * cpp);
  }
  int k = kcap;
  if (nrhs_dev) k = min(k, nrhs_dev[mi] - col0);
  if (k <= 0) return;
  const int n = d.n, w = d.w;
  if (n <= 0) return;
  const int ld = d.ld;
  const T* L = base + d.off;
  double* X = xbase + xoff[mi] + (int64_t)col0 * n;
  const int rmask = ring - 1;  // ring is a power of two >= w + 2 SNB

  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);                      // kStages
  T* stage = reinterpret_cast<T*>(smem_raw + 128);                             // kStages * SNB * ld
  A* win = reinterpret_cast<A*>(stage + (size_t)kStages * kSNB * ld);         // k columns of ring rows
  A* blk = win + (size_t)ring * k;                                             // SNB * k
  A* red = blk + (size_t)kSNB * k;                                             // 4 * kThreads
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = kThreads >> 5;
  const int nb = (n + kSNB - 1) / kSNB;
  const int nvis = 2 * nb;

  for (int idx = tid; idx < ring * k; idx += kThreads) win[idx] = A();
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 1);
    fence_barrier_init();
  }
  __syncthreads();
  auto issue = [&](int v) {
    const int kb = visit_block(v, nb) * kSNB;
    const int b = min(kSNB, n - kb);
    const int s = v % kStages;
    const uint32_t bytes = (uint32_t)((size_t)b * ld * sizeof(T));
    fence_proxy_async();
    mbar_arrive_expect_tx(&bars[s], bytes);
    bulk_load(stage + (size_t)s * kSNB * ld, L + (int64_t)kb * ld, bytes, &bars[s]);
  };
  int issued = 0;  // copies issued by thread 0
  if (tid == 0)
    for (; issued < min(kStages - 1, nvis); ++issued) issue(issued);
  bool ok = true;
  int waited = 0;  // stages this thread has waited for
  int lo = n;  // lowest row held in the ring during the backward sweep

  for (int v = 0; v < nvis; ++v) {
    const int s = v % kStages;
    const uint32_t parity = (uint32_t)((v / kStages) & 1);
    if (tid == 0 && ok && issued < nvis) issue(issued++);
    const int kb = visit_block(v, nb) * kSNB;
    const int b = min(kSNB, n - kb);
    if (v < nb) {
      // ---------------- forward, rows kb..kb+b-1 (left-looking)
      // right-hand sides of this block, fetched before the wait (lane i of
      // the warp owning right-hand side c holds b[kb + i][c])
      A xb[kMaxRhsPerWarp];
#pragma unroll
      for (int u = 0; u < kMaxRhsPerWarp; ++u) {
        const int c = wid + u * nw;
        xb[u] = (c < k && lane < b) ? to_arith<A>(X[(int64_t)c * n + kb + lane]) : A();
      }
      if (ok) {
        ok = mbar_wait_bounded(&bars[s], parity, st, d.id, v);
        waited += ok ? 1 : 0;
      }
      const T* S = stage + (size_t)s * kSNB * ld;
      // dot products with the solved rows [kb + i - w, kb) held in the ring:
      // a (b x w) x (w x k) product; a thread owns one row and CT right-hand
      // sides over one segment of the band, partials summed by the warp that
      // owns the right-hand side
      const int ct = k == 1 ? 1 : 4;
      const int ntc = (k + ct - 1) / ct;
      const int ntiles = b * ntc;
      const int nseg = max(1, min(32, kThreads / ntiles));
      for (int task = tid; task < ntiles * nseg; task += kThreads) {
        const int tile = task % ntiles, seg = task / ntiles;
        const int i = tile % b, c0 = (tile / b) * ct;
        const int r = kb + i;
        const int olo = max(0, w - r), ohi = w - i;  // columns r - w + oo in [0, kb)
        const int len = max(0, ohi - olo);
        const int s0 = olo + (int)((int64_t)len * seg / nseg);
        const int s1 = olo + (int)((int64_t)len * (seg + 1) / nseg);
        const T* srow = S + (size_t)i * ld;
        A a0 = A(), a1 = A(), a2 = A(), a3 = A();
        if (ct == 1) {
          const A* wc = win + (size_t)c0 * ring;
          int oo = s0;
          for (; oo + 1 < s1; oo += 2) {
            a0 += to_arith<A>(srow[oo]) * wc[(r - w + oo) & rmask];
            a1 += to_arith<A>(srow[oo + 1]) * wc[(r - w + oo + 1) & rmask];
          }
          if (oo < s1) a0 += to_arith<A>(srow[oo]) * wc[(r - w + oo) & rmask];
          a0 += a1;
          a1 = A();
        } else {
          const A* w0 = win + (size_t)c0 * ring;
          const bool h1 = c0 + 1 < k, h2 = c0 + 2 < k, h3 = c0 + 3 < k;
          const A* w1 = h1 ? w0 + ring : w0;
          const A* w2 = h2 ? w0 + 2 * ring : w0;
          const A* w3 = h3 ? w0 + 3 * ring : w0;
          for (int oo = s0; oo < s1; ++oo) {
            const A sv = to_arith<A>(srow[oo]);
            const int q = (r - w + oo) & rmask;
            a0 += sv * w0[q];
            a1 += sv * w1[q];
            a2 += sv * w2[q];
            a3 += sv * w3[q];
          }
        }
        A* rd = red + (size_t)(seg * ntiles + tile) * 4;
        rd[0] = a0;
        rd[1] = a1;
        rd[2] = a2;
        rd[3] = a3;
      }
      __syncthreads();
      // diagonal block by the warp owning each right-hand side: row of L and
      // the reciprocal pivot in registers, substitution by shuffles
      A lrow[kSNB];
#pragma unroll
      for (int t = 0; t < kSNB; ++t)
        lrow[t] = (lane < b && t < lane && lane - t <= w) ? to_arith<A>(S[lane * ld + (w - lane + t)]) : A();
      const A dinv = lane < b ? recip_arith<A>(S[lane * ld + w]) : A();
#pragma unroll
      for (int u = 0; u < kMaxRhsPerWarp; ++u) {
        const int c = wid + u * nw;
        if (c >= k) break;
        A y = A();
        if (lane < b) {
          const int tile = lane + (c / ct) * b, q = c % ct;
          A acc = A();
          for (int seg = 0; seg < nseg; ++seg) acc += red[(size_t)(seg * ntiles + tile) * 4 + q];
          y = xb[u] - acc;
        }
#pragma unroll
        for (int t = 0; t < kSNB; ++t) {
          if (t < b) {
            if (lane == t) y *= dinv;
            const A yt = shfl(y, t);
            if (lane > t) y -= lrow[t] * yt;
          }
        }
        if (lane < b) {
          win[(size_t)c * ring + ((kb + lane) & rmask)] = y;
          X[(int64_t)c * n + kb + lane] = to_double(y);
        }
      }
      if (v == nb - 1) lo = max(0, kb - w);  // the ring holds rows [lo, n) for the backward sweep
    } else {
      // ---------------- backward, block kb (right-looking on L^T)
      if (ok) {
        ok = mbar_wait_bounded(&bars[s], parity, st, d.id, v);
        waited += ok ? 1 : 0;
      }
      const T* S = stage + (size_t)s * kSNB * ld;
      A lcol[kSNB];
#pragma unroll
      for (int t = 0; t < kSNB; ++t)
        lcol[t] = (t < b && lane < t && t - lane <= w) ? to_arith<A>(S[t * ld + (w - t + lane)]) : A();
      const A dinv = lane < b ? recip_arith<A>(S[lane * ld + w]) : A();
      for (int c = wid; c < k; c += nw) {
        A y = lane < b ? win[(size_t)c * ring + ((kb + lane) & rmask)] : A();
#pragma unroll
        for (int t = kSNB - 1; t >= 0; --t) {
          if (t < b) {
            if (lane == t) y *= dinv;
            const A xt = shfl(y, t);
            if (lane < t) y -= lcol[t] * xt;
          }
        }
        if (lane < b) {
          blk[lane * k + c] = y;
          X[(int64_t)c * n + kb + lane] = to_double(y);
        }
      }
      __syncthreads();
      // rows [lo, kb) of the ring: y -= sum_t L(kb + t, row) x_t; at the same
      // time the rows the next block adds to the ring come from X (forward
      // results, not yet finalised by this sweep)
      const int cnt = kb - lo;
      const int ncg = (k + 3) / 4;
      for (int idx = tid; idx < cnt * ncg; idx += kThreads) {
        const int rr = lo + idx % cnt, c0 = (idx / cnt) * 4;
        A a0 = A(), a1 = A(), a2 = A(), a3 = A();
        const int tmax = min(b - 1, rr - kb + w);
        for (int t = 0; t <= tmax; ++t) {
          const A sv = to_arith<A>(S[t * ld + (rr - kb - t + w)]);
          const A* bt = blk + t * k + c0;
          a0 += sv * bt[0];
          if (c0 + 1 < k) a1 += sv * bt[1];
          if (c0 + 2 < k) a2 += sv * bt[2];
          if (c0 + 3 < k) a3 += sv * bt[3];
        }
        const int q = rr & rmask;
        win[(size_t)c0 * ring + q] -= a0;
        if (c0 + 1 < k) win[(size_t)(c0 + 1) * ring + q] -= a1;
        if (c0 + 2 < k) win[(size_t)(c0 + 2) * ring + q] -= a2;
        if (c0 + 3 < k) win[(size_t)(c0 + 3) * ring + q] -= a3;
      }
      if (kb > 0) {
        const int nlo = max(0, kb - kSNB - w);
        const int ncnt = lo - nlo;
        for (int idx = tid; idx < ncnt * k; idx += kThreads) {
          const int rr = nlo + idx % ncnt, c = idx / ncnt;
          win[(size_t)c * ring + (rr & rmask)] = to_arith<A>(X[(int64_t)c * n + rr]);
        }
        lo = nlo;
      }
    }
    __syncthreads();
  }
  // after a timed-out wait, let the copies still in flight land (bounded)
  if (tid == 0 && !ok)
    for (int v = waited; v < issued; ++v)
      mbar_wait_bounded(&bars[v % kStages], (uint32_t)((v / kStages) & 1), st, d.id, v);
}

// One right-hand side with the whole vector resident in shared memory (the
// preconditioner's local solves and the coarse solve).  The vector is read
// once at the start and written once at the end, so no global access sits on
// the sequential path of the sweeps; only the factor (band rows and the
// inverted diagonal block) streams in.  Forward block (left-looking): row i
// of the block is a dot product over the w solved entries to its left, split
// over a half-warp (16 segments, shuffle reduction), then the inverted
// diagonal block is applied.  Backward block (right-looking): the transposed
// inverse is applied, then every thread updates rows above the block.
template <typename T, int kStages>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 2 : 1)
k_band_solve_res(const T* __restrict__ base, const BandDesc* __restrict__ descs,
                 double* __restrict__ xbase, const int64_t* __restrict__ xoff,
                 const int32_t* __restrict__ nrhs_dev, const int32_t* __restrict__ skip, DevStatus* st) {
  constexpr int SNB = 16;
  const BandDesc d = descs[blockIdx.x];
  // vectors, counts and skip flags are indexed by the subdomain id (a
  // batch may hold a subset of the subdomains)
  const int mi = d.id >= 0 ? d.id : (int)blockIdx.x;
  if (skip && skip[mi]) return;
  if (nrhs_dev && nrhs_dev[mi] <= 0) return;
  const int n = d.n, w = d.w;
  if (n <= 0) return;
  const int ld = d.ld;
  const T* L = base + d.off;
  const T* Dg = base + d.dinv;
  double* X = xbase + xoff[mi];

  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);             // kStages
  T* stage = reinterpret_cast<T*>(smem_raw + 128);                    // kStages * SNB * ld
  T* dstage = stage + (size_t)kStages * SNB * ld;                     // kStages * 256
  T* vec = dstage + (size_t)kStages * 256;                            // n (padded to 4)
  T* zb = vec + ((n + 3) & ~3);                                       // SNB
  const int tid = threadIdx.x;
  const int nb = (n + SNB - 1) / SNB;
  const int nvis = 2 * nb;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 1);
    fence_barrier_init();
  }
  __syncthreads();
  auto issue = [&](int v) {
    const int blk = visit_block(v, nb), kb = blk * SNB;
    const int b = min(SNB, n - kb);
    const int s = v % kStages;
    const uint32_t bytes = (uint32_t)((size_t)b * ld * sizeof(T));
    fence_proxy_async();
    mbar_arrive_expect_tx(&bars[s], bytes + 256 * (uint32_t)sizeof(T));
    bulk_load(stage + (size_t)s * SNB * ld, L + (int64_t)kb * ld, bytes, &bars[s]);
    bulk_load(dstage + (size_t)s * 256, Dg + (int64_t)blk * 256, 256 * sizeof(T), &bars[s]);
  };
  int issued = 0;  // copies issued by thread 0
  if (tid == 0)
    for (; issued < min(kStages - 1, nvis); ++issued) issue(issued);
  const T* Sg = d.scl >= 0 ? base + d.scl : nullptr;  // equilibrated band: solve with S A S
  for (int i = tid; i < n; i += kThreads) vec[i] = Sg ? (T)X[i] * Sg[i] : (T)X[i];
  __syncthreads();
  bool ok = true;
  int waited = 0;  // stages this thread has waited for

  for (int v = 0; v < nvis; ++v) {
    const int s = v % kStages;
    const uint32_t parity = (uint32_t)((v / kStages) & 1);
    if (tid == 0 && ok && issued < nvis) issue(issued++);
    const int kb = visit_block(v, nb) * SNB;
    const int b = min(SNB, n - kb);
    if (ok) {
      ok = mbar_wait_bounded(&bars[s], parity, st, d.id, v);
      waited += ok ? 1 : 0;
    }
    const T* S = stage + (size_t)s * SNB * ld;
    const T* D = dstage + (size_t)s * 256;   // M(i, t) at D[16 t + i]
    if (v < nb) {
      // ---------------- forward: z_i = b_i - sum_{c < kb} L(kb+i, c) y_c
      const int i = tid >> 4, sl = tid & 15;
      T acc = T(0);
      if (i < b) {
        const int r = kb + i;
        const int olo = max(0, w - r), ohi = w - i;  // band offsets of the columns [r - w, kb)
        const int len = ohi - olo;
        const T* sp = S + (size_t)i * ld + olo;
        const T* vp = vec + (r - w + olo);
        T a1 = T(0);
        int j = sl;
        for (; j + 16 < len; j += 32) {
          acc += sp[j] * vp[j];
          a1 += sp[j + 16] * vp[j + 16];
        }
        if (j < len) acc += sp[j] * vp[j];
        acc += a1;
      }
#pragma unroll
      for (int off = 8; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off, 16);
      if (sl == 0 && i < b) zb[i] = vec[kb + i] - acc;
      __syncthreads();
      // y = M z
      if (tid < b) {
        T y = T(0);
#pragma unroll
        for (int t = 0; t < SNB; ++t)
          if (t <= tid) y += D[t * SNB + tid] * zb[t];
        vec[kb + tid] = y;
      }
    } else {
      // ---------------- backward: x = M^T y, then rows above the block
      if (tid < b) {
        T x = T(0);
#pragma unroll
        for (int j = 0; j < SNB; ++j) {
          const int i = (tid + j) & (SNB - 1);  // rotated: conflict-free reads of M
          if (i >= tid && i < b) x += D[tid * SNB + i] * vec[kb + i];
        }
        zb[tid] = x;
      }
      __syncthreads();
      if (tid < b) vec[kb + tid] = zb[tid];
      // y_rr -= sum_t L(kb + t, rr) x_{kb+t} for rr in [kb - w, kb)
      const int lo = max(0, kb - w);
      for (int rr = lo + tid; rr < kb; rr += kThreads) {
        const int tmax = min(b - 1, rr - kb + w);
        T a0 = T(0), a1 = T(0);
        int t = 0;
        for (; t + 1 <= tmax; t += 2) {
          a0 += S[t * ld + (rr - kb - t + w)] * zb[t];
          a1 += S[(t + 1) * ld + (rr - kb - t - 1 + w)] * zb[t + 1];
        }
        if (t <= tmax) a0 += S[t * ld + (rr - kb - t + w)] * zb[t];
        vec[rr] -= a0 + a1;
      }
    }
    __syncthreads();
  }
  // after a timed-out wait, let the copies still in flight land (bounded)
  if (tid == 0 && !ok)
    for (int v = waited; v < issued; ++v)
      mbar_wait_bounded(&bars[v % kStages], (uint32_t)((v / kStages) & 1), st, d.id, v);
  if (!ok) return;
  for (int i = tid; i < n; i += kThreads) X[i] = Sg ? (double)(vec[i] * Sg[i]) : (double)vec[i];
}

// One right-hand side for bands whose whole vector does not fit in shared
// memory next to the staged rows (wide bands, long subdomains, FP64).  The
// sweeps are those of k_band_solve_res (forward left-looking with the
// inverted 16 x 16 diagonal blocks, backward right-looking), with the
// vector kept as a window of the rows [kb - w - 16, kb + 16) in a ring of
// `ring` slots (a power of two >= w + 32): the forward results go to X as
// they are formed and come back into the ring during the backward sweep, one
// block ahead.  The band rows stream in as half blocks of 8 rows through kHS
// shared stages; warp 8 (one lane) issues the bulk copies as soon as a stage
// is released (full / empty mbarriers, the empty ones counted by the 256
// compute threads), so a stage is refilled while the other half of the
// block is still being used.  The first half block of every block also
// carries that block's inverted diagonal block.  Every wait is bounded; a
// wait that gives up records GENEO_ERR_TIMEOUT and raises a block-wide
// abort flag, and the copies already issued are waited for before exit.
template <typename T, int kHS>
__global__ void __launch_bounds__(kThreads + 32, 1)
k_band_solve_ring(const T* __restrict__ base, const BandDesc* __restrict__ descs,
                  double* __restrict__ xbase, const int64_t* __restrict__ xoff,
                  const int32_t* __restrict__ nrhs_dev, const int32_t* __restrict__ skip, int ring,
                  DevStatus* st) {
  constexpr int SNB = 16, HB = 8;
  const BandDesc d = descs[blockIdx.x];
  const int mi = d.id >= 0 ? d.id : (int)blockIdx.x;
  if (skip && skip[mi]) return;
  if (nrhs_dev && nrhs_dev[mi] <= 0) return;
  const int n = d.n, w = d.w;
  if (n <= 0) return;
  const int ld = d.ld;
  const T* L = base + d.off;
  const T* Dg = base + d.dinv;
  const T* Sg = d.scl >= 0 ? base + d.scl : nullptr;  // equilibrated band: solve with S A S
  double* X = xbase + xoff[mi];
  const int rmask = ring - 1;

  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);  // kHS
  uint64_t* empty = full + kHS;                             // kHS
  volatile int* abort = reinterpret_cast<volatile int*>(empty + kHS);
  T* stage = reinterpret_cast<T*>(smem_raw + 256);          // kHS * (HB * ld + 256)
  const size_t hs_len = (size_t)HB * ld + 256;              // rows, then the diagonal block
  T* vec = stage + (size_t)kHS * hs_len;                    // ring
  T* zb = vec + ring;                                       // SNB
  T* xs = zb + SNB;                                         // SNB
  T* rhs = xs + SNB;                                        // SNB: right-hand side of the next block
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nb = (n + SNB - 1) / SNB;
  const int nvis = 2 * nb;
  const int nhv = 2 * nvis;

  if (tid == 0) {
    for (int i = 0; i < kHS; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kThreads);
    }
    *abort = 0;
    fence_barrier_init();
  }
  for (int i = tid; i < ring; i += blockDim.x) vec[i] = T(0);
  for (int i = tid; i < SNB; i += blockDim.x) rhs[i] = (i < n) ? (Sg ? (T)X[i] * Sg[i] : (T)X[i]) : T(0);
  __syncthreads();

  auto bounded = [&](uint64_t* bar, uint32_t parity, int64_t where) -> bool {
    for (int it = 0; it < (1 << 22); ++it) {
      if (mbar_try_wait(bar, parity)) return true;
      if ((it & 1023) == 1023 && *abort) return false;
    }
    *abort = 1;
    record_error(st, GENEO_ERR_TIMEOUT, d.id, where);
    return false;
  };

  if (wid == kThreads / 32) {
    // ------------------------------------------------------------ copies
    if (lane == 0) {
      uint32_t iss[kHS];
#pragma unroll
      for (int i = 0; i < kHS; ++i) iss[i] = 0;
      for (int hv = 0; hv < nhv && !*abort; ++hv) {
        const int sl = hv % kHS;
        if (hv >= kHS && !bounded(&empty[sl], (uint32_t)((hv / kHS - 1) & 1), hv)) break;
        const int v = hv >> 1, h = hv & 1;
        const int blk = visit_block(v, nb), kb = blk * SNB;
        const int r0 = kb + HB * h, rows = max(0, min(HB, n - r0));
        const uint32_t bytes = (uint32_t)((size_t)rows * ld * sizeof(T));
        const uint32_t dbytes = h == 0 ? 256u * (uint32_t)sizeof(T) : 0u;
        T* dst = stage + (size_t)sl * hs_len;
        fence_proxy_async();
        mbar_arrive_expect_tx(&full[sl], bytes + dbytes);
        if (bytes) bulk_load(dst, L + (int64_t)r0 * ld, bytes, &full[sl]);
        if (dbytes) bulk_load(dst + (size_t)HB * ld, Dg + (int64_t)blk * 256, dbytes, &full[sl]);
        ++iss[sl];
      }
      // let every copy issued land before the block exits
#pragma unroll
      for (int i = 0; i < kHS; ++i)
        if (iss[i] > 0)
          for (int it = 0; it < (1 << 22) && !mbar_try_wait(&full[i], (iss[i] - 1) & 1); ++it) {
          }
    }
    return;
  }

  // ------------------------------------------------------------ sweeps
  int lo = n;  // lowest row in the ring during the backward sweep
  for (int v = 0; v < nvis; ++v) {
    const int kb = visit_block(v, nb) * SNB;
    const int b = min(SNB, n - kb);
    const int hv0 = 2 * v, s0 = hv0 % kHS, s1 = (hv0 + 1) % kHS;
    const uint32_t p0 = (uint32_t)((hv0 / kHS) & 1), p1 = (uint32_t)(((hv0 + 1) / kHS) & 1);
    const T* H0 = stage + (size_t)s0 * hs_len;  // rows kb .. kb + 7, then M
    const T* H1 = stage + (size_t)s1 * hs_len;  // rows kb + 8 .. kb + 15
    const T* D = H0 + (size_t)HB * ld;           // M(i, t) at D[16 t + i]
    if (v < nb) {
      // ---------------- forward: z_i = b_i - sum_{c < kb} L(kb+i, c) y_c
      T nxt = T(0);  // right-hand side of the next block (thread i < 16)
      if (tid < SNB && v + 1 < nb && kb + SNB + tid < n) {
        const int r = kb + SNB + tid;
        nxt = Sg ? (T)X[r] * Sg[r] : (T)X[r];
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (!*abort) bounded(h ? &full[s1] : &full[s0], h ? p1 : p0, v);
        const T* S = h ? H1 : H0;
        const int i = HB * h + wid;  // one row per warp
        T acc = T(0);
        if (i < b) {
          const int r = kb + i;
          const int olo = max(0, w - r), ohi = w - i;  // band offsets of the columns [r - w, kb)
          const T* sp = S + (size_t)wid * ld;
          T a1 = T(0);
          int j = olo + lane;
          for (; j + 32 < ohi; j += 64) {
            acc += sp[j] * vec[(r - w + j) & rmask];
            a1 += sp[j + 32] * vec[(r - w + j + 32) & rmask];
          }
          if (j < ohi) acc += sp[j] * vec[(r - w + j) & rmask];
          acc += a1;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0 && i < b) zb[i] = rhs[i] - acc;
        if (h == 1) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[s1])) : "memory");
      }
      asm volatile("bar.sync 1, 256;" ::: "memory");
      // y = M z
      if (tid < b) {
        T y = T(0);
#pragma unroll
        for (int t = 0; t < SNB; ++t)
          if (t <= tid) y += D[t * SNB + tid] * zb[t];
        vec[(kb + tid) & rmask] = y;
        X[kb + tid] = (double)y;
      }
      if (tid < SNB) rhs[tid] = nxt;
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[s0])) : "memory");
      if (v == nb - 1) lo = max(0, kb - w);
    } else {
      // ---------------- backward: x = M^T y, then rows above the block
      const int nlo = max(0, kb - SNB - w);
      T er = T(0);  // row entering the ring (forward result)
      if (tid < lo - nlo) er = (T)X[nlo + tid];
      if (!*abort) bounded(&full[s0], p0, v);
      if (!*abort) bounded(&full[s1], p1, v);
      if (tid < b) {
        T x = T(0);
#pragma unroll
        for (int j = 0; j < SNB; ++j) {
          const int i = (tid + j) & (SNB - 1);  // rotated: conflict-free reads of M
          if (i >= tid && i < b) x += D[tid * SNB + i] * vec[(kb + i) & rmask];
        }
        xs[tid] = x;
        X[kb + tid] = Sg ? (double)(x * Sg[kb + tid]) : (double)x;
      }
      asm volatile("bar.sync 1, 256;" ::: "memory");
      // y_rr -= sum_t L(kb + t, rr) x_t for rr in [lo, kb)
      for (int rr = lo + tid; rr < kb; rr += kThreads) {
        const int tmax = min(b - 1, rr - kb + w);
        T a0 = T(0), a1 = T(0);
        int t = 0;
        for (; t + 1 <= tmax; t += 2) {
          const T* r0p = t < HB ? H0 + (size_t)t * ld : H1 + (size_t)(t - HB) * ld;
          const T* r1p = t + 1 < HB ? H0 + (size_t)(t + 1) * ld : H1 + (size_t)(t + 1 - HB) * ld;
          a0 += r0p[rr - kb - t + w] * xs[t];
          a1 += r1p[rr - kb - t - 1 + w] * xs[t + 1];
        }
        if (t <= tmax) {
          const T* r0p = t < HB ? H0 + (size_t)t * ld : H1 + (size_t)(t - HB) * ld;
          a0 += r0p[rr - kb - t + w] * xs[t];
        }
        vec[rr & rmask] -= a0 + a1;
      }
      if (tid < lo - nlo) vec[(nlo + tid) & rmask] = er;
      lo = nlo;
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[s0])) : "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[s1])) : "memory");
    }
    asm volatile("bar.sync 1, 256;" ::: "memory");
  }
}

// Several right-hand sides (the eigensolver's K_j^{-1} blocks), at most
// 2 CT per launch.  The solved rows of the last w + 32 block rows sit in a
// shared ring stored row-major (row stride KP = 2 CT + 4 values, so rows
// taken by consecutive threads fall in distinct banks).
// Forward block: the (16 x w) x (w x k) product with the solved rows is cut
// into eight ranges of the band, one per warp; lane (i, g) owns row i and
// columns [g CT, g CT + CT), reads one factor value and CT/4 four-wide ring
// vectors per band position, and the warps' partial sums are added in a
// fixed order; the inverted diagonal block is then applied (one output per
// thread).  Backward block: the transposed inverse is applied, then the ring
// rows above the block are updated, one (row, four columns) item per thread.
// Right-hand sides of the next block and the rows that enter the ring are
// loaded one block ahead.
template <typename T, typename A, int CT, int kStages>
__global__ void __launch_bounds__(kThreads, 1)
k_band_solve_multi(const T* __restrict__ base, const BandDesc* __restrict__ descs,
                   double* __restrict__ xbase, const int64_t* __restrict__ xoff, int col0, int kcap,
                   const int32_t* __restrict__ nrhs_dev, const int32_t* __restrict__ skip, int ring,
                   DevStatus* st) {
  constexpr int SNB = 16;
  constexpr int KP = 2 * CT + 4;
  constexpr int NW = kThreads / 32;
  const BandDesc d = descs[blockIdx.x];
  // vectors, counts and skip flags are indexed by the subdomain id (a
  // batch may hold a subset of the subdomains)
  const int mi = d.id >= 0 ? d.id : (int)blockIdx.x;
  if (skip && skip[mi]) return;
  // column split: block y takes the columns [2 CT y, 2 CT (y + 1)) of the kcap
  col0 += (int)blockIdx.y * 2 * CT;
  kcap -= (int)blockIdx.y * 2 * CT;
  int k = min(kcap, 2 * CT);
  if (nrhs_dev) k = min(k, nrhs_dev[mi] - col0);
  if (k <= 0) return;
  const int n = d.n, w = d.w;
  if (n <= 0) return;
  const int ld = d.ld;
  const T* L = base + d.off;
  const T* Dg = base + d.dinv;
  double* X = xbase + xoff[mi] + (int64_t)col0 * n;
  const int rmask = ring - 1;  // ring: power of two >= w + 2 SNB

  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);      // kStages
  T* stage = reinterpret_cast<T*>(smem_raw + 128);             // kStages * SNB * ld
  T* dstage = stage + (size_t)kStages * SNB * ld;              // kStages * 256
  A* win = reinterpret_cast<A*>(dstage + (size_t)kStages * 256);  // ring * KP
  A* red = win + (size_t)ring * KP;                               // NW * SNB * KP
  A* zb = red + (size_t)NW * SNB * KP;                            // SNB * KP
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nb = (n + SNB - 1) / SNB;
  const int nvis = 2 * nb;

  for (int idx = tid; idx < ring * KP; idx += kThreads) win[idx] = A();
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 1);
    fence_barrier_init();
  }
  __syncthreads();
  auto issue = [&](int v) {
    const int blk = visit_block(v, nb), kb = blk * SNB;
    const int b = min(SNB, n - kb);
    const int s = v % kStages;
    const uint32_t bytes = (uint32_t)((size_t)b * ld * sizeof(T));
    fence_proxy_async();
    mbar_arrive_expect_tx(&bars[s], bytes + 256 * (uint32_t)sizeof(T));
    bulk_load(stage + (size_t)s * SNB * ld, L + (int64_t)kb * ld, bytes, &bars[s]);
    bulk_load(dstage + (size_t)s * 256, Dg + (int64_t)blk * 256, 256 * sizeof(T), &bars[s]);
  };
  int issued = 0;
  if (tid == 0)
    for (; issued < min(kStages - 1, nvis); ++issued) issue(issued);
  // element e of a (16 rows x k columns) block handled by this thread:
  // idx = tid + e * kThreads, column idx >> 4, row idx & 15
  auto load_rows = [&](int r0, int cnt, A* out) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int idx = tid + e * kThreads, c = idx >> 4, t = idx & 15;
      out[e] = (c < k && t < cnt) ? to_arith<A>(X[(int64_t)c * n + r0 + t]) : A();
    }
  };
  A xr[2];
  load_rows(0, min(SNB, n), xr);
  bool ok = true;
  int waited = 0;
  int lo = n;

  for (int v = 0; v < nvis; ++v) {
    const int s = v % kStages;
    const uint32_t parity = (uint32_t)((v / kStages) & 1);
    if (tid == 0 && ok && issued < nvis) issue(issued++);
    const int kb = visit_block(v, nb) * SNB;
    const int b = min(SNB, n - kb);
    const T* S = stage + (size_t)s * SNB * ld;
    const T* D = dstage + (size_t)s * 256;   // M(i, t) at D[16 t + i]
    if (v < nb) {
      // ---------------- forward
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int idx = tid + e * kThreads, c = idx >> 4, t = idx & 15;
        if (c < k) zb[t * KP + c] = xr[e];
      }
      if (v + 1 < nb) load_rows(kb + SNB, min(SNB, n - kb - SNB), xr);
      if (ok) {
        ok = mbar_wait_bounded(&bars[s], parity, st, d.id, v);
        waited += ok ? 1 : 0;
      }
      {
        const int i = lane & 15, g = lane >> 4;
        A acc[CT];
#pragma unroll
        for (int c = 0; c < CT; ++c) acc[c] = A();
        if (i < b) {
          const int ua = (int)((int64_t)w * wid / NW), ub = (int)((int64_t)w * (wid + 1) / NW);
          const int u0 = max(ua, max(i, w - kb));
          const T* srow = S + (size_t)i * ld - i;   // srow[u] = L(kb + i, kb - w + u)
          for (int u = u0; u < ub; ++u) {
            const A a = to_arith<A>(srow[u]);
            const A* rr = win + (size_t)((kb - w + u) & rmask) * KP + g * CT;
#pragma unroll
            for (int q = 0; q < CT / 4; ++q) {
              A xv[4];
              load4(rr + 4 * q, xv);
#pragma unroll
              for (int z = 0; z < 4; ++z) acc[4 * q + z] += a * xv[z];
            }
          }
        }
        A* rp = red + (size_t)(wid * SNB + i) * KP + g * CT;
#pragma unroll
        for (int q = 0; q < CT / 4; ++q) store4(rp + 4 * q, acc + 4 * q);
      }
      __syncthreads();
      for (int idx = tid; idx < SNB * k; idx += kThreads) {
        const int c = idx >> 4, t = idx & 15;
        A sum = A();
#pragma unroll
        for (int ww = 0; ww < NW; ++ww) sum += red[(size_t)(ww * SNB + t) * KP + c];
        zb[t * KP + c] -= sum;
      }
      __syncthreads();
      // y = M z: one (row, column) output per thread
      for (int idx = tid; idx < SNB * k; idx += kThreads) {
        const int c = idx >> 4, i = idx & 15;
        if (i < b) {
          A y = A();
#pragma unroll
          for (int t = 0; t < SNB; ++t)
            if (t <= i) y += to_arith<A>(D[t * SNB + i]) * zb[t * KP + c];
          win[(size_t)((kb + i) & rmask) * KP + c] = y;
          X[(int64_t)c * n + kb + i] = to_double(y);
        }
      }
      if (v == nb - 1) lo = max(0, kb - w);
    } else {
      // ---------------- backward
      const int nlo = max(0, kb - SNB - w);
      A er[2];
      load_rows(nlo, lo - nlo, er);  // rows entering the ring (forward results)
      if (ok) {
        ok = mbar_wait_bounded(&bars[s], parity, st, d.id, v);
        waited += ok ? 1 : 0;
      }
      // x = M^T y into zb (the ring rows of the block are not needed again)
      for (int idx = tid; idx < SNB * k; idx += kThreads) {
        const int c = idx >> 4, t = idx & 15;
        A x = A();
        if (t < b) {
#pragma unroll
          for (int j = 0; j < SNB; ++j) {
            const int i = (t + j) & (SNB - 1);  // rotated: conflict-free reads of M
            if (i >= t && i < b) x += to_arith<A>(D[t * SNB + i]) * win[(size_t)((kb + i) & rmask) * KP + c];
          }
          X[(int64_t)c * n + kb + t] = to_double(x);
        }
        zb[t * KP + c] = x;
      }
      __syncthreads();
      // rows [lo, kb): y_rr -= sum_t L(kb + t, rr) x_{kb+t}, items (row, four columns)
      const int cnt = kb - lo, nq = (k + 3) >> 2;
      for (int it = tid; it < cnt * nq; it += kThreads) {
        const int rr = lo + it % cnt, q = it / cnt;
        const int tmax = min(b - 1, rr - kb + w);
        A* yrow = win + (size_t)(rr & rmask) * KP + 4 * q;
        A acc[4];
        load4(yrow, acc);
        for (int t = 0; t <= tmax; ++t) {
          const A lv = to_arith<A>(S[t * ld + (rr - kb - t + w)]);
          A xv[4];
          load4(zb + t * KP + 4 * q, xv);
#pragma unroll
          for (int z = 0; z < 4; ++z) acc[z] -= lv * xv[z];
        }
        store4(yrow, acc);
      }
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int idx = tid + e * kThreads, c = idx >> 4, t = idx & 15;
        if (c < k && t < lo - nlo) win[(size_t)((nlo + t) & rmask) * KP + c] = er[e];
      }
      lo = nlo;
    }
    __syncthreads();
  }
  if (tid == 0 && !ok)
    for (int v = waited; v < issued; ++v)
      mbar_wait_bounded(&bars[v % kStages], (uint32_t)((v / kStages) & 1), st, d.id, v);
}

// Tensor-core variant of the multi-right-hand-side solve for FP32 factors:
// the same sweeps as k_band_solve_multi, with the two contractions done by
// m16n8k8 TF32 MMAs in three passes (hi*hi + hi*lo + lo*hi, about FP32
// accuracy):
//  forward  (16 x w) x (w x k): rows of the block against the solved ring
//           rows, the band cut into eight k-ranges (one per warp), partial
//           sums added in a fixed order;
//  backward (w x 16) x (16 x k): ring rows above the block minus L^T x, one
//           16-row tile per warp at a time, the ring values as the MMA's C.
// k <= 8 NT columns per launch.  The ring holds row r at slot r mod ring
// (ring a power of two >= w + 2 SNB); its row stride RP puts the four
// k-rows of a B fragment in distinct eight-bank groups: by padding (8, 24,
// 40 values for NT = 1, 3, 4) or, for NT = 2, with 16 values and the column
// halves swapped (column c at c ^ 8) on slots with bit 1 set.  With NT <= 2
// the block is sized for two resident blocks per SM.
template <int NT>
struct MtcKP { static constexpr int v = NT == 1 ? 8 : (NT == 4 ? 40 : 24); };
template <int NT>
struct MtcRP { static constexpr int v = NT == 2 ? 16 : MtcKP<NT>::v; };

template <int NT, int kStages, int PASSES>
__global__ void __launch_bounds__(kThreads, NT <= 2 ? 2 : 1)
k_band_solve_mtc(const float* __restrict__ base, const BandDesc* __restrict__ descs,
                 double* __restrict__ xbase, const int64_t* __restrict__ xoff, int col0, int kcap,
                 const int32_t* __restrict__ nrhs_dev, const int32_t* __restrict__ skip, int ring,
                 DevStatus* st) {
  constexpr int SNB = 16;
  constexpr int KP = MtcKP<NT>::v;   // row stride of zb and of the partial sums
  constexpr int RP = MtcRP<NT>::v;   // row stride of the ring
  constexpr bool SWZ = NT == 2;
  constexpr int NW = kThreads / 32;
  const BandDesc d = descs[blockIdx.x];
  // vectors, counts and skip flags are indexed by the subdomain id (a
  // batch may hold a subset of the subdomains)
  const int mi = d.id >= 0 ? d.id : (int)blockIdx.x;
  if (skip && skip[mi]) return;
  // column split: block y takes the columns [8 NT y, 8 NT (y + 1)) of the kcap
  col0 += (int)blockIdx.y * 8 * NT;
  kcap -= (int)blockIdx.y * 8 * NT;
  int k = min(kcap, 8 * NT);
  if (nrhs_dev) k = min(k, nrhs_dev[mi] - col0);
  if (k <= 0) return;
  const int n = d.n, w = d.w;
  if (n <= 0) return;
  const int ld = d.ld;
  const float* L = base + d.off;
  const float* Dg = base + d.dinv;
  double* X = xbase + xoff[mi] + (int64_t)col0 * n;
  const int rmask = ring - 1;
  auto slot = [&](int r) { return r & rmask; };

  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);      // kStages
  float* stage = reinterpret_cast<float*>(smem_raw + 128);     // kStages * SNB * ld
  float* dstage = stage + (size_t)kStages * SNB * ld;          // kStages * 256
  float* win = dstage + (size_t)kStages * 256;                 // ring * RP
  float* red = win + (size_t)ring * RP;                        // NW * SNB * KP
  float* zb = red + (size_t)NW * SNB * KP;                     // SNB * KP
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int g = lane >> 2, tg = lane & 3;
  const int nb = (n + SNB - 1) / SNB;
  const int nvis = 2 * nb;

  // columns >= k stay zero in the ring and in zb
  for (int idx = tid; idx < ring * RP; idx += kThreads) win[idx] = 0.f;
  auto rptr = [&](int r, int c) -> float* {
    const int sl = slot(r);
    return win + (size_t)sl * RP + (SWZ ? (c ^ ((sl << 2) & 8)) : c);
  };
  for (int idx = tid; idx < SNB * KP; idx += kThreads) zb[idx] = 0.f;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 1);
    fence_barrier_init();
  }
  __syncthreads();
  auto issue = [&](int v) {
    const int blk = visit_block(v, nb), kb = blk * SNB;
    const int b = min(SNB, n - kb);
    const int s = v % kStages;
    const uint32_t bytes = (uint32_t)((size_t)b * ld * sizeof(float));
    fence_proxy_async();
    mbar_arrive_expect_tx(&bars[s], bytes + 256 * (uint32_t)sizeof(float));
    bulk_load(stage + (size_t)s * SNB * ld, L + (int64_t)kb * ld, bytes, &bars[s]);
    bulk_load(dstage + (size_t)s * 256, Dg + (int64_t)blk * 256, 256 * sizeof(float), &bars[s]);
  };
  int issued = 0;
  if (tid == 0)
    for (; issued < min(kStages - 1, nvis); ++issued) issue(issued);
  const float* Sg = d.scl >= 0 ? base + d.scl : nullptr;  // equilibrated band: solve with S A S
  // rows of the (16 x k) block of this thread; `scaled` multiplies by s
  // (right-hand sides), the forward results re-entering the ring are not
  auto load_rows = [&](int r0, int cnt, float* out, bool scaled) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int idx = tid + e * kThreads, c = idx >> 4, t = idx & 15;
      float v = 0.f;
      if (c < k && t < cnt) {
        v = (float)X[(int64_t)c * n + r0 + t];
        if (scaled && Sg) v *= Sg[r0 + t];
      }
      out[e] = v;
    }
  };
  float xr[2];
  load_rows(0, min(SNB, n), xr, true);
  bool ok = true;
  int waited = 0;
  int lo = n;
  const int nsteps = (w + 7) >> 3;  // k-steps of eight band positions
  const int s0 = (nsteps * wid) / NW, s1 = (nsteps * (wid + 1)) / NW;

  for (int v = 0; v < nvis; ++v) {
    const int s = v % kStages;
    const uint32_t parity = (uint32_t)((v / kStages) & 1);
    if (tid == 0 && ok && issued < nvis) issue(issued++);
    const int kb = visit_block(v, nb) * SNB;
    const int b = min(SNB, n - kb);
    const float* S = stage + (size_t)s * SNB * ld;
    const float* D = dstage + (size_t)s * 256;   // M(i, t) at D[16 t + i]
    if (v < nb) {
      // ---------------- forward
      // right-hand sides of this block (element e of this thread), kept in
      // registers while the next block's are fetched
      float bcur[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) bcur[e] = xr[e];
      if (v + 1 < nb) load_rows(kb + SNB, min(SNB, n - kb - SNB), xr, true);
      if (ok) {
        ok = mbar_wait_bounded(&bars[s], parity, st, d.id, v);
        waited += ok ? 1 : 0;
      }
      {
        // A(i, u) = L(kb + i, kb - w + u) = S[i ld + u - i] for u >= i and
        // u >= w - kb (rows i = g, g + 8); B(u, c) = ring row kb - w + u
        float acc[NT][3][4];
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
          for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[nt][p][q] = 0.f;
        const bool va = g < b, vb = g + 8 < b;
        const int ia = g * (ld - 1), ib = (g + 8) * (ld - 1);
        const int kfull = max(15, w - kb);   // from here every row's element is in band
        for (int st8 = s0; st8 < s1; ++st8) {
          const int u0 = 8 * st8;
          const int k1 = u0 + tg, k2 = u0 + tg + 4;
          const bool masked = u0 < kfull || u0 + 8 > w;
          float x[4];
          if (!masked) {
            x[0] = va ? S[ia + k1] : 0.f;
            x[1] = vb ? S[ib + k1] : 0.f;
            x[2] = va ? S[ia + k2] : 0.f;
            x[3] = vb ? S[ib + k2] : 0.f;
          } else {
            const int lo0 = max(0, w - kb);
            x[0] = (va && k1 < w && k1 >= g && k1 >= lo0) ? S[ia + k1] : 0.f;
            x[1] = (vb && k1 < w && k1 >= g + 8 && k1 >= lo0) ? S[ib + k1] : 0.f;
            x[2] = (va && k2 < w && k2 >= g && k2 >= lo0) ? S[ia + k2] : 0.f;
            x[3] = (vb && k2 < w && k2 >= g + 8 && k2 >= lo0) ? S[ib + k2] : 0.f;
          }
          uint32_t ah[4], al[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) split_tf32(x[q], ah[q], al[q]);
          const int sl1 = slot(kb - w + k1), sl2 = slot(kb - w + k2);
          const float* r1 = win + (size_t)sl1 * RP + g;
          const float* r2 = win + (size_t)sl2 * RP + g;
          const int x1 = SWZ ? ((sl1 >> 1) & 1) : 0, x2 = SWZ ? ((sl2 >> 1) & 1) : 0;
#pragma unroll
          for (int nt = 0; nt < NT; ++nt) {
            uint32_t bh[2], bl[2];
            split_tf32(r1[8 * (nt ^ x1)], bh[0], bl[0]);
            split_tf32(r2[8 * (nt ^ x2)], bh[1], bl[1]);
            if (PASSES == 3) {
              mma_tf32(acc[nt][0], al, bh);
              mma_tf32(acc[nt][1], ah, bl);
            }
            mma_tf32(acc[nt][2], ah, bh);
          }
        }
        // partial sums: rows g, g + 8, columns 8 nt + 2 tg (+1)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int row = g + ((q & 2) ? 8 : 0), col = 8 * nt + 2 * tg + (q & 1);
            red[(size_t)(wid * SNB + row) * KP + col] = (acc[nt][0][q] + acc[nt][1][q]) + acc[nt][2][q];
          }
      }
      __syncthreads();
      // z = b - (the warps' partial sums) and y = M z for element (row t,
      // column c) of this thread: the 16 rows of a column are the 16 lanes
      // of one half-warp, which pass z to each other by shuffles (rows past
      // the block end hold z = 0)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int idx = tid + e * kThreads;
        if (idx < SNB * k) {
          const int c = idx >> 4, t = idx & 15;
          float sum = 0.f;
#pragma unroll
          for (int ww = 0; ww < NW; ++ww) sum += red[(size_t)(ww * SNB + t) * KP + c];
          const float z = bcur[e] - sum;
          const unsigned hm = 0xffffu << (lane & 16);
          float y = 0.f;
#pragma unroll
          for (int u = 0; u < SNB; ++u) {
            const float zu = __shfl_sync(hm, z, u, 16);
            if (u <= t) y += D[u * SNB + t] * zu;
          }
          if (t < b) {
            *rptr(kb + t, c) = y;
            X[(int64_t)c * n + kb + t] = (double)y;
          }
        }
      }
      if (v == nb - 1) lo = max(0, kb - w);
    } else {
      // ---------------- backward
      const int nlo = max(0, kb - SNB - w);
      float er[2];
      load_rows(nlo, lo - nlo, er, false);  // rows entering the ring (forward results)
      if (ok) {
        ok = mbar_wait_bounded(&bars[s], parity, st, d.id, v);
        waited += ok ? 1 : 0;
      }
      // x = M^T y into zb (the ring rows of the block are not needed again)
      for (int idx = tid; idx < SNB * k; idx += kThreads) {
        const int c = idx >> 4, t = idx & 15;
        float x = 0.f;
        if (t < b) {
#pragma unroll
          for (int j = 0; j < SNB; ++j) {
            const int i = (t + j) & (SNB - 1);  // rotated: conflict-free reads of M
            if (i >= t && i < b) x += D[t * SNB + i] * *rptr(kb + i, c);
          }
          X[(int64_t)c * n + kb + t] = Sg ? (double)(x * Sg[kb + t]) : (double)x;
        }
        zb[t * KP + c] = x;
      }
      __syncthreads();
      // rows [lo, kb): y_rr -= sum_t L(kb + t, rr) x_t, 16-row tiles
      {
        uint32_t bh[2][NT][2], bl[2][NT][2];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int nt = 0; nt < NT; ++nt) {
            split_tf32(zb[(8 * h + tg) * KP + 8 * nt + g], bh[h][nt][0], bl[h][nt][0]);
            split_tf32(zb[(8 * h + tg + 4) * KP + 8 * nt + g], bh[h][nt][1], bl[h][nt][1]);
          }
        const int cnt = kb - lo;
        const int ntile = (cnt + 15) >> 4;
        for (int tile = wid; tile < ntile; tile += NW) {
          const int ra = lo + 16 * tile + g, rb = ra + 8;
          float cacc[NT][4];
#pragma unroll
          for (int nt = 0; nt < NT; ++nt) {
            const int col = 8 * nt + 2 * tg;
            const float2 ya = ra < kb ? *reinterpret_cast<const float2*>(rptr(ra, col)) : make_float2(0.f, 0.f);
            const float2 yb = rb < kb ? *reinterpret_cast<const float2*>(rptr(rb, col)) : make_float2(0.f, 0.f);
            cacc[nt][0] = ya.x; cacc[nt][1] = ya.y; cacc[nt][2] = yb.x; cacc[nt][3] = yb.y;
          }
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            // A(rr, t) = -L(kb + t, rr) = -S[t ld + rr - kb - t + w], t <= min(b - 1, rr - kb + w)
            float x[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int rr = (q & 1) ? rb : ra;
              const int t = 8 * h + tg + ((q & 2) ? 4 : 0);
              const int off = rr - kb - t + w;
              x[q] = (rr < kb && t < b && off >= 0) ? -S[t * ld + off] : 0.f;
            }
            uint32_t ah[4], al[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) split_tf32(x[q], ah[q], al[q]);
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
              if (PASSES == 3) {
                mma_tf32(cacc[nt], al, bh[h][nt]);
                mma_tf32(cacc[nt], ah, bl[h][nt]);
              }
              mma_tf32(cacc[nt], ah, bh[h][nt]);
            }
          }
#pragma unroll
          for (int nt = 0; nt < NT; ++nt) {
            const int col = 8 * nt + 2 * tg;
            if (ra < kb) *reinterpret_cast<float2*>(rptr(ra, col)) = make_float2(cacc[nt][0], cacc[nt][1]);
            if (rb < kb) *reinterpret_cast<float2*>(rptr(rb, col)) = make_float2(cacc[nt][2], cacc[nt][3]);
          }
        }
      }
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int idx = tid + e * kThreads, c = idx >> 4, t = idx & 15;
        if (c < k && t < lo - nlo) *rptr(nlo + t, c) = er[e];
      }
      lo = nlo;
    }
    __syncthreads();
  }
  if (tid == 0 && !ok)
    for (int v = waited; v < issued; ++v)
      mbar_wait_bounded(&bars[v % kStages], (uint32_t)((v / kStages) & 1), st, d.id, v);
}

constexpr int kNB = 32;
constexpr size_t kSmemCap = 200 * 1024;

inline int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

}  // namespace

template <typename T>
geneo_status_t band_potrf(T* base, const BandDesc* d_desc, int count, int max_w, int max_n,
                          DevStatus* st, cudaStream_t s, bool equil, int32_t* weak, float weak_tol,
                          const Tc5Plan* tc5) {
  if (count <= 0) return GENEO_OK;
  // FP32: fifth-generation tensor cores (tcgen05, TMA) when the batch fits;
  // the packing into the tiled band applies the equilibration
  if constexpr (sizeof(T) == 4) {
    if (tc5 && tc5->ok) {
      if (equil && max_n > 0) {
        k_band_equil_s<T><<<dim3((max_n + 255) / 256, count), 256, 0, s>>>(base, d_desc); note_launch();
        GENEO_CUDA(cudaGetLastError());
      }
      GENEO_TRY(tc5_factor(*tc5, base, d_desc, st, s, weak, weak_tol * kTf32PivotScale));
      if (max_n > 0) {
        const int nb = (max_n + 15) / 16;
        k_band_dinv<T><<<dim3((nb + 15) / 16, count), 256, 0, s>>>(base, d_desc); note_launch();
        GENEO_CUDA(cudaGetLastError());
      }
      return GENEO_OK;
    }
  }
  if (equil && max_n > 0) {
    k_band_equil_s<T><<<dim3((max_n + 255) / 256, count), 256, 0, s>>>(base, d_desc); note_launch();
    k_band_equil_a<T><<<dim3((max_n + 15) / 16, count), 256, 0, s>>>(base, d_desc); note_launch();
    GENEO_CUDA(cudaGetLastError());
  }
  // FP32: left-looking tensor-core kernel when a panel's rows and two chunk
  // buffers fit in shared memory
  if constexpr (sizeof(T) == 4) {
    const size_t tc_smem = potrf_tc_smem(max_w);
    if (tc_smem <= 227 * 1024) {
      GENEO_CUDA(allow_smem(k_band_potrf_tc));
      k_band_potrf_tc<<<count, kThreads, tc_smem, s>>>(base, d_desc, st, weak, weak_tol * kTf32PivotScale);
      note_launch();
      GENEO_CUDA(cudaGetLastError());
      if (max_n > 0) {
        const int nb = (max_n + 15) / 16;
        k_band_dinv<T><<<dim3((nb + 15) / 16, count), 256, 0, s>>>(base, d_desc); note_launch();
        GENEO_CUDA(cudaGetLastError());
      }
      return GENEO_OK;
    }
  }
  // one large matrix (the coarse matrix): spread each panel's update over SMs
  if (count == 1 && max_n > 256 && max_w >= 128 && !weak) {
    constexpr int PB = 32;
    for (int kb = 0; kb < max_n; kb += PB) {
      k_band_panel_diag<T, PB><<<1, 32, 0, s>>>(base, d_desc, kb, st); note_launch();
      const int b = std::min(PB, max_n - kb);
      const int h = std::min(max_w, max_n - kb - b);
      if (h > 0) {
        k_band_panel_rows<T, PB><<<(h + 31) / 32, 32, 0, s>>>(base, d_desc, kb); note_launch();
        const int T64 = (h + 63) / 64;
        k_band_trail<T, PB><<<T64 * (T64 + 1) / 2, kThreads, 0, s>>>(base, d_desc, kb); note_launch();
      }
    }
    GENEO_CUDA(cudaGetLastError());
    const int nb = (max_n + 15) / 16;
    k_band_dinv<T><<<dim3((nb + 15) / 16, 1), 256, 0, s>>>(base, d_desc); note_launch();
    GENEO_CUDA(cudaGetLastError());
    return GENEO_OK;
  }
  // the panel starts at a 16-byte boundary (diag block: 32 x 33 values) and
  // its row stride phmax is a multiple of 4
  const size_t diag = (size_t)kNB * (kNB + 1) * sizeof(T);
  const int phmax = (max_w + 3) & ~3;
  const size_t panel = (size_t)phmax * kNB * sizeof(T);
  if (diag + panel <= kSmemCap) {
    auto kern = k_band_potrf<T, kNB, true>;
    GENEO_CUDA(allow_smem(kern));
    kern<<<count, kThreads, diag + panel, s>>>(base, d_desc, phmax, st, weak, weak_tol); note_launch();
  } else {
    auto kern = k_band_potrf<T, kNB, false>;
    kern<<<count, kThreads, diag, s>>>(base, d_desc, 0, st, weak, weak_tol); note_launch();
  }
  GENEO_CUDA(cudaGetLastError());
  if (max_n > 0) {
    const int nb = (max_n + 15) / 16;
    k_band_dinv<T><<<dim3((nb + 15) / 16, count), 256, 0, s>>>(base, d_desc); note_launch();
    GENEO_CUDA(cudaGetLastError());
  }
  return GENEO_OK;
}

// Shared memory of one solve launch with k right-hand sides.
template <typename T>
size_t solve_smem(int max_w, int k, int ring, int snb, int stages) {
  const int ld = band_ld(max_w);
  return 128 + sizeof(T) * ((size_t)stages * snb * ld + (size_t)ring * k + (size_t)snb * k + 4 * kThreads);
}

// Shared memory of the register-tiled multi-right-hand-side solve.
template <typename T>
size_t multi_smem(int max_w, int ring, int CT, int stages) {
  const int ld = band_ld(max_w);
  const int KP = 2 * CT + 4;
  return 128 + sizeof(T) * ((size_t)stages * (16 * ld + 256) + (size_t)ring * KP +
                            (size_t)(kThreads / 32 + 1) * 16 * KP);
}

// Column split of a multi-right-hand-side launch: when a batch holds at most
// half as many matrices as the GPU has SMs, each matrix's columns are cut
// into parts (grid y) that run on otherwise idle SMs, each part a shorter
// dependent sweep with less work per step; at most `units` parts and no more
// blocks than SMs.
inline int sm_count() {
  static int sms[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (!sms[dev] && cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 152;
  }
  return sms[dev];
}
inline int split_parts(int count, int units) {
  const int sms = sm_count();
  if (count <= 0 || 2 * count > sms || units <= 1) return 1;
  return std::max(1, std::min(units, sms / count));
}

template <typename T, typename A, int CT, int kStages>
geneo_status_t launch_multi_t(dim3 grid, size_t smem, cudaStream_t s, const T* base, const BandDesc* d_desc,
                              double* xbase, const int64_t* xoff, int c0, int kc,
                              const int32_t* nrhs_dev, const int32_t* skip_dev, int ring, DevStatus* st) {
  auto kern = k_band_solve_multi<T, A, CT, kStages>;
  GENEO_CUDA(allow_smem(kern));
  kern<<<grid, kThreads, smem, s>>>(base, d_desc, xbase, xoff, c0, kc, nrhs_dev, skip_dev, ring, st);
  note_launch();
  GENEO_CUDA(cudaGetLastError());
  return GENEO_OK;
}

template <typename T, typename A = T>
geneo_status_t launch_multi(int CT, int stages, dim3 grid, size_t smem, cudaStream_t s, const T* base,
                            const BandDesc* d_desc, double* xbase, const int64_t* xoff, int c0, int kc,
                            const int32_t* nrhs_dev, const int32_t* skip_dev, int ring, DevStatus* st) {
#define GENEO_MULTI(ct, sg)                                                                       \
  if (CT == ct && stages == sg)                                                                  \
    return launch_multi_t<T, A, ct, sg>(grid, smem, s, base, d_desc, xbase, xoff, c0, kc, nrhs_dev, \
                                     skip_dev, ring, st);
  GENEO_MULTI(4, 2) GENEO_MULTI(4, 4) GENEO_MULTI(8, 2) GENEO_MULTI(8, 4)
  if constexpr (sizeof(T) == 4) {
    GENEO_MULTI(12, 2) GENEO_MULTI(12, 4) GENEO_MULTI(16, 2) GENEO_MULTI(16, 4)
  }
#undef GENEO_MULTI
  return GENEO_ERR_ARG;
}

// Shared memory of the tensor-core multi-right-hand-side solve (ring and
// partial-sum strides as in MtcRP / MtcKP).
inline size_t mtc_smem(int max_w, int ring, int NT, int stages) {
  const int ld = band_ld(max_w);
  const int KP = NT == 1 ? 8 : (NT == 4 ? 40 : 24);
  const int RP = NT == 2 ? 16 : KP;
  return 128 + sizeof(float) * ((size_t)stages * (16 * ld + 256) + (size_t)ring * RP +
                                (size_t)(kThreads / 32 + 1) * 16 * KP);
}
// Shared memory per block that still lets two blocks share an SM.
constexpr size_t kTwoPerSm = 112 * 1024;

template <int NT, int kStages, int PASSES>
geneo_status_t launch_mtc_t(dim3 grid, size_t smem, cudaStream_t s, const float* base, const BandDesc* d_desc,
                            double* xbase, const int64_t* xoff, int c0, int kc,
                            const int32_t* nrhs_dev, const int32_t* skip_dev, int ring, DevStatus* st) {
  auto kern = k_band_solve_mtc<NT, kStages, PASSES>;
  GENEO_CUDA(allow_smem(kern));
  kern<<<grid, kThreads, smem, s>>>(base, d_desc, xbase, xoff, c0, kc, nrhs_dev, skip_dev, ring, st);
  note_launch();
  GENEO_CUDA(cudaGetLastError());
  return GENEO_OK;
}

geneo_status_t launch_mtc(int NT, int stages, int passes, dim3 grid, size_t smem, cudaStream_t s,
                          const float* base, const BandDesc* d_desc, double* xbase, const int64_t* xoff,
                          int c0, int kc, const int32_t* nrhs_dev, const int32_t* skip_dev, int ring,
                          DevStatus* st) {
#define GENEO_MTC(nt, sg)                                                                              \
  if (NT == nt && stages == sg)                                                                        \
    return passes == 1 ? launch_mtc_t<nt, sg, 1>(grid, smem, s, base, d_desc, xbase, xoff, c0, kc,    \
                                                 nrhs_dev, skip_dev, ring, st)                         \
                       : launch_mtc_t<nt, sg, 3>(grid, smem, s, base, d_desc, xbase, xoff, c0, kc,    \
                                                 nrhs_dev, skip_dev, ring, st);
  GENEO_MTC(1, 2) GENEO_MTC(1, 3) GENEO_MTC(1, 4) GENEO_MTC(2, 2) GENEO_MTC(2, 3) GENEO_MTC(2, 4)
  GENEO_MTC(3, 2) GENEO_MTC(3, 3) GENEO_MTC(3, 4) GENEO_MTC(4, 2) GENEO_MTC(4, 3) GENEO_MTC(4, 4)
#undef GENEO_MTC
  return GENEO_ERR_ARG;
}

// Shared memory of the resident-vector one-right-hand-side solve.
template <typename T>
size_t res_smem(int max_w, int max_n, int snb, int stages) {
  const int ld = band_ld(max_w);
  return 128 + sizeof(T) * ((size_t)stages * (snb * ld + 256) + (size_t)((max_n + 3) & ~3) + snb);
}

// Shared memory of the ring one-right-hand-side solve: barriers, hs half
// blocks of 8 rows with a diagonal block each, the ring, three 16-vectors.
template <typename T>
size_t ring_smem(int max_w, int ring, int hs) {
  const int ld = band_ld(max_w);
  return 256 + sizeof(T) * ((size_t)hs * (8 * (size_t)ld + 256) + (size_t)ring + 48);
}

// Solves with the kernels that do not apply a band's row scaling (the
// caller scales the vectors around them).
template <typename T, typename A = T>
geneo_status_t band_solve_plain(const T* base, const BandDesc* d_desc, int count, int max_w,
                                double* xbase, const int64_t* xoff, int nrhs, const int32_t* nrhs_dev,
                                const int32_t* skip_dev, DevStatus* st, cudaStream_t s, int live = 0) {
  if (live <= 0) live = count;
  if (nrhs == 1) {
    int snb = 16;
    if (solve_smem<T>(max_w, 1, next_pow2(max_w + 32), 16, 2) > kSmemCap) snb = 4;
    const int ring = next_pow2(max_w + 2 * snb);
    const size_t smem = solve_smem<T>(max_w, 1, ring, snb, 2);
    if (smem > 227 * 1024) return GENEO_ERR_ARG;
    auto kern = snb == 16 ? k_band_solve<T, A, 16, 1, 2> : k_band_solve<T, A, 4, 1, 2>;
    GENEO_CUDA(allow_smem(kern));
    kern<<<count, kThreads, smem, s>>>(base, d_desc, xbase, xoff, 0, 1, nrhs_dev, skip_dev, ring, st); note_launch();
    GENEO_CUDA(cudaGetLastError());
    return GENEO_OK;
  }
  // register-tiled kernel: up to 32 (FP32) or 16 (FP64) columns per launch
  {
    const int ring = next_pow2(max_w + 32);
    const int kmax = std::min(nrhs, sizeof(T) == 4 ? 32 : 16);
    const int CT0 = (((kmax + 1) / 2) + 3) & ~3;
    if (multi_smem<T>(max_w, ring, CT0, 2) <= 227 * 1024) {
      for (int c0 = 0; c0 < nrhs; c0 += kmax) {
        const int kc = std::min(kmax, nrhs - c0);
        int CT = (((kc + 1) / 2) + 3) & ~3;
        // parts of 8 k columns (CT a multiple of 4)
        const int units = (kc + 7) / 8, parts = split_parts(live, units);
        int nsplit = 1;
        if (parts > 1) {
          CT = 4 * ((units + parts - 1) / parts);
          nsplit = (kc + 2 * CT - 1) / (2 * CT);
        }
        const int stages = multi_smem<T>(max_w, ring, CT, 4) <= 227 * 1024 ? 4 : 2;
        const geneo_status_t rc = launch_multi<T, A>(CT, stages, dim3(count, nsplit),
                                                      multi_smem<T>(max_w, ring, CT, stages), s, base, d_desc,
                                                      xbase, xoff, c0, kc, nrhs_dev, skip_dev, ring, st);
        if (rc != GENEO_OK) return rc;
      }
      return GENEO_OK;
    }
  }
  constexpr int stg = Stages<T>::v;
  int snb = 16;
  if (solve_smem<T>(max_w, 1, next_pow2(max_w + 32), 16, stg) > kSmemCap) snb = 4;
  const int ring = next_pow2(max_w + 2 * snb);
  // right-hand sides per launch: as many as fit in shared memory, at most 64
  // (8 warps x 8 register slots; the forward partial-sum buffer holds
  // 4 * kThreads values for b * ceil(k / 4) <= kThreads tiles)
  int kmax = std::min(nrhs, 64);
  while (kmax > 1 && solve_smem<T>(max_w, kmax, ring, snb, stg) > kSmemCap) kmax = (kmax + 1) / 2;
  const size_t smem = solve_smem<T>(max_w, kmax, ring, snb, stg);
  if (smem > 227 * 1024) return GENEO_ERR_ARG;  // band too wide for the streamed solve
  auto kern = snb == 16 ? k_band_solve<T, A, 16, 8, stg> : k_band_solve<T, A, 4, 8, stg>;
  GENEO_CUDA(allow_smem(kern));
  for (int c0 = 0; c0 < nrhs; c0 += kmax) {
    const int kc = std::min(kmax, nrhs - c0);
    const int nsplit = split_parts(live, (kc + 3) / 4);  // parts of at least 4 columns
    kern<<<dim3(count, nsplit), kThreads, smem, s>>>(base, d_desc, xbase, xoff, c0, kc, nrhs_dev, skip_dev, ring,
                                                     st);
    note_launch();
    GENEO_CUDA(cudaGetLastError());
  }
  return GENEO_OK;
}

template <typename T, typename A>
geneo_status_t band_solve_impl(const T* base, const BandDesc* d_desc, int count, int max_w,
                               double* xbase, const int64_t* xoff, int nrhs, const int32_t* nrhs_dev,
                               const int32_t* skip_dev, DevStatus* st, cudaStream_t s, int max_n, int tc_passes,
                               int res_stages, int active) {
  if (count <= 0 || nrhs <= 0) return GENEO_OK;
  // double-single arithmetic covers the multi-column solves; one right-hand
  // side keeps the FP64 kernels
  if constexpr (!std::is_same_v<A, T>) {
    if (nrhs == 1)
      return band_solve_impl<T, T>(base, d_desc, count, max_w, xbase, xoff, nrhs, nrhs_dev, skip_dev, st, s, max_n,
                                   tc_passes, res_stages, active);
  }
  // matrices to solve (the others are skipped by their blocks at once): the
  // column split and the pipeline depth follow this number
  const int live = active > 0 ? std::min(active, count) : count;
  // One right-hand side (the preconditioner's local solves): two stages and
  // one register slot per warp keep the block small enough for several
  // blocks per SM, which hides the latency of the sequential sweep.
  if (nrhs == 1) {
    // whole vector resident in shared memory when it fits; the deepest
    // pipeline (at most four stages) that keeps two blocks per SM for FP32
    // batches (one for FP64 or a small batch) hides the latency of the
    // factor stream
    if (max_n > 0) {
      const size_t budget = (sizeof(T) == 4 && count > 152) ? 112 * 1024 : 226 * 1024;
      int stages = 4;
      while (stages > 2 && res_smem<T>(max_w, max_n, 16, stages) > budget) --stages;
      // a depth chosen by the autotuner (solve.cu) when it fits
      if (res_stages >= 2 && res_stages <= 4 && res_smem<T>(max_w, max_n, 16, res_stages) <= 227 * 1024)
        stages = res_stages;
      const size_t smem = res_smem<T>(max_w, max_n, 16, stages);
      if (smem <= 227 * 1024) {
        auto kern = stages == 4 ? k_band_solve_res<T, 4>
                  : stages == 3 ? k_band_solve_res<T, 3> : k_band_solve_res<T, 2>;
        GENEO_CUDA(allow_smem(kern));
        kern<<<count, kThreads, smem, s>>>(base, d_desc, xbase, xoff, nrhs_dev, skip_dev, st); note_launch();
        GENEO_CUDA(cudaGetLastError());
        return GENEO_OK;
      }
    }
    // the vector does not fit: a window of it in a ring, the band in
    // half-block stages, as many as fit
    const int ring = next_pow2(max_w + 32);
    int hs = 6;
    while (hs > 2 && ring_smem<T>(max_w, ring, hs) > 227 * 1024) hs = hs == 6 ? 4 : hs - 1;
    const size_t smem = ring_smem<T>(max_w, ring, hs);
    if (smem <= 227 * 1024) {
      auto kern = hs == 6 ? k_band_solve_ring<T, 6>
                : hs == 4 ? k_band_solve_ring<T, 4>
                : hs == 3 ? k_band_solve_ring<T, 3> : k_band_solve_ring<T, 2>;
      GENEO_CUDA(allow_smem(kern));
      kern<<<count, kThreads + 32, smem, s>>>(base, d_desc, xbase, xoff, nrhs_dev, skip_dev, ring, st);
      note_launch();
      GENEO_CUDA(cudaGetLastError());
      return GENEO_OK;
    }
  }
  // FP32 factors: tensor-core kernel, up to 32 columns per launch
  if constexpr (sizeof(T) == 4) {
    const int ring = next_pow2(max_w + 32);
    if (mtc_smem(max_w, ring, 1, 2) <= 227 * 1024) {
      for (int c0 = 0; c0 < nrhs; c0 += 32) {
        const int kc = std::min(32, nrhs - c0);
        int NT = (kc + 7) / 8;
        while (NT > 1 && mtc_smem(max_w, ring, NT, 2) > 227 * 1024) --NT;
        const int kk = std::min(kc, 8 * NT);
        // column parts of 8 NT columns for small batches
        int nsplit = 1;
        {
          const int parts = split_parts(live, NT);
          if (parts > 1) {
            NT = (NT + parts - 1) / parts;
            nsplit = (kk + 8 * NT - 1) / (8 * NT);
          }
        }
        // the deepest pipeline that keeps two blocks per SM when the batch
        // fills more than one wave of single blocks (NT <= 2), else the
        // deepest that fits
        int stages = 4;
        const size_t cap = (NT <= 2 && live > 152 && mtc_smem(max_w, ring, NT, 2) <= kTwoPerSm) ? kTwoPerSm
                                                                                                : 227 * 1024;
        while (stages > 2 && mtc_smem(max_w, ring, NT, stages) > cap) --stages;
        GENEO_TRY(launch_mtc(NT, stages, tc_passes, dim3(count, nsplit), mtc_smem(max_w, ring, NT, stages), s,
                             base, d_desc, xbase, xoff, c0, kk, nrhs_dev, skip_dev, ring, st));
        if (kk < kc) c0 -= kc - kk;  // the rest of this chunk goes in the next launch
      }
      return GENEO_OK;
    }
  }
  // other kernels: the vectors are scaled around the solve where the bands
  // are equilibrated (FP32 factors)
  if constexpr (sizeof(T) == 4) {
    const int gx = std::max(1, std::min(64, (max_n > 0 ? max_n : 4096) * nrhs / 256));
    k_band_scale_x<T><<<dim3(gx, count), 256, 0, s>>>(base, d_desc, xbase, xoff, 0, nrhs, nrhs_dev, skip_dev);
    note_launch();
    GENEO_TRY(band_solve_plain<T>(base, d_desc, count, max_w, xbase, xoff, nrhs, nrhs_dev, skip_dev, st, s, live));
    k_band_scale_x<T><<<dim3(gx, count), 256, 0, s>>>(base, d_desc, xbase, xoff, 0, nrhs, nrhs_dev, skip_dev);
    note_launch();
    GENEO_CUDA(cudaGetLastError());
    return GENEO_OK;
  } else {
    return band_solve_plain<T, A>(base, d_desc, count, max_w, xbase, xoff, nrhs, nrhs_dev, skip_dev, st, s, live);
  }
}

template <typename T>
geneo_status_t band_solve(const T* base, const BandDesc* d_desc, int count, int max_w,
                          double* xbase, const int64_t* xoff, int nrhs, const int32_t* nrhs_dev,
                          const int32_t* skip_dev, DevStatus* st, cudaStream_t s, int max_n, int tc_passes,
                          int res_stages, int active) {
  return band_solve_impl<T, T>(base, d_desc, count, max_w, xbase, xoff, nrhs, nrhs_dev, skip_dev, st, s, max_n,
                               tc_passes, res_stages, active);
}

geneo_status_t band_solve_ds(const double* base, const BandDesc* d_desc, int count, int max_w, double* xbase,
                             const int64_t* xoff, int nrhs, const int32_t* nrhs_dev, const int32_t* skip_dev,
                             DevStatus* st, cudaStream_t s, int max_n, int active) {
  return band_solve_impl<double, dsv>(base, d_desc, count, max_w, xbase, xoff, nrhs, nrhs_dev, skip_dev, st, s,
                                      max_n, 3, 0, active);
}

template geneo_status_t band_potrf<double>(double*, const BandDesc*, int, int, int, DevStatus*,
                                           cudaStream_t, bool, int32_t*, float, const Tc5Plan*);
template geneo_status_t band_potrf<float>(float*, const BandDesc*, int, int, int, DevStatus*,
                                          cudaStream_t, bool, int32_t*, float, const Tc5Plan*);
template geneo_status_t band_solve<double>(const double*, const BandDesc*, int, int, double*,
                                           const int64_t*, int, const int32_t*, const int32_t*,
                                           DevStatus*, cudaStream_t, int, int, int, int);
template geneo_status_t band_solve<float>(const float*, const BandDesc*, int, int, double*,
                                          const int64_t*, int, const int32_t*, const int32_t*,
                                          DevStatus*, cudaStream_t, int, int, int, int);

}  // namespace geneo
