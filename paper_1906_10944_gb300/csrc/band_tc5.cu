// Batched FP32 band Cholesky on the fifth-generation tensor cores: tcgen05
// MMAs with TMEM accumulators, fed by tensor-map bulk copies (TMA).
//
// The local matrices factored here are the shifted Neumann matrices
// K_j = Atilde_j - sigma B_j of the spectral transformation (Section 4.4) and
// the Dirichlet matrices A_j (Section 3), equilibrated to a unit diagonal
// (S A S); see band.cu for the band storage the solves use.
//
// Storage while factoring ("tiled band"): each matrix is cut into row blocks
// of 32 rows; row block I holds the dense 32 x (W + 32) rectangle of the
// columns [32 I - W, 32 I + 32), W = the batch's largest half bandwidth
// rounded up to 32, row-major.  Entries outside the band are zero and stay
// zero.  In this layout the columns [c - W, c) of any row block form a plain
// 2D box, so the panel update of a left-looking Cholesky is a sequence of
// boxed tiles.  Each value x is kept in two planes, hi = x with the low 13
// mantissa bits cleared (a TF32 value) and lo = x - hi (exact), so the
// three-pass TF32 product hi*hi + hi*lo + lo*hi, about FP32 accuracy, needs no
// splitting on chip.  The row blocks of a whole batch form one 3D tensor
// (x: W + 32 columns, y: 32 rows, z: row block) described by two tensor maps
// (hi, lo) with 128-byte swizzle, the layout the MMA descriptors read.
//
// Panel J (columns c0 = 32 J .. c0 + 31; rows [c0, c0 + R),
// R = min(n, c0 + 32 + w) - c0, in chunks h of 128 rows = four row blocks):
//   D_h = sum over k-chunks q of A_h(q) B(q)^T      (TMEM, M 128 x N 32)
// with A_h(q) = the chunk's rows at the columns c0 - W + 32 q .. + 31 (row
// block I: box x = 32 (J + q - I), negative x reads zeros) and B(q) = row
// block J at box x = 32 q.  Each tile is four K = 8 steps times three passes
// of tcgen05.mma kind::tf32.  Tiles whose row blocks all lie outside the
// band (4 h > q) are skipped.  Thread 0 issues the copies and thread 32 the
// MMAs through a ring of kStages stages (full / empty mbarriers;
// tcgen05.commit releases a stage and finally signals the accumulators).
// Then every thread reads its TMEM lane (tcgen05.ld), forms U = A - D in
// shared memory, one warp factors the 32 x 32 diagonal block in registers,
// the rows below are solved against it, and the panel's columns return to
// both planes (generic stores and a proxy fence before the next panel's
// copies read them).
//
// Every mbarrier wait is bounded; a wait that gives up records
// GENEO_ERR_TIMEOUT, raises a CTA-wide abort flag so the other roles stop
// waiting, and the kernel still drains the copies it issued, lets its MMAs
// finish and frees its TMEM before it exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "ptx.cuh"

namespace geneo {
namespace {

constexpr int kT5 = 256;                       // threads (8 warps)
constexpr int kPB5 = 32;                       // panel width = row block height
constexpr int kSt5 = 3;                        // pipeline stages
constexpr int kUS5 = kPB5 + 1;                 // row stride of the panel block in shared memory
constexpr uint32_t kBox5 = 32u * 32u * 4u;     // one 32 x 32 FP32 box (4 KB)
constexpr uint32_t kTileA5 = 4 * kBox5;        // 128 rows x 32 columns
constexpr uint32_t kTileB5 = kBox5;            // 32 rows x 32 columns
constexpr uint32_t kStage5 = 2 * kTileA5 + 2 * kTileB5;  // hi and lo of A and B: 40 KB
constexpr uint32_t kIdesc5 = umma_idesc_tf32(128, 32);

size_t tc5_smem(int W) {
  return 1024 + (size_t)kSt5 * kStage5 + (size_t)(kPB5 + W) * kUS5 * sizeof(float) + kPB5 * sizeof(float) +
         (2 * kSt5 + 2) * sizeof(uint64_t) + 16;
}

// Bounded wait that also gives up early once another role has aborted.
__device__ __forceinline__ bool wait5(uint64_t* bar, uint32_t parity, volatile int* abort, DevStatus* st,
                                      int id, int64_t where) {
  for (int it = 0; it < (1 << 22); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 1023) == 1023 && *abort) return false;
  }
  *abort = 1;
  record_error(st, GENEO_ERR_TIMEOUT, id, where);
  return false;
}

__device__ __forceinline__ bool finite_pos5(float v) { return v > 0.f && isfinite(v); }

__global__ void __launch_bounds__(kT5, 1)
k_band_potrf_tc5(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo,
                 float* __restrict__ phi, float* __restrict__ plo, const BandDesc* __restrict__ descs,
                 const int64_t* __restrict__ zoff, int W, uint32_t tmem_cols, DevStatus* st,
                 int32_t* __restrict__ weak, float weak_tol) {
  const BandDesc d = descs[blockIdx.x];
  const int n = d.n, w = d.w;
  const int64_t z0 = zoff[blockIdx.x];
  const int Wt = W + kPB5;
  const int QW = W / kPB5;  // k-chunks in a full window
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  unsigned char* base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  unsigned char* stages = base;
  float* Us = reinterpret_cast<float*>(base + kSt5 * kStage5);
  float* Dinv = Us + (size_t)(kPB5 + W) * kUS5;
  uint64_t* full = reinterpret_cast<uint64_t*>(Dinv + kPB5);
  uint64_t* empty = full + kSt5;
  uint64_t* accum = empty + kSt5;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(accum + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
  volatile uint32_t* inited_s = reinterpret_cast<volatile uint32_t*>(tslot + 2);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

  if (tid == 0) {
    for (int i = 0; i < kSt5; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(accum, 1);
    *abort = 0;
    *inited_s = 0;
    fence_barrier_init();
  }
  if (wid == 0) tmem_alloc(tslot, tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  uint32_t issued[kSt5] = {0, 0, 0};  // thread 0: copies issued into each stage
  uint32_t t_issue = 0;               // thread 0: tiles issued (all panels)
  uint32_t t_mma = 0;                 // thread 32: tiles consumed
  uint32_t n_commit = 0;              // thread 32: commits to `accum`
  uint32_t n_acc = 0;                 // all threads: accumulator phases waited

  for (int J = 0; J * kPB5 < n; ++J) {
    const int c0 = J * kPB5;
    const int b = min(kPB5, n - c0);
    const int R = min(n, c0 + kPB5 + w) - c0;
    const int nh = ((R + 31) / 32 + 3) / 4;   // 128-row chunks
    const int q0 = max(0, QW - J);            // first k-chunk with columns >= 0
    const bool any = q0 < QW;
    if (tid == 0 && any) {
      // ---- producer: tiles (q, h) for q in [q0, QW), h < min(nh, q / 4 + 1)
      for (int q = q0; q < QW; ++q) {
        const int hmax = min(nh, q / 4 + 1);
        for (int hh = 0; hh < hmax; ++hh) {
          const uint32_t s = t_issue % kSt5;
          bool go = !*abort;
          if (go && t_issue >= (uint32_t)kSt5)
            go = wait5(&empty[s], ((t_issue / kSt5) - 1) & 1, abort, st, d.id, c0);
          if (go) {
            unsigned char* sb = stages + s * kStage5;
            mbar_arrive_expect_tx(&full[s], kStage5);
            for (int i = 0; i < 4; ++i) {
              const int I = J + 4 * hh + i;
              const int x = 32 * (J + q - I);
              tma_load_3d(sb + i * kBox5, &tm_hi, x, 0, (int)(z0 + I), &full[s]);
              tma_load_3d(sb + kTileA5 + i * kBox5, &tm_lo, x, 0, (int)(z0 + I), &full[s]);
            }
            tma_load_3d(sb + 2 * kTileA5, &tm_hi, 32 * q, 0, (int)(z0 + J), &full[s]);
            tma_load_3d(sb + 2 * kTileA5 + kTileB5, &tm_lo, 32 * q, 0, (int)(z0 + J), &full[s]);
            ++issued[s];
          }
          ++t_issue;
        }
      }
    }
    if (tid == 32 && any) {
      // ---- MMA issuer
      uint32_t inited = 0;  // bit h: D_h written in this panel
      for (int q = q0; q < QW; ++q) {
        const int hmax = min(nh, q / 4 + 1);
        for (int hh = 0; hh < hmax; ++hh) {
          const uint32_t s = t_mma % kSt5;
          bool go = !*abort;
          if (go) go = wait5(&full[s], (t_mma / kSt5) & 1, abort, st, d.id, c0);
          if (go) {
            tc_fence_after();
            const uint32_t sa = smem_u32(stages + s * kStage5);
            const uint32_t dt = tmem + 32u * hh;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t ah = umma_desc_sw128(sa + 32 * kk);
              const uint64_t al = umma_desc_sw128(sa + kTileA5 + 32 * kk);
              const uint64_t bh = umma_desc_sw128(sa + 2 * kTileA5 + 32 * kk);
              const uint64_t bl = umma_desc_sw128(sa + 2 * kTileA5 + kTileB5 + 32 * kk);
              const uint32_t acc = ((inited >> hh) & 1u) | (kk > 0 ? 1u : 0u);
              umma_tf32(dt, al, bh, kIdesc5, acc);
              umma_tf32(dt, ah, bl, kIdesc5, 1u);
              umma_tf32(dt, ah, bh, kIdesc5, 1u);
            }
            inited |= 1u << hh;
            umma_commit(&empty[s]);
          }
          ++t_mma;
        }
      }
      *inited_s = inited;
      umma_commit(accum);  // arrives once every MMA issued so far has finished
      ++n_commit;
    }
    __syncthreads();
    uint32_t inited = 0;
    if (any) {
      wait5(accum, n_acc & 1, abort, st, d.id, c0);
      ++n_acc;
      tc_fence_after();
      inited = *inited_s;
    }
    // ---- U = A - D for the panel rows.  Warp w reads TMEM lanes
    // 32 (w % 4) .. + 31 of the chunks h = w / 4, w / 4 + 2, ...
    __syncwarp();
    for (int hh = wid >> 2; hh < nh; hh += 2) {
      const int row = 128 * hh + 32 * (wid & 3) + lane;
      float dv[32];
      if ((inited >> hh) & 1u) {
        tmem_ld32(tmem + ((uint32_t)(32 * (wid & 3)) << 16) + 32u * hh, dv);
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) dv[i] = 0.f;
      }
      if (row < R) {
        const int I = J + row / 32;
        const int64_t o = ((z0 + I) * 32 + (row & 31)) * (int64_t)Wt + (W - 32 * (I - J));
#pragma unroll
        for (int col = 0; col < 32; ++col) {
          float u = 0.f;
          if (col < b && col <= row && row - col <= w) u = (phi[o + col] + plo[o + col]) - dv[col];
          Us[(size_t)row * kUS5 + col] = u;
        }
      }
    }
    tc_fence_before();
    __syncthreads();
    // ---- the 32 x 32 diagonal block in warp 0: lane r holds row r; step t
    // takes pivot t from lane t (a pivot that is not positive is reported
    // and replaced by 1), scales column t and updates the trailing part
    if (wid == 0) {
      float a[kPB5];
#pragma unroll
      for (int u = 0; u < kPB5; ++u) a[u] = (lane < b && u <= lane) ? Us[lane * kUS5 + u] : 0.f;
#pragma unroll
      for (int t = 0; t < kPB5; ++t) {
        if (t < b) {
          float p = __shfl_sync(0xffffffffu, a[t], t);
          if (weak) {
            if (lane == 0 && !(p > weak_tol)) weak[d.id] = 1;
            if (!finite_pos5(p)) p = 1.f;
          } else if (!finite_pos5(p)) {
            if (lane == 0) record_error(st, isfinite(p) ? GENEO_ERR_NOT_SPD : GENEO_ERR_NONFINITE, d.id,
                                        (int64_t)c0 + t);
            p = 1.f;
          }
          const float inv = rsqrtf(p);
          if (lane == t) {
            a[t] = p * inv;
            Dinv[t] = inv;
          } else if (lane > t) {
            a[t] *= inv;
          }
#pragma unroll
          for (int u = t + 1; u < kPB5; ++u) {
            const float lut = __shfl_sync(0xffffffffu, a[t], u);
            if (lane >= u) a[u] -= a[t] * lut;
          }
        }
      }
      if (lane < b) {
#pragma unroll
        for (int u = 0; u < kPB5; ++u)
          if (u <= lane) Us[lane * kUS5 + u] = a[u];
      } else {
        Dinv[lane] = 0.f;
      }
    }
    __syncthreads();
    // ---- rows below: x L_JJ^T = u, one row per thread
    for (int i = b + tid; i < R; i += kT5) {
      float* ur = Us + (size_t)i * kUS5;
      float x[kPB5];
#pragma unroll
      for (int t = 0; t < kPB5; ++t) x[t] = ur[t];
#pragma unroll
      for (int t = 0; t < kPB5; ++t) {
        if (t < b) {
          float v = x[t];
#pragma unroll
          for (int u = 0; u < t; ++u) v -= x[u] * Us[t * kUS5 + u];
          x[t] = v * Dinv[t];
        }
      }
#pragma unroll
      for (int t = 0; t < kPB5; ++t) ur[t] = x[t];
    }
    __syncthreads();
    // ---- the panel's columns back to both planes (warp per row, coalesced)
    for (int i = wid; i < R; i += kT5 / 32) {
      const int r = c0 + i, c = c0 + lane;
      if (lane < b && c <= r && r - c <= w) {
        const int I = J + i / 32;
        const int64_t o = ((z0 + I) * 32 + (i & 31)) * (int64_t)Wt + (W - 32 * (I - J)) + lane;
        const float x = Us[(size_t)i * kUS5 + lane];
        const float xh = __uint_as_float(__float_as_uint(x) & 0xffffe000u);
        phi[o] = xh;
        plo[o] = x - xh;
      }
    }
    fence_proxy_async_global();  // the next panel's copies read these columns
    __syncthreads();
  }
  // ---- drain: the last phase of every stage's copies, and every MMA issued
  if (tid == 0)
    for (int s = 0; s < kSt5; ++s)
      if (issued[s] > 0)
        for (int it = 0; it < (1 << 22) && !mbar_try_wait(&full[s], (issued[s] - 1) & 1); ++it) {
        }
  if (tid == 32) {
    umma_commit(accum);
    const uint32_t ph = n_commit & 1;  // phase index n_commit completes with this commit
    for (int it = 0; it < (1 << 22) && !mbar_try_wait(accum, ph); ++it) {
    }
  }
  tc_fence_before();
  __syncthreads();
  if (wid == 0) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, tmem_cols);
  }
}

// band (skewed rows, BandDesc) -> tiled-band planes; one warp per row
__global__ void __launch_bounds__(256)
k_tb_pack(const float* __restrict__ band, const BandDesc* __restrict__ descs, const int64_t* __restrict__ zoff,
          int W, float* __restrict__ phi, float* __restrict__ plo) {
  const BandDesc d = descs[blockIdx.y];
  const int Wt = W + kPB5;
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < d.n; r += nw) {
    const int I = r / 32;
    const float* src = band + d.off + (int64_t)r * d.ld;
    float* dh = phi + ((zoff[blockIdx.y] + I) * 32 + (r & 31)) * (int64_t)Wt;
    float* dl = plo + ((zoff[blockIdx.y] + I) * 32 + (r & 31)) * (int64_t)Wt;
    for (int c = max(0, r - d.w) + lane; c <= r; c += 32) {
      const float x = src[c - r + d.w];
      const float xh = __uint_as_float(__float_as_uint(x) & 0xffffe000u);
      const int xx = c - 32 * I + W;
      dh[xx] = xh;
      dl[xx] = x - xh;
    }
  }
}

// tiled-band planes -> band: x = hi + lo on the band
__global__ void __launch_bounds__(256)
k_tb_unpack(float* __restrict__ band, const BandDesc* __restrict__ descs, const int64_t* __restrict__ zoff,
            int W, const float* __restrict__ phi, const float* __restrict__ plo) {
  const BandDesc d = descs[blockIdx.y];
  const int Wt = W + kPB5;
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < d.n; r += nw) {
    const int I = r / 32;
    float* dst = band + d.off + (int64_t)r * d.ld;
    const int64_t o = ((zoff[blockIdx.y] + I) * 32 + (r & 31)) * (int64_t)Wt;
    for (int c = max(0, r - d.w) + lane; c <= r; c += 32) {
      const int xx = c - 32 * I + W;
      dst[c - r + d.w] = phi[o + xx] + plo[o + xx];
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  return fn;
}

// 3D tensor map over the tiled-band planes: x = W + 32 columns, y = 32 rows,
// z = row blocks; 32 x 32 x 1 boxes, 128-byte swizzle, zeros out of range
bool encode_tb_map(CUtensorMap* m, float* base, int W, int64_t Z) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t Wt = (cuuint64_t)W + kPB5;
  const cuuint64_t dims[3] = {Wt, 32, (cuuint64_t)Z};
  const cuuint64_t strides[2] = {Wt * sizeof(float), Wt * 32 * sizeof(float)};
  const cuuint32_t box[3] = {32, 32, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

geneo_status_t tc5_prepare(const BandDesc* h_desc, int count, int max_w, DevMem& tmp, cudaStream_t s,
                           Tc5Plan* p) {
  p->ok = false;
  if (count <= 0) return GENEO_OK;
  const int W = (max_w + 31) & ~31;
  const size_t smem = tc5_smem(W);
  if (W < kPB5 || smem > 227 * 1024) return GENEO_OK;  // the older kernels take it
  const int nh = (kPB5 + W + 127) / 128;
  uint32_t cols = 32;
  while (cols < (uint32_t)(32 * nh)) cols <<= 1;
  if (cols > 512) return GENEO_OK;
  std::vector<int64_t> zo(count);
  int64_t Z = 0;
  int max_n = 0;
  for (int i = 0; i < count; ++i) {
    zo[i] = Z;
    Z += (h_desc[i].n + 31) / 32;
    max_n = std::max(max_n, h_desc[i].n);
  }
  if (Z <= 0 || Z > (int64_t)INT32_MAX) return GENEO_OK;
  const size_t plane = (size_t)Z * 32 * (W + kPB5);
  GENEO_TRY(tmp.get(&p->phi, plane));
  GENEO_TRY(tmp.get(&p->plo, plane));
  GENEO_TRY(tmp.get(&p->dz, (size_t)count));
  if (!encode_tb_map(&p->mhi, p->phi, W, Z) || !encode_tb_map(&p->mlo, p->plo, W, Z)) return GENEO_OK;
  GENEO_CUDA(cudaMemcpyAsync(p->dz, zo.data(), sizeof(int64_t) * count, cudaMemcpyHostToDevice, s));
  GENEO_CUDA(cudaMemsetAsync(p->phi, 0, sizeof(float) * plane, s));
  GENEO_CUDA(cudaMemsetAsync(p->plo, 0, sizeof(float) * plane, s));
  p->W = W;
  p->cols = cols;
  p->smem = smem;
  p->count = count;
  p->max_n = max_n;
  p->ok = true;
  return GENEO_OK;
}

geneo_status_t tc5_factor(const Tc5Plan& p, float* band, const BandDesc* d_desc, DevStatus* st, cudaStream_t s,
                          int32_t* weak, float weak_tol) {
  const dim3 gp((unsigned)std::min(64, (p.max_n + 7) / 8), (unsigned)p.count);
  k_tb_pack<<<gp, 256, 0, s>>>(band, d_desc, p.dz, p.W, p.phi, p.plo); note_launch();
  GENEO_CUDA(cudaGetLastError());
  GENEO_CUDA(allow_smem(k_band_potrf_tc5));
  k_band_potrf_tc5<<<p.count, kT5, p.smem, s>>>(p.mhi, p.mlo, p.phi, p.plo, d_desc, p.dz, p.W, p.cols, st,
                                                 weak, weak_tol);
  note_launch();
  GENEO_CUDA(cudaGetLastError());
  k_tb_unpack<<<gp, 256, 0, s>>>(band, d_desc, p.dz, p.W, p.phi, p.plo); note_launch();
  GENEO_CUDA(cudaGetLastError());
  return GENEO_OK;
}

}  // namespace geneo
