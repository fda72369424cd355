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
// boxed tiles.  Each value x is kept in two planes, hi and lo, both TF32
// (split_tf32_rn), so the three-pass TF32 product hi*hi + hi*lo + lo*hi
// (error at most 3 * 2^-22 of the product) needs no splitting on chip.  The row blocks of a whole batch form one 3D tensor
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
// band (4 h > q) are skipped.  The tensor cores add each MMA's products into
// the FP32 accumulator with truncation, a bias that grows with the number of
// MMAs summed into one accumulator; so every chunk has 1 + P accumulators:
// slot 0 takes the small terms (lo*hi + hi*lo), slot 1 + (q mod P) the
// hi*hi terms of k-chunk q, and the panel threads add the slots in FP32
// (small terms first).  Thread 0 issues the copies and thread 32 the
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

constexpr int kEpi5 = 256;                     // epilogue / panel threads (warps 0-7)
constexpr int kT5 = kEpi5 + 64;                // + copy warp 8 + MMA warp 9
constexpr int kPB5 = 32;                       // panel width = row block height
constexpr int kMaxStA5 = 4;                    // A-tile stages (4, or fewer for the widest bands)
constexpr int kStB5 = 2;                       // B-tile stages
constexpr int kUS5 = kPB5 + 1;                 // row stride of the panel block in shared memory
constexpr uint32_t kBox5 = 32u * 32u * 4u;     // one 32 x 32 FP32 box (4 KB)
constexpr uint32_t kTileA5 = 4 * kBox5;        // 128 rows x 32 columns
constexpr uint32_t kTileB5 = kBox5;            // 32 rows x 32 columns
constexpr uint32_t kStageA5 = 2 * kTileA5;     // hi and lo of an A tile: 32 KB
constexpr uint32_t kStageB5 = 2 * kTileB5;     // hi and lo of a B tile: 8 KB
constexpr uint32_t kIdesc5 = umma_idesc_tf32(128, 32);
constexpr int kMaxPar5 = 7;                    // at most this many hi*hi accumulators per chunk
// afull, aempty, bfull, bempty, acc_full[2], acc_empty[2], pdone, fin
constexpr int bars5(int sta) { return 2 * sta + 2 * kStB5 + 2 + 2 + 2; }

size_t tc5_smem(int W, int sta) {
  return 1024 + (size_t)sta * kStageA5 + (size_t)kStB5 * kStageB5 + (size_t)(kPB5 + W) * kUS5 * sizeof(float) +
         2 * kPB5 * sizeof(float) + bars5(sta) * sizeof(uint64_t) + 16;
}
// the most A stages (4, 3, 2) whose shared memory fits a class of width W;
// 0 when none does
int tc5_stages(int W) {
  for (int sta = kMaxStA5; sta >= 2; --sta)
    if (tc5_smem(W, sta) <= 227 * 1024) return sta;
  return 0;
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

__device__ __forceinline__ void arrive5(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// barrier among the 256 panel threads only (the copy and MMA warps run on)
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

__device__ __forceinline__ bool finite_pos5(float v) { return v > 0.f && isfinite(v); }

// x into the two planes: hi = x rounded to TF32, lo = x - hi rounded to
// TF32 (split_tf32_rn); with bf16 = 1 the value is first rounded to BF16 (to nearest, ties
// to even, by integer arithmetic on the bit pattern), which a TF32 plane
// holds exactly, and lo is 0 (the factor then holds BF16 values)
__device__ __forceinline__ void split5(float x, int bf16, float& h, float& l) {
  if (bf16) {
    uint32_t u = __float_as_uint(x);
    if (isfinite(x)) u = (u + 0x7fffu + ((u >> 16) & 1u)) & 0xffff0000u;
    h = __uint_as_float(u);
    l = 0.f;
  } else {
    split_tf32_rn(x, h, l);
  }
}

// Warp-specialised: warp 8 (one lane) streams the tiles of panel after
// panel, warp 9 (one lane) issues the MMAs into one of nbuf (1 or 2) TMEM
// accumulator buffers (panel G uses buffer G % nbuf), and warps 0-7 run the panel
// steps.  A tiles go through a ring of kStA5 stages (4, or 3 or 2 for the
// widest classes, whose panel block takes the room), the B tile of each
// k-chunk (shared by the chunk's row tiles) through a ring of kStB5.  The
// tiles of panel J + 1 that do not read panel J's columns (all k-chunks but
// the last) are loaded and multiplied while panel J is being factored; the
// last k-chunk waits for panel J's write-back (pdone).  Barriers: afull /
// aempty and bfull / bempty (stage rings), acc_full[b] (MMA -> panel
// threads), acc_empty[b] (panel threads -> MMA: buffer b read), pdone
// (panel written).
template <int kStA5>
__global__ void __launch_bounds__(kT5, 1)
k_band_potrf_tc5(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo,
                 float* __restrict__ phi, float* __restrict__ plo, const BandDesc* __restrict__ descs,
                 const int64_t* __restrict__ zoff, int count, int32_t* __restrict__ queue, int W,
                 uint32_t tmem_cols, int nbuf, int P, DevStatus* st, int32_t* __restrict__ weak, float weak_tol,
                 int bf16) {
  const int Wt = W + kPB5;
  const int QW = W / kPB5;                    // k-chunks in a full window
  const uint32_t bufcols = tmem_cols / nbuf;  // columns of one accumulator buffer
  const uint32_t chcols = 32u * (1 + P);      // columns of one chunk's accumulators
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  unsigned char* base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  unsigned char* stA = base;
  unsigned char* stB = base + kStA5 * kStageA5;
  float* Us = reinterpret_cast<float*>(stB + kStB5 * kStageB5);
  float* Dinv = Us + (size_t)(kPB5 + W) * kUS5;
  uint64_t* afull = reinterpret_cast<uint64_t*>(Dinv + 2 * kPB5);
  uint64_t* aempty = afull + kStA5;
  uint64_t* bfull = aempty + kStA5;
  uint64_t* bempty = bfull + kStB5;
  uint64_t* acc_full = bempty + kStB5;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* pdone = acc_empty + 2;
  uint64_t* fin = pdone + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(fin + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
  volatile int* item_s = reinterpret_cast<volatile int*>(tslot + 2);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

  if (tid == 0) {
    for (int i = 0; i < kStA5; ++i) {
      mbar_init(&afull[i], 1);
      mbar_init(&aempty[i], 1);
    }
    for (int i = 0; i < kStB5; ++i) {
      mbar_init(&bfull[i], 1);
      mbar_init(&bempty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], kEpi5);
    }
    mbar_init(pdone, kEpi5);
    mbar_init(fin, 1);
    *abort = 0;
    fence_barrier_init();
  }
  if (wid == 9) tmem_alloc(tslot, tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  // role state carried over the matrices this CTA takes from the queue
  uint32_t issA[kStA5], issB[kStB5] = {0, 0};  // copy lane: arms per stage
#pragma unroll
  for (int i = 0; i < kStA5; ++i) issA[i] = 0;
  uint32_t ta = 0, tb = 0;  // copy and MMA lanes: A tiles and B tiles so far
  int pb = 0;               // panels of the earlier matrices (barrier phases run on)
  for (;;) {
    // work queue: the next matrix in batch order (largest first)
    if (tid == 0) *item_s = atomicAdd(queue, 1);
    __syncthreads();
    const int item = *item_s;
    __syncthreads();
    if (item >= count) break;
    const BandDesc d = descs[item];
    const int n = d.n, w = d.w;
    const int64_t z0 = zoff[item];
    const int np = (n + kPB5 - 1) / kPB5;  // panels
    if (wid == 8) {
      // ------------------------------------------------------------ copies
      if (lane == 0) {
        for (int J = 0; J < np; ++J) {
          const int c0 = J * kPB5;
          const int R = min(n, c0 + kPB5 + w) - c0;
          const int nh = ((R + 31) / 32 + 3) / 4;
          const int q0 = max(0, QW - J);
          for (int q = q0; q < QW; ++q, ++tb) {
            // the last k-chunk holds panel J - 1's columns
            if (q == QW - 1 && J >= 1 && !*abort) wait5(pdone, (pb + J - 1) & 1, abort, st, d.id, c0);
            {
              const uint32_t sb = tb % kStB5;
              if (!*abort && (tb < (uint32_t)kStB5 || wait5(&bempty[sb], ((tb / kStB5) - 1) & 1, abort, st, d.id, c0))) {
                unsigned char* dst = stB + sb * kStageB5;
                mbar_arrive_expect_tx(&bfull[sb], kStageB5);
                tma_load_3d(dst, &tm_hi, 32 * q, 0, (int)(z0 + J), &bfull[sb]);
                tma_load_3d(dst + kTileB5, &tm_lo, 32 * q, 0, (int)(z0 + J), &bfull[sb]);
                ++issB[sb];
              }
            }
            const int hmax = min(nh, q / 4 + 1);
            for (int hh = 0; hh < hmax; ++hh, ++ta) {
              const uint32_t sa = ta % kStA5;
              if (*abort) continue;
              if (ta >= (uint32_t)kStA5 && !wait5(&aempty[sa], ((ta / kStA5) - 1) & 1, abort, st, d.id, c0)) continue;
              unsigned char* dst = stA + sa * kStageA5;
              mbar_arrive_expect_tx(&afull[sa], kStageA5);
              for (int i = 0; i < 4; ++i) {
                const int I = J + 4 * hh + i;
                const int x = 32 * (J + q - I);
                tma_load_3d(dst + i * kBox5, &tm_hi, x, 0, (int)(z0 + I), &afull[sa]);
                tma_load_3d(dst + kTileA5 + i * kBox5, &tm_lo, x, 0, (int)(z0 + I), &afull[sa]);
              }
              ++issA[sa];
            }
          }
        }
      }
    } else if (wid == 9) {
      // ------------------------------------------------------------ MMAs
      if (lane == 0) {
        for (int J = 0; J < np; ++J) {
          const int c0 = J * kPB5;
          const int R = min(n, c0 + kPB5 + w) - c0;
          const int nh = ((R + 31) / 32 + 3) / 4;
          const int q0 = max(0, QW - J);
          const int G = pb + J;  // panel index over this CTA's matrices
          const int b = G % nbuf;
          if (G >= nbuf && !*abort) wait5(&acc_empty[b], ((G / nbuf) - 1) & 1, abort, st, d.id, c0);
          tc_fence_after();
          const uint32_t dbuf = tmem + (uint32_t)b * bufcols;
          uint64_t inited = 0;  // bit (1 + P) hh + slot: accumulator written
          for (int q = q0; q < QW; ++q, ++tb) {
            const uint32_t sb = tb % kStB5;
            const bool bok = !*abort && wait5(&bfull[sb], (tb / kStB5) & 1, abort, st, d.id, c0);
            const uint32_t bsa = smem_u32(stB + sb * kStageB5);
            const int hmax = min(nh, q / 4 + 1);
            for (int hh = 0; hh < hmax; ++hh, ++ta) {
              const uint32_t sa = ta % kStA5;
              if (!bok || *abort || !wait5(&afull[sa], (ta / kStA5) & 1, abort, st, d.id, c0)) continue;
              tc_fence_after();
              const uint32_t asa = smem_u32(stA + sa * kStageA5);
              const int ss = 1 + q % P;  // the hi*hi slot of this k-chunk
              const int bs = (1 + P) * hh, bb = bs + ss;
              const uint32_t ds = dbuf + chcols * hh, db = ds + 32u * ss;
              const uint32_t acs = (uint32_t)((inited >> bs) & 1u), acb = (uint32_t)((inited >> bb) & 1u);
  #pragma unroll
              for (int kk = 0; kk < 4; ++kk) {
                const uint64_t ah = umma_desc_sw128(asa + 32 * kk);
                const uint64_t al = umma_desc_sw128(asa + kTileA5 + 32 * kk);
                const uint64_t bh = umma_desc_sw128(bsa + 32 * kk);
                const uint64_t bl = umma_desc_sw128(bsa + kTileB5 + 32 * kk);
                umma_tf32(ds, al, bh, kIdesc5, acs | (kk > 0 ? 1u : 0u));
                umma_tf32(ds, ah, bl, kIdesc5, 1u);
                umma_tf32(db, ah, bh, kIdesc5, acb | (kk > 0 ? 1u : 0u));
              }
              inited |= (1ull << bs) | (1ull << bb);
              umma_commit(&aempty[sa]);
            }
            if (bok) umma_commit(&bempty[sb]);  // the k-chunk's row tiles are all issued
          }
          umma_commit(&acc_full[b]);  // every MMA of this panel has finished
        }
      }
    } else {
      // ------------------------------------------------------------ panels
      for (int J = 0; J < np; ++J) {
        const int c0 = J * kPB5;
        const int b = min(kPB5, n - c0);
        const int R = min(n, c0 + kPB5 + w) - c0;
        const int nh = ((R + 31) / 32 + 3) / 4;
        const int q0 = max(0, QW - J);
        const int G = pb + J;
        const int buf = G % nbuf;
        // the panel's entries of A (both planes) into Us: eight lanes per row,
        // four columns each (16-byte loads), four row groups of 32 rows per
        // batch in flight; entries outside the band are zero in the planes
        {
          const int rsub = lane >> 3, cg = 4 * (lane & 7);
          for (int i0 = 4 * wid + rsub; i0 < R; i0 += 4 * kEpi5 / 8) {
            float4 vh[4], vl[4];
  #pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int i = i0 + u * (kEpi5 / 8);
              vh[u] = make_float4(0.f, 0.f, 0.f, 0.f);
              vl[u] = vh[u];
              if (i < R) {
                const int I = J + i / 32;
                const int64_t o = ((z0 + I) * 32 + (i & 31)) * (int64_t)Wt + (W - 32 * (I - J)) + cg;
                vh[u] = *reinterpret_cast<const float4*>(phi + o);
                vl[u] = *reinterpret_cast<const float4*>(plo + o);
              }
            }
  #pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int i = i0 + u * (kEpi5 / 8);
              if (i < R) {
                float* ur = Us + (size_t)i * kUS5 + cg;
                ur[0] = vh[u].x + vl[u].x;
                ur[1] = vh[u].y + vl[u].y;
                ur[2] = vh[u].z + vl[u].z;
                ur[3] = vh[u].w + vl[u].w;
              }
            }
          }
        }
        if (!*abort) wait5(&acc_full[buf], (G / nbuf) & 1, abort, st, d.id, c0);
        tc_fence_after();
        epi_sync();
        // U = A - D.  Warp w reads TMEM lanes 32 (w % 4) .. + 31 of the
        // chunks h = w / 4, w / 4 + 2, ...; chunk h holds data when one of its
        // tiles was multiplied (some k-chunk q >= 4 h exists), and its hi*hi
        // slot 1 + r when one of those q has q mod P = r.  D = small terms +
        // the hi*hi slots, summed in FP32.
        __syncwarp();
        for (int hh = wid >> 2; hh < nh; hh += 2) {
          const int qlo = max(q0, 4 * hh);
          if (qlo >= QW) continue;
          const uint32_t ta0 = tmem + (uint32_t)buf * bufcols + ((uint32_t)(32 * (wid & 3)) << 16) + chcols * hh;
          float dv[32], dt[32];
          tmem_ld32(ta0, dv);
          for (int r = 0; r < P; ++r) {
            if (qlo + ((r - qlo % P) + P) % P >= QW) continue;  // no k-chunk of this parity
            tmem_ld32(ta0 + 32u * (1 + r), dt);
  #pragma unroll
            for (int col = 0; col < 32; ++col) dv[col] += dt[col];
          }
          const int row = 128 * hh + 32 * (wid & 3) + lane;
          if (row < R) {
            float* ur = Us + (size_t)row * kUS5;
  #pragma unroll
            for (int col = 0; col < 32; ++col)
              if (col < b && col <= row && row - col <= w) ur[col] -= dv[col];
          }
        }
        tc_fence_before();
        arrive5(&acc_empty[buf]);  // the MMAs may refill this buffer
        epi_sync();
        // ---- the 32 x 32 diagonal block in warp 0: lane r holds row r; step t
        // takes pivot t from lane t (a pivot that is not positive is reported
        // and replaced by 1), scales column t and updates the trailing part
        if (wid == 0) {
          // lane r holds row r; step t publishes the scaled column t in Dcol
          // (shared memory) and every lane updates its row from it
          float* Dcol = Dinv + kPB5;  // kPB5 scratch values after Dinv
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
              Dcol[lane] = a[t];
              __syncwarp();
  #pragma unroll
              for (int u = t + 1; u < kPB5; ++u)
                if (lane >= u) a[u] -= a[t] * Dcol[u];
              __syncwarp();
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
        epi_sync();
        // ---- rows below: x L_JJ^T = u, one row per thread
        for (int i = b + tid; i < R; i += kEpi5) {
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
        epi_sync();
        // ---- the panel's columns back to both planes: eight lanes per row,
        // 16-byte stores.  Us holds exact zeros outside the band (A is zero
        // there and every update of such an entry is 0 - 0), which is also
        // what the planes hold there.
        {
          const int rsub = lane >> 3, cg = 4 * (lane & 7);
          for (int i = 4 * wid + rsub; i < R; i += kEpi5 / 8) {
            const int I = J + i / 32;
            const int64_t o = ((z0 + I) * 32 + (i & 31)) * (int64_t)Wt + (W - 32 * (I - J)) + cg;
            const float* ur = Us + (size_t)i * kUS5 + cg;
            float4 xh, xl;
            split5(ur[0], bf16, xh.x, xl.x);
            split5(ur[1], bf16, xh.y, xl.y);
            split5(ur[2], bf16, xh.z, xl.z);
            split5(ur[3], bf16, xh.w, xl.w);
            *reinterpret_cast<float4*>(phi + o) = xh;
            *reinterpret_cast<float4*>(plo + o) = xl;
          }
        }
        fence_proxy_async_global();  // the next panel's copies read these columns
        arrive5(pdone);
        epi_sync();                  // Us is refilled by the next panel
      }
    }
    pb += np;
  }
  // drain: the last phase of every stage's copies, and every MMA issued
  if (tid == 8 * 32) {
    for (int i = 0; i < kStA5; ++i)
      if (issA[i] > 0)
        for (int it = 0; it < (1 << 22) && !mbar_try_wait(&afull[i], (issA[i] - 1) & 1); ++it) {
        }
    for (int i = 0; i < kStB5; ++i)
      if (issB[i] > 0)
        for (int it = 0; it < (1 << 22) && !mbar_try_wait(&bfull[i], (issB[i] - 1) & 1); ++it) {
        }
  }
  if (tid == 9 * 32) {
    umma_commit(fin);
    for (int it = 0; it < (1 << 22) && !mbar_try_wait(fin, 0); ++it) {
    }
  }
  tc_fence_before();
  __syncthreads();
  if (wid == 9) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, tmem_cols);
  }
}

// band (skewed rows, BandDesc) -> tiled-band planes, every entry of every
// row block (zeros outside the band and beyond n), one warp per row.  With
// a row scaling (d.scl >= 0) the planes receive s_r s_c a_rc, the
// equilibrated matrix S A S.
__global__ void __launch_bounds__(256)
k_tb_pack(const float* __restrict__ band, const BandDesc* __restrict__ descs, const int64_t* __restrict__ zoff,
          int W, float* __restrict__ phi, float* __restrict__ plo, int bf16) {
  const BandDesc d = descs[blockIdx.y];
  const int Wt = W + kPB5;
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const float* S = d.scl >= 0 ? band + d.scl : nullptr;
  const int rows = (d.n + 31) & ~31;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < rows; r += nw) {
    const int I = r / 32;
    const float* src = band + d.off + (int64_t)r * d.ld;
    const int64_t o = ((zoff[blockIdx.y] + I) * 32 + (r & 31)) * (int64_t)Wt;
    const float sr = (S && r < d.n) ? S[r] : 1.f;
    for (int xx = lane; xx < Wt; xx += 32) {
      const int c = xx + 32 * I - W;
      float x = 0.f;
      if (r < d.n && c >= 0 && c <= r && r - c <= d.w) {
        x = src[c - r + d.w];
        if (S) x *= sr * S[c];
      }
      float xh, xl;
      split5(x, bf16, xh, xl);
      phi[o + xx] = xh;
      plo[o + xx] = xl;
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

// TMEM layout of the accumulators for nh 128-row chunks: two buffers when
// each buffer can hold at least one hi*hi slot next to the small-term slot,
// else one; then as many hi*hi slots per chunk (P <= kMaxPar5) as the 512
// columns allow.  False when not even one buffer with P = 1 fits.
bool tc5_acc_layout(int nh, int* nbuf, int* P) {
  for (int nb = 2; nb >= 1; --nb) {
    const int slots = 512 / (nb * 32 * nh);  // 1 + P
    if (slots >= 2) {
      *nbuf = nb;
      *P = std::min(kMaxPar5, slots - 1);
      return true;
    }
  }
  return false;
}

bool tc5_fits(int w) {
  const int W = (w + 31) & ~31;
  const int nh = (kPB5 + W + 127) / 128;
  int nb = 0, P = 0;
  return W >= kPB5 && tc5_stages(W) > 0 && tc5_acc_layout(nh, &nb, &P);
}

geneo_status_t tc5_prepare(const BandDesc* h_desc, int count, int max_w, DevMem& tmp, cudaStream_t s,
                           Tc5Plan* p) {
  p->ok = false;
  if (count <= 0) return GENEO_OK;
  const int W = (max_w + 31) & ~31;
  const int sta = tc5_stages(W);
  if (W < kPB5 || sta == 0) return GENEO_OK;  // the older kernels take it
  const size_t smem = tc5_smem(W, sta);
  const int nh = (kPB5 + W + 127) / 128;
  int nbuf = 0, P = 0;
  if (!tc5_acc_layout(nh, &nbuf, &P)) return GENEO_OK;
  uint32_t cols = 32;
  while (cols < (uint32_t)(nbuf * 32 * nh * (1 + P))) cols <<= 1;
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
  GENEO_TRY(tmp.get(&p->queue, 1));
  if (!encode_tb_map(&p->mhi, p->phi, W, Z) || !encode_tb_map(&p->mlo, p->plo, W, Z)) return GENEO_OK;
  GENEO_CUDA(cudaMemcpyAsync(p->dz, zo.data(), sizeof(int64_t) * count, cudaMemcpyHostToDevice, s));
  p->W = W;
  p->cols = cols;
  p->nbuf = nbuf;
  p->par = P;
  p->smem = smem;
  p->sta = sta;
  p->count = count;
  p->max_n = max_n;
  p->ok = true;
  return GENEO_OK;
}

geneo_status_t tc5_factor(const Tc5Plan& p, float* band, const BandDesc* d_desc, DevStatus* st, cudaStream_t s,
                          int32_t* weak, float weak_tol) {
  const int bf16 = p.bf16 ? 1 : 0;
  const dim3 gp((unsigned)std::min(64, (p.max_n + 7) / 8), (unsigned)p.count);
  k_tb_pack<<<gp, 256, 0, s>>>(band, d_desc, p.dz, p.W, p.phi, p.plo, bf16); note_launch();
  GENEO_CUDA(cudaGetLastError());
  auto kern = p.sta == 4 ? k_band_potrf_tc5<4> : p.sta == 3 ? k_band_potrf_tc5<3> : k_band_potrf_tc5<2>;
  GENEO_CUDA(allow_smem(kern));
  // persistent CTAs, one per SM (the shared memory allows no more), taking
  // matrices from the queue in batch order
  int dev = 0, sms = 0;
  GENEO_CUDA(cudaGetDevice(&dev));
  GENEO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  GENEO_CUDA(cudaMemsetAsync(p.queue, 0, sizeof(int32_t), s));
  kern<<<std::min(p.count, sms), kT5, p.smem, s>>>(p.mhi, p.mlo, p.phi, p.plo, d_desc, p.dz, p.count, p.queue, p.W,
                                                    p.cols, p.nbuf, p.par, st, weak, weak_tol, bf16);
  note_launch();
  GENEO_CUDA(cudaGetLastError());
  k_tb_unpack<<<gp, 256, 0, s>>>(band, d_desc, p.dz, p.W, p.phi, p.plo); note_launch();
  GENEO_CUDA(cudaGetLastError());
  return GENEO_OK;
}

}  // namespace geneo
