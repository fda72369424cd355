// Internal declarations shared by the translation units of libgeneo.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>
#include <vector>

#include "geneo.h"

namespace geneo {

// --------------------------------------------------------------------------
// Status handling.  Device code records the first error it meets in a small
// status block (code, where, index); host code returns geneo_status_t.
// --------------------------------------------------------------------------
struct DevStatus {
  int32_t code;    // geneo_status_t, 0 = OK
  int32_t where;   // subdomain / matrix id
  int64_t index;   // row, iteration or other index
};

__device__ __forceinline__ void record_error(DevStatus* st, int code, int where, int64_t index) {
  if (atomicCAS(&st->code, 0, code) == 0) {
    st->where = where;
    st->index = index;
  }
}

#define GENEO_CUDA(call)                                \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) {                            \
      geneo::set_cuda_error(e_, #call, __FILE__, __LINE__); \
      return GENEO_ERR_CUDA;                            \
    }                                                   \
  } while (0)

#define GENEO_TRY(expr)                      \
  do {                                       \
    geneo_status_t s_ = (expr);              \
    if (s_ != GENEO_OK) return s_;           \
  } while (0)

void set_cuda_error(cudaError_t e, const char* what, const char* file, int line);
// process-wide count of kernel launches made by this library
void note_launch();
int64_t launch_count();

// Accumulates CUDA-event time of selected launches on one stream.
struct EventTimer {
  cudaEvent_t a = nullptr, b = nullptr;
  double ms = 0.0;
  cudaStream_t s = 0;
  void start(cudaStream_t st) {
    s = st;
    if (!a) { cudaEventCreate(&a); cudaEventCreate(&b); }
    cudaEventRecord(a, s);
  }
  void stop() {
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float t = 0.f;
    cudaEventElapsedTime(&t, a, b);
    ms += t;
  }
  ~EventTimer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};
const std::string& last_cuda_error();

// Opt-in per-family timing: event pairs recorded around launches, summed
// when the owner synchronises (no synchronisation per launch).
struct KernelProfiler {
  struct Rec { int fam; cudaEvent_t a, b; double flops, bytes; };
  bool on = false;
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  double ms[GENEO_PROF_COUNT] = {0}, flops[GENEO_PROF_COUNT] = {0}, bytes[GENEO_PROF_COUNT] = {0};
  int64_t launches[GENEO_PROF_COUNT] = {0};
  cudaEvent_t get() {
    if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  // returns the index of the open record or -1
  int begin(int fam, double fl, double by, cudaStream_t s) {
    if (!on) return -1;
    Rec r{fam, get(), get(), fl, by};
    cudaEventRecord(r.a, s);
    pending.push_back(r);
    return (int)pending.size() - 1;
  }
  void end(int idx, cudaStream_t s) {
    if (idx < 0) return;
    cudaEventRecord(pending[idx].b, s);
  }
  void collect() {
    for (Rec& r : pending) {
      cudaEventSynchronize(r.b);
      float t = 0.f;
      cudaEventElapsedTime(&t, r.a, r.b);
      ms[r.fam] += t;
      flops[r.fam] += r.flops;
      bytes[r.fam] += r.bytes;
      launches[r.fam] += 1;
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    pending.clear();
  }
  ~KernelProfiler() {
    for (Rec& r : pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

// --------------------------------------------------------------------------
// Per-subdomain descriptor (device and host copies).
// --------------------------------------------------------------------------
struct SubDesc {
  int64_t offN;    // offset of subdomain rows in N-indexed arrays
  int64_t offE;    // offset into sub_elem
  int64_t bandA;   // element offset of the Dirichlet band factor
  int64_t bandK;   // element offset of the shifted Neumann band factor
  int64_t offZ;    // element offset of Z_j (nD x m, column-major)
  int64_t offY;    // element offset of Y_j = A Z_j (nN x m, column-major)
  int32_t nN, nD, nE;
  int32_t wA, wK;  // half bandwidths
  int32_t s;       // eigensolver block width actually used
  int32_t m;       // coarse vectors taken
  int32_t offH;    // first coarse index of this subdomain
};

// Band matrix descriptor for the batched Cholesky / triangular solves.
// Lower band stored by rows: entry (r, c), 0 <= r - c <= w, at
// base[r * ld + (c - r + w)]; ld = w + 1 rounded up to a multiple of 4, so
// every row (and every block of rows) starts on a 16-byte boundary (32 for
// FP64) and can be moved by one bulk copy.  Slots with c < 0 are zero.
// Beside the band, the factorisation stores the inverses of the 16 x 16
// diagonal blocks of L (block b: rows and columns 16 b .. 16 b + 15; entry
// (i, t) at dinv + 256 b + 16 i + t, zero outside the lower triangle and
// beyond n), which the solves apply instead of substituting.
struct BandDesc {
  int64_t off;     // element offset of the band (a multiple of 4)
  int32_t n, w;
  int32_t id;      // reported in errors; the solves index vectors, counts and
                   // skip flags by id when it is >= 0 (subdomain index), by
                   // the position in the batch otherwise
  int32_t ld;      // row stride
  int64_t dinv;    // element offset of the inverted diagonal blocks
  int64_t scl;     // element offset of the row scaling s = diag^{-1/2} of an
                   // equilibrated band (the factor is that of S A S), or -1
};

__host__ __device__ __forceinline__ int band_ld(int w) { return (w + 4) & ~3; }
// elements of the inverted diagonal blocks of an order-n band
__host__ __device__ __forceinline__ int64_t dinv_elems(int n) { return (int64_t)((n + 15) / 16) * 256; }
// elements of the row scaling of an order-n band (a multiple of 4)
__host__ __device__ __forceinline__ int64_t scl_elems(int n) { return (int64_t)((n + 3) & ~3); }

// --------------------------------------------------------------------------
// Device helpers.
// --------------------------------------------------------------------------
__device__ __forceinline__ int lower_bound_i32(const int32_t* a, int n, int32_t key) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// index of key in sorted a[0..n) or -1
__device__ __forceinline__ int find_i32(const int32_t* a, int n, int32_t key) {
  int p = lower_bound_i32(a, n, key);
  return (p < n && a[p] == key) ? p : -1;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum (deterministic: fixed tree).  `red` needs blockDim/32 slots.
template <typename T>
__device__ T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T t = (threadIdx.x < nw) ? red[threadIdx.x] : T(0);
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  T r = red[0];
  __syncthreads();
  return r;
}

// x = hi + lo for three-pass TF32 tensor-core products: hi = x rounded to
// TF32 (10 explicit mantissa bits, to nearest), lo = x - hi (exact in FP32)
// rounded to TF32 too, so both are exact MMA operands.  hi*y_hi + hi*y_lo +
// lo*y_hi then differs from x*y by the dropped lo*y_lo and the two roundings
// of lo: at most 3 * 2^-22 |x y|, of either sign (no bias from truncation).
__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
__device__ __forceinline__ void split_tf32_rn(float x, float& hi, float& lo) {
  hi = tf32_rn(x);
  lo = tf32_rn(x - hi);
}
// A matrix factored with those products is sent to FP64 when a pivot is at
// or below this multiple of the FP32 pivot tolerance: the tolerance stands
// for (condition) x (unit roundoff), and the product error bound above is
// 12 times an FP32 FMA's 2^-24.
constexpr float kTf32PivotScale = 12.f;

// SplitMix64 (Steele, Lea, Flood 2014): counter -> 64 random bits.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Algorithmic work of the banded kernels for an n x n band of half width w:
// column c has h_c = min(w, n-1-c) entries below the diagonal.
// Cholesky: 1 sqrt, h_c divisions, h_c (h_c + 1)/2 fused multiply-adds of
// the trailing update -> sum_c (h_c + 1)^2 flops.
inline double band_factor_flops(double n, double w) {
  if (n <= 0) return 0.0;
  if (w >= n) w = n - 1;
  return (n - w) * (w + 1) * (w + 1) + w * (w + 1) * (2 * w + 1) / 6.0;
}
// Forward plus backward substitution, one right-hand side: 2 sum_c (2 h_c + 1).
inline double band_solve_flops(double n, double w) {
  if (n <= 0) return 0.0;
  if (w >= n) w = n - 1;
  const double sum_h = (n - w) * w + w * (w - 1) / 2.0;
  return 2.0 * (2.0 * sum_h + n);
}
// Stored entries of the band, sum_c (h_c + 1).
inline double band_entries(double n, double w) {
  if (n <= 0) return 0.0;
  if (w >= n) w = n - 1;
  return (n - w) * (w + 1) + w * (w + 1) / 2.0;
}

// --------------------------------------------------------------------------
// Simple owning device buffer.
// --------------------------------------------------------------------------
// Device allocations from the stream-ordered pool: allocated and freed in
// the order of `stream` (set by the owner before use), so a free does not
// synchronise the device and concurrent handles on other streams keep
// running; the pool keeps freed memory for the next allocation.
struct DevMem {
  std::vector<void*> ptrs;
  int64_t bytes = 0;
  cudaStream_t stream = nullptr;
  geneo_status_t alloc(void** p, size_t n);
  template <typename T>
  geneo_status_t get(T** p, size_t count) {
    return alloc(reinterpret_cast<void**>(p), count * sizeof(T));
  }
  void release(void* p);
  void free_all();
};

// Allow a kernel all the dynamic shared memory the device can give it (the
// opt-in maximum less its static shared memory).  The limit belongs to the
// kernel and is shared by every host thread, so it is not set to one
// launch's size, which would race with concurrent launches of other sizes on
// other streams; each launch still requests only what it uses.
template <typename K>
inline cudaError_t allow_smem(K kern) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, kern);
  if (e != cudaSuccess) return e;
  int dev = 0, v = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, v - (int)a.sharedSizeBytes);
}

// --------------------------------------------------------------------------
// Kernel launchers implemented in the .cu files.
// --------------------------------------------------------------------------
// scan.cu: exclusive prefix sum of n int64 (out may alias in); returns total.
geneo_status_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total,
                                  DevMem& tmp, cudaStream_t st);

// band_tc5.cu: FP32 band Cholesky on the fifth-generation tensor cores.
// tc5_prepare allocates the tiled-band planes of a batch (host descriptors in
// batch order) and their tensor maps on stream s; p->ok stays false when the
// batch does not fit the kernel (the older kernels then factor it).
// tc5_factor (after equilibration) packs the bands, factors them and unpacks
// the factors back into the bands.
struct Tc5Plan {
  CUtensorMap mhi, mlo;
  bool ok = false;
  int W = 0, count = 0, max_n = 0;
  uint32_t cols = 0;  // TMEM columns allocated
  int nbuf = 0;       // accumulator buffers (panels in flight)
  int sta = 4;        // A-tile stages of the kernel
  int par = 0;        // hi*hi accumulators per 128-row chunk
  size_t smem = 0;
  float* phi = nullptr;
  float* plo = nullptr;
  int64_t* dz = nullptr;
  int32_t* queue = nullptr;  // work counter of the persistent launch
  bool bf16 = false;         // factor values rounded to BF16 (precision study)
};
geneo_status_t tc5_prepare(const BandDesc* h_desc, int count, int max_w, DevMem& tmp, cudaStream_t s,
                           Tc5Plan* p);
// whether a band of half bandwidth w fits the kernel (shared memory, TMEM)
bool tc5_fits(int w);
geneo_status_t tc5_factor(const Tc5Plan& p, float* band, const BandDesc* d_desc, DevStatus* st, cudaStream_t s,
                          int32_t* weak, float weak_tol);

// band.cu
// Batched Cholesky.  equil: factor S A S (s = diag^{-1/2}) and keep s.
// weak (may be NULL): instead of reporting GENEO_ERR_NOT_SPD, matrix d sets
// weak[d.id] = 1 when one of its pivots is not above weak_tol (relative to
// the unit diagonal of an equilibrated band); the caller factors those
// matrices again in FP64.
// tc5 (FP32, may be NULL): a prepared plan sends the factorisation to the
// fifth-generation tensor-core kernel.
template <typename T>
geneo_status_t band_potrf(T* base, const BandDesc* d_desc, int count, int max_w, int max_n,
                          DevStatus* st, cudaStream_t s, bool equil = false,
                          int32_t* weak = nullptr, float weak_tol = 0.f, const Tc5Plan* tc5 = nullptr);
// Solve L L^T X = X in place for `nrhs` columns per matrix (column-major,
// leading dimension = matrix n, column stride = n); X for matrix i (i = the
// descriptor's id when >= 0, else its batch position) starts at
// xbase + xoff[i]; nrhs_dev (may be NULL) gives per-matrix column counts
// capped by nrhs; skip_dev (may be NULL) skips matrices with a non-zero flag;
// a descriptor with n = 0 is skipped.
// max_n (largest matrix order, 0 if unknown) enables the one-right-hand-side
// solve with the vector resident in shared memory.  tc_passes (FP32 factors,
// several right-hand sides): 3 = each tensor-core product as three TF32
// passes (about FP32 accuracy), 1 = one TF32 pass.  res_stages (one
// right-hand side with the vector resident, 2-4; 0 = by shared memory): the
// pipeline depth of that kernel, as an autotuner picked it.  active (0 =
// count): how many of the matrices skip_dev leaves to solve, which sizes the
// column split of the multi-column kernels.
template <typename T>
geneo_status_t band_solve(const T* base, const BandDesc* d_desc, int count, int max_w,
                          double* xbase, const int64_t* xoff, int nrhs, const int32_t* nrhs_dev,
                          const int32_t* skip_dev, DevStatus* st, cudaStream_t s, int max_n = 0,
                          int tc_passes = 3, int res_stages = 0, int active = 0);

// FP64 factors solved in double-single arithmetic on the FP32 pipe (about
// 46 significant bits) for several right-hand sides: the FP64 fallback
// factors of the FP32 mode, where FP64's 1/64 rate on GB300 bounds the
// sweeps; one right-hand side is solved in FP64.
geneo_status_t band_solve_ds(const double* base, const BandDesc* d_desc, int count, int max_w, double* xbase,
                             const int64_t* xoff, int nrhs, const int32_t* nrhs_dev, const int32_t* skip_dev,
                             DevStatus* st, cudaStream_t s, int max_n, int active = 0);

// solve_set.cu
// A batch of band factors cut into classes of similar half bandwidth for
// band_solve (each class launched with its own widest band and longest
// vector), the classes spread over lanes: lane 0 = the caller's stream,
// lane l > 0 = SolveStreams::s[l - 1].
struct SolveClass {
  const void* base = nullptr;  // float or double band storage
  bool f64 = false;
  bool ds = false;             // FP64 factors, several right-hand sides in double-single
  BandDesc* d = nullptr;       // the class's descriptors (device), largest sweep first
  int count = 0, max_w = 0, max_n = 0;
  double cost = 0.0;           // bytes of one forward and backward sweep over the class
  int lane = 0;
};
struct SolveSet {
  std::vector<SolveClass> cls;
  int lanes = 1;
};
constexpr int kSolveStreams = 4;
struct SolveStreams {
  cudaStream_t s[kSolveStreams] = {};
  cudaEvent_t ev[kSolveStreams] = {};
  cudaEvent_t fork = nullptr;
};
// The classes of the band batch (base, f64, d_desc, count) and, in FP32 mode,
// of the FP64 refactorisations (base64, d_desc64, count64; may be empty),
// whose multi-column solves run in double-single arithmetic when ds64;
// descriptors with n = 0 are left out.  Device descriptor arrays come from
// mem; the call synchronises s once (it reads the descriptors back).
geneo_status_t make_solve_set(const void* base, bool f64, const BandDesc* d_desc, int count,
                              const double* base64, const BandDesc* d_desc64, int count64, DevMem& mem,
                              cudaStream_t s, SolveSet* out, bool ds64 = false);
// band_solve over every class, ordered after the work already on s; the
// work of every lane is joined back into s before the call returns.  active
// (0 = all): an upper bound of the matrices of any class that skip_dev leaves
// to solve.
geneo_status_t solve_set_run(const SolveSet& ss, const SolveStreams& pool, double* xbase, const int64_t* xoff,
                             int nrhs, const int32_t* nrhs_dev, const int32_t* skip_dev, DevStatus* st,
                             cudaStream_t s, int tc_passes = 3, int res_stages = 0, int active = 0);

}  // namespace geneo
