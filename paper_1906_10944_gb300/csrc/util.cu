// Device memory bookkeeping, error strings and a device-wide exclusive scan.
#include <atomic>
#include <cstdio>

#include "common.cuh"

namespace geneo {

static std::atomic<int64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(); }

static thread_local std::string g_last_cuda_error;

void set_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s: %s (%s:%d)", cudaGetErrorString(e), what, file, line);
  g_last_cuda_error = buf;
}

const std::string& last_cuda_error() { return g_last_cuda_error; }

geneo_status_t DevMem::alloc(void** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 16;
  cudaError_t e = cudaMallocAsync(p, n, stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_cuda_error(e, "cudaMallocAsync", __FILE__, __LINE__);
    *p = nullptr;
    return GENEO_ERR_OOM;
  }
  ptrs.push_back(*p);
  bytes += (int64_t)n;
  return GENEO_OK;
}

void DevMem::release(void* p) {
  for (auto& q : ptrs) {
    if (q == p) {
      cudaFreeAsync(q, stream);
      q = nullptr;
    }
  }
}

void DevMem::free_all() {
  for (void* p : ptrs)
    if (p) cudaFreeAsync(p, stream);
  ptrs.clear();
  bytes = 0;
}

namespace {
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;   // items per thread
constexpr int kScanTile = kScanThreads * kScanItems;

// Per tile: exclusive scan in place, tile total to sums[blockIdx.x].
__global__ void __launch_bounds__(kScanThreads)
k_scan_tiles(const int64_t* __restrict__ in, int64_t* __restrict__ out, int64_t n,
             int64_t* __restrict__ sums) {
  __shared__ int64_t warp_tot[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t local = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t idx = base + i;
    v[i] = idx < n ? in[idx] : 0;
    local += v[i];
  }
  // inclusive warp scan of per-thread totals
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t incl = local;
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int64_t t = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int64_t u = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += u;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = t;  // inclusive
  }
  __syncthreads();
  int64_t run = incl - local + (wid > 0 ? warp_tot[wid - 1] : 0);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t idx = base + i;
    const int64_t x = v[i];
    if (idx < n) out[idx] = run;
    run += x;
  }
  if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = run;
}

__global__ void k_add_offsets(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ offs) {
  const int64_t idx = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
  const int64_t add = offs[blockIdx.x];
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t j = idx + (int64_t)i * kScanThreads;
    if (j < n && j < (int64_t)(blockIdx.x + 1) * kScanTile) out[j] += add;
  }
}
}  // namespace

geneo_status_t exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total,
                                  DevMem& tmp, cudaStream_t st) {
  if (n <= 0) {
    if (total) *total = 0;
    return GENEO_OK;
  }
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  int64_t* sums = nullptr;
  GENEO_TRY(tmp.get(&sums, (size_t)tiles + 1));
  k_scan_tiles<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, out, n, sums); note_launch();
  GENEO_CUDA(cudaGetLastError());
  if (tiles > 1) {
    int64_t* offs = nullptr;
    GENEO_TRY(tmp.get(&offs, (size_t)tiles + 1));
    int64_t t2 = 0;
    GENEO_TRY(exclusive_scan_i64(sums, offs, tiles, &t2, tmp, st));
    k_add_offsets<<<(unsigned)tiles, kScanThreads, 0, st>>>(out, n, offs); note_launch();
    GENEO_CUDA(cudaGetLastError());
    if (total) *total = t2;
  } else if (total) {
    GENEO_CUDA(cudaMemcpyAsync(total, sums, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    GENEO_CUDA(cudaStreamSynchronize(st));
  }
  return GENEO_OK;
}

}  // namespace geneo
