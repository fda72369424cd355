// Size classes of a batch of band factors for the solves.
//
// The local solves of the preconditioner (A_j^{-1}, Section 3) and the block
// solves of the eigensolver (K_j^{-1}, Section 4.4) run one thread block per
// subdomain, and band_solve picks one kernel and one shared-memory size for a
// whole launch from the widest band and the longest vector of the batch.  In
// a batch of very uneven subdomains one large box would then send every
// subdomain to the streamed kernels and size every block for itself.  A
// SolveSet cuts the batch (the FP32 part and the FP64 part separately) into
// classes of similar half bandwidth, each launched with its own maxima, and
// runs the classes concurrently: the largest on the caller's stream, the
// others on the handle's solve streams, assigned longest-first to the least
// loaded stream.  Inside a class the subdomains are ordered by cost, largest
// first, so that the longest sweeps start first.
#include <algorithm>
#include <numeric>
#include <vector>

#include "common.cuh"

namespace geneo {
namespace {

constexpr double kClassRatio = 0.6;  // a class holds half bandwidths down to this fraction of its widest
constexpr int kMaxClassesPerPart = 6;

double sweep_bytes(const BandDesc& b, double esz) {
  return 2.0 * esz * (double)b.n * (double)(b.w + 1);
}

geneo_status_t add_part(const void* base, bool f64, bool ds, const BandDesc* d_desc, int count, DevMem& mem,
                        cudaStream_t s, std::vector<SolveClass>& out) {
  if (!base || !d_desc || count <= 0) return GENEO_OK;
  std::vector<BandDesc> h(count);
  GENEO_CUDA(cudaMemcpyAsync(h.data(), d_desc, sizeof(BandDesc) * count, cudaMemcpyDeviceToHost, s));
  GENEO_CUDA(cudaStreamSynchronize(s));
  std::vector<BandDesc> live;
  for (const BandDesc& b : h)
    if (b.n > 0) live.push_back(b);
  if (live.empty()) return GENEO_OK;
  std::stable_sort(live.begin(), live.end(), [](const BandDesc& a, const BandDesc& b) {
    return a.w != b.w ? a.w > b.w : a.n > b.n;
  });
  const double esz = f64 ? 8.0 : 4.0;
  std::vector<std::vector<BandDesc>> groups;
  int top = -1;
  for (const BandDesc& b : live) {
    if (groups.empty() || ((double)b.w < kClassRatio * top && (int)groups.size() < kMaxClassesPerPart)) {
      groups.emplace_back();
      top = b.w;
    }
    groups.back().push_back(b);
  }
  for (auto& g : groups) {
    std::stable_sort(g.begin(), g.end(), [&](const BandDesc& a, const BandDesc& b) {
      return sweep_bytes(a, esz) > sweep_bytes(b, esz);
    });
    SolveClass c;
    c.base = base;
    c.f64 = f64;
    c.ds = ds;
    c.count = (int)g.size();
    for (const BandDesc& b : g) {
      c.max_w = std::max(c.max_w, b.w);
      c.max_n = std::max(c.max_n, b.n);
      c.cost += sweep_bytes(b, esz);
    }
    GENEO_TRY(mem.get(&c.d, g.size()));
    GENEO_CUDA(cudaMemcpyAsync(c.d, g.data(), sizeof(BandDesc) * g.size(), cudaMemcpyHostToDevice, s));
    out.push_back(c);
  }
  return GENEO_OK;
}

geneo_status_t run_class(const SolveClass& c, double* xbase, const int64_t* xoff, int nrhs,
                         const int32_t* nrhs_dev, const int32_t* skip_dev, DevStatus* st, cudaStream_t s,
                         int tc_passes, int res_stages, int active) {
  const int act = active > 0 ? std::min(active, c.count) : 0;
  if (c.ds && nrhs > 1)
    return band_solve_ds(static_cast<const double*>(c.base), c.d, c.count, c.max_w, xbase, xoff, nrhs, nrhs_dev,
                         skip_dev, st, s, c.max_n, act);
  if (c.f64)
    return band_solve<double>(static_cast<const double*>(c.base), c.d, c.count, c.max_w, xbase, xoff, nrhs,
                              nrhs_dev, skip_dev, st, s, c.max_n, tc_passes, res_stages, act);
  return band_solve<float>(static_cast<const float*>(c.base), c.d, c.count, c.max_w, xbase, xoff, nrhs,
                           nrhs_dev, skip_dev, st, s, c.max_n, tc_passes, res_stages, act);
}

}  // namespace

geneo_status_t make_solve_set(const void* base, bool f64, const BandDesc* d_desc, int count,
                              const double* base64, const BandDesc* d_desc64, int count64, DevMem& mem,
                              cudaStream_t s, SolveSet* out, bool ds64) {
  out->cls.clear();
  out->lanes = 1;
  GENEO_TRY(add_part(base, f64, false, d_desc, count, mem, s, out->cls));
  GENEO_TRY(add_part(base64, true, ds64, d_desc64, count64, mem, s, out->cls));
  // longest first onto the least loaded lane (lane 0 = the caller's stream)
  std::vector<size_t> order(out->cls.size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](size_t a, size_t b) { return out->cls[a].cost > out->cls[b].cost; });
  const int lanes = std::min<int>(1 + kSolveStreams, (int)out->cls.size());
  std::vector<double> load(std::max(lanes, 1), 0.0);
  std::vector<SolveClass> sorted;
  for (size_t i : order) {
    const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[l] += out->cls[i].cost;
    out->cls[i].lane = l;
    sorted.push_back(out->cls[i]);
  }
  out->cls.swap(sorted);
  out->lanes = std::max(lanes, 1);
  return GENEO_OK;
}

geneo_status_t solve_set_run(const SolveSet& ss, const SolveStreams& pool, double* xbase, const int64_t* xoff,
                             int nrhs, const int32_t* nrhs_dev, const int32_t* skip_dev, DevStatus* st,
                             cudaStream_t s, int tc_passes, int res_stages, int active) {
  if (ss.cls.empty() || nrhs <= 0) return GENEO_OK;
  if (ss.lanes > 1) {
    GENEO_CUDA(cudaEventRecord(pool.fork, s));
    for (int l = 1; l < ss.lanes; ++l) GENEO_CUDA(cudaStreamWaitEvent(pool.s[l - 1], pool.fork, 0));
  }
  geneo_status_t rc = GENEO_OK;
  for (const SolveClass& c : ss.cls) {
    const cudaStream_t cs = c.lane == 0 ? s : pool.s[c.lane - 1];
    rc = run_class(c, xbase, xoff, nrhs, nrhs_dev, skip_dev, st, cs, tc_passes, res_stages, active);
    if (rc != GENEO_OK) break;
  }
  // join every lane, also after a failed launch, so that no work is left
  // unordered with the caller's stream
  for (int l = 1; l < ss.lanes; ++l) {
    GENEO_CUDA(cudaEventRecord(pool.ev[l - 1], pool.s[l - 1]));
    GENEO_CUDA(cudaStreamWaitEvent(s, pool.ev[l - 1], 0));
  }
  return rc;
}

}  // namespace geneo
