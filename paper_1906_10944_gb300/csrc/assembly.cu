// Subdomain structure, partition of unity and local matrices.
//
// Section 3: Omega_j is a union of elements; R_j restricts to the dofs of
// V_{h,0}(Omega_j), here D_j = the dofs of N_j (closure of Omega_j without
// global Dirichlet dofs) all of whose elements lie in Omega_j.
// Section 4.3: the discrete partition of unity X_j is 1/c_k on D_j, where c_k
// counts the subdomains whose D contains dof k (the "sum of ones"), and 0 on
// the subdomain boundary; the Neumann matrix Atilde_j is assembled from all
// elements of Omega_j, the overlap matrix A_j^o from the elements that belong
// to more than one subdomain.  Section 4.4: K_j = Atilde_j - sigma B_j with
// B_j = X_j A_j^o X_j is the operator of the shift-and-invert transformation.
//
// All scatter steps are written in gather form (one thread owns one output
// row and sums its contributions in a fixed order), so the results are
// bitwise reproducible.  Integer counters use atomics, which is exact.
#include <algorithm>
#include <chrono>

#include "handle.cuh"

namespace geneo {
namespace {

constexpr int kT = 256;

__global__ void k_count_i32(const int32_t* __restrict__ idx, int64_t m, int32_t* __restrict__ cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[idx[i]], 1);
}

__global__ void k_i32_to_i64(const int32_t* __restrict__ a, int64_t* __restrict__ b, int64_t m) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}

// cnt_j[a] = number of elements of Omega_j containing N-row a.
__global__ void k_sub_elem_counts(const SubDesc* __restrict__ sub, const int32_t* __restrict__ sub_elem,
                                  const int32_t* __restrict__ elem_dofs, int ke,
                                  const int32_t* __restrict__ Nlist, int32_t* __restrict__ cnt_j) {
  const SubDesc d = sub[blockIdx.x];
  const int32_t* Nj = Nlist + d.offN;
  const int64_t tot = (int64_t)d.nE * ke;
  for (int64_t i = threadIdx.x; i < tot; i += blockDim.x) {
    const int32_t e = sub_elem[d.offE + i / ke];
    const int32_t k = elem_dofs[(int64_t)e * ke + (i % ke)];
    const int loc = find_i32(Nj, d.nN, k);
    if (loc >= 0) atomicAdd(&cnt_j[d.offN + loc], 1);
  }
}

// D_j = N-rows whose element count inside Omega_j equals the global count.
// Ordered compaction with a block scan; writes Dlist, dpos, nToD and nD.
__global__ void k_dirichlet_set(const SubDesc* __restrict__ sub, const int32_t* __restrict__ Nlist,
                                const int32_t* __restrict__ cnt_j, const int32_t* __restrict__ cnt_all,
                                int32_t* __restrict__ Dlist, int32_t* __restrict__ dpos,
                                int32_t* __restrict__ nToD, int32_t* __restrict__ nD_out) {
  __shared__ int32_t wsum[kT / 32];
  __shared__ int32_t carry;
  const SubDesc d = sub[blockIdx.x];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int base = 0; base < d.nN; base += blockDim.x) {
    const int a = base + threadIdx.x;
    int flag = 0;
    if (a < d.nN) flag = cnt_j[d.offN + a] == cnt_all[Nlist[d.offN + a]];
    unsigned ball = __ballot_sync(0xffffffffu, flag);
    int pre = __popc(ball & ((1u << lane) - 1u));
    if (lane == 0) wsum[wid] = __popc(ball);
    __syncthreads();
    int woff = 0;
    for (int w2 = 0; w2 < wid; ++w2) woff += wsum[w2];
    int tot = 0;
    for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) tot += wsum[w2];
    const int pos = carry + woff + pre;
    if (a < d.nN) {
      if (flag) {
        Dlist[d.offN + pos] = Nlist[d.offN + a];
        dpos[d.offN + pos] = a;
        nToD[d.offN + a] = pos;
      } else {
        nToD[d.offN + a] = -1;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) nD_out[blockIdx.x] = carry;
}

__global__ void k_count_D(const SubDesc* __restrict__ sub, const int32_t* __restrict__ Dlist,
                          int32_t* __restrict__ cmul) {
  const SubDesc d = sub[blockIdx.x];
  for (int i = threadIdx.x; i < d.nD; i += blockDim.x) atomicAdd(&cmul[Dlist[d.offN + i]], 1);
}

// Every free dof must lie in some D_j (Section 4.3: the weights sum to one).
__global__ void k_check_cover(const int32_t* __restrict__ cmul, const uint8_t* __restrict__ dir,
                              int64_t n, DevStatus* st) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    if (!dir[k] && cmul[k] == 0) record_error(st, GENEO_ERR_ARG, -1, k);
}

// X_j = 1/c_k on D_j, 0 elsewhere on N_j.
__global__ void k_pu(const SubDesc* __restrict__ sub, const int32_t* __restrict__ Nlist,
                     const int32_t* __restrict__ nToD, const int32_t* __restrict__ cmul,
                     double* __restrict__ pu) {
  const SubDesc d = sub[blockIdx.x];
  for (int a = threadIdx.x; a < d.nN; a += blockDim.x) {
    const int64_t r = d.offN + a;
    pu[r] = nToD[r] >= 0 ? 1.0 / (double)cmul[Nlist[r]] : 0.0;
  }
}

// Caller weights (Definition 3): each X_j(k) in [0, 1] and zero on the
// inner boundary of Omega_j (the N-rows outside D_j).
__global__ void k_check_pu_local(const SubDesc* __restrict__ sub, const int32_t* __restrict__ nToD,
                                 const double* __restrict__ pu, DevStatus* st) {
  const SubDesc d = sub[blockIdx.x];
  for (int a = threadIdx.x; a < d.nN; a += blockDim.x) {
    const int64_t r = d.offN + a;
    const double v = pu[r];
    if (!(v >= 0.0 && v <= 1.0) || (nToD[r] < 0 && v != 0.0)) record_error(st, GENEO_ERR_ARG, blockIdx.x, a);
  }
}

// ... and sum_j X_j(k) = 1 (to 1e-12) on every non-Dirichlet dof, summed in
// the fixed order of the inverse map.
__global__ void k_check_pu_sum(int64_t n, const uint8_t* __restrict__ dir, const int64_t* __restrict__ invD_ptr,
                               const int32_t* __restrict__ invD_sub, const int32_t* __restrict__ invD_loc,
                               const SubDesc* __restrict__ sub, const int32_t* __restrict__ dpos,
                               const double* __restrict__ pu, DevStatus* st) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    if (dir[k]) continue;
    double sum = 0.0;
    for (int64_t t = invD_ptr[k]; t < invD_ptr[k + 1]; ++t) {
      const SubDesc& d = sub[invD_sub[t]];
      sum += pu[d.offN + dpos[d.offN + invD_loc[t]]];
    }
    if (!(fabs(sum - 1.0) <= 1e-12)) record_error(st, GENEO_ERR_ARG, -1, k);
  }
}

// Smooth (Sarkis) partition of unity, Section 3 (Fig. 2, right).
// Step 1: d_j(a) = element layers between N-row a and the inner boundary of
// Omega_j (the N-rows outside D_j, d = 0), by breadth-first levels over the
// local pattern: every coupling of a D_j row comes from an element of
// Omega_j, so these are distances through Omega_j.  A subdomain without
// inner boundary takes d = 1 everywhere.  The level loop is bounded by nN.
__global__ void __launch_bounds__(kT)
k_sarkis_dist(const SubDesc* __restrict__ sub, const int32_t* __restrict__ nToD,
              const int64_t* __restrict__ lrow, const int32_t* __restrict__ lcol, int32_t* __restrict__ dist) {
  const SubDesc d = sub[blockIdx.x];
  int32_t* dj = dist + d.offN;
  int inner = 0;
  for (int a = threadIdx.x; a < d.nN; a += blockDim.x) {
    const bool b = nToD[d.offN + a] < 0;
    dj[a] = b ? 0 : -1;
    inner |= b;
  }
  if (!__syncthreads_or(inner)) {
    for (int a = threadIdx.x; a < d.nN; a += blockDim.x) dj[a] = 1;
    return;
  }
  for (int level = 1; level <= d.nN; ++level) {
    int changed = 0;
    for (int a = threadIdx.x; a < d.nN; a += blockDim.x) {
      if (dj[a] >= 0) continue;
      // a row set at this level never equals level - 1, so rows written in
      // this sweep do not feed it
      for (int64_t e = lrow[d.offN + a]; e < lrow[d.offN + a + 1]; ++e)
        if (dj[lcol[e]] == level - 1) {
          dj[a] = level;
          changed = 1;
          break;
        }
    }
    if (!__syncthreads_or(changed)) break;
  }
}

// Step 2: total(k) = sum_i d_i(k) over the subdomains whose D holds k (the
// others contribute d = 0 or do not hold k).
__global__ void k_sarkis_total(int64_t n, const int64_t* __restrict__ invD_ptr, const int32_t* __restrict__ invD_sub,
                               const int32_t* __restrict__ invD_loc, const SubDesc* __restrict__ sub,
                               const int32_t* __restrict__ dpos, const int32_t* __restrict__ dist,
                               double* __restrict__ total) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    double sum = 0.0;
    for (int64_t t = invD_ptr[k]; t < invD_ptr[k + 1]; ++t) {
      const SubDesc& d = sub[invD_sub[t]];
      sum += (double)dist[d.offN + dpos[d.offN + invD_loc[t]]];
    }
    total[k] = sum;
  }
}

// Step 3: X_j = d_j / total on D_j, 0 on the inner boundary.
__global__ void k_sarkis_pu(const SubDesc* __restrict__ sub, const int32_t* __restrict__ Nlist,
                            const int32_t* __restrict__ nToD, const int32_t* __restrict__ dist,
                            const double* __restrict__ total, double* __restrict__ pu) {
  const SubDesc d = sub[blockIdx.x];
  for (int a = threadIdx.x; a < d.nN; a += blockDim.x) {
    const int64_t r = d.offN + a;
    pu[r] = nToD[r] >= 0 ? (double)dist[r] / total[Nlist[r]] : 0.0;
  }
}

__global__ void k_fill_inv(const SubDesc* __restrict__ sub, const int32_t* __restrict__ list,
                           const int32_t* __restrict__ counts_per_sub, int use_nD,
                           const int64_t* __restrict__ ptr, int32_t* __restrict__ cursor,
                           int32_t* __restrict__ inv_sub, int32_t* __restrict__ inv_loc) {
  const SubDesc d = sub[blockIdx.x];
  const int cnt = use_nD ? d.nD : d.nN;
  (void)counts_per_sub;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    const int32_t k = list[d.offN + i];
    const int pos = atomicAdd(&cursor[k], 1);
    inv_sub[ptr[k] + pos] = blockIdx.x;
    inv_loc[ptr[k] + pos] = i;
  }
}

// Sort each short inverse list by key (insertion sort; lists hold at most a
// few dozen entries).  Makes every later gather order deterministic.
__global__ void k_sort_lists(const int64_t* __restrict__ ptr, int64_t n, int32_t* __restrict__ key,
                             int32_t* __restrict__ val) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = ptr[k], e = ptr[k + 1];
    for (int64_t i = b + 1; i < e; ++i) {
      const int32_t kk = key[i];
      const int32_t vv = val ? val[i] : 0;
      int64_t j = i - 1;
      while (j >= b && key[j] > kk) {
        key[j + 1] = key[j];
        if (val) val[j + 1] = val[j];
        --j;
      }
      key[j + 1] = kk;
      if (val) val[j + 1] = vv;
    }
  }
}

__global__ void k_fill_dof_elem(const int32_t* __restrict__ elem_dofs, int64_t n_elem, int ke,
                                const int64_t* __restrict__ ptr, int32_t* __restrict__ cursor,
                                int32_t* __restrict__ de) {
  const int64_t tot = n_elem * ke;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t k = elem_dofs[i];
    const int pos = atomicAdd(&cursor[k], 1);
    de[ptr[k] + pos] = (int32_t)(i / ke);
  }
}

// Local CSR pattern: row a of subdomain j holds the columns of global row
// N_j[a] that are in N_j.  pass 0 counts, pass 1 fills and records the
// half bandwidth max |a - b|.
template <int PASS>
__global__ void k_local_csr(const SubDesc* __restrict__ sub, const int32_t* __restrict__ Nlist,
                            const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            const double* __restrict__ val, int64_t* __restrict__ lcnt,
                            const int64_t* __restrict__ lrow, int32_t* __restrict__ lcol,
                            double* __restrict__ lA, int32_t* __restrict__ wK) {
  const SubDesc d = sub[blockIdx.x];
  const int32_t* Nj = Nlist + d.offN;
  int wmax = 0;
  for (int a = threadIdx.x; a < d.nN; a += blockDim.x) {
    const int32_t k = Nj[a];
    int c = 0;
    int64_t out = PASS ? lrow[d.offN + a] : 0;
    for (int64_t e = rowptr[k]; e < rowptr[k + 1]; ++e) {
      const int b = find_i32(Nj, d.nN, col[e]);
      if (b < 0) continue;
      if (PASS) {
        lcol[out] = b;
        lA[out] = val[e];
        ++out;
        wmax = max(wmax, abs(a - b));
      }
      ++c;
    }
    if (!PASS) lcnt[d.offN + a] = c;
  }
  if (PASS) {
    wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, 16));
    wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, 8));
    wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, 4));
    wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, 2));
    wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, 1));
    if ((threadIdx.x & 31) == 0) atomicMax(&wK[blockIdx.x], wmax);
  }
}

// Half bandwidth of A_j in D numbering.
__global__ void k_band_width_A(const SubDesc* __restrict__ sub, const int32_t* __restrict__ dpos,
                               const int32_t* __restrict__ nToD, const int64_t* __restrict__ lrow,
                               const int32_t* __restrict__ lcol, int32_t* __restrict__ wA) {
  const SubDesc d = sub[blockIdx.x];
  int wmax = 0;
  for (int i = threadIdx.x; i < d.nD; i += blockDim.x) {
    const int a = dpos[d.offN + i];
    for (int64_t e = lrow[d.offN + a]; e < lrow[d.offN + a + 1]; ++e) {
      const int i2 = nToD[d.offN + lcol[e]];
      if (i2 >= 0) wmax = max(wmax, abs(i - i2));
    }
  }
  for (int o = 16; o > 0; o >>= 1) wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&wA[blockIdx.x], wmax);
}

// Local (N_j) index of every dof of every element of Omega_j, -1 for a
// global Dirichlet dof: eloc[(offE + e) * ke + b] for element Ej[e].  One
// lookup per (element, dof) instead of one per (row, element, dof).
__global__ void k_elem_local(const SubDesc* __restrict__ sub, const int32_t* __restrict__ Nlist,
                             const int32_t* __restrict__ sub_elem, const int32_t* __restrict__ elem_dofs,
                             int ke, int32_t* __restrict__ eloc) {
  const SubDesc d = sub[blockIdx.x];
  const int32_t* Nj = Nlist + d.offN;
  const int32_t* Ej = sub_elem + d.offE;
  const int64_t items = (int64_t)d.nE * ke;
  for (int64_t t = threadIdx.x; t < items; t += blockDim.x) {
    const int64_t e = t / ke;
    const int b = (int)(t - e * ke);
    eloc[d.offE * ke + t] = find_i32(Nj, d.nN, elem_dofs[(int64_t)Ej[e] * ke + b]);
  }
}

// Element assembly in gather form: row a of Omega_j sums, over the elements
// of its dof that belong to Omega_j (ascending element id), the element
// matrix row.  lK receives Atilde_j, lB receives A_j^o (overlap elements).
// The local column of an element dof comes from eloc, its slot in row a
// (columns ascending) by binary search.
__global__ void k_assemble(const SubDesc* __restrict__ sub, const int32_t* __restrict__ Nlist,
                           const int32_t* __restrict__ sub_elem, const int64_t* __restrict__ de_ptr,
                           const int32_t* __restrict__ de, const int32_t* __restrict__ eloc,
                           const double* __restrict__ elem_mats, int ke,
                           const int32_t* __restrict__ e_tau, const int64_t* __restrict__ lrow,
                           const int32_t* __restrict__ lcol, double* __restrict__ lK,
                           double* __restrict__ lB, DevStatus* st) {
  const SubDesc d = sub[blockIdx.x];
  const int32_t* Nj = Nlist + d.offN;
  const int32_t* Ej = sub_elem + d.offE;
  for (int a = threadIdx.x; a < d.nN; a += blockDim.x) {
    const int32_t k = Nj[a];
    const int64_t r0 = lrow[d.offN + a], r1 = lrow[d.offN + a + 1];
    const int rl = (int)(r1 - r0);
    const int32_t* rc = lcol + r0;
    for (int64_t e = r0; e < r1; ++e) {
      lK[e] = 0.0;
      lB[e] = 0.0;
    }
    for (int64_t t = de_ptr[k]; t < de_ptr[k + 1]; ++t) {
      const int32_t el = de[t];
      const int pe = find_i32(Ej, d.nE, el);
      if (pe < 0) continue;
      const int32_t* loc = eloc + (d.offE + pe) * (int64_t)ke;
      int ak = 0;
      while (ak < ke && loc[ak] != a) ++ak;
      if (ak == ke) continue;  // cannot happen: dof k of this element is row a
      const double* Krow = elem_mats + ((int64_t)el * ke + ak) * ke;
      const bool ovl = e_tau[el] > 1;
      for (int bq = 0; bq < ke; ++bq) {
        const int bl = loc[bq];
        if (bl < 0) continue;
        const int sl = lower_bound_i32(rc, rl, bl);
        if (sl >= rl || rc[sl] != bl) continue;  // cannot happen when A holds every element coupling
        const int64_t slot = r0 + sl;
        const double v = Krow[bq];
        if (!isfinite(v)) record_error(st, GENEO_ERR_NONFINITE, blockIdx.x, el);
        lK[slot] += v;
        if (ovl) lB[slot] += v;
      }
    }
  }
}

// B = X M X with M = A^o (paper form) or Atilde (full form); K = Atilde - sigma B.
__global__ void k_pencil(const SubDesc* __restrict__ sub, const double* __restrict__ pu,
                         const int64_t* __restrict__ lrow, const int32_t* __restrict__ lcol,
                         double* __restrict__ lK, double* __restrict__ lB, double sigma, int full) {
  const SubDesc d = sub[blockIdx.x];
  for (int a = threadIdx.x; a < d.nN; a += blockDim.x) {
    const double xa = pu[d.offN + a];
    for (int64_t e = lrow[d.offN + a]; e < lrow[d.offN + a + 1]; ++e) {
      const double at = lK[e];
      const double m = full ? at : lB[e];
      const double b = xa * m * pu[d.offN + lcol[e]];
      lB[e] = b;
      lK[e] = at - sigma * b;
    }
  }
}

// Band entries of K_j / A_j for the batch `bd` (descriptor id = subdomain).
template <typename T>
__global__ void k_band_fill_K(const SubDesc* __restrict__ sub, const BandDesc* __restrict__ bd,
                              const int64_t* __restrict__ lrow, const int32_t* __restrict__ lcol,
                              const double* __restrict__ lK, T* __restrict__ band) {
  const BandDesc b = bd[blockIdx.x];
  const SubDesc d = sub[b.id];
  const int64_t ld = b.ld;
  T* L = band + b.off;
  for (int a = threadIdx.x; a < d.nN; a += blockDim.x)
    for (int64_t e = lrow[d.offN + a]; e < lrow[d.offN + a + 1]; ++e) {
      const int c = lcol[e];
      if (c <= a) L[(int64_t)a * ld + (c - a + b.w)] = (T)lK[e];
    }
}

template <typename T>
__global__ void k_band_fill_A(const SubDesc* __restrict__ sub, const BandDesc* __restrict__ bd,
                              const int32_t* __restrict__ dpos, const int32_t* __restrict__ nToD,
                              const int64_t* __restrict__ lrow, const int32_t* __restrict__ lcol,
                              const double* __restrict__ lA, T* __restrict__ band) {
  const BandDesc b = bd[blockIdx.x];
  const SubDesc d = sub[b.id];
  const int64_t ld = b.ld;
  T* L = band + b.off;
  for (int i = threadIdx.x; i < d.nD; i += blockDim.x) {
    const int a = dpos[d.offN + i];
    for (int64_t e = lrow[d.offN + a]; e < lrow[d.offN + a + 1]; ++e) {
      const int i2 = nToD[d.offN + lcol[e]];
      if (i2 >= 0 && i2 <= i) L[(int64_t)i * ld + (i2 - i + b.w)] = (T)lA[e];
    }
  }
}

inline int grid_for(int64_t m) { return (int)std::min<int64_t>(std::max<int64_t>(1, (m + kT - 1) / kT), 152 * 16); }

double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// Adaptive precision per subdomain: an FP32 factorisation with a weak pivot
// (coefficient contrast beyond what FP32 resolves) is redone in FP64 from
// the FP64 local matrix, and its FP32 descriptor gets n = 0 so the FP32
// solves skip it.  Descriptor ids stay the subdomain indices, so the FP64
// batch solves into the same vectors.
struct Refactor {
  double* band = nullptr;
  BandDesc* desc = nullptr;
  int count = 0, maxw = 0, maxn = 0;
};

geneo_status_t refactor_fp64(geneo_handle_s* h, const AssemblyOut& a, const int32_t* weak_dev, bool isK,
                             std::vector<BandDesc>& hmain, BandDesc* dmain, DevMem& mem, cudaStream_t s,
                             Refactor* r) {
  const int N = h->N;
  std::vector<int32_t> flag(N);
  GENEO_CUDA(cudaMemcpyAsync(flag.data(), weak_dev, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, s));
  GENEO_CUDA(cudaStreamSynchronize(s));
  std::vector<BandDesc> rd;
  int64_t tot = 0;
  for (int j = 0; j < N; ++j) {
    if (!flag[j]) continue;
    const SubDesc& d = h->hsub[j];
    const int n = isK ? d.nN : d.nD, w = isK ? d.wK : d.wA;
    rd.push_back(BandDesc{tot, n, w, j, band_ld(w), 0, -1});
    tot += (int64_t)n * band_ld(w);
    r->maxw = std::max(r->maxw, w);
    r->maxn = std::max(r->maxn, n);
  }
  r->count = (int)rd.size();
  if (rd.empty()) return GENEO_OK;
  int64_t dv = tot;
  for (BandDesc& b : rd) {
    b.dinv = dv;
    dv += dinv_elems(b.n);
  }
  GENEO_TRY(mem.get(&r->band, (size_t)dv));
  GENEO_TRY(mem.get(&r->desc, rd.size()));
  GENEO_CUDA(cudaMemsetAsync(r->band, 0, sizeof(double) * tot, s));
  GENEO_CUDA(cudaMemcpyAsync(r->desc, rd.data(), sizeof(BandDesc) * rd.size(), cudaMemcpyHostToDevice, s));
  const int R = r->count;
  if (isK)
    k_band_fill_K<double><<<R, kT, 0, s>>>(h->dsub, r->desc, a.lrow, a.lcol, a.lK, r->band);
  else
    k_band_fill_A<double><<<R, kT, 0, s>>>(h->dsub, r->desc, h->dpos, h->nToD, a.lrow, a.lcol, a.lA, r->band);
  note_launch();
  GENEO_CUDA(cudaGetLastError());
  GENEO_TRY(band_potrf<double>(r->band, r->desc, R, r->maxw, r->maxn, h->dstat, s));
  for (const BandDesc& b : rd) hmain[b.id].n = 0;
  GENEO_CUDA(cudaMemcpyAsync(dmain, hmain.data(), sizeof(BandDesc) * N, cudaMemcpyHostToDevice, s));
  return GENEO_OK;
}

// A factorisation batch: descriptors (host and device copies) of one size
// class, largest factorisations first, and its tensor-core plan.
struct FactorBatch {
  std::vector<BandDesc> h;
  BandDesc* d = nullptr;
  int maxw = 0, maxn = 0;
  Tc5Plan plan;
};

// Size classes of a cost-sorted batch for the fifth-generation tensor-core
// kernel: the widths that kernel takes are grouped so that no class pads a
// band to more than 1/0.6 of its own width (rounded up to 32), each class
// with its own tiled-band planes; the widths it does not take form one
// batch for the older kernels.  Without the kernel: one batch.
geneo_status_t factor_batches(const std::vector<BandDesc>& sorted, bool tc5_on, bool bf16, DevMem& tmp,
                              cudaStream_t s, std::vector<FactorBatch>& out) {
  out.clear();
  std::vector<std::vector<BandDesc>> groups;
  std::vector<BandDesc> rest;
  if (!tc5_on) {
    rest = sorted;
  } else {
    std::vector<int> widths;
    for (const BandDesc& b : sorted)
      if (tc5_fits(b.w)) widths.push_back((b.w + 31) & ~31);
    std::sort(widths.begin(), widths.end(), std::greater<int>());
    widths.erase(std::unique(widths.begin(), widths.end()), widths.end());
    std::vector<int> tops;  // the W of each class, descending
    for (int W : widths)
      if (tops.empty() || W < 0.6 * tops.back()) tops.push_back(W);
    groups.resize(tops.size());
    for (const BandDesc& b : sorted) {
      if (!tc5_fits(b.w)) {
        rest.push_back(b);
        continue;
      }
      const int W = (b.w + 31) & ~31;
      size_t g = 0;  // the smallest class top that still covers W
      for (size_t i = 0; i < tops.size(); ++i)
        if (tops[i] >= W) g = i;
      groups[g].push_back(b);
    }
  }
  if (!rest.empty()) groups.push_back(rest);
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    if (groups[gi].empty()) continue;
    FactorBatch fb;
    fb.h = groups[gi];
    for (const BandDesc& b : fb.h) {
      fb.maxw = std::max(fb.maxw, b.w);
      fb.maxn = std::max(fb.maxn, b.n);
    }
    GENEO_TRY(tmp.get(&fb.d, fb.h.size()));
    GENEO_CUDA(cudaMemcpyAsync(fb.d, fb.h.data(), sizeof(BandDesc) * fb.h.size(), cudaMemcpyHostToDevice, s));
    const bool is_rest = tc5_on && gi + 1 == groups.size() && !rest.empty();
    if (tc5_on && !is_rest) {
      GENEO_TRY(tc5_prepare(fb.h.data(), (int)fb.h.size(), fb.maxw, tmp, s, &fb.plan));
      fb.plan.bf16 = bf16;
    }
    out.push_back(std::move(fb));
  }
  return GENEO_OK;
}

}  // namespace

geneo_status_t build_structure(geneo_handle_s* h, const geneo_problem_t* p, AssemblyOut& a_out,
                               DevMem& tmp, cudaStream_t s) {
  const int N = h->N;
  const int64_t n = h->n;
  const int ke = p->elem_ndof;
  DevMem& M = h->mem;
  GENEO_TRY(M.get(&h->Nlist, (size_t)h->sumN));
  GENEO_TRY(M.get(&h->Dlist, (size_t)h->sumN));
  GENEO_TRY(M.get(&h->dpos, (size_t)h->sumN));
  GENEO_TRY(M.get(&h->nToD, (size_t)h->sumN));
  GENEO_TRY(M.get(&h->pu, (size_t)h->sumN));
  GENEO_CUDA(cudaMemcpyAsync(h->Nlist, p->sub_dof, sizeof(int32_t) * h->sumN,
                             cudaMemcpyDeviceToDevice, s));

  // element multiplicity e_tau (R5) and global element counts per dof
  GENEO_TRY(tmp.get(&a_out.e_tau, (size_t)p->n_elem));
  GENEO_TRY(tmp.get(&a_out.cnt_all, (size_t)n));
  GENEO_CUDA(cudaMemsetAsync(a_out.e_tau, 0, sizeof(int32_t) * p->n_elem, s));
  GENEO_CUDA(cudaMemsetAsync(a_out.cnt_all, 0, sizeof(int32_t) * n, s));
  const int64_t n_sub_elem = h->hsub.back().offE + h->hsub.back().nE;
  k_count_i32<<<grid_for(n_sub_elem), kT, 0, s>>>(p->sub_elem, n_sub_elem, a_out.e_tau); note_launch();
  k_count_i32<<<grid_for(p->n_elem * ke), kT, 0, s>>>(p->elem_dofs, p->n_elem * ke, a_out.cnt_all); note_launch();
  GENEO_CUDA(cudaGetLastError());

  // D_j (Section 3) from element counts inside / outside Omega_j
  int32_t* cnt_j = nullptr;
  int32_t* nD_dev = nullptr;
  GENEO_TRY(tmp.get(&cnt_j, (size_t)h->sumN));
  GENEO_TRY(tmp.get(&nD_dev, (size_t)N));
  GENEO_CUDA(cudaMemsetAsync(cnt_j, 0, sizeof(int32_t) * h->sumN, s));
  k_sub_elem_counts<<<N, kT, 0, s>>>(h->dsub, p->sub_elem, p->elem_dofs, ke, h->Nlist, cnt_j); note_launch();
  k_dirichlet_set<<<N, kT, 0, s>>>(h->dsub, h->Nlist, cnt_j, a_out.cnt_all, h->Dlist, h->dpos,
                                   h->nToD, nD_dev); note_launch();
  GENEO_CUDA(cudaGetLastError());
  std::vector<int32_t> nD(N);
  GENEO_CUDA(cudaMemcpyAsync(nD.data(), nD_dev, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, s));
  GENEO_CUDA(cudaStreamSynchronize(s));
  for (int j = 0; j < N; ++j) {
    h->hsub[j].nD = nD[j];
    if (nD[j] == 0) return GENEO_ERR_ARG;  // a subdomain without interior dofs
  }
  GENEO_CUDA(cudaMemcpyAsync(h->dsub, h->hsub.data(), sizeof(SubDesc) * N, cudaMemcpyHostToDevice, s));

  // multiplicity c_k and partition of unity (Section 4.3)
  int32_t* cmul = nullptr;
  GENEO_TRY(tmp.get(&cmul, (size_t)n));
  GENEO_CUDA(cudaMemsetAsync(cmul, 0, sizeof(int32_t) * n, s));
  k_count_D<<<N, kT, 0, s>>>(h->dsub, h->Dlist, cmul); note_launch();
  k_check_cover<<<grid_for(n), kT, 0, s>>>(cmul, h->dir, n, h->dstat); note_launch();
  if (p->pu_weights) {  // caller weights (device view of the problem's array)
    GENEO_CUDA(cudaMemcpyAsync(h->pu, p->pu_weights, sizeof(double) * h->sumN, cudaMemcpyDeviceToDevice, s));
    k_check_pu_local<<<N, kT, 0, s>>>(h->dsub, h->nToD, h->pu, h->dstat); note_launch();
  } else {
    k_pu<<<N, kT, 0, s>>>(h->dsub, h->Nlist, h->nToD, cmul, h->pu); note_launch();
  }
  GENEO_CUDA(cudaGetLastError());

  // inverse map dof -> (j, D index), sorted by j
  int64_t* cnt64 = nullptr;
  GENEO_TRY(M.get(&h->invD_ptr, (size_t)n + 1));
  GENEO_TRY(tmp.get(&cnt64, (size_t)n + 1));
  k_i32_to_i64<<<grid_for(n), kT, 0, s>>>(cmul, cnt64, n); note_launch();
  GENEO_CUDA(cudaMemsetAsync(cnt64 + n, 0, sizeof(int64_t), s));
  int64_t totD = 0;
  GENEO_TRY(exclusive_scan_i64(cnt64, h->invD_ptr, n + 1, &totD, tmp, s));
  GENEO_TRY(M.get(&h->invD_sub, (size_t)totD));
  GENEO_TRY(M.get(&h->invD_loc, (size_t)totD));
  int32_t* cursor = nullptr;
  GENEO_TRY(tmp.get(&cursor, (size_t)n));
  GENEO_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int32_t) * n, s));
  k_fill_inv<<<N, kT, 0, s>>>(h->dsub, h->Dlist, nullptr, 1, h->invD_ptr, cursor, h->invD_sub,
                              h->invD_loc); note_launch();
  k_sort_lists<<<grid_for(n), kT, 0, s>>>(h->invD_ptr, n, h->invD_sub, h->invD_loc); note_launch();
  if (p->pu_weights) {
    k_check_pu_sum<<<grid_for(n), kT, 0, s>>>(n, h->dir, h->invD_ptr, h->invD_sub, h->invD_loc, h->dsub,
                                              h->dpos, h->pu, h->dstat); note_launch();
  }
  GENEO_CUDA(cudaGetLastError());
  return check_status(h, s);
}

geneo_status_t assemble_local(geneo_handle_s* h, const geneo_problem_t* p, AssemblyOut& out,
                              DevMem& tmp, cudaStream_t s, double* ms_assembly, double* ms_factor) {
  AssemblyOut& a_out = out;
  auto t0 = std::chrono::steady_clock::now();
  const int N = h->N;
  const int64_t n = h->n;
  const int ke = p->elem_ndof;

  // dof -> element lists (ascending element id)
  int64_t* de_cnt = nullptr;
  int64_t* de_ptr = nullptr;
  int32_t* de = nullptr;
  int32_t* cursor = nullptr;
  GENEO_TRY(tmp.get(&de_cnt, (size_t)n + 1));
  GENEO_TRY(tmp.get(&de_ptr, (size_t)n + 1));
  k_i32_to_i64<<<grid_for(n), kT, 0, s>>>(a_out.cnt_all, de_cnt, n); note_launch();
  GENEO_CUDA(cudaMemsetAsync(de_cnt + n, 0, sizeof(int64_t), s));
  int64_t tot = 0;
  GENEO_TRY(exclusive_scan_i64(de_cnt, de_ptr, n + 1, &tot, tmp, s));
  GENEO_TRY(tmp.get(&de, (size_t)tot));
  GENEO_TRY(tmp.get(&cursor, (size_t)n));
  GENEO_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int32_t) * n, s));
  k_fill_dof_elem<<<grid_for(p->n_elem * ke), kT, 0, s>>>(p->elem_dofs, p->n_elem, ke, de_ptr,
                                                          cursor, de); note_launch();
  k_sort_lists<<<grid_for(n), kT, 0, s>>>(de_ptr, n, de, nullptr); note_launch();
  GENEO_CUDA(cudaGetLastError());

  // local CSR pattern over N-rows
  int64_t* lcnt = nullptr;
  GENEO_TRY(tmp.get(&lcnt, (size_t)h->sumN + 1));
  GENEO_TRY(tmp.get(&out.lrow, (size_t)h->sumN + 1));
  GENEO_CUDA(cudaMemsetAsync(lcnt + h->sumN, 0, sizeof(int64_t), s));
  k_local_csr<0><<<N, kT, 0, s>>>(h->dsub, h->Nlist, h->rowptr, h->col, h->val, lcnt, nullptr,
                                  nullptr, nullptr, nullptr); note_launch();
  GENEO_CUDA(cudaGetLastError());
  GENEO_TRY(exclusive_scan_i64(lcnt, out.lrow, h->sumN + 1, &out.lnnz, tmp, s));
  int32_t *wK = nullptr, *wA = nullptr;
  GENEO_TRY(tmp.get(&out.lcol, (size_t)out.lnnz));
  GENEO_TRY(tmp.get(&out.lA, (size_t)out.lnnz));
  double* lA = out.lA;
  GENEO_TRY(tmp.get(&wK, (size_t)N));
  GENEO_TRY(tmp.get(&wA, (size_t)N));
  GENEO_CUDA(cudaMemsetAsync(wK, 0, sizeof(int32_t) * N, s));
  GENEO_CUDA(cudaMemsetAsync(wA, 0, sizeof(int32_t) * N, s));
  k_local_csr<1><<<N, kT, 0, s>>>(h->dsub, h->Nlist, h->rowptr, h->col, h->val, nullptr, out.lrow,
                                  out.lcol, lA, wK); note_launch();
  k_band_width_A<<<N, kT, 0, s>>>(h->dsub, h->dpos, h->nToD, out.lrow, out.lcol, wA); note_launch();
  GENEO_CUDA(cudaGetLastError());
  std::vector<int32_t> hwK(N), hwA(N);
  GENEO_CUDA(cudaMemcpyAsync(hwK.data(), wK, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, s));
  GENEO_CUDA(cudaMemcpyAsync(hwA.data(), wA, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, s));
  GENEO_CUDA(cudaStreamSynchronize(s));
  int64_t bandK_tot = 0, bandA_tot = 0;
  out.maxwK = 0;
  h->maxwA = 0;
  h->maxnD = 0;
  for (int j = 0; j < N; ++j) {
    SubDesc& d = h->hsub[j];
    d.wK = hwK[j];
    d.wA = hwA[j];
    d.bandK = bandK_tot;
    d.bandA = bandA_tot;
    bandK_tot += (int64_t)d.nN * band_ld(d.wK);
    bandA_tot += (int64_t)d.nD * band_ld(d.wA);
    out.maxwK = std::max(out.maxwK, d.wK);
    h->maxwA = std::max(h->maxwA, d.wA);
    h->maxnD = std::max(h->maxnD, d.nD);
  }
  GENEO_CUDA(cudaMemcpyAsync(h->dsub, h->hsub.data(), sizeof(SubDesc) * N, cudaMemcpyHostToDevice, s));

  // smooth partition of unity (when chosen and no caller weights)
  if (!p->pu_weights && h->opt.pu_kind == GENEO_PU_SARKIS) {
    int32_t* dist = nullptr;
    double* total = nullptr;
    GENEO_TRY(tmp.get(&dist, (size_t)h->sumN));
    GENEO_TRY(tmp.get(&total, (size_t)n));
    k_sarkis_dist<<<N, kT, 0, s>>>(h->dsub, h->nToD, out.lrow, out.lcol, dist); note_launch();
    k_sarkis_total<<<grid_for(n), kT, 0, s>>>(n, h->invD_ptr, h->invD_sub, h->invD_loc, h->dsub, h->dpos,
                                              dist, total); note_launch();
    k_sarkis_pu<<<N, kT, 0, s>>>(h->dsub, h->Nlist, h->nToD, dist, total, h->pu); note_launch();
    GENEO_CUDA(cudaGetLastError());
  }
  // numeric assembly of Atilde_j, A_j^o, then B_j and K_j
  GENEO_TRY(tmp.get(&out.lK, (size_t)out.lnnz));
  GENEO_TRY(tmp.get(&out.lB, (size_t)out.lnnz));
  int32_t* eloc = nullptr;
  int64_t sumE = 0;
  for (const SubDesc& d : h->hsub) sumE += d.nE;
  GENEO_TRY(tmp.get(&eloc, (size_t)std::max<int64_t>(sumE * ke, 1)));
  k_elem_local<<<N, kT, 0, s>>>(h->dsub, h->Nlist, p->sub_elem, p->elem_dofs, ke, eloc); note_launch();
  k_assemble<<<N, kT, 0, s>>>(h->dsub, h->Nlist, p->sub_elem, de_ptr, de, eloc,
                              p->elem_mats, ke, a_out.e_tau, out.lrow, out.lcol, out.lK, out.lB,
                              h->dstat); note_launch();
  k_pencil<<<N, kT, 0, s>>>(h->dsub, h->pu, out.lrow, out.lcol, out.lK, out.lB, h->opt.sigma,
                            h->opt.eig_form == GENEO_EIG_FULL); note_launch();
  GENEO_CUDA(cudaGetLastError());

  // band storage, descriptors
  const size_t esz = h->fp32 ? sizeof(float) : sizeof(double);
  // the inverted diagonal blocks follow all bands in the same allocation
  // with FP32 factors the bands are equilibrated (S A S, s = diag^{-1/2}):
  // FP32 Cholesky of the unscaled matrices breaks down at coefficient
  // contrasts near 1e8; the row scalings follow the inverted blocks
  const bool equil = h->fp32;
  int64_t dinvK_tot = 0, dinvA_tot = 0;
  int maxnK = 0;
  for (const SubDesc& d : h->hsub) {
    dinvK_tot += dinv_elems(d.nN) + (equil ? scl_elems(d.nN) : 0);
    dinvA_tot += dinv_elems(d.nD) + (equil ? scl_elems(d.nD) : 0);
    maxnK = std::max(maxnK, d.nN);
  }
  GENEO_TRY(tmp.alloc(&out.bandK, esz * (size_t)std::max<int64_t>(bandK_tot + dinvK_tot, 1)));
  GENEO_TRY(h->mem.alloc(&h->bandA, esz * (size_t)std::max<int64_t>(bandA_tot + dinvA_tot, 1)));
  GENEO_CUDA(cudaMemsetAsync(out.bandK, 0, esz * bandK_tot, s));
  GENEO_CUDA(cudaMemsetAsync(h->bandA, 0, esz * bandA_tot, s));
  std::vector<BandDesc> bk(N), ba(N);
  int64_t dK = bandK_tot, dA = bandA_tot;
  for (int j = 0; j < N; ++j) {
    const SubDesc& d = h->hsub[j];
    bk[j] = BandDesc{d.bandK, d.nN, d.wK, j, band_ld(d.wK), dK, equil ? dK + dinv_elems(d.nN) : -1};
    ba[j] = BandDesc{d.bandA, d.nD, d.wA, j, band_ld(d.wA), dA, equil ? dA + dinv_elems(d.nD) : -1};
    dK += dinv_elems(d.nN) + (equil ? scl_elems(d.nN) : 0);
    dA += dinv_elems(d.nD) + (equil ? scl_elems(d.nD) : 0);
  }
  // largest factorisations first: blocks are dispatched in index order, so
  // this shortens the tail of the last wave (descriptors carry their id)
  auto by_cost = [](const BandDesc& x, const BandDesc& y) {
    const double cx = band_factor_flops(x.n, x.w), cy = band_factor_flops(y.n, y.w);
    return cx > cy || (cx == cy && x.id < y.id);
  };
  std::vector<BandDesc> bkf = bk, baf = ba;
  std::sort(bkf.begin(), bkf.end(), by_cost);
  std::sort(baf.begin(), baf.end(), by_cost);
  BandDesc *fdK = nullptr, *fdA = nullptr;
  GENEO_TRY(tmp.get(&fdK, (size_t)N));
  GENEO_TRY(tmp.get(&fdA, (size_t)N));
  GENEO_CUDA(cudaMemcpyAsync(fdK, bkf.data(), sizeof(BandDesc) * N, cudaMemcpyHostToDevice, s));
  GENEO_CUDA(cudaMemcpyAsync(fdA, baf.data(), sizeof(BandDesc) * N, cudaMemcpyHostToDevice, s));
  GENEO_TRY(tmp.get(&out.dbandK, (size_t)N));
  GENEO_TRY(h->mem.get(&h->dbandA, (size_t)N));
  GENEO_CUDA(cudaMemcpyAsync(out.dbandK, bk.data(), sizeof(BandDesc) * N, cudaMemcpyHostToDevice, s));
  GENEO_CUDA(cudaMemcpyAsync(h->dbandA, ba.data(), sizeof(BandDesc) * N, cudaMemcpyHostToDevice, s));
  out.hbandK = bk;
  out.hbandA = ba;
  if (h->fp32) {
    GENEO_TRY(tmp.get(&out.weak, (size_t)2 * N));
    GENEO_CUDA(cudaMemsetAsync(out.weak, 0, sizeof(int32_t) * 2 * N, s));
  }
  if (h->fp32) {
    k_band_fill_K<float><<<N, kT, 0, s>>>(h->dsub, out.dbandK, out.lrow, out.lcol, out.lK,
                                          (float*)out.bandK); note_launch();
    k_band_fill_A<float><<<N, kT, 0, s>>>(h->dsub, h->dbandA, h->dpos, h->nToD, out.lrow, out.lcol, lA,
                                          (float*)h->bandA); note_launch();
  } else {
    k_band_fill_K<double><<<N, kT, 0, s>>>(h->dsub, out.dbandK, out.lrow, out.lcol, out.lK,
                                           (double*)out.bandK); note_launch();
    k_band_fill_A<double><<<N, kT, 0, s>>>(h->dsub, h->dbandA, h->dpos, h->nToD, out.lrow, out.lcol, lA,
                                           (double*)h->bandA); note_launch();
  }
  GENEO_CUDA(cudaGetLastError());
  GENEO_TRY(check_status(h, s));
  *ms_assembly = ms_since(t0);

  // batched Cholesky of A_j and K_j (Sections 3 and 4.4)
  auto t1 = std::chrono::steady_clock::now();
  EventTimer ev;
  ev.start(s);
  // FP32 factors: size classes of the half bandwidth for the
  // fifth-generation tensor-core factorisation (each class padded to its own
  // W), their tiled-band planes allocated on the main stream before the fork
  std::vector<FactorBatch> batK, batA;
  const bool tc5_on = h->fp32 && h->opt.factor_kernel != 1;
  const bool bf16 = h->fp32 && h->opt.factor_bf16;
  GENEO_TRY(factor_batches(bkf, tc5_on || bf16, bf16, tmp, s, batK));
  GENEO_TRY(factor_batches(baf, tc5_on || bf16, bf16, tmp, s, batA));
  // K_j on the main stream, A_j concurrently on the auxiliary stream
  GENEO_CUDA(cudaEventRecord(h->ev_fork, s));
  GENEO_CUDA(cudaStreamWaitEvent(h->aux, h->ev_fork, 0));
  double flK = 0, flA = 0, byK = 0, byA = 0;
  for (const SubDesc& d : h->hsub) {
    flK += band_factor_flops(d.nN, d.wK);
    flA += band_factor_flops(d.nD, d.wA);
    byK += 2.0 * esz * band_entries(d.nN, d.wK);
    byA += 2.0 * esz * band_entries(d.nD, d.wA);
  }
  const int pK = h->prof.begin(GENEO_PROF_FACTOR, flK, byK, s);
  const int pA = h->prof.begin(GENEO_PROF_FACTOR, flA, byA, h->aux);
  if (h->fp32) {
    // a weak pivot flags the matrix for an FP64 factorisation instead of
    // failing the setup
    const float wt = (float)h->opt.fp32_pivot_tol;
    for (const FactorBatch& fb : batK)
      GENEO_TRY(band_potrf<float>((float*)out.bandK, fb.d, (int)fb.h.size(), fb.maxw, fb.maxn, h->dstat, s, equil,
                                  out.weak, wt, fb.plan.ok ? &fb.plan : nullptr));
    for (const FactorBatch& fb : batA)
      GENEO_TRY(band_potrf<float>((float*)h->bandA, fb.d, (int)fb.h.size(), fb.maxw, fb.maxn, h->dstat, h->aux,
                                  equil, out.weak + N, wt, fb.plan.ok ? &fb.plan : nullptr));
    h->factor_classes = (int)(batK.size() + batA.size());
  } else {
    GENEO_TRY(band_potrf<double>((double*)out.bandK, fdK, N, out.maxwK, maxnK, h->dstat, s));
    GENEO_TRY(band_potrf<double>((double*)h->bandA, fdA, N, h->maxwA, h->maxnD, h->dstat, h->aux));
  }
  h->prof.end(pK, s);
  h->prof.end(pA, h->aux);
  // the A_j factors are only needed by the solves: their factorisation keeps
  // running on the aux stream beside the eigensolver and is joined at the
  // end of the setup
  GENEO_CUDA(cudaEventRecord(h->ev_afac, h->aux));
  ev.stop();
  h->factor_ms = ev.ms;
  h->factor_flops = 0.0;
  for (const SubDesc& d : h->hsub)
    h->factor_flops += band_factor_flops(d.nD, d.wA) + band_factor_flops(d.nN, d.wK);
  GENEO_TRY(check_status(h, s));
  if (h->fp32) {
    Refactor r;
    GENEO_TRY(refactor_fp64(h, out, out.weak, true, out.hbandK, out.dbandK, tmp, s, &r));
    out.bandK64 = r.band;
    out.dbandK64 = r.desc;
    out.nK64 = h->nK64 = r.count;
    out.maxwK64 = r.maxw;
    out.maxnK64 = r.maxn;
    GENEO_TRY(check_status(h, s));
  }
  *ms_factor = ms_since(t1);
  return GENEO_OK;
}

geneo_status_t refactor_weak_A(geneo_handle_s* h, AssemblyOut& a, DevMem& tmp, cudaStream_t s) {
  if (!h->fp32 || !a.weak) return GENEO_OK;
  Refactor r;
  GENEO_TRY(refactor_fp64(h, a, a.weak + h->N, false, a.hbandA, h->dbandA, h->mem, s, &r));
  h->bandA64 = r.band;
  h->dbandA64 = r.desc;
  h->nA64 = r.count;
  h->maxwA64 = r.maxw;
  h->maxnA64 = r.maxn;
  h->a64.assign(h->N, 0);
  std::vector<BandDesc> rd(r.count);
  if (r.count) {
    GENEO_CUDA(cudaMemcpyAsync(rd.data(), r.desc, sizeof(BandDesc) * r.count, cudaMemcpyDeviceToHost, s));
    GENEO_CUDA(cudaStreamSynchronize(s));
  }
  for (const BandDesc& b : rd) h->a64[b.id] = 1;
  (void)tmp;
  return GENEO_OK;
}

}  // namespace geneo
