// Overlapping subdomains from a non-overlapping element partition.
//
// Section 3: each part Omega'_j (a union of elements) is grown by a number
// of element layers; one layer adds every element that shares a vertex with
// the current set.  The dof lists hold the dofs of the grown subdomain's
// elements (its closure) without global Dirichlet dofs.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

#include "geneo.h"

namespace {

template <typename T>
T* copy_out(const std::vector<T>& v) {
  T* p = static_cast<T*>(std::malloc(sizeof(T) * std::max<size_t>(v.size(), 1)));
  if (p && !v.empty()) std::memcpy(p, v.data(), sizeof(T) * v.size());
  return p;
}

}  // namespace

extern "C" geneo_status_t geneo_grow_partition(int64_t n, int64_t n_elem, int32_t elem_ndof,
                                               const int32_t* elem_dofs, const uint8_t* dirichlet,
                                               const int32_t* part, int32_t n_parts, int32_t overlap,
                                               int64_t** sub_elem_ptr, int32_t** sub_elem,
                                               int64_t** sub_dof_ptr, int32_t** sub_dof) {
  if (n <= 0 || n_elem <= 0 || elem_ndof <= 0 || !elem_dofs || !dirichlet || !part || n_parts <= 0 ||
      overlap < 0 || !sub_elem_ptr || !sub_elem || !sub_dof_ptr || !sub_dof)
    return GENEO_ERR_ARG;
  for (int64_t e = 0; e < n_elem; ++e)
    if (part[e] < 0 || part[e] >= n_parts) return GENEO_ERR_ARG;
  for (int64_t i = 0; i < n_elem * elem_ndof; ++i)
    if (elem_dofs[i] < 0 || elem_dofs[i] >= n) return GENEO_ERR_ARG;
  // dof -> elements
  std::vector<int64_t> dptr(n + 1, 0);
  for (int64_t i = 0; i < n_elem * elem_ndof; ++i) ++dptr[elem_dofs[i] + 1];
  for (int64_t k = 0; k < n; ++k) dptr[k + 1] += dptr[k];
  std::vector<int32_t> delem(dptr[n]);
  {
    std::vector<int64_t> cur(dptr.begin(), dptr.end() - 1);
    for (int64_t e = 0; e < n_elem; ++e)
      for (int a = 0; a < elem_ndof; ++a) {
        const int32_t k = elem_dofs[e * elem_ndof + a];
        if (cur[k] == dptr[k] || delem[cur[k] - 1] != (int32_t)e) delem[cur[k]++] = (int32_t)e;
      }
    // unused tail entries (an element listing a dof twice) stay beyond cur; mark them
    for (int64_t k = 0; k < n; ++k)
      for (int64_t t = cur[k]; t < dptr[k + 1]; ++t) delem[t] = -1;
  }
  // initial parts
  std::vector<std::vector<int32_t>> elems(n_parts), dofs(n_parts);
  for (int64_t e = 0; e < n_elem; ++e) elems[part[e]].push_back((int32_t)e);
  const int nthreads = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  auto work = [&](int tid) {
    std::vector<uint32_t> emark(n_elem, 0), dmark(n, 0);
    uint32_t stamp = 0;
    for (int p = tid; p < n_parts; p += nthreads) {
      std::vector<int32_t> cur = elems[p];
      for (int layer = 0; layer < overlap; ++layer) {
        ++stamp;
        for (int32_t e : cur) emark[e] = stamp;
        std::vector<int32_t> next = cur;
        for (int32_t e : cur)
          for (int a = 0; a < elem_ndof; ++a) {
            const int32_t k = elem_dofs[(int64_t)e * elem_ndof + a];
            if (dmark[k] == stamp) continue;
            dmark[k] = stamp;
            for (int64_t t = dptr[k]; t < dptr[k + 1]; ++t) {
              const int32_t e2 = delem[t];
              if (e2 >= 0 && emark[e2] != stamp) {
                emark[e2] = stamp;
                next.push_back(e2);
              }
            }
          }
        cur.swap(next);
      }
      std::sort(cur.begin(), cur.end());
      ++stamp;
      std::vector<int32_t> dl;
      for (int32_t e : cur)
        for (int a = 0; a < elem_ndof; ++a) {
          const int32_t k = elem_dofs[(int64_t)e * elem_ndof + a];
          if (dmark[k] != stamp && !dirichlet[k]) {
            dmark[k] = stamp;
            dl.push_back(k);
          }
        }
      std::sort(dl.begin(), dl.end());
      elems[p].swap(cur);
      dofs[p].swap(dl);
    }
  };
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t) th.emplace_back(work, t);
  for (auto& t : th) t.join();
  std::vector<int64_t> ep(n_parts + 1, 0), dp(n_parts + 1, 0);
  std::vector<int32_t> ev, dv;
  for (int p = 0; p < n_parts; ++p) {
    ep[p + 1] = ep[p] + (int64_t)elems[p].size();
    dp[p + 1] = dp[p] + (int64_t)dofs[p].size();
    ev.insert(ev.end(), elems[p].begin(), elems[p].end());
    dv.insert(dv.end(), dofs[p].begin(), dofs[p].end());
  }
  *sub_elem_ptr = copy_out(ep);
  *sub_elem = copy_out(ev);
  *sub_dof_ptr = copy_out(dp);
  *sub_dof = copy_out(dv);
  if (!*sub_elem_ptr || !*sub_elem || !*sub_dof_ptr || !*sub_dof) {
    std::free(*sub_elem_ptr);
    std::free(*sub_elem);
    std::free(*sub_dof_ptr);
    std::free(*sub_dof);
    *sub_elem_ptr = nullptr;
    *sub_elem = nullptr;
    *sub_dof_ptr = nullptr;
    *sub_dof = nullptr;
    return GENEO_ERR_OOM;
  }
  return GENEO_OK;
}
