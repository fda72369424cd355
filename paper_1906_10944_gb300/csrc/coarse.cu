// Coarse space: basis Z, coarse matrix A_H = Z^T A Z and its factor.
//
// Definition 4 and Section 4.4: the coarse basis vectors are R_j^T X_j p_k
// normalised in l2; the sign is fixed so that the entry of largest
// magnitude is positive (first such entry on ties).  Z_j is stored on the
// rows D_j, where X_j is non-zero.
// Section 4.5: (A_H)_{ik} = phi_i^T A phi_k is zero unless the supports meet;
// Y_j = A R_j^T Z_j lives on N_j (the rows of A touching D_j), so block
// (i, j) is the sum over dofs of D_i that are in N_j.  Blocks are computed
// one thread block per subdomain pair, each output entry summed by one thread
// in ascending row order (deterministic), and written into the banded
// storage of A_H (coarse dofs ordered by subdomain).
#include <algorithm>
#include <chrono>

#include "handle.cuh"

namespace geneo {
namespace {

constexpr int kT = 256;
constexpr int kChunk = 64;
constexpr int kMaxM = 40;

// Z_j[:, k] = X_j P[:, k] restricted to D_j, l2-normalised, sign-fixed.
__global__ void __launch_bounds__(kT)
k_basis(const SubDesc* __restrict__ sub, const double* __restrict__ X, int W, const double* __restrict__ pu,
        const int32_t* __restrict__ dpos, double* __restrict__ Z) {
  const int j = blockIdx.x;
  const SubDesc d = sub[j];
  __shared__ double red[kT / 32];
  __shared__ double best_v[kT / 32];
  __shared__ int best_i[kT / 32];
  const double* xj = X + d.offN * (int64_t)W;
  double* zj = Z + d.offZ;
  for (int k = 0; k < d.m; ++k) {
    const double* xc = xj + (int64_t)k * d.nN;
    double* zc = zj + (int64_t)k * d.nD;
    double ss = 0.0, bv = -1.0;
    int bi = 0x7fffffff;
    for (int i = threadIdx.x; i < d.nD; i += blockDim.x) {
      const int a = dpos[d.offN + i];
      const double v = pu[d.offN + a] * xc[a];
      zc[i] = v;
      ss += v * v;
      const double av = fabs(v);
      if (av > bv) { bv = av; bi = i; }
    }
    const double nrm2 = block_sum(ss, red);
    // argmax |v|, smallest index on ties
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { best_v[wid] = bv; best_i[wid] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double v0 = best_v[0];
      int i0 = best_i[0];
      for (int w2 = 1; w2 < (int)(blockDim.x >> 5); ++w2)
        if (best_v[w2] > v0 || (best_v[w2] == v0 && best_i[w2] < i0)) { v0 = best_v[w2]; i0 = best_i[w2]; }
      best_i[0] = i0;
    }
    __syncthreads();
    const int imax = best_i[0];
    const double nrm = sqrt(nrm2);
    const double sgn = (imax < d.nD && zc[imax] < 0.0) ? -1.0 : 1.0;
    const double scale = nrm > 0.0 ? sgn / nrm : 0.0;
    __syncthreads();
    for (int i = threadIdx.x; i < d.nD; i += blockDim.x) zc[i] *= scale;
    __syncthreads();
  }
}

// Y_j = A R_j^T Z_j on the N-rows of subdomain j (local pattern holds A).
__global__ void __launch_bounds__(kT)
k_AZ(const SubDesc* __restrict__ sub, const int64_t* __restrict__ lrow, const int32_t* __restrict__ lcol,
     const double* __restrict__ lA, const int32_t* __restrict__ nToD, const double* __restrict__ Z,
     double* __restrict__ Y) {
  const int j = blockIdx.y;
  const SubDesc d = sub[j];
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= d.nN || d.m == 0) return;
  const int64_t e0 = lrow[d.offN + a], e1 = lrow[d.offN + a + 1];
  const double* zj = Z + d.offZ;
  for (int c = 0; c < d.m; ++c) {
    double acc = 0.0;
    for (int64_t e = e0; e < e1; ++e) {
      const int di = nToD[d.offN + lcol[e]];
      if (di >= 0) acc += lA[e] * zj[(int64_t)c * d.nD + di];
    }
    Y[d.offY + (int64_t)c * d.nN + a] = acc;
  }
}

// mark[i*N + j] = 1 when D_i meets N_j
__global__ void k_pairs(const SubDesc* __restrict__ sub, const int32_t* __restrict__ Nlist,
                        const int64_t* __restrict__ invD_ptr, const int32_t* __restrict__ invD_sub,
                        int nsub, uint8_t* __restrict__ mark) {
  const int j = blockIdx.x;
  const SubDesc d = sub[j];
  for (int a = threadIdx.x; a < d.nN; a += blockDim.x) {
    const int32_t k = Nlist[d.offN + a];
    for (int64_t t = invD_ptr[k]; t < invD_ptr[k + 1]; ++t) mark[(int64_t)invD_sub[t] * nsub + j] = 1;
  }
}

// Block (i, j) of A_H = Z_i^T Y_j over rows k in D_i and N_j; i >= j.
__global__ void __launch_bounds__(kT)
k_coarse_block(const SubDesc* __restrict__ sub, const int2* __restrict__ pairs,
               const int32_t* __restrict__ Nlist, const int64_t* __restrict__ invD_ptr,
               const int32_t* __restrict__ invD_sub, const int32_t* __restrict__ invD_loc,
               const double* __restrict__ Z, const double* __restrict__ Y, double* __restrict__ band,
               int wH) {
  const int2 pr = pairs[blockIdx.x];
  const int i = pr.x, j = pr.y;
  const SubDesc di = sub[i], dj = sub[j];
  const int mi = di.m, mj = dj.m;
  __shared__ int rowD[kChunk];
  __shared__ double Zs[kChunk][kMaxM];
  __shared__ double Ys[kChunk][kMaxM];
  constexpr int kOut = (kMaxM * kMaxM + kT - 1) / kT;
  double acc[kOut];
#pragma unroll
  for (int u = 0; u < kOut; ++u) acc[u] = 0.0;
  const double* zi = Z + di.offZ;
  const double* yj = Y + dj.offY;
  for (int base = 0; base < dj.nN; base += kChunk) {
    const int nr = min(kChunk, dj.nN - base);
    __syncthreads();
    if (threadIdx.x < kChunk) {
      int found = -1;
      if ((int)threadIdx.x < nr) {
        const int32_t k = Nlist[dj.offN + base + threadIdx.x];
        for (int64_t t = invD_ptr[k]; t < invD_ptr[k + 1]; ++t)
          if (invD_sub[t] == i) { found = invD_loc[t]; break; }
      }
      rowD[threadIdx.x] = found;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < kChunk * mi; idx += blockDim.x) {
      const int r = idx % kChunk, c = idx / kChunk;
      Zs[r][c] = (r < nr && rowD[r] >= 0) ? zi[(int64_t)c * di.nD + rowD[r]] : 0.0;
    }
    for (int idx = threadIdx.x; idx < kChunk * mj; idx += blockDim.x) {
      const int r = idx % kChunk, c = idx / kChunk;
      Ys[r][c] = (r < nr && rowD[r] >= 0) ? yj[(int64_t)c * dj.nN + base + r] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kOut; ++u) {
      const int o = threadIdx.x + u * kT;
      if (o >= mi * mj) continue;
      const int a = o % mi, b = o / mi;
      double s = acc[u];
      for (int r = 0; r < nr; ++r) s += Zs[r][a] * Ys[r][b];
      acc[u] = s;
    }
  }
  const int64_t ld = band_ld(wH);
#pragma unroll
  for (int u = 0; u < kOut; ++u) {
    const int o = threadIdx.x + u * kT;
    if (o >= mi * mj) continue;
    const int a = o % mi, b = o / mi;
    const int r = di.offH + a, c = dj.offH + b;
    if (r >= c && r - c <= wH) band[(int64_t)r * ld + (c - r + wH)] = acc[u];
  }
}

inline double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// X = I (dim x dim, column-major)
__global__ void k_identity(double* __restrict__ X, int dim) {
  const int64_t tot = (int64_t)dim * dim;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x)
    X[i] = (i % dim == i / dim) ? 1.0 : 0.0;
}

}  // namespace


geneo_status_t build_coarse(geneo_handle_s* h, const AssemblyOut& asmb, const double* X, DevMem& tmp,
                            cudaStream_t s, double* ms_basis, double* ms_matrix, double* ms_factor) {
  auto t0 = std::chrono::steady_clock::now();
  const int N = h->N;
  const geneo_options_t& o = h->opt;
  // selection (Theorem 1 with the threshold tau, capped at nev_max)
  int off = 0;
  int64_t zoff = 0, yoff = 0;
  h->maxm = 0;
  int maxn = 0;
  for (int j = 0; j < N; ++j) {
    SubDesc& d = h->hsub[j];
    int m = 0;
    const int lim = std::min(o.nev_max, d.s);
    if (o.fixed_nev) {
      m = lim;
    } else {
      while (m < lim && h->lambda_host[(size_t)j * h->s_block + m] < o.tau) ++m;
    }
    d.m = m;
    d.offH = off;
    d.offZ = zoff;
    d.offY = yoff;
    off += m;
    zoff += (int64_t)d.nD * m;
    yoff += (int64_t)d.nN * m;
    h->maxm = std::max(h->maxm, m);
    maxn = std::max(maxn, d.nN);
  }
  if (h->maxm > kMaxM) return GENEO_ERR_ARG;
  h->dimH = off;
  GENEO_CUDA(cudaMemcpyAsync(h->dsub, h->hsub.data(), sizeof(SubDesc) * N, cudaMemcpyHostToDevice, s));
  GENEO_TRY(h->mem.get(&h->Z, (size_t)std::max<int64_t>(zoff, 1)));
  if (h->dimH == 0) {
    *ms_basis = ms_since(t0);
    return GENEO_OK;
  }
  k_basis<<<N, kT, 0, s>>>(h->dsub, X, 3 * h->s_block, h->pu, h->dpos, h->Z); note_launch();
  GENEO_CUDA(cudaGetLastError());
  GENEO_TRY(check_status(h, s));
  *ms_basis = ms_since(t0);

  auto t1 = std::chrono::steady_clock::now();
  double* Y = nullptr;
  GENEO_TRY(tmp.get(&Y, (size_t)yoff));
  k_AZ<<<dim3(ceil_div(maxn, kT), N), kT, 0, s>>>(h->dsub, asmb.lrow, asmb.lcol, asmb.lA, h->nToD,
                                                   h->Z, Y); note_launch();
  uint8_t* mark = nullptr;
  GENEO_TRY(tmp.get(&mark, (size_t)N * N));
  GENEO_CUDA(cudaMemsetAsync(mark, 0, (size_t)N * N, s));
  k_pairs<<<N, kT, 0, s>>>(h->dsub, h->Nlist, h->invD_ptr, h->invD_sub, N, mark); note_launch();
  GENEO_CUDA(cudaGetLastError());
  std::vector<uint8_t> hmark((size_t)N * N);
  GENEO_CUDA(cudaMemcpyAsync(hmark.data(), mark, (size_t)N * N, cudaMemcpyDeviceToHost, s));
  GENEO_CUDA(cudaStreamSynchronize(s));
  std::vector<int2> pairs;
  int wH = 0;
  for (int i = 0; i < N; ++i) {
    const SubDesc& di = h->hsub[i];
    if (di.m == 0) continue;
    for (int j = 0; j <= i; ++j) {
      const SubDesc& dj = h->hsub[j];
      if (dj.m == 0 || !hmark[(size_t)i * N + j]) continue;
      pairs.push_back(make_int2(i, j));
      wH = std::max(wH, di.offH + di.m - 1 - dj.offH);
    }
  }
  h->wH = wH;
  GENEO_TRY(h->mem.get(&h->bandH, (size_t)h->dimH * band_ld(wH) + dinv_elems(h->dimH)));
  GENEO_CUDA(cudaMemsetAsync(h->bandH, 0, sizeof(double) * h->dimH * band_ld(wH), s));
  int2* dpairs = nullptr;
  GENEO_TRY(tmp.get(&dpairs, pairs.size()));
  GENEO_CUDA(cudaMemcpyAsync(dpairs, pairs.data(), sizeof(int2) * pairs.size(), cudaMemcpyHostToDevice, s));
  k_coarse_block<<<(unsigned)pairs.size(), kT, 0, s>>>(h->dsub, dpairs, h->Nlist, h->invD_ptr,
                                                       h->invD_sub, h->invD_loc, h->Z, Y, h->bandH, wH); note_launch();
  GENEO_CUDA(cudaGetLastError());
  GENEO_TRY(check_status(h, s));
  *ms_matrix = ms_since(t1);

  auto t2 = std::chrono::steady_clock::now();
  BandDesc bh{0, h->dimH, wH, -2, band_ld(wH), (int64_t)h->dimH * band_ld(wH), -1};
  GENEO_TRY(h->mem.get(&h->dbandH, 1));
  GENEO_CUDA(cudaMemcpyAsync(h->dbandH, &bh, sizeof(BandDesc), cudaMemcpyHostToDevice, s));
  const int pf = h->prof.begin(GENEO_PROF_FACTOR, band_factor_flops(h->dimH, wH),
                               2.0 * 8.0 * band_entries(h->dimH, wH), s);
  GENEO_TRY(band_potrf<double>(h->bandH, h->dbandH, 1, wH, h->dimH, h->dstat, s));
  h->prof.end(pf, s);
  GENEO_TRY(check_status(h, s));
  // The preconditioner's coarse solve A_H y = c runs on one small band, a
  // chain of dependent steps on one SM; instead A_H^{-1} is formed once here
  // (A_H X = I solved with the factor, 16 columns per block, all column
  // blocks in one launch) and each apply is a dense FP64 matrix-vector
  // product spread over the GPU.  Kept up to 16384 coarse dofs (2 GB).
  if (h->dimH <= 16384) {
    const int dim = h->dimH, nc = (dim + 15) / 16;
    std::vector<BandDesc> rep(nc, bh);
    std::vector<int64_t> xo(nc);
    std::vector<int32_t> cnt(nc);
    for (int i = 0; i < nc; ++i) {
      rep[i].id = -1;  // vectors indexed by the position in the batch
      xo[i] = (int64_t)i * 16 * dim;
      cnt[i] = std::min(16, dim - 16 * i);
    }
    BandDesc* drep = nullptr;
    int64_t* dxo = nullptr;
    int32_t* dcnt = nullptr;
    GENEO_TRY(tmp.get(&drep, (size_t)nc));
    GENEO_TRY(tmp.get(&dxo, (size_t)nc));
    GENEO_TRY(tmp.get(&dcnt, (size_t)nc));
    GENEO_TRY(h->mem.get(&h->Hinv, (size_t)dim * dim));
    GENEO_TRY(h->mem.get(&h->yH, (size_t)dim));
    GENEO_CUDA(cudaMemcpyAsync(drep, rep.data(), sizeof(BandDesc) * nc, cudaMemcpyHostToDevice, s));
    GENEO_CUDA(cudaMemcpyAsync(dxo, xo.data(), sizeof(int64_t) * nc, cudaMemcpyHostToDevice, s));
    GENEO_CUDA(cudaMemcpyAsync(dcnt, cnt.data(), sizeof(int32_t) * nc, cudaMemcpyHostToDevice, s));
    k_identity<<<(unsigned)std::min<int64_t>(((int64_t)dim * dim + kT - 1) / kT, 152 * 16), kT, 0, s>>>(
        h->Hinv, dim); note_launch();
    GENEO_CUDA(cudaGetLastError());
    // FP32 mode: the columns of A_H^{-1} in double-single arithmetic on the
    // FP32 pipe (about 46 bits; GB300 issues FP64 at 1/64 of the FP32 rate),
    // an error far below the FP32 local solves' beside it in M^{-1}
    if (h->fp32)
      GENEO_TRY(band_solve_ds(h->bandH, drep, nc, wH, h->Hinv, dxo, 16, dcnt, nullptr, h->dstat, s, 0));
    else
      GENEO_TRY(band_solve<double>(h->bandH, drep, nc, wH, h->Hinv, dxo, 16, dcnt, nullptr, h->dstat, s, 0));
    GENEO_TRY(check_status(h, s));
  }
  *ms_factor = ms_since(t2);
  tmp.release(Y);
  return GENEO_OK;
}

}  // namespace geneo
