// C ABI: argument checking, setup orchestration and handle lifetime.
#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <new>

#include "handle.cuh"

using geneo::DevMem;
using geneo::SubDesc;

namespace geneo {

geneo_status_t check_status(geneo_handle_s* h, cudaStream_t s) {
  GENEO_CUDA(cudaStreamSynchronize(s));
  GENEO_CUDA(cudaMemcpy(&h->hstat, h->dstat, sizeof(DevStatus), cudaMemcpyDeviceToHost));
  if (h->hstat.code != 0) return (geneo_status_t)h->hstat.code;
  return GENEO_OK;
}

}  // namespace geneo

namespace {

// details of the last geneo_setup on this thread that failed (its handle is
// gone by then), for geneo_last_error(NULL, ...)
thread_local geneo::DevStatus g_setup_error{0, 0, 0};

double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// Copy (or reference) one problem array on the device.
template <typename T>
geneo_status_t to_device(const T* src, int64_t count, bool host, DevMem& tmp, cudaStream_t s,
                         const T** out) {
  if (!host) {
    *out = src;
    return GENEO_OK;
  }
  T* d = nullptr;
  GENEO_TRY(tmp.get(&d, (size_t)std::max<int64_t>(count, 1)));
  if (count > 0) GENEO_CUDA(cudaMemcpyAsync(d, src, sizeof(T) * count, cudaMemcpyHostToDevice, s));
  *out = d;
  return GENEO_OK;
}

template <typename T>
geneo_status_t to_host(const T* src, int64_t count, bool host, cudaStream_t s, std::vector<T>& out) {
  out.resize(count);
  if (host) {
    std::memcpy(out.data(), src, sizeof(T) * count);
    return GENEO_OK;
  }
  GENEO_CUDA(cudaMemcpyAsync(out.data(), src, sizeof(T) * count, cudaMemcpyDeviceToHost, s));
  GENEO_CUDA(cudaStreamSynchronize(s));
  return GENEO_OK;
}

geneo_status_t setup_impl(geneo_handle_s* h, const geneo_problem_t* p, cudaStream_t s) {
  auto t_all = std::chrono::steady_clock::now();
  const bool host = p->mem == GENEO_MEM_HOST;
  DevMem tmp;
  tmp.stream = s;
  h->mem.stream = s;
  // on every exit: the aux stream (A_j factorisation) finishes before the
  // temporaries it may read are freed
  struct Guard {
    DevMem& t;
    cudaStream_t a;
    ~Guard() {
      if (a) cudaStreamSynchronize(a);
      t.free_all();
    }
  } guard{tmp, h->aux};
  h->n = p->n;
  h->nnz = p->nnz;
  h->N = p->n_sub;
  const int N = h->N;
  // host copies of the subdomain offsets
  std::vector<int64_t> sep, sdp;
  GENEO_TRY(to_host(p->sub_elem_ptr, N + 1, host, s, sep));
  GENEO_TRY(to_host(p->sub_dof_ptr, N + 1, host, s, sdp));
  if (sep[0] != 0 || sdp[0] != 0) return GENEO_ERR_ARG;
  h->hsub.assign(N, SubDesc{});
  for (int j = 0; j < N; ++j) {
    SubDesc& d = h->hsub[j];
    d.offE = sep[j];
    d.nE = (int32_t)(sep[j + 1] - sep[j]);
    d.offN = sdp[j];
    d.nN = (int32_t)(sdp[j + 1] - sdp[j]);
    if (d.nE <= 0 || d.nN <= 0) return GENEO_ERR_ARG;
  }
  h->sumN = sdp[N];
  // device views of the inputs
  geneo_problem_t dp = *p;
  GENEO_TRY(to_device(p->elem_dofs, p->n_elem * p->elem_ndof, host, tmp, s, &dp.elem_dofs));
  GENEO_TRY(to_device(p->elem_mats, p->n_elem * p->elem_ndof * p->elem_ndof, host, tmp, s, &dp.elem_mats));
  GENEO_TRY(to_device(p->sub_elem, sep[N], host, tmp, s, &dp.sub_elem));
  GENEO_TRY(to_device(p->sub_dof, sdp[N], host, tmp, s, &dp.sub_dof));
  if (p->pu_weights) GENEO_TRY(to_device(p->pu_weights, sdp[N], host, tmp, s, &dp.pu_weights));
  // the handle keeps A and the Dirichlet mask
  DevMem& M = h->mem;
  GENEO_TRY(M.get(&h->rowptr, (size_t)h->n + 1));
  GENEO_TRY(M.get(&h->col, (size_t)h->nnz));
  GENEO_TRY(M.get(&h->val, (size_t)h->nnz));
  GENEO_TRY(M.get(&h->dir, (size_t)h->n));
  const cudaMemcpyKind kind = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  GENEO_CUDA(cudaMemcpyAsync(h->rowptr, p->row_ptr, sizeof(int64_t) * (h->n + 1), kind, s));
  GENEO_CUDA(cudaMemcpyAsync(h->col, p->col, sizeof(int32_t) * h->nnz, kind, s));
  GENEO_CUDA(cudaMemcpyAsync(h->val, p->val, sizeof(double) * h->nnz, kind, s));
  GENEO_CUDA(cudaMemcpyAsync(h->dir, p->dirichlet, sizeof(uint8_t) * h->n, kind, s));
  GENEO_TRY(M.get(&h->dstat, 1));
  GENEO_CUDA(cudaMemsetAsync(h->dstat, 0, sizeof(geneo::DevStatus), s));
  GENEO_TRY(M.get(&h->dsub, (size_t)N));
  GENEO_CUDA(cudaMemcpyAsync(h->dsub, h->hsub.data(), sizeof(SubDesc) * N, cudaMemcpyHostToDevice, s));

  // a1: D_j, multiplicities, partition of unity, inverse map
  auto t0 = std::chrono::steady_clock::now();
  geneo::AssemblyOut asmb;
  GENEO_TRY(geneo::build_structure(h, &dp, asmb, tmp, s));
  h->setup_ms[0] = ms_since(t0);
  // a2-a4: local matrices and factorisations
  GENEO_TRY(geneo::assemble_local(h, &dp, asmb, tmp, s, &h->setup_ms[1], &h->setup_ms[2]));
  // a5: local eigenproblems
  double* X = nullptr;
  if (h->opt.nev_max > 0) {
    int64_t unused = 0;
    GENEO_TRY(geneo::local_eigensolve(h, asmb, tmp, s, &X, &unused));
  } else {
    h->lambda_host.clear();
    for (auto& d : h->hsub) d.s = 0;
  }
  // eigensolver cap reached: an error only when the caller asks for it
  if (h->opt.eig_strict && h->eig_unconv > 0) return GENEO_ERR_EIG_NOCONV;
  // a6-a7: coarse basis, coarse matrix, factorisation
  GENEO_TRY(geneo::build_coarse(h, asmb, X, tmp, s, &h->setup_ms[4], &h->setup_ms[5], &h->setup_ms[6]));
  // join the A_j factorisation (aux stream) before the temporaries go; A_j
  // whose FP32 factor had a weak pivot are factored again in FP64
  GENEO_CUDA(cudaStreamWaitEvent(s, h->ev_afac, 0));
  GENEO_TRY(geneo::check_status(h, s));
  GENEO_TRY(geneo::refactor_weak_A(h, asmb, tmp, s));
  GENEO_TRY(geneo::alloc_solver(h));
  GENEO_TRY(geneo::check_status(h, s));
  if (h->opt.autotune) GENEO_TRY(geneo::tune_local_solve(h));
  h->setup_ms[7] = ms_since(t_all);
  h->prof.collect();
  return GENEO_OK;
}

}  // namespace

extern "C" {

void geneo_default_options(geneo_options_t* o) {
  if (!o) return;
  o->tau = 0.3;
  o->sigma = -0.01;
  o->eig_tol = 1e-6;
  o->nev_max = 10;
  o->fixed_nev = 0;
  o->eig_form = GENEO_EIG_PAPER;
  o->eig_maxit = 100;
  o->guard = -1;
  o->precision = GENEO_PREC_FP64;
  o->profile = 0;
  o->first_nev = -1;
  o->fp32_pivot_tol = 1e-4;
  o->seed = 0x5EED5EEDull;
  o->pu_kind = GENEO_PU_STANDARD;
  o->eig_strict = 0;
  o->deterministic = 1;
  o->eig_solve_tf32 = 1;
  o->factor_kernel = 0;
  o->autotune = 1;
  o->factor_bf16 = 0;
  o->reserved = 0;
}

geneo_status_t geneo_setup(const geneo_problem_t* prob, const geneo_options_t* opt, void* stream,
                           geneo_handle_t* out) {
  if (!out) return GENEO_ERR_ARG;
  *out = nullptr;
  if (!prob || prob->n <= 0 || prob->nnz <= 0 || prob->n_sub <= 0 || prob->n_elem <= 0 ||
      prob->elem_ndof <= 0 || prob->elem_ndof > 64 || !prob->row_ptr || !prob->col || !prob->val ||
      !prob->dirichlet || !prob->elem_dofs || !prob->elem_mats || !prob->sub_elem_ptr ||
      !prob->sub_elem || !prob->sub_dof_ptr || !prob->sub_dof ||
      (prob->mem != GENEO_MEM_HOST && prob->mem != GENEO_MEM_DEVICE) || prob->n > INT32_MAX)
    return GENEO_ERR_ARG;
  geneo_options_t o;
  geneo_default_options(&o);
  if (opt) o = *opt;
  if (o.nev_max < 0 || o.nev_max > 34 || !(o.sigma < 0.0) || !(o.eig_tol > 0.0) || o.eig_maxit < 1 ||
      !(o.fp32_pivot_tol >= 0.0 && o.fp32_pivot_tol < 1.0) ||
      (o.eig_form != GENEO_EIG_PAPER && o.eig_form != GENEO_EIG_FULL) ||
      (o.precision != GENEO_PREC_FP64 && o.precision != GENEO_PREC_FP32) ||
      (o.pu_kind != GENEO_PU_STANDARD && o.pu_kind != GENEO_PU_SARKIS) ||
      (o.eig_strict != 0 && o.eig_strict != 1) || (o.deterministic != 0 && o.deterministic != 1) ||
      (o.eig_solve_tf32 != 0 && o.eig_solve_tf32 != 1) || (o.factor_kernel != 0 && o.factor_kernel != 1) ||
      (o.autotune != 0 && o.autotune != 1) || (o.factor_bf16 != 0 && o.factor_bf16 != 1) || o.reserved != 0)
    return GENEO_ERR_ARG;
  // keep freed device memory in the stream-ordered pool for the next setup
  {
    int dev = 0;
    cudaMemPool_t pool;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
  }
  geneo_handle_s* h = new (std::nothrow) geneo_handle_s();
  if (!h) return GENEO_ERR_OOM;
  h->opt = o;
  h->fp32 = o.precision == GENEO_PREC_FP32;
  h->prof.on = o.profile != 0;
  const int guard = o.guard >= 0 ? o.guard : std::min(3, o.nev_max);
  h->s_block = std::min(o.nev_max + guard, 34);
  h->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return GENEO_ERR_CUDA;
  }
  if (cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_afac, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->solve_streams.fork, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    geneo_destroy(h);
    return GENEO_ERR_CUDA;
  }
  for (int i = 0; i < geneo::kSolveStreams; ++i)
    if (cudaStreamCreateWithFlags(&h->solve_streams.s[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->solve_streams.ev[i], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      geneo_destroy(h);
      return GENEO_ERR_CUDA;
    }
  geneo_status_t st = setup_impl(h, prob, h->stream);
  if (st != GENEO_OK) {
    cudaStreamSynchronize(h->stream);
    g_setup_error = h->hstat;
    if (g_setup_error.code == 0) g_setup_error = geneo::DevStatus{(int32_t)st, -1, -1};
    geneo_destroy(h);
    return st;
  }
  g_setup_error = geneo::DevStatus{0, 0, 0};
  *out = h;
  return GENEO_OK;
}

geneo_status_t geneo_apply(geneo_handle_t h, const double* r_dev, double* z_dev, int32_t nrhs,
                           void* stream) {
  if (!h || !r_dev || !z_dev || nrhs < 0) return GENEO_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  h->mem.stream = s;  // the handle's last stream (see geneo_destroy)
  for (int i = 0; i < nrhs; ++i)
    GENEO_TRY(geneo::apply_prec(h, r_dev + (int64_t)i * h->n, z_dev + (int64_t)i * h->n, s));
  return GENEO_OK;
}

geneo_status_t geneo_pcg_solve(geneo_handle_t h, const double* b, double* x, int32_t nrhs, double tol,
                               int32_t maxit, int32_t mem, geneo_solve_info_t* info, void* stream) {
  if (!h || !b || !x || nrhs < 0 || !(tol > 0.0) || maxit < 0 ||
      (mem != GENEO_MEM_HOST && mem != GENEO_MEM_DEVICE))
    return GENEO_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = h->n;
  geneo_status_t worst = GENEO_OK;
  double *db = nullptr, *dx = nullptr;
  DevMem tmp;
  tmp.stream = s;
  // several right-hand sides: solved together, up to kBlk at a time (the
  // dense coarse inverse is needed, which every coarse space up to 16384
  // vectors has)
  if (nrhs >= 2 && (h->dimH == 0 || h->Hinv)) {
    const int kb = std::min(nrhs, geneo::kBlk);
    if (mem == GENEO_MEM_HOST) {
      GENEO_TRY(tmp.get(&db, (size_t)n * kb));
      GENEO_TRY(tmp.get(&dx, (size_t)n * kb));
    }
    for (int i0 = 0; i0 < nrhs; i0 += kb) {
      const int k = std::min(kb, nrhs - i0);
      const double* bi = b + (int64_t)i0 * n;
      double* xi = x + (int64_t)i0 * n;
      if (mem == GENEO_MEM_HOST) {
        cudaError_t e = cudaMemcpyAsync(db, bi, sizeof(double) * n * k, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) { tmp.free_all(); return GENEO_ERR_CUDA; }
        bi = db;
        xi = dx;
      }
      geneo_status_t st = geneo::pcg_block(h, bi, xi, k, tol, maxit, info, s);
      if (mem == GENEO_MEM_HOST) {
        cudaError_t e = cudaMemcpyAsync(x + (int64_t)i0 * n, dx, sizeof(double) * n * k, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { tmp.free_all(); return GENEO_ERR_CUDA; }
      }
      if (st != GENEO_OK && worst == GENEO_OK) worst = st;
      if (st == GENEO_ERR_CUDA || st == GENEO_ERR_OOM || st == GENEO_ERR_ARG) break;
    }
    tmp.free_all();
    return worst;
  }
  if (mem == GENEO_MEM_HOST) {
    GENEO_TRY(tmp.get(&db, (size_t)n));
    GENEO_TRY(tmp.get(&dx, (size_t)n));
  }
  for (int i = 0; i < nrhs; ++i) {
    const double* bi = b + (int64_t)i * n;
    double* xi = x + (int64_t)i * n;
    if (mem == GENEO_MEM_HOST) {
      cudaError_t e = cudaMemcpyAsync(db, bi, sizeof(double) * n, cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) { tmp.free_all(); return GENEO_ERR_CUDA; }
      bi = db;
      xi = dx;
    }
    geneo_status_t st = geneo::pcg(h, bi, xi, tol, maxit, info, s);
    if (mem == GENEO_MEM_HOST) {
      cudaError_t e = cudaMemcpyAsync(x + (int64_t)i * n, dx, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) { tmp.free_all(); return GENEO_ERR_CUDA; }
    }
    if (st != GENEO_OK && worst == GENEO_OK) worst = st;
  }
  tmp.free_all();
  return worst;
}

geneo_status_t geneo_query(geneo_handle_t h, geneo_coarse_info_t* info) {
  if (!h || !info) return GENEO_ERR_ARG;
  info->n_sub = h->N;
  info->dim_coarse = h->dimH;
  info->coarse_bandwidth = h->wH;
  info->eig_iterations = h->eig_iters;
  info->block_size = h->s_block;
  info->fp64_factors_K = h->nK64;
  info->fp64_factors_A = h->nA64;
  info->fp64_ortho = h->eig_o64;
  info->eig_unconverged = h->eig_unconv;
  info->factor_classes = h->factor_classes;
  info->local_solve_stages = h->local_stages;
  info->device_bytes = h->mem.bytes;
  for (int i = 0; i < 8; ++i) info->setup_ms[i] = h->setup_ms[i];
  info->factor_flops = h->factor_flops;
  info->factor_event_ms = h->factor_ms;
  info->eigsolve_flops = h->eig_flops;
  info->eigsolve_event_ms = h->eig_ms;
  info->apply_flops = h->apply_flops;
  info->apply_bytes = h->apply_bytes;
  cudaDeviceSynchronize();
  h->prof.collect();
  for (int i = 0; i < GENEO_PROF_COUNT; ++i) {
    info->prof_ms[i] = h->prof.ms[i];
    info->prof_flops[i] = h->prof.flops[i];
    info->prof_bytes[i] = h->prof.bytes[i];
    info->prof_launches[i] = h->prof.launches[i];
  }
  return GENEO_OK;
}

int64_t geneo_launch_count(void) { return geneo::launch_count(); }

int32_t geneo_struct_sizes(int64_t* out, int32_t n) {
  const int64_t sz[4] = {(int64_t)sizeof(geneo_problem_t), (int64_t)sizeof(geneo_options_t),
                         (int64_t)sizeof(geneo_solve_info_t), (int64_t)sizeof(geneo_coarse_info_t)};
  if (!out || n <= 0) return 0;
  const int32_t k = n < 4 ? n : 4;
  for (int32_t i = 0; i < k; ++i) out[i] = sz[i];
  return k;
}

geneo_status_t geneo_get_subdomain(geneo_handle_t h, int32_t j, int32_t* n_neu, int32_t* n_dir,
                                   int32_t* m, int32_t* s, int32_t* dir_dofs, int64_t dir_cap,
                                   double* pu, int64_t pu_cap, double* lambda, int64_t lambda_cap,
                                   double* Z, int64_t z_cap) {
  if (!h || j < 0 || j >= h->N) return GENEO_ERR_ARG;
  const SubDesc& d = h->hsub[j];
  if (n_neu) *n_neu = d.nN;
  if (n_dir) *n_dir = d.nD;
  if (m) *m = d.m;
  if (s) *s = d.s;
  GENEO_CUDA(cudaDeviceSynchronize());
  if (dir_dofs && dir_cap >= d.nD)
    GENEO_CUDA(cudaMemcpy(dir_dofs, h->Dlist + d.offN, sizeof(int32_t) * d.nD, cudaMemcpyDeviceToHost));
  if (pu && pu_cap >= d.nN)
    GENEO_CUDA(cudaMemcpy(pu, h->pu + d.offN, sizeof(double) * d.nN, cudaMemcpyDeviceToHost));
  if (lambda && lambda_cap >= d.s && !h->lambda_host.empty())
    std::memcpy(lambda, h->lambda_host.data() + (size_t)j * h->s_block, sizeof(double) * d.s);
  if (Z && z_cap >= (int64_t)d.nD * d.m && d.m > 0)
    GENEO_CUDA(cudaMemcpy(Z, h->Z + d.offZ, sizeof(double) * d.nD * d.m, cudaMemcpyDeviceToHost));
  return GENEO_OK;
}

void geneo_destroy(geneo_handle_t h) {
  if (!h) return;
  // the handle's memory goes back to the pool in the order of the stream of
  // its last call, after that call's work
  if (h->aux) cudaStreamSynchronize(h->aux);
  for (int i = 0; i < geneo::kSolveStreams; ++i)
    if (h->solve_streams.s[i]) cudaStreamSynchronize(h->solve_streams.s[i]);
  cudaStreamSynchronize(h->mem.stream);
  h->mem.free_all();
  cudaStreamSynchronize(h->mem.stream);
  for (int i = 0; i < geneo::kSolveStreams; ++i) {
    if (h->solve_streams.ev[i]) cudaEventDestroy(h->solve_streams.ev[i]);
    if (h->solve_streams.s[i]) cudaStreamDestroy(h->solve_streams.s[i]);
  }
  if (h->solve_streams.fork) cudaEventDestroy(h->solve_streams.fork);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->ev_afac) cudaEventDestroy(h->ev_afac);
  if (h->aux) cudaStreamDestroy(h->aux);
  if (h->hpin) cudaFreeHost(h->hpin);
  delete h;
}

const char* geneo_status_str(geneo_status_t s) {
  switch (s) {
    case GENEO_OK: return "ok";
    case GENEO_ERR_ARG: return "invalid argument";
    case GENEO_ERR_OOM: return "device out of memory";
    case GENEO_ERR_NOT_SPD: return "non-positive pivot in a Cholesky factorisation";
    case GENEO_ERR_EIG_NOCONV: return "local eigensolver did not converge";
    case GENEO_ERR_PCG_NOCONV: return "PCG did not reach the tolerance";
    case GENEO_ERR_BREAKDOWN: return "PCG breakdown";
    case GENEO_ERR_CUDA: return "CUDA runtime error";
    case GENEO_ERR_TIMEOUT: return "bounded device wait timed out";
    case GENEO_ERR_NONFINITE: return "non-finite value";
  }
  return "unknown status";
}

geneo_status_t geneo_last_error(geneo_handle_t h, int32_t* code, int32_t* where, int64_t* index) {
  const geneo::DevStatus& e = h ? h->hstat : g_setup_error;
  if (code) *code = e.code;
  if (where) *where = e.where;
  if (index) *index = e.index;
  return GENEO_OK;
}

void geneo_free_host(void* p) { std::free(p); }

}  // extern "C"
