// C-ABI entry points: plan life cycle, window export, potential, apply, preconditioner.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "blockops.cuh"
#include "common.cuh"

namespace iwf {

namespace {
thread_local std::string g_last_error;
}

iwf_status fail(iwf_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

iwf_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return IWF_ERR_CUDA;
}

void clear_error() { g_last_error.clear(); }

iwf_status ensure_workspace(iwf_plan* p, size_t bytes) {
  if (p->work_bytes >= bytes) return IWF_OK;
  if (p->d_work) { cudaFree(p->d_work); p->d_work = nullptr; p->work_bytes = 0; }
  cudaError_t e = cudaMalloc(&p->d_work, bytes);
  if (e != cudaSuccess) { p->d_work = nullptr; return fail(IWF_ERR_ALLOC, "workspace allocation failed"); }
  p->work_bytes = bytes;
  return IWF_OK;
}

namespace {

// Q = P_I^{-1} P_II by LU with partial pivoting (d > 1) or one division per entry (d = 1).
iwf_status split_q(int d, int n, const double* P, double* Q) {
  const int m = n - d;
  if (d == 1) {
    if (!(std::fabs(P[0]) > 0.0)) return fail(IWF_ERR_SINGULAR_PI, "P_I is zero");
    for (int i = 0; i < m; ++i) Q[i] = P[1 + i] / P[0];
    return IWF_OK;
  }
  std::vector<double> A(d * d), B(d * m), inv(d * d, 0.0);
  for (int r = 0; r < d; ++r) {
    for (int c = 0; c < d; ++c) A[r * d + c] = P[r * n + c];
    for (int c = 0; c < m; ++c) B[r * m + c] = P[r * n + d + c];
    inv[r * d + r] = 1.0;
  }
  double norm1 = 0.0;
  for (int c = 0; c < d; ++c) {
    double s = 0.0;
    for (int r = 0; r < d; ++r) s += std::fabs(A[r * d + c]);
    norm1 = std::fmax(norm1, s);
  }
  // Gauss-Jordan with partial pivoting on [A | B | I]
  for (int c = 0; c < d; ++c) {
    int piv = c;
    for (int r = c + 1; r < d; ++r)
      if (std::fabs(A[r * d + c]) > std::fabs(A[piv * d + c])) piv = r;
    if (!(std::fabs(A[piv * d + c]) > 0.0)) return fail(IWF_ERR_SINGULAR_PI, "P_I is singular");
    if (piv != c) {
      for (int k = 0; k < d; ++k) { std::swap(A[c * d + k], A[piv * d + k]); std::swap(inv[c * d + k], inv[piv * d + k]); }
      for (int k = 0; k < m; ++k) std::swap(B[c * m + k], B[piv * m + k]);
    }
    const double pv = A[c * d + c];
    for (int r = 0; r < d; ++r) {
      if (r == c) continue;
      const double f = A[r * d + c] / pv;
      if (f == 0.0) continue;
      for (int k = 0; k < d; ++k) { A[r * d + k] -= f * A[c * d + k]; inv[r * d + k] -= f * inv[c * d + k]; }
      for (int k = 0; k < m; ++k) B[r * m + k] -= f * B[c * m + k];
    }
  }
  double ninv = 0.0;
  for (int c = 0; c < d; ++c) {
    double s = 0.0;
    for (int r = 0; r < d; ++r) s += std::fabs(inv[r * d + c] / A[r * d + r]);
    ninv = std::fmax(ninv, s);
  }
  if (norm1 * ninv > 1e12) return fail(IWF_ERR_SINGULAR_PI, "P_I is ill-conditioned (cond > 1e12)");
  for (int r = 0; r < d; ++r)
    for (int k = 0; k < m; ++k) Q[r * m + k] = B[r * m + k] / A[r * d + r];
  return IWF_OK;
}

iwf_status plan_create(iwf_plan** out, int d, int n, const double* P, const int* K, const int* L,
                       const iwf_plan_opts* opts) {
  if (!out) return fail(IWF_ERR_ARG, "iwf_plan_create: plan pointer is NULL");
  *out = nullptr;
  if (!P || !K || !L) return fail(IWF_ERR_ARG, "iwf_plan_create: NULL P, K or L");
  if (d < 1 || n <= d || n > IWF_MAX_N)
    return fail(IWF_ERR_ARG, "iwf_plan_create: need 1 <= d < n <= 8");
  iwf_plan_opts o{IWF_METHOD_IWFPM, IWF_SHIFT_EXACT, 0};
  if (opts) o = *opts;
  if (o.method != IWF_METHOD_IWFPM && o.method != IWF_METHOD_PM)
    return fail(IWF_ERR_ARG, "iwf_plan_create: unknown method");
  if (o.shift_round != IWF_SHIFT_EXACT && o.shift_round != IWF_SHIFT_ROUND)
    return fail(IWF_ERR_ARG, "iwf_plan_create: unknown shift mode");
  for (int i = 0; i < d * n; ++i)
    if (!std::isfinite(P[i])) return fail(IWF_ERR_NONFINITE, "iwf_plan_create: non-finite P");
  int ndev = 0;
  IWF_CUDA(cudaGetDeviceCount(&ndev));
  if (o.device < 0 || o.device >= ndev) return fail(IWF_ERR_ARG, "iwf_plan_create: bad device");

  Geom g{};
  g.d = d; g.n = n; g.N = 1; g.MI = 1; g.MII = 1;
  for (int j = 0; j < n; ++j) {
    const int h = j < d ? K[j] : L[j - d];
    if (h < 1) return fail(IWF_ERR_ARG, "iwf_plan_create: K and L must be >= 1");
    if (!axis_len_ok(2 * h))
      return fail(IWF_ERR_UNSUPPORTED, "iwf_plan_create: axis length 2K or 2L above 8192, or "
                                       "above 32 with a prime factor above 7");
    g.half[j] = h;
    g.lens[j] = 2 * h;
    g.N *= 2 * h;
    if (j < d) g.MI *= 2 * h; else g.MII *= 2 * h;
  }
  if (g.MI > IWF_MAX_GROUP)
    return fail(IWF_ERR_UNSUPPORTED, "iwf_plan_create: (2K)^d above 8192");

  iwf_plan* p = new (std::nothrow) iwf_plan();
  if (!p) return fail(IWF_ERR_ALLOC, "iwf_plan_create: host allocation failed");
  p->device = o.device;
  p->method = o.method;
  p->shift_round = o.shift_round;
  p->g = g;
  std::memcpy(p->P, P, sizeof(double) * d * n);
  if (o.method == IWF_METHOD_IWFPM) {
    iwf_status st = split_q(d, n, P, p->Q);
    if (st != IWF_OK) { delete p; return st; }
  }
  DeviceGuard guard(p->device);
  iwf_status st = IWF_OK;
  if (cudaMalloc((void**)&p->d_err, sizeof(int)) != cudaSuccess) st = fail(IWF_ERR_ALLOC, "cudaMalloc");
  if (st == IWF_OK && cudaMalloc((void**)&p->d_apply_err, sizeof(int)) != cudaSuccess)
    st = fail(IWF_ERR_ALLOC, "cudaMalloc");
  if (st == IWF_OK && cudaMemset(p->d_apply_err, 0, sizeof(int)) != cudaSuccess)
    st = fail(IWF_ERR_CUDA, "cudaMemset");
  if (st == IWF_OK && cudaMalloc((void**)&p->d_field, 4 * sizeof(unsigned long long)) != cudaSuccess)
    st = fail(IWF_ERR_ALLOC, "cudaMalloc");
  if (st == IWF_OK) st = build_window_tables(p);
  if (st == IWF_OK) st = build_long_twiddles(p);
  if (st != IWF_OK) { iwf_plan_destroy(p); return st; }
  *out = p;
  return IWF_OK;
}

}  // namespace
}  // namespace iwf

using namespace iwf;

extern "C" {

int iwf_version(void) { return 100; }

const char* iwf_last_error(void) { return g_last_error.c_str(); }

iwf_status iwf_plan_create(iwf_plan** plan, int d, int n, const double* P, const int* K,
                           const int* L, const iwf_plan_opts* opts) {
  clear_error();
  return plan_create(plan, d, n, P, K, L, opts);
}

void iwf_plan_trim(iwf_plan* p) {
  if (!p) return;
  DeviceGuard guard(p->device);
  for (auto& b : p->solve_ws) cudaFree(b.ptr);
  p->solve_ws.clear();
}

void iwf_plan_destroy(iwf_plan* p) {
  if (!p) return;
  DeviceGuard guard(p->device);
  cudaFree(p->d_lo);
  cudaFree(p->d_lam64);
  cudaFree(p->d_lam32);
  cudaFree(p->d_err);
  cudaFree(p->d_apply_err);
  cudaFree(p->d_stencil_m);
  cudaFree(p->d_stencil_c);
  cudaFree(p->d_eval_part);
  cudaFree(p->d_field);
  for (int j = 0; j < IWF_MAX_N; ++j) {
    cudaFree(p->d_ltw64[j]);
    cudaFree(p->d_ltw32[j]);
  }
  release_host_pipeline(p);
  cudaFree(p->d_tab64);
  cudaFree(p->d_tab32);
  cudaFree(p->d_grid64);
  cudaFree(p->d_grid32);
  cudaFree(p->d_work);
  for (auto& b : p->solve_ws) cudaFree(b.ptr);
  delete p;
}

iwf_status iwf_plan_size(const iwf_plan* p, long long* N) {
  if (!p || !N) return fail(IWF_ERR_ARG, "iwf_plan_size: NULL argument");
  *N = p->g.N;
  return IWF_OK;
}

iwf_status iwf_plan_lens(const iwf_plan* p, int* lens) {
  if (!p || !lens) return fail(IWF_ERR_ARG, "iwf_plan_lens: NULL argument");
  for (int j = 0; j < p->g.n; ++j) lens[j] = p->g.lens[j];
  return IWF_OK;
}

iwf_status iwf_window(const iwf_plan* p, int* k) {
  if (!p || !k) return fail(IWF_ERR_ARG, "iwf_window: NULL argument");
  DeviceGuard guard(p->device);
  return export_window(p, k);
}

iwf_status iwf_coef_extent(const iwf_plan* p, const void* coef, double threshold, int* need,
                           void* stream) {
  clear_error();
  return coef_extent(p, coef, threshold, need, (cudaStream_t)stream);
}

iwf_status iwf_kinetic(const iwf_plan* p, double* lam) {
  if (!p || !lam) return fail(IWF_ERR_ARG, "iwf_kinetic: NULL argument");
  DeviceGuard guard(p->device);
  IWF_CUDA(cudaMemcpy(lam, p->d_lam64, sizeof(double) * p->g.N, cudaMemcpyDeviceToHost));
  return IWF_OK;
}

iwf_status iwf_set_potential(iwf_plan* p, int nmodes, const int* m, const double* re,
                             const double* im) {
  clear_error();
  if (!p || nmodes < 0 || (nmodes > 0 && (!m || !re || !im)))
    return fail(IWF_ERR_ARG, "iwf_set_potential: bad arguments");
  DeviceGuard guard(p->device);
  return build_potential(p, nmodes, m, re, im);
}

iwf_status iwf_apply(iwf_plan* p, int precision, const void* psi, void* hpsi, int nvec,
                     void* stream) {
  if (!p) return fail(IWF_ERR_ARG, "iwf_apply: NULL plan");
  DeviceGuard guard(p->device);
  return apply_impl(p, precision, psi, hpsi, nvec, (cudaStream_t)stream);
}

iwf_status iwf_apply_profile(iwf_plan* p, int precision, const void* psi, void* hpsi, int nvec,
                             void* stream, double* pass_ms, int* launches) {
  if (!p) return fail(IWF_ERR_ARG, "iwf_apply_profile: NULL plan");
  DeviceGuard guard(p->device);
  PassTimer t;
  IWF_CUDA(cudaEventCreate(&t.ev[0]));
  if (cudaEventCreate(&t.ev[1]) != cudaSuccess) {
    cudaEventDestroy(t.ev[0]);
    return fail(IWF_ERR_CUDA, "cudaEventCreate");
  }
  iwf_status st = apply_impl(p, precision, psi, hpsi, nvec, (cudaStream_t)stream, &t);
  cudaEventDestroy(t.ev[0]);
  cudaEventDestroy(t.ev[1]);
  if (st != IWF_OK) return st;
  IWF_TRY(check_apply_error(p, (cudaStream_t)stream));
  for (int i = 0; i < 3; ++i) {
    if (pass_ms) pass_ms[i] = t.ms[i];
    if (launches) launches[i] = t.launches[i];
  }
  return IWF_OK;
}

long long iwf_kernel_launches(void) { return launch_count(); }

iwf_status iwf_plan_autotune(iwf_plan* p, int precision, int nvec, double* best_ms, int* best,
                             void* stream) {
  clear_error();
  if (!p) return fail(IWF_ERR_ARG, "iwf_plan_autotune: NULL plan");
  DeviceGuard guard(p->device);
  return autotune_impl(p, precision, nvec, best_ms, best, (cudaStream_t)stream);
}

iwf_status iwf_plan_set_schedule(iwf_plan* p, int precision, int threads, int tile_kb,
                                 int chunk_mb) {
  if (!p) return fail(IWF_ERR_ARG, "iwf_plan_set_schedule: NULL plan");
  return set_schedule_impl(p, precision, threads, tile_kb, chunk_mb);
}

iwf_status iwf_apply_host(iwf_plan* p, int precision, const void* psi_host, void* hpsi_host,
                          int nvec, void* stream) {
  clear_error();
  if (!p) return fail(IWF_ERR_ARG, "iwf_apply_host: NULL plan");
  DeviceGuard guard(p->device);
  return apply_host_impl(p, precision, psi_host, hpsi_host, nvec, (cudaStream_t)stream);
}

iwf_status iwf_apply_stencil(iwf_plan* p, int precision, const void* psi, void* hpsi, int nvec,
                             void* stream) {
  clear_error();
  if (!p) return fail(IWF_ERR_ARG, "iwf_apply_stencil: NULL plan");
  DeviceGuard guard(p->device);
  return apply_stencil_impl(p, precision, psi, hpsi, nvec, (cudaStream_t)stream);
}

iwf_status iwf_evaluate(iwf_plan* p, const void* coef, const double* x, long long M,
                        void* u, void* stream) {
  clear_error();
  if (!p) return fail(IWF_ERR_ARG, "iwf_evaluate: NULL plan");
  DeviceGuard guard(p->device);
  return evaluate_impl(p, coef, x, M, u, (cudaStream_t)stream);
}

iwf_status iwf_evaluate_grid(iwf_plan* p, const void* coef, const double* origin,
                             const double* step, const int* count, void* u, void* stream) {
  clear_error();
  if (!p) return fail(IWF_ERR_ARG, "iwf_evaluate_grid: NULL plan");
  DeviceGuard guard(p->device);
  return evaluate_grid_impl(p, coef, origin, step, count, u, (cudaStream_t)stream);
}

iwf_status iwf_field_normalize(iwf_plan* p, void* u, long long M, long long at, double* rho,
                               long long* argmax, void* stream) {
  clear_error();
  if (!p) return fail(IWF_ERR_ARG, "iwf_field_normalize: NULL plan");
  DeviceGuard guard(p->device);
  return field_normalize_impl(p, u, M, at, rho, argmax, (cudaStream_t)stream);
}

iwf_status iwf_field_distance(iwf_plan* p, const void* u, const void* v, long long M,
                              double* dist, void* stream) {
  clear_error();
  if (!p) return fail(IWF_ERR_ARG, "iwf_field_distance: NULL plan");
  DeviceGuard guard(p->device);
  return field_distance_impl(p, u, v, M, dist, (cudaStream_t)stream);
}

iwf_status iwf_plan_set_path(iwf_plan* p, int precision, int path) {
  clear_error();
  if (!p) return fail(IWF_ERR_ARG, "iwf_plan_set_path: NULL plan");
  return set_path_impl(p, precision, path);
}

iwf_status iwf_plan_set_arith(iwf_plan* p, int arith) {
  clear_error();
  if (!p) return fail(IWF_ERR_ARG, "iwf_plan_set_arith: NULL plan");
  return set_arith_impl(p, arith);
}

iwf_status iwf_plan_get_schedule(const iwf_plan* p, int precision, int* sched) {
  clear_error();
  if (!p) return fail(IWF_ERR_ARG, "iwf_plan_get_schedule: NULL plan");
  return get_schedule_impl(p, precision, sched);
}

iwf_status iwf_batch_eigensolve(iwf_plan* p, int nprob, const int* nmodes, const int* m,
                                const double* re, const double* im, const iwf_solve_opts* opts,
                                const void* X0, double* evals, void* evecs, double* resid,
                                int* iters, iwf_solve_info* info, void* stream) {
  clear_error();
  if (!p) return fail(IWF_ERR_ARG, "iwf_batch_eigensolve: NULL plan");
  DeviceGuard guard(p->device);
  return batch_eigensolve_impl(p, nprob, nmodes, m, re, im, opts, X0, evals, evecs, resid,
                               iters, info, (cudaStream_t)stream);
}

iwf_status iwf_batch_solve(int nplans, iwf_plan* const* plans, const iwf_solve_opts* opts,
                           const void* const* X0, double* evals, void* const* evecs,
                           double* resid, int* iters, iwf_solve_info* info, void* stream) {
  clear_error();
  return batch_solve_impl(nplans, plans, opts, X0, evals, evecs, resid, iters, info,
                          (cudaStream_t)stream);
}

iwf_status iwf_eigensolve(iwf_plan* p, const iwf_solve_opts* opts, const void* X0, double* evals,
                          void* evecs, double* resid, iwf_solve_info* info, void* stream) {
  clear_error();
  if (!p) return fail(IWF_ERR_ARG, "iwf_eigensolve: NULL plan");
  DeviceGuard guard(p->device);
  return eigensolve_impl(p, opts, X0, evals, evecs, resid, info, (cudaStream_t)stream);
}

iwf_status iwf_apply_noalloc(iwf_plan* p, int precision, const void* psi, void* hpsi, int nvec,
                             void* stream) {
  if (!p) return fail(IWF_ERR_ARG, "iwf_apply_noalloc: NULL plan");
  DeviceGuard guard(p->device);
  return apply_noalloc_impl(p, precision, psi, hpsi, nvec, (cudaStream_t)stream);
}

iwf_status iwf_plan_check(iwf_plan* p, void* stream) {
  clear_error();
  if (!p) return fail(IWF_ERR_ARG, "iwf_plan_check: NULL plan");
  DeviceGuard guard(p->device);
  return check_apply_error(p, (cudaStream_t)stream);
}

iwf_status iwf_plan_set_wait_limit(iwf_plan* p, long long rounds) {
  clear_error();
  if (!p) return fail(IWF_ERR_ARG, "iwf_plan_set_wait_limit: NULL plan");
  p->wait_rounds = rounds < 0 ? -1 : rounds;
  return IWF_OK;
}

iwf_status iwf_preconditioner(const iwf_plan* p, double* M, double* sigma) {
  if (!p) return fail(IWF_ERR_ARG, "iwf_preconditioner: NULL plan");
  if (p->pot_kind == 0) return fail(IWF_ERR_ARG, "iwf_preconditioner: no potential set");
  const double sg = p->voff_abs - p->vg0 + 1.0;
  if (sigma) *sigma = sg;
  if (M) {
    DeviceGuard guard(p->device);
    std::vector<double> lam(p->g.N);
    IWF_CUDA(cudaMemcpy(lam.data(), p->d_lam64, sizeof(double) * p->g.N, cudaMemcpyDeviceToHost));
    for (long long i = 0; i < p->g.N; ++i) {
      const double h = lam[i] + p->vg0 + sg;
      M[i] = h / (h * h + p->voff_sq);
    }
  }
  return IWF_OK;
}

}  // extern "C"

// ---- the eigensolver's contractions as entry points (iwf_gram, iwf_block_update) ----------
namespace {
struct Scratch {
  std::vector<void*> ptrs;
  ~Scratch() { for (void* p : ptrs) cudaFree(p); }
  iwf_status get(void** out, size_t bytes) {
    if (cudaMalloc(out, bytes) != cudaSuccess) return iwf::fail(IWF_ERR_ALLOC, "contraction scratch");
    ptrs.push_back(*out);
    return IWF_OK;
  }
};

iwf_status contract_batch(int engine, Scratch& sc, iwf::Batch* bt) {
  if (engine != IWF_CONTRACT_TENSOR && engine != IWF_CONTRACT_DF && engine != IWF_CONTRACT_F64)
    return iwf::fail(IWF_ERR_ARG, "unknown contraction engine");
  bt->nprob = 1;
  bt->pstride = 0;
  bt->active = nullptr;
  bt->engine = engine == IWF_CONTRACT_TENSOR ? iwf::kEngineTensor
               : engine == IWF_CONTRACT_DF   ? iwf::kEngineDF
                                             : iwf::kEngineF64;
  void *e = nullptr, *w = nullptr;
  IWF_TRY(sc.get(&e, sizeof(int) * 2 * iwf::kMaxSmall));
  IWF_TRY(sc.get(&w, sizeof(int)));
  IWF_CUDA(cudaMemset(w, 0, sizeof(int)));
  bt->exps = static_cast<int*>(e);
  bt->err = static_cast<int*>(w);
  return IWF_OK;
}

iwf_status contract_finish(const iwf::Batch& bt, cudaStream_t st) {
  int h = 0;
  IWF_CUDA(cudaMemcpyAsync(&h, bt.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  IWF_CUDA(cudaStreamSynchronize(st));
  if (h) return iwf::fail(IWF_ERR_TIMEOUT, "tensor-core contraction: a bounded wait ran out");
  return IWF_OK;
}
}  // namespace

extern "C" {

iwf_status iwf_gram(int engine, long long nrows, const void* A, int ma, const void* B, int mb,
                    void* G, int device, void* stream) {
  clear_error();
  if (!A || !B || !G || nrows < 1 || ma < 1 || mb < 1 || ma > kMaxSmall || mb > kMaxSmall)
    return fail(IWF_ERR_ARG, "iwf_gram: bad arguments");
  DeviceGuard guard(device);
  cudaStream_t st = (cudaStream_t)stream;
  Scratch sc;
  Batch bt;
  IWF_TRY(contract_batch(engine, sc, &bt));
  const int slots = 608;
  void *part = nullptr, *out = nullptr;
  IWF_TRY(sc.get(&part, sizeof(double2) * (size_t)slots * kCapG));
  IWF_TRY(sc.get(&out, sizeof(double2) * kCapG));
  BlockList LA{}, LB{};
  LA.p[0] = A; LA.nb = 1; LA.b = ma;
  LB.p[0] = B; LB.nb = 1; LB.b = mb;
  IWF_TRY(gram<double>(bt, LA, LB, nrows, static_cast<double2*>(out),
                       static_cast<double2*>(part), slots, st, false));
  IWF_CUDA(cudaMemcpyAsync(G, out, sizeof(double2) * (size_t)ma * mb, cudaMemcpyDeviceToDevice, st));
  return contract_finish(bt, st);
}

iwf_status iwf_block_update(int engine, long long nrows, const void* S, int m, const void* C,
                            int q, void* Y, int subtract, int device, void* stream) {
  clear_error();
  if (!S || !C || !Y || nrows < 1 || m < 1 || m > kMaxSmall || q < 1 || q > kMaxBlock)
    return fail(IWF_ERR_ARG, "iwf_block_update: bad arguments");
  DeviceGuard guard(device);
  cudaStream_t st = (cudaStream_t)stream;
  Scratch sc;
  Batch bt;
  IWF_TRY(contract_batch(engine, sc, &bt));
  BlockList LS{};
  LS.p[0] = S; LS.nb = 1; LS.b = m;
  IWF_TRY(block_update<double>(bt, LS, nrows, static_cast<const double2*>(C), nullptr, m * q, q,
                               Y, nullptr, subtract != 0, st));
  return contract_finish(bt, st);
}

}  // extern "C"
