// Block LOBPCG for the lowest eigenpairs of H~ (Sec. 4.1, Alg. 2 in block form), for one
// problem or a batch of problems sharing one plan's geometry (different potentials).
//
// Every iteration keeps an orthonormal basis S = [X W P] of each problem's trial subspace:
//   R = H X - X diag(theta), W = M R            (preconditioner of Eq. precond, shifted)
//   W <- W - [X P]([X P]^H W), twice            (classical Gram-Schmidt, reorthogonalised)
//   W <- W D U S^{-1/2}, twice                   (SVQB; dependent directions dropped)
//   HW = H W                                      (the FFT apply)
//   A = S^H [HX HW HP]; A = Y diag(theta) Y^H     (one-CTA Jacobi per problem, FP64)
//   X <- S Yx, P <- S Yp with Yp orthonormalised against Yx in the coefficient space, so
//   that [X P] stays orthonormal without touching the long vectors again.
// All problems advance in lockstep through the same kernels (problem index in the grid);
// converged problems are switched off by a device flag every kernel reads. The steady-state
// iteration is captured once into two CUDA graphs (the buffer sets alternate) and replayed;
// the host reads only the residual norms after each replay.
// Mixed precision: a first phase stores the blocks in complex float and applies H in
// complex float (Gram sums in float within 16-row tiles, double across tiles); its X then
// seeds the FP64 phase, which runs to the requested tolerance.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "blockops.cuh"
#include "common.cuh"

namespace iwf {

namespace {

// IWF_LOG=1: one line per iteration on stderr; IWF_LOG=2: also every residual.
int log_level() {
  static const int level = [] {
    const char* e = std::getenv("IWF_LOG");
    return e ? std::atoi(e) : 0;
  }();
  return level;
}

bool graphs_enabled() {
  static const bool on = [] { return std::getenv("IWF_NO_GRAPH") == nullptr; }();
  return on;
}

template <typename T> constexpr int prec_of() { return sizeof(T) == 8 ? IWF_PREC_F64 : IWF_PREC_C64; }

// Device buffers of one solve. With a plan, they come from the plan's workspace: the i-th
// request of a solve reuses the plan's i-th buffer when it is large enough (a solve of the
// same shape allocates nothing), else that buffer is replaced. Without a plan (the groups of
// iwf_batch_solve, whose memory must return before the next group starts) they are
// allocated here and freed with the arena.
struct Arena {
  iwf_plan* plan = nullptr;
  size_t next = 0;
  std::vector<void*> own;
  explicit Arena(iwf_plan* p = nullptr) : plan(p) {}
  ~Arena() { for (void* q : own) cudaFree(q); }
  Arena(const Arena&) = delete;
  Arena& operator=(const Arena&) = delete;
  template <typename U>
  iwf_status get(U** out, size_t count) {
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(U);
    void* q = nullptr;
    if (!plan) {
      if (cudaMalloc(&q, bytes) != cudaSuccess)
        return fail(IWF_ERR_ALLOC, "eigensolver workspace allocation failed");
      own.push_back(q);
      *out = reinterpret_cast<U*>(q);
      return IWF_OK;
    }
    auto& ws = plan->solve_ws;
    if (next < ws.size() && ws[next].bytes >= bytes) {
      *out = reinterpret_cast<U*>(ws[next++].ptr);
      return IWF_OK;
    }
    if (next < ws.size()) {
      cudaFree(ws[next].ptr);
      ws[next] = {nullptr, 0};
    } else {
      ws.push_back({nullptr, 0});
    }
    if (cudaMalloc(&q, bytes) != cudaSuccess) {
      (void)cudaGetLastError();
      return fail(IWF_ERR_ALLOC, "eigensolver workspace allocation failed");
    }
    ws[next] = {q, bytes};
    *out = reinterpret_cast<U*>(ws[next++].ptr);
    return IWF_OK;
  }
};

// Per-problem small buffers (fixed capacities, see blockops.cuh) and problem parameters.
struct Small {
  int nprob = 1;
  int slots = 608;             // Gram / residual partial slots per problem
  double2 *G, *Cx, *Cp, *T, *partial;
  double *theta, *resid, *rpartial;
  int *mask, *maskw, *maskp, *status, *active;
  int* exps;                   // column scales of the tensor-core Gram products
  double *shift, *off2;        // preconditioner parameters per problem
};

iwf_status alloc_small(Arena& ar, Small& s, int nprob) {
  s.nprob = nprob;
  s.slots = std::max(8, std::min(608, (4 * 608) / nprob));
  IWF_TRY(ar.get(&s.G, (size_t)nprob * kCapG));
  IWF_TRY(ar.get(&s.Cx, (size_t)nprob * kCapC));
  IWF_TRY(ar.get(&s.Cp, (size_t)nprob * kCapC));
  IWF_TRY(ar.get(&s.T, (size_t)nprob * kCapT));
  IWF_TRY(ar.get(&s.theta, (size_t)nprob * kMaxBlock));
  IWF_TRY(ar.get(&s.resid, (size_t)nprob * kMaxBlock));
  IWF_TRY(ar.get(&s.mask, (size_t)nprob * kMaxSmall));
  IWF_TRY(ar.get(&s.maskw, (size_t)nprob * kMaxBlock));
  IWF_TRY(ar.get(&s.maskp, (size_t)nprob * kMaxBlock));
  IWF_TRY(ar.get(&s.status, (size_t)nprob));
  IWF_TRY(ar.get(&s.active, (size_t)nprob));
  IWF_TRY(ar.get(&s.shift, (size_t)nprob));
  IWF_TRY(ar.get(&s.off2, (size_t)nprob));
  IWF_TRY(ar.get(&s.exps, (size_t)nprob * 2 * kMaxSmall));
  IWF_TRY(ar.get(&s.partial, (size_t)nprob * s.slots * kCapG));
  IWF_TRY(ar.get(&s.rpartial, (size_t)nprob * s.slots * kMaxBlock));
  return IWF_OK;
}

struct PhaseResult {
  std::vector<int> iters;        // per problem: iterations until it converged (or stopped)
  std::vector<int> converged;
  long long applies = 0;
  int rounds = 0;                // lockstep iterations of the phase
  std::vector<double> theta, resid;  // nprob x kMaxBlock
};

BlockList blocks(std::initializer_list<const void*> ps, int b) {
  BlockList L{};
  int i = 0;
  for (const void* p : ps) L.p[i++] = p;
  L.nb = i;
  L.b = b;
  return L;
}

struct Graph {
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  long long kernels = 0;
  ~Graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
};

// One LOBPCG phase with blocks stored as T for nprob problems (problem p's block at
// X + p*N*b). Stops per problem when its first nev residuals are <= tol (verified with a
// fresh H X), when `stall` > 0 and its worst residual has not dropped by 30 % in `stall`
// iterations (a floor: ordinary convergence here runs at about 0.88 per iteration, so a
// halving test would stop it), or after maxit lockstep iterations.
template <typename T>
iwf_status run_phase(iwf_plan* p, const ApplyBatch* ab, int b, int nev, int maxit, double tol,
                     int stall, void* Xio, Small& sm, Arena& ar, cudaStream_t st,
                     PhaseResult& res, int engine) {
  using V2 = typename Cplx<T>::type;
  const int np = sm.nprob;
  const long long N = p->g.N;
  const size_t blk = (size_t)N * b;
  const size_t all = blk * np;
  V2 *X, *HX, *W, *HW, *P, *HP, *X2, *HX2, *P2, *HP2, *W2;
  IWF_TRY(ar.get(&HX, all)); IWF_TRY(ar.get(&W, all)); IWF_TRY(ar.get(&HW, all));
  IWF_TRY(ar.get(&P, all)); IWF_TRY(ar.get(&HP, all)); IWF_TRY(ar.get(&X2, all));
  IWF_TRY(ar.get(&HX2, all)); IWF_TRY(ar.get(&P2, all)); IWF_TRY(ar.get(&HP2, all));
  IWF_TRY(ar.get(&W2, all));
  X = reinterpret_cast<V2*>(Xio);
  Batch bt{np, (long long)blk, sm.active, engine, sm.exps, p->d_apply_err};
  const int prec = prec_of<T>();
  std::vector<double> h_resid((size_t)np * kMaxBlock), h_theta((size_t)np * kMaxBlock);
  std::vector<int> h_status(np), h_active(np, 1);
  res.iters.assign(np, 0);
  res.converged.assign(np, 0);
  std::vector<int> pending(np, 0);      // met tol once; waiting for a verified residual
  std::vector<double> best(np, INFINITY);
  std::vector<int> best_it(np, 0);

  auto upload_active = [&]() -> iwf_status {
    IWF_CUDA(cudaMemcpyAsync(sm.active, h_active.data(), sizeof(int) * np, cudaMemcpyHostToDevice, st));
    return IWF_OK;
  };
  auto count_applies = [&]() {
    int nact = 0;
    for (int q = 0; q < np; ++q) nact += h_active[q];
    res.applies += (long long)b * nact;
  };
  auto orthonormalize = [&](V2* Y, V2* Y2, int* mask) -> iwf_status {
    for (int pass = 0; pass < 2; ++pass) {
      IWF_TRY(gram<T>(bt, blocks({Y}, b), blocks({Y}, b), N, sm.G, sm.partial, sm.slots, st, true));
      IWF_TRY(svqb_small(bt, sm.G, b, 1e-14, sm.T, mask, sm.status, st));
      IWF_TRY(block_update<T>(bt, blocks({Y}, b), N, sm.T, nullptr, kCapT, b, Y2, nullptr, false, st));
      IWF_CUDA(cudaMemcpyAsync(Y, Y2, sizeof(V2) * all, cudaMemcpyDeviceToDevice, st));
    }
    return IWF_OK;
  };
  // Rayleigh-Ritz on X alone: X <- X Y, HX <- HX Y, theta (results land back in X, HX)
  auto rr_x = [&](V2* Xc, V2* HXc, V2* T1, V2* T2) -> iwf_status {
    IWF_TRY(gram<T>(bt, blocks({Xc}, b), blocks({HXc}, b), N, sm.G, sm.partial, sm.slots, st, true));
    IWF_TRY(set_mask(bt, sm.mask, 0, b, 1, nullptr, st));
    IWF_TRY(rayleigh_ritz_small(bt, sm.G, b, b, sm.mask, b, sm.theta, sm.Cx, sm.Cp, sm.maskp,
                                sm.status, st));
    IWF_TRY(block_update<T>(bt, blocks({Xc}, b), N, sm.Cx, nullptr, kCapC, b, T1, nullptr, false, st));
    IWF_TRY(block_update<T>(bt, blocks({HXc}, b), N, sm.Cx, nullptr, kCapC, b, T2, nullptr, false, st));
    IWF_CUDA(cudaMemcpyAsync(Xc, T1, sizeof(V2) * all, cudaMemcpyDeviceToDevice, st));
    IWF_CUDA(cudaMemcpyAsync(HXc, T2, sizeof(V2) * all, cudaMemcpyDeviceToDevice, st));
    return IWF_OK;
  };
  auto residual = [&](const V2* Xc, const V2* HXc) -> iwf_status {
    return residual_precond<T>(bt, Xc, HXc, sm.theta, p->d_lam64, sm.shift, sm.off2, W, N, b,
                               sm.rpartial, sm.slots, sm.resid, st);
  };
  // one iteration from (Xa, HXa, Pa, HPa) into (Xb, HXb, Pb, HPb), then the new residual
  auto iterate = [&](V2* Xa, V2* HXa, V2* Pa, V2* HPa, V2* Xb, V2* HXb, V2* Pb, V2* HPb,
                     bool hasP) -> iwf_status {
    for (int pass = 0; pass < 2; ++pass) {
      const BlockList XP = hasP ? blocks({Xa, Pa}, b) : blocks({Xa}, b);
      IWF_TRY(gram<T>(bt, XP, blocks({W}, b), N, sm.G, sm.partial, sm.slots, st));
      IWF_TRY(block_update<T>(bt, XP, N, sm.G, nullptr, kCapG, b, W, nullptr, true, st));
    }
    for (int pass = 0; pass < 2; ++pass) {
      IWF_TRY(gram<T>(bt, blocks({W}, b), blocks({W}, b), N, sm.G, sm.partial, sm.slots, st, true));
      IWF_TRY(svqb_small(bt, sm.G, b, 1e-14, sm.T, sm.maskw, sm.status, st));
      IWF_TRY(block_update<T>(bt, blocks({W}, b), N, sm.T, nullptr, kCapT, b, W2, nullptr, false, st));
      std::swap(W, W2);
    }
    IWF_TRY(apply_impl(p, prec, W, HW, b * np, st, nullptr, ab));
    const int m = hasP ? 3 * b : 2 * b;
    const BlockList S = hasP ? blocks({Xa, W, Pa}, b) : blocks({Xa, W}, b);
    const BlockList HS = hasP ? blocks({HXa, HW, HPa}, b) : blocks({HXa, HW}, b);
    // S^H H S is Hermitian (H is): only its upper 24 x 24 blocks are formed
    IWF_TRY(gram<T>(bt, S, HS, N, sm.G, sm.partial, sm.slots, st, true));
    IWF_TRY(set_mask(bt, sm.mask, 0, b, 1, nullptr, st));
    IWF_TRY(set_mask(bt, sm.mask, b, b, 0, sm.maskw, st));
    if (hasP) IWF_TRY(set_mask(bt, sm.mask, 2 * b, b, 0, sm.maskp, st));
    IWF_TRY(rayleigh_ritz_small(bt, sm.G, m, b, sm.mask, b, sm.theta, sm.Cx, sm.Cp, sm.maskp,
                                sm.status, st));
    IWF_TRY(block_update<T>(bt, S, N, sm.Cx, sm.Cp, kCapC, b, Xb, Pb, false, st));
    IWF_TRY(block_update<T>(bt, HS, N, sm.Cx, sm.Cp, kCapC, b, HXb, HPb, false, st));
    return residual(Xb, HXb);
  };
  auto read_small = [&]() -> iwf_status {
    IWF_CUDA(cudaMemcpyAsync(h_resid.data(), sm.resid, sizeof(double) * np * kMaxBlock, cudaMemcpyDeviceToHost, st));
    IWF_CUDA(cudaMemcpyAsync(h_theta.data(), sm.theta, sizeof(double) * np * kMaxBlock, cudaMemcpyDeviceToHost, st));
    IWF_CUDA(cudaMemcpyAsync(h_status.data(), sm.status, sizeof(int) * np, cudaMemcpyDeviceToHost, st));
    // the apply's device error word (a pipelined pass that gave up waiting), read at the
    // same synchronisation point
    return check_apply_error(p, st);
  };
  auto worst_of = [&](int q) {
    double w = 0;
    for (int j = 0; j < nev; ++j) {
      const double r = h_resid[(size_t)q * kMaxBlock + j];
      w = std::isfinite(r) ? std::max(w, r) : INFINITY;
    }
    return w;
  };

  IWF_TRY(upload_active());
  IWF_CUDA(cudaMemsetAsync(sm.status, 0, sizeof(int) * np, st));
  IWF_TRY(orthonormalize(X, X2, sm.maskw));
  count_applies();
  IWF_TRY(apply_impl(p, prec, X, HX, b * np, st, nullptr, ab));
  IWF_TRY(rr_x(X, HX, X2, HX2));
  IWF_TRY(residual(X, HX));
  bool hasP = false;
  int parity = 0;                // 0: current iterate in (X, HX, P, HP), 1: in the *2 set
  Graph graphs[2];
  for (int it = 0;; ++it) {
    IWF_TRY(read_small());
    bool any_pending = false, any_active = false;
    for (int q = 0; q < np; ++q) {
      if (!h_active[q]) continue;
      const double w = worst_of(q);
      if (!std::isfinite(w)) return fail(IWF_ERR_NONFINITE, "non-finite residual in the eigensolver");
      if (h_status[q] != 0) return fail(IWF_ERR_BREAKDOWN, "Rayleigh-Ritz subspace lost rank");
      res.iters[q] = it;
      if (w <= tol) {
        if (pending[q]) { res.converged[q] = 1; h_active[q] = 0; pending[q] = 0; continue; }
        pending[q] = 1;
        any_pending = true;
      } else {
        pending[q] = 0;
        if (stall > 0) {
          if (w < 0.7 * best[q]) { best[q] = w; best_it[q] = it; }
          else if (it - best_it[q] >= stall) { h_active[q] = 0; continue; }
        }
      }
      any_active = true;
    }
    if (log_level() > 0) {
      int nact = 0;
      double worst = 0;
      for (int q = 0; q < np; ++q) if (h_active[q]) { ++nact; worst = std::max(worst, worst_of(q)); }
      std::fprintf(stderr, "[iwf] %s it %d active %d worst %.3e theta0 %.12f\n",
                   sizeof(T) == 8 ? "f64" : "c64", it, nact, worst, h_theta[0]);
      if (log_level() > 1)
        for (int q = 0; q < np; ++q) {
          for (int j = 0; j < b; ++j) std::fprintf(stderr, " %.2e", h_resid[(size_t)q * kMaxBlock + j]);
          std::fprintf(stderr, "\n");
        }
    }
    res.rounds = it;
    if (!any_active || it >= maxit) break;
    IWF_TRY(upload_active());
    V2 *Xa = parity ? X2 : X, *HXa = parity ? HX2 : HX, *Pa = parity ? P2 : P, *HPa = parity ? HP2 : HP;
    V2 *Xb = parity ? X : X2, *HXb = parity ? HX : HX2, *Pb = parity ? P : P2, *HPb = parity ? HP : HP2;
    if (any_pending) {
      // fresh H X for every active problem (removes drift of the implicit HX updates); the
      // spare buffer set (Xb, HXb) is scratch here
      count_applies();
      IWF_TRY(apply_impl(p, prec, Xa, HXa, b * np, st, nullptr, ab));
      IWF_TRY(rr_x(Xa, HXa, Xb, HXb));
      IWF_TRY(residual(Xa, HXa));
      --it;
      continue;
    }
    count_applies();
    if (hasP && graphs_enabled()) {
      Graph& g = graphs[parity];
      if (!g.exec) {
        const long long k0 = launch_count();
        IWF_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        const iwf_status s = iterate(Xa, HXa, Pa, HPa, Xb, HXb, Pb, HPb, true);
        const cudaError_t e = cudaStreamEndCapture(st, &g.graph);
        if (s != IWF_OK) return s;
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        IWF_CUDA(cudaGraphInstantiate(&g.exec, g.graph, 0));
        g.kernels = launch_count() - k0;
      } else {
        for (long long k = 0; k < g.kernels; ++k) count_launch();
      }
      IWF_CUDA(cudaGraphLaunch(g.exec, st));
    } else {
      IWF_TRY(iterate(Xa, HXa, Pa, HPa, Xb, HXb, Pb, HPb, hasP));
    }
    hasP = true;
    parity ^= 1;
  }
  res.theta = h_theta;
  res.resid = h_resid;
  if (parity)
    IWF_CUDA(cudaMemcpyAsync(X, X2, sizeof(V2) * all, cudaMemcpyDeviceToDevice, st));
  IWF_CUDA(cudaStreamSynchronize(st));
  return IWF_OK;
}

// ---- returned eigenvalues: FP64 Rayleigh quotients of the returned vectors ----
// theta_j = Re(x_j^H (H x)_j) / (x_j^H x_j) with H x applied afresh. The Ritz values of the
// double-float Rayleigh-Ritz carry its rounding (a few 1e-12 when the projected matrix has
// large entries); these quotients carry only FP64 rounding of two dot products and of one
// apply, and differ from the exact eigenvalue by O(residual^2 / gap).
constexpr int kRqThreads = 256;

// vector v = q * nev + j (problem q, column j < nev) at offset (q * b + j) * N in X and Y;
// block c of vector v writes its partial (num, den) to part[v * chunks + c]
__global__ void __launch_bounds__(kRqThreads) rq_partial_kernel(
    const double2* __restrict__ X, const double2* __restrict__ Y, long long N, int b, int nev,
    int chunks, double2* __restrict__ part) {
  const int v = blockIdx.y;
  const int q = v / nev, j = v - q * nev;
  const size_t off = ((size_t)q * b + j) * (size_t)N;
  double num = 0.0, den = 0.0;
  for (long long i = (long long)blockIdx.x * kRqThreads + threadIdx.x; i < N;
       i += (long long)chunks * kRqThreads) {
    const double2 x = X[off + i], y = Y[off + i];
    num = fma(x.x, y.x, fma(x.y, y.y, num));
    den = fma(x.x, x.x, fma(x.y, x.y, den));
  }
  for (int o = 16; o; o >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, o);
    den += __shfl_xor_sync(0xffffffffu, den, o);
  }
  __shared__ double sn[kRqThreads / 32], sd[kRqThreads / 32];
  if ((threadIdx.x & 31) == 0) { sn[threadIdx.x >> 5] = num; sd[threadIdx.x >> 5] = den; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int w = 0; w < kRqThreads / 32; ++w) { a += sn[w]; c += sd[w]; }
    part[(size_t)v * chunks + blockIdx.x] = make_double2(a, c);
  }
}

__global__ void rq_final_kernel(const double2* __restrict__ part, int chunks, int nvec,
                                double* __restrict__ theta) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvec) return;
  double a = 0.0, c = 0.0;
  for (int k = 0; k < chunks; ++k) {
    const double2 t = part[(size_t)v * chunks + k];
    a += t.x;
    c += t.y;
  }
  theta[v] = a / c;
}

// Rayleigh quotients of the first nev columns of every problem's block X (b columns each).
iwf_status rayleigh_quotients(iwf_plan* p, const ApplyBatch* ab, Small& sm, Arena& ar,
                              const double2* X, int b, int nev, double* out, long long* applies,
                              cudaStream_t st) {
  const int np = sm.nprob;
  const long long N = p->g.N;
  // one problem: apply only its nev columns; a batch: the whole block (its layout), with
  // every problem switched on again
  const int nvec = ab ? b * np : nev;
  double2 *HX, *part;
  double* d_theta;
  IWF_TRY(ar.get(&HX, (size_t)N * nvec));
  const int chunks = (int)std::min<long long>(512, (N + kRqThreads - 1) / kRqThreads);
  IWF_TRY(ar.get(&part, (size_t)np * nev * chunks));
  IWF_TRY(ar.get(&d_theta, (size_t)np * nev));
  if (ab) {
    const std::vector<int> ones(np, 1);
    IWF_CUDA(cudaMemcpyAsync(sm.active, ones.data(), sizeof(int) * np, cudaMemcpyHostToDevice, st));
  }
  IWF_TRY(apply_impl(p, IWF_PREC_F64, X, HX, nvec, st, nullptr, ab));
  *applies += nvec;
  rq_partial_kernel<<<dim3((unsigned)chunks, (unsigned)(np * nev)), kRqThreads, 0, st>>>(
      X, HX, N, ab ? b : nev, nev, chunks, part);
  IWF_CUDA(cudaGetLastError());
  count_launch();
  rq_final_kernel<<<(np * nev + 127) / 128, 128, 0, st>>>(part, chunks, np * nev, d_theta);
  IWF_CUDA(cudaGetLastError());
  count_launch();
  IWF_CUDA(cudaMemcpyAsync(out, d_theta, sizeof(double) * np * nev, cudaMemcpyDeviceToHost, st));
  return check_apply_error(p, st);
}

// Shared driver: problems 0..np-1 with preconditioner parameters already on the device.
iwf_status solve_problems(iwf_plan* p, const ApplyBatch* ab, const iwf_solve_opts* o,
                          Small& sm, Arena& ar, const void* X0, double* evals, void* evecs,
                          double* resid, int* iters_out, iwf_solve_info* info, cudaStream_t st) {
  const int np = sm.nprob;
  const int nev = o->nev;
  const int b = o->block > 0 ? o->block : nev;
  const double tol = o->tol > 0 ? o->tol : 1e-10;
  const int maxit = o->maxit > 0 ? o->maxit : 1000;
  const long long N = p->g.N;
  const size_t all = (size_t)N * b * np;
  const auto t0 = std::chrono::steady_clock::now();
  double2* X;
  int* flag;
  IWF_TRY(ar.get(&X, all));
  IWF_TRY(ar.get(&flag, 1));     // requested either way: the workspace sequence stays fixed
  if (X0) {
    // a non-finite start block is an input error (it would otherwise surface later, or be
    // masked by the orthonormalisation dropping its columns)
    int h_flag = 0;
    IWF_TRY(any_nonfinite(reinterpret_cast<const double*>(X0), 2 * (long long)all, flag, st));
    IWF_CUDA(cudaMemcpyAsync(&h_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    IWF_CUDA(cudaStreamSynchronize(st));
    if (h_flag) return fail(IWF_ERR_NONFINITE, "iwf_eigensolve: non-finite start block X0");
  }
  PhaseResult r1, r2;
  if (o->precision == IWF_PREC_C64) {
    float2* Xf;
    IWF_TRY(ar.get(&Xf, all));
    if (X0) IWF_TRY((convert_block<double, float>(X0, Xf, 2 * (long long)all, st)));
    else IWF_TRY(random_block<float>(Xf, N, b * np, o->seed, st));
    const double tol1 = std::max(tol, o->c64_tol > 0 ? o->c64_tol : 1e-5);
    IWF_TRY(run_phase<float>(p, ab, b, nev, maxit, tol1, 10, Xf, sm, ar, st, r1, kEngineTensor));
    IWF_TRY((convert_block<float, double>(Xf, X, 2 * (long long)all, st)));
  } else {
    if (X0) IWF_CUDA(cudaMemcpyAsync(X, X0, sizeof(double2) * all, cudaMemcpyDeviceToDevice, st));
    else IWF_TRY(random_block<double>(X, N, b * np, o->seed, st));
  }
  const int left = std::max(1, maxit - r1.rounds);
  const int engine = o->precision == IWF_PREC_F64_EXACT ? kEngineF64
                     : o->precision == IWF_PREC_F64_DF  ? kEngineDF
                                                        : kEngineTensor;
  IWF_TRY(run_phase<double>(p, ab, b, nev, left, tol, 0, X, sm, ar, st, r2, engine));
  std::vector<double> rq((size_t)np * nev);
  long long rq_applies = 0;
  IWF_TRY(rayleigh_quotients(p, ab, sm, ar, X, b, nev, rq.data(), &rq_applies, st));
  if (evecs) {
    for (int q = 0; q < np; ++q)
      IWF_CUDA(cudaMemcpyAsync(reinterpret_cast<double2*>(evecs) + (size_t)q * N * nev,
                               X + (size_t)q * N * b, sizeof(double2) * N * nev,
                               cudaMemcpyDeviceToDevice, st));
  }
  IWF_CUDA(cudaStreamSynchronize(st));
  bool all_conv = true;
  double worst = 0;
  for (int q = 0; q < np; ++q) {
    for (int j = 0; j < nev; ++j) {
      evals[(size_t)q * nev + j] = rq[(size_t)q * nev + j];
      const double r = r2.resid[(size_t)q * kMaxBlock + j];
      if (resid) resid[(size_t)q * nev + j] = r;
      worst = std::max(worst, r);
    }
    if (iters_out) iters_out[q] = (r1.iters.empty() ? 0 : r1.iters[q]) + r2.iters[q];
    all_conv = all_conv && r2.converged[q];
  }
  if (info) {
    info->iters = r1.rounds + r2.rounds;
    info->iters_c64 = r1.rounds;
    info->applies = r1.applies + r2.applies + rq_applies;
    info->converged = all_conv ? 1 : 0;
    info->max_resid = worst;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (!all_conv) return fail(IWF_ERR_NOCONV, "eigensolver reached maxit before tol");
  return IWF_OK;
}

iwf_status check_opts(const iwf_plan* p, const iwf_solve_opts* o) {
  if (!o) return fail(IWF_ERR_ARG, "iwf_eigensolve: NULL options");
  const int nev = o->nev;
  const int b = o->block > 0 ? o->block : nev;
  if (nev < 1 || b < nev || b > kMaxBlock)
    return fail(IWF_ERR_ARG, "iwf_eigensolve: need 1 <= nev <= block <= 24");
  if ((long long)3 * b > p->g.N) return fail(IWF_ERR_ARG, "iwf_eigensolve: window too small for the block");
  if (o->precision != IWF_PREC_F64 && o->precision != IWF_PREC_C64 &&
      o->precision != IWF_PREC_F64_EXACT && o->precision != IWF_PREC_F64_DF)
    return fail(IWF_ERR_ARG, "iwf_eigensolve: unknown precision");
  return IWF_OK;
}

// The solve runs on a library stream ordered after the caller's stream (so it can be
// captured into graphs whatever stream the caller uses).
struct SolveStream {
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  ~SolveStream() {
    if (ev) cudaEventDestroy(ev);
    if (s) cudaStreamDestroy(s);
  }
  iwf_status open(cudaStream_t caller) {
    IWF_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    IWF_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    IWF_CUDA(cudaEventRecord(ev, caller));
    IWF_CUDA(cudaStreamWaitEvent(s, ev, 0));
    return IWF_OK;
  }
};

}  // namespace

iwf_status eigensolve_impl(iwf_plan* p, const iwf_solve_opts* o, const void* X0, double* evals,
                           void* evecs, double* resid, iwf_solve_info* info, cudaStream_t st) {
  IWF_TRY(check_opts(p, o));
  if (!evals || !evecs) return fail(IWF_ERR_ARG, "iwf_eigensolve: NULL output");
  if (p->pot_kind == 0) return fail(IWF_ERR_ARG, "iwf_eigensolve: no potential set");
  SolveStream ss;
  IWF_TRY(ss.open(st));
  Arena ar(p);
  Small sm;
  IWF_TRY(alloc_small(ar, sm, 1));
  const double sigma = p->voff_abs - p->vg0 + 1.0;
  const double shift = p->vg0 + sigma, off2 = p->voff_sq;
  IWF_CUDA(cudaMemcpyAsync(sm.shift, &shift, sizeof(double), cudaMemcpyHostToDevice, ss.s));
  IWF_CUDA(cudaMemcpyAsync(sm.off2, &off2, sizeof(double), cudaMemcpyHostToDevice, ss.s));
  int iters = 0;
  return solve_problems(p, nullptr, o, sm, ar, X0, evals, evecs, resid, &iters, info, ss.s);
}

iwf_status batch_eigensolve_impl(iwf_plan* p, int nprob, const int* nmodes, const int* m,
                                 const double* re, const double* im, const iwf_solve_opts* o,
                                 const void* X0, double* evals, void* evecs, double* resid,
                                 int* iters, iwf_solve_info* info, cudaStream_t st) {
  IWF_TRY(check_opts(p, o));
  if (nprob < 1 || !nmodes || !evals) return fail(IWF_ERR_ARG, "iwf_batch_eigensolve: bad arguments");
  const int b = o->block > 0 ? o->block : o->nev;
  if ((long long)nprob * b > 65535) return fail(IWF_ERR_ARG, "iwf_batch_eigensolve: nprob * block > 65535");
  SolveStream ss;
  IWF_TRY(ss.open(st));
  Arena ar(p);
  Small sm;
  IWF_TRY(alloc_small(ar, sm, nprob));
  long long stride = 0;
  for (int j = 0; j < p->g.n; ++j) stride += p->g.lens[j];
  double* tab64;
  float* tab32;
  IWF_TRY(ar.get(&tab64, (size_t)nprob * stride));
  IWF_TRY(ar.get(&tab32, (size_t)nprob * stride));
  std::vector<double> shift(nprob), off2(nprob);
  long long mo = 0;
  for (int q = 0; q < nprob; ++q) {
    if (nmodes[q] < 0 || (nmodes[q] > 0 && (!m || !re || !im)))
      return fail(IWF_ERR_ARG, "iwf_batch_eigensolve: bad mode list");
    PotSummary s;
    IWF_TRY(potential_tables(p, nmodes[q], m + mo * p->g.n, re + mo, im + mo,
                             tab64 + (size_t)q * stride, tab32 + (size_t)q * stride, &s, ss.s));
    const double sigma = s.off_abs - s.vg0 + 1.0;
    shift[q] = s.vg0 + sigma;
    off2[q] = s.off_sq;
    mo += nmodes[q];
  }
  IWF_CUDA(cudaMemcpyAsync(sm.shift, shift.data(), sizeof(double) * nprob, cudaMemcpyHostToDevice, ss.s));
  IWF_CUDA(cudaMemcpyAsync(sm.off2, off2.data(), sizeof(double) * nprob, cudaMemcpyHostToDevice, ss.s));
  ApplyBatch ab{tab64, tab32, stride, b, sm.active};
  return solve_problems(p, &ab, o, sm, ar, X0, evals, evecs, resid, iters, info, ss.s);
}

// ---------------------------------------------------------------------------------------
// Many plans in one call. Plans with the same geometry (P, K, L, method, shift) form a group
// that runs as one lockstep batch (per-problem potential tables, captured graphs); groups run
// side by side on their own streams and host threads, as many at a time as fit in about 60 %
// of the free device memory, largest first.
namespace {

bool same_geometry(const iwf_plan* a, const iwf_plan* b) {
  if (a->device != b->device || a->method != b->method || a->shift_round != b->shift_round ||
      a->g.d != b->g.d || a->g.n != b->g.n)
    return false;
  for (int j = 0; j < a->g.n; ++j)
    if (a->g.lens[j] != b->g.lens[j]) return false;
  return std::memcmp(a->P, b->P, sizeof(double) * a->g.d * a->g.n) == 0;
}

struct GroupJob {
  std::vector<int> idx;        // plans of the group, in call order
  size_t bytes = 0;            // device memory estimate of its solve
  iwf_status st = IWF_OK;
  std::string msg;
  iwf_solve_info info{};
};

iwf_status run_group(iwf_plan* const* plans, GroupJob& job, const iwf_solve_opts* o,
                     const void* const* X0, double* evals, void* const* evecs, double* resid,
                     int* iters, cudaStream_t caller) {
  iwf_plan* gp = plans[job.idx[0]];
  DeviceGuard guard(gp->device);
  const int np = (int)job.idx.size();
  const int nev = o->nev;
  const int b = o->block > 0 ? o->block : nev;
  const long long N = gp->g.N;
  IWF_TRY(check_opts(gp, o));
  SolveStream ss;
  IWF_TRY(ss.open(caller));
  Arena ar;
  Small sm;
  IWF_TRY(alloc_small(ar, sm, np));
  long long stride = 0;
  for (int j = 0; j < gp->g.n; ++j) stride += gp->g.lens[j];
  double* tab64;
  float* tab32;
  IWF_TRY(ar.get(&tab64, (size_t)np * stride));
  IWF_TRY(ar.get(&tab32, (size_t)np * stride));
  // each plan's per-axis tables, with its constant term folded into axis 0 (the batched
  // apply's convention), and its preconditioner parameters
  std::vector<double> t64((size_t)np * stride), shift(np), off2(np);
  std::vector<float> t32((size_t)np * stride);
  for (int q = 0; q < np; ++q) {
    const iwf_plan* p = plans[job.idx[q]];
    IWF_CUDA(cudaMemcpy(t64.data() + (size_t)q * stride, p->d_tab64, sizeof(double) * stride,
                        cudaMemcpyDeviceToHost));
    const double c = p->vconst / (double)N;
    for (int l = 0; l < gp->g.lens[0]; ++l) t64[(size_t)q * stride + p->tab_off[0] + l] += c;
    const double sigma = p->voff_abs - p->vg0 + 1.0;
    shift[q] = p->vg0 + sigma;
    off2[q] = p->voff_sq;
  }
  for (size_t i = 0; i < t64.size(); ++i) t32[i] = (float)t64[i];
  IWF_CUDA(cudaMemcpyAsync(tab64, t64.data(), sizeof(double) * t64.size(), cudaMemcpyHostToDevice, ss.s));
  IWF_CUDA(cudaMemcpyAsync(tab32, t32.data(), sizeof(float) * t32.size(), cudaMemcpyHostToDevice, ss.s));
  IWF_CUDA(cudaMemcpyAsync(sm.shift, shift.data(), sizeof(double) * np, cudaMemcpyHostToDevice, ss.s));
  IWF_CUDA(cudaMemcpyAsync(sm.off2, off2.data(), sizeof(double) * np, cudaMemcpyHostToDevice, ss.s));
  // start blocks: the caller's where given, else the seeded random block
  double2* X0cat = nullptr;
  bool any_x0 = false;
  for (int q = 0; q < np && X0; ++q) any_x0 = any_x0 || X0[job.idx[q]] != nullptr;
  if (any_x0) {
    IWF_TRY(ar.get(&X0cat, (size_t)np * b * N));
    for (int q = 0; q < np; ++q) {
      double2* dst = X0cat + (size_t)q * b * N;
      const void* src = X0[job.idx[q]];
      if (src) IWF_CUDA(cudaMemcpyAsync(dst, src, sizeof(double2) * b * N, cudaMemcpyDeviceToDevice, ss.s));
      else IWF_TRY(random_block<double>(dst, N, b, o->seed + 7919ull * (unsigned long long)q, ss.s));
    }
  }
  double2* V = nullptr;
  bool any_v = false;
  for (int q = 0; q < np && evecs; ++q) any_v = any_v || evecs[job.idx[q]] != nullptr;
  if (any_v) IWF_TRY(ar.get(&V, (size_t)np * nev * N));
  std::vector<double> ev((size_t)np * nev), rs((size_t)np * nev);
  std::vector<int> it(np);
  ApplyBatch ab{tab64, tab32, stride, b, sm.active};
  const iwf_status st = solve_problems(gp, &ab, o, sm, ar, X0cat, ev.data(), V, rs.data(),
                                       it.data(), &job.info, ss.s);
  if (st != IWF_OK && st != IWF_ERR_NOCONV) return st;
  for (int q = 0; q < np; ++q) {
    const int k = job.idx[q];
    for (int j = 0; j < nev; ++j) {
      evals[(size_t)k * nev + j] = ev[(size_t)q * nev + j];
      if (resid) resid[(size_t)k * nev + j] = rs[(size_t)q * nev + j];
    }
    if (iters) iters[k] = it[q];
    if (V && evecs[k])
      IWF_CUDA(cudaMemcpyAsync(evecs[k], V + (size_t)q * nev * N, sizeof(double2) * nev * N,
                               cudaMemcpyDeviceToDevice, ss.s));
  }
  IWF_CUDA(cudaStreamSynchronize(ss.s));
  return st;
}

}  // namespace

iwf_status batch_solve_impl(int nplans, iwf_plan* const* plans, const iwf_solve_opts* o,
                            const void* const* X0, double* evals, void* const* evecs,
                            double* resid, int* iters, iwf_solve_info* info,
                            cudaStream_t st) {
  if (nplans < 1 || !plans || !o || !evals) return fail(IWF_ERR_ARG, "iwf_batch_solve: bad arguments");
  const auto t0 = std::chrono::steady_clock::now();
  const int nev = o->nev;
  const int b = o->block > 0 ? o->block : nev;
  std::vector<GroupJob> jobs;
  for (int k = 0; k < nplans; ++k) {
    iwf_plan* p = plans[k];
    if (!p) return fail(IWF_ERR_ARG, "iwf_batch_solve: NULL plan");
    if (p->pot_kind == 0) return fail(IWF_ERR_ARG, "iwf_batch_solve: a plan has no potential");
    if (p->pot_kind != 1)
      return fail(IWF_ERR_UNSUPPORTED, "iwf_batch_solve: every potential must be a sum of "
                                       "single-axis modes (per-axis tables)");
    if (p->device != plans[0]->device)
      return fail(IWF_ERR_ARG, "iwf_batch_solve: all plans must live on one device");
    IWF_TRY(check_opts(p, o));
    bool placed = false;
    for (auto& j : jobs)
      if (same_geometry(plans[j.idx[0]], p)) { j.idx.push_back(k); placed = true; break; }
    if (!placed) { jobs.emplace_back(); jobs.back().idx.push_back(k); }
  }
  for (auto& j : jobs) {
    const size_t N = (size_t)plans[j.idx[0]]->g.N;
    // complex-double blocks (12) and, in the mixed mode, complex-float ones (11)
    const size_t per = (size_t)b * N * (12 * 16 + (o->precision == IWF_PREC_C64 ? 11 * 8 : 0));
    j.bytes = per * j.idx.size();
    if ((long long)j.idx.size() * b > 65535) return fail(IWF_ERR_ARG, "iwf_batch_solve: a group exceeds 65535 vectors");
  }
  std::sort(jobs.begin(), jobs.end(), [](const GroupJob& a, const GroupJob& c) { return a.bytes > c.bytes; });
  size_t free_b = 0, total_b = 0;
  {
    DeviceGuard guard(plans[0]->device);
    IWF_CUDA(cudaMemGetInfo(&free_b, &total_b));
  }
  const size_t budget = (size_t)(0.6 * (double)free_b);
  // launch groups while their estimates fit; the first one always runs
  std::vector<std::thread> running;
  std::vector<size_t> run_bytes;
  size_t in_use = 0;
  std::mutex mu;
  size_t next = 0;
  while (next < jobs.size() || !running.empty()) {
    while (next < jobs.size() && (running.empty() || in_use + jobs[next].bytes <= budget)) {
      GroupJob& j = jobs[next];
      in_use += j.bytes;
      running.emplace_back([&, jp = &j]() {
        jp->st = run_group(plans, *jp, o, X0, evals, evecs, resid, iters, st);
        if (jp->st != IWF_OK) jp->msg = iwf_last_error();
      });
      run_bytes.push_back(j.bytes);
      ++next;
    }
    // wait for the oldest running group, then admit more
    running.front().join();
    in_use -= run_bytes.front();
    running.erase(running.begin());
    run_bytes.erase(run_bytes.begin());
  }
  iwf_status out = IWF_OK;
  std::string msg;
  long long applies = 0;
  int max_it = 0, conv = 1;
  double worst = 0.0;
  for (const auto& j : jobs) {
    if (j.st != IWF_OK && (out == IWF_OK || out == IWF_ERR_NOCONV)) { out = j.st; msg = j.msg; }
    applies += j.info.applies;
    max_it = std::max(max_it, j.info.iters);
    conv = conv && j.info.converged;
    worst = std::max(worst, j.info.max_resid);
  }
  if (info) {
    info->iters = max_it;
    info->iters_c64 = 0;
    info->applies = applies;
    info->converged = conv;
    info->max_resid = worst;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (out != IWF_OK) return fail(out, msg);
  return IWF_OK;
}

}  // namespace iwf
