// Block LOBPCG for the lowest eigenpairs of H~ (Sec. 4.1, Alg. 2 in block form).
//
// Every iteration keeps an orthonormal basis S = [X W P] of the trial subspace:
//   R = H X - X diag(theta), W = M R            (preconditioner of Eq. precond, shifted)
//   W <- W - [X P]([X P]^H W), twice            (classical Gram-Schmidt, reorthogonalised)
//   W <- W D U S^{-1/2}, twice                   (SVQB; dependent directions dropped)
//   HW = H W                                      (the FFT apply)
//   A = S^H [HX HW HP]; A = Y diag(theta) Y^H     (one-CTA Jacobi, FP64)
//   X <- S Yx, P <- S Yp with Yp orthonormalised against Yx in the small space, so that
//   [X P] stays orthonormal without touching the long vectors again.
// Mixed precision: a first phase stores the blocks in complex float and applies H in
// complex float (Gram sums in float within 16-row tiles, double across tiles); its X then
// seeds the FP64 phase, which runs to the requested tolerance.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cmath>
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

template <typename T> constexpr int prec_of() { return sizeof(T) == 8 ? IWF_PREC_F64 : IWF_PREC_C64; }

struct SmallBufs {
  double2* G = nullptr;       // kMaxSmall^2
  double2* Cx = nullptr;      // kMaxSmall x kMaxBlock
  double2* Cp = nullptr;
  double2* T = nullptr;       // kMaxBlock^2
  double* theta = nullptr;    // kMaxBlock
  double* resid = nullptr;    // kMaxBlock
  int* mask = nullptr;        // kMaxSmall (X | W | P)
  int* maskw = nullptr;       // kMaxBlock
  int* maskp = nullptr;       // kMaxBlock
  int* status = nullptr;
  double2* partial = nullptr; // slots x kMaxSmall^2
  double* rpartial = nullptr; // slots x kMaxBlock
  int slots = 608;
};

struct Arena {
  std::vector<void*> ptrs;
  ~Arena() { for (void* p : ptrs) cudaFree(p); }
  template <typename U>
  iwf_status get(U** out, size_t count) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(U));
    if (e != cudaSuccess) return fail(IWF_ERR_ALLOC, "eigensolver workspace allocation failed");
    ptrs.push_back(p);
    *out = reinterpret_cast<U*>(p);
    return IWF_OK;
  }
};

iwf_status alloc_small(Arena& ar, SmallBufs& s) {
  IWF_TRY(ar.get(&s.G, kMaxSmall * kMaxSmall));
  IWF_TRY(ar.get(&s.Cx, kMaxSmall * kMaxBlock));
  IWF_TRY(ar.get(&s.Cp, kMaxSmall * kMaxBlock));
  IWF_TRY(ar.get(&s.T, kMaxBlock * kMaxBlock));
  IWF_TRY(ar.get(&s.theta, kMaxBlock));
  IWF_TRY(ar.get(&s.resid, kMaxBlock));
  IWF_TRY(ar.get(&s.mask, kMaxSmall));
  IWF_TRY(ar.get(&s.maskw, kMaxBlock));
  IWF_TRY(ar.get(&s.maskp, kMaxBlock));
  IWF_TRY(ar.get(&s.status, 1));
  IWF_TRY(ar.get(&s.partial, (size_t)s.slots * kMaxSmall * kMaxSmall));
  IWF_TRY(ar.get(&s.rpartial, (size_t)s.slots * kMaxBlock));
  return IWF_OK;
}

struct PhaseResult {
  int iters = 0;
  long long applies = 0;
  bool converged = false;
  std::vector<double> theta, resid;
};

BlockList blocks(std::initializer_list<const void*> ps, int b) {
  BlockList L{};
  int i = 0;
  for (const void* p : ps) L.p[i++] = p;
  L.nb = i;
  L.b = b;
  return L;
}

// One LOBPCG phase with blocks stored as T. X (N x b) is the start block (overwritten by
// the result); stops when the first nev residuals are <= tol, after maxit iterations, or
// (when stall > 0) when the largest of them has not halved over `stall` iterations.
template <typename T>
iwf_status run_phase(iwf_plan* p, int b, int nev, int maxit, double tol, int stall, void* Xio,
                     const SmallBufs& sb, Arena& ar, cudaStream_t st, PhaseResult& res) {
  using V2 = typename Cplx<T>::type;
  const long long N = p->g.N;
  const size_t blk = (size_t)N * b;
  V2 *X, *HX, *W, *HW, *P, *HP, *X2, *HX2, *P2, *HP2, *W2;
  T* M;
  IWF_TRY(ar.get(&HX, blk)); IWF_TRY(ar.get(&W, blk)); IWF_TRY(ar.get(&HW, blk));
  IWF_TRY(ar.get(&P, blk)); IWF_TRY(ar.get(&HP, blk)); IWF_TRY(ar.get(&X2, blk));
  IWF_TRY(ar.get(&HX2, blk)); IWF_TRY(ar.get(&P2, blk)); IWF_TRY(ar.get(&HP2, blk));
  IWF_TRY(ar.get(&W2, blk)); IWF_TRY(ar.get(&M, (size_t)N));
  X = reinterpret_cast<V2*>(Xio);
  V2* Xorig = X;
  const double sigma = p->voff_abs - p->vg0 + 1.0;
  IWF_TRY(precond_diag<T>(p->d_lam64, p->vg0 + sigma, p->voff_sq, N, M, st));
  const int prec = prec_of<T>();
  std::vector<double> h_resid(b), h_theta(b);
  int h_status = 0;

  auto orthonormalize = [&](V2*& Y, V2*& Y2, int* mask) -> iwf_status {
    for (int pass = 0; pass < 2; ++pass) {
      IWF_TRY(gram<T>(blocks({Y}, b), blocks({Y}, b), N, sb.G, sb.partial, sb.slots, st));
      IWF_TRY(svqb_small(sb.G, b, 1e-14, sb.T, mask, sb.status, st));
      IWF_TRY(block_update<T>(blocks({Y}, b), N, sb.T, nullptr, b, Y2, nullptr, false, st));
      std::swap(Y, Y2);
    }
    return IWF_OK;
  };
  // Rayleigh-Ritz on X alone: X <- X Y, HX <- HX Y, theta
  auto rr_x = [&]() -> iwf_status {
    IWF_TRY(gram<T>(blocks({X}, b), blocks({HX}, b), N, sb.G, sb.partial, sb.slots, st));
    IWF_TRY(set_mask(sb.mask, b, 1, st));
    IWF_TRY(rayleigh_ritz_small(sb.G, b, b, sb.mask, b, sb.theta, sb.Cx, sb.Cp, sb.maskp,
                                sb.status, st));
    IWF_TRY(block_update<T>(blocks({X}, b), N, sb.Cx, nullptr, b, X2, nullptr, false, st));
    IWF_TRY(block_update<T>(blocks({HX}, b), N, sb.Cx, nullptr, b, HX2, nullptr, false, st));
    std::swap(X, X2);
    std::swap(HX, HX2);
    return IWF_OK;
  };
  auto apply = [&](const V2* in, V2* out) -> iwf_status {
    IWF_TRY(apply_impl(p, prec, in, out, b, st));
    res.applies += b;
    return IWF_OK;
  };
  auto read_small = [&]() -> iwf_status {
    IWF_CUDA(cudaMemcpyAsync(h_resid.data(), sb.resid, sizeof(double) * b, cudaMemcpyDeviceToHost, st));
    IWF_CUDA(cudaMemcpyAsync(h_theta.data(), sb.theta, sizeof(double) * b, cudaMemcpyDeviceToHost, st));
    IWF_CUDA(cudaMemcpyAsync(&h_status, sb.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    IWF_CUDA(cudaStreamSynchronize(st));
    return IWF_OK;
  };

  // start: orthonormalise X, apply, Rayleigh-Ritz on X
  IWF_TRY(orthonormalize(X, X2, sb.maskw));
  IWF_TRY(apply(X, HX));
  IWF_TRY(rr_x());
  bool hasP = false;
  double best = INFINITY;
  int best_it = 0;
  bool verified = false;
  for (int it = 0; it <= maxit; ++it) {
    IWF_TRY(residual_precond<T>(X, HX, sb.theta, M, W, N, b, sb.rpartial, sb.slots, sb.resid, st));
    IWF_TRY(read_small());
    if (h_status != 0) return fail(IWF_ERR_BREAKDOWN, "Rayleigh-Ritz subspace lost rank");
    double worst = 0;
    for (int j = 0; j < nev; ++j) {
      if (!std::isfinite(h_resid[j]) || !std::isfinite(h_theta[j]))
        return fail(IWF_ERR_NONFINITE, "non-finite residual in the eigensolver");
      worst = std::max(worst, h_resid[j]);
    }
    res.iters = it;
    if (log_level() > 0) {
      std::fprintf(stderr, "[iwf] %s it %d worst %.3e theta0 %.12f theta%d %.12f\n",
                   sizeof(T) == 8 ? "f64" : "c64", it, worst, h_theta[0], nev - 1, h_theta[nev - 1]);
      if (log_level() > 1) {
        for (int j = 0; j < b; ++j) std::fprintf(stderr, " %.2e", h_resid[j]);
        std::fprintf(stderr, "\n");
      }
    }
    if (worst <= tol) {
      if (verified) { res.converged = true; break; }
      // recompute H X explicitly (removes drift of the implicit HX updates), re-check
      IWF_TRY(apply(X, HX));
      IWF_TRY(rr_x());
      verified = true;
      --it;
      continue;
    }
    verified = false;
    if (it == maxit) break;
    if (stall > 0) {
      if (worst < 0.5 * best) { best = worst; best_it = it; }
      else if (it - best_it >= stall) break;
    }
    // W <- W - [X P]([X P]^H W), twice
    for (int pass = 0; pass < 2; ++pass) {
      const BlockList XP = hasP ? blocks({X, P}, b) : blocks({X}, b);
      IWF_TRY(gram<T>(XP, blocks({W}, b), N, sb.G, sb.partial, sb.slots, st));
      IWF_TRY(block_update<T>(XP, N, sb.G, nullptr, b, W, nullptr, true, st));
    }
    IWF_TRY(orthonormalize(W, W2, sb.maskw));
    IWF_TRY(apply(W, HW));
    const int m = hasP ? 3 * b : 2 * b;
    const BlockList S = hasP ? blocks({X, W, P}, b) : blocks({X, W}, b);
    const BlockList HS = hasP ? blocks({HX, HW, HP}, b) : blocks({HX, HW}, b);
    IWF_TRY(gram<T>(S, HS, N, sb.G, sb.partial, sb.slots, st));
    IWF_TRY(set_mask(sb.mask, b, 1, st));
    IWF_CUDA(cudaMemcpyAsync(sb.mask + b, sb.maskw, sizeof(int) * b, cudaMemcpyDeviceToDevice, st));
    if (hasP)
      IWF_CUDA(cudaMemcpyAsync(sb.mask + 2 * b, sb.maskp, sizeof(int) * b, cudaMemcpyDeviceToDevice, st));
    IWF_TRY(rayleigh_ritz_small(sb.G, m, b, sb.mask, b, sb.theta, sb.Cx, sb.Cp, sb.maskp,
                                sb.status, st));
    IWF_TRY(block_update<T>(S, N, sb.Cx, sb.Cp, b, X2, P2, false, st));
    IWF_TRY(block_update<T>(HS, N, sb.Cx, sb.Cp, b, HX2, HP2, false, st));
    std::swap(X, X2); std::swap(HX, HX2); std::swap(P, P2); std::swap(HP, HP2);
    hasP = true;
  }
  res.theta = h_theta;
  res.resid = h_resid;
  if (X != Xorig)
    IWF_CUDA(cudaMemcpyAsync(Xorig, X, sizeof(V2) * blk, cudaMemcpyDeviceToDevice, st));
  IWF_CUDA(cudaStreamSynchronize(st));
  return IWF_OK;
}

}  // namespace

iwf_status eigensolve_impl(iwf_plan* p, const iwf_solve_opts* o, const void* X0, double* evals,
                           void* evecs, double* resid, iwf_solve_info* info, cudaStream_t st) {
  if (!o) return fail(IWF_ERR_ARG, "iwf_eigensolve: NULL options");
  const int nev = o->nev;
  const int b = o->block > 0 ? o->block : nev;
  if (nev < 1 || b < nev || b > kMaxBlock)
    return fail(IWF_ERR_ARG, "iwf_eigensolve: need 1 <= nev <= block <= 24");
  if ((long long)3 * b > p->g.N) return fail(IWF_ERR_ARG, "iwf_eigensolve: window too small for the block");
  if (!evals || !evecs) return fail(IWF_ERR_ARG, "iwf_eigensolve: NULL output");
  if (p->pot_kind == 0) return fail(IWF_ERR_ARG, "iwf_eigensolve: no potential set");
  if (o->precision != IWF_PREC_F64 && o->precision != IWF_PREC_C64)
    return fail(IWF_ERR_ARG, "iwf_eigensolve: unknown precision");
  const double tol = o->tol > 0 ? o->tol : 1e-10;
  const int maxit = o->maxit > 0 ? o->maxit : 1000;
  const long long N = p->g.N;
  const auto t0 = std::chrono::steady_clock::now();

  Arena ar;
  SmallBufs sb;
  IWF_TRY(alloc_small(ar, sb));
  double2* X;
  IWF_TRY(ar.get(&X, (size_t)N * b));
  PhaseResult r1, r2;
  if (o->precision == IWF_PREC_C64) {
    float2* Xf;
    IWF_TRY(ar.get(&Xf, (size_t)N * b));
    if (X0) IWF_TRY((convert_block<double, float>(X0, Xf, 2 * N * b, st)));
    else IWF_TRY(random_block<float>(Xf, N, b, o->seed, st));
    const double tol1 = std::max(tol, o->c64_tol > 0 ? o->c64_tol : 1e-4);
    IWF_TRY(run_phase<float>(p, b, nev, maxit, tol1, 5, Xf, sb, ar, st, r1));
    IWF_TRY((convert_block<float, double>(Xf, X, 2 * N * b, st)));
  } else {
    if (X0) IWF_CUDA(cudaMemcpyAsync(X, X0, sizeof(double2) * N * b, cudaMemcpyDeviceToDevice, st));
    else IWF_TRY(random_block<double>(X, N, b, o->seed, st));
  }
  IWF_TRY(run_phase<double>(p, b, nev, std::max(1, maxit - r1.iters), tol, 0, X, sb, ar, st, r2));
  IWF_CUDA(cudaMemcpyAsync(evecs, X, sizeof(double2) * N * nev, cudaMemcpyDeviceToDevice, st));
  IWF_CUDA(cudaStreamSynchronize(st));
  for (int j = 0; j < nev; ++j) {
    evals[j] = r2.theta[j];
    if (resid) resid[j] = r2.resid[j];
  }
  if (info) {
    info->iters = r1.iters + r2.iters;
    info->iters_c64 = r1.iters;
    info->applies = r1.applies + r2.applies;
    info->converged = r2.converged ? 1 : 0;
    double w = 0;
    for (int j = 0; j < nev; ++j) w = std::max(w, r2.resid[j]);
    info->max_resid = w;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (!r2.converged) return fail(IWF_ERR_NOCONV, "eigensolver reached maxit before tol");
  return IWF_OK;
}

}  // namespace iwf
