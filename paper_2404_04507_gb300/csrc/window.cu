// Window construction on the device (Sec. 3.1-3.2) and the lifted potential (Sec. 4.1).
//
// For each k_II slice the window holds the k_I with k_I + Q k_II in [-K, K)^d, i.e. the 2K_j
// consecutive integers from lo_j = ceil(-K_j - q_j), q = Q k_II (exact shift), or
// lo_j = -K_j - round(q_j) (rounded shift). q is summed left to right with every product
// and sum rounded separately (__dmul_rn / __dadd_rn, no contraction), so the
// classification is reproducible. The true index of window position t in a slice is
// k_j = lo_j + t_j, which is the inverse of the index-shift map rho (Eqs. inverse1-3).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "common.cuh"

namespace iwf {

namespace {

constexpr double kTieEps = 1e-9;

struct WinArgs {
  Geom g;
  double Q[IWF_MAX_N * IWF_MAX_N];
  double P[IWF_MAX_N * IWF_MAX_N];
  int shift_round;
};

// k_II of slice s (C order over the k_II positions p_j = k_j + L_j).
__device__ __forceinline__ void slice_kII(const Geom& g, long long s, int* k) {
  for (int j = g.n - 1; j >= g.d; --j) {
    const int len = g.lens[j];
    k[j] = (int)(s % len) - g.half[j];
    s /= len;
  }
}

__device__ __forceinline__ double round_half_away(double q) {
  const double r = trunc(q);
  const double f = __dadd_rn(q, -r);
  return fabs(f) >= 0.5 ? __dadd_rn(r, copysign(1.0, q)) : r;
}

__global__ void lo_kernel(WinArgs a, int* lo, int* err) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= a.g.MII) return;
  int k[IWF_MAX_N];
  slice_kII(a.g, s, k);
  const int d = a.g.d, m = a.g.n - d;
  for (int j = 0; j < d; ++j) {
    double q = 0.0;
    for (int i = 0; i < m; ++i) {
      const double prod = __dmul_rn(a.Q[j * m + i], (double)k[d + i]);
      q = i ? __dadd_rn(q, prod) : prod;
    }
    const int K = a.g.half[j];
    int l;
    if (a.shift_round) {
      const double h = q - floor(q) - 0.5;
      if (fabs(h) < kTieEps && h != 0.0) atomicOr(err, 1);
      l = -K - (int)round_half_away(q);
    } else {
      const double t = __dadd_rn(-(double)K, -q);
      const double dist = fabs(t - rint(t));
      if (dist < kTieEps && dist != 0.0) atomicOr(err, 1);
      l = (int)ceil(t);
    }
    lo[s * d + j] = l;
  }
}

// True index of window position e (slice-major, k_I C order inside the slice).
__device__ __forceinline__ void window_index(const Geom& g, const int* lo, long long e, int* k) {
  const long long s = e / g.MI;
  long long t = e - s * g.MI;
  for (int j = g.d - 1; j >= 0; --j) {
    const int len = g.lens[j];
    k[j] = lo[s * g.d + j] + (int)(t % len);
    t /= len;
  }
  slice_kII(g, s, k);
}

__global__ void kinetic_kernel(WinArgs a, const int* lo, double* lam64, float* lam32) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= a.g.N) return;
  int k[IWF_MAX_N];
  window_index(a.g, lo, e, k);
  double s2 = 0.0;
  for (int r = 0; r < a.g.d; ++r) {
    double x = 0.0;
    for (int j = 0; j < a.g.n; ++j) x += a.P[r * a.g.n + j] * (double)k[j];
    s2 += x * x;
  }
  const double lam = 0.5 * s2;
  lam64[e] = lam;
  lam32[e] = (float)lam;
}

__global__ void export_kernel(Geom g, const int* lo, int* kout) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= g.N) return;
  int k[IWF_MAX_N];
  window_index(g, lo, e, k);
  for (int j = 0; j < g.n; ++j) kout[e * g.n + j] = k[j];
}

// V(y_l) for one grid point from the folded mode list: Re sum_m c_m exp(2 pi i sum_j m_j l_j / len_j).
struct ModeArgs {
  Geom g;
  int nmodes;
  const int* m;        // nmodes x n, already reduced to [0, len_j)
  const double* re;
  const double* im;
  double scale;        // 1/N
};

__device__ double mode_sum(const ModeArgs& a, const int* l) {
  double v = 0.0;
  for (int q = 0; q < a.nmodes; ++q) {
    double frac = 0.0;
    for (int j = 0; j < a.g.n; ++j) {
      const int len = a.g.lens[j];
      const int ph = (int)(((long long)a.m[q * a.g.n + j] * l[j]) % len);
      frac += (double)ph / (double)len;
    }
    frac -= floor(frac);
    double s, c;
    sincospi(2.0 * frac, &s, &c);
    v += a.re[q] * c - a.im[q] * s;
  }
  return v;
}

// Per-axis tables: entry (axis j, l) = V restricted to the modes on axis j, at y_j = 2 pi l/len_j.
__global__ void axis_table_kernel(ModeArgs a, const int* mode_axis, int total, const int* tab_axis,
                                  const int* tab_l, double* t64, float* t32, int fold_const) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int ax = tab_axis[i];
  int l[IWF_MAX_N] = {0};
  l[ax] = tab_l[i];
  double v = 0.0;
  for (int q = 0; q < a.nmodes; ++q) {
    if (fold_const && ax == 0 && mode_axis[q] < 0) { v += a.re[q]; continue; }
    if (mode_axis[q] != ax) continue;
    const int len = a.g.lens[ax];
    const int ph = (int)(((long long)a.m[q * a.g.n + ax] * l[ax]) % len);
    double s, c;
    sincospi(2.0 * (double)ph / (double)len, &s, &c);
    v += a.re[q] * c - a.im[q] * s;
  }
  v *= a.scale;
  t64[i] = v;
  t32[i] = (float)v;
}

// Full grid in data layout: l_II (slow, C order) then l_I (fast, C order).
__global__ void grid_kernel(ModeArgs a, double* g64, float* g32) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= a.g.N) return;
  int l[IWF_MAX_N];
  long long r = e;
  for (int j = a.g.d - 1; j >= 0; --j) { l[j] = (int)(r % a.g.lens[j]); r /= a.g.lens[j]; }
  for (int j = a.g.n - 1; j >= a.g.d; --j) { l[j] = (int)(r % a.g.lens[j]); r /= a.g.lens[j]; }
  const double v = mode_sum(a, l) * a.scale;
  g64[e] = v;
  g32[e] = (float)v;
}

template <typename T>
iwf_status dev_alloc(T** ptr, size_t count) {
  if (*ptr) { cudaFree(*ptr); *ptr = nullptr; }
  if (count == 0) return IWF_OK;
  cudaError_t e = cudaMalloc((void**)ptr, count * sizeof(T));
  if (e != cudaSuccess) { *ptr = nullptr; return cuda_fail(e, "cudaMalloc"); }
  return IWF_OK;
}

template <typename T>
struct DevBuf {
  T* p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
};

}  // namespace

iwf_status build_window_tables(iwf_plan* p) {
  const Geom& g = p->g;
  WinArgs a{};
  a.g = g;
  a.shift_round = p->shift_round;
  for (int i = 0; i < g.d * (g.n - g.d); ++i) a.Q[i] = p->Q[i];
  for (int i = 0; i < g.d * g.n; ++i) a.P[i] = p->P[i];
  IWF_TRY(dev_alloc(&p->d_lo, (size_t)g.MII * g.d));
  IWF_TRY(dev_alloc(&p->d_lam64, (size_t)g.N));
  IWF_TRY(dev_alloc(&p->d_lam32, (size_t)g.N));
  IWF_CUDA(cudaMemset(p->d_err, 0, sizeof(int)));
  const int T = 256;
  lo_kernel<<<(unsigned)((g.MII + T - 1) / T), T>>>(a, p->d_lo, p->d_err);
  IWF_CUDA(cudaGetLastError());
  kinetic_kernel<<<(unsigned)((g.N + T - 1) / T), T>>>(a, p->d_lo, p->d_lam64, p->d_lam32);
  IWF_CUDA(cudaGetLastError());
  int err = 0;
  IWF_CUDA(cudaMemcpy(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) return fail(IWF_ERR_WINDOW_TIE, "a window bound lies within 1e-9 of an integer");
  return IWF_OK;
}

iwf_status export_window(const iwf_plan* p, int* k_host) {
  const Geom& g = p->g;
  DevBuf<int> buf;
  IWF_CUDA(cudaMalloc((void**)&buf.p, (size_t)g.N * g.n * sizeof(int)));
  const int T = 256;
  export_kernel<<<(unsigned)((g.N + T - 1) / T), T>>>(g, p->d_lo, buf.p);
  IWF_CUDA(cudaGetLastError());
  IWF_CUDA(cudaMemcpy(k_host, buf.p, (size_t)g.N * g.n * sizeof(int), cudaMemcpyDeviceToHost));
  return IWF_OK;
}

namespace {
struct Folded {
  std::vector<int> m;          // modes reduced to [0, len_j), merged
  std::vector<double> re, im;
  std::vector<int> axis;       // -1 constant, j single-axis, -2 several axes
  double vg0 = 0, off_abs = 0, off_sq = 0, vconst = 0;
  bool separable = true;
};

// Fold the modes onto the grid (aliasing rule), merge duplicates, check that V is real and
// classify every mode by the lifted axes it touches.
iwf_status fold_modes(const Geom& g, int nmodes, const int* m, const double* re,
                      const double* im, Folded& out) {
  const int n = g.n;
  std::vector<int>& fm = out.m;
  std::vector<double>& fre = out.re;
  std::vector<double>& fim = out.im;
  for (int q = 0; q < nmodes; ++q) {
    if (!std::isfinite(re[q]) || !std::isfinite(im[q]))
      return fail(IWF_ERR_NONFINITE, "iwf_set_potential: non-finite coefficient");
    int red[IWF_MAX_N];
    for (int j = 0; j < n; ++j) {
      const int len = g.lens[j];
      int v = m[q * n + j] % len;
      red[j] = v < 0 ? v + len : v;
    }
    int hit = -1;
    for (size_t r = 0; r < fre.size(); ++r) {
      bool same = true;
      for (int j = 0; j < n && same; ++j) same = fm[r * n + j] == red[j];
      if (same) { hit = (int)r; break; }
    }
    if (hit < 0) {
      fm.insert(fm.end(), red, red + n);
      fre.push_back(re[q]);
      fim.push_back(im[q]);
    } else {
      fre[hit] += re[q];
      fim[hit] += im[q];
    }
  }
  // reality check: Vg_{-m} = conj(Vg_m) on the grid
  double scale = 0.0;
  for (size_t r = 0; r < fre.size(); ++r) scale = std::fmax(scale, std::hypot(fre[r], fim[r]));
  for (size_t r = 0; r < fre.size(); ++r) {
    int neg[IWF_MAX_N];
    for (int j = 0; j < n; ++j) neg[j] = (g.lens[j] - fm[r * n + j]) % g.lens[j];
    double cre = 0.0, cim = 0.0;
    for (size_t s = 0; s < fre.size(); ++s) {
      bool same = true;
      for (int j = 0; j < n && same; ++j) same = fm[s * n + j] == neg[j];
      if (same) { cre = fre[s]; cim = fim[s]; break; }
    }
    if (std::fabs(cre - fre[r]) > 1e-12 * scale || std::fabs(cim + fim[r]) > 1e-12 * scale)
      return fail(IWF_ERR_ARG, "iwf_set_potential: V is not real (modes must come in +-m "
                               "pairs with conjugate coefficients)");
  }
  // preconditioner summaries and the axis classification
  out.axis.assign(fre.size(), -1);
  for (size_t r = 0; r < fre.size(); ++r) {
    int nz = 0, ax = -1;
    for (int j = 0; j < n; ++j) if (fm[r * n + j] != 0) { ++nz; ax = j; }
    const double a2 = fre[r] * fre[r] + fim[r] * fim[r];
    if (nz == 0) { out.vg0 = fre[r]; out.vconst = fre[r]; continue; }
    out.off_abs += std::sqrt(a2);
    out.off_sq += a2;
    if (nz > 1) { out.separable = false; ax = -2; }
    out.axis[r] = ax;
  }
  return IWF_OK;
}
}  // namespace

iwf_status build_potential(iwf_plan* p, int nmodes, const int* m, const double* re,
                           const double* im) {
  const Geom& g = p->g;
  const int n = g.n;
  Folded F;
  IWF_TRY(fold_modes(g, nmodes, m, re, im, F));
  const std::vector<int>& fm = F.m;
  const std::vector<double>& fre = F.re;
  const std::vector<double>& fim = F.im;
  const std::vector<int>& mode_axis = F.axis;
  const bool separable = F.separable;
  p->vg0 = F.vg0; p->voff_abs = F.off_abs; p->voff_sq = F.off_sq; p->vconst = F.vconst;

  DevBuf<int> d_m, d_axis, d_tax, d_tl;
  DevBuf<double> d_re, d_im;
  const size_t nm = fre.size();
  if (nm) {
    IWF_CUDA(cudaMalloc((void**)&d_m.p, nm * n * sizeof(int)));
    IWF_CUDA(cudaMalloc((void**)&d_axis.p, nm * sizeof(int)));
    IWF_CUDA(cudaMalloc((void**)&d_re.p, nm * sizeof(double)));
    IWF_CUDA(cudaMalloc((void**)&d_im.p, nm * sizeof(double)));
    IWF_CUDA(cudaMemcpy(d_m.p, fm.data(), nm * n * sizeof(int), cudaMemcpyHostToDevice));
    IWF_CUDA(cudaMemcpy(d_axis.p, mode_axis.data(), nm * sizeof(int), cudaMemcpyHostToDevice));
    IWF_CUDA(cudaMemcpy(d_re.p, fre.data(), nm * sizeof(double), cudaMemcpyHostToDevice));
    IWF_CUDA(cudaMemcpy(d_im.p, fim.data(), nm * sizeof(double), cudaMemcpyHostToDevice));
  }
  ModeArgs a{};
  a.g = g; a.nmodes = (int)nm; a.m = d_m.p; a.re = d_re.p; a.im = d_im.p;
  a.scale = 1.0 / (double)g.N;
  const int T = 256;
  IWF_TRY(dev_alloc(&p->d_tab64, 0));
  IWF_TRY(dev_alloc(&p->d_tab32, 0));
  IWF_TRY(dev_alloc(&p->d_grid64, 0));
  IWF_TRY(dev_alloc(&p->d_grid32, 0));
  if (separable) {
    std::vector<int> tax, tl;
    int total = 0;
    for (int j = 0; j < n; ++j) {
      p->tab_off[j] = total;
      for (int l = 0; l < g.lens[j]; ++l) { tax.push_back(j); tl.push_back(l); }
      total += g.lens[j];
    }
    IWF_TRY(dev_alloc(&p->d_tab64, (size_t)total));
    IWF_TRY(dev_alloc(&p->d_tab32, (size_t)total));
    IWF_CUDA(cudaMalloc((void**)&d_tax.p, total * sizeof(int)));
    IWF_CUDA(cudaMalloc((void**)&d_tl.p, total * sizeof(int)));
    IWF_CUDA(cudaMemcpy(d_tax.p, tax.data(), total * sizeof(int), cudaMemcpyHostToDevice));
    IWF_CUDA(cudaMemcpy(d_tl.p, tl.data(), total * sizeof(int), cudaMemcpyHostToDevice));
    axis_table_kernel<<<(total + T - 1) / T, T>>>(a, d_axis.p, total, d_tax.p, d_tl.p,
                                                  p->d_tab64, p->d_tab32, 0);
    IWF_CUDA(cudaGetLastError());
    p->pot_kind = 1;
  } else {
    IWF_TRY(dev_alloc(&p->d_grid64, (size_t)g.N));
    IWF_TRY(dev_alloc(&p->d_grid32, (size_t)g.N));
    grid_kernel<<<(unsigned)((g.N + T - 1) / T), T>>>(a, p->d_grid64, p->d_grid32);
    IWF_CUDA(cudaGetLastError());
    p->pot_kind = 2;
  }
  // the folded modes themselves, for the direct-convolution apply
  cudaFree(p->d_stencil_m);
  cudaFree(p->d_stencil_c);
  p->d_stencil_m = nullptr;
  p->d_stencil_c = nullptr;
  p->stencil_nm = 0;
  if (nm) {
    std::vector<double2> coef(nm);
    for (size_t q = 0; q < nm; ++q) coef[q] = make_double2(fre[q], fim[q]);
    IWF_CUDA(cudaMalloc((void**)&p->d_stencil_m, nm * n * sizeof(int)));
    IWF_CUDA(cudaMalloc((void**)&p->d_stencil_c, nm * sizeof(double2)));
    IWF_CUDA(cudaMemcpy(p->d_stencil_m, fm.data(), nm * n * sizeof(int), cudaMemcpyHostToDevice));
    IWF_CUDA(cudaMemcpy(p->d_stencil_c, coef.data(), nm * sizeof(double2), cudaMemcpyHostToDevice));
  }
  p->stencil_nm = (int)nm;
  IWF_CUDA(cudaDeviceSynchronize());
  return IWF_OK;
}

iwf_status potential_tables(const iwf_plan* p, int nmodes, const int* m, const double* re,
                            const double* im, double* tab64, float* tab32, PotSummary* sum,
                            cudaStream_t s) {
  const Geom& g = p->g;
  const int n = g.n;
  Folded F;
  IWF_TRY(fold_modes(g, nmodes, m, re, im, F));
  if (!F.separable)
    return fail(IWF_ERR_UNSUPPORTED, "batched solves need potentials whose modes each lie on one "
                                     "lifted axis");
  sum->vg0 = F.vg0; sum->off_abs = F.off_abs; sum->off_sq = F.off_sq; sum->separable = true;
  const size_t nm = F.re.size();
  std::vector<int> tax, tl;
  int total = 0;
  for (int j = 0; j < n; ++j) {
    for (int l = 0; l < g.lens[j]; ++l) { tax.push_back(j); tl.push_back(l); }
    total += g.lens[j];
  }
  DevBuf<int> d_m, d_axis, d_tax, d_tl;
  DevBuf<double> d_re, d_im;
  IWF_CUDA(cudaMalloc((void**)&d_m.p, std::max<size_t>(nm, 1) * n * sizeof(int)));
  IWF_CUDA(cudaMalloc((void**)&d_axis.p, std::max<size_t>(nm, 1) * sizeof(int)));
  IWF_CUDA(cudaMalloc((void**)&d_re.p, std::max<size_t>(nm, 1) * sizeof(double)));
  IWF_CUDA(cudaMalloc((void**)&d_im.p, std::max<size_t>(nm, 1) * sizeof(double)));
  IWF_CUDA(cudaMalloc((void**)&d_tax.p, total * sizeof(int)));
  IWF_CUDA(cudaMalloc((void**)&d_tl.p, total * sizeof(int)));
  if (nm) {
    IWF_CUDA(cudaMemcpy(d_m.p, F.m.data(), nm * n * sizeof(int), cudaMemcpyHostToDevice));
    IWF_CUDA(cudaMemcpy(d_axis.p, F.axis.data(), nm * sizeof(int), cudaMemcpyHostToDevice));
    IWF_CUDA(cudaMemcpy(d_re.p, F.re.data(), nm * sizeof(double), cudaMemcpyHostToDevice));
    IWF_CUDA(cudaMemcpy(d_im.p, F.im.data(), nm * sizeof(double), cudaMemcpyHostToDevice));
  }
  IWF_CUDA(cudaMemcpy(d_tax.p, tax.data(), total * sizeof(int), cudaMemcpyHostToDevice));
  IWF_CUDA(cudaMemcpy(d_tl.p, tl.data(), total * sizeof(int), cudaMemcpyHostToDevice));
  ModeArgs a{};
  a.g = g; a.nmodes = (int)nm; a.m = d_m.p; a.re = d_re.p; a.im = d_im.p;
  a.scale = 1.0 / (double)g.N;
  axis_table_kernel<<<(total + 255) / 256, 256, 0, s>>>(a, d_axis.p, total, d_tax.p, d_tl.p,
                                                        tab64, tab32, 1);
  IWF_CUDA(cudaGetLastError());
  IWF_CUDA(cudaStreamSynchronize(s));
  return IWF_OK;
}

// ---------------------------------------------------------------------------------------
// Extent of the concentrated coefficients (the "concentrated area" of Sec. 4.2): for every
// axis the smallest half-width of a window with this plan's centring that holds every point
// with |c_k|^2 >= thr2. In window order a point's k_I offset o_j = k_I,j - lo_j lies in
// [0, 2K_j) and needs half-width max(K_j - o_j, o_j - K_j + 1); its k_II coordinate t_j - L_j
// (digit t_j in [0, 2L_j)) needs max(L_j - t_j, t_j - L_j + 1). Maxima over points by warp
// shuffles and one atomicMax per warp and axis; need[] must start at 0.
namespace {
__global__ void coef_extent_kernel(Geom g, const double2* c, double thr2, int* need) {
  int loc[IWF_MAX_N];
#pragma unroll
  for (int j = 0; j < IWF_MAX_N; ++j) loc[j] = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 v = c[i];
    if (!(fma(v.x, v.x, v.y * v.y) >= thr2)) continue;
    long long rem = i % g.MI;                   // in-slice index: k_I offsets, last axis fastest
    for (int j = g.d - 1; j >= 0; --j) {
      const int o = (int)(rem % g.lens[j]);
      rem /= g.lens[j];
      loc[j] = max(loc[j], max(g.half[j] - o, o - g.half[j] + 1));
    }
    rem = i / g.MI;                             // slice index: k_II digits, last axis fastest
    for (int j = g.n - 1; j >= g.d; --j) {
      const int t = (int)(rem % g.lens[j]);
      rem /= g.lens[j];
      loc[j] = max(loc[j], max(g.half[j] - t, t - g.half[j] + 1));
    }
  }
  for (int j = 0; j < g.n; ++j) {
    int m = loc[j];
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(need + j, m);
  }
}
}  // namespace

iwf_status coef_extent(const iwf_plan* p, const void* coef, double threshold, int* need,
                       cudaStream_t s) {
  if (!p || !coef || !need) return fail(IWF_ERR_ARG, "iwf_coef_extent: NULL argument");
  if (!(threshold >= 0.0) || !std::isfinite(threshold))
    return fail(IWF_ERR_ARG, "iwf_coef_extent: threshold must be finite and >= 0");
  if (reinterpret_cast<uintptr_t>(coef) & 15)
    return fail(IWF_ERR_ARG, "iwf_coef_extent: coefficients must be 16-byte aligned");
  DeviceGuard guard(p->device);
  int* d_need = nullptr;
  IWF_CUDA(cudaMalloc((void**)&d_need, IWF_MAX_N * sizeof(int)));
  iwf_status st = IWF_OK;
  const int blocks = (int)std::max<long long>(1, std::min<long long>((p->g.N + 255) / 256, 8 * 152));
  if (cudaMemsetAsync(d_need, 0, IWF_MAX_N * sizeof(int), s) != cudaSuccess) st = fail(IWF_ERR_CUDA, "iwf_coef_extent");
  if (st == IWF_OK) {
    coef_extent_kernel<<<blocks, 256, 0, s>>>(p->g, reinterpret_cast<const double2*>(coef),
                                              threshold * threshold, d_need);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) st = fail(IWF_ERR_CUDA, "iwf_coef_extent launch");
  }
  if (st == IWF_OK &&
      (cudaMemcpyAsync(need, d_need, p->g.n * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
       cudaStreamSynchronize(s) != cudaSuccess))
    st = fail(IWF_ERR_CUDA, "iwf_coef_extent readback");
  cudaFree(d_need);
  return st;
}

}  // namespace iwf
