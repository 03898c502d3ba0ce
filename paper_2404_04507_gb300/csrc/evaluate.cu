// Physical-space values of a quasiperiodic function from its window coefficients:
// u(x) = sum_{k in K_{K,L}} c_k exp(i (P k).x) (Sec. 3.1, Eq. int; the paper's accuracy
// metric E_f of Sec. 4.2 compares such values on a uniform grid). With y = P^T x,
// (P k).x = k.y, so the sum runs over the window in window order: per slice (fixed k_II) the
// k_I box [lo, lo + 2K)^d, rows of which run along the fastest k_I axis.
//
// Each row is a polynomial in z = exp(i y_f) (y_f: the fastest k_I axis). It is summed by
// Horner's rule in conj(z), in storage order, which leaves the row sum divided by the phase
// of the row's last coefficient; one complex multiplication by that phase adds the row to
// the point's total (4 FP64 fmas per coefficient). Row phases advance by exp(i y_s) along the
// second-fastest k_I axis and are evaluated exactly with sincos whenever that axis wraps
// (every row when d = 1). FP64 throughout. Direct summation: O(N M).
//
// Grid: x over tiles of kEvalThreads points (one point per thread), y over groups of
// consecutive slices. With one group the kernel writes u; with several each group writes a
// partial sum and reduce_groups adds them in group order, so results do not depend on timing.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace iwf {

namespace {

constexpr int kEvalThreads = 256;
constexpr int kEvalChunk = 2048;            // coefficients staged per step (32 KB)
constexpr size_t kEvalPartMax = size_t(256) << 20;   // cap on the partial-sum scratch

struct EvalArgs {
  Geom g;
  double P[IWF_MAX_N * IWF_MAX_N];          // d x n, row-major
  const int* lo;                            // MII x d
  const double2* coef;                      // N, window order
  const double* x;                          // M x d, row-major
  long long M;
  long long o_per;                          // slices per group
  double2* out;                             // u (one group) or partials, group g at g*M
};

__global__ void __launch_bounds__(kEvalThreads) evaluate_kernel(EvalArgs a) {
  __shared__ double2 s_c[kEvalChunk];
  const Geom& g = a.g;
  const int d = g.d, n = g.n;
  const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = m < a.M;
  double y[IWF_MAX_N];
  for (int j = 0; j < n; ++j) {
    double v = 0.0;
    if (active)
      for (int r = 0; r < d; ++r) v = fma(a.P[r * n + j], a.x[m * d + r], v);
    y[j] = v;
  }
  const int lf = g.lens[d - 1];
  const int ls = d >= 2 ? g.lens[d - 2] : 1;  // rows between exact row phases
  double sf, cf, ss = 0.0, cs = 1.0;
  sincos(y[d - 1], &sf, &cf);
  if (d >= 2) sincos(y[d - 2], &ss, &cs);
  double accr = 0.0, acci = 0.0;
  const long long o0 = (long long)blockIdx.y * a.o_per;
  const long long o1 = min(g.MII, o0 + a.o_per);
  for (long long o = o0; o < o1; ++o) {
    // phase of the slice's first row at its last coefficient: k_II.y_II + lo.y_I +
    // (2K_f - 1) y_f, with k_II,j = pos_j - L_j (C order over the k_II axes, last fastest)
    double th_slice = (double)(lf - 1) * y[d - 1];
    {
      long long rem = o;
      for (int j = n - 1; j >= d; --j) {
        const int len = g.lens[j];
        const int pos = (int)(rem % len);
        rem /= len;
        th_slice = fma((double)(pos - g.half[j]), y[j], th_slice);
      }
      for (int j = 0; j < d; ++j) th_slice = fma((double)a.lo[o * d + j], y[j], th_slice);
    }
    double hr = 0.0, hi = 0.0;              // Horner sum of the current row
    double qr = 0.0, qi = 0.0;              // phase of the current row's last coefficient
    int wf = 0;                             // position along the fastest axis
    int row = 0;                            // row of the slice
    int ws = 0;                             // position along the second-fastest axis
    for (long long c0 = 0; c0 < g.MI; c0 += kEvalChunk) {
      const int cnt = (int)min((long long)kEvalChunk, g.MI - c0);
      __syncthreads();
      for (int e = threadIdx.x; e < cnt; e += blockDim.x) s_c[e] = a.coef[o * g.MI + c0 + e];
      __syncthreads();
      if (!active) continue;
      for (int e = 0; e < cnt; ++e) {
        const double2 c = s_c[e];
        const double nr = fma(hr, cf, fma(hi, sf, c.x));
        hi = fma(hi, cf, fma(-hr, sf, c.y));
        hr = nr;
        if (++wf == lf) {
          if (ws == 0) {
            double th = th_slice;
            int rem = row;
            for (int j = d - 2; j >= 0; --j) {
              const int len = g.lens[j];
              th = fma((double)(rem % len), y[j], th);
              rem /= len;
            }
            sincos(th, &qi, &qr);
          } else {
            const double t = qr * cs - qi * ss;
            qi = fma(qr, ss, qi * cs);
            qr = t;
          }
          accr = fma(hr, qr, accr); accr = fma(-hi, qi, accr);
          acci = fma(hr, qi, acci); acci = fma(hi, qr, acci);
          hr = hi = 0.0;
          wf = 0;
          ++row;
          if (++ws == ls) ws = 0;
        }
      }
    }
  }
  if (active) a.out[(long long)blockIdx.y * a.M + m] = make_double2(accr, acci);
}

__global__ void reduce_groups_kernel(const double2* __restrict__ part, long long M, int groups,
                                     double2* __restrict__ u) {
  const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  double2 s = part[m];
  for (int q = 1; q < groups; ++q) {
    const double2 v = part[(long long)q * M + m];
    s.x += v.x;
    s.y += v.y;
  }
  u[m] = s;
}

// ---- values on a uniform grid in 2D with a diagonal P_I (the observation grids of Sec. 4.2) --
// With P_I = diag(p00, p11), (P k).x = x_0 (p00 k_1 + A_s) + x_1 (p11 k_2 + B_s), where
// A_s = sum_{j>=2} P_0j k_j and B_s = sum_{j>=2} P_1j k_j depend only on the slice s (fixed
// k_II). Within a slice k_I runs over the box [lo_1, lo_1 + 2K_1) x [lo_2, lo_2 + 2K_2), so the
// slice's share of u on the grid x_0(a) = o_0 + a h_0, x_1(b) = o_1 + b h_1 is the product
// E0_s C_s E1_s^T with C_s the slice's 2K_1 x 2K_2 coefficients, E0_s[a][i] =
// exp(i x_0(a) (p00 (lo_1 + i) + A_s)) and E1_s[i][b] = exp(i x_1(b) (p11 (lo_2 + i) + B_s)).
// Per slice and tile of kGA x kGT points: T = C_s E1_s^T (2K_1 x kGT), then u += E0_s T, i.e.
// 2K_1 (1 + 2K_2 / kGA) complex multiply-adds per point instead of the 2K_1 2K_2 of direct
// summation. Phase tables: one exact sincos per row or column and slice, then a recurrence of
// at most 31 complex multiplications. FP64 throughout.
constexpr int kGT = 64;              // output tile: kGA rows x kGT columns
constexpr int kGA = 128;
constexpr int kGThreads = 512;
constexpr int kGMaxLen = 32;         // largest 2K_j of the fast path
constexpr int kGRows = kGThreads / kGT;          // 8 row groups of threads
constexpr int kGAcc = kGA / kGRows;              // 16 accumulators per thread
constexpr size_t kGSmem =
    sizeof(double2) * (size_t)(kGMaxLen * kGMaxLen + 2 * kGMaxLen * kGT + kGA * kGMaxLen);

struct GridArgs {
  Geom g;
  double p00, p11;
  double pa[IWF_MAX_N], pb[IWF_MAX_N];   // P_0j, P_1j of the k_II axes (index j)
  double o0, o1, h0, h1;                 // grid origin and steps
  int G0, G1;                            // points per axis
  int tiles1;                            // tiles along axis 1
  const int* lo;                         // MII x 2
  const double2* coef;
  long long o_per;
  double2* out;                          // u (one group) or partials, group g at g * G0 * G1
};

__device__ __forceinline__ double2 cmul2(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

__global__ void __launch_bounds__(kGThreads, 1) evaluate_grid_kernel(GridArgs a) {
  extern __shared__ __align__(16) unsigned char g_raw[];
  double2* s_c = reinterpret_cast<double2*>(g_raw);          // [i0][i1], len1 stride
  double2* s_e1 = s_c + kGMaxLen * kGMaxLen;                  // [i1][b]
  double2* s_e0 = s_e1 + kGMaxLen * kGT;                      // [a][i0], kGMaxLen stride
  double2* s_t = s_e0 + kGA * kGMaxLen;                       // [i0][b]
  const Geom& g = a.g;
  const int len0 = g.lens[0], len1 = g.lens[1];
  const int MI = len0 * len1;
  const int t = threadIdx.x;
  const int tb = t % kGT, tr = t / kGT;                       // column and row group
  const int ta0 = (blockIdx.x / a.tiles1) * kGA, tb0 = (blockIdx.x % a.tiles1) * kGT;
  // grid coordinates of this thread's table row (t < kGT: column b = t; kGT <= t < kGT + kGA:
  // row a = t - kGT), with the same rounding as origin + index * step on the host
  double xc = 0.0, zr = 1.0, zi = 0.0;                        // coordinate and step phase
  if (t < kGT + kGA) {
    xc = t < kGT ? __dadd_rn(a.o1, __dmul_rn((double)(tb0 + t), a.h1))
                 : __dadd_rn(a.o0, __dmul_rn((double)(ta0 + t - kGT), a.h0));
    sincos(xc * (t < kGT ? a.p11 : a.p00), &zi, &zr);
  }
  double2 acc[kGAcc];
#pragma unroll
  for (int j = 0; j < kGAcc; ++j) acc[j] = make_double2(0.0, 0.0);
  const long long s0 = (long long)blockIdx.y * a.o_per;
  const long long s1 = min(g.MII, s0 + a.o_per);
  for (long long o = s0; o < s1; ++o) {
    __syncthreads();                                          // previous slice's tables read
    for (int e = t; e < MI; e += kGThreads) s_c[e] = a.coef[o * MI + e];
    if (t < kGT + kGA) {
      // slice constants: A_s or B_s from k_II = pos - L (C order, last axis fastest)
      double sab = 0.0;
      long long rem = o;
      for (int j = g.n - 1; j >= 2; --j) {
        const int len = g.lens[j];
        const int kj = (int)(rem % len) - g.half[j];
        rem /= len;
        sab = fma(t < kGT ? a.pb[j] : a.pa[j], (double)kj, sab);
      }
      const bool col = t < kGT;
      const int lo = a.lo[o * 2 + (col ? 1 : 0)];
      const double freq = fma(col ? a.p11 : a.p00, (double)lo, sab);
      double pr, pi;
      sincos(xc * freq, &pi, &pr);
      const int len = col ? len1 : len0;
      for (int i = 0; i < len; ++i) {
        if (col) s_e1[i * kGT + t] = make_double2(pr, pi);
        else s_e0[(t - kGT) * kGMaxLen + i] = make_double2(pr, pi);
        const double nr = fma(pr, zr, -pi * zi);
        pi = fma(pr, zi, pi * zr);
        pr = nr;
      }
    }
    __syncthreads();
    // T = C_s E1_s^T for this thread's column tb
    for (int i0 = tr; i0 < len0; i0 += kGRows) {
      double2 sum = make_double2(0.0, 0.0);
      for (int i1 = 0; i1 < len1; ++i1) {
        const double2 c = s_c[i0 * len1 + i1], e = s_e1[i1 * kGT + tb];
        sum.x = fma(c.x, e.x, sum.x); sum.x = fma(-c.y, e.y, sum.x);
        sum.y = fma(c.x, e.y, sum.y); sum.y = fma(c.y, e.x, sum.y);
      }
      s_t[i0 * kGT + tb] = sum;
    }
    __syncthreads();
    // u += E0_s T for rows tr, tr + kGRows, ...
    for (int i0 = 0; i0 < len0; ++i0) {
      const double2 tv = s_t[i0 * kGT + tb];
#pragma unroll
      for (int j = 0; j < kGAcc; ++j) {
        const double2 e = s_e0[(tr + kGRows * j) * kGMaxLen + i0];
        acc[j].x = fma(e.x, tv.x, acc[j].x); acc[j].x = fma(-e.y, tv.y, acc[j].x);
        acc[j].y = fma(e.x, tv.y, acc[j].y); acc[j].y = fma(e.y, tv.x, acc[j].y);
      }
    }
  }
  const long long M = (long long)a.G0 * a.G1;
  const int b = tb0 + tb;
  if (b < a.G1) {
#pragma unroll
    for (int j = 0; j < kGAcc; ++j) {
      const int ra = ta0 + tr + kGRows * j;
      if (ra < a.G0) a.out[(long long)blockIdx.y * M + (long long)ra * a.G1 + b] = acc[j];
    }
  }
}

// ---- normalised fields, density and E_f (Sec. 4.2) ----
// |u|^2 with each product and the sum rounded separately (no fused multiply-add), so that
// the choice of the maximal point is reproducible by any IEEE implementation.
__device__ __forceinline__ double abs2_rn(double2 v) {
  return __dadd_rn(__dmul_rn(v.x, v.x), __dmul_rn(v.y, v.y));
}

constexpr unsigned long long kNoIndex = ~0ull;

// w[0] <- max over m of the bits of |u_m|^2 (non-negative doubles order like their bits);
// NaNs are skipped by fmax.
__global__ void field_max_kernel(const double2* __restrict__ u, long long M,
                                 unsigned long long* w) {
  double best = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += stride)
    best = fmax(best, abs2_rn(u[m]));
  for (int off = 16; off; off >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, off));
  if ((threadIdx.x & 31) == 0) atomicMax(&w[0], (unsigned long long)__double_as_longlong(best));
}

// w[1] <- the first m with |u_m|^2 equal to the maximum
__global__ void field_argmax_kernel(const double2* __restrict__ u, long long M,
                                    unsigned long long* w) {
  const unsigned long long key = w[0];
  unsigned long long first = kNoIndex;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += stride)
    if ((unsigned long long)__double_as_longlong(abs2_rn(u[m])) == key) {
      first = (unsigned long long)m;        // a thread's points ascend: its first match
      break;
    }
  for (int off = 16; off; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, first, off);
    first = o < first ? o : first;
  }
  if ((threadIdx.x & 31) == 0 && first != kNoIndex) atomicMin(&w[1], first);
}

// one thread: the multiplier conj(s) / |s|^2 with s = u at the chosen point (`at` if it is
// >= 0, else the maximal point; 1 when that value is zero or no point matched), stored at
// w[2..3]; the index to *argmax
__global__ void field_pick_kernel(const double2* __restrict__ u, unsigned long long* w,
                                  long long at, long long* argmax) {
  const unsigned long long i = at >= 0 ? (unsigned long long)at : w[1];
  double2 f = make_double2(1.0, 0.0);
  if (i != kNoIndex) {
    const double2 s = u[i];
    const double a = abs2_rn(s);
    if (a > 0.0) f = make_double2(s.x / a, -s.y / a);
  }
  reinterpret_cast<double2*>(w + 2)[0] = f;
  if (argmax) *argmax = i == kNoIndex ? -1 : (long long)i;
}

__global__ void field_scale_kernel(double2* __restrict__ u, long long M,
                                   const unsigned long long* w, double* __restrict__ rho) {
  const double2 f = reinterpret_cast<const double2*>(w + 2)[0];
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += stride) {
    const double2 v = u[m];
    const double2 r = make_double2(v.x * f.x - v.y * f.y, v.x * f.y + v.y * f.x);
    u[m] = r;
    if (rho) rho[m] = abs2_rn(r);
  }
}

// w[0] <- max over m of the bits of |u_m - v_m|^2
__global__ void field_diff_kernel(const double2* __restrict__ u, const double2* __restrict__ v,
                                  long long M, unsigned long long* w) {
  double best = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += stride) {
    const double2 a = u[m], b = v[m];
    best = fmax(best, abs2_rn(make_double2(a.x - b.x, a.y - b.y)));
  }
  for (int off = 16; off; off >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, off));
  if ((threadIdx.x & 31) == 0) atomicMax(&w[0], (unsigned long long)__double_as_longlong(best));
}

__global__ void field_sqrt_kernel(const unsigned long long* w, double* dist) {
  *dist = sqrt(__longlong_as_double((long long)w[0]));
}

unsigned reduce_blocks(long long M, int device) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    sms = 1;
  const long long b = (M + kEvalThreads - 1) / kEvalThreads;
  return (unsigned)std::max(1LL, std::min(b, 8LL * sms));
}

}  // namespace

iwf_status evaluate_impl(iwf_plan* p, const void* coef, const double* x, long long M, void* u,
                         cudaStream_t stream) {
  if (M < 0) return fail(IWF_ERR_ARG, "iwf_evaluate: M < 0");
  if (M == 0) return IWF_OK;
  if (!coef || !x || !u) return fail(IWF_ERR_ARG, "iwf_evaluate: null pointer");
  const long long tiles = (M + kEvalThreads - 1) / kEvalThreads;
  if (tiles > 2147483647LL) return fail(IWF_ERR_ARG, "iwf_evaluate: too many points");
  const Geom& g = p->g;
  // slice groups: enough CTAs for about eight per SM, at most one group per slice, and a
  // bounded partial-sum scratch
  int sms = 0;
  IWF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
  long long groups = std::max(1LL, (8LL * sms + tiles - 1) / tiles);
  groups = std::min(groups, g.MII);
  groups = std::min(groups, std::max(1LL, (long long)(kEvalPartMax / (16 * (size_t)M))));
  groups = std::min(groups, 65535LL);
  const long long o_per = (g.MII + groups - 1) / groups;
  groups = (g.MII + o_per - 1) / o_per;
  EvalArgs a{};
  a.g = g;
  for (int i = 0; i < g.d * g.n; ++i) a.P[i] = p->P[i];
  a.lo = p->d_lo;
  a.coef = reinterpret_cast<const double2*>(coef);
  a.x = x;
  a.M = M;
  a.o_per = o_per;
  if (groups == 1) {
    a.out = reinterpret_cast<double2*>(u);
  } else {
    const size_t need = (size_t)groups * (size_t)M * sizeof(double2);
    if (need > p->eval_part_bytes) {
      cudaFree(p->d_eval_part);
      p->d_eval_part = nullptr;
      p->eval_part_bytes = 0;
      IWF_CUDA(cudaMalloc(&p->d_eval_part, need));
      p->eval_part_bytes = need;
    }
    a.out = p->d_eval_part;
  }
  evaluate_kernel<<<dim3((unsigned)tiles, (unsigned)groups), kEvalThreads, 0, stream>>>(a);
  IWF_CUDA(cudaGetLastError());
  count_launch();
  if (groups > 1) {
    reduce_groups_kernel<<<(unsigned)tiles, kEvalThreads, 0, stream>>>(
        p->d_eval_part, M, (int)groups, reinterpret_cast<double2*>(u));
    IWF_CUDA(cudaGetLastError());
    count_launch();
  }
  return IWF_OK;
}

}  // namespace iwf

namespace iwf {

iwf_status field_normalize_impl(iwf_plan* p, void* u, long long M, long long at, double* rho,
                                long long* argmax, cudaStream_t stream) {
  if (M < 0) return fail(IWF_ERR_ARG, "iwf_field_normalize: M < 0");
  if (at >= M) return fail(IWF_ERR_ARG, "iwf_field_normalize: at >= M");
  if (M == 0) return IWF_OK;
  if (!u) return fail(IWF_ERR_ARG, "iwf_field_normalize: null field");
  double2* f = reinterpret_cast<double2*>(u);
  unsigned long long* w = p->d_field;
  const unsigned blocks = reduce_blocks(M, p->device);
  if (at < 0) {
    IWF_CUDA(cudaMemsetAsync(w, 0, sizeof(unsigned long long), stream));
    IWF_CUDA(cudaMemsetAsync(w + 1, 0xff, sizeof(unsigned long long), stream));
    field_max_kernel<<<blocks, kEvalThreads, 0, stream>>>(f, M, w);
    field_argmax_kernel<<<blocks, kEvalThreads, 0, stream>>>(f, M, w);
    count_launch();
    count_launch();
  }
  field_pick_kernel<<<1, 1, 0, stream>>>(f, w, at, argmax);
  field_scale_kernel<<<blocks, kEvalThreads, 0, stream>>>(f, M, w, rho);
  IWF_CUDA(cudaGetLastError());
  count_launch();
  count_launch();
  return IWF_OK;
}

iwf_status field_distance_impl(iwf_plan* p, const void* u, const void* v, long long M,
                               double* dist, cudaStream_t stream) {
  if (M < 0) return fail(IWF_ERR_ARG, "iwf_field_distance: M < 0");
  if (!dist || (M > 0 && (!u || !v)))
    return fail(IWF_ERR_ARG, "iwf_field_distance: null pointer");
  unsigned long long* w = p->d_field;
  IWF_CUDA(cudaMemsetAsync(w, 0, sizeof(unsigned long long), stream));
  if (M > 0)
    field_diff_kernel<<<reduce_blocks(M, p->device), kEvalThreads, 0, stream>>>(
        reinterpret_cast<const double2*>(u), reinterpret_cast<const double2*>(v), M, w);
  field_sqrt_kernel<<<1, 1, 0, stream>>>(w, dist);
  IWF_CUDA(cudaGetLastError());
  count_launch();
  if (M > 0) count_launch();
  return IWF_OK;
}

}  // namespace iwf

namespace iwf {

iwf_status evaluate_grid_impl(iwf_plan* p, const void* coef, const double* origin,
                              const double* step, const int* count, void* u,
                              cudaStream_t stream) {
  const Geom& g = p->g;
  if (!origin || !step || !count) return fail(IWF_ERR_ARG, "iwf_evaluate_grid: null argument");
  if (g.d != 2 || g.n < 3)
    return fail(IWF_ERR_UNSUPPORTED, "iwf_evaluate_grid: needs d = 2 (use iwf_evaluate)");
  if (p->P[1] != 0.0 || p->P[g.n] != 0.0)
    return fail(IWF_ERR_UNSUPPORTED, "iwf_evaluate_grid: P_I not diagonal (use iwf_evaluate)");
  if (g.lens[0] > kGMaxLen || g.lens[1] > kGMaxLen)
    return fail(IWF_ERR_UNSUPPORTED, "iwf_evaluate_grid: 2K above 32 (use iwf_evaluate)");
  if (count[0] < 0 || count[1] < 0) return fail(IWF_ERR_ARG, "iwf_evaluate_grid: count < 0");
  for (int r = 0; r < 2; ++r)
    if (!std::isfinite(origin[r]) || !std::isfinite(step[r]))
      return fail(IWF_ERR_NONFINITE, "iwf_evaluate_grid: non-finite origin or step");
  const long long M = (long long)count[0] * count[1];
  if (M == 0) return IWF_OK;
  if (!coef || !u) return fail(IWF_ERR_ARG, "iwf_evaluate_grid: null pointer");
  const long long tiles0 = (count[0] + kGA - 1) / kGA, tiles1 = (count[1] + kGT - 1) / kGT;
  if (tiles0 * tiles1 > 2147483647LL) return fail(IWF_ERR_ARG, "iwf_evaluate_grid: grid too large");
  const long long tiles = tiles0 * tiles1;
  int sms = 0;
  IWF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
  // one CTA per SM: about four waves of slice groups
  long long groups = std::max(1LL, (4LL * sms + tiles - 1) / tiles);
  groups = std::min(groups, g.MII);
  groups = std::min(groups, std::max(1LL, (long long)(kEvalPartMax / (16 * (size_t)M))));
  groups = std::min(groups, 65535LL);
  const long long o_per = (g.MII + groups - 1) / groups;
  groups = (g.MII + o_per - 1) / o_per;
  GridArgs a{};
  a.g = g;
  a.p00 = p->P[0];
  a.p11 = p->P[g.n + 1];
  for (int j = 2; j < g.n; ++j) { a.pa[j] = p->P[j]; a.pb[j] = p->P[g.n + j]; }
  a.o0 = origin[0]; a.o1 = origin[1]; a.h0 = step[0]; a.h1 = step[1];
  a.G0 = count[0]; a.G1 = count[1];
  a.tiles1 = (int)tiles1;
  a.lo = p->d_lo;
  a.coef = reinterpret_cast<const double2*>(coef);
  a.o_per = o_per;
  if (groups == 1) {
    a.out = reinterpret_cast<double2*>(u);
  } else {
    const size_t need = (size_t)groups * (size_t)M * sizeof(double2);
    if (need > p->eval_part_bytes) {
      cudaFree(p->d_eval_part);
      p->d_eval_part = nullptr;
      p->eval_part_bytes = 0;
      IWF_CUDA(cudaMalloc(&p->d_eval_part, need));
      p->eval_part_bytes = need;
    }
    a.out = p->d_eval_part;
  }
  static bool attr[64] = {};
  if (p->device >= 0 && p->device < 64 && !attr[p->device]) {
    IWF_CUDA(cudaFuncSetAttribute(evaluate_grid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kGSmem));
    attr[p->device] = true;
  }
  evaluate_grid_kernel<<<dim3((unsigned)tiles, (unsigned)groups), kGThreads, kGSmem, stream>>>(a);
  IWF_CUDA(cudaGetLastError());
  count_launch();
  if (groups > 1) {
    reduce_groups_kernel<<<(unsigned)((M + kEvalThreads - 1) / kEvalThreads), kEvalThreads, 0,
                           stream>>>(p->d_eval_part, M, (int)groups, reinterpret_cast<double2*>(u));
    IWF_CUDA(cudaGetLastError());
    count_launch();
  }
  return IWF_OK;
}

}  // namespace iwf
