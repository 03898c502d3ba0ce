// Direct-convolution apply: H~ psi = Lambda psi + sum_m Vg_m psi(k* - m), the cyclic
// convolution on the K* grid with the potential's folded modes that F V F^{-1} equals
// (Sec. 3.3, Sec. 4.1; App. C for the folding). It is the ablation of the three FFT passes for
// potentials with few modes (every config's V is a sum of cosines: 8 or 12 modes): one read
// of psi and one write of H psi per point, plus the neighbours' reads from L1/L2.
//
// In window order, grid point k* of slice o (k_II window position pos) sits at k_I window
// position w_j = (k*_j - lo_j(o)) mod 2K_j. The neighbour k* - m lies in slice o' with
// pos'_j = (pos_j - m_{II,j}) mod 2L_j, at k_I window position
// (w_j + lo_j(o) - lo_j(o') - m_{I,j}) mod 2K_j: each mode is a cyclic shift of whole slices,
// fixed per (slice, mode) pair.
#include <cstdint>
#include <string>

#include "common.cuh"

namespace iwf {

namespace {

constexpr int kStencilMaxModes = 256;
constexpr int kStencilRows = 8;            // blockDim.y; blockDim.x = fast k_I axis length

template <typename T> struct SVec2;
template <> struct SVec2<double> { using type = double2; };
template <> struct SVec2<float> { using type = float2; };

struct StencilArgs {
  Geom g;
  const int* lo;          // MII x d
  const int* modes;       // nmodes x n, folded
  const double2* coef;    // nmodes
  int nmodes;
  const void* psi;
  void* out;
  const void* lam;
  long long ld;           // N
};

// CTA (slice o = blockIdx.x, vector blockIdx.y). Threads: x along the fastest k_I axis,
// y over the rows formed by the slower k_I axes. D: number of k_I axes when it is 1, 2 or 3
// (the index arithmetic then stays in registers); 0 handles any d.
template <typename T, int D>
__global__ void __launch_bounds__(32 * kStencilRows) stencil_kernel(StencilArgs a) {
  using V2 = typename SVec2<T>::type;
  __shared__ int s_o[kStencilMaxModes];                       // neighbour slice
  __shared__ int s_d[kStencilMaxModes][IWF_MAX_N];            // k_I shift per axis
  __shared__ V2 s_c[kStencilMaxModes];
  const Geom& g = a.g;
  const int d = D > 0 ? D : g.d, nII = g.n - d;
  const long long o = blockIdx.x;
  const int vec = blockIdx.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  for (int q = tid; q < a.nmodes; q += nt) {
    // k_II window position of slice o (C order, last k_II axis fastest), shifted by -m_II
    long long rem = o, op = 0, stride = 1;
    for (int j = nII - 1; j >= 0; --j) {
      const int len = g.lens[d + j];
      const int pos = (int)(rem % len);
      rem /= len;
      int np = pos - a.modes[q * g.n + d + j];
      if (np < 0) np += len;
      op += (long long)np * stride;
      stride *= len;
    }
    s_o[q] = (int)op;
    for (int j = 0; j < d; ++j) {
      const int len = g.lens[j];
      int sh = (a.lo[o * d + j] - a.lo[op * d + j] - a.modes[q * g.n + j]) % len;
      if (sh < 0) sh += len;
      s_d[q][j] = sh;
    }
    const double2 c = a.coef[q];
    V2 cv; cv.x = (T)c.x; cv.y = (T)c.y;
    s_c[q] = cv;
  }
  __syncthreads();
  const int lf = g.lens[d - 1];               // fastest k_I axis
  const int rows = (int)(g.MI / lf);
  const int MI = (int)g.MI;
  const V2* psi = reinterpret_cast<const V2*>(a.psi) + (size_t)vec * a.ld;
  V2* out = reinterpret_cast<V2*>(a.out) + (size_t)vec * a.ld + (size_t)o * MI;
  const T* lam = reinterpret_cast<const T*>(a.lam) + (size_t)o * MI;
  const int x = threadIdx.x;
  if (x >= lf) return;
  const int l0 = g.lens[0], l1 = D == 3 ? g.lens[1] : 1;
  for (int r = threadIdx.y; r < rows; r += blockDim.y) {
    // row r -> coordinates of the slower k_I axes (C order)
    int w0 = 0, w1 = 0;
    int wc[IWF_MAX_N];
    if (D == 2) {
      w0 = r;
    } else if (D == 3) {
      w0 = r / l1; w1 = r - w0 * l1;
    } else if (D == 0) {
      int rr = r;
      for (int j = d - 2; j >= 0; --j) { wc[j] = rr % g.lens[j]; rr /= g.lens[j]; }
    }
    const int w = r * lf + x;
    const V2 p0 = psi[(size_t)o * MI + w];
    const T l = lam[w];
    T accr = l * p0.x, acci = l * p0.y;
    // modes in batches of kBatch: all loads of a batch are issued before its products, so
    // each thread keeps kBatch neighbour reads in flight
    constexpr int kBatch = 8;
    for (int q0 = 0; q0 < a.nmodes; q0 += kBatch) {
      V2 v[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int q = q0 + u;
        if (q < a.nmodes) {
          int xs = x + s_d[q][d - 1];
          if (xs >= lf) xs -= lf;
          int rs = 0;
          if (D == 2) {
            rs = w0 + s_d[q][0];
            if (rs >= l0) rs -= l0;
          } else if (D == 3) {
            int t0 = w0 + s_d[q][0], t1 = w1 + s_d[q][1];
            if (t0 >= l0) t0 -= l0;
            if (t1 >= l1) t1 -= l1;
            rs = t0 * l1 + t1;
          } else if (D == 0) {
            for (int j = 0; j < d - 1; ++j) {
              int t = wc[j] + s_d[q][j];
              if (t >= g.lens[j]) t -= g.lens[j];
              rs = rs * g.lens[j] + t;
            }
          }
          v[u] = psi[(size_t)s_o[q] * MI + rs * lf + xs];
        }
      }
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        if (q0 + u < a.nmodes) {
          const V2 c = s_c[q0 + u];
          accr = fma(c.x, v[u].x, accr); accr = fma(-c.y, v[u].y, accr);
          acci = fma(c.x, v[u].y, acci); acci = fma(c.y, v[u].x, acci);
        }
      }
    }
    V2 res; res.x = accr; res.y = acci;
    out[w] = res;
  }
}

template <typename T>
void launch_stencil(const StencilArgs& a, dim3 grid, dim3 block, cudaStream_t s) {
  switch (a.g.d) {
    case 1: stencil_kernel<T, 1><<<grid, block, 0, s>>>(a); break;
    case 2: stencil_kernel<T, 2><<<grid, block, 0, s>>>(a); break;
    case 3: stencil_kernel<T, 3><<<grid, block, 0, s>>>(a); break;
    default: stencil_kernel<T, 0><<<grid, block, 0, s>>>(a); break;
  }
}

}  // namespace

iwf_status apply_stencil_impl(iwf_plan* p, int precision, const void* psi, void* hpsi, int nvec,
                              cudaStream_t stream) {
  if (nvec < 0) return fail(IWF_ERR_ARG, "iwf_apply_stencil: nvec < 0");
  if (nvec == 0) return IWF_OK;
  if (!psi || !hpsi) return fail(IWF_ERR_ARG, "iwf_apply_stencil: null vector pointer");
  if (precision != IWF_PREC_F64 && precision != IWF_PREC_C64)
    return fail(IWF_ERR_ARG, "iwf_apply_stencil: unknown precision");
  if (p->pot_kind == 0) return fail(IWF_ERR_ARG, "iwf_apply_stencil: no potential set");
  if (nvec > 65535) return fail(IWF_ERR_ARG, "iwf_apply_stencil: nvec > 65535");
  if (p->stencil_nm > kStencilMaxModes)
    return fail(IWF_ERR_UNSUPPORTED, "iwf_apply_stencil: more than " +
                std::to_string(kStencilMaxModes) + " folded modes (use iwf_apply)");
  const size_t bytes = (size_t)p->g.N * nvec * (precision == IWF_PREC_F64 ? 16 : 8);
  const uintptr_t ua = reinterpret_cast<uintptr_t>(psi), ub = reinterpret_cast<uintptr_t>(hpsi);
  if (ua < ub + bytes && ub < ua + bytes) return fail(IWF_ERR_ARG, "iwf_apply_stencil: psi and hpsi overlap");
  const int lf = p->g.lens[p->g.d - 1];
  if (lf > 32) return fail(IWF_ERR_UNSUPPORTED, "iwf_apply_stencil: axis longer than 32");
  StencilArgs a{};
  a.g = p->g; a.lo = p->d_lo; a.modes = p->d_stencil_m; a.coef = p->d_stencil_c;
  a.nmodes = p->stencil_nm; a.psi = psi; a.out = hpsi; a.ld = p->g.N;
  const dim3 block(lf, kStencilRows), grid((unsigned)p->g.MII, (unsigned)nvec);
  if (p->g.MII > 2147483647LL) return fail(IWF_ERR_UNSUPPORTED, "iwf_apply_stencil: too many slices");
  if (precision == IWF_PREC_F64) {
    a.lam = p->d_lam64;
    launch_stencil<double>(a, grid, block, stream);
  } else {
    a.lam = p->d_lam32;
    launch_stencil<float>(a, grid, block, stream);
  }
  IWF_CUDA(cudaGetLastError());
  count_launch();
  return IWF_OK;
}

}  // namespace iwf
