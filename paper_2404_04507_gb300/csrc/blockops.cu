// Block kernels of the eigensolver (declarations and layout conventions in blockops.cuh).
#include <algorithm>
#include <cmath>

#include "blockops.cuh"

namespace iwf {

namespace {

constexpr int kGramRows = 16;      // rows staged per Gram tile
constexpr int kGramTx = 24;        // 24 x 24 threads, 3 x 3 outputs each -> up to 72 x 72
constexpr int kGramThreads = kGramTx * kGramTx;

template <typename T> struct Acc { using type = double; };
template <> struct Acc<float> { using type = float; };

// ---- double-float arithmetic ------------------------------------------------------------
// A double x is carried as an unevaluated sum hi + lo of two floats (hi = x rounded to float,
// lo = the rest rounded to float: 48 significant bits). Products of two such pairs are formed
// with the exact float product error from fma (Dekker); sums keep their rounding error with
// TwoSum (Knuth). FP64 on this GPU runs at 1/62 of the FP32 rate, so a complex multiply-add in
// this form (about 48 FP32 operations) costs about a fifth of its 4 FP64 fmas.
struct DF4 { float rh, rl, ih, il; };              // complex: re (hi, lo), im (hi, lo)

// x = hi + lo with integer and FP32 operations only: conversions between double and float,
// and double arithmetic, issue on the slow FP64 pipe and made the staging of a tile cost as
// much as its products. hi is x truncated to 24 significant bits (built from x's sign,
// exponent and top fraction bits); lo is the remaining 29 fraction bits rounded to a float
// (two exact 23-bit integer-to-float conversions by the 2^23 bias trick and one fma) times
// the exact power of two 2^(e - 52). |x| < 2^-126 gives (0, 0); below 2^-75 lo is 0.
__device__ __forceinline__ void split_bits(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int hw = (unsigned int)(b >> 32), lw = (unsigned int)b;
  const int e = (int)((hw >> 20) & 0x7ffu);          // biased exponent
  const unsigned int sign = hw & 0x80000000u;
  if (e < 1023 - 126) { hi = 0.f; lo = 0.f; return; }
  const unsigned int top23 = ((hw & 0xfffffu) << 3) | (lw >> 29);
  hi = __uint_as_float(sign | ((unsigned int)(e - 1023 + 127) << 23) | top23);
  const unsigned int rest = lw & 0x1fffffffu;
  const float rh = __uint_as_float(0x4B000000u | (rest >> 23)) - 8388608.f;      // exact
  const float rl = __uint_as_float(0x4B000000u | (rest & 0x7fffffu)) - 8388608.f;  // exact
  const float r = fmaf(rh, 8388608.f, rl);
  const int se = e - 1075 + 127;
  const float scale = se > 0 ? __uint_as_float((unsigned int)se << 23) : 0.f;
  lo = r * scale;
  if (sign) lo = -lo;
}
__device__ __forceinline__ DF4 df_split(double2 v) {
  DF4 o;
  split_bits(v.x, o.rh, o.rl);
  split_bits(v.y, o.ih, o.il);
  return o;
}
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// (sh, sl) += (xh + xl)(yh + yl), dropping xl*yl (below 2^-48 relative)
__device__ __forceinline__ void df_mac(float& sh, float& sl, float xh, float xl, float yh, float yl) {
  const float p = xh * yh;
  float t = fmaf(xh, yh, -p);                      // exact: xh*yh = p + t
  t = fmaf(xh, yl, t);
  t = fmaf(xl, yh, t);
  float s, e;
  two_sum(sh, p, s, e);
  sh = s;
  sl += e + t;
}
__device__ __forceinline__ double df_value(float h, float l) { return (double)h + (double)l; }

// G_partial[cta] = sum over this CTA's rows of conj(A_i,a) * B_i,c.
// 24 x 24 threads; each owns a U x V micro-tile (outputs ty + 24u, tx + 24v), so the
// launch picks U = ceil(ma/24), V = ceil(mb/24) and no thread multiplies padding.
// HERM (the product is Hermitian, ma == mb): only the 24 x 24 output blocks u <= v are
// formed; reduce_partials mirrors the others.
template <typename T, int U, int V, bool HERM>
__global__ void __launch_bounds__(kGramThreads)
gram_kernel(Batch bt, BlockList A, BlockList B, int ma, int mb, long long N, double2* partial) {
  static_assert(U > 0 && V > 0 && (!HERM || U == V), "tile");
  using V2 = typename Cplx<T>::type;
  using AT = typename Acc<T>::type;
  const int prob = blockIdx.y;
  if (bt.active && !bt.active[prob]) return;
  const size_t poff = (size_t)prob * bt.pstride;
  for (int i = 0; i < A.nb; ++i) A.p[i] = reinterpret_cast<const V2*>(A.p[i]) + poff;
  for (int i = 0; i < B.nb; ++i) B.p[i] = reinterpret_cast<const V2*>(B.p[i]) + poff;
  __shared__ V2 sa[kGramRows][kMaxSmall + 1];
  __shared__ V2 sb[kGramRows][kMaxSmall + 1];
  const int tx = threadIdx.x % kGramTx, ty = threadIdx.x / kGramTx;
  // running sums across tiles: double for double blocks; for float blocks a float pair
  // (hi, lo) kept with TwoSum, because adding into doubles would put one FP64 addition per
  // output and tile on the slow FP64 pipe
  AT sumr[U][V], sumi[U][V], lor[U][V], loi[U][V];
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int v = 0; v < V; ++v) { sumr[u][v] = 0; sumi[u][v] = 0; lor[u][v] = 0; loi[u][v] = 0; }
  const long long ntiles = (N + kGramRows - 1) / kGramRows;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const long long r0 = t * kGramRows;
    for (int e = threadIdx.x; e < kGramRows * ma; e += blockDim.x) {
      const int k = e / kGramRows, r = e % kGramRows;
      V2 v; v.x = 0; v.y = 0;
      if (r0 + r < N) v = col_ptr<T>(A, k, N)[r0 + r];
      sa[r][k] = v;
    }
    for (int e = threadIdx.x; e < kGramRows * mb; e += blockDim.x) {
      const int k = e / kGramRows, r = e % kGramRows;
      V2 v; v.x = 0; v.y = 0;
      if (r0 + r < N) v = col_ptr<T>(B, k, N)[r0 + r];
      sb[r][k] = v;
    }
    __syncthreads();
    AT accr[U][V], acci[U][V];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int v = 0; v < V; ++v) { accr[u][v] = 0; acci[u][v] = 0; }
    for (int r = 0; r < kGramRows; ++r) {
      V2 av[U], bv[V];
#pragma unroll
      for (int u = 0; u < U; ++u) av[u] = sa[r][min(ty + kGramTx * u, kMaxSmall)];
#pragma unroll
      for (int v = 0; v < V; ++v) bv[v] = sb[r][min(tx + kGramTx * v, kMaxSmall)];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int v = 0; v < V; ++v) {
          if (HERM && u > v) continue;
          // conj(a) * b: re = ax bx + ay by, im = ax by - ay bx
          accr[u][v] = fma((AT)av[u].x, (AT)bv[v].x, accr[u][v]);
          accr[u][v] = fma((AT)av[u].y, (AT)bv[v].y, accr[u][v]);
          acci[u][v] = fma((AT)av[u].x, (AT)bv[v].y, acci[u][v]);
          acci[u][v] = fma(-(AT)av[u].y, (AT)bv[v].x, acci[u][v]);
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int v = 0; v < V; ++v) {
        if (HERM && u > v) continue;
        if constexpr (sizeof(AT) == 4) {
          float t, e;
          two_sum(sumr[u][v], accr[u][v], t, e); sumr[u][v] = t; lor[u][v] += e;
          two_sum(sumi[u][v], acci[u][v], t, e); sumi[u][v] = t; loi[u][v] += e;
        } else {
          sumr[u][v] += accr[u][v]; sumi[u][v] += acci[u][v];
        }
      }
    __syncthreads();
  }
  double2* out = partial + ((size_t)prob * gridDim.x + blockIdx.x) * ma * mb;
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int a = ty + kGramTx * u, c = tx + kGramTx * v;
      if (a < ma && c < mb && !(HERM && u > v))
        out[a * mb + c] = make_double2((double)sumr[u][v] + (double)lor[u][v],
                                       (double)sumi[u][v] + (double)loi[u][v]);
    }
}

// Double-float variant of gram_kernel for complex-double blocks: the staged rows are split into
// float pairs once, every product and sum runs on the FP32 pipes into one double-float
// accumulator per output (TwoSum keeps each addition exact in the high part), and the CTA's
// total is written as double.
template <int U, int V, bool HERM>
__global__ void __launch_bounds__(kGramThreads)
gram_df_kernel(Batch bt, BlockList A, BlockList B, int ma, int mb, long long N, double2* partial) {
  static_assert(!HERM || U == V, "tile");
  const int prob = blockIdx.y;
  if (bt.active && !bt.active[prob]) return;
  const size_t poff = (size_t)prob * bt.pstride;
  for (int i = 0; i < A.nb; ++i) A.p[i] = reinterpret_cast<const double2*>(A.p[i]) + poff;
  for (int i = 0; i < B.nb; ++i) B.p[i] = reinterpret_cast<const double2*>(B.p[i]) + poff;
  __shared__ DF4 sa[kGramRows][kMaxSmall + 1];
  __shared__ DF4 sb[kGramRows][kMaxSmall + 1];
  const int tx = threadIdx.x % kGramTx, ty = threadIdx.x / kGramTx;
  float srh[U][V], srl[U][V], sih[U][V], sil[U][V];
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int v = 0; v < V; ++v) { srh[u][v] = srl[u][v] = sih[u][v] = sil[u][v] = 0.f; }
  const long long ntiles = (N + kGramRows - 1) / kGramRows;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const long long r0 = t * kGramRows;
    for (int e = threadIdx.x; e < kGramRows * ma; e += blockDim.x) {
      const int k = e / kGramRows, r = e % kGramRows;
      double2 v = make_double2(0.0, 0.0);
      if (r0 + r < N) v = col_ptr<double>(A, k, N)[r0 + r];
      sa[r][k] = df_split(v);
    }
    for (int e = threadIdx.x; e < kGramRows * mb; e += blockDim.x) {
      const int k = e / kGramRows, r = e % kGramRows;
      double2 v = make_double2(0.0, 0.0);
      if (r0 + r < N) v = col_ptr<double>(B, k, N)[r0 + r];
      sb[r][k] = df_split(v);
    }
    __syncthreads();
    for (int r = 0; r < kGramRows; ++r) {
      DF4 av[U], bv[V];
#pragma unroll
      for (int u = 0; u < U; ++u) av[u] = sa[r][min(ty + kGramTx * u, kMaxSmall)];
#pragma unroll
      for (int v = 0; v < V; ++v) bv[v] = sb[r][min(tx + kGramTx * v, kMaxSmall)];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int v = 0; v < V; ++v) {
          if (HERM && u > v) continue;
          // conj(a) * b: re = ar br + ai bi, im = ar bi - ai br
          df_mac(srh[u][v], srl[u][v], av[u].rh, av[u].rl, bv[v].rh, bv[v].rl);
          df_mac(srh[u][v], srl[u][v], av[u].ih, av[u].il, bv[v].ih, bv[v].il);
          df_mac(sih[u][v], sil[u][v], av[u].rh, av[u].rl, bv[v].ih, bv[v].il);
          df_mac(sih[u][v], sil[u][v], -av[u].ih, -av[u].il, bv[v].rh, bv[v].rl);
        }
    }
    __syncthreads();
  }
  double2* out = partial + ((size_t)prob * gridDim.x + blockIdx.x) * ma * mb;
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int a = ty + kGramTx * u, c = tx + kGramTx * v;
      if (a < ma && c < mb && !(HERM && u > v))
        out[a * mb + c] = make_double2(df_value(srh[u][v], srl[u][v]), df_value(sih[u][v], sil[u][v]));
    }
}

// Sum the per-CTA partials in a fixed order (deterministic); problem blockIdx.y.
// herm: entries in 24 x 24 blocks below the block diagonal were not formed; they are the
// conjugates of their mirror images (mb = row length).
__global__ void reduce_partials(Batch bt, const double2* partial, int slots, int count,
                                double2* out, bool herm, int mb) {
  const int prob = blockIdx.y;
  if (bt.active && !bt.active[prob]) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  int src = e;
  bool conj = false;
  if (herm) {
    const int a = e / mb, c = e % mb;
    if (a / kGramTx > c / kGramTx) { src = c * mb + a; conj = true; }
  }
  const double2* pp = partial + (size_t)prob * slots * count;
  double re = 0, im = 0;
  for (int s = 0; s < slots; ++s) {
    const double2 v = pp[(size_t)s * count + src];
    re += v.x; im += v.y;
  }
  out[(size_t)prob * kCapG + e] = make_double2(re, conj ? -im : im);
}

constexpr int kUpdRows = 16;
constexpr int kUpdThreads = kUpdRows * kMaxBlock;

// out1[:, j] (=|-=) sum_k S[:, k] C1[k, j]; out2 likewise with C2. C row-major m x q.
template <typename T, bool SUB>
__global__ void __launch_bounds__(kUpdThreads)
update_kernel(Batch bt, BlockList S, int m, long long N, const double2* C1, const double2* C2,
              int cstride, int q, typename Cplx<T>::type* out1, typename Cplx<T>::type* out2) {
  using V2 = typename Cplx<T>::type;
  using AT = typename Acc<T>::type;
  const int prob = blockIdx.y;
  if (bt.active && !bt.active[prob]) return;
  const size_t poff = (size_t)prob * bt.pstride;
  for (int i = 0; i < S.nb; ++i) S.p[i] = reinterpret_cast<const V2*>(S.p[i]) + poff;
  out1 += poff;
  if (out2) out2 += poff;
  C1 += (size_t)prob * cstride;
  if (C2) C2 += (size_t)prob * cstride;
  extern __shared__ __align__(16) unsigned char upd_raw[];
  using C2T = typename Cplx<AT>::type;            // coefficients in the arithmetic type
  C2T* sc1 = reinterpret_cast<C2T*>(upd_raw);
  C2T* sc2 = sc1 + kMaxSmall * kMaxBlock;
  constexpr int rows = kUpdRows;                  // one thread per (row, j)
  __shared__ V2 ss[rows][kMaxSmall + 1];
  for (int e = threadIdx.x; e < m * q; e += blockDim.x) {
    C2T c; c.x = (AT)C1[e].x; c.y = (AT)C1[e].y;
    sc1[e] = c;
    if (C2) { C2T c2; c2.x = (AT)C2[e].x; c2.y = (AT)C2[e].y; sc2[e] = c2; }
  }
  const int r = threadIdx.x / kMaxBlock, j = threadIdx.x % kMaxBlock;  // r < kUpdRows
  const long long ntiles = (N + rows - 1) / rows;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const long long r0 = t * rows;
    __syncthreads();
    for (int e = threadIdx.x; e < rows * m; e += blockDim.x) {
      const int k = e / rows, rr = e % rows;
      V2 v; v.x = 0; v.y = 0;
      if (r0 + rr < N) v = col_ptr<T>(S, k, N)[r0 + rr];
      ss[rr][k] = v;
    }
    __syncthreads();
    if (j < q && r0 + r < N) {
      AT a1r = 0, a1i = 0, a2r = 0, a2i = 0;
      for (int k = 0; k < m; ++k) {
        const V2 sv = ss[r][k];
        const C2T c1 = sc1[k * q + j];
        a1r = fma((AT)sv.x, (AT)c1.x, a1r);
        a1r = fma(-(AT)sv.y, (AT)c1.y, a1r);
        a1i = fma((AT)sv.x, (AT)c1.y, a1i);
        a1i = fma((AT)sv.y, (AT)c1.x, a1i);
        if (C2) {
          const C2T c2 = sc2[k * q + j];
          a2r = fma((AT)sv.x, (AT)c2.x, a2r);
          a2r = fma(-(AT)sv.y, (AT)c2.y, a2r);
          a2i = fma((AT)sv.x, (AT)c2.y, a2i);
          a2i = fma((AT)sv.y, (AT)c2.x, a2i);
        }
      }
      const size_t gi = (size_t)j * N + r0 + r;
      if (SUB) {
        V2 o = out1[gi];
        o.x = (T)((AT)o.x - a1r); o.y = (T)((AT)o.y - a1i);
        out1[gi] = o;
      } else {
        V2 o; o.x = (T)a1r; o.y = (T)a1i;
        out1[gi] = o;
        if (C2) { V2 o2; o2.x = (T)a2r; o2.y = (T)a2i; out2[gi] = o2; }
      }
    }
  }
}

// Double-float variant of update_kernel for complex-double blocks (same layout and
// semantics; see gram_df_kernel for the arithmetic). One output element per thread is a sum of
// at most 72 products, kept in one double-float accumulator.
template <bool SUB>
__global__ void __launch_bounds__(kUpdThreads)
update_df_kernel(Batch bt, BlockList S, int m, long long N, const double2* C1, const double2* C2,
                 int cstride, int q, double2* out1, double2* out2) {
  const int prob = blockIdx.y;
  if (bt.active && !bt.active[prob]) return;
  const size_t poff = (size_t)prob * bt.pstride;
  for (int i = 0; i < S.nb; ++i) S.p[i] = reinterpret_cast<const double2*>(S.p[i]) + poff;
  out1 += poff;
  if (out2) out2 += poff;
  C1 += (size_t)prob * cstride;
  if (C2) C2 += (size_t)prob * cstride;
  extern __shared__ __align__(16) unsigned char upd_raw[];
  DF4* sc1 = reinterpret_cast<DF4*>(upd_raw);
  DF4* sc2 = sc1 + kMaxSmall * kMaxBlock;
  constexpr int rows = kUpdRows;
  __shared__ DF4 ss[rows][kMaxSmall + 1];
  for (int e = threadIdx.x; e < m * q; e += blockDim.x) {
    sc1[e] = df_split(C1[e]);
    if (C2) sc2[e] = df_split(C2[e]);
  }
  const int r = threadIdx.x / kMaxBlock, j = threadIdx.x % kMaxBlock;
  const long long ntiles = (N + rows - 1) / rows;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const long long r0 = t * rows;
    __syncthreads();
    for (int e = threadIdx.x; e < rows * m; e += blockDim.x) {
      const int k = e / rows, rr = e % rows;
      double2 v = make_double2(0.0, 0.0);
      if (r0 + rr < N) v = col_ptr<double>(S, k, N)[r0 + rr];
      ss[rr][k] = df_split(v);
    }
    __syncthreads();
    if (j < q && r0 + r < N) {
      float a1rh = 0, a1rl = 0, a1ih = 0, a1il = 0, a2rh = 0, a2rl = 0, a2ih = 0, a2il = 0;
      for (int k = 0; k < m; ++k) {
        const DF4 sv = ss[r][k];
        const DF4 c1 = sc1[k * q + j];
        // s * c: re = sr cr - si ci, im = sr ci + si cr
        df_mac(a1rh, a1rl, sv.rh, sv.rl, c1.rh, c1.rl);
        df_mac(a1rh, a1rl, -sv.ih, -sv.il, c1.ih, c1.il);
        df_mac(a1ih, a1il, sv.rh, sv.rl, c1.ih, c1.il);
        df_mac(a1ih, a1il, sv.ih, sv.il, c1.rh, c1.rl);
        if (C2) {
          const DF4 c2 = sc2[k * q + j];
          df_mac(a2rh, a2rl, sv.rh, sv.rl, c2.rh, c2.rl);
          df_mac(a2rh, a2rl, -sv.ih, -sv.il, c2.ih, c2.il);
          df_mac(a2ih, a2il, sv.rh, sv.rl, c2.ih, c2.il);
          df_mac(a2ih, a2il, sv.ih, sv.il, c2.rh, c2.rl);
        }
      }
      const size_t gi = (size_t)j * N + r0 + r;
      if (SUB) {
        double2 o = out1[gi];
        o.x -= df_value(a1rh, a1rl);
        o.y -= df_value(a1ih, a1il);
        out1[gi] = o;
      } else {
        out1[gi] = make_double2(df_value(a1rh, a1rl), df_value(a1ih, a1il));
        if (C2) out2[gi] = make_double2(df_value(a2rh, a2rl), df_value(a2ih, a2il));
      }
    }
  }
}

constexpr int kResThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kResThreads)
residual_kernel(Batch bt, const typename Cplx<T>::type* X, const typename Cplx<T>::type* HX,
                const double* theta, const double* lam, const double* shift, const double* off2,
                typename Cplx<T>::type* W, long long N, int b, double* partial) {
  using V2 = typename Cplx<T>::type;
  using AT = typename Acc<T>::type;
  const int prob = blockIdx.y;
  if (bt.active && !bt.active[prob]) return;
  const size_t poff = (size_t)prob * bt.pstride;
  X += poff; HX += poff; W += poff;
  theta += (size_t)prob * kMaxBlock;
  const double sh = shift[prob], o2 = off2[prob];
  __shared__ double red[kResThreads / 32][kMaxBlock];  // b <= kMaxBlock
  AT acc[kMaxBlock];
#pragma unroll
  for (int j = 0; j < kMaxBlock; ++j) acc[j] = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const double h = lam[i] + sh;
    const T mi = (T)(h / (h * h + o2));
#pragma unroll
    for (int j = 0; j < kMaxBlock; ++j) {
      if (j >= b) break;
      const size_t gi = (size_t)j * N + i;
      const V2 x = X[gi], h = HX[gi];
      const T th = (T)theta[j];
      V2 r; r.x = h.x - th * x.x; r.y = h.y - th * x.y;
      acc[j] += (AT)r.x * (AT)r.x + (AT)r.y * (AT)r.y;
      V2 w; w.x = mi * r.x; w.y = mi * r.y;
      W[gi] = w;
    }
  }
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
#pragma unroll
  for (int j = 0; j < kMaxBlock; ++j) {
    if (j >= b) break;
    double v = (double)acc[j];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][j] = v;
  }
  __syncthreads();
  if (threadIdx.x < b) {
    double v = 0;
    for (int w = 0; w < kResThreads / 32; ++w) v += red[w][threadIdx.x];
    partial[((size_t)prob * gridDim.x + blockIdx.x) * b + threadIdx.x] = v;
  }
}

__global__ void resid_finish(Batch bt, const double* partial, int slots, int b, double* resid) {
  const int prob = blockIdx.x;
  if (bt.active && !bt.active[prob]) return;
  const int j = threadIdx.x;
  if (j >= b) return;
  double s = 0;
  for (int c = 0; c < slots; ++c) s += partial[((size_t)prob * slots + c) * b + j];
  resid[(size_t)prob * kMaxBlock + j] = sqrt(s);
}

// ---------------------------------------------------------------------------------------
// One-CTA dense Hermitian eigensolver: parallel cyclic Jacobi (round-robin pairing), FP64.
// A (n x n, row-major, leading dimension ld) is overwritten; V receives the eigenvectors.
constexpr int kSmallThreads = 512;

struct SmallShared {
  double2 A[kMaxSmall * kMaxSmall];
  double2 V[kMaxSmall * kMaxSmall];
  double2 B[kMaxSmall * kMaxBlock];   // m x b scratch (the P coefficients)
  double w[kMaxSmall];
  double w2[kMaxSmall];
  double d[kMaxSmall];
  float4 rot_cs[kMaxSmall / 2 + 1];   // Jacobi: c and s as float pairs (c.h, c.l, s.h, s.l)
  float4 rot_ph[kMaxSmall / 2 + 1];   // Jacobi: e^{-i phi} as float pairs (re.h, re.l, im.h, im.l)
  int rp[kMaxSmall / 2 + 1], rq[kMaxSmall / 2 + 1];
  int idx[kMaxSmall];
  int perm[kMaxSmall];
  double red[kSmallThreads / 32];
  int flag;
  int rot;
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = v;
  __syncthreads();
  double s = 0;
  for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += red[w];
  __syncthreads();
  return s;
}

// ---- double-float scalars for the Jacobi rotations ---------------------------------------
struct DF { float h, l; };
__device__ __forceinline__ DF df_of(double x) {
  DF o;
  o.h = __double2float_rn(x);
  o.l = __double2float_rn(x - (double)o.h);
  return o;
}
__device__ __forceinline__ double df_dbl(DF a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ DF df_norm(float s, float e) {   // fast two-sum, |s| >= |e|
  DF o;
  o.h = s + e;
  o.l = e - (o.h - s);
  return o;
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return df_norm(p, e);
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e += a.l + b.l;
  return df_norm(s, e);
}
__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.h, -a.l}; }
// complex double-float, stored in the 16 bytes of a double2
struct CDF { DF re, im; };
__device__ __forceinline__ CDF cdf_mul(CDF a, CDF b) {
  return CDF{df_add(df_mul(a.re, b.re), df_neg(df_mul(a.im, b.im))),
             df_add(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
// c a - s t and s a + c t for real c, s
__device__ __forceinline__ void cdf_rot(CDF a, CDF t, DF c, DF s, CDF& a2, CDF& t2) {
  a2 = CDF{df_add(df_mul(c, a.re), df_neg(df_mul(s, t.re))),
           df_add(df_mul(c, a.im), df_neg(df_mul(s, t.im)))};
  t2 = CDF{df_add(df_mul(s, a.re), df_mul(c, t.re)), df_add(df_mul(s, a.im), df_mul(c, t.im))};
}
__device__ __forceinline__ CDF& cdf_at(double2* base, int e) {
  return *reinterpret_cast<CDF*>(base + e);
}
__device__ __forceinline__ CDF cdf_of(double2 v) { return CDF{df_of(v.x), df_of(v.y)}; }
__device__ __forceinline__ double2 dbl_of(CDF v) { return make_double2(df_dbl(v.re), df_dbl(v.im)); }

// Eigen-decomposition of the Hermitian n x n matrix in sh.A (row-major, ld = n).
// On return sh.w holds ascending eigenvalues and sh.V (row-major) the eigenvectors as columns.
// The rotations run in double-float arithmetic on the FP32 pipes (A and V are held as float
// pairs in place of their double2 entries while the sweeps run): this one-CTA solve sits on
// the critical path of every iteration, and FP64 on this GPU issues at 1/62 of the FP32 rate.
// Rotation angles are computed in FP64 from the double-float entries.
__device__ void jacobi_eig(SmallShared& sh, int n) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < n * n; e += nt) {
    const int i = e / n, j = e % n;
    sh.V[e] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    // symmetrise: A = (A + A^H)/2
    if (i < j) {
      const double2 a = sh.A[i * n + j], c = sh.A[j * n + i];
      const double2 m = make_double2(0.5 * (a.x + c.x), 0.5 * (a.y - c.y));
      sh.A[i * n + j] = m;
      sh.A[j * n + i] = cconj(m);
    } else if (i == j) {
      sh.A[e].y = 0.0;
    }
  }
  __syncthreads();
  if (n == 1) {
    if (tid == 0) sh.w[0] = sh.A[0].x;
    __syncthreads();
    return;
  }
  for (int e = tid; e < n * n; e += nt) {
    cdf_at(sh.A, e) = cdf_of(sh.A[e]);
    cdf_at(sh.V, e) = cdf_of(sh.V[e]);
  }
  __syncthreads();
  const int ne = n + (n & 1);       // players, with one dummy when n is odd
  const int np = ne / 2;
  for (int sweep = 0; sweep < 40; ++sweep) {
    // convergence: off-diagonal Frobenius norm relative to the whole matrix, at the level
    // double-float entries resolve (about 2^-46 each)
    // (in double: the entries of a Gram of tiny columns would underflow when squared in float)
    double off = 0, tot = 0;
    for (int e = tid; e < n * n; e += nt) {
      const CDF a = cdf_at(sh.A, e);
      const double v = (double)a.re.h * a.re.h + (double)a.im.h * a.im.h;
      tot += v;
      if (e / n != e % n) off += v;
    }
    off = block_sum(off, sh.red);
    tot = block_sum(tot, sh.red);
    if (off <= 1e-25 * tot || off == 0.0) break;
    if (tid == 0) sh.rot = 0;
    __syncthreads();
    for (int round = 0; round < ne - 1; ++round) {
      if (tid < np) {
        const int k = tid;
        const int posa = k, posb = ne - 1 - k;
        const int p = posa == 0 ? 0 : ((posa - 1 + round) % (ne - 1)) + 1;
        const int q = ((posb - 1 + round) % (ne - 1)) + 1;
        // rotation annihilating a_pq, stored as float pairs for the row and column updates.
        // The angle t = tan(theta) only needs to be close (a rotation by a slightly wrong
        // angle leaves a tiny a_pq for the next sweep), so it is taken in FP32; c, s and the
        // unit phase e^{-i phi} must be orthonormal to working precision and are formed in
        // FP64 from that t (double-float arithmetic would leave c^2 + s^2 - 1 near 1.5e-14,
        // four times the FP64 rounding, which stalled the 32^4 solves). This keeps the chain
        // of dependent FP64 operations per round short: it is the latency of every round.
        double c = 1.0, s = 0.0;
        double2 eph = make_double2(1.0, 0.0);   // e^{-i phi}
        int pp = p < q ? p : q, qq = p < q ? q : p;
        if (qq < n) {
          const double2 apq = dbl_of(cdf_at(sh.A, pp * n + qq));
          const double r2 = fma(apq.x, apq.x, apq.y * apq.y);
          const DF ad = cdf_at(sh.A, pp * n + pp).re, bd = cdf_at(sh.A, qq * n + qq).re;
          const double a = df_dbl(ad), bq = df_dbl(bd);
          if (r2 > 1e-300 && r2 > 1.6e-27 * fabs(a * bq)) {
            sh.rot = 1;
            const double inv_r = rsqrt(r2);
            eph = make_double2(apq.x * inv_r, -apq.y * inv_r);
            // tau = (a_qq - a_pp) / (2 |a_pq|) and t in FP32
            const float tau = (float)((bq - a) * 0.5) * (float)inv_r;
            const float at = fabsf(tau);
            float tf = at > 1e15f ? 0.5f / at : 1.f / (at + sqrtf(fmaf(at, at, 1.f)));
            if (tau < 0.f) tf = -tf;
            const double t = (double)tf;
            c = rsqrt(fma(t, t, 1.0));
            s = t * c;
          }
        } else {
          pp = -1;
        }
        sh.rp[k] = pp; sh.rq[k] = qq;
        const DF cf = df_of(c), sf = df_of(s);
        const CDF pf = cdf_of(eph);
        sh.rot_cs[k] = make_float4(cf.h, cf.l, sf.h, sf.l);
        sh.rot_ph[k] = make_float4(pf.re.h, pf.re.l, pf.im.h, pf.im.l);
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int e = tid; e < n * np; e += nt) {
        const int i = e / np, k = e % np;
        const int p = sh.rp[k];
        if (p < 0 || sh.rot_cs[k].z == 0.f) continue;
        const int q = sh.rq[k];
        const float4 cs = sh.rot_cs[k], ph = sh.rot_ph[k];
        const DF c{cs.x, cs.y}, s{cs.z, cs.w};
        const CDF eph{DF{ph.x, ph.y}, DF{ph.z, ph.w}};
        {
          CDF& aip = cdf_at(sh.A, i * n + p);
          CDF& aiq = cdf_at(sh.A, i * n + q);
          const CDF t = cdf_mul(aiq, eph);
          CDF a2, t2;
          cdf_rot(aip, t, c, s, a2, t2);
          aip = a2; aiq = t2;
        }
        {
          CDF& vip = cdf_at(sh.V, i * n + p);
          CDF& viq = cdf_at(sh.V, i * n + q);
          const CDF t = cdf_mul(viq, eph);
          CDF a2, t2;
          cdf_rot(vip, t, c, s, a2, t2);
          vip = a2; viq = t2;
        }
      }
      __syncthreads();
      // rows: A <- J^H A. Consecutive threads walk along a row (j fastest): rows start n
      // entries of 16 B apart, so threads of one column in different rows would share banks.
      for (int e = tid; e < n * np; e += nt) {
        const int k = e / n, j = e % n;
        const int p = sh.rp[k];
        if (p < 0 || sh.rot_cs[k].z == 0.f) continue;
        const int q = sh.rq[k];
        const float4 cs = sh.rot_cs[k], ph = sh.rot_ph[k];
        const DF c{cs.x, cs.y}, s{cs.z, cs.w};
        const CDF ephc{DF{ph.x, ph.y}, DF{-ph.z, -ph.w}};   // e^{+i phi}
        CDF& apj = cdf_at(sh.A, p * n + j);
        CDF& aqj = cdf_at(sh.A, q * n + j);
        const CDF t = cdf_mul(aqj, ephc);
        CDF a2, t2;
        cdf_rot(apj, t, c, s, a2, t2);
        apj = a2; aqj = t2;
      }
      __syncthreads();
    }
    if (sh.rot == 0) break;
    __syncthreads();
  }
  // back to double: eigenvalues on the diagonal, eigenvectors in V
  for (int e = tid; e < n * n; e += nt) {
    sh.A[e] = dbl_of(cdf_at(sh.A, e));
    sh.V[e] = dbl_of(cdf_at(sh.V, e));
  }
  __syncthreads();
  // sort ascending: rank of every eigenvalue (ties by index)
  for (int i = tid; i < n; i += nt) sh.w2[i] = sh.A[i * n + i].x;
  __syncthreads();
  for (int i = tid; i < n; i += nt) {
    int rank = 0;
    const double wi = sh.w2[i];
    for (int j = 0; j < n; ++j) {
      const double wj = sh.w2[j];
      rank += (wj < wi) || (wj == wi && j < i);
    }
    sh.perm[rank] = i;
  }
  __syncthreads();
  // A (no longer needed) <- V[:, perm], then V <- A
  for (int e = tid; e < n * n; e += nt) {
    const int i = e / n, r = e % n;
    sh.A[e] = sh.V[i * n + sh.perm[r]];
  }
  for (int r = tid; r < n; r += nt) sh.w[r] = sh.w2[sh.perm[r]];
  __syncthreads();
  for (int e = tid; e < n * n; e += nt) sh.V[e] = sh.A[e];
  __syncthreads();
}

// Orthonormalising transform of a block from its Gram matrix (SVQB):
// D = diag(G)^{-1/2}, D G D = U S U^H, T = D U S^{-1/2} restricted to S > drop * max(S).
// Columns of T beyond the kept rank are zero and their mask entry is 0.
__global__ void __launch_bounds__(kSmallThreads)
svqb_kernel(Batch bt, const double2* G, int b, double drop, double2* T, int* mask, int* status) {
  extern __shared__ __align__(16) unsigned char raw[];
  SmallShared& sh = *reinterpret_cast<SmallShared*>(raw);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int prob = blockIdx.x;
  if (bt.active && !bt.active[prob]) return;
  G += (size_t)prob * kCapG;
  T += (size_t)prob * kCapT;
  mask += (size_t)prob * kMaxBlock;
  if (status) status += prob;
  for (int i = tid; i < b; i += nt) {
    const double g = G[i * b + i].x;
    sh.w[i] = g > 1e-300 ? 1.0 / sqrt(g) : 0.0;
  }
  __syncthreads();
  for (int e = tid; e < b * b; e += nt) {
    const int i = e / b, j = e % b;
    const double2 g = G[e];
    sh.A[e] = make_double2(g.x * sh.w[i] * sh.w[j], g.y * sh.w[i] * sh.w[j]);
  }
  // keep D while the eigensolver reuses w
  for (int i = tid; i < b; i += nt) sh.d[i] = sh.w[i];
  __syncthreads();
  jacobi_eig(sh, b);
  const double smax = sh.w[b - 1];
  for (int e = tid; e < b * b; e += nt) {
    const int i = e / b, k = e % b;   // T[i][k]; eigenvalues ascending, keep the largest
    const int col = b - 1 - k;        // output column k <- eigenpair b-1-k (descending)
    const double sk = sh.w[col];
    const double di = sh.d[i];
    double2 t = make_double2(0, 0);
    if (smax > 0 && sk > drop * smax) {
      const double f = di / sqrt(sk);
      const double2 u = sh.V[i * b + col];
      t = make_double2(u.x * f, u.y * f);
    }
    T[e] = t;
  }
  for (int k = tid; k < b; k += nt) {
    const double sk = sh.w[b - 1 - k];
    mask[k] = (smax > 0 && sk > drop * smax) ? 1 : 0;
  }
  if (tid == 0 && status) *status = 0;
}

// Rayleigh-Ritz on the orthonormal basis S (m columns, `mask` marks the active ones):
// eigenpairs of the compacted Hermitian A; theta and Cx (m x b) take the lowest b.
// Cp: Cx with its first x_rows rows zeroed (the W and P parts), orthogonalised against Cx
// and orthonormalised in the coefficient space, so that S Cp is orthonormal and orthogonal
// to S Cx; dependent columns are zero with mask_p = 0.
__global__ void __launch_bounds__(kSmallThreads)
rr_kernel(Batch bt, const double2* Ain, int m, int b, const int* mask, int x_rows,
          double* theta, double2* Cx, double2* Cp, int* mask_p, int* status) {
  extern __shared__ __align__(16) unsigned char raw[];
  SmallShared& sh = *reinterpret_cast<SmallShared*>(raw);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int prob = blockIdx.x;
  if (bt.active && !bt.active[prob]) return;
  Ain += (size_t)prob * kCapG;
  mask += (size_t)prob * kMaxSmall;
  theta += (size_t)prob * kMaxBlock;
  Cx += (size_t)prob * kCapC;
  Cp += (size_t)prob * kCapC;
  mask_p += (size_t)prob * kMaxBlock;
  status += prob;
  if (tid == 0) {
    int na = 0;
    for (int i = 0; i < m; ++i) if (mask[i]) sh.idx[na++] = i;
    sh.flag = na;
  }
  __syncthreads();
  const int na = sh.flag;
  if (na < b) {
    if (tid == 0) *status = 1;
    return;
  }
  for (int e = tid; e < na * na; e += nt) {
    const int i = e / na, j = e % na;
    sh.A[e] = Ain[sh.idx[i] * m + sh.idx[j]];
  }
  __syncthreads();
  jacobi_eig(sh, na);
  // Cx (m x b): rows of inactive columns are zero
  for (int e = tid; e < m * b; e += nt) Cx[e] = make_double2(0, 0);
  __syncthreads();
  for (int e = tid; e < na * b; e += nt) {
    const int i = e / b, k = e % b;
    Cx[sh.idx[i] * b + k] = sh.V[i * na + k];
  }
  for (int k = tid; k < b; k += nt) theta[k] = sh.w[k];
  __syncthreads();
  __threadfence_block();
  // Cp: two rounds of (orthogonalise against Cx twice, then orthonormalise). The second
  // round acts on unit columns, so the rounding left by normalising tiny first-round
  // columns (norm down to 1e-12) cannot survive as a loss of orthogonality to Cx.
  for (int rep = 0; rep < 2; ++rep) {
    for (int e = tid; e < m * b; e += nt) {
      const double2 c = Cx[e];
      sh.A[e] = c;
      sh.B[e] = rep ? Cp[e] : ((e / b) < x_rows ? make_double2(0, 0) : c);
    }
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
      for (int e = tid; e < b * b; e += nt) {
        const int r = e / b, c = e % b;
        double2 s = make_double2(0, 0);
        for (int i = 0; i < m; ++i) {
          const double2 t = cmul(cconj(sh.A[i * b + r]), sh.B[i * b + c]);
          s.x += t.x; s.y += t.y;
        }
        sh.V[e] = s;
      }
      __syncthreads();
      for (int e = tid; e < m * b; e += nt) {
        const int i = e / b, c = e % b;
        double2 s = make_double2(0, 0);
        for (int r = 0; r < b; ++r) {
          const double2 t = cmul(sh.A[i * b + r], sh.V[r * b + c]);
          s.x += t.x; s.y += t.y;
        }
        sh.V[b * b + e] = make_double2(sh.B[e].x - s.x, sh.B[e].y - s.y);
      }
      __syncthreads();
      for (int e = tid; e < m * b; e += nt) sh.B[e] = sh.V[b * b + e];
      __syncthreads();
    }
    // Gram of Cp, then its SVQB transform in the coefficient space
    for (int e = tid; e < b * b; e += nt) {
      const int r = e / b, c = e % b;
      double2 s = make_double2(0, 0);
      for (int i = 0; i < m; ++i) {
        const double2 t = cmul(cconj(sh.B[i * b + r]), sh.B[i * b + c]);
        s.x += t.x; s.y += t.y;
      }
      sh.V[b * b + m * b + e] = s;
    }
    __syncthreads();
    for (int e = tid; e < m * b; e += nt) Cp[e] = sh.B[e];
    for (int e = tid; e < b * b; e += nt) sh.A[e] = sh.V[b * b + m * b + e];
    __syncthreads();
    jacobi_eig(sh, b);
    // keep columns of norm > 1e-12 in the first round, near-unit columns in the second
    const double keep = rep ? 1e-2 : 1e-24;
    for (int e = tid; e < b * b; e += nt) {
      const int i = e / b, k = e % b;
      const int col = b - 1 - k;
      const double sk = sh.w[col];
      double2 t = make_double2(0, 0);
      if (sk > keep) {
        const double f = 1.0 / sqrt(sk);
        const double2 u = sh.V[i * b + col];
        t = make_double2(u.x * f, u.y * f);
      }
      sh.A[e] = t;
    }
    for (int k = tid; k < b; k += nt) mask_p[k] = sh.w[b - 1 - k] > keep ? 1 : 0;
    __syncthreads();
    for (int e = tid; e < m * b; e += nt) sh.B[e] = Cp[e];
    __syncthreads();
    for (int e = tid; e < m * b; e += nt) {
      const int i = e / b, c = e % b;
      double2 s = make_double2(0, 0);
      for (int r = 0; r < b; ++r) {
        const double2 t = cmul(sh.B[i * b + r], sh.A[r * b + c]);
        s.x += t.x; s.y += t.y;
      }
      Cp[e] = s;
    }
    __syncthreads();
  }
  if (tid == 0) *status = 0;
}

template <typename Tin, typename Tout>
__global__ void convert_kernel(const Tin* in, Tout* out, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (Tout)in[i];
}

// splitmix64 (Steele, Lea, Flood 2014) as a counter-based generator of start vectors.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename T>
__global__ void random_kernel(typename Cplx<T>::type* X, long long count, unsigned long long seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long a = splitmix64(seed ^ (2ull * (unsigned long long)i));
    const unsigned long long c = splitmix64(seed ^ (2ull * (unsigned long long)i + 1ull));
    typename Cplx<T>::type v;
    v.x = (T)((double)(a >> 11) * (1.0 / 9007199254740992.0) - 0.5);
    v.y = (T)((double)(c >> 11) * (1.0 / 9007199254740992.0) - 0.5);
    X[i] = v;
  }
}

// flag = 1 when any of the count doubles is NaN or infinite
__global__ void nonfinite_kernel(const double* x, long long count, int* flag) {
  int bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    bad |= !isfinite(x[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

__global__ void mask_kernel(int nprob, int* mask, int off, int b, int value, const int* src) {
  const int prob = blockIdx.x;
  const int j = threadIdx.x;
  if (prob >= nprob || j >= b) return;
  mask[(size_t)prob * kMaxSmall + off + j] = src ? src[(size_t)prob * kMaxBlock + j] : value;
}

int grid_for(long long work, int per_block) {
  long long g = (work + per_block - 1) / per_block;
  if (g > 4 * 152) g = 4 * 152;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

template <typename T>
iwf_status gram(const Batch& bt, const BlockList& A, const BlockList& B, long long N, double2* out,
                double2* partial, int slots_per_prob, cudaStream_t s, bool herm) {
  const int ma = A.nb * A.b, mb = B.nb * B.b;
  if (ma > kMaxSmall || mb > kMaxSmall) return fail(IWF_ERR_ARG, "gram: too many columns");
  if (herm && ma != mb) return fail(IWF_ERR_ARG, "gram: a Hermitian product must be square");
  if (sizeof(T) == 8 && bt.engine == kEngineTensor)
    return gram_tc(bt, A, B, N, out, reinterpret_cast<double*>(partial), slots_per_prob, bt.err, s,
                   herm);
  int g = grid_for(N, kGramRows);
  if (g > slots_per_prob) g = slots_per_prob;
  const int U = (ma + kGramTx - 1) / kGramTx, V = (mb + kGramTx - 1) / kGramTx;
  const dim3 grid(g, bt.nprob);
  const bool df = sizeof(T) == 8 && bt.engine == kEngineDF;
  switch (U * 4 + V + (herm ? 100 : 0)) {
#define IWF_GRAM(U_, V_, H_) \
    case U_ * 4 + V_ + (H_ ? 100 : 0): \
      if (df) gram_df_kernel<U_, V_, H_><<<grid, kGramThreads, 0, s>>>(bt, A, B, ma, mb, N, partial); \
      else gram_kernel<T, U_, V_, H_><<<grid, kGramThreads, 0, s>>>(bt, A, B, ma, mb, N, partial); \
      break;
    IWF_GRAM(1, 1, false) IWF_GRAM(1, 2, false) IWF_GRAM(1, 3, false) IWF_GRAM(2, 1, false)
    IWF_GRAM(2, 2, false) IWF_GRAM(2, 3, false) IWF_GRAM(3, 1, false) IWF_GRAM(3, 2, false)
    IWF_GRAM(3, 3, false) IWF_GRAM(1, 1, true) IWF_GRAM(2, 2, true) IWF_GRAM(3, 3, true)
#undef IWF_GRAM
    default: return fail(IWF_ERR_ARG, "gram: shape");
  }
  IWF_CUDA(cudaGetLastError());
  count_launch();
  const int cnt = ma * mb;
  reduce_partials<<<dim3((cnt + 255) / 256, bt.nprob), 256, 0, s>>>(bt, partial, g, cnt, out,
                                                                      herm, mb);
  IWF_CUDA(cudaGetLastError());
  count_launch();
  return IWF_OK;
}

template <typename T>
iwf_status block_update(const Batch& bt, const BlockList& S, long long N, const double2* C1,
                        const double2* C2, int cstride, int q, void* out1, void* out2,
                        bool subtract, cudaStream_t s) {
  // (the static attribute flags below are per instantiation of T)
  using V2 = typename Cplx<T>::type;
  const int m = S.nb * S.b;
  if (m > kMaxSmall || q > kMaxBlock || q < 1) return fail(IWF_ERR_ARG, "block_update: shape");
  if (cstride < m * q) return fail(IWF_ERR_ARG, "block_update: coefficient stride too small");
  if (sizeof(T) == 8 && bt.engine == kEngineTensor)
    return update_tc(bt, S, N, C1, C2, cstride, q, reinterpret_cast<double2*>(out1),
                     reinterpret_cast<double2*>(out2), subtract, bt.err, s);
  int g0 = grid_for(N, kUpdRows);
  if (bt.nprob > 1) g0 = std::max(1, std::min(g0, (8 * 152 + bt.nprob - 1) / bt.nprob));
  const dim3 g(g0, bt.nprob);
  const size_t dyn = 2 * sizeof(double2) * kMaxSmall * kMaxBlock;
  static bool attr[2] = {false, false};
  if (!attr[subtract]) {
    if (subtract)
      IWF_CUDA(cudaFuncSetAttribute(update_kernel<T, true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    else
      IWF_CUDA(cudaFuncSetAttribute(update_kernel<T, false>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    attr[subtract] = true;
  }
  if (sizeof(T) == 8 && bt.engine == kEngineDF) {
    static bool attr_df[2] = {false, false};
    if (!attr_df[subtract]) {
      if (subtract)
        IWF_CUDA(cudaFuncSetAttribute(update_df_kernel<true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
      else
        IWF_CUDA(cudaFuncSetAttribute(update_df_kernel<false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
      attr_df[subtract] = true;
    }
    if (subtract)
      update_df_kernel<true><<<g, kUpdThreads, dyn, s>>>(bt, S, m, N, C1, nullptr, cstride, q,
                                                         reinterpret_cast<double2*>(out1), nullptr);
    else
      update_df_kernel<false><<<g, kUpdThreads, dyn, s>>>(bt, S, m, N, C1, C2, cstride, q,
                                                          reinterpret_cast<double2*>(out1),
                                                          reinterpret_cast<double2*>(out2));
    IWF_CUDA(cudaGetLastError());
    count_launch();
    return IWF_OK;
  }
  if (subtract)
    update_kernel<T, true><<<g, kUpdThreads, dyn, s>>>(bt, S, m, N, C1, nullptr, cstride, q,
                                                       reinterpret_cast<V2*>(out1), nullptr);
  else
    update_kernel<T, false><<<g, kUpdThreads, dyn, s>>>(bt, S, m, N, C1, C2, cstride, q,
                                                        reinterpret_cast<V2*>(out1),
                                                        reinterpret_cast<V2*>(out2));
  IWF_CUDA(cudaGetLastError());
  count_launch();
  return IWF_OK;
}

template <typename T>
iwf_status residual_precond(const Batch& bt, const void* X, const void* HX, const double* theta,
                            const double* lam, const double* shift, const double* off2,
                            void* W, long long N, int b, double* partial, int slots_per_prob,
                            double* resid, cudaStream_t s) {
  using V2 = typename Cplx<T>::type;
  int g = grid_for(N, kResThreads);
  if (g > slots_per_prob) g = slots_per_prob;
  residual_kernel<T><<<dim3(g, bt.nprob), kResThreads, 0, s>>>(
      bt, reinterpret_cast<const V2*>(X), reinterpret_cast<const V2*>(HX), theta, lam, shift,
      off2, reinterpret_cast<V2*>(W), N, b, partial);
  IWF_CUDA(cudaGetLastError());
  count_launch();
  resid_finish<<<bt.nprob, 32, 0, s>>>(bt, partial, g, b, resid);
  IWF_CUDA(cudaGetLastError());
  count_launch();
  return IWF_OK;
}

static iwf_status small_smem_attr(const void* fn) {
  IWF_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(SmallShared)));
  return IWF_OK;
}

iwf_status svqb_small(const Batch& bt, const double2* G, int b, double drop, double2* T,
                      int* mask, int* status, cudaStream_t s) {
  static bool attr = false;
  if (!attr) { IWF_TRY(small_smem_attr((const void*)svqb_kernel)); attr = true; }
  svqb_kernel<<<bt.nprob, kSmallThreads, sizeof(SmallShared), s>>>(bt, G, b, drop, T, mask, status);
  IWF_CUDA(cudaGetLastError());
  count_launch();
  return IWF_OK;
}

iwf_status rayleigh_ritz_small(const Batch& bt, const double2* A, int m, int b, const int* mask,
                               int x_rows, double* theta, double2* Cx, double2* Cp,
                               int* mask_p, int* status, cudaStream_t s) {
  static bool attr = false;
  if (!attr) { IWF_TRY(small_smem_attr((const void*)rr_kernel)); attr = true; }
  rr_kernel<<<bt.nprob, kSmallThreads, sizeof(SmallShared), s>>>(bt, A, m, b, mask, x_rows, theta,
                                                                 Cx, Cp, mask_p, status);
  IWF_CUDA(cudaGetLastError());
  count_launch();
  return IWF_OK;
}

template <typename Tin, typename Tout>
iwf_status convert_block(const void* in, void* out, long long count, cudaStream_t s) {
  convert_kernel<Tin, Tout><<<grid_for(count, 256), 256, 0, s>>>(
      reinterpret_cast<const Tin*>(in), reinterpret_cast<Tout*>(out), count);
  IWF_CUDA(cudaGetLastError());
  count_launch();
  return IWF_OK;
}

template <typename T>
iwf_status random_block(void* X, long long N, int b, unsigned long long seed, cudaStream_t s) {
  const long long count = N * b;
  random_kernel<T><<<grid_for(count, 256), 256, 0, s>>>(
      reinterpret_cast<typename Cplx<T>::type*>(X), count, seed);
  IWF_CUDA(cudaGetLastError());
  count_launch();
  return IWF_OK;
}

iwf_status any_nonfinite(const double* x, long long count, int* flag, cudaStream_t s) {
  IWF_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
  nonfinite_kernel<<<grid_for(count, 256), 256, 0, s>>>(x, count, flag);
  IWF_CUDA(cudaGetLastError());
  count_launch();
  return IWF_OK;
}

iwf_status set_mask(const Batch& bt, int* mask, int off, int b, int value, const int* src,
                    cudaStream_t s) {
  mask_kernel<<<bt.nprob, 32, 0, s>>>(bt.nprob, mask, off, b, value, src);
  IWF_CUDA(cudaGetLastError());
  count_launch();
  return IWF_OK;
}

template iwf_status gram<double>(const Batch&, const BlockList&, const BlockList&, long long,
                                 double2*, double2*, int, cudaStream_t, bool);
template iwf_status gram<float>(const Batch&, const BlockList&, const BlockList&, long long,
                                double2*, double2*, int, cudaStream_t, bool);
template iwf_status block_update<double>(const Batch&, const BlockList&, long long, const double2*,
                                         const double2*, int, int, void*, void*, bool,
                                         cudaStream_t);
template iwf_status block_update<float>(const Batch&, const BlockList&, long long, const double2*,
                                        const double2*, int, int, void*, void*, bool,
                                        cudaStream_t);
template iwf_status residual_precond<double>(const Batch&, const void*, const void*, const double*,
                                             const double*, const double*, const double*, void*,
                                             long long, int, double*, int, double*, cudaStream_t);
template iwf_status residual_precond<float>(const Batch&, const void*, const void*, const double*,
                                            const double*, const double*, const double*, void*,
                                            long long, int, double*, int, double*, cudaStream_t);
template iwf_status convert_block<double, float>(const void*, void*, long long, cudaStream_t);
template iwf_status convert_block<float, double>(const void*, void*, long long, cudaStream_t);
template iwf_status random_block<double>(void*, long long, int, unsigned long long, cudaStream_t);
template iwf_status random_block<float>(void*, long long, int, unsigned long long, cudaStream_t);

}  // namespace iwf
