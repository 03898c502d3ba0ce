// Register-resident DFT codelets for the axis lengths of the lifted grid (2 <= len <= 32).
//
// A codelet transforms one pencil held in two register arrays (re, im) in place:
//   X[k] = sum_n x[n] w^{n k},  w = exp(S * 2 pi i / len),  S = +1 (inverse, unnormalised)
//                                                          S = -1 (forward, unnormalised).
// It recurses by decimation in time, len = R * M with R = 4 when 4 | len, else 2, else the
// smallest odd prime factor; every loop is unrolled, so all indices and twiddle exponents
// are compile-time constants and trivial twiddles (1, -1, +-i) cost nothing. Non-trivial
// twiddles come from a per-length table in constant memory (uniform across a warp, so the
// constant cache broadcasts them and they feed the FMA directly).
//
// The tables live in this translation unit: include this header from exactly one .cu file.
#pragma once

#include <cuda_runtime.h>

namespace iwf {

constexpr int kTwTotal = IWF_MAX_LEN * (IWF_MAX_LEN + 1) / 2;  // sum of len over 1..32

// entry (len, j) at len*(len-1)/2 + j holds (cos 2 pi j/len, sin 2 pi j/len); the
// double-float table holds (cos.h, cos.l, sin.h, sin.l)
static __constant__ double2 c_tw64[kTwTotal];
static __constant__ float2 c_tw32[kTwTotal];
static __constant__ float4 c_twdf[kTwTotal];

__host__ __device__ constexpr int tw_off(int len) { return len * (len - 1) / 2; }

__host__ __device__ constexpr int radix_of(int n) {
  return (n % 4 == 0) ? 4
         : (n % 2 == 0) ? 2
         : (n % 3 == 0) ? 3
         : (n % 5 == 0) ? 5
         : (n % 7 == 0) ? 7
         : (n % 11 == 0) ? 11
         : (n % 13 == 0) ? 13
         : (n % 17 == 0) ? 17
         : (n % 19 == 0) ? 19
         : (n % 23 == 0) ? 23
         : (n % 29 == 0) ? 29
         : n;
}

// Double-float scalar for the DFTs of an FP64-storage apply run on the FP32 pipes: the value
// h + l with |l| <= ulp(h) / 2, about 48 significant bits. Addition keeps the rounding error
// of the high parts by Knuth's TwoSum and adds the low parts to it (no cancellation-proof
// renormalisation: the error stays below about 2^-45 of |a| + |b|, the norm-wise bound an FFT
// needs); multiplication forms the high product exactly with fma (Dekker/Kahan).
struct dfl {
  float h, l;
  dfl() = default;
  __device__ __forceinline__ constexpr dfl(float a, float b) : h(a), l(b) {}
  __device__ __forceinline__ explicit constexpr dfl(int z) : h((float)z), l(0.f) {}
};
__device__ __forceinline__ dfl dfl_quick(float s, float e) {
  const float h = s + e;
  return dfl(h, e - (h - s));
}
__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
  const float s = a.h + b.h;
  const float bb = s - a.h;
  float e = (a.h - (s - bb)) + (b.h - bb);
  e += a.l + b.l;
  return dfl_quick(s, e);
}
__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.h, -a.l); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + dfl(-b.h, -b.l); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return dfl_quick(p, e);
}
__device__ __forceinline__ dfl& operator+=(dfl& a, dfl b) { a = a + b; return a; }

// FP64 <-> double-float in integer arithmetic (no FP64 instruction: on this GPU those issue
// at 1/64 of the FP32 rate). to_dfl: h = x rounded to 24 significant bits (ties away from
// zero), l = the exact remainder rounded to a float; values below 2^-100 in magnitude, and
// denormals, become 0 (an apply's vectors are normalised; such entries are far below the
// double-float resolution of any vector that holds them), values above 2^127 saturate.
__device__ __forceinline__ dfl to_dfl(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int hi = (unsigned int)(b >> 32), lo = (unsigned int)b;
  const int e = (int)((hi >> 20) & 0x7FFu);
  if (e < 1023 - 100) return dfl(0.f, 0.f);
  const unsigned int sign = hi & 0x80000000u;
  const int fe = e < 1023 + 127 ? e - 1023 + 127 : 254;
  // top 23 stored mantissa bits and the 29 below them; round on bit 28
  const unsigned int m23 = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  const unsigned int rest = lo & 0x1FFFFFFFu;
  const unsigned int up = rest >> 28;                     // 1: round the magnitude up
  const unsigned int hb = sign | ((unsigned int)fe << 23) | m23;
  const float h = __uint_as_float(hb + up);               // a carry moves into the exponent
  // remainder x - h = (rest - up 2^29) 2^(e - 1075), |.| <= 2^28 units: exact as an int,
  // rounded once to a float, scaled by 2^(e - 1075) through its exponent field
  const int r = (int)rest - (int)(up << 29);
  if (r == 0) return dfl(h, 0.f);
  float l = (float)r;                                     // |l| < 2^29: exponent <= 127 + 28
  const int le = (int)((__float_as_uint(l) >> 23) & 0xFFu) + (e - 1075);
  l = le > 0 ? __uint_as_float(__float_as_uint(l) + (unsigned int)((e - 1075) << 23)) : 0.f;
  return dfl(h, sign ? -l : l);
}
// h + l rounded to FP64: the float h widened exactly, l added at its place below h's last
// bit with one 64-bit integer add and a final round on the dropped bits (|l| <= ulp(h) / 2).
__device__ __forceinline__ double from_dfl(dfl v) {
  const unsigned int hb = __float_as_uint(v.h);
  const int fe = (int)((hb >> 23) & 0xFFu);
  if (fe == 0) return 0.0;                                // h = 0 (or a denormal: below 2^-126)
  const unsigned long long sign = (unsigned long long)(hb & 0x80000000u) << 32;
  // |h| as a 53-bit significand M (implicit bit included) times 2^(fe - 127 - 52)
  long long M = (long long)(((hb & 0x7FFFFFu) | 0x800000u)) << 29;
  const unsigned int lb = __float_as_uint(v.l);
  const int le = (int)((lb >> 23) & 0xFFu);
  if (le != 0) {
    // l = +-ml 2^(le - 127 - 23); in units of 2^(fe - 127 - 52): shift by (le - 23) - (fe - 52)
    long long ml = (long long)((lb & 0x7FFFFFu) | 0x800000u);
    const int sh = (le - 23) - (fe - 52);
    if (sh >= 0) ml <<= sh;
    else ml = sh > -64 ? ((ml >> (-sh - 1)) + 1) >> 1 : 0;  // round half up on the dropped bits
    // the sign of l relative to h
    M += ((lb ^ hb) & 0x80000000u) ? -ml : ml;
  }
  // renormalise M (it stays within [2^51, 2^54) since |l| <= ulp(h) / 2)
  int de = 0;
  if (M >= (1LL << 53)) { M = (M + 1) >> 1; de = 1; }
  else if (M < (1LL << 52)) { M <<= 1; de = -1; }
  const long long e64 = (long long)fe - 127 + 1023 + de;
  return __longlong_as_double((long long)(sign | ((unsigned long long)e64 << 52) |
                                           ((unsigned long long)M & 0xFFFFFFFFFFFFFull)));
}

template <typename T> __device__ __forceinline__ T tw_cos(int off);
template <typename T> __device__ __forceinline__ T tw_sin(int off);
template <> __device__ __forceinline__ double tw_cos<double>(int off) { return c_tw64[off].x; }
template <> __device__ __forceinline__ double tw_sin<double>(int off) { return c_tw64[off].y; }
template <> __device__ __forceinline__ float tw_cos<float>(int off) { return c_tw32[off].x; }
template <> __device__ __forceinline__ float tw_sin<float>(int off) { return c_tw32[off].y; }
template <> __device__ __forceinline__ dfl tw_cos<dfl>(int off) {
  const float4 t = c_twdf[off];
  return dfl(t.x, t.y);
}
template <> __device__ __forceinline__ dfl tw_sin<dfl>(int off) {
  const float4 t = c_twdf[off];
  return dfl(t.z, t.w);
}

template <int S, typename T> __device__ __forceinline__ T sgn(T x) {
  if constexpr (S > 0) return x; else return -x;
}

// (re + i im) *= exp(S * 2 pi i j / LEN) for a compile-time-constant j after unrolling.
template <int LEN, int S, typename T>
__device__ __forceinline__ void twiddle(int j, T& re, T& im) {
  j %= LEN;
  if (j == 0) return;
  if (2 * j == LEN) { re = -re; im = -im; return; }
  if (4 * j == LEN) {            // w = S i
    T t = re; re = sgn<-S>(im); im = sgn<S>(t); return;
  }
  if (4 * j == 3 * LEN) {        // w = -S i
    T t = re; re = sgn<S>(im); im = sgn<-S>(t); return;
  }
  const T c = tw_cos<T>(tw_off(LEN) + j);
  const T s = sgn<S>(tw_sin<T>(tw_off(LEN) + j));
  const T r = re * c - im * s;
  im = re * s + im * c;
  re = r;
}

// In-place small DFT of size R (the combine step of one decimation level).
template <int R, int S, typename T> struct Butterfly {
  // odd R: pair up t_j and t_{R-j}; X_q = A_q + S i B_q, X_{R-q} = A_q - S i B_q
  static __device__ __forceinline__ void run(T (&xr)[R], T (&xi)[R]) {
    constexpr int H = (R - 1) / 2;
    T sr[H + 1], si[H + 1], dr[H + 1], di[H + 1];
#pragma unroll
    for (int j = 1; j <= H; ++j) {
      sr[j] = xr[j] + xr[R - j]; si[j] = xi[j] + xi[R - j];
      dr[j] = xr[j] - xr[R - j]; di[j] = xi[j] - xi[R - j];
    }
    T or_[R], oi[R];
    T a0r = xr[0], a0i = xi[0];
#pragma unroll
    for (int j = 1; j <= H; ++j) { a0r += sr[j]; a0i += si[j]; }
    or_[0] = a0r; oi[0] = a0i;
#pragma unroll
    for (int q = 1; q <= H; ++q) {
      T ar = xr[0], ai = xi[0], br = T(0), bi = T(0);
#pragma unroll
      for (int j = 1; j <= H; ++j) {
        const int e = (j * q) % R;
        const T c = tw_cos<T>(tw_off(R) + e), s = tw_sin<T>(tw_off(R) + e);
        ar += c * sr[j]; ai += c * si[j];
        br += s * dr[j]; bi += s * di[j];
      }
      // S i B = (-S bi, S br)
      or_[q] = ar + sgn<-S>(bi); oi[q] = ai + sgn<S>(br);
      or_[R - q] = ar + sgn<S>(bi); oi[R - q] = ai + sgn<-S>(br);
    }
#pragma unroll
    for (int q = 0; q < R; ++q) { xr[q] = or_[q]; xi[q] = oi[q]; }
  }
};

template <int S, typename T> struct Butterfly<2, S, T> {
  static __device__ __forceinline__ void run(T (&xr)[2], T (&xi)[2]) {
    const T ar = xr[0], ai = xi[0];
    xr[0] = ar + xr[1]; xi[0] = ai + xi[1];
    xr[1] = ar - xr[1]; xi[1] = ai - xi[1];
  }
};

template <int S, typename T> struct Butterfly<4, S, T> {
  static __device__ __forceinline__ void run(T (&xr)[4], T (&xi)[4]) {
    const T s0r = xr[0] + xr[2], s0i = xi[0] + xi[2];
    const T d0r = xr[0] - xr[2], d0i = xi[0] - xi[2];
    const T s1r = xr[1] + xr[3], s1i = xi[1] + xi[3];
    const T d1r = xr[1] - xr[3], d1i = xi[1] - xi[3];
    xr[0] = s0r + s1r; xi[0] = s0i + s1i;
    xr[2] = s0r - s1r; xi[2] = s0i - s1i;
    // X1 = d0 + S i d1, X3 = d0 - S i d1
    xr[1] = d0r + sgn<-S>(d1i); xi[1] = d0i + sgn<S>(d1r);
    xr[3] = d0r + sgn<S>(d1i);  xi[3] = d0i + sgn<-S>(d1r);
  }
};

template <int N, int S, typename T> struct Dft {
  static __device__ __forceinline__ void run(T (&xr)[N], T (&xi)[N]) {
    constexpr int R = radix_of(N);
    constexpr int M = N / R;
    if constexpr (M == 1) {
      Butterfly<R, S, T>::run(xr, xi);
    } else {
      T yr[R][M], yi[R][M];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int m = 0; m < M; ++m) { yr[r][m] = xr[R * m + r]; yi[r][m] = xi[R * m + r]; }
#pragma unroll
      for (int r = 0; r < R; ++r) Dft<M, S, T>::run(yr[r], yi[r]);
#pragma unroll
      for (int k = 0; k < M; ++k) {
        T tr[R], ti[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          tr[r] = yr[r][k]; ti[r] = yi[r][k];
          twiddle<N, S, T>(r * k, tr[r], ti[r]);
        }
        Butterfly<R, S, T>::run(tr, ti);
#pragma unroll
        for (int q = 0; q < R; ++q) { xr[k + M * q] = tr[q]; xi[k + M * q] = ti[q]; }
      }
    }
  }
};

template <int S, typename T> struct Dft<1, S, T> {
  static __device__ __forceinline__ void run(T (&)[1], T (&)[1]) {}
};

}  // namespace iwf
