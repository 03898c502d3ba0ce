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

// entry (len, j) at len*(len-1)/2 + j holds (cos 2 pi j/len, sin 2 pi j/len)
static __constant__ double2 c_tw64[kTwTotal];
static __constant__ float2 c_tw32[kTwTotal];

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

template <typename T> __device__ __forceinline__ T tw_cos(int off);
template <typename T> __device__ __forceinline__ T tw_sin(int off);
template <> __device__ __forceinline__ double tw_cos<double>(int off) { return c_tw64[off].x; }
template <> __device__ __forceinline__ double tw_sin<double>(int off) { return c_tw64[off].y; }
template <> __device__ __forceinline__ float tw_cos<float>(int off) { return c_tw32[off].x; }
template <> __device__ __forceinline__ float tw_sin<float>(int off) { return c_tw32[off].y; }

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
