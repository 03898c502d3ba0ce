/*
 * CPU oracle: H~ psi as a direct spectral convolution, in plain C with OpenMP.
 * TEST INFRASTRUCTURE ONLY (tests/, smoke() and bench.py's CPU baseline call it; the CUDA
 * library never does).
 *
 * Sec. 4.1 (Eq. pseudospectral vector) defines H~ U~ = Lambda U~ + F V F^{-1} U~ with F = T F*
 * (Sec. 3.3, Eq. F). In exact arithmetic the potential term is the cyclic convolution on the
 * K* grid with the grid Fourier coefficients Vg of V (App. C folds each parent mode onto the
 * grid):  (F V F^{-1} U~)_i = sum_m Vg_m U~*_{(k*_i - m) mod lens}, where U~* places U~_j at
 * the grid position k*_j of window point j (the index-shift map of Sec. 3.2). This file
 * writes that sum out for every window point: the same operator as oracle/operator.py's
 * apply_stencil, the modes taken in the caller's order, each point independent (the points
 * are spread over the host's cores).
 *
 *   N, n          window points, lifted dimension
 *   lens[n]       grid side lengths (2K_1..2K_d, 2L_1..2L_{n-d})
 *   kstar[N*n]    grid position of each window point (row-major)
 *   lam[N]        Lambda_k = 1/2 |P k|^2 (Eq. discrete_Lambda)
 *   nm, shift[nm*n], vre[nm], vim[nm]   the nonzero grid coefficients Vg_m and their m
 *   nvec, psi, out  column-major N x nvec complex blocks, interleaved (re, im)
 */
#include <stdlib.h>

int oracle_apply(long long N, int n, const int* lens, const int* kstar, const double* lam,
                 int nm, const int* shift, const double* vre, const double* vim, int nvec,
                 const double* psi, double* out) {
  long long G = 1;
  for (int a = 0; a < n; ++a) G *= lens[a];
  long long* pos = (long long*)malloc(sizeof(long long) * (size_t)N);  /* flat grid index */
  long long* grid = (long long*)malloc(sizeof(long long) * (size_t)G);  /* window index or -1 */
  if (!pos || !grid) { free(pos); free(grid); return -1; }
  for (long long g = 0; g < G; ++g) grid[g] = -1;
  for (long long i = 0; i < N; ++i) {
    long long f = 0;
    for (int a = 0; a < n; ++a) f = f * lens[a] + kstar[i * n + a];
    pos[i] = f;
    grid[f] = i;
  }
  for (int c = 0; c < nvec; ++c) {
    const double* x = psi + 2 * (size_t)N * c;
    double* y = out + 2 * (size_t)N * c;
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < N; ++i) {
      double re = 0.0, im = 0.0;
      for (int q = 0; q < nm; ++q) {
        /* grid point k*_i - m (cyclic), then the window point stored there (if any) */
        long long f = 0;
        for (int a = 0; a < n; ++a) {
          int v = (kstar[i * n + a] - shift[q * n + a]) % lens[a];
          if (v < 0) v += lens[a];
          f = f * lens[a] + v;
        }
        const long long j = grid[f];
        if (j < 0) continue;
        const double xr = x[2 * j], xi = x[2 * j + 1];
        re += vre[q] * xr - vim[q] * xi;
        im += vre[q] * xi + vim[q] * xr;
      }
      y[2 * i] = re + lam[i] * x[2 * i];
      y[2 * i + 1] = im + lam[i] * x[2 * i + 1];
    }
  }
  free(pos);
  free(grid);
  return 0;
}
