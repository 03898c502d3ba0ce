// Tall-skinny block kernels of the eigensolver: Gram products, block updates, the fused
// residual / preconditioner step, and the one-CTA dense Hermitian eigensolver used for the
// small Rayleigh-Ritz and orthonormalisation problems.
//
// A block of b vectors of length N is column-major (column j at offset j*N). A "block list"
// concatenates up to four blocks of equal width b into one logical N x (nb*b) matrix.
// Small matrices are complex double, row-major.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace iwf {

constexpr int kMaxBlock = 24;              // b, the eigensolver block size
constexpr int kMaxSmall = 3 * kMaxBlock;   // m = 3b, size of the Rayleigh-Ritz problem

template <typename T> struct Cplx;
template <> struct Cplx<double> { using type = double2; };
template <> struct Cplx<float> { using type = float2; };

struct BlockList {
  const void* p[4];
  int nb;       // number of blocks
  int b;        // columns per block
};

// Column k of a block list.
template <typename T>
__device__ __forceinline__ const typename Cplx<T>::type* col_ptr(const BlockList& L, int k,
                                                                 long long N) {
  using V2 = typename Cplx<T>::type;
  return reinterpret_cast<const V2*>(L.p[k / L.b]) + (size_t)(k % L.b) * N;
}

// Host-side launchers (defined in blockops.cu).
template <typename T>
iwf_status gram(const BlockList& A, const BlockList& B, long long N, double2* out,
                double2* partial, int partial_slots, cudaStream_t s);
// out = S C1 (and out2 = S C2 when C2 != nullptr); subtract: out -= S C1 instead.
template <typename T>
iwf_status block_update(const BlockList& S, long long N, const double2* C1, const double2* C2,
                        int q, void* out1, void* out2, bool subtract, cudaStream_t s);
// R = HX - X diag(theta); W = M R; partial squared column norms of R -> resid (sqrt'ed).
template <typename T>
iwf_status residual_precond(const void* X, const void* HX, const double* theta, const T* M,
                            void* W, long long N, int b, double* partial, int partial_slots,
                            double* resid, cudaStream_t s);
iwf_status svqb_small(const double2* G, int b, double drop, double2* T, int* mask,
                      int* status, cudaStream_t s);
iwf_status rayleigh_ritz_small(const double2* A, int m, int b, const int* mask, int x_rows,
                               double* theta, double2* Cx, double2* Cp, int* mask_p,
                               int* status, cudaStream_t s);
template <typename T>
iwf_status precond_diag(const double* lam, double shift, double off2, long long N, T* M,
                        cudaStream_t s);
template <typename Tin, typename Tout>
iwf_status convert_block(const void* in, void* out, long long count, cudaStream_t s);
template <typename T>
iwf_status random_block(void* X, long long N, int b, unsigned long long seed, cudaStream_t s);
iwf_status set_mask(int* mask, int b, int value, cudaStream_t s);

}  // namespace iwf
