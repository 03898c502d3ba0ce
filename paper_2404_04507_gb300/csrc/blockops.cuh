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

// A batch of nprob independent problems with the same geometry. Problem p's long blocks
// start pstride elements after problem p-1's (every BlockList pointer is problem 0's).
// Small per-problem matrices sit at fixed capacities: G kMaxSmall^2, C kMaxSmall*kMaxBlock,
// T kMaxBlock^2, theta/resid kMaxBlock, masks kMaxSmall. active (may be null): problems
// with active[p] == 0 are skipped by every kernel.
// Engines of the complex-double Gram products and block updates.
enum { kEngineTensor = 0,   // tcgen05 tensor cores, Ozaki scheme I (bf16 slices, ozaki.cu)
       kEngineDF = 1,       // double-float arithmetic on the FP32 pipes (about 48 bits)
       kEngineF64 = 2 };    // FP64 arithmetic
struct Batch {
  int nprob;
  long long pstride;
  const int* active;
  int engine = kEngineTensor;
  int* exps = nullptr;      // tensor engine: column scales, nprob x 2 kMaxSmall ints
  int* err = nullptr;       // tensor engine: device error word for a bounded wait that ran out
};
constexpr int kCapG = kMaxSmall * kMaxSmall;
constexpr int kCapC = kMaxSmall * kMaxBlock;
constexpr int kCapT = kMaxBlock * kMaxBlock;

// Host-side launchers (defined in blockops.cu).
// herm: the product is Hermitian (A^H A, or X^H H X for Hermitian H): only the blocks on and
// above the 24 x 24 block diagonal are formed, the rest are mirrored.
template <typename T>
iwf_status gram(const Batch& bt, const BlockList& A, const BlockList& B, long long N, double2* out,
                double2* partial, int slots_per_prob, cudaStream_t s, bool herm = false);
// out = S C1 (and out2 = S C2 when C2 != nullptr); subtract: out -= S C1 instead.
// Problem p's coefficient matrices start at C1 + p*cstride (kCapG for Gram outputs,
// kCapT for SVQB transforms, kCapC for Rayleigh-Ritz coefficients).
template <typename T>
iwf_status block_update(const Batch& bt, const BlockList& S, long long N, const double2* C1,
                        const double2* C2, int cstride, int q, void* out1, void* out2,
                        bool subtract, cudaStream_t s);
// R = HX - X diag(theta); W = M R with M_k = h/(h^2 + off2[p]), h = lam_k + shift[p]
// (Eq. precond, shifted); squared column norms of R -> resid (sqrt'ed).
template <typename T>
iwf_status residual_precond(const Batch& bt, const void* X, const void* HX, const double* theta,
                            const double* lam, const double* shift, const double* off2,
                            void* W, long long N, int b, double* partial, int slots_per_prob,
                            double* resid, cudaStream_t s);
iwf_status svqb_small(const Batch& bt, const double2* G, int b, double drop, double2* T,
                      int* mask, int* status, cudaStream_t s);
iwf_status rayleigh_ritz_small(const Batch& bt, const double2* A, int m, int b, const int* mask,
                               int x_rows, double* theta, double2* Cx, double2* Cp,
                               int* mask_p, int* status, cudaStream_t s);
template <typename Tin, typename Tout>
iwf_status convert_block(const void* in, void* out, long long count, cudaStream_t s);
template <typename T>
iwf_status random_block(void* X, long long N, int b, unsigned long long seed, cudaStream_t s);
// Tensor-core (Ozaki scheme I) versions of gram<double> and block_update<double> (ozaki.cu);
// partial holds nprob x slots_cap x 2 kCapG doubles.
iwf_status gram_tc(const Batch& bt, const BlockList& A, const BlockList& B, long long N,
                   double2* out, double* partial, int slots_cap, int* err, cudaStream_t s,
                   bool herm);
iwf_status update_tc(const Batch& bt, const BlockList& S, long long N, const double2* C1,
                     const double2* C2, int cstride, int q, double2* out1, double2* out2,
                     bool subtract, int* err, cudaStream_t s);
// *flag = 1 (device int) when any of count doubles at x is NaN or infinite, else 0.
iwf_status any_nonfinite(const double* x, long long count, int* flag, cudaStream_t s);
// mask[p*kMaxSmall + off + j] = value (or src[p*kMaxBlock + j]) for j < b, every problem.
iwf_status set_mask(const Batch& bt, int* mask, int off, int b, int value, const int* src,
                    cudaStream_t s);

}  // namespace iwf
