// Shared host/device definitions of the IWFPM library: the plan object, error plumbing and
// small complex helpers. Every translation unit of the library includes this header.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/iwfpm.h"

#define IWF_MAX_N 8
#define IWF_MAX_LEN 32       // largest axis length handled by the register DFT codelets
#define IWF_MAX_GROUP 8192   // largest point count of one axis group staged in shared memory
#define IWF_MAX_RADIX 7      // largest prime factor of an axis longer than IWF_MAX_LEN

namespace iwf {

// Radices of the shared-memory FFT of axes longer than IWF_MAX_LEN, in stage order: 4 while
// it divides, then 2, 3, 5, 7.
__host__ __device__ constexpr int long_radix(int n) {
  return (n % 4 == 0) ? 4 : (n % 2 == 0) ? 2 : (n % 3 == 0) ? 3 : (n % 5 == 0) ? 5
         : (n % 7 == 0) ? 7 : n;
}

// Values one thread holds for a stage of radix R: whole butterflies, at most 16 values.
__host__ __device__ constexpr int long_stage_values(int R) { return R * (16 / R); }

// true if an axis of this length is handled (short: codelets; long: prime factors <= 7)
inline bool axis_len_ok(int len) {
  if (len < 1 || len > IWF_MAX_GROUP) return false;
  if (len <= IWF_MAX_LEN) return true;
  for (int r = len; r > 1;) {
    const int R = long_radix(r);
    if (R > IWF_MAX_RADIX) return false;
    r /= R;
  }
  return true;
}

// Smallest long_stage_values over the radices of an axis (16 for a power of two).
inline int long_axis_values(int len) {
  int v = 16;
  for (int r = len; r > 1;) {
    const int R = long_radix(r);
    if (long_stage_values(R) < v) v = long_stage_values(R);
    r /= R;
  }
  return v;
}

// Records a message for iwf_last_error() and returns the status unchanged.
iwf_status fail(iwf_status st, const std::string& msg);
iwf_status cuda_fail(cudaError_t e, const char* what);
void clear_error();

#define IWF_CUDA(call)                                                   \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) return ::iwf::cuda_fail(e_, #call);           \
  } while (0)

#define IWF_TRY(call)                                                    \
  do {                                                                   \
    iwf_status s_ = (call);                                              \
    if (s_ != IWF_OK) return s_;                                         \
  } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Geometry of the lifted grid, passed by value to kernels.
struct Geom {
  int d, n;
  int lens[IWF_MAX_N];     // 2K_1..2K_d, 2L_1..2L_{n-d}
  int half[IWF_MAX_N];     // K_1..K_d, L_1..L_{n-d}
  long long N;             // total points
  long long MI;            // (2K)^d, points of one k_I slice
  long long MII;           // (2L)^{n-d}, number of slices
};

// Potential representation on the grid G_{K,L}, already multiplied by 1/N.
struct PotDev {
  int kind;                // 1: per-axis tables, 2: full grid
  int tab_off[IWF_MAX_N];  // offset of axis j's table (length lens[j]) in tab
  const double* tab64;     // per-axis tables (kind 1)
  const float* tab32;
  double c64;              // constant term (kind 1)
  float c32;
  const double* grid64;    // kind 2: N values, data layout (l_II slow, l_I fast)
  const float* grid32;
  long long tab_stride;    // batches: table entries between consecutive problems
  int vecs_per_prob;       // batches: vectors per problem (0: one problem)
  const int* active;       // batches: problem p skipped when active[p] == 0 (may be null)
};

// Per-problem potential tables of a batch of problems sharing one plan's geometry: problem
// p's axis tables (constant term folded into axis 0) start at p * tab_stride.
struct ApplyBatch {
  const double* tab64;
  const float* tab32;
  long long tab_stride;
  int vecs_per_prob;
  const int* active;
};

}  // namespace iwf

struct iwf_plan {
  int device = 0;
  int method = IWF_METHOD_IWFPM;
  int shift_round = IWF_SHIFT_EXACT;
  iwf::Geom g{};
  double P[IWF_MAX_N * IWF_MAX_N] = {};
  double Q[IWF_MAX_N * IWF_MAX_N] = {};   // d x (n-d), row-major; zero for PM
  int* d_lo = nullptr;                    // MII x d slice lower bounds lo_j(k_II)
  double* d_lam64 = nullptr;              // N kinetic diagonal
  float* d_lam32 = nullptr;
  int* d_err = nullptr;                   // device error word
  int* d_apply_err = nullptr;             // set by an apply kernel whose bounded wait ran out
  long long wait_rounds = -1;             // main-wait bound of pipelined passes (-1: default)
  // potential
  int pot_kind = 0;                       // 0 unset, 1 tables, 2 grid
  double* d_tab64 = nullptr;
  float* d_tab32 = nullptr;
  double* d_grid64 = nullptr;
  float* d_grid32 = nullptr;
  double vconst = 0.0;                    // constant term of V (unscaled)
  double vg0 = 0.0;                       // Re Vg_0
  double voff_abs = 0.0;                  // sum_{m != 0} |Vg_m|
  double voff_sq = 0.0;                   // sum_{m != 0} |Vg_m|^2
  int tab_off[IWF_MAX_N] = {};
  // folded modes of the potential for the direct-convolution apply (iwf_apply_stencil):
  // stencil_m[q*n + j] in [0, lens[j]), coefficient stencil_c[q] = Vg (re, im)
  int stencil_nm = 0;
  int* d_stencil_m = nullptr;
  double2* d_stencil_c = nullptr;
  // exp(2 pi i j / len), j < len, for every axis of a group with an axis longer than
  // IWF_MAX_LEN (null otherwise)
  double2* d_ltw64[IWF_MAX_N] = {};
  float2* d_ltw32[IWF_MAX_N] = {};
  // partial sums of iwf_evaluate's slice groups, grown on demand
  double2* d_eval_part = nullptr;
  size_t eval_part_bytes = 0;
  // four words for the field reductions: max key, first index, multiplier (double2)
  unsigned long long* d_field = nullptr;
  // workspace for the apply
  void* d_work = nullptr;
  size_t work_bytes = 0;
  // apply launch schedule per precision (0: FP64, 1: complex64), set by iwf_plan_autotune
  int tune_threads[2] = {256, 256};
  int tune_tile_kb[2] = {160, 160};
  int tune_chunk_mb[2] = {48, 48};
  // host-block pipeline (iwf_apply_host): two input and two output chunk buffers, streams for
  // host-to-device copies, compute and device-to-host copies, and the events that order them;
  // created on first use
  void* d_hin[2] = {nullptr, nullptr};
  void* d_hout[2] = {nullptr, nullptr};
  size_t host_chunk_bytes = 0;
  cudaStream_t host_stream[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t host_ev[9] = {};
  // apply kernels per precision: IWF_PATH_AUTO (pencil path where the geometry allows it),
  // IWF_PATH_TILED or IWF_PATH_PENCIL
  int path[2] = {IWF_PATH_AUTO, IWF_PATH_AUTO};
  // DFT arithmetic of FP64 applies on the pencil path (IWF_ARITH_F64 or IWF_ARITH_DF)
  int fft_arith = IWF_ARITH_F64;
  // eigensolver workspace of iwf_eigensolve / iwf_batch_eigensolve, kept between solves: the
  // buffers in the order a solve requests them, each reused while large enough
  struct SolveBuf { void* ptr; size_t bytes; };
  std::vector<SolveBuf> solve_ws;
};

namespace iwf {
iwf_status ensure_workspace(iwf_plan* p, size_t bytes);
// Optional per-pass timing of one apply (events on the launching stream).
struct PassTimer {
  cudaEvent_t ev[2] = {nullptr, nullptr};
  double ms[3] = {0, 0, 0};
  int launches[3] = {0, 0, 0};
};
iwf_status apply_impl(iwf_plan* p, int precision, const void* psi, void* hpsi, int nvec,
                      cudaStream_t stream, PassTimer* timer = nullptr,
                      const ApplyBatch* batch = nullptr);
iwf_status apply_noalloc_impl(iwf_plan* p, int precision, const void* psi, void* hpsi, int nvec,
                              cudaStream_t stream);
iwf_status apply_host_impl(iwf_plan* p, int precision, const void* psi_host, void* hpsi_host,
                           int nvec, cudaStream_t stream);
iwf_status apply_stencil_impl(iwf_plan* p, int precision, const void* psi, void* hpsi, int nvec,
                              cudaStream_t stream);
iwf_status evaluate_impl(iwf_plan* p, const void* coef, const double* x, long long M,
                         void* u, cudaStream_t stream);
void release_host_pipeline(iwf_plan* p);
iwf_status build_long_twiddles(iwf_plan* p);
iwf_status evaluate_grid_impl(iwf_plan* p, const void* coef, const double* origin,
                              const double* step, const int* count, void* u, cudaStream_t stream);
iwf_status field_normalize_impl(iwf_plan* p, void* u, long long M, long long at, double* rho,
                                long long* argmax, cudaStream_t stream);
iwf_status field_distance_impl(iwf_plan* p, const void* u, const void* v, long long M,
                               double* dist, cudaStream_t stream);
iwf_status eigensolve_impl(iwf_plan* p, const iwf_solve_opts* o, const void* X0, double* evals,
                           void* evecs, double* resid, iwf_solve_info* info, cudaStream_t st);
iwf_status batch_eigensolve_impl(iwf_plan* p, int nprob, const int* nmodes, const int* m,
                                 const double* re, const double* im, const iwf_solve_opts* o,
                                 const void* X0, double* evals, void* evecs, double* resid,
                                 int* iters, iwf_solve_info* info, cudaStream_t st);
iwf_status batch_solve_impl(int nplans, iwf_plan* const* plans, const iwf_solve_opts* o,
                            const void* const* X0, double* evals, void* const* evecs,
                            double* resid, int* iters, iwf_solve_info* info, cudaStream_t st);
iwf_status autotune_impl(iwf_plan* p, int precision, int nvec, double* best_ms, int* best,
                         cudaStream_t stream);
iwf_status set_schedule_impl(iwf_plan* p, int precision, int threads, int tile_kb, int chunk_mb);
iwf_status set_path_impl(iwf_plan* p, int precision, int path);
// Reads (and clears) the apply error word after synchronising `stream`: IWF_ERR_TIMEOUT when
// a pipelined apply kernel gave up waiting for one of its copies.
iwf_status check_apply_error(iwf_plan* p, cudaStream_t stream);
iwf_status get_schedule_impl(const iwf_plan* p, int precision, int* sched);
iwf_status set_arith_impl(iwf_plan* p, int arith);
void count_launch();
long long launch_count();
iwf_status build_window_tables(iwf_plan* p);          // lo table, Lambda; sets d_err on ties
iwf_status export_window(const iwf_plan* p, int* k_host);
iwf_status coef_extent(const iwf_plan* p, const void* coef, double threshold, int* need,
                       cudaStream_t s);
iwf_status build_potential(iwf_plan* p, int nmodes, const int* m, const double* re,
                           const double* im);
// Potential summaries used by the preconditioner (Eq. precond): Re Vg_0, sum |Vg_m|,
// sum |Vg_m|^2 over m != 0 after folding onto the grid.
struct PotSummary {
  double vg0 = 0, off_abs = 0, off_sq = 0;
  bool separable = true;
};
// Per-axis tables (scaled by 1/N, constant folded into axis 0) of one separable potential,
// written at tab64/tab32 (length sum of lens); the host summary goes to *sum.
iwf_status potential_tables(const iwf_plan* p, int nmodes, const int* m, const double* re,
                            const double* im, double* tab64, float* tab32, PotSummary* sum,
                            cudaStream_t s);
}  // namespace iwf
