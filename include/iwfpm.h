/*
 * iwfpm.h -- C ABI of the GB300 (sm_103a) implementation of the irrational-window-filter
 * projection method (IWFPM) for quasiperiodic Schroedinger eigenproblems
 * (Jiang, Li, Ma, Zhang, Zhang, Zhou, arXiv 2404.04507).
 *
 * Conventions shared by every entry point
 *   - Every call returns an iwf_status. Nothing aborts or exits; after a failure
 *     iwf_last_error() returns a thread-local message describing it.
 *   - "host" pointers are ordinary CPU memory, "device" pointers are CUDA global memory on
 *     the plan's device. The caller owns every buffer it passes in; the library owns a plan
 *     and its workspace and frees them in iwf_plan_destroy.
 *   - Coefficient vectors hold U~_k for k in the window K_{K,L} in WINDOW ORDER: k_II
 *     lexicographic (slowest), then k_I lexicographic, each k_I axis running over its 2K_j
 *     consecutive integers from the slice's lower bound. Element type: complex double
 *     (interleaved re,im; 16 bytes) for IWF_PREC_F64, complex float (8 bytes) for
 *     IWF_PREC_C64. A block of nvec vectors is column-major: vector v starts at element v*N.
 *   - "stream" is a cudaStream_t (NULL = the legacy default stream). Calls that take a
 *     stream enqueue their GPU work on it; they return after enqueueing unless stated.
 */
#ifndef IWFPM_H
#define IWFPM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IWF_OK = 0,
  IWF_ERR_ARG = -1,           /* invalid argument (null pointer, size, shape)              */
  IWF_ERR_SINGULAR_PI = -2,   /* P_I (first d columns of P) singular or cond > 1e12        */
  IWF_ERR_ALLOC = -3,         /* device or host allocation failed                          */
  IWF_ERR_CUDA = -4,          /* a CUDA runtime call failed                                */
  IWF_ERR_NONFINITE = -5,     /* NaN/Inf met in the input or during a solve                */
  IWF_ERR_BREAKDOWN = -6,     /* Gram matrix not positive definite after re-orthogonalising */
  IWF_ERR_NOCONV = -7,        /* eigensolver hit maxit; partial results are returned       */
  IWF_ERR_TIMEOUT = -8,       /* a bounded device wait ran out                             */
  IWF_ERR_WINDOW_TIE = -9,    /* a window bound lies within 1e-9 of an integer             */
  IWF_ERR_UNSUPPORTED = -10   /* shape outside what the kernels support (see iwf_plan_create) */
} iwf_status;

enum { IWF_METHOD_IWFPM = 0, IWF_METHOD_PM = 1 };
enum { IWF_SHIFT_EXACT = 0, IWF_SHIFT_ROUND = 1 };
enum { IWF_PREC_F64 = 0, IWF_PREC_C64 = 1, IWF_PREC_F64_EXACT = 2, IWF_PREC_F64_DF = 3 };

typedef struct iwf_plan iwf_plan; /* opaque, library-owned */

typedef struct {
  int method;      /* IWF_METHOD_IWFPM (irrational window) or IWF_METHOD_PM (box)          */
  int shift_round; /* IWF_SHIFT_EXACT: lower bound ceil(-K - (Q k_II)_j) as in Sec. 3.2;
                      IWF_SHIFT_ROUND: -K - round((Q k_II)_j), round half away from zero   */
  int device;      /* CUDA device ordinal the plan lives on                                */
} iwf_plan_opts;

/* Library version as major*10000 + minor*100 + patch. */
int iwf_version(void);

/* Thread-local description of the last failure on this thread ("" if none). */
const char* iwf_last_error(void);

/*
 * Build a plan for the lifted operator of Sec. 3.1-3.2 and Sec. 4.1.
 *   d, n   physical and lifted dimension, 1 <= d < n <= 8.
 *   P      host, d*n doubles, row-major: the projection matrix (Def. 2.1). Its first d
 *          columns P_I must be invertible (Sec. 3.1); reorder columns otherwise.
 *   K, L   host, d and n-d ints >= 1: window sizes (vector form, Remark after Fig. 1).
 *          IWFPM: k_II in [-L,L)^{n-d}, k_I + Q k_II in [-K,K)^d with Q = P_I^{-1} P_II.
 *          PM: the box [-K,K)^d x [-L,L)^{n-d}.
 *   opts   host, may be NULL (IWFPM, exact shift, device 0).
 * Supported: every axis length 2K_j, 2L_j in [2, 32], or in (32, 8192] with no prime factor
 * above 7 (e.g. 40, 120, 1280, 8192); (2K)^d at most 8192. Axis groups with an axis above 32
 * run a shared-memory FFT instead of the register codelets. A k_II group too large for one
 * shared-memory tile ((2L)^{n-d} above 8192 points, or above 16 x 512 points per radix
 * stage of its FFT) runs as one pass per k_II axis; a k_I group that large gives
 * IWF_ERR_UNSUPPORTED at the apply.
 * The window, its slice bounds and Lambda = 1/2 |P k|^2 (Eq. discrete_Lambda)
 * are built on the device; the call synchronises the device.
 * Errors: IWF_ERR_ARG, IWF_ERR_SINGULAR_PI, IWF_ERR_UNSUPPORTED, IWF_ERR_WINDOW_TIE,
 * IWF_ERR_ALLOC, IWF_ERR_CUDA. On error *plan is set to NULL.
 */
iwf_status iwf_plan_create(iwf_plan** plan, int d, int n, const double* P, const int* K,
                           const int* L, const iwf_plan_opts* opts);

/* Release the plan and all device memory it owns. NULL is ignored. */
void iwf_plan_destroy(iwf_plan* plan);

/* N = (2K)^d (2L)^{n-d}, the number of window points (DOF, Sec. 3.3). */
iwf_status iwf_plan_size(const iwf_plan* plan, long long* N);

/* The n grid side lengths (2K_1..2K_d, 2L_1..2L_{n-d}) of K*_{K,L} (Sec. 3.2). */
iwf_status iwf_plan_lens(const iwf_plan* plan, int* lens);

/*
 * The window K_{K,L} itself: host output k of N*n ints, row k[i*n + j] = component j of the
 * true index of window position i (the inverse of the index-shift map, Eqs. inverse1-3).
 * Synchronises the device.
 */
iwf_status iwf_window(const iwf_plan* plan, int* k);

/* Lambda_k = 1/2 |P k|^2 for every window position, host output of N doubles. */
iwf_status iwf_kinetic(const iwf_plan* plan, double* lam);

/*
 * Extent of the concentrated coefficients of a vector on this window (the "concentrated
 * area" of the Fourier coefficients, Sec. 4.2, Example 4.1): need[j] is the smallest half-
 * width K'_j (j < d) or L'_j (j >= d) of a window with this plan's centring that contains
 * every position with |coef_k| >= threshold. For a k_I axis a position at offset o in its
 * slice (o = k_I,j - lo_j in [0, 2K_j)) needs max(K_j - o, o - K_j + 1); for a k_II axis
 * the coordinate k_II,j needs max(-k_II,j, k_II,j + 1). need[j] = K_j (or L_j) means the
 * concentrated coefficients reach the window's edge along axis j; 0 that no position
 * passes the threshold. Used to size windows automatically from the decay of a solution.
 *   coef       device, N complex doubles (window order), 16-byte aligned.
 *   threshold  absolute magnitude, finite and >= 0.
 *   need       host, n ints.
 * Synchronises `stream`. Errors: IWF_ERR_ARG, IWF_ERR_CUDA. Library extension (the paper
 * reads the concentrated area off its figures).
 */
iwf_status iwf_coef_extent(const iwf_plan* plan, const void* coef, double threshold, int* need,
                           void* stream);

/*
 * Set the lifted potential V(y) = sum_m c_m exp(i m.y) (Sec. 4.1, V sampled on G_{K,L}).
 *   nmodes >= 0; m host nmodes*n ints (row per mode); re, im host nmodes doubles.
 * V must be real: every mode m != 0 must come with -m and the conjugate coefficient
 * (checked to 1e-12 relative; IWF_ERR_ARG otherwise). Modes are folded onto the grid by
 * the aliasing rule of App. C. When every mode lies on one lifted axis, V is kept as n
 * per-axis tables; otherwise as a full grid of N values per precision.
 * Synchronises the device.
 */
iwf_status iwf_set_potential(iwf_plan* plan, int nmodes, const int* m, const double* re,
                             const double* im);

/*
 * hpsi = H~ psi = Lambda psi + F V F^{-1} psi for nvec vectors (Sec. 4.1, Eq. pseudospectral
 * vector), with F = T F* (Sec. 3.3, Eq. F): gather through the index shift, inverse n-D
 * FFT, multiply by V, forward n-D FFT, scatter back to the window and add Lambda psi.
 *   precision  IWF_PREC_F64 (complex double I/O and arithmetic) or IWF_PREC_C64
 *              (complex float I/O and arithmetic, Lambda applied in float).
 *   psi, hpsi  device, N*nvec elements each, column-major, window order; must not overlap.
 *              Both must be 16-byte aligned.
 *   nvec >= 0; stream as above. Uses the plan's workspace: calls on one plan must not run
 *   concurrently on different streams.
 * Errors: IWF_ERR_ARG (no potential set, bad pointers), IWF_ERR_ALLOC, IWF_ERR_CUDA.
 */
iwf_status iwf_apply(iwf_plan* plan, int precision, const void* psi, void* hpsi, int nvec,
                     void* stream);

/*
 * Diagonal preconditioner of Eq. precond, M_kk = h_k / (h_k^2 + sum_{m != 0} |Vg_m|^2),
 * h_k = Lambda_k + Vg_0 + sigma with sigma = sum_{m != 0}|Vg_m| - Vg_0 + 1 (a shift that
 * makes V + sigma >= 1; it changes no eigenvector). Host outputs: M (N doubles, may be NULL)
 * and *sigma (may be NULL). Synchronises the device.
 */
iwf_status iwf_preconditioner(const iwf_plan* plan, double* M, double* sigma);

typedef struct {
  int nev;          /* eigenpairs wanted, 1 <= nev <= block                                 */
  int block;        /* LOBPCG block size b (0: b = nev), at most 24                          */
  int maxit;        /* iteration limit over both phases (0: 1000)                            */
  double tol;       /* stop when |H~x_i - lambda_i x_i|_2 <= tol for i < nev, |x_i|_2 = 1
                       (0: 1e-10)                                                           */
  int precision;    /* IWF_PREC_F64: every phase in complex double; the tall-skinny Gram
                       products and block updates run on the tensor cores (tcgen05) by the
                       Ozaki scheme: each FP64 value as seven 7-bit bf16 slices under a
                       shared power-of-two scale, exact fp32 sums per slice level, about 49
                       significant bits relative to the scales (iwf_gram).
                       IWF_PREC_F64_DF: the same contractions in double-float arithmetic on the
                       FP32 pipes (products exact by fma, sums by TwoSum: about 48 bits).
                       IWF_PREC_F64_EXACT: FP64 arithmetic in those contractions (slow on this
                       GPU, whose FP64 rate is 1/62 of FP32).
                       IWF_PREC_C64: a first phase with complex-float blocks and apply (FP64
                       small problems) until the residuals reach c64_tol or stall, then the
                       IWF_PREC_F64 phase to tol. Small problems are always FP64.          */
  double c64_tol;   /* residual target of the complex-float phase (0: 1e-5); the phase also
                       ends when its worst residual stops improving (a 30 % drop within
                       10 iterations)                                                      */
  unsigned long long seed; /* seed of the start block when X0 is NULL                       */
} iwf_solve_opts;

typedef struct {
  int iters;        /* LOBPCG iterations, both phases                                       */
  int iters_c64;    /* of which in the complex-float phase                                  */
  long long applies;/* vectors passed through H~                                            */
  int converged;    /* 1 when every wanted residual reached tol                             */
  double max_resid; /* largest final residual among the nev wanted pairs                    */
  double seconds;   /* wall time of the call                                                */
} iwf_solve_info;

/*
 * Lowest nev eigenpairs of H~ (Sec. 4.1) by block LOBPCG (Alg. 2 in block form, Knyazev's
 * method cited there) with the diagonal preconditioner of Eq. precond, shifted as described
 * for iwf_preconditioner. Every step runs on the device: the FFT apply, the residual and
 * preconditioner, Gram products and block updates (IWF_PREC_F64: tensor cores, FP64 values
 * split into 56-bit fixed-point bf16 digits, Ozaki scheme), orthonormalisation and the small
 * Rayleigh-Ritz eigenproblem (one-CTA Jacobi, FP64 angles, double-float rotations); the host
 * reads only the residual norms once per iteration.
 *   X0     device, N*block complex doubles (window order, column-major) or NULL for a seeded
 *          random start (splitmix64 counter generator).
 *   evals  host, nev doubles, ascending.   resid host, nev doubles (may be NULL).
 *          Each is the FP64 Rayleigh quotient x^H H~ x / x^H x of its returned vector, with
 *          H~ x applied afresh after the iteration: O(resid^2 / gap) from the exact
 *          eigenvalue, free of the Rayleigh-Ritz rounding (Ritz values differ by up to a few
 *          1e-12 once the projected matrix has large entries).
 *   evecs  device, N*nev complex doubles, orthonormal, column-major, window order.
 *   info   host (may be NULL).
 * The workspace (about 12 blocks of N*block complex values) stays on the plan after the call,
 * so a later solve of the same shape allocates nothing; iwf_plan_trim frees it. One solve at a
 * time per plan. The call synchronises `stream` before returning.
 * Errors: IWF_ERR_ARG, IWF_ERR_ALLOC, IWF_ERR_CUDA, IWF_ERR_NONFINITE (a NaN or Inf in X0,
 * checked on the device before the first iteration, or a non-finite residual), IWF_ERR_TIMEOUT
 * (an apply gave up waiting for a copy, read at the per-iteration synchronisation),
 * IWF_ERR_BREAKDOWN, IWF_ERR_NOCONV (outputs then hold the last iterate).
 */
iwf_status iwf_eigensolve(iwf_plan* plan, const iwf_solve_opts* opts, const void* X0,
                          double* evals, void* evecs, double* resid, iwf_solve_info* info,
                          void* stream);

/*
 * Lowest nev eigenpairs of nprob problems that share the plan's P, K, L and method but
 * each have their own lifted potential (for example a sweep over potential strengths and
 * phases). The problems advance in lockstep through the same kernels -- the apply takes
 * each vector's potential table from its problem, Gram products and updates carry the
 * problem in the grid, the small Rayleigh-Ritz problems run one CTA per problem -- and a
 * converged problem drops out by a device flag. The steady-state iteration is captured
 * into a CUDA graph and replayed. Same method, options and tolerance as iwf_eigensolve.
 *   nmodes  host, nprob ints; m (sum(nmodes) * n ints), re, im (sum(nmodes) doubles): the
 *           problems' mode lists, concatenated in problem order, as for iwf_set_potential.
 *           Every mode must lie on a single lifted axis (IWF_ERR_UNSUPPORTED otherwise).
 *   evals   host, nprob*nev (problem-major).  resid host, nprob*nev (may be NULL).
 *   evecs   device, nprob*N*nev complex doubles (problem p at offset p*N*nev), or NULL.
 *   iters   host, nprob ints (may be NULL): iterations each problem needed.
 *   info    host (may be NULL): totals over the batch (iters = lockstep iterations).
 *   X0      device, nprob*block*N complex doubles (problem p's start block at p*block*N,
 *           column-major, window order) or NULL for the seeded random start.
 * nprob * block <= 65535. The workspace stays on the plan, as for iwf_eigensolve.
 * Synchronises `stream`.
 */
iwf_status iwf_batch_eigensolve(iwf_plan* plan, int nprob, const int* nmodes, const int* m,
                                const double* re, const double* im, const iwf_solve_opts* opts,
                                const void* X0, double* evals, void* evecs, double* resid,
                                int* iters, iwf_solve_info* info, void* stream);

/*
 * Lowest nev eigenpairs of nplans independent problems, each given by its own plan (its own
 * window K, L, method and potential: for example a sweep over potential strengths, phases
 * and window cutoffs with uneven numbers of DOF). Each problem is Sec. 4.1's eigenproblem,
 * solved by the method and options of iwf_eigensolve. Plans with the same P, K, L, method and
 * shift form a group that advances in lockstep as one batch (as in iwf_batch_eigensolve);
 * groups run side by side on their own streams, as many as fit in about 60 % of the free
 * device memory, the largest first.
 *   plans   host, nplans plan pointers, all on one device; every potential must be a sum of
 *           single-axis modes (IWF_ERR_UNSUPPORTED otherwise). A plan may appear only once.
 *   X0      host array of nplans device pointers (each N_p*block complex doubles) or NULL;
 *           NULL entries (or X0 == NULL) take the seeded random start.
 *   evals   host, nplans*nev (plan-major).   resid host, nplans*nev (may be NULL).
 *   evecs   host array of nplans device pointers (each N_p*nev complex doubles, may be NULL),
 *           or NULL.   iters host, nplans ints (may be NULL).
 *   info    host (may be NULL): iters = the longest group's lockstep iterations, applies
 *           summed, converged = all, max_resid over all, seconds = wall time of the call.
 * The plans' workspaces are used: the caller must not apply with them meanwhile.
 * Synchronises `stream` (every group starts after the work already on it).
 * Errors: as iwf_eigensolve (IWF_ERR_NOCONV when some problem stopped at maxit; every
 * output is still written).
 */
iwf_status iwf_batch_solve(int nplans, iwf_plan* const* plans, const iwf_solve_opts* opts,
                           const void* const* X0, double* evals, void* const* evecs,
                           double* resid, int* iters, iwf_solve_info* info, void* stream);

/*
 * Frees the eigensolver workspace that iwf_eigensolve and iwf_batch_eigensolve keep on the
 * plan (iwf_batch_solve allocates its groups' workspaces per call and frees them before it
 * returns). The plan stays usable; the next solve allocates again. Waits for the plan's
 * device work (cudaFree). Library extension: the paper has no counterpart.
 */
void iwf_plan_trim(iwf_plan* plan);

/*
 * Learned warm start (no counterpart in the paper, whose start vector is e_1; Sec. 4.1):
 * an MLP from a potential's parameters to the lowest eigenvectors on a small "core" window.
 * Dense layers use bfloat16 weights and inputs with float32 accumulation on the tensor
 * cores (tcgen05.mma, accumulators in tensor memory; K split across CTAs when a layer has
 * few output tiles), GELU between layers, a linear output; float32 master weights and AdamW.
 * predict, loss_grad and train synchronise `stream` and return IWF_ERR_TIMEOUT when a GEMM's
 * bounded wait ran out (the word is then cleared).
 *   dims: nlayers+1 sizes, every one a multiple of 64 (pad the features with zeros).
 *   Output layout per sample: 2*nvec*ncore floats, (v*ncore + i)*2 + {0: re, 1: im}.
 * Loss per sample: |X X^H - Y Y^H|_F^2 / nvec for reference X and prediction Y on the core,
 * averaged over the batch (independent of each eigenvector's phase and of rotations inside
 * degenerate eigenspaces). Parameters are one flat float32 vector: per layer W (out x in,
 * row-major) then b (out). Batch sizes are multiples of 64. All pointers are device
 * pointers unless named host.
 */
typedef struct iwf_ws iwf_ws;
iwf_status iwf_ws_create(iwf_ws** ws, int nlayers, const int* dims, unsigned long long seed,
                         int device);
void iwf_ws_destroy(iwf_ws* ws);
iwf_status iwf_ws_num_params(const iwf_ws* ws, long long* n);
iwf_status iwf_ws_get_params(const iwf_ws* ws, float* host);            /* host nparams */
iwf_status iwf_ws_set_params(iwf_ws* ws, const float* host);            /* host nparams */
/* out (nsamples x dims[nlayers]) = MLP(feat (nsamples x dims[0])). */
iwf_status iwf_ws_predict(iwf_ws* ws, int nsamples, const float* feat, float* out, void* stream);
/* Loss (host scalar, may be NULL) and gradient (host nparams, may be NULL) of one batch. */
iwf_status iwf_ws_loss_grad(iwf_ws* ws, int nsamples, const float* feat, const float* target,
                            int nvec, int ncore, float* loss, float* grads_host, void* stream);
/* AdamW (beta 0.9/0.999, eps 1e-8, weight decay wd on W only) over shuffled batches;
   loss_hist host (epochs), mean batch loss per epoch (may be NULL). Synchronises. */
iwf_status iwf_ws_train(iwf_ws* ws, int nsamples, const float* feat, const float* target,
                        int nvec, int ncore, int epochs, int batch, float lr, float wd,
                        unsigned long long seed, float* loss_hist, void* stream);
/*
 * Embed vectors on the window of plan `core` into the window of plan `big` by true index k
 * (zero elsewhere). in: nprob*nvec vectors of core N; out: nprob*nvec vectors of big N
 * (complex double). The core window must lie inside the big one (IWF_ERR_ARG otherwise).
 */
iwf_status iwf_ws_embed(const iwf_plan* core, const iwf_plan* big, int nprob, int nvec,
                        const void* in, void* out, void* stream);
/*
 * vecs[p][v][k] *= exp(i * sign * k . phi_p) on the plan's window (true index k), in place:
 * nprob*nvec complex-double vectors, phases host nprob*n doubles, sign = +1 or -1.
 * A shift of the potential's phases, V(y) = sum_m c_m e^{i m.(y + phi)}, is this diagonal
 * unitary (H_phi = D H_0 D^H, D = diag(e^{i k.phi})) up to the grid wrap-around, so the
 * warm-start network needs to learn only the phase-free problem. Synchronises `stream`.
 */
iwf_status iwf_ws_phase(const iwf_plan* plan, int nprob, int nvec, const double* phases,
                        int sign, void* vecs, void* stream);

/*
 * Same computation as iwf_apply, with CUDA events recorded on `stream` around every pass
 * kernel (pass A: inverse DFT along k_I with the gather; pass B: k_II inverse DFT, V,
 * k_II forward DFT; pass C: forward DFT along k_I with the scatter and Lambda psi).
 * Synchronises the stream. Host outputs (may be NULL): pass_ms[3] = summed device time of
 * each pass in this call (ms), launches[3] = number of kernel launches of each pass.
 */
iwf_status iwf_apply_profile(iwf_plan* plan, int precision, const void* psi, void* hpsi,
                             int nvec, void* stream, double* pass_ms, int* launches);

/*
 * H~ psi (Sec. 4.1) for a block held in HOST memory.
 *   psi_host, hpsi_host  host, N*nvec elements each, column-major, window order, complex
 *                        double (IWF_PREC_F64) or complex float (IWF_PREC_C64); must not
 *                        overlap. Page-locked memory gives the full copy bandwidth; pageable
 *                        memory works, slower.
 * The block crosses the device in chunks of vectors: the host-to-device copy of one chunk,
 * the apply of the previous one and the device-to-host copy of the one before overlap on
 * internal streams. Two input and two output chunk buffers are allocated by the plan on first
 * use and kept until iwf_plan_destroy. The work is ordered after earlier work on `stream`
 * (NULL: the legacy default stream) and the call returns when hpsi_host is complete. Same
 * results as iwf_apply.
 */
iwf_status iwf_apply_host(iwf_plan* plan, int precision, const void* psi_host, void* hpsi_host,
                          int nvec, void* stream);

/*
 * Physical-space values u(x) = sum_{k in K_{K,L}} coef_k exp(i (P k).x) of the quasiperiodic
 * function with window coefficients coef (Sec. 3.1, Eq. int), e.g. an eigenvector, at M
 * points: the input of the paper's eigenfunction error E_f and density rho (Sec. 4.2).
 *   coef  device, N complex double, window order
 *   x     device, M x d doubles, row-major (point m at x + m*d)
 *   u     device, M complex double (output)
 * Direct summation in FP64, O(N M): each row along the fastest k_I axis by Horner's rule,
 * row phases exact (sincos) whenever the second-fastest k_I axis wraps and advanced by one
 * complex multiplication in between. Absolute errors are about (l_f + l_s + |theta|_max) eps
 * sum|coef|, with l_f, l_s the two fastest k_I extents and theta = (P k).x.
 * When M points fill too few CTAs, groups of slices are summed separately into a plan-owned
 * scratch (at most 256 MiB, allocated on first need, freed by iwf_plan_destroy) and added in
 * a fixed order: results do not depend on timing. Calls on one plan that overlap on the GPU
 * share that scratch and race. Enqueues on `stream`; M = 0 is a no-op; M < 0 or a NULL
 * pointer gives IWF_ERR_ARG.
 */
iwf_status iwf_evaluate(iwf_plan* plan, const void* coef, const double* x, long long M,
                        void* u, void* stream);

/*
 * The same values as iwf_evaluate on a uniform 2D grid, x = origin + (a step_0, b step_1) for
 * 0 <= a < count[0], 0 <= b < count[1] (the observation grids of Sec. 4.2), for plans with
 * d = 2, a diagonal P_I (P_01 = P_10 = 0, as in every example of the paper) and 2K_1, 2K_2 <= 32.
 * Then (P k).x separates over the two grid axes within each k_II slice, and the slice's share
 * of u is a product E0 C E1^T of its 2K_1 x 2K_2 coefficients with two phase tables: about 2K_2
 * times fewer operations per point than iwf_evaluate, in FP64.
 *   coef    device, N complex double, window order
 *   origin, step   host, 2 doubles each;  count  host, 2 ints
 *   u       device, count[0]*count[1] complex double, row-major (the last axis fastest)
 * Scratch and stream rules as iwf_evaluate. Errors: IWF_ERR_UNSUPPORTED for other plans (use
 * iwf_evaluate), IWF_ERR_ARG (NULL pointers with points to compute, negative counts),
 * IWF_ERR_NONFINITE (origin or step). No points: a no-op.
 */
iwf_status iwf_evaluate_grid(iwf_plan* plan, const void* coef, const double* origin,
                             const double* step, const int* count, void* u, void* stream);

/*
 * Normalises a physical-space field in place as the eigenfunction metrics of Sec. 4.2 do:
 * u <- u / u(xi*), xi* the first point of largest |u|, so that max|u| = 1 and u is real and
 * positive at xi* (the paper divides by the maximal modulus and leaves the phase free; fixing
 * it there is this library's reading). |u|^2 is formed with each product and the sum rounded
 * separately, so xi* is the same on any IEEE implementation; NaN points are never chosen; a
 * field that is zero everywhere is left unchanged.
 * To compare two fields (E_f), normalise both at one point: pass the reference's xi* as `at`.
 * For an even real potential u(-x) = conj(u(x)), so mirror points tie in modulus exactly and
 * fields normalised at different twins differ by a phase factor.
 *   u       device, M complex double, in place
 *   at      index of xi* to use, or -1 to search for the first point of largest |u|
 *   rho     device, M doubles: the density |u|^2 after normalisation, or NULL
 *   argmax  device, one long long: the index of xi* (-1 if no point qualified), or NULL
 * Uses four words of plan-owned scratch: calls on one plan that overlap on the GPU race.
 * Enqueues on `stream`; M = 0 is a no-op; M < 0, at >= M or u == NULL gives IWF_ERR_ARG.
 */
iwf_status iwf_field_normalize(iwf_plan* plan, void* u, long long M, long long at, double* rho,
                               long long* argmax, void* stream);

/*
 * E_f = max_m |u_m - v_m| of two fields of M complex doubles (Sec. 4.2), written to `dist`
 * (device, one double; 0 for M = 0, when u and v may be NULL). The square root is taken once,
 * of the largest |u - v|^2. Same scratch and stream rules as iwf_field_normalize; M < 0 or a
 * NULL dist gives IWF_ERR_ARG.
 */
iwf_status iwf_field_distance(iwf_plan* plan, const void* u, const void* v, long long M,
                              double* dist, void* stream);

/*
 * H~ psi by direct convolution instead of the FFT passes: Lambda psi + sum_m Vg_m psi(k* - m),
 * the cyclic convolution on the K* grid with the potential's folded modes that F V F^{-1}
 * equals (Sec. 3.3, Sec. 4.1, App. C). An ablation for potentials with few modes (at most
 * 256 folded modes, else IWF_ERR_UNSUPPORTED; fastest k_I axis at most 32): its cost per
 * point grows with the number of modes, the FFT passes' does not. Same arguments, layout and
 * results (up to rounding) as iwf_apply; enqueues on `stream`.
 */
iwf_status iwf_apply_stencil(iwf_plan* plan, int precision, const void* psi, void* hpsi,
                             int nvec, void* stream);

/*
 * Apply kernels. Both compute the same three passes (Sec. 4.1); they differ in how a pass
 * moves data:
 *   IWF_PATH_TILED   stages shared-memory tiles and runs every axis of a group on them; any
 *                    geometry (every supported axis length);
 *   IWF_PATH_PENCIL  keeps one pencil per thread in registers, loaded from and stored to
 *                    global memory directly, with one shared-memory transpose per pass;
 *                    needs n = 4, d = 2 with 2K_1 = 2K_2 and 2L_1 = 2L_2, each 16 or 32;
 *   IWF_PATH_AUTO    the pencil path where the geometry allows it, else the tiled path.
 */
enum { IWF_PATH_AUTO = 0, IWF_PATH_TILED = 1, IWF_PATH_PENCIL = 2 };

/*
 * Apply schedule autotuner. Times iwf_apply on an nvec block (scratch buffers allocated and
 * freed by the call) for every candidate schedule and keeps the fastest for this plan and
 * precision. Candidates: the tiled path with threads per CTA {128, 256}, shared-memory tile
 * budget {24, 48, 96, 160} KB and L2 chunk of vectors between passes {24, 48, 96} MB; where
 * the geometry allows it, the pencil path with chunks {12, 24, 48, 96} MB. Host outputs
 * (may be NULL): *best_ms per apply, best[3] = {threads, tile_kb, chunk_mb} (threads and
 * tile_kb are 0 when the pencil path won; iwf_plan_get_schedule reports the path). Needs a
 * potential. Results are identical for every schedule up to floating-point summation order;
 * synchronises.
 */
iwf_status iwf_plan_autotune(iwf_plan* plan, int precision, int nvec, double* best_ms,
                             int* best, void* stream);

/* Set the apply schedule directly (threads 128 or 256, tile_kb 8..200, chunk_mb >= 1). The
 * threads and tile budget are used by the tiled path, the chunk by both; the path is kept. */
iwf_status iwf_plan_set_schedule(iwf_plan* plan, int precision, int threads, int tile_kb,
                                 int chunk_mb);

/* Choose the apply kernels (IWF_PATH_*). IWF_PATH_PENCIL on a geometry it does not cover
 * returns IWF_ERR_UNSUPPORTED and leaves the plan unchanged. */
iwf_status iwf_plan_set_path(iwf_plan* plan, int precision, int path);

/*
 * Arithmetic of the DFTs of an FP64 (complex double) apply on the pencil path:
 *   IWF_ARITH_F64  FP64 (the default);
 *   IWF_ARITH_DF   double-float on the FP32 pipes: each value h + l of two floats (about
 *                  48 significant bits), split from and joined back to FP64 in integer
 *                  arithmetic at the pass boundaries. Storage, the potential tables and the
 *                  kinetic term Lambda psi stay FP64; the DFTs' errors grow from about 2^-53
 *                  to about 2^-45 of the vector's norm. On this GPU FP64 issues at 1/64 of
 *                  the FP32 rate, which bounds the FP64 passes.
 * Applies to iwf_apply, iwf_apply_host, iwf_apply_noalloc and the eigensolvers' complex-
 * double phase on this plan. IWF_ARITH_DF on a geometry without the pencil path, or with
 * the path set to IWF_PATH_TILED, returns IWF_ERR_UNSUPPORTED (the tiled kernels compute in
 * FP64). Library extension: the paper's FFTs are FP64 (MATLAB).
 */
enum { IWF_ARITH_F64 = 0, IWF_ARITH_DF = 1 };
iwf_status iwf_plan_set_arith(iwf_plan* plan, int arith);

/* The schedule iwf_apply will use: sched[4] = {threads, tile_kb, chunk_mb, path}, path
 * being IWF_PATH_TILED or IWF_PATH_PENCIL (IWF_PATH_AUTO resolved for this geometry). */
iwf_status iwf_plan_get_schedule(const iwf_plan* plan, int precision, int* sched);

/* Number of kernels this library has launched in this process (all devices, all plans). */
long long iwf_kernel_launches(void);

/*
 * iwf_apply without any device allocation. The paper has no counterpart: this entry point
 * exists for callers that must not allocate device memory while they run -- for example a
 * program whose device memory belongs to a pool or framework allocator that forbids direct
 * cudaMalloc/cudaFree, or a latency-critical loop where the implicit device
 * synchronisation of cudaMalloc/cudaFree would stall other work. iwf_apply may grow the
 * plan's workspace on a call with a larger block; this call never does.
 *   Same arguments, layout and result as iwf_apply.
 *   Scratch: the block between the passes lives in a fixed 32 MiB array compiled into the
 *   library (every GPU that loads the library holds it until the process exits). One
 *   vector must fit: N * 16 bytes (IWF_PREC_F64) or N * 8 bytes (IWF_PREC_C64) at most
 *   33554432; larger plans return IWF_ERR_UNSUPPORTED with the sizes in the message.
 *   Blocks are processed a chunk of vectors at a time; nothing in the array needs to start
 *   at zero, and each call overwrites what the previous one left there.
 *   The first call on a device looks up the array's device address (no allocation); make
 *   that first call before starting any stream capture on that device.
 *   All calls share the one array: calls whose GPU work overlaps (different streams, or
 *   different host threads, without ordering between them) race and give wrong results.
 *   Order them on one stream or with events.
 * Errors: as iwf_apply, plus IWF_ERR_UNSUPPORTED for a plan too large for the array.
 */
iwf_status iwf_apply_noalloc(iwf_plan* plan, int precision, const void* psi, void* hpsi,
                             int nvec, void* stream);

/*
 * Device-side failures of the apply. The pipelined pass C (complex-float pencil path) waits on
 * its bulk copies with bounded waits; a wait that runs out records IWF_ERR_TIMEOUT in the
 * plan's device error word and the kernel returns without storing the rest of H~ psi
 * (failure detection; the paper has no counterpart). iwf_apply and
 * iwf_apply_noalloc only enqueue work, so they cannot see the word; it is read and cleared at
 * the plan's next synchronisation point: iwf_apply_host, iwf_apply_profile, iwf_eigensolve
 * and iwf_batch_eigensolve (every iteration), or this call.
 * iwf_plan_check synchronises `stream` and returns IWF_ERR_TIMEOUT (clearing the word) when
 * an apply on the plan gave up waiting since the last check, IWF_OK otherwise.
 */
iwf_status iwf_plan_check(iwf_plan* plan, void* stream);

/*
 * Bound on the main waits of the plan's pipelined passes, in try_wait rounds (rounds < 0: the
 * default of 2^20, far above any real copy latency). A fault-injection knob for tests: with 0
 * every pipelined pass gives up at its first wait, so the apply reports IWF_ERR_TIMEOUT at the
 * next check. The drain of copies already in flight keeps the default bound, so the kernel
 * still lets them land before it exits.
 */
iwf_status iwf_plan_set_wait_limit(iwf_plan* plan, long long rounds);

/*
 * The tall-skinny contractions of the eigensolver's Rayleigh-Ritz step (Sec. 4.1, Alg. 2 in
 * block form: the Gram matrices S^H S and S^H H S and the updates X <- S C), exposed for
 * direct use, testing and measurement. Engines:
 *   IWF_CONTRACT_TENSOR  tcgen05 tensor cores, Ozaki scheme I: every FP64 value becomes the
 *                        integer round(v 2^(48-E)) under a power-of-two scale 2^E shared by
 *                        its group (a column for iwf_gram, a row of S and a column of C for
 *                        iwf_block_update), written as seven balanced 7-bit digits stored as
 *                        bf16; digit pairs of one level are summed exactly in fp32 tensor
 *                        memory (levels 2..6; 7..9 share one accumulator; pairs above 9 are
 *                        dropped). Error about 2^-49 of the product of the two scales per
 *                        term, random in sign.
 *   IWF_CONTRACT_DF      double-float arithmetic on the FP32 pipes (about 48 bits).
 *   IWF_CONTRACT_F64     FP64 arithmetic.
 * Matrices: A (nrows x ma), B (nrows x mb), S (nrows x m) and Y (nrows x q) are device,
 * complex double, column-major with leading dimension nrows; G (ma x mb) and C (m x q) are
 * device, complex double, row-major. ma, mb, m <= 72, q <= 24, nrows >= 1.
 * Each call allocates and frees its scratch (a few MB) and synchronises `stream`.
 * Errors: IWF_ERR_ARG (shape, NULL), IWF_ERR_ALLOC, IWF_ERR_CUDA, IWF_ERR_TIMEOUT (a bounded
 * wait of the tensor-core pipeline ran out).
 */
enum { IWF_CONTRACT_TENSOR = 0, IWF_CONTRACT_DF = 1, IWF_CONTRACT_F64 = 2 };
/* G = A^H B. */
iwf_status iwf_gram(int engine, long long nrows, const void* A, int ma, const void* B, int mb,
                    void* G, int device, void* stream);
/* Y = S C, or Y = Y - S C when subtract != 0 (Y must not overlap S). */
iwf_status iwf_block_update(int engine, long long nrows, const void* S, int m, const void* C,
                            int q, void* Y, int subtract, int device, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* IWFPM_H */
