// FP64-accurate tall-skinny contractions of the eigensolver on the tcgen05 tensor cores
// (Ozaki scheme I with fixed-point bf16 slices):
//   Gram   G = A^H B      (A: N x ma, B: N x mb complex double, contraction over N rows)
//   update Y = S C        (S: N x m, C: m x q complex double, contraction over m)
// These are the dense contractions of the Rayleigh-Ritz step of LOBPCG (Sec. 4.1, Alg. 2
// in block form).
//
// Slicing. Every value v of a group that shares one scale 2^E (a column of a Gram operand,
// a row of an update operand; |v| < 2^E) becomes the 56-bit integer I = round(v 2^(55-E)),
// written in balanced base-128 digits I = sum_k d_k 2^(56-7k), k = 1..8, |d_k| <= 64. Digit k
// is stored as the bf16 value D_k = d_k 2^(-7(k-1)) (exact: at most 7 significant bits), so
// v = 2^(E-6) sum_k D_k. A product of two values expands into digit pairs (k, l); pairs of one
// level k + l are integer multiples of one unit 2^(-7(k+l-2)). The tensor core multiplies
// bf16 pairs exactly and adds them in fp32; with |d| <= 64 a level's sum over a bounded
// number of rows stays below 2^24 units, so levels 2..6 are exact in their fp32 accumulators
// in tensor memory (one per level), and the rounding of levels 7..10 sits below 2^-56 of the
// scales' product. Pairs with k + l >= 11 are dropped (below 2^-62). The one rounding that
// matters is that of v to I: 2^-56 of the group's scale. Exact level sums are moved into
// double-float registers (Gram: every few hundred rows) or assembled into FP64 (update).
// Fifty-six bits rather than the fifty-three of FP64: a scale is the largest magnitude of a
// whole column or row, and H~ amplifies the high-frequency rows of H~W, so errors relative
// to the scales must sit well below the FP64 rounding of the entries that matter.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "blockops.cuh"
#include "common.cuh"
#include "tc.cuh"

namespace iwf {

namespace {

constexpr int kDig = 8;                 // digits per value
constexpr int kMaxLvl = 10;             // pairs k + l <= 10
constexpr long long kTcSpin = 1LL << 22;  // bounded mbarrier waits (try_wait rounds)
constexpr int kErrTimeout = 1;
constexpr int kSmemCap = 227 * 1024 - 2048;  // dynamic shared memory per CTA (227 KB less the
                                              // kernels' static shared memory)

// Balanced base-128 digits of round(v 2^(55-E)), where the group's largest biased exponent is
// maxb (E = maxb - 1022, so |v| < 2^E), as the bit patterns of the floats
// D_k = d_k 2^(-7(k-1)), |d_k| <= 64 (at most 7 significant bits: the top half is bf16).
// The scaling is an integer add to v's exponent field and the rounding one hardware
// conversion to a 64-bit integer (measured faster here than a rounded shift of the mantissa in
// 64-bit integer arithmetic, with either the tensor-core issue or the slicing as the
// bottleneck); the digits then come from two 28-bit halves in 32-bit arithmetic.
// Zeros, denormals and values below 2^(E-56) give zero digits.
__device__ __forceinline__ void digits8(double v, int maxb, uint32_t (&f)[kDig]) {
  const long long bits = __double_as_longlong(v);
  const int hi = (int)(bits >> 32);
  const int e = (hi >> 20) & 0x7FF;
  const int sh = 1077 - maxb;                     // v 2^(55-E) = v 2^(sh)
  long long I = 0;
  if (e != 0 && e + sh > 0)
    I = __double2ll_rn(__hiloint2double(hi + (sh << 20), (int)bits));
  // I = q 2^28 + r with r in [-2^27, 2^27)
  const int r0 = ((int)((unsigned int)I << 4)) >> 4;
  int q = (int)((I - r0) >> 28);
  int r = r0;
  int d[kDig];
  d[0] = (q + (1 << 20)) >> 21; q -= d[0] << 21;
  d[1] = (q + (1 << 13)) >> 14; q -= d[1] << 14;
  d[2] = (q + (1 << 6)) >> 7;   q -= d[2] << 7;
  d[3] = q;
  d[4] = (r + (1 << 20)) >> 21; r -= d[4] << 21;
  d[5] = (r + (1 << 13)) >> 14; r -= d[5] << 14;
  d[6] = (r + (1 << 6)) >> 7;   r -= d[6] << 7;
  d[7] = r;
  // d 2^(-7k) exactly: add d to the bits of m = 1.5 2^(23-7k) (whose last place is 2^(-7k)),
  // then subtract m
#pragma unroll
  for (int k = 0; k < kDig; ++k) {
    const float m = __int_as_float(((150 - 7 * k) << 23) | 0x400000);
    f[k] = __float_as_uint(__int_as_float(__float_as_int(m) + d[k]) - m);
  }
}

__device__ __forceinline__ uint32_t pack2(uint32_t lo, uint32_t hi) {
  return __byte_perm(lo, hi, 0x7632);
}

// Digits of 8 consecutive values of one group, written as the 16-byte K-row of one tile row
// in each of the digit tiles (tile k at base + k * tile_stride).
__device__ __forceinline__ void store_digits8(const double (&v)[8], int maxb, unsigned char* base,
                                              uint32_t tile_stride, uint32_t off) {
  uint32_t w[kDig][4];
#pragma unroll
  for (int j = 0; j < 8; j += 2) {
    uint32_t a[kDig], b[kDig];
    digits8(v[j], maxb, a);
    digits8(v[j + 1], maxb, b);
#pragma unroll
    for (int k = 0; k < kDig; ++k) w[k][j / 2] = pack2(a[k], b[k]);
  }
#pragma unroll
  for (int k = 0; k < kDig; ++k)
    *reinterpret_cast<uint4*>(base + (size_t)k * tile_stride + off) =
        make_uint4(w[k][0], w[k][1], w[k][2], w[k][3]);
}

using tc::tile_off;

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ bool wait_bounded(uint32_t bar, uint32_t parity) {
  for (long long r = 0; r < kTcSpin; ++r)
    if (tc::bar_try_wait(bar, parity)) return true;
  return false;
}
// The same for waits that usually last many microseconds (the accumulator hand-over): the
// warp sleeps between polls instead of taking issue slots from the slicing warps. Bounded by
// the same number of polls (about a second at the 256 ns sleep).
__device__ __forceinline__ bool wait_bounded_sleep(uint32_t bar, uint32_t parity) {
  for (long long r = 0; r < kTcSpin; ++r) {
    if (tc::bar_try_wait(bar, parity)) return true;
    __nanosleep(256);
  }
  return false;
}

// 16-byte asynchronous global -> shared copy; src_bytes = 0 fills zeros (src is not read).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
               "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait1() {
  asm volatile("cp.async.wait_group 1;" ::: "memory");
}

__host__ __device__ constexpr int round8(int x) { return (x + 7) & ~7; }


// The MMAs of one K16 step, for A digits k and runs of B digits l0..l0+n-1 (consecutive levels
// k + l, whose accumulators sit next to each other): entry = A tile index k - 1, B tile
// index l0 - 1, first accumulator k + l0 - 2, run length n, and whether the run's
// accumulators already hold partial sums. The plan of the first step of an accumulation
// (every accumulator fresh) differs from that of any later step. A run covers at most
// max_cat B digits (N = n NMMA <= 256). Built at compile time.
struct MmaStep { uint8_t a, b, acc, n, add; };
constexpr int kMaxPlan = 24;
struct MmaPlan { MmaStep s[kMaxPlan]; int n; };
__host__ __device__ constexpr MmaPlan make_plan(bool first, int max_cat) {
  MmaPlan P{};
  uint32_t started = first ? 0u : 0xFFFFFFFFu;
  int cnt = 0;
  for (int k = 1; k <= kDig; ++k) {
    const int lmax = (kDig < kMaxLvl - k) ? kDig : kMaxLvl - k;
    int l = 1;
    while (l <= lmax) {
      const int l0 = l;
      const uint32_t st0 = (started >> (k + l0 - 2)) & 1u;
      while (l <= lmax && l - l0 < max_cat && ((started >> (k + l - 2)) & 1u) == st0) ++l;
      const int n = l - l0;
      P.s[cnt].a = (uint8_t)(k - 1);
      P.s[cnt].b = (uint8_t)(l0 - 1);
      P.s[cnt].acc = (uint8_t)(k + l0 - 2);
      P.s[cnt].n = (uint8_t)n;
      P.s[cnt].add = (uint8_t)st0;
      ++cnt;
      started |= ((1u << n) - 1u) << (k + l0 - 2);
    }
  }
  P.n = cnt;
  return P;
}
template <int NMMA> constexpr int max_cat() { return 256 / NMMA < kDig ? 256 / NMMA : kDig; }
static_assert(make_plan(true, 5).n <= kMaxPlan && make_plan(false, 5).n <= kMaxPlan &&
                  make_plan(true, 8).n <= kMaxPlan && make_plan(false, 8).n <= kMaxPlan,
              "plan size");

// The MMAs of one K16 step, unrolled at compile time from the plan: A digit tiles every
// a_unit * 16 bytes from dA, B digit tiles of NMMA rows from dB, accumulators NMMA columns
// apart from tmem.
template <int NMMA, bool FIRST, int I = 0>
__device__ __forceinline__ void issue_plan(uint32_t tmem, uint64_t dA, uint64_t dB, uint32_t a_unit) {
  constexpr MmaPlan P = make_plan(FIRST, max_cat<NMMA>());
  if constexpr (I < P.n) {
    constexpr MmaStep m = P.s[I];
    tc::mma_bf16(tmem + (uint32_t)(m.acc * NMMA), dA + (uint64_t)(m.a * a_unit),
                 dB + (uint64_t)((m.b * NMMA * tc::kTileRowBytes) >> 4),
                 tc::idesc_bf16(128, m.n * NMMA, false), m.add != 0);
    issue_plan<NMMA, FIRST, I + 1>(tmem, dA, dB, a_unit);
  }
}

// ---------------------------------------------------------------------------------------
// Column scales of both Gram operands: exps[c] (c < ma: column c of A) and
// exps[kMaxSmall + c] (column c of B) = largest biased FP64 exponent over the re and im parts
// of the column (2047 when it holds an Inf or NaN, 0 for a zero column). With same = 1 (A and
// B are one block list) only A is read and both slots are written. exps must start at 0.
__global__ void colexp_kernel(Batch bt, BlockList A, BlockList B, int ma, int same, long long N,
                              int* exps) {
  const int prob = blockIdx.z, c = blockIdx.y;
  if (bt.active && !bt.active[prob]) return;
  const bool isA = c < ma;
  const int cc = isA ? c : c - ma;
  const void* base = isA ? A.p[cc / A.b] : B.p[cc / B.b];
  const double2* col = reinterpret_cast<const double2*>(base) + (size_t)prob * bt.pstride +
                       (size_t)(cc % (isA ? A.b : B.b)) * N;
  unsigned int m = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 v = col[i];
    const unsigned int hx = (unsigned int)(__double_as_longlong(v.x) >> 32);
    const unsigned int hy = (unsigned int)(__double_as_longlong(v.y) >> 32);
    m = max(m, max((hx >> 20) & 0x7FFu, (hy >> 20) & 0x7FFu));
  }
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m) {
    int* e = exps + (size_t)prob * 2 * kMaxSmall;
    atomicMax(e + (isA ? cc : kMaxSmall + cc), (int)m);
    if (same) atomicMax(e + kMaxSmall + cc, (int)m);
  }
}

// ---------------------------------------------------------------------------------------
// Gram kernel. The product is cut into sub-Grams of at most 48 A columns and 24 B columns,
// D = [Ar; Ai]^T [Br, Bi] (M = 2na <= 96 lanes, N = 2nb <= 48 columns per level), one per
// blockIdx.z; for a Hermitian product the sub-Grams below the block diagonal are skipped and
// mirrored by the reduction. Each level 2..10 has its own accumulator (N columns apart in
// tensor memory), so for one A digit k the B digits l of consecutive levels k + l sit next
// to each other along N and one MMA covers up to 256 / N of them.
// Roles: warps 0..7 slice 16-row stages of A and B into the digit tiles (the FP64 rows of
// the next stage are already on their way into a staging buffer by cp.async); warp 8 issues
// the MMAs; warps 9..16 move the level accumulators into double-float running sums every
// 512 rows and write the CTA's partial at the end.
// A tiles hold only the rows in use (rounded to 8); the MMA (M = 128) reads on into the
// following tiles, whose values land in accumulator lanes nobody reads.
constexpr int kProdWarps = 10, kEpiWarps = 8;
constexpr int kGramThreads = (kProdWarps + 1 + kEpiWarps) * 32;
constexpr int kMaxStages = 4;
constexpr int kStageRows = 32;           // rows per stage: two K16 steps
constexpr int kGuard = 4096;             // tail room for the MMAs' reads past the last tile
constexpr int kNumLvl = kMaxLvl - 1;     // accumulators, levels 2..10
constexpr int kChunkRows = 512;          // a level sum over 512 rows stays below 2^24 units
constexpr int kMaxSub = 12;
static_assert((kStageRows / 8) * (48 + 24) <= kProdWarps * 32, "one staging item per producer thread");

struct SubGram { int a0, na, b0, nb, poff; };
struct SubList {
  SubGram s[kMaxSub];
  int n;
  int slot_size;        // doubles of one slot's partials, over all sub-Grams
  int herm;
};

template <int NMMA>
struct GramLayout {
  int rowsA, rowsB, tileA, stage, items, staging;
  __host__ __device__ GramLayout(int na, int nb) {
    rowsA = 2 * na;
    rowsB = 2 * nb;
    tileA = round8(rowsA) * tc::kTileRowBytes;
    // [A tiles: K16 step t, digit k][B tiles: t, digit l]
    stage = (kStageRows / 16) * kDig * (tileA + NMMA * tc::kTileRowBytes);
    items = (kStageRows / 8) * (na + nb);   // (column, 8-row group)
    staging = items * 128;
  }
  __host__ __device__ int smem(int S) const { return S * stage + 2 * staging + kGuard; }
};

template <int NMMA>
__global__ void __launch_bounds__(kGramThreads, 1)
gram_tc_kernel(Batch bt, BlockList A, BlockList B, long long N, long long rows_per_slot, int S,
               SubList subs, double* partial, int* err) {
  constexpr int kTileB = NMMA * tc::kTileRowBytes;
  const int prob = blockIdx.y, slot = blockIdx.x, sub = blockIdx.z;
  if (bt.active && !bt.active[prob]) return;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) unsigned long long full_bar[kMaxStages], empty_bar[kMaxStages];
  __shared__ __align__(8) unsigned long long accf_bar, acce_bar, done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const SubGram sg = subs.s[sub];
  const int na = sg.na, nb = sg.nb;
  const GramLayout<NMMA> Lo(na, nb);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t poff = (size_t)prob * bt.pstride;
  const int* expA = bt.exps + (size_t)prob * 2 * kMaxSmall;
  const int* expB = expA + kMaxSmall;
  const long long r_begin = (long long)slot * rows_per_slot;
  const long long r_end = min(N, r_begin + rows_per_slot);
  const long long nrows = r_end > r_begin ? r_end - r_begin : 0;
  const int nstages = (int)((nrows + kStageRows - 1) / kStageRows);
  constexpr int kStagesPerChunk = kChunkRows / kStageRows;
  constexpr int kSteps = kStageRows / 16;
  __shared__ int sexpA[48], sexpB[24];
  for (int i = threadIdx.x; i < na; i += blockDim.x) sexpA[i] = expA[sg.a0 + i];
  for (int i = threadIdx.x; i < nb; i += blockDim.x) sexpB[i] = expB[sg.b0 + i];
  const int nchunks = (nstages + kStagesPerChunk - 1) / kStagesPerChunk;
  unsigned char* staging = smem + (size_t)S * Lo.stage;

  // zero the digit stages and the guard (B padding rows stay zero; reads past the tiles stay
  // inside the allocation), barriers, tensor memory
  for (int i = threadIdx.x; i < S * Lo.stage / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
  for (int i = threadIdx.x; i < kGuard / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(staging + 2 * Lo.staging)[i] = make_uint4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      tc::bar_init(tc::smem_u32(&full_bar[s]), kProdWarps * 32);
      tc::bar_init(tc::smem_u32(&empty_bar[s]), 1);
    }
    tc::bar_init(tc::smem_u32(&accf_bar), 1);
    tc::bar_init(tc::smem_u32(&acce_bar), kEpiWarps * 32);
    tc::bar_init(tc::smem_u32(&done_bar), 1);
    tc::bar_init_fence();
    abort_flag = 0;
  }
  if (warp == 0) {
    tc::tmem_alloc(tc::smem_u32(&tmem_base), 512);
    tc::tmem_relinquish();
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  volatile int* abort_v = &abort_flag;

  if (warp < kProdWarps) {
    // ---- producers: item = (column, 8-row group) of A or B, 8 rows x (re, im); thread tid
    // owns item tid in every stage (items <= 4 (48 + 24) < kProdWarps * 32), so it only ever
    // reads the staging slots it filled itself. Staging is [row u][item], so that a warp's
    // reads are consecutive. Item it: K half h = it & 1, column cc = (it >> 1) % ncols, K16
    // step t = (it >> 1) / ncols, so that a warp's tile stores cover whole 256-byte atoms of
    // one step ----
    const int it = threadIdx.x;
    const int ncols = na + nb;
    const bool has = it < Lo.items;
    const int cc = (it >> 1) % ncols;
    const int grp = 2 * ((it >> 1) / ncols) + (it & 1), t = grp >> 1, h = grp & 1;
    const bool isA = cc < na;
    const int c = isA ? cc : cc - na;
    const int gcol = isA ? sg.a0 + c : sg.b0 + c;
    const double2* col = nullptr;
    if (has) {
      const void* gbase = isA ? A.p[gcol / A.b] : B.p[gcol / B.b];
      col = reinterpret_cast<const double2*>(gbase) + poff + (size_t)(gcol % (isA ? A.b : B.b)) * N;
    }
    const int maxb = has ? (isA ? sexpA[c] : sexpB[c]) : 0;
    const uint32_t tstride = isA ? (uint32_t)Lo.tileA : (uint32_t)kTileB;
    // byte offsets of this item's re and im rows inside the step-t digit tiles of a stage
    const size_t tbase = isA ? (size_t)t * kDig * Lo.tileA
                             : (size_t)kSteps * kDig * Lo.tileA + (size_t)t * kDig * kTileB;
    const uint32_t off_re = tile_off(c, h), off_im = tile_off(c + (isA ? na : nb), h);
    const uint32_t stg = tc::smem_u32(staging) + (uint32_t)it * 16;
    const auto issue = [&](int j) {
      if (has) {
        const uint32_t dst = stg + (uint32_t)((j & 1) * Lo.staging);
        const long long r0 = r_begin + (long long)kStageRows * j + 8 * grp;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const long long r = r0 + u;
          const bool in = r < r_end;
          cp_async16(dst + (uint32_t)(u * Lo.items * 16), col + (in ? r : r_begin), in ? 16 : 0);
        }
      }
      cp_async_commit();
    };
    if (nstages > 0) issue(0);
    for (int j = 0; j < nstages; ++j) {
      const int st = j % S;
      if (j + 1 < nstages) issue(j + 1);
      else cp_async_commit();                      // an empty group keeps the count uniform
      cp_async_wait1();                            // this thread's copies of stage j landed
      if (!wait_bounded(tc::smem_u32(&empty_bar[st]), (uint32_t)(((j / S) & 1) ^ 1))) {
        atomicExch(&abort_flag, 1);
        break;
      }
      if (*abort_v) break;
      if (has) {
        const double2* sv =
            reinterpret_cast<const double2*>(staging + (size_t)(j & 1) * Lo.staging) + it;
        double re[8], im[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) { const double2 v = sv[u * Lo.items]; re[u] = v.x; im[u] = v.y; }
        unsigned char* tb = smem + (size_t)st * Lo.stage + tbase;
        store_digits8(re, maxb, tb, tstride, off_re);
        store_digits8(im, maxb, tb, tstride, off_im);
      }
      tc::fence_async_smem();
      tc::bar_arrive(tc::smem_u32(&full_bar[st]));
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else if (warp == kProdWarps) {
    // ---- MMA issuer: the compile-time plan of each K16 step ----
    if (lane == 0) {
      const uint32_t a_unit = (uint32_t)Lo.tileA >> 4;
      for (int j = 0; j < nstages && !*abort_v; ++j) {
        const int st = j % S;
        const int chunk = j / kStagesPerChunk;
        const bool fresh = j % kStagesPerChunk == 0;
        if (fresh && chunk > 0 &&
            !wait_bounded(tc::smem_u32(&acce_bar), (uint32_t)((chunk - 1) & 1))) {
          atomicExch(&abort_flag, 1);
          break;
        }
        if (!wait_bounded(tc::smem_u32(&full_bar[st]), (uint32_t)((j / S) & 1))) {
          atomicExch(&abort_flag, 1);
          break;
        }
        tc::fence_after_sync();
        const uint32_t aBase = tc::smem_u32(smem + (size_t)st * Lo.stage);
        const uint32_t bBase = aBase + kSteps * kDig * Lo.tileA;
#pragma unroll
        for (int t = 0; t < kSteps; ++t) {
          const uint64_t dA = tc::sdesc(aBase + t * kDig * Lo.tileA);
          const uint64_t dB = tc::sdesc(bBase + t * kDig * kTileB);
          if (fresh && t == 0) issue_plan<NMMA, true>(tmem, dA, dB, a_unit);
          else issue_plan<NMMA, false>(tmem, dA, dB, a_unit);
        }
        tc::mma_commit(tc::smem_u32(&empty_bar[st]));
        if (j % kStagesPerChunk == kStagesPerChunk - 1 || j == nstages - 1)
          tc::mma_commit(tc::smem_u32(&accf_bar));
      }
      // every MMA issued has completed before the kernel releases tensor memory
      tc::mma_commit(tc::smem_u32(&done_bar));
      wait_bounded(tc::smem_u32(&done_bar), 0);
    }
    __syncwarp();
  } else {
    // ---- epilogue: level accumulators -> double-float running sums ----
    const int e = warp - kProdWarps - 1;            // 0..7
    const int q = warp & 3;                         // TMEM lane quarter of this warp
    const int half = e >= 4 ? 1 : 0;
    constexpr int G = NMMA / 8;                     // 8-column groups
    constexpr int GH = (G + 1) / 2;
    const int g0 = half ? GH : 0, g1 = half ? G : GH;
    const int lane_row = 32 * q + lane;             // accumulator row
    float hi[GH * 8], lo[GH * 8];
#pragma unroll
    for (int i = 0; i < GH * 8; ++i) { hi[i] = 0.f; lo[i] = 0.f; }
    const bool live = 32 * q < Lo.rowsA;            // lanes beyond 2na hold garbage
    for (int c = 0; c < nchunks && !*abort_v; ++c) {
      if (!wait_bounded_sleep(tc::smem_u32(&accf_bar), (uint32_t)(c & 1))) {
        atomicExch(&abort_flag, 1);
        break;
      }
      tc::fence_after_sync();
      if (live) {
#pragma unroll
        for (int gi = 0; gi < GH; ++gi) {
          const int g = g0 + gi;
          if (g < g1) {
#pragma unroll
            for (int a = 0; a < kNumLvl; ++a) {
              float v[8];
              tc::tmem_ld8(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(a * NMMA + 8 * g), v);
              tc::tmem_wait_ld();
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                float s, er;
                two_sum(hi[gi * 8 + u], v[u], s, er);
                hi[gi * 8 + u] = s;
                lo[gi * 8 + u] += er;
              }
            }
          }
        }
      }
      tc::fence_before_sync();
      tc::bar_arrive(tc::smem_u32(&acce_bar));
    }
    // partial of this CTA and sub-Gram: rows 2na x cols 2nb
    const int Ncols = Lo.rowsB;
    double* out = partial + ((size_t)prob * gridDim.x + slot) * subs.slot_size + sg.poff;
    if (lane_row < Lo.rowsA) {
#pragma unroll
      for (int gi = 0; gi < GH; ++gi) {
        const int g = g0 + gi;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int col = 8 * g + u;
          if (g < g1 && col < Ncols)
            out[(size_t)lane_row * Ncols + col] = (double)hi[gi * 8 + u] + (double)lo[gi * 8 + u];
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (*abort_v && threadIdx.x == 0) atomicExch(err, kErrTimeout);
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, 512);
  }
}

// G[prob] (ma x mb, row-major, complex double at out + prob * kCapG) from the slot partials of
// the sub-Grams, with the column scales 2^(Ea + Eb - 12), E = maxb - 1022. An entry of a
// skipped (Hermitian) block is the conjugate of its mirror image.
__global__ void gram_tc_reduce(Batch bt, const double* partial, int slots, int ma, int mb,
                               SubList subs, double2* out) {
  const int prob = blockIdx.y;
  if (bt.active && !bt.active[prob]) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ma * mb) return;
  int a = e / mb, b = e % mb;
  int si = -1;
  bool mirror = false;
  for (int t = 0; t < subs.n && si < 0; ++t) {
    const SubGram& g = subs.s[t];
    if (a >= g.a0 && a < g.a0 + g.na && b >= g.b0 && b < g.b0 + g.nb) si = t;
  }
  if (si < 0 && subs.herm) {
    for (int t = 0; t < subs.n && si < 0; ++t) {
      const SubGram& g = subs.s[t];
      if (b >= g.a0 && b < g.a0 + g.na && a >= g.b0 && a < g.b0 + g.nb) si = t;
    }
    mirror = true;
    const int tmp = a; a = b; b = tmp;
  }
  double2 r = make_double2(nan(""), nan(""));
  if (si >= 0) {
    const SubGram g = subs.s[si];
    const int ia = a - g.a0, ib = b - g.b0, Nc = 2 * g.nb;
    const double* p = partial + (size_t)prob * slots * subs.slot_size + g.poff;
    double re = 0.0, im = 0.0;
    for (int s = 0; s < slots; ++s, p += subs.slot_size) {
      re += p[(size_t)ia * Nc + ib] + p[(size_t)(ia + g.na) * Nc + ib + g.nb];
      im += p[(size_t)ia * Nc + ib + g.nb] - p[(size_t)(ia + g.na) * Nc + ib];
    }
    const int* expA = bt.exps + (size_t)prob * 2 * kMaxSmall;
    const int ea = expA[a], eb = expA[kMaxSmall + b];
    if (ea < 2047 && eb < 2047) {
      const double sc = ldexp(1.0, ea + eb - 2044 - 12);
      r = make_double2(re * sc, mirror ? -im * sc : im * sc);
    }
  }
  out[(size_t)prob * kCapG + e] = r;
}

// ---------------------------------------------------------------------------------------
// Update kernel: Y_o = S C_o (or Y_0 -= S C_0) for 128-row tiles of S. MMA M = 128 rows,
// N = 2q (row 2j of B gives Re Y_j, row 2j+1 Im Y_j), K = 2m with the re and im parts of each
// S column interleaved. Row scales of S come from a first pass over the tile (its data then
// sits in L2 for the second pass that slices it); column scales of C are computed once per
// CTA. One CTA per SM, persistent over tiles; blockIdx.x = 2 * slot + o for two outputs, so
// that the two CTAs reading one tile run side by side. Roles: warps 0..7 slice (K16 slices of
// 8 S columns into a 3-slot ring), warp 8 issues the MMAs, warps 9..12 assemble the FP64
// outputs from the level accumulators with integer arithmetic.
constexpr int kUpdProd = 8, kUpdEpi = 4;
constexpr int kUpdThreads = (kUpdProd + 1 + kUpdEpi) * 32;
constexpr int kUpdSlots = 3;
constexpr int kRxRing = 2;                               // row-scale buffers in flight
constexpr int kTileA = 128 * tc::kTileRowBytes;          // 4 KB: 128 rows x K16
constexpr int kUpdSliceBytes = kDig * kTileA;            // digit tiles of one K16 slice

template <int NMMA>
struct UpdCfg {
  static constexpr int kTileB = NMMA * tc::kTileRowBytes;
  static constexpr int kMaxSlices = kMaxSmall / 8;        // K = 2m <= 144
  static constexpr int kBBytes = kDig * kMaxSlices * kTileB;
  static constexpr int kSmem = kBBytes + kUpdSlots * kUpdSliceBytes + 1024;
};

// FP64 value of T * 2^(sh) for a 64-bit integer T (round to nearest; 0 below the normal range).
__device__ __forceinline__ double ll_to_double_scaled(long long T, int sh) {
  if (T == 0) return 0.0;
  const unsigned long long sign = T < 0 ? (1ull << 63) : 0ull;
  unsigned long long U = T < 0 ? (unsigned long long)(-T) : (unsigned long long)T;
  const int lz = __clzll((long long)U);
  int top = 63 - lz;                       // position of the leading one
  unsigned long long M;
  if (top > 52) {
    const int r = top - 52;
    M = (U + (1ull << (r - 1))) >> r;      // may carry into bit 53
    if (M >> 53) { M >>= 1; ++top; }
  } else {
    M = U << (52 - top);
  }
  const int e = top + sh + 1023;
  if (e <= 0) return 0.0;
  if (e >= 2047) return __longlong_as_double((long long)(sign | (0x7FFull << 52)));
  return __longlong_as_double((long long)(sign | ((unsigned long long)e << 52) |
                                          (M & 0xFFFFFFFFFFFFFull)));
}

// round(x * scale) for |x scale| < 2^22 (exact when x scale is an integer)
__device__ __forceinline__ int magic_int(float x, float scale) {
  return __float_as_int(fmaf(x, scale, 12582912.0f)) - 0x4B400000;
}

template <int NMMA, bool SUB>
__global__ void __launch_bounds__(kUpdThreads, 1)
update_tc_kernel(Batch bt, BlockList S, int m, long long N, const double2* C1, const double2* C2,
                 int cstride, int q, double2* out1, double2* out2, int nout, int* err) {
  using Cfg = UpdCfg<NMMA>;
  const int prob = blockIdx.y;
  if (bt.active && !bt.active[prob]) return;
  const int o = blockIdx.x % nout, slot = blockIdx.x / nout, nslots = gridDim.x / nout;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) unsigned long long full_bar[kUpdSlots], empty_bar[kUpdSlots];
  __shared__ __align__(8) unsigned long long accf_bar, acce_bar, done_bar;
  __shared__ __align__(8) unsigned long long rxf_bar[kRxRing], rxe_bar[kRxRing];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ int rowexp[kRxRing][128];
  __shared__ int colexpB[NMMA];
  __shared__ const double2* scol[kMaxSmall];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t poff = (size_t)prob * bt.pstride;
  const double2* C = (o == 0 ? C1 : C2) + (size_t)prob * cstride;
  double2* Y = (o == 0 ? out1 : out2) + poff;
  const int nsl = (m + 7) / 8;                  // K16 slices (8 S columns each)
  const long long ntiles = (N + 127) / 128;
  unsigned char* Bt = smem;                     // [slice][digit] B tiles
  unsigned char* ring = smem + Cfg::kBBytes;    // [slot][digit] A tiles

  // ---- set-up: column scales and digits of B (from C), barriers, tensor memory ----
  for (int i = threadIdx.x; i < (Cfg::kBBytes + kUpdSlots * kUpdSliceBytes) / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
  for (int n = threadIdx.x; n < NMMA; n += blockDim.x) {
    int mx = 0;
    if (n < 2 * q) {
      const int j = n >> 1;
      for (int c = 0; c < m; ++c) {
        const double2 v = C[(size_t)c * q + j];
        const unsigned int hx = (unsigned int)(__double_as_longlong(v.x) >> 32);
        const unsigned int hy = (unsigned int)(__double_as_longlong(v.y) >> 32);
        mx = max(mx, (int)max((hx >> 20) & 0x7FFu, (hy >> 20) & 0x7FFu));
      }
    }
    colexpB[n] = mx;
  }
  if (threadIdx.x == 0) {
    for (int sl = 0; sl < kUpdSlots; ++sl) {
      tc::bar_init(tc::smem_u32(&full_bar[sl]), kUpdProd * 32);
      tc::bar_init(tc::smem_u32(&empty_bar[sl]), 1);
    }
    tc::bar_init(tc::smem_u32(&accf_bar), 1);
    tc::bar_init(tc::smem_u32(&acce_bar), kUpdEpi * 32);
    tc::bar_init(tc::smem_u32(&done_bar), 1);
    for (int i = 0; i < kRxRing; ++i) {
      tc::bar_init(tc::smem_u32(&rxf_bar[i]), kUpdProd * 32);
      tc::bar_init(tc::smem_u32(&rxe_bar[i]), kUpdEpi * 32);
    }
    tc::bar_init_fence();
    abort_flag = 0;
  }
  // the base pointer of every S column (so that no thread indexes the parameter block)
  for (int c = threadIdx.x; c < m; c += blockDim.x)
    scol[c] = reinterpret_cast<const double2*>(S.p[c / S.b]) + poff + (size_t)(c % S.b) * N;
  __syncthreads();
  // B row n, K-elements 16 s + 8 h .. + 7 = S columns c = 8 s + 4 h + u (re, im interleaved):
  // row 2j:   Re Y_j = sum_c Re S_c Re C_cj - Im S_c Im C_cj
  // row 2j+1: Im Y_j = sum_c Re S_c Im C_cj + Im S_c Re C_cj
  for (int it = threadIdx.x; it < 2 * q * nsl * 2; it += blockDim.x) {
    const int h = it & 1, sl = (it >> 1) % nsl, n = (it >> 1) / nsl;
    const int j = n >> 1;
    double v[8];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = 8 * sl + 4 * h + u;
      double2 cv = make_double2(0.0, 0.0);
      if (c < m) cv = C[(size_t)c * q + j];
      if ((n & 1) == 0) { v[2 * u] = cv.x; v[2 * u + 1] = -cv.y; }
      else { v[2 * u] = cv.y; v[2 * u + 1] = cv.x; }
    }
    store_digits8(v, colexpB[n], Bt + (size_t)sl * kDig * Cfg::kTileB, Cfg::kTileB,
                  tile_off(n, h));
  }
  if (warp == 0) {
    tc::tmem_alloc(tc::smem_u32(&tmem_base), 512);
    tc::tmem_relinquish();
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  volatile int* abort_v = &abort_flag;

  if (warp < kUpdProd) {
    // ---- producers: thread (rho, hh) owns row rho of the tile and half of its columns;
    // both halves of a row sit in one warp, so the row's scale is a shuffle away ----
    const int rho = warp * 16 + (lane & 15), hh = lane >> 4;
    const auto ld = [&](int c, long long r) { return scol[c][r]; };
    int j = 0;                                  // slices produced so far (ring position)
    int tcount = 0;
    for (long long t = slot; t < ntiles && !*abort_v; t += nslots, ++tcount) {
      const long long r = t * 128 + rho;
      const bool live = r < N;
      // pass 1: this row's largest exponent over all of S's columns, eight loads in flight
      unsigned int mx = 0;
      if (live) {
        for (int c0 = hh; c0 < m; c0 += 16) {
          double2 v[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int c = c0 + 2 * u;
            v[u] = c < m ? ld(c, r) : make_double2(0.0, 0.0);
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const unsigned int hx = (unsigned int)(__double_as_longlong(v[u].x) >> 32);
            const unsigned int hy = (unsigned int)(__double_as_longlong(v[u].y) >> 32);
            mx = max(mx, max((hx >> 20) & 0x7FFu, (hy >> 20) & 0x7FFu));
          }
        }
      }
      mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 16));
      const int maxb = (int)mx;
      // the row scales travel to the epilogue through a ring of buffers
      const int rb = tcount % kRxRing;
      if (!wait_bounded(tc::smem_u32(&rxe_bar[rb]), (uint32_t)(((tcount / kRxRing) & 1) ^ 1))) {
        atomicExch(&abort_flag, 1);
        break;
      }
      if (hh == 0) rowexp[rb][rho] = maxb;
      tc::bar_arrive(tc::smem_u32(&rxf_bar[rb]));
      // pass 2: slices of 8 columns (this thread: 4 columns, re and im, of its row); the next
      // slice's values are loaded before this one is sliced
      double2 cur[4], nxt[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = 4 * hh + u;
        cur[u] = (live && c < m) ? ld(c, r) : make_double2(0.0, 0.0);
      }
      bool ok = true;
      for (int sl = 0; sl < nsl; ++sl, ++j) {
        const int st = j % kUpdSlots;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c = 8 * (sl + 1) + 4 * hh + u;
          nxt[u] = (live && c < m) ? ld(c, r) : make_double2(0.0, 0.0);
        }
        if (!wait_bounded(tc::smem_u32(&empty_bar[st]), (uint32_t)(((j / kUpdSlots) & 1) ^ 1))) {
          atomicExch(&abort_flag, 1);
          ok = false;
          break;
        }
        double v[8];
#pragma unroll
        for (int u = 0; u < 4; ++u) { v[2 * u] = cur[u].x; v[2 * u + 1] = cur[u].y; }
        store_digits8(v, maxb, ring + (size_t)st * kUpdSliceBytes, kTileA, tile_off(rho, hh));
        tc::fence_async_smem();
        tc::bar_arrive(tc::smem_u32(&full_bar[st]));
#pragma unroll
        for (int u = 0; u < 4; ++u) cur[u] = nxt[u];
      }
      if (!ok) break;
    }
  } else if (warp == kUpdProd) {
    // ---- MMA issuer ----
    if (lane == 0) {
      const uint32_t idn = tc::idesc_bf16(128, NMMA, false);
      int j = 0, tcount = 0;
      for (long long t = slot; t < ntiles && !*abort_v; t += nslots, ++tcount) {
        if (tcount > 0 &&
            !wait_bounded(tc::smem_u32(&acce_bar), (uint32_t)((tcount - 1) & 1))) {
          atomicExch(&abort_flag, 1);
          break;
        }
        bool ok = true;
        for (int sl = 0; sl < nsl; ++sl, ++j) {
          const int st = j % kUpdSlots;
          if (!wait_bounded(tc::smem_u32(&full_bar[st]), (uint32_t)((j / kUpdSlots) & 1))) {
            atomicExch(&abort_flag, 1);
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint64_t dA = tc::sdesc(tc::smem_u32(ring + (size_t)st * kUpdSliceBytes));
          const uint64_t dB = tc::sdesc(tc::smem_u32(Bt + (size_t)sl * kDig * Cfg::kTileB));
          if (sl == 0) issue_plan<NMMA, true>(tmem, dA, dB, (uint32_t)kTileA >> 4);
          else issue_plan<NMMA, false>(tmem, dA, dB, (uint32_t)kTileA >> 4);
          tc::mma_commit(tc::smem_u32(&empty_bar[st]));
        }
        if (!ok) break;
        tc::mma_commit(tc::smem_u32(&accf_bar));
      }
      tc::mma_commit(tc::smem_u32(&done_bar));
      wait_bounded(tc::smem_u32(&done_bar), 0);
    }
    __syncwarp();
  } else {
    // ---- epilogue: lanes are rows; FP64 assembly with integer arithmetic ----
    const int qd = warp & 3;
    const int rho = 32 * qd + lane;
    int tcount = 0;
    for (long long t = slot; t < ntiles && !*abort_v; t += nslots, ++tcount) {
      if (!wait_bounded_sleep(tc::smem_u32(&accf_bar), (uint32_t)(tcount & 1))) {
        atomicExch(&abort_flag, 1);
        break;
      }
      tc::fence_after_sync();
      const long long r = t * 128 + rho;
      const int rb = tcount % kRxRing;
      if (!wait_bounded(tc::smem_u32(&rxf_bar[rb]), (uint32_t)((tcount / kRxRing) & 1))) {
        atomicExch(&abort_flag, 1);
        break;
      }
      const int er = rowexp[rb][rho];
      tc::bar_arrive(tc::smem_u32(&rxe_bar[rb]));
      constexpr int G = NMMA / 8;
      for (int g = 0; g < G; ++g) {
        float a[kNumLvl][8];
#pragma unroll
        for (int ac = 0; ac < kNumLvl; ++ac)
          tc::tmem_ld8(tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(ac * NMMA + 8 * g), a[ac]);
        tc::tmem_wait_ld();
        if (g == G - 1) {
          tc::fence_before_sync();
          tc::bar_arrive(tc::smem_u32(&acce_bar));
        }
        // levels 7..10 together (their rounding sits far below the result's last bit)
#pragma unroll
        for (int u = 0; u < 8; ++u) a[5][u] = (a[5][u] + a[6][u]) + (a[7][u] + a[8][u]);
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
          const int jc = (8 * g + u) >> 1;       // complex output column
          if (jc >= q || r >= N) continue;
          double val[2];
#pragma unroll
          for (int w = 0; w < 2; ++w) {
            const int n = 8 * g + u + w;
            // Th = 2^28 x (levels 2..6): the level-l sum is an integer multiple of 2^(-7(l-2))
            // below 2^22 of its unit, so Th is exact (below 2^48). The shared levels 7..10 are
            // added at a finer unit 2^(-28-k), k as large as keeps the sum in 62 bits.
            const long long Th =
                ((long long)magic_int(a[0][u + w], 1.0f) << 28) +
                ((long long)magic_int(a[1][u + w], 128.0f) << 21) +
                ((long long)magic_int(a[2][u + w], 16384.0f) << 14) +
                ((long long)magic_int(a[3][u + w], 2097152.0f) << 7) +
                (long long)magic_int(a[4][u + w], 268435456.0f);
            const unsigned long long ua = Th < 0 ? (unsigned long long)(-Th) : (unsigned long long)Th;
            const int nb = 64 - __clzll((long long)ua);
            const int k = min(21, 62 - nb);
            const long long T = Th * (1LL << k) +
                                __float2ll_rn(a[5][u + w] * __int_as_float((127 + 28 + k) << 23));
            // value = T 2^(-28-k) 2^(Er + En - 12), E = maxb - 1022
            const int en = colexpB[n];
            val[w] = (er >= 2047 || en >= 2047)
                         ? nan("")
                         : ll_to_double_scaled(T, er + en - 2044 - 12 - 28 - k);
          }
          double2* dst = Y + (size_t)jc * N + r;
          if (SUB) {
            const double2 old = *dst;
            *dst = make_double2(old.x - val[0], old.y - val[1]);
          } else {
            *dst = make_double2(val[0], val[1]);
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (*abort_v && threadIdx.x == 0) atomicExch(err, kErrTimeout);
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, 512);
  }
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
      n = 152;
  }
  return n;
}

template <int NMMA>
iwf_status launch_gram_tc(const Batch& bt, const BlockList& A, const BlockList& B,
                          const SubList& subs, int ma, int mb, long long N, double2* out,
                          double* partial, long long partial_cap, int* err, cudaStream_t s) {
  static bool attr[64] = {};
  int dev = 0;
  IWF_CUDA(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64 && !attr[dev]) {
    IWF_CUDA(cudaFuncSetAttribute(gram_tc_kernel<NMMA>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap));
    attr[dev] = true;
  }
  int na_max = 0, nb_max = 0;
  for (int t = 0; t < subs.n; ++t) {
    na_max = std::max(na_max, subs.s[t].na);
    nb_max = std::max(nb_max, subs.s[t].nb);
  }
  // the shared-memory layout of the largest sub-Gram serves them all
  const GramLayout<NMMA> Lo(na_max, nb_max);
  int S = kMaxStages;
  while (S > 2 && Lo.smem(S) > kSmemCap) --S;
  if (Lo.smem(S) > kSmemCap) return fail(IWF_ERR_ARG, "gram_tc: tiles exceed shared memory");
  const long long chunks = (N + kChunkRows - 1) / kChunkRows;
  long long want = std::max(1, sm_count() / (subs.n * std::max(1, bt.nprob)));
  want = std::min<long long>(want, std::max<long long>(1, chunks));
  want = std::min<long long>(want, std::max<long long>(
                                       1, partial_cap / ((long long)subs.slot_size * bt.nprob)));
  const long long per = (chunks + want - 1) / want * kChunkRows;
  const int slots = (int)((N + per - 1) / per);
  dim3 grid((unsigned)std::max(1, slots), (unsigned)bt.nprob, (unsigned)subs.n);
  gram_tc_kernel<NMMA><<<grid, kGramThreads, Lo.smem(S), s>>>(bt, A, B, N, per, S, subs, partial,
                                                              err);
  IWF_CUDA(cudaGetLastError());
  count_launch();
  gram_tc_reduce<<<dim3((ma * mb + 255) / 256, bt.nprob), 256, 0, s>>>(
      bt, partial, std::max(1, slots), ma, mb, subs, out);
  IWF_CUDA(cudaGetLastError());
  count_launch();
  return IWF_OK;
}

template <int NMMA, bool SUB>
iwf_status launch_update_tc(const Batch& bt, const BlockList& S, int m, long long N,
                            const double2* C1, const double2* C2, int cstride, int q,
                            double2* out1, double2* out2, int* err, cudaStream_t s) {
  using Cfg = UpdCfg<NMMA>;
  static bool attr[64] = {};
  int dev = 0;
  IWF_CUDA(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64 && !attr[dev]) {
    IWF_CUDA(cudaFuncSetAttribute(update_tc_kernel<NMMA, SUB>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::kSmem));
    attr[dev] = true;
  }
  const int nout = (!SUB && C2) ? 2 : 1;
  const long long ntiles = (N + 127) / 128;
  long long slots = std::max(1, sm_count() / (nout * std::max(1, bt.nprob)));
  slots = std::min(slots, ntiles);
  dim3 grid((unsigned)(slots * nout), (unsigned)bt.nprob);
  update_tc_kernel<NMMA, SUB><<<grid, kUpdThreads, Cfg::kSmem, s>>>(bt, S, m, N, C1, C2, cstride,
                                                                    q, out1, out2, nout, err);
  IWF_CUDA(cudaGetLastError());
  count_launch();
  return IWF_OK;
}

}  // namespace

// Column scales of A and B (one memset of the problems' scale slots, one kernel)
iwf_status colexp(const Batch& bt, const BlockList& A, const BlockList& B, long long N,
                  cudaStream_t s) {
  const int ma = A.nb * A.b, mb = B.nb * B.b;
  bool same = ma == mb && A.b == B.b;
  for (int i = 0; same && i < A.nb; ++i) same = A.p[i] == B.p[i];
  IWF_CUDA(cudaMemsetAsync(bt.exps, 0, sizeof(int) * 2 * kMaxSmall * (size_t)bt.nprob, s));
  const long long blocks = std::max<long long>(1, std::min<long long>(64, (N + 4095) / 4096));
  colexp_kernel<<<dim3((unsigned)blocks, (unsigned)(same ? ma : ma + mb), (unsigned)bt.nprob),
                  256, 0, s>>>(bt, A, B, ma, same ? 1 : 0, N, bt.exps);
  IWF_CUDA(cudaGetLastError());
  count_launch();
  return IWF_OK;
}

iwf_status gram_tc(const Batch& bt, const BlockList& A, const BlockList& B, long long N,
                   double2* out, double* partial, int slots_cap, int* err, cudaStream_t s,
                   bool herm) {
  const int ma = A.nb * A.b, mb = B.nb * B.b;
  if (!bt.exps) return fail(IWF_ERR_ARG, "gram_tc: no exponent scratch");
  if (ma > kMaxSmall || mb > kMaxSmall) return fail(IWF_ERR_ARG, "gram_tc: shape");
  IWF_TRY(colexp(bt, A, B, N, s));
  // sub-Grams: A in blocks of 48 columns, B in blocks of 24 (the last ones shorter)
  const int nA = (ma + 47) / 48, nB = (mb + 23) / 24;
  SubList subs{};
  subs.herm = herm ? 1 : 0;
  int off = 0, nbmax = 0;
  for (int i = 0; i < nA; ++i) {
    const int a0 = 48 * i, a1 = std::min(ma, a0 + 48);
    for (int j = 0; j < nB; ++j) {
      const int b0 = 24 * j, b1 = std::min(mb, b0 + 24);
      if (herm && a0 >= b1) continue;              // entirely below the diagonal: mirrored
      if (subs.n >= kMaxSub) return fail(IWF_ERR_ARG, "gram_tc: too many sub-Grams");
      subs.s[subs.n++] = SubGram{a0, a1 - a0, b0, b1 - b0, off};
      off += 4 * (a1 - a0) * (b1 - b0);
      nbmax = std::max(nbmax, b1 - b0);
    }
  }
  subs.slot_size = off;
  const long long cap = (long long)bt.nprob * slots_cap * 2 * kCapG;
  const int nm = ((2 * nbmax + 15) / 16) * 16;
  if (nm == 16) return launch_gram_tc<16>(bt, A, B, subs, ma, mb, N, out, partial, cap, err, s);
  if (nm == 32) return launch_gram_tc<32>(bt, A, B, subs, ma, mb, N, out, partial, cap, err, s);
  return launch_gram_tc<48>(bt, A, B, subs, ma, mb, N, out, partial, cap, err, s);
}

iwf_status update_tc(const Batch& bt, const BlockList& S, long long N, const double2* C1,
                     const double2* C2, int cstride, int q, double2* out1, double2* out2,
                     bool subtract, int* err, cudaStream_t s) {
  const int m = S.nb * S.b;
  if (m > kMaxSmall || q < 1 || q > kMaxBlock) return fail(IWF_ERR_ARG, "update_tc: shape");
  const int nm = ((2 * q + 15) / 16) * 16;
#define IWF_UPD(NM)                                                                        \
  if (nm == NM) {                                                                          \
    if (subtract)                                                                          \
      return launch_update_tc<NM, true>(bt, S, m, N, C1, nullptr, cstride, q, out1, nullptr, \
                                        err, s);                                           \
    return launch_update_tc<NM, false>(bt, S, m, N, C1, C2, cstride, q, out1, out2, err, s); \
  }
  IWF_UPD(16) IWF_UPD(32) IWF_UPD(48)
#undef IWF_UPD
  return fail(IWF_ERR_ARG, "update_tc: shape");
}

}  // namespace iwf
