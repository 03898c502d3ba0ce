// H~ psi = Lambda psi + F V F^{-1} psi on the GPU (Sec. 4.1), with F = T F* (Sec. 3.3).
//
// The lifted grid is split into two axis groups: the d k_I axes (innermost in memory, one
// contiguous slice of (2K)^d points per k_II) and the n-d k_II axes (outermost). One apply is
// three passes over global memory, each staging tiles in shared memory and running the
// register DFT codelets of dft.cuh along every axis of its group:
//   pass A  (k_I group)   window order -> cyclic roll by the slice bound lo_j(k_II) (the
//                         index shift T^{-1}, Eq. index mod) -> inverse DFT along k_I axes;
//   pass B  (k_II group)  roll by L_j -> inverse DFT along k_II axes -> multiply by V(y)/N on
//                         G_{K,L} -> forward DFT along k_II axes -> roll back; in place;
//   pass C  (k_I group)   forward DFT along k_I axes -> roll back by lo_j (the scatter T) ->
//                         add Lambda_k psi_k.
// A k_II group too large for one shared-memory tile (more than 8192 points, Example 4.3 from
// L = 20) runs as per-axis passes: inverse DFTs along its slower axes one at a time (KIND 0
// on a one-axis group), the last axis with the multiply by V as pass B, then the forward DFTs
// back along the slower axes (KIND 3).
// Rolls are index permutations inside a pencil and cost no arithmetic. Vectors are processed
// in chunks sized so that the intermediate block stays resident in the 129 MB L2.
//
// Two kernel sets implement the passes. The tiled set (pass_kernel) stages whole tiles in
// shared memory and handles every geometry. The pencil set (pencil_*) covers two k_I and two
// k_II axes of equal lengths 16 or 32 (the 2D moire family): one pencil per thread in
// registers, global loads and stores straight from registers, one swizzled shared-memory
// transpose per axis change, and for complex float a bulk-copy pipeline in pass C.
#include <atomic>
#include <mutex>
#include <string>
#include <cmath>
#include <cstdio>
#include <cstring>

#include <vector>

#include "common.cuh"
#include "dft.cuh"

namespace iwf {

namespace {

constexpr int kThreads = 256;
constexpr int kLongThreads = 512;   // pass kernels of axis groups with a long axis

template <typename T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

// Shared-memory padding: one spare slot every 32 elements breaks power-of-two strides.
__device__ __forceinline__ int padx(int i) { return i + (i >> 5); }

// Static description of one axis group inside a tile.
struct GroupDesc {
  int ng;                   // axes in the group
  int len[IWF_MAX_N];       // slowest first
  int gs[IWF_MAX_N];        // stride of each axis in units of group points (C order)
  int kI[IWF_MAX_N];        // >= 0: k_I axis index j (roll from the lo table); -1: k_II axis
  int Lroll[IWF_MAX_N];     // k_II axes: roll offset L_j
};

struct PassArgs {
  Geom g;
  GroupDesc grp;
  int M;                    // points of the group (product of len)
  long long inner;          // points of all faster axes
  int C;                    // inner chunk per tile (a power of two)
  int lc;                   // log2(C)
  int Ot;                   // outer indices per tile
  long long outer;          // number of outer indices
  long long tiles_inner;    // inner chunks per outer index
  const void* in;
  void* out;
  const void* psi;          // pass C only
  const void* lam;          // pass C only
  const int* lo;            // MII x d
  PotDev pot;               // pass B only (tables); all passes (batch skipping)
  long long ld;             // element stride between vectors (= N)
  int tile_bytes;           // shared-memory bytes of the tile (pass B's V tables follow it)
  int vec_base;             // index of the launch's first vector in the whole block
  const void* ltw[IWF_MAX_N];  // group axes longer than IWF_MAX_LEN: exp(2 pi i j / len)
  // pass B split into per-axis passes (a k_II group too large for one tile): the group is
  // k_II axes [ii0, ii0 + ng); the slower k_II axes index the outer range, the faster ones
  // the inner range above the k_I slice (0 and ng for the unsplit pass B)
  int ii0;
};

// Roll offset of axis a for outer tile index o: pencil element k* lives at (k* + off) mod len.
__device__ __forceinline__ int roll_off(const PassArgs& a, int ax, long long o) {
  const int len = a.grp.len[ax];
  if (a.grp.kI[ax] >= 0) {
    const int lo = a.lo[o * a.g.d + a.grp.kI[ax]];
    int off = (-lo) % len;
    return off < 0 ? off + len : off;
  }
  return a.grp.Lroll[ax] % len;
}

// One DFT of length LEN along group axis `ax` for every pencil of the tile.
// ROLL_LOAD: gather with the roll (inverse direction); ROLL_STORE: scatter with it (forward).
template <typename T, int LEN, int S, bool ROLL_LOAD, bool ROLL_STORE>
__device__ void axis_dft(typename Vec2<T>::type* tile, const PassArgs& a, int ax, long long o0,
                         const int* s_off) {
  using V2 = typename Vec2<T>::type;
  const int lc = a.lc, M = a.M;
  const int gs = a.grp.gs[ax];
  const int step = gs << lc;                       // tile distance between pencil elements
  const int per_o = (M / LEN) << lc;
  const int npen = per_o * a.Ot;
  for (int p = threadIdx.x; p < npen; p += blockDim.x) {
    const int ot = p / per_o;
    const int rem = p - ot * per_o;
    const int c = rem & ((1 << lc) - 1);
    const int rest = rem >> lc;
    const int q = rest / gs;
    const int g0 = q * gs * LEN + (rest - q * gs);
    const int base = ((ot * M + g0) << lc) + c;
    const int off = (ROLL_LOAD || ROLL_STORE) ? s_off[ot * IWF_MAX_N + ax] : 0;
    T xr[LEN], xi[LEN];
#pragma unroll
    for (int i = 0; i < LEN; ++i) {
      int src = i;
      if (ROLL_LOAD) { src = i + off; if (src >= LEN) src -= LEN; }
      const V2 v = tile[padx(base + src * step)];
      xr[i] = v.x; xi[i] = v.y;
    }
    Dft<LEN, S, T>::run(xr, xi);
#pragma unroll
    for (int i = 0; i < LEN; ++i) {
      int dst = i;
      if (ROLL_STORE) { dst = i + off; if (dst >= LEN) dst -= LEN; }
      V2 v; v.x = xr[i]; v.y = xi[i];
      tile[padx(base + dst * step)] = v;
    }
  }
}

template <typename T, int S, bool RL, bool RS>
__device__ void axis_dispatch(typename Vec2<T>::type* tile, const PassArgs& a, int ax, long long o0,
                              const int* s_off) {
  switch (a.grp.len[ax]) {
#define IWF_CASE(L_) case L_: axis_dft<T, L_, S, RL, RS>(tile, a, ax, o0, s_off); break;
    IWF_CASE(2) IWF_CASE(4) IWF_CASE(6) IWF_CASE(8) IWF_CASE(10) IWF_CASE(12) IWF_CASE(14)
    IWF_CASE(16) IWF_CASE(18) IWF_CASE(20) IWF_CASE(22) IWF_CASE(24) IWF_CASE(26) IWF_CASE(28)
    IWF_CASE(30) IWF_CASE(32)
#undef IWF_CASE
    default: break;  // lengths are validated on the host
  }
}

// ---- axes longer than the codelets: in-place mixed-radix Stockham FFT in shared memory ----
// A stage of radix R works on sub-transforms of size Ns (the product of the earlier radices).
// Butterfly j of a pencil takes the elements j + r LEN/R (r < R), multiplies element r by
// w^(r k LEN/(Ns R)) with k = j mod Ns and w = exp(S 2 pi i / LEN), combines them by an
// R-point DFT and writes output r to (j / Ns) Ns R + k + r Ns. After the last stage the
// pencil holds its DFT in natural order. Every thread first reads all its butterflies of a
// stage into registers, the block synchronises, and then they are written, so the stages run
// in place; the host keeps a tile at most long_stage_values(R) x blockDim elements. The roll
// acts on the first stage's reads (gather) and on the last stage's writes (scatter), as in
// axis_dft.
__device__ __forceinline__ int pencil_base(const PassArgs& a, int gs, int len, int per_o, int p,
                                           int* ot) {
  const int o = p / per_o;
  const int rem = p - o * per_o;
  const int c = rem & ((1 << a.lc) - 1);
  const int rest = rem >> a.lc;
  const int q = rest / gs;
  const int g0 = q * gs * len + (rest - q * gs);
  *ot = o;
  return ((o * a.M + g0) << a.lc) + c;
}

template <typename T, int R, int S, bool RL, bool RS>
__device__ __forceinline__ void long_stage(typename Vec2<T>::type* tile, const PassArgs& a, int ax, int len,
                           int Ns, bool first, bool last, const int* s_off) {
  using V2 = typename Vec2<T>::type;
  constexpr int NB = 16 / R;                       // butterflies per thread and stage
  const V2* __restrict__ tw = reinterpret_cast<const V2*>(a.ltw[ax]);
  const int gs = a.grp.gs[ax];
  const int step = gs << a.lc;
  const int per_o = (a.M / len) << a.lc;
  const int bpp = len / R;                         // butterflies per pencil
  const int total = per_o * a.Ot * bpp;
  const int tws = len / (Ns * R);
  T vr[NB][R], vi[NB][R];
#pragma unroll
  for (int bb = 0; bb < NB; ++bb) {
    const int b = threadIdx.x + bb * blockDim.x;
    if (b < total) {
      const int p = b / bpp, j = b - p * bpp;
      int ot;
      const int base = pencil_base(a, gs, len, per_o, p, &ot);
      const int off = (RL && first) ? s_off[ot * IWF_MAX_N + ax] : 0;
      const int k = j % Ns;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        int i = j + r * bpp;
        if (RL && first) { i += off; if (i >= len) i -= len; }
        const V2 v = tile[padx(base + i * step)];
        T xr = v.x, xi = v.y;
        const int e = r * k * tws;
        if (e) {
          const V2 w = __ldg(tw + e);
          const T c = w.x, sn = S > 0 ? w.y : -w.y;
          const T t = xr * c - xi * sn;
          xi = xr * sn + xi * c;
          xr = t;
        }
        vr[bb][r] = xr; vi[bb][r] = xi;
      }
      Butterfly<R, S, T>::run(vr[bb], vi[bb]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int bb = 0; bb < NB; ++bb) {
    const int b = threadIdx.x + bb * blockDim.x;
    if (b < total) {
      const int p = b / bpp, j = b - p * bpp;
      int ot;
      const int base = pencil_base(a, gs, len, per_o, p, &ot);
      const int off = (RS && last) ? s_off[ot * IWF_MAX_N + ax] : 0;
      const int k = j % Ns;
      const int o0 = (j / Ns) * Ns * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        int o = o0 + r * Ns;
        if (RS && last) { o += off; if (o >= len) o -= len; }
        V2 v; v.x = vr[bb][r]; v.y = vi[bb][r];
        tile[padx(base + o * step)] = v;
      }
    }
  }
  __syncthreads();
}

template <typename T, int S, bool RL, bool RS>
__device__ __forceinline__ void long_axis_fft(typename Vec2<T>::type* tile, const PassArgs& a, int ax,
                              const int* s_off) {
  const int len = a.grp.len[ax];
  int Ns = 1;
  for (int rem = len; rem > 1;) {
    const int R = long_radix(rem);
    const bool first = Ns == 1, last = rem == R;
    switch (R) {
#define IWF_STAGE(R_) case R_: long_stage<T, R_, S, RL, RS>(tile, a, ax, len, Ns, first, last, s_off); break;
      IWF_STAGE(4) IWF_STAGE(2) IWF_STAGE(3) IWF_STAGE(5) IWF_STAGE(7)
#undef IWF_STAGE
      default: return;  // lengths are validated on the host
    }
    Ns *= R;
    rem /= R;
  }
}

// One axis of a group: register codelets, or in the LONG instantiation of the pass kernel
// (groups with an axis longer than IWF_MAX_LEN) the shared-memory FFT for every axis of the
// group, so that neither instantiation carries the other's register demand. Ends with the
// block synchronised.
template <typename T, int S, bool RL, bool RS, bool LONG>
__device__ __forceinline__ void run_axis(typename Vec2<T>::type* tile, const PassArgs& a, int ax,
                                         long long o0, const int* s_off) {
  if constexpr (LONG) {
    if (a.grp.len[ax] > 1) long_axis_fft<T, S, RL, RS>(tile, a, ax, s_off);
  } else {
    axis_dispatch<T, S, RL, RS>(tile, a, ax, o0, s_off);
    __syncthreads();
  }
}

template <typename T> __device__ __forceinline__ T pot_tab(const PotDev& p, long long off);
template <> __device__ __forceinline__ double pot_tab<double>(const PotDev& p, long long off) { return p.tab64[off]; }
template <> __device__ __forceinline__ float pot_tab<float>(const PotDev& p, long long off) { return p.tab32[off]; }
template <typename T> __device__ __forceinline__ T pot_grid(const PotDev& p, long long i);
template <> __device__ __forceinline__ double pot_grid<double>(const PotDev& p, long long i) { return p.grid64[i]; }
template <> __device__ __forceinline__ float pot_grid<float>(const PotDev& p, long long i) { return p.grid32[i]; }
template <typename T> __device__ __forceinline__ T pot_const(const PotDev& p);
template <> __device__ __forceinline__ double pot_const<double>(const PotDev& p) { return p.c64; }
template <> __device__ __forceinline__ float pot_const<float>(const PotDev& p) { return p.c32; }

// KIND 0: pass A, KIND 1: pass B, KIND 2: pass C. LONG: the group has an axis longer than
// IWF_MAX_LEN (run by pass_long_kernel).
template <typename T, int KIND, bool LONG>
__device__ __forceinline__ void pass_body(const PassArgs& a) {
  using V2 = typename Vec2<T>::type;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  V2* tile = reinterpret_cast<V2*>(smem_raw);
  __shared__ int s_off[64 * IWF_MAX_N];

  const long long tile_id = blockIdx.x;
  const long long o0 = (tile_id / a.tiles_inner) * a.Ot;
  const long long c0 = (tile_id % a.tiles_inner) * a.C;
  const int Ot = (int)min((long long)a.Ot, a.outer - o0);
  const int vec = blockIdx.y;
  int prob = 0;
  if (a.pot.vecs_per_prob > 0) {
    prob = (a.vec_base + vec) / a.pot.vecs_per_prob;
    if (a.pot.active && !a.pot.active[prob]) return;
  }
  const V2* in = reinterpret_cast<const V2*>(a.in) + (size_t)vec * a.ld;
  V2* out = reinterpret_cast<V2*>(a.out) + (size_t)vec * a.ld;

  // roll offsets of every outer slot of the tile; the slots past the last outer index of a
  // partial tile get 0, so that the DFTs run on them (on unused data) stay inside the tile
  for (int t = threadIdx.x; t < a.Ot * a.grp.ng; t += blockDim.x) {
    const int ot = t / a.grp.ng, ax = t % a.grp.ng;
    s_off[ot * IWF_MAX_N + ax] = ot < Ot ? roll_off(a, ax, o0 + ot) : 0;
  }
  // stage the tile: rows of C contiguous elements, one row per (outer, group point);
  // element e of the tile sits at (e >> lc) * inner + (e & (C-1)) from the tile's origin
  const int C = a.C, M = a.M, lc = a.lc;
  const int nel = Ot * M * C;
  const size_t org = (size_t)o0 * M * a.inner + c0;
  const V2* tin = in + org;
  const bool contig = a.inner == C;                // the whole tile is one contiguous run
  auto gidx = [&](int e) -> size_t {
    return contig ? (size_t)e : (size_t)(e >> lc) * a.inner + (e & (C - 1));
  };
  // complex float: two neighbours of a row (or of a contiguous tile) move as one 16-byte word
  const bool pairs = sizeof(T) == 4 && (contig || C >= 2) && (nel % 2 == 0);
  bool staged = false;
  if constexpr (sizeof(T) == 4) {
    if (pairs) {
      for (int e = 2 * threadIdx.x; e < nel; e += 2 * blockDim.x) {
        const float4 w = *reinterpret_cast<const float4*>(tin + gidx(e));
        tile[padx(e)] = make_float2(w.x, w.y);
        tile[padx(e + 1)] = make_float2(w.z, w.w);
      }
      staged = true;
    }
  }
  if (!staged)
    for (int e = threadIdx.x; e < nel; e += blockDim.x) tile[padx(e)] = tin[gidx(e)];
  __syncthreads();

  if (KIND == 0) {
    for (int ax = 0; ax < a.grp.ng; ++ax) run_axis<T, +1, true, false, LONG>(tile, a, ax, o0, s_off);
  } else if (KIND == 3) {
    for (int ax = 0; ax < a.grp.ng; ++ax) run_axis<T, -1, false, true, LONG>(tile, a, ax, o0, s_off);
  } else if (KIND == 1) {
    for (int ax = 0; ax < a.grp.ng; ++ax) run_axis<T, +1, true, false, LONG>(tile, a, ax, o0, s_off);
    // multiply by V(y_l)/N: l_II from the group point, l_I from the inner index. With
    // per-axis tables V = [const + sum over k_I axes] + [sum over k_II axes]; both parts are
    // tabulated once per tile (vI over the C inner indices, vII over the M group points).
    // (Ot = 1 here: the inner range is above one point.) With a split k_II group the slower
    // k_II axes come from the outer index o0 and the faster ones from the inner index above
    // the k_I slice.
    const int nII = a.g.n - a.g.d, ii1 = a.ii0 + a.grp.ng;
    if (a.pot.kind == 1) {
      T* vII = reinterpret_cast<T*>(smem_raw + a.tile_bytes);
      T* vI = vII + M;
      const long long tbase = (long long)prob * a.pot.tab_stride;
      T vout = pot_const<T>(a.pot);          // slower k_II axes (outer index, C order)
      {
        long long rem = o0;
        for (int j = a.ii0 - 1; j >= 0; --j) {
          const int lj = (int)(rem % a.g.lens[a.g.d + j]);
          rem /= a.g.lens[a.g.d + j];
          vout += pot_tab<T>(a.pot, tbase + a.pot.tab_off[a.g.d + j] + lj);
        }
      }
      for (int c = threadIdx.x; c < C; c += blockDim.x) {
        T v = vout;
        long long rem = c0 + c;              // inner index -> l_I, then faster l_II (C order)
        for (int j = a.g.d - 1; j >= 0; --j) {
          const int lj = (int)(rem % a.g.lens[j]);
          rem /= a.g.lens[j];
          v += pot_tab<T>(a.pot, tbase + a.pot.tab_off[j] + lj);
        }
        for (int j = nII - 1; j >= ii1; --j) {
          const int lj = (int)(rem % a.g.lens[a.g.d + j]);
          rem /= a.g.lens[a.g.d + j];
          v += pot_tab<T>(a.pot, tbase + a.pot.tab_off[a.g.d + j] + lj);
        }
        vI[c] = v;
      }
      for (int g = threadIdx.x; g < M; g += blockDim.x) {
        T v = T(0);
        int gr = g;                          // group point -> l_II coordinates
        for (int ax = a.grp.ng - 1; ax >= 0; --ax) {
          const int lj = gr % a.grp.len[ax];
          gr /= a.grp.len[ax];
          v += pot_tab<T>(a.pot, tbase + a.pot.tab_off[a.g.d + a.ii0 + ax] + lj);
        }
        vII[g] = v;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < nel; e += blockDim.x) {
        const T v = vI[e & (C - 1)] + vII[e >> lc];
        V2 x = tile[padx(e)];
        x.x *= v; x.y *= v;
        tile[padx(e)] = x;
      }
    } else {
      for (int e = threadIdx.x; e < nel; e += blockDim.x) {
        const T v = pot_grid<T>(a.pot, ((long long)o0 * M + (e >> lc)) * a.inner + c0 +
                                           (e & (C - 1)));
        V2 x = tile[padx(e)];
        x.x *= v; x.y *= v;
        tile[padx(e)] = x;
      }
    }
    __syncthreads();
    for (int ax = 0; ax < a.grp.ng; ++ax) run_axis<T, -1, false, true, LONG>(tile, a, ax, o0, s_off);
  } else {
    for (int ax = 0; ax < a.grp.ng; ++ax) run_axis<T, -1, false, true, LONG>(tile, a, ax, o0, s_off);
  }

  V2* tout = out + org;
  if (KIND == 2) {
    const V2* psi = reinterpret_cast<const V2*>(a.psi) + (size_t)vec * a.ld + org;
    const T* lam = reinterpret_cast<const T*>(a.lam) + org;
    for (int e = threadIdx.x; e < nel; e += blockDim.x) {
      const size_t gi = gidx(e);
      const V2 x = tile[padx(e)];
      const V2 p = psi[gi];
      const T l = lam[gi];
      V2 r; r.x = x.x + l * p.x; r.y = x.y + l * p.y;
      tout[gi] = r;
    }
  } else {
    bool done = false;
    if constexpr (sizeof(T) == 4) {
      if (pairs) {
        for (int e = 2 * threadIdx.x; e < nel; e += 2 * blockDim.x) {
          const V2 u0 = tile[padx(e)], u1 = tile[padx(e + 1)];
          *reinterpret_cast<float4*>(tout + gidx(e)) = make_float4(u0.x, u0.y, u1.x, u1.y);
        }
        done = true;
      }
    }
    if (!done)
      for (int e = threadIdx.x; e < nel; e += blockDim.x) tout[gidx(e)] = tile[padx(e)];
  }
}

template <typename T, int KIND>
__global__ void __launch_bounds__(kThreads) pass_kernel(PassArgs a) { pass_body<T, KIND, false>(a); }

// One CTA per SM is enough for these (a long axis fills the tile); the bound lets each thread
// keep a whole FFT stage (16 complex values) in registers.
template <typename T, int KIND>
__global__ void __launch_bounds__(kLongThreads, 1) pass_long_kernel(PassArgs a) {
  pass_body<T, KIND, true>(a);
}

// ---------------------------------------------------------------------------------------
// Pencil path for the common geometry of two k_I axes of length LI and two k_II axes of
// length LII (LI, LII in {16, 32}; the 2D moire family). Every thread holds one whole
// pencil in registers: the first axis is loaded straight from global memory (L independent
// loads per thread, coalesced because the lanes run along the other, contiguous axis), one
// XOR-swizzled shared-memory transpose switches to the second axis, and results leave
// registers straight for global memory. The intermediate block uses its own slice layout:
// position l1 * LI + l0 for the k_I grid point (l0, l1), i.e. each slice is stored
// transposed, which makes pass A's stores and pass C's loads coalesced.
//
// Bank conflicts: a warp-wide access of 8-byte (16-byte) elements is served in wavefronts of
// G = 16 (8) lanes; the swizzles make the G element indices of every wavefront distinct
// modulo G, both when a pencil is written and when the transposed pencil is read.
// Compute type of the pencil DFTs: the storage type itself, or the double-float dfl for
// FP64 storage (IWF_ARITH_DF: the FP32 pipes instead of the FP64 one). A shared-memory
// complex element is 16 bytes in both FP64 forms, so the layouts and swizzles are shared.
template <typename U> struct SmemCplx;
template <> struct SmemCplx<double> { using type = double2; };
template <> struct SmemCplx<float> { using type = float2; };
template <> struct SmemCplx<dfl> { using type = float4; };
__device__ __forceinline__ double2 mkc(double r, double i) { return make_double2(r, i); }
__device__ __forceinline__ float2 mkc(float r, float i) { return make_float2(r, i); }
__device__ __forceinline__ float4 mkc(dfl r, dfl i) { return make_float4(r.h, r.l, i.h, i.l); }
__device__ __forceinline__ void unc(double2 v, double& r, double& i) { r = v.x; i = v.y; }
__device__ __forceinline__ void unc(float2 v, float& r, float& i) { r = v.x; i = v.y; }
__device__ __forceinline__ void unc(float4 v, dfl& r, dfl& i) { r = dfl(v.x, v.y); i = dfl(v.z, v.w); }
// storage value -> compute value, and back
__device__ __forceinline__ void ld_u(double x, double& u) { u = x; }
__device__ __forceinline__ void ld_u(float x, float& u) { u = x; }
__device__ __forceinline__ void ld_u(double x, dfl& u) { u = to_dfl(x); }
__device__ __forceinline__ double st_t(double u) { return u; }
__device__ __forceinline__ float st_t(float u) { return u; }
__device__ __forceinline__ double st_t(dfl u) { return from_dfl(u); }

struct PencilArgs {
  const void* in;
  void* out;
  const void* psi;          // pass C
  const void* lam;          // pass C
  const int* lo;            // MII x 2 slice bounds (passes A and C)
  PotDev pot;               // pass B tables or grid; batch skipping in every pass
  long long ld;             // N, elements between vectors
  long long MI, MII;        // LI^2, LII^2
  int vec_base;
  long long spin;           // pipelined pass C: try_wait rounds of each main wait
};

template <typename T> constexpr int wave_lanes() { return sizeof(T) == 4 ? 16 : 8; }

__device__ __forceinline__ bool pencil_skip(const PencilArgs& a, int vec) {
  if (a.pot.vecs_per_prob <= 0 || !a.pot.active) return false;
  return !a.pot.active[(a.vec_base + vec) / a.pot.vecs_per_prob];
}

__device__ __forceinline__ int roll_of(int lo, int len) {
  int off = (-lo) % len;
  return off < 0 ? off + len : off;
}

// Pass A (KIND 0) and pass C (KIND 2) over whole slices. A warp owns 32 / L slices; lane
// (s, p) of it loads grid column p of slice s along axis 0, so each load instruction reads
// whole 32-element rows of the slice (a permutation of them, because of the roll).
template <typename T, int L, int KIND, typename U = T>
__global__ void __launch_bounds__(256) pencil_ac_kernel(PencilArgs a) {
  using V2 = typename Vec2<T>::type;
  using SC = typename SmemCplx<U>::type;
  static_assert(sizeof(SC) == sizeof(V2), "shared-memory element size");
  constexpr int SPW = 32 / L, LL = L * L;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = lane / L, p = lane % L;
  const long long o = ((long long)blockIdx.x * (blockDim.x >> 5) + warp) * SPW + s;
  const int vec = blockIdx.y;
  if (pencil_skip(a, vec)) return;
  if (((long long)blockIdx.x * (blockDim.x >> 5) + warp) * SPW >= a.MII) return;  // whole warp idle
  const bool valid = o < a.MII;
  SC* S = reinterpret_cast<SC*>(smem_raw) + (size_t)threadIdx.x / L * LL;  // this slice's buffer
  int off0 = 0, off1 = 0;
  if (valid) { off0 = roll_of(a.lo[2 * o], L); off1 = roll_of(a.lo[2 * o + 1], L); }
  const size_t sbase = (size_t)vec * a.ld + (size_t)o * LL;
  U xr[L], xi[L];
  if (KIND == 0) {
    // window order -> grid: grid (i, p) sits at window ((i + off0) mod L, (p + off1) mod L)
    const V2* in = reinterpret_cast<const V2*>(a.in) + sbase;
    const int col = (p + off1) & (L - 1);
#pragma unroll
    for (int i = 0; i < L; ++i) {
      V2 v{};
      if (valid) v = in[((i + off0) & (L - 1)) * L + col];
      ld_u(v.x, xr[i]); ld_u(v.y, xi[i]);
    }
    Dft<L, +1, U>::run(xr, xi);                         // along axis 0: lane p has column p
#pragma unroll
    for (int i = 0; i < L; ++i) S[i * L + (p ^ i)] = mkc(xr[i], xi[i]);
    __syncwarp();
#pragma unroll
    for (int j = 0; j < L; ++j) unc(S[p * L + (j ^ p)], xr[j], xi[j]);
    Dft<L, +1, U>::run(xr, xi);                         // along axis 1: lane p has row l0 = p
    if (valid) {
      V2* out = reinterpret_cast<V2*>(a.out) + sbase;
#pragma unroll
      for (int j = 0; j < L; ++j) { V2 v; v.x = st_t(xr[j]); v.y = st_t(xi[j]); out[j * L + p] = v; }
    }
  } else {
    const V2* in = reinterpret_cast<const V2*>(a.in) + sbase;
#pragma unroll
    for (int j = 0; j < L; ++j) {
      V2 v{};
      if (valid) v = in[j * L + p];
      ld_u(v.x, xr[j]); ld_u(v.y, xi[j]);
    }
    Dft<L, -1, U>::run(xr, xi);                         // along axis 1 for row l0 = p
#pragma unroll
    for (int j = 0; j < L; ++j) S[p * L + (j ^ p)] = mkc(xr[j], xi[j]);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < L; ++i) unc(S[i * L + (p ^ i)], xr[i], xi[i]);
    Dft<L, -1, U>::run(xr, xi);                         // along axis 0 for column p
    if (valid) {
      // grid -> window order, + Lambda psi at the same window positions. psi and H psi never
      // overlap (checked on the host), so the loads of a batch are all issued before its
      // stores instead of one load round trip per element.
      const V2* __restrict__ psi = reinterpret_cast<const V2*>(a.psi) + sbase;
      const T* __restrict__ lam = reinterpret_cast<const T*>(a.lam) + (size_t)o * LL;
      V2* __restrict__ out = reinterpret_cast<V2*>(a.out) + sbase;
      const int col = (p + off1) & (L - 1);
      constexpr int kBatch = 8;
#pragma unroll
      for (int i0 = 0; i0 < L; i0 += kBatch) {
        V2 q[kBatch];
        T l[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
          const int w = ((i0 + u + off0) & (L - 1)) * L + col;
          q[u] = psi[w];
          l[u] = lam[w];
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
          const int w = ((i0 + u + off0) & (L - 1)) * L + col;
          V2 r; r.x = st_t(xr[i0 + u]) + l[u] * q[u].x; r.y = st_t(xi[i0 + u]) + l[u] * q[u].y;
          out[w] = r;
        }
      }
    }
  }
}

// ---- asynchronous bulk copies (TMA) and mbarriers -------------------------------------
// Every wait is bounded: after kSpinRounds unsuccessful try_wait rounds the kernel records
// kApplyTimeout in the plan's apply error word and stops.
constexpr long long kSpinRounds = 1LL << 20;
constexpr int kApplyTimeout = 1;

__device__ __forceinline__ uint32_t smem_addr(const void* ptr) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(ptr));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void proxy_fence() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
// Drops a 128-byte line of scratch data from L2 without writing it back (its value becomes
// undefined): the intermediate block is dead once pass C has read it.
__device__ __forceinline__ void discard_l2(const void* line) {
  asm volatile("discard.global.L2 [%0], 128;" ::"l"(line));
}
__device__ __forceinline__ void store_streaming(float2* p, float2 v) { __stcs(p, v); }
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for phase `parity` of the barrier (at most `rounds` try_wait rounds); false
// when the bound ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          long long rounds = kSpinRounds) {
  for (long long r = 0; r < rounds; ++r)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// Global -> shared bulk copy completing on `bar` (16-byte aligned addresses and size).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// Pipelined pass C. Each warp is persistent over units of 32 / L slices of one vector (32 L
// elements, contiguous in the intermediate block) and keeps STAGES - 1 units in flight: lane 0
// copies unit k + STAGES - 1 into shared memory with one bulk copy while the warp transforms
// unit k. The staged unit is read once into registers and its buffer then serves the
// transpose; its lines are then dropped from L2 (the intermediate block is dead after this
// pass). The unit's psi and Lambda are copied into a per-warp buffer as soon as the unit
// starts, so that the copy overlaps the two DFTs, and H psi leaves with streaming stores. Each
// unit's slice bounds are loaded before its wait. Units of inactive batch problems are
// skipped.
//
// Shared memory: per warp STAGES staged units and psi and Lambda of one unit (56 KB per CTA
// for complex float at L = 32: four CTAs per SM).
template <typename T>
__host__ __device__ constexpr size_t pipe_warp_bytes(int L, int stages) {
  return (size_t)stages * 32 * L * sizeof(typename Vec2<T>::type) +
         (size_t)32 * L * (sizeof(typename Vec2<T>::type) + sizeof(T));
}

template <typename T, int L, int WARPS, int STAGES>
__global__ void __launch_bounds__(WARPS * 32) pencil_c_pipe_kernel(PencilArgs a, int nvec,
                                                                   int* err) {
  using V2 = typename Vec2<T>::type;
  constexpr int SPW = 32 / L, LL = L * L, UNIT = 32 * L;
  constexpr uint32_t UBYTES = UNIT * sizeof(V2), LBYTES = UNIT * sizeof(T);
  constexpr size_t WBYTES = pipe_warp_bytes<T>(L, STAGES);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bars[WARPS][STAGES + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = lane / L, p = lane % L;
  unsigned char* wbase = smem_raw + (size_t)warp * WBYTES;
  V2* stages = reinterpret_cast<V2*>(wbase);
  V2* psi_s = stages + STAGES * UNIT;
  T* lam_s = reinterpret_cast<T*>(psi_s + UNIT);
  if (lane == 0)
    for (int st = 0; st <= STAGES; ++st) mbar_init(smem_addr(&bars[warp][st]), 1);
  mbar_init_fence();
  __syncthreads();

  const long long upv = a.MII / SPW;                 // units per vector
  const long long total = upv * nvec;
  const long long nw = (long long)gridDim.x * WARPS;
  const long long first = (long long)blockIdx.x * WARPS + warp;
  // j-th candidate unit of this warp, and the next candidate >= j whose problem is active
  const auto unit_of = [&](long long j) { return first + j * nw; };
  const auto next_active = [&](long long j) {
    while (unit_of(j) < total && pencil_skip(a, (int)(unit_of(j) / upv))) ++j;
    return j;
  };
  const auto unit_offset = [&](long long j) {
    const long long u = unit_of(j);
    return (size_t)(u / upv) * a.ld + (size_t)(u % upv) * UNIT;
  };
  const auto issue = [&](long long j, int st) {       // lane 0: unit j -> stage st
    const uint32_t bar = smem_addr(&bars[warp][st]);
    proxy_fence();                                     // generic accesses before the async write
    mbar_expect_tx(bar, UBYTES);
    bulk_load(smem_addr(stages + st * UNIT), reinterpret_cast<const V2*>(a.in) + unit_offset(j),
              UBYTES, bar);
  };

  long long jp = next_active(0);   // next unit to prefetch
  int kp = 0;                      // unit copies issued
  for (; kp < STAGES - 1 && unit_of(jp) < total; ++kp) {
    if (lane == 0) issue(jp, kp % STAGES);
    jp = next_active(jp + 1);
  }
  long long jc = next_active(0);
  int k = 0;
  bool ok = true, psi_pending = false;
  for (; unit_of(jc) < total; ++k, jc = next_active(jc + 1)) {
    __syncwarp();                  // unit k - 1 is done with its stage and the psi buffer
    if (unit_of(jp) < total) {     // refill the stage unit k - 1 used
      if (lane == 0) issue(jp, kp % STAGES);
      ++kp;
      jp = next_active(jp + 1);
    }
    const long long u = unit_of(jc);
    const size_t uoff = unit_offset(jc);
    if (lane == 0) {               // psi and Lambda of this unit, consumed after the DFTs
      const uint32_t bar = smem_addr(&bars[warp][STAGES]);
      proxy_fence();
      mbar_expect_tx(bar, UBYTES + LBYTES);
      bulk_load(smem_addr(psi_s), reinterpret_cast<const V2*>(a.psi) + uoff, UBYTES, bar);
      bulk_load(smem_addr(lam_s), reinterpret_cast<const T*>(a.lam) + (size_t)(u % upv) * UNIT,
                LBYTES, bar);
    }
    psi_pending = true;
    const long long o = (u % upv) * SPW + s;          // slice of this lane
    const int lo0 = a.lo[2 * o], lo1 = a.lo[2 * o + 1];  // issued before the wait, which hides them
    const int st = k % STAGES;
    ok = mbar_wait(smem_addr(&bars[warp][st]), (uint32_t)((k / STAGES) & 1), a.spin);
    if (__any_sync(0xffffffffu, !ok)) { ok = false; break; }
    V2* U = stages + st * UNIT + s * LL;               // this lane's slice in the stage
    const int off0 = roll_of(lo0, L), off1 = roll_of(lo1, L);
    T xr[L], xi[L];
    {
#pragma unroll
      for (int j = 0; j < L; ++j) { const V2 v = U[j * L + p]; xr[j] = v.x; xi[j] = v.y; }
      // the unit's intermediate values now live in registers: drop its lines from L2
      {
        const unsigned char* g = reinterpret_cast<const unsigned char*>(
            reinterpret_cast<const V2*>(a.in) + uoff);
#pragma unroll
        for (int t = 0; t < (int)(UBYTES / (32 * 128)); ++t) discard_l2(g + (t * 32 + lane) * 128);
      }
      Dft<L, -1, T>::run(xr, xi);
      __syncwarp();
#pragma unroll
      for (int j = 0; j < L; ++j) { V2 v; v.x = xr[j]; v.y = xi[j]; U[p * L + (j ^ p)] = v; }
      __syncwarp();
#pragma unroll
      for (int i = 0; i < L; ++i) { const V2 v = U[i * L + (p ^ i)]; xr[i] = v.x; xi[i] = v.y; }
      Dft<L, -1, T>::run(xr, xi);
      ok = mbar_wait(smem_addr(&bars[warp][STAGES]), (uint32_t)(k & 1), a.spin);
      if (__any_sync(0xffffffffu, !ok)) { ok = false; break; }
      psi_pending = false;
      // grid -> window order, + Lambda psi at the same window positions
      const V2* ps = psi_s + s * LL;
      const T* ls = lam_s + s * LL;
      V2* out = reinterpret_cast<V2*>(a.out) + uoff + (size_t)s * LL;
      const int col = (p + off1) & (L - 1);
#pragma unroll
      for (int i = 0; i < L; ++i) {
        const int w = ((i + off0) & (L - 1)) * L + col;
        const V2 q = ps[w];
        const T l = ls[w];
        V2 r; r.x = xr[i] + l * q.x; r.y = xi[i] + l * q.y;
        store_streaming(out + w, r);
      }
    }
  }
  if (!ok) {
    // record the timeout, then give the copies still in flight a bounded time to land (the
    // full bound, whatever a.spin is)
    if (lane == 0) atomicExch(err, kApplyTimeout);
    if (psi_pending) mbar_wait(smem_addr(&bars[warp][STAGES]), (uint32_t)(k & 1));
    for (; k < kp; ++k) mbar_wait(smem_addr(&bars[warp][k % STAGES]), (uint32_t)((k / STAGES) & 1));
  }
}

// Swizzled column of group point (k, a) of tile column c: a ^ f(c, k), a bijection in a.
template <int C, int G>
__device__ __forceinline__ int pencil_sw(int a, int c, int k) {
  if constexpr (C >= G) return a ^ (c & (G - 1));
  else return a ^ (c * (G / C)) ^ (k & (G / C - 1));
}

// Pass B (in place) on a tile of C consecutive slice positions x all LII^2 k_II points.
// Thread (a, c) first holds the pencil along k_II axis 0 at axis-1 window coordinate a; after
// the transpose, thread (k, c) holds the pencil along k_II axis 1 at axis-0 grid index k.
template <typename T, int L, int C, typename U = T>
__global__ void __launch_bounds__(C * L) pencil_b_kernel(PencilArgs a) {
  using V2 = typename Vec2<T>::type;
  using SC = typename SmemCplx<U>::type;
  static_assert(sizeof(SC) == sizeof(V2) && sizeof(U) == sizeof(T), "shared-memory sizes");
  constexpr int LL = L * L, H = L / 2, G = wave_lanes<T>();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  SC* S = reinterpret_cast<SC*>(smem_raw);
  U* vI = reinterpret_cast<U*>(S + C * LL);   // C slice positions
  U* v0 = vI + C;                             // k_II axis 0 table (L)
  U* v1 = v0 + L;                             // k_II axis 1 table (L)
  const int c = threadIdx.x % C, ta = threadIdx.x / C;
  const long long c0 = (long long)blockIdx.x * C;
  const int vec = blockIdx.y;
  if (pencil_skip(a, vec)) return;
  const int prob = a.pot.vecs_per_prob > 0 ? (a.vec_base + vec) / a.pot.vecs_per_prob : 0;
  const int LI = a.MI == 256 ? 16 : 32;
  if (a.pot.kind == 1) {
    const long long tb = (long long)prob * a.pot.tab_stride;
    if (threadIdx.x < C) {
      const int pos = (int)(c0 + threadIdx.x);      // slice layout: pos = l1 * LI + l0
      ld_u(pot_const<T>(a.pot) + pot_tab<T>(a.pot, tb + a.pot.tab_off[0] + pos % LI) +
               pot_tab<T>(a.pot, tb + a.pot.tab_off[1] + pos / LI), vI[threadIdx.x]);
    } else if (threadIdx.x < C + L) {
      const int l = threadIdx.x - C;
      ld_u(pot_tab<T>(a.pot, tb + a.pot.tab_off[2] + l), v0[l]);
    } else if (threadIdx.x < C + 2 * L) {
      const int l = threadIdx.x - C - L;
      ld_u(pot_tab<T>(a.pot, tb + a.pot.tab_off[3] + l), v1[l]);
    }
  }
  // in place (a.in == a.out): every load of the tile precedes the first barrier, every store
  // follows the second
  V2* col = reinterpret_cast<V2*>(a.out) + (size_t)vec * a.ld + c0 + c + (size_t)ta * a.MI;
  const int rstride = L * (int)a.MI;              // k_II axis 0 stride (N < 2^31 on this path)
  // Shared-memory indices. Element (k, a) of column c sits at c*LL + k*L + (a ^ f(c, k)),
  // f = pencil_sw(0, c, k). Both index families below are one XOR with an immediate on a
  // thread constant; the constants are made opaque before each loop so that the compiler
  // recomputes the 32 indices instead of keeping them live across the DFTs.
  constexpr int M = (C >= G) ? 0 : G / C - 1;     // bits of k that enter f
  int t0 = c * LL + pencil_sw<C, G>(ta, c, 0);     // (i, ta): (t0 ^ (i & M)) + i * L
  U xr[L], xi[L];
  // grid index i along k_II axis 0 sits at window row (i + L/2) mod L (roll by L_j)
#pragma unroll
  for (int i = 0; i < L; ++i) {
    const V2 v = col[((i + H) & (L - 1)) * rstride];
    ld_u(v.x, xr[i]); ld_u(v.y, xi[i]);
  }
  Dft<L, +1, U>::run(xr, xi);
#pragma unroll
  for (int i = 0; i < L; ++i) {
    S[(t0 ^ (i & M)) + i * L] = mkc(xr[i], xi[i]);
  }
  __syncthreads();
  const int k = ta;
  int r1 = (c * LL + k * L) | pencil_sw<C, G>(0, c, k);   // (k, a): r1 ^ a
#pragma unroll
  for (int j = 0; j < L; ++j) {
    unc(S[r1 ^ ((j + H) & (L - 1))], xr[j], xi[j]);
  }
  Dft<L, +1, U>::run(xr, xi);
  // x V(y_l) / N at l_II = (k, j) and the tile column's k_I grid point
  if (a.pot.kind == 1) {
    const U base = vI[c] + v0[k];
#pragma unroll
    for (int j = 0; j < L; ++j) { const U v = base + v1[j]; xr[j] = xr[j] * v; xi[j] = xi[j] * v; }
  } else {
    const int pos = (int)(c0 + c);
    const long long lI = (long long)(pos % LI) * LI + pos / LI;   // natural k_I order
#pragma unroll
    for (int j = 0; j < L; ++j) {
      U v;
      ld_u(pot_grid<T>(a.pot, (long long)(k * L + j) * a.MI + lI), v);
      xr[j] = xr[j] * v; xi[j] = xi[j] * v;
    }
  }
  Dft<L, -1, U>::run(xr, xi);
  asm volatile("" : "+r"(r1));
#pragma unroll
  for (int j = 0; j < L; ++j) {
    S[r1 ^ ((j + H) & (L - 1))] = mkc(xr[j], xi[j]);
  }
  __syncthreads();
  asm volatile("" : "+r"(t0));
#pragma unroll
  for (int i = 0; i < L; ++i) {
    unc(S[(t0 ^ (i & M)) + i * L], xr[i], xi[i]);
  }
  Dft<L, -1, U>::run(xr, xi);
  // make the tile pointer opaque so that the load addresses are recomputed here instead of
  // being kept live across the DFTs
  asm volatile("" : "+l"(col));
#pragma unroll
  for (int i = 0; i < L; ++i) {
    V2 v; v.x = st_t(xr[i]); v.y = st_t(xi[i]);
    col[((i + H) & (L - 1)) * rstride] = v;
  }
}

// Per-device flag for the twiddle tables, guarded by a mutex so that first calls from several
// host threads fill the tables once. The flags assume the device's primary context is never
// reset while the library is loaded.
std::mutex g_tw_mu;
bool g_tw_ready[64] = {};

iwf_status init_twiddles(int device) {
  std::lock_guard<std::mutex> lock(g_tw_mu);
  if (device >= 0 && device < 64 && g_tw_ready[device]) return IWF_OK;
  std::vector<double2> h64(kTwTotal);
  std::vector<float2> h32(kTwTotal);
  std::vector<float4> hdf(kTwTotal);
  const long double two_pi = 6.283185307179586476925286766559005768L;
  for (int len = 1; len <= IWF_MAX_LEN; ++len) {
    for (int j = 0; j < len; ++j) {
      long double c, s;
      if (j == 0) { c = 1; s = 0; }
      else if (2 * j == len) { c = -1; s = 0; }
      else if (4 * j == len) { c = 0; s = 1; }
      else if (4 * j == 3 * len) { c = 0; s = -1; }
      else { const long double t = two_pi * j / len; c = cosl(t); s = sinl(t); }
      h64[tw_off(len) + j] = make_double2((double)c, (double)s);
      h32[tw_off(len) + j] = make_float2((float)c, (float)s);
      const float ch = (float)c, sh = (float)s;
      hdf[tw_off(len) + j] = make_float4(ch, (float)(c - (long double)ch), sh,
                                         (float)(s - (long double)sh));
    }
  }
  IWF_CUDA(cudaMemcpyToSymbol(c_tw64, h64.data(), sizeof(double2) * kTwTotal));
  IWF_CUDA(cudaMemcpyToSymbol(c_tw32, h32.data(), sizeof(float2) * kTwTotal));
  IWF_CUDA(cudaMemcpyToSymbol(c_twdf, hdf.data(), sizeof(float4) * kTwTotal));
  if (device >= 0 && device < 64) g_tw_ready[device] = true;
  return IWF_OK;
}

// Values per thread the group's long axes allow for a stage (0: no axis above IWF_MAX_LEN).
int long_group_values(const PassArgs& a) {
  bool any = false;
  for (int ax = 0; ax < a.grp.ng; ++ax) any = any || a.grp.len[ax] > IWF_MAX_LEN;
  if (!any) return 0;
  int v = 16;
  for (int ax = 0; ax < a.grp.ng; ++ax) {
    const int w = long_axis_values(a.grp.len[ax]);
    v = w < v ? w : v;
  }
  return v;
}

// Choose C (inner chunk) and Ot (outer indices) for a group pass within tile_kb of smem.
template <typename T>
void choose_tile(PassArgs& a, int tile_kb) {
  // pass B (inner > 1) also keeps its group's V table (M values) next to the tile
  long long kb = (long long)tile_kb * 1024 - (a.inner > 1 ? (long long)a.M * sizeof(T) : 0);
  if (kb < 0) kb = 0;
  size_t budget = (size_t)kb / sizeof(typename Vec2<T>::type) * 32 / 33;
  // a group with a long axis keeps every value of a shared-memory FFT stage in registers
  const int vmin = long_group_values(a);
  if (vmin > 0 && budget > (size_t)vmin * kLongThreads) budget = (size_t)vmin * kLongThreads;
  if (a.inner == 1) {
    a.C = 1;
    long long ot = (long long)(budget / a.M);
    ot = ot < 1 ? 1 : ot;
    // keep several tiles per SM worth of parallelism
    const long long want = (a.outer + 4 * 152 - 1) / (4 * 152);
    if (ot > want) ot = want < 1 ? 1 : want;
    if (ot > 64) ot = 64;
    a.Ot = (int)ot;
  } else {
    a.Ot = 1;
    long long c = (long long)(budget / a.M);
    if (c > a.inner) c = a.inner;
    // largest power of two <= c that divides inner, so chunks tile the inner range exactly
    long long p = 1;
    while (p * 2 <= c && a.inner % (p * 2) == 0) p *= 2;
    a.C = (int)p;
  }
  a.lc = 0;
  while ((1 << a.lc) < a.C) ++a.lc;
  a.tiles_inner = a.inner / a.C;
}

// Closes the event pair opened before a launch and adds the elapsed time to pass `kind`.
iwf_status stop_timer(PassTimer* timer, int kind, cudaStream_t stream) {
  IWF_CUDA(cudaEventRecord(timer->ev[1], stream));
  IWF_CUDA(cudaEventSynchronize(timer->ev[1]));
  float ms = 0.f;
  IWF_CUDA(cudaEventElapsedTime(&ms, timer->ev[0], timer->ev[1]));
  timer->ms[kind] += ms;
  timer->launches[kind] += 1;
  return IWF_OK;
}

// tkind: the pass (0 A, 1 B, 2 C) whose time the launch counts toward (-1: its own KIND)
template <typename T, int KIND>
iwf_status launch_pass(PassArgs a, int nvec, cudaStream_t stream, PassTimer* timer, int threads,
                       int tkind = -1) {
  const size_t elems = (size_t)a.Ot * a.M * a.C;
  const size_t tbytes = ((elems + elems / 32 + 1) * sizeof(typename Vec2<T>::type) + 15) / 16 * 16;
  a.tile_bytes = (int)tbytes;
  const size_t bytes = tbytes + (KIND == 1 ? (size_t)(a.M + a.C) * sizeof(T) : 0);
  if (bytes > 200 * 1024) return fail(IWF_ERR_UNSUPPORTED, "apply: tile exceeds shared memory");
  const int vmin = long_group_values(a);
  if (vmin > 0) {
    threads = kLongThreads;
    if (elems > (size_t)vmin * kLongThreads)
      return fail(IWF_ERR_UNSUPPORTED, "apply: axis group too large for the shared-memory FFT");
  }
  static bool attr_set[2][4][2] = {};
  const int ti = sizeof(T) == 8 ? 0 : 1;
  const int li = vmin > 0 ? 1 : 0;
  auto kern = vmin > 0 ? pass_long_kernel<T, KIND> : pass_kernel<T, KIND>;
  if (!attr_set[ti][KIND][li]) {
    IWF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set[ti][KIND][li] = true;
  }
  const long long tiles = ((a.outer + a.Ot - 1) / a.Ot) * a.tiles_inner;
  dim3 grid((unsigned)tiles, (unsigned)nvec);
  if (timer) IWF_CUDA(cudaEventRecord(timer->ev[0], stream));
  kern<<<grid, threads, bytes, stream>>>(a);
  IWF_CUDA(cudaGetLastError());
  count_launch();
  return timer ? stop_timer(timer, tkind >= 0 ? tkind : KIND, stream) : IWF_OK;
}

// Whether pass B's whole k_II group fits one shared-memory tile (else it runs per axis).
template <typename T>
bool group_fits(const PassArgs& a) {
  const size_t el = sizeof(typename Vec2<T>::type);
  const size_t tbytes = ((size_t)a.M + a.M / 32 + 1) * el + (size_t)(a.M + 1) * sizeof(T);
  if (tbytes > 200 * 1024) return false;
  const int vmin = long_group_values(a);
  return vmin == 0 || (size_t)a.M <= (size_t)vmin * kLongThreads;
}

// Pencil path: two k_I axes of one length and two k_II axes of one length, each 16 or 32.
bool pencil_geometry(const Geom& g, int* LI, int* LII) {
  if (g.n != 4 || g.d != 2) return false;
  if (g.lens[0] != g.lens[1] || g.lens[2] != g.lens[3]) return false;
  const auto ok = [](int l) { return l == 16 || l == 32; };
  if (!ok(g.lens[0]) || !ok(g.lens[2])) return false;
  *LI = g.lens[0];
  *LII = g.lens[2];
  return true;
}

// Threads of a pass A/C CTA and tile columns of a pass B CTA: 64 KB of shared memory each.
template <typename T> constexpr int pencil_threads() { return sizeof(T) == 4 ? 256 : 128; }

// Raises the kernel's dynamic shared-memory limit on the current device to `bytes` when the
// limit set so far (allowed[dev], per kernel and device) is smaller.
template <typename K>
iwf_status allow_smem(K* kernel, size_t bytes, size_t* allowed) {
  int dev = 0;
  IWF_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(IWF_ERR_ARG, "device ordinal out of range");
  if (allowed[dev] < bytes) {
    IWF_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    allowed[dev] = bytes;
  }
  return IWF_OK;
}

// Pipelined pass C configuration: 2 warps per CTA, 2 stages per warp (56 KB with the psi and
// Lambda buffers for complex float at L = 32: four CTAs per SM).
constexpr int kPipeWarps = 2, kPipeStages = 2;

// Resident CTAs of `kernel` on the current device times its SM count, cached per device for
// the shared-memory size it was computed with.
struct OccCache {
  size_t smem[64] = {};
  int ctas[64] = {};
};
template <typename K>
iwf_status persistent_ctas(K* kernel, int threads, size_t smem, OccCache* cache, int* out) {
  int dev = 0;
  IWF_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(IWF_ERR_ARG, "device ordinal out of range");
  if (!cache->ctas[dev] || cache->smem[dev] != smem) {
    int per_sm = 0, sms = 0;
    IWF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem));
    IWF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (per_sm < 1) return fail(IWF_ERR_UNSUPPORTED, "pencil pass: kernel does not fit an SM");
    cache->ctas[dev] = per_sm * sms;
    cache->smem[dev] = smem;
  }
  *out = cache->ctas[dev];
  return IWF_OK;
}

// Which pass A/C kernel runs: the pipelined one for complex-float pass C, whose psi and Lambda
// loads it takes off the critical path; the direct one elsewhere (pass A, where it measured
// no faster, and complex double, whose larger stages would leave too few warps for the FP64
// units).
template <typename T, int KIND> constexpr bool use_pipe() { return sizeof(T) == 4 && KIND == 2; }

template <typename T, int L, int KIND, typename U = T>
iwf_status launch_pencil_direct(const PencilArgs& a, int nvec, cudaStream_t stream,
                                PassTimer* timer) {
  using V2 = typename Vec2<T>::type;
  constexpr int threads = pencil_threads<T>();
  constexpr int per_cta = threads / 32 * (32 / L);          // slices per CTA
  const size_t smem = (size_t)threads * L * sizeof(V2);
  static size_t allowed[64] = {};
  IWF_TRY(allow_smem(pencil_ac_kernel<T, L, KIND, U>, smem, allowed));
  dim3 grid((unsigned)((a.MII + per_cta - 1) / per_cta), (unsigned)nvec);
  if (timer) IWF_CUDA(cudaEventRecord(timer->ev[0], stream));
  pencil_ac_kernel<T, L, KIND, U><<<grid, threads, smem, stream>>>(a);
  IWF_CUDA(cudaGetLastError());
  count_launch();
  return timer ? stop_timer(timer, KIND, stream) : IWF_OK;
}

template <typename T, int L>
iwf_status launch_pencil_c_pipe(const PencilArgs& a, int nvec, int* err, cudaStream_t stream,
                                PassTimer* timer) {
  constexpr int W = kPipeWarps, SPW = 32 / L;
  const auto kernel = pencil_c_pipe_kernel<T, L, W, kPipeStages>;
  const size_t smem = (size_t)W * pipe_warp_bytes<T>(L, kPipeStages);
  static size_t allowed[64] = {};
  static OccCache occ;
  IWF_TRY(allow_smem(kernel, smem, allowed));
  int max_ctas = 0;
  IWF_TRY(persistent_ctas(kernel, W * 32, smem, &occ, &max_ctas));
  if (a.MII % SPW) return fail(IWF_ERR_UNSUPPORTED, "pencil pass: slices not a multiple of a unit");
  const long long units = a.MII / SPW * nvec;
  const long long want = (units + W - 1) / W;
  const unsigned grid = (unsigned)(want < max_ctas ? want : max_ctas);
  if (timer) IWF_CUDA(cudaEventRecord(timer->ev[0], stream));
  kernel<<<grid, W * 32, smem, stream>>>(a, nvec, err);
  IWF_CUDA(cudaGetLastError());
  count_launch();
  return timer ? stop_timer(timer, 2, stream) : IWF_OK;
}

template <typename T, int L, int KIND, typename U = T>
iwf_status launch_pencil_ac(const PencilArgs& a, int nvec, int* err, cudaStream_t stream,
                            PassTimer* timer) {
  if constexpr (use_pipe<T, KIND>()) return launch_pencil_c_pipe<T, L>(a, nvec, err, stream, timer);
  else return launch_pencil_direct<T, L, KIND, U>(a, nvec, stream, timer);
}

template <typename T, int L, typename U = T>
iwf_status launch_pencil_b(const PencilArgs& a, int nvec, cudaStream_t stream, PassTimer* timer) {
  using V2 = typename Vec2<T>::type;
  constexpr int C = pencil_threads<T>() / L;
  const size_t smem = (size_t)C * L * L * sizeof(V2) + (size_t)(C + 2 * L) * sizeof(T);
  static size_t allowed[64] = {};
  IWF_TRY(allow_smem(pencil_b_kernel<T, L, C, U>, smem, allowed));
  if (a.MI % C) return fail(IWF_ERR_UNSUPPORTED, "pencil pass B: slice not a multiple of the tile");
  dim3 grid((unsigned)(a.MI / C), (unsigned)nvec);
  if (timer) IWF_CUDA(cudaEventRecord(timer->ev[0], stream));
  pencil_b_kernel<T, L, C, U><<<grid, C * L, smem, stream>>>(a);
  IWF_CUDA(cudaGetLastError());
  count_launch();
  return timer ? stop_timer(timer, 1, stream) : IWF_OK;
}

// One chunk of vectors through the three pencil passes (DFTs in the compute type U).
template <typename T, typename U = T>
iwf_status pencil_chunk(PencilArgs a, int LI, int LII, const void* in, void* wk, void* out,
                        const void* lam, int nv, int* err, cudaStream_t stream, PassTimer* timer) {
  a.in = in; a.out = wk;
  IWF_TRY(LI == 16 ? (launch_pencil_ac<T, 16, 0, U>(a, nv, err, stream, timer))
                   : (launch_pencil_ac<T, 32, 0, U>(a, nv, err, stream, timer)));
  a.in = wk; a.out = wk;
  IWF_TRY(LII == 16 ? (launch_pencil_b<T, 16, U>(a, nv, stream, timer))
                    : (launch_pencil_b<T, 32, U>(a, nv, stream, timer)));
  a.in = wk; a.out = out; a.psi = in; a.lam = lam;
  return LI == 16 ? launch_pencil_ac<T, 16, 2, U>(a, nv, err, stream, timer)
                  : launch_pencil_ac<T, 32, 2, U>(a, nv, err, stream, timer);
}

template <typename T>
iwf_status apply_typed(iwf_plan* p, const void* psi, void* hpsi, int nvec, cudaStream_t stream,
                       PassTimer* timer, void* ext_work = nullptr, size_t ext_bytes = 0,
                       const ApplyBatch* batch = nullptr) {
  using V2 = typename Vec2<T>::type;
  const Geom& g = p->g;
  const int d = g.d, n = g.n;
  const int ti = sizeof(T) == 8 ? 0 : 1;
  const int threads = p->tune_threads[ti], tile_kb = p->tune_tile_kb[ti];
  // chunk of vectors whose intermediate block fits comfortably in L2
  const size_t vbytes = (size_t)g.N * sizeof(V2);
  int chunk = (int)(((size_t)p->tune_chunk_mb[ti] << 20) / vbytes);
  if (chunk < 1) chunk = 1;
  if (chunk > nvec) chunk = nvec;
  if (chunk > 65535) chunk = 65535;
  void* work = ext_work;
  if (ext_work) {
    const int fit = (int)(ext_bytes / vbytes);
    if (fit < 1) return fail(IWF_ERR_UNSUPPORTED, "caller workspace smaller than one vector");
    if (chunk > fit) chunk = fit;
  } else {
    IWF_TRY(ensure_workspace(p, vbytes * chunk));
    work = p->d_work;
  }

  PotDev pot{};
  pot.kind = p->pot_kind;
  for (int j = 0; j < n; ++j) pot.tab_off[j] = p->tab_off[j];
  pot.tab64 = p->d_tab64; pot.tab32 = p->d_tab32;
  pot.grid64 = p->d_grid64; pot.grid32 = p->d_grid32;
  pot.c64 = p->vconst / (double)g.N;
  pot.c32 = (float)pot.c64;
  if (batch) {
    // batch tables: axis j's table follows axes 0..j-1 (lens[0] + ... + lens[j-1])
    int off = 0;
    for (int j = 0; j < n; ++j) { pot.tab_off[j] = off; off += g.lens[j]; }
    pot.kind = 1;
    pot.tab64 = batch->tab64; pot.tab32 = batch->tab32;
    pot.c64 = 0.0; pot.c32 = 0.f;             // folded into the tables
    pot.tab_stride = batch->tab_stride;
    pot.vecs_per_prob = batch->vecs_per_prob;
    pot.active = batch->active;
  }

  PassArgs A{};
  A.g = g; A.lo = p->d_lo; A.ld = g.N; A.pot = pot;
  A.grp.ng = d; A.M = (int)g.MI; A.inner = 1; A.outer = g.MII;
  for (int j = 0; j < d; ++j) { A.grp.len[j] = g.lens[j]; A.grp.kI[j] = j; A.grp.Lroll[j] = 0; }
  {
    int s = 1;
    for (int j = d - 1; j >= 0; --j) { A.grp.gs[j] = s; s *= g.lens[j]; }
  }
  for (int j = 0; j < d; ++j)
    A.ltw[j] = sizeof(T) == 8 ? (const void*)p->d_ltw64[j] : (const void*)p->d_ltw32[j];
  choose_tile<T>(A, tile_kb);

  PassArgs B{};
  B.g = g; B.lo = p->d_lo; B.ld = g.N; B.pot = pot;
  B.grp.ng = n - d; B.M = (int)g.MII; B.inner = g.MI; B.outer = 1;
  for (int j = 0; j < n - d; ++j) {
    B.grp.len[j] = g.lens[d + j]; B.grp.kI[j] = -1; B.grp.Lroll[j] = g.half[d + j];
  }
  {
    int s = 1;
    for (int j = n - d - 1; j >= 0; --j) { B.grp.gs[j] = s; s *= g.lens[d + j]; }
  }
  for (int j = 0; j < n - d; ++j)
    B.ltw[j] = sizeof(T) == 8 ? (const void*)p->d_ltw64[d + j] : (const void*)p->d_ltw32[d + j];
  B.ii0 = 0;
  // a k_II group too large for one tile: one pass per k_II axis (slower axes outer, faster
  // axes and the k_I slice inner)
  const bool split = !group_fits<T>(B);
  PassArgs Bs[IWF_MAX_N];
  if (split) {
    long long outer = 1;
    for (int j = 0; j < n - d; ++j) {
      PassArgs& q = Bs[j];
      q = B;
      q.grp.ng = 1;
      q.grp.len[0] = g.lens[d + j]; q.grp.gs[0] = 1; q.grp.kI[0] = -1; q.grp.Lroll[0] = g.half[d + j];
      q.ltw[0] = B.ltw[j];
      q.M = g.lens[d + j];
      q.outer = outer;
      q.inner = g.MII / outer / g.lens[d + j] * g.MI;
      q.ii0 = j;
      outer *= g.lens[d + j];
      choose_tile<T>(q, tile_kb);
    }
  } else {
    choose_tile<T>(B, tile_kb);
  }

  PassArgs Cp = A;
  Cp.lam = sizeof(T) == 8 ? (const void*)p->d_lam64 : (const void*)p->d_lam32;

  int LI = 0, LII = 0;
  if (p->path[ti] != IWF_PATH_TILED && pencil_geometry(g, &LI, &LII)) {
    // pencil geometry: N = LI^2 LII^2 <= 2^20, so in-vector offsets fit in int
    PencilArgs pa{};
    pa.lo = p->d_lo; pa.pot = pot; pa.ld = g.N; pa.MI = g.MI; pa.MII = g.MII;
    pa.spin = p->wait_rounds >= 0 ? p->wait_rounds : kSpinRounds;
    for (int v0 = 0; v0 < nvec; v0 += chunk) {
      const int nv = nvec - v0 < chunk ? nvec - v0 : chunk;
      pa.vec_base = v0;
      const void* cin = reinterpret_cast<const V2*>(psi) + (size_t)v0 * g.N;
      void* cout = reinterpret_cast<V2*>(hpsi) + (size_t)v0 * g.N;
      if constexpr (sizeof(T) == 8) {
        if (p->fft_arith == IWF_ARITH_DF) {
          IWF_TRY((pencil_chunk<T, dfl>(pa, LI, LII, cin, work, cout, Cp.lam, nv, p->d_apply_err,
                                        stream, timer)));
          continue;
        }
      }
      IWF_TRY(pencil_chunk<T>(pa, LI, LII, cin, work, cout, Cp.lam, nv, p->d_apply_err, stream,
                              timer));
    }
    return IWF_OK;
  }

  for (int v0 = 0; v0 < nvec; v0 += chunk) {
    const int nv = nvec - v0 < chunk ? nvec - v0 : chunk;
    const V2* in = reinterpret_cast<const V2*>(psi) + (size_t)v0 * g.N;
    V2* out = reinterpret_cast<V2*>(hpsi) + (size_t)v0 * g.N;
    V2* wk = reinterpret_cast<V2*>(work);
    A.vec_base = v0; B.vec_base = v0; Cp.vec_base = v0;
    A.in = in; A.out = wk;
    IWF_TRY((launch_pass<T, 0>(A, nv, stream, timer, threads)));
    if (split) {
      const int m = n - d;
      for (int j = 0; j < m; ++j) { Bs[j].vec_base = v0; Bs[j].in = wk; Bs[j].out = wk; }
      for (int j = 0; j + 1 < m; ++j) IWF_TRY((launch_pass<T, 0>(Bs[j], nv, stream, timer, threads, 1)));
      IWF_TRY((launch_pass<T, 1>(Bs[m - 1], nv, stream, timer, threads)));
      for (int j = m - 2; j >= 0; --j) IWF_TRY((launch_pass<T, 3>(Bs[j], nv, stream, timer, threads, 1)));
    } else {
      B.in = wk; B.out = wk;
      IWF_TRY((launch_pass<T, 1>(B, nv, stream, timer, threads)));
    }
    Cp.in = wk; Cp.out = out; Cp.psi = in;
    IWF_TRY((launch_pass<T, 2>(Cp, nv, stream, timer, threads)));
  }
  return IWF_OK;
}

}  // namespace

namespace {
std::atomic<long long> g_launches{0};
}
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

// True when the nvec-vector blocks at psi and hpsi share any byte.
static bool blocks_overlap(const iwf_plan* p, int precision, const void* psi, const void* hpsi,
                           int nvec) {
  const uintptr_t bytes = (uintptr_t)p->g.N * nvec * (precision == IWF_PREC_F64 ? 16 : 8);
  const uintptr_t a = reinterpret_cast<uintptr_t>(psi), b = reinterpret_cast<uintptr_t>(hpsi);
  return a < b + bytes && b < a + bytes;
}

iwf_status apply_impl(iwf_plan* p, int precision, const void* psi, void* hpsi, int nvec,
                      cudaStream_t stream, PassTimer* timer, const ApplyBatch* batch) {
  if (nvec < 0) return fail(IWF_ERR_ARG, "iwf_apply: nvec < 0");
  if (nvec == 0) return IWF_OK;
  if (!psi || !hpsi) return fail(IWF_ERR_ARG, "iwf_apply: null vector pointer");
  if ((reinterpret_cast<uintptr_t>(psi) | reinterpret_cast<uintptr_t>(hpsi)) & 15)
    return fail(IWF_ERR_ARG, "iwf_apply: vectors must be 16-byte aligned");
  if (p->pot_kind == 0 && !batch) return fail(IWF_ERR_ARG, "iwf_apply: no potential set");
  if (nvec > 65535) return fail(IWF_ERR_ARG, "iwf_apply: nvec > 65535");
  if (blocks_overlap(p, precision, psi, hpsi, nvec))
    return fail(IWF_ERR_ARG, "iwf_apply: psi and hpsi overlap");
  IWF_TRY(init_twiddles(p->device));
  if (precision == IWF_PREC_F64)
    return apply_typed<double>(p, psi, hpsi, nvec, stream, timer, nullptr, 0, batch);
  if (precision == IWF_PREC_C64)
    return apply_typed<float>(p, psi, hpsi, nvec, stream, timer, nullptr, 0, batch);
  return fail(IWF_ERR_ARG, "iwf_apply: unknown precision");
}

// ---------------------------------------------------------------------------------------
// Schedule autotuner: time the apply of an nvec block for every candidate (threads per CTA,
// shared-memory tile budget, L2 chunk) and keep the fastest for this plan and precision.
iwf_status autotune_impl(iwf_plan* p, int precision, int nvec, double* best_ms, int* best,
                         cudaStream_t stream) {
  if (precision != IWF_PREC_F64 && precision != IWF_PREC_C64)
    return fail(IWF_ERR_ARG, "iwf_plan_autotune: unknown precision");
  if (p->pot_kind == 0) return fail(IWF_ERR_ARG, "iwf_plan_autotune: no potential set");
  if (nvec < 1 || nvec > 65535) return fail(IWF_ERR_ARG, "iwf_plan_autotune: bad nvec");
  const int ti = precision == IWF_PREC_F64 ? 0 : 1;
  const size_t elt = precision == IWF_PREC_F64 ? 16 : 8;
  const size_t bytes = (size_t)p->g.N * nvec * elt;
  void *x = nullptr, *y = nullptr;
  if (cudaMalloc(&x, bytes) != cudaSuccess) return fail(IWF_ERR_ALLOC, "autotune buffers");
  if (cudaMalloc(&y, bytes) != cudaSuccess) { cudaFree(x); return fail(IWF_ERR_ALLOC, "autotune buffers"); }
  cudaMemsetAsync(x, 0, bytes, stream);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int threads[] = {128, 256};
  const int tiles[] = {24, 48, 96, 160};
  const int chunks[] = {24, 48, 96};
  const int pencil_chunks[] = {12, 24, 48, 96};
  double best_t = 1e30;
  int bt = p->tune_threads[ti], bk = p->tune_tile_kb[ti], bc = p->tune_chunk_mb[ti];
  int bp = IWF_PATH_TILED;
  const int saved_path = p->path[ti];
  iwf_status st = IWF_OK;
  // times one candidate (the plan already holds it); keeps it if it is the fastest so far
  const auto trial = [&](int path, int th, int tk, int ch) {
    if (st != IWF_OK) return;
    p->path[ti] = path;
    p->tune_threads[ti] = th; p->tune_tile_kb[ti] = tk; p->tune_chunk_mb[ti] = ch;
    st = apply_impl(p, precision, x, y, nvec, stream);             // warm-up (and workspace)
    if (st != IWF_OK) return;
    cudaEventRecord(e0, stream);
    for (int r = 0; r < 3 && st == IWF_OK; ++r) st = apply_impl(p, precision, x, y, nvec, stream);
    cudaEventRecord(e1, stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) { st = fail(IWF_ERR_CUDA, "autotune timing"); return; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms / 3 < best_t) { best_t = ms / 3; bt = th; bk = tk; bc = ch; bp = path; }
  };
  // double-float DFTs exist on the pencil path only: no tiled candidates then
  const bool df_only = precision == IWF_PREC_F64 && p->fft_arith == IWF_ARITH_DF;
  if (saved_path != IWF_PATH_PENCIL && !df_only)
    for (int th : threads)
      for (int tk : tiles)
        for (int ch : chunks) trial(IWF_PATH_TILED, th, tk, ch);
  int LI = 0, LII = 0;
  if (saved_path != IWF_PATH_TILED && pencil_geometry(p->g, &LI, &LII))
    for (int ch : pencil_chunks) trial(IWF_PATH_PENCIL, p->tune_threads[ti], p->tune_tile_kb[ti], ch);
  p->tune_threads[ti] = bt; p->tune_tile_kb[ti] = bk; p->tune_chunk_mb[ti] = bc;
  p->path[ti] = bp;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(x);
  cudaFree(y);
  if (st != IWF_OK) { p->path[ti] = saved_path; return st; }
  if (best_ms) *best_ms = best_t;
  if (best) {
    best[0] = bp == IWF_PATH_PENCIL ? 0 : bt;
    best[1] = bp == IWF_PATH_PENCIL ? 0 : bk;
    best[2] = bc;
  }
  return IWF_OK;
}

// exp(2 pi i j / len), j < len, in FP64 and FP32 (rounded from long double; the quarter
// points are exact) for every axis of an axis group (k_I or k_II) that has an axis longer
// than IWF_MAX_LEN: such groups run the shared-memory FFT on all their axes.
iwf_status build_long_twiddles(iwf_plan* p) {
  const long double two_pi = 6.283185307179586476925286766559005768L;
  bool long_grp[2] = {false, false};
  for (int j = 0; j < p->g.n; ++j)
    if (p->g.lens[j] > IWF_MAX_LEN) long_grp[j < p->g.d ? 0 : 1] = true;
  for (int j = 0; j < p->g.n; ++j) {
    const int len = p->g.lens[j];
    if (!long_grp[j < p->g.d ? 0 : 1]) continue;
    std::vector<double2> h64(len);
    std::vector<float2> h32(len);
    for (int e = 0; e < len; ++e) {
      long double c, sn;
      if (e == 0) { c = 1; sn = 0; }
      else if (2 * e == len) { c = -1; sn = 0; }
      else if (4 * e == len) { c = 0; sn = 1; }
      else if (4 * e == 3 * len) { c = 0; sn = -1; }
      else { const long double t = two_pi * e / len; c = cosl(t); sn = sinl(t); }
      h64[e] = make_double2((double)c, (double)sn);
      h32[e] = make_float2((float)c, (float)sn);
    }
    IWF_CUDA(cudaMalloc(&p->d_ltw64[j], len * sizeof(double2)));
    IWF_CUDA(cudaMalloc(&p->d_ltw32[j], len * sizeof(float2)));
    IWF_CUDA(cudaMemcpy(p->d_ltw64[j], h64.data(), len * sizeof(double2), cudaMemcpyHostToDevice));
    IWF_CUDA(cudaMemcpy(p->d_ltw32[j], h32.data(), len * sizeof(float2), cudaMemcpyHostToDevice));
  }
  return IWF_OK;
}

iwf_status check_apply_error(iwf_plan* p, cudaStream_t stream) {
  if (!p->d_apply_err) return IWF_OK;
  int err = 0;
  IWF_CUDA(cudaMemcpyAsync(&err, p->d_apply_err, sizeof(int), cudaMemcpyDeviceToHost, stream));
  IWF_CUDA(cudaStreamSynchronize(stream));
  if (err == 0) return IWF_OK;
  IWF_CUDA(cudaMemsetAsync(p->d_apply_err, 0, sizeof(int), stream));
  IWF_CUDA(cudaStreamSynchronize(stream));
  return fail(IWF_ERR_TIMEOUT, "apply: a pipelined pass gave up waiting for a bulk copy");
}

iwf_status set_path_impl(iwf_plan* p, int precision, int path) {
  if (precision != IWF_PREC_F64 && precision != IWF_PREC_C64)
    return fail(IWF_ERR_ARG, "iwf_plan_set_path: unknown precision");
  if (path != IWF_PATH_AUTO && path != IWF_PATH_TILED && path != IWF_PATH_PENCIL)
    return fail(IWF_ERR_ARG, "iwf_plan_set_path: unknown path");
  int LI = 0, LII = 0;
  if (path == IWF_PATH_PENCIL && !pencil_geometry(p->g, &LI, &LII))
    return fail(IWF_ERR_UNSUPPORTED,
                "iwf_plan_set_path: the pencil path needs n = 4, d = 2 and two equal axis "
                "lengths per group, each 16 or 32");
  if (path == IWF_PATH_TILED && precision == IWF_PREC_F64 && p->fft_arith == IWF_ARITH_DF)
    return fail(IWF_ERR_UNSUPPORTED,
                "iwf_plan_set_path: double-float DFTs are set on this plan and need the pencil path");
  p->path[precision == IWF_PREC_F64 ? 0 : 1] = path;
  return IWF_OK;
}

iwf_status set_arith_impl(iwf_plan* p, int arith) {
  if (arith != IWF_ARITH_F64 && arith != IWF_ARITH_DF)
    return fail(IWF_ERR_ARG, "iwf_plan_set_arith: unknown arithmetic");
  int LI = 0, LII = 0;
  if (arith == IWF_ARITH_DF && (!pencil_geometry(p->g, &LI, &LII) || p->path[0] == IWF_PATH_TILED))
    return fail(IWF_ERR_UNSUPPORTED,
                "iwf_plan_set_arith: double-float DFTs need the pencil path (n = 4, d = 2, two "
                "equal axis lengths per group, each 16 or 32)");
  p->fft_arith = arith;
  return IWF_OK;
}

iwf_status get_schedule_impl(const iwf_plan* p, int precision, int* sched) {
  if (precision != IWF_PREC_F64 && precision != IWF_PREC_C64)
    return fail(IWF_ERR_ARG, "iwf_plan_get_schedule: unknown precision");
  if (!sched) return fail(IWF_ERR_ARG, "iwf_plan_get_schedule: NULL output");
  const int ti = precision == IWF_PREC_F64 ? 0 : 1;
  int LI = 0, LII = 0;
  const bool pencil = p->path[ti] != IWF_PATH_TILED && pencil_geometry(p->g, &LI, &LII);
  sched[0] = p->tune_threads[ti];
  sched[1] = p->tune_tile_kb[ti];
  sched[2] = p->tune_chunk_mb[ti];
  sched[3] = pencil ? IWF_PATH_PENCIL : IWF_PATH_TILED;
  return IWF_OK;
}

iwf_status set_schedule_impl(iwf_plan* p, int precision, int threads, int tile_kb, int chunk_mb) {
  if (precision != IWF_PREC_F64 && precision != IWF_PREC_C64)
    return fail(IWF_ERR_ARG, "iwf_plan_set_schedule: unknown precision");
  if ((threads != 128 && threads != 256) || tile_kb < 8 || tile_kb > 200 || chunk_mb < 1)
    return fail(IWF_ERR_ARG, "iwf_plan_set_schedule: threads 128 or 256, tile_kb 8..200, chunk_mb >= 1");
  const int ti = precision == IWF_PREC_F64 ? 0 : 1;
  p->tune_threads[ti] = threads; p->tune_tile_kb[ti] = tile_kb; p->tune_chunk_mb[ti] = chunk_mb;
  return IWF_OK;
}

// ---------------------------------------------------------------------------------------
// Allocation-free apply. The intermediate block lives in a fixed array compiled into this
// library instead of the plan's workspace, so the call never allocates device memory.
// The array is created on every GPU that loads the library and stays until the process
// exits. Its device address is looked up once per device, on that device's first call.
constexpr size_t kStaticScratchBytes = size_t(32) << 20;   // 32 MiB
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace {
std::mutex g_scratch_mu;
void* g_scratch_addr[64] = {};
}  // namespace

// Device address of the fixed array on the current device (the caller makes it current).
static iwf_status static_scratch_address(int device, void** out) {
  if (device < 0 || device >= 64) return fail(IWF_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[device]) {
    void* addr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&addr, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
    g_scratch_addr[device] = addr;
  }
  *out = g_scratch_addr[device];
  return IWF_OK;
}

iwf_status apply_noalloc_impl(iwf_plan* p, int precision, const void* psi, void* hpsi, int nvec,
                              cudaStream_t stream) {
  if (nvec < 0) return fail(IWF_ERR_ARG, "iwf_apply_noalloc: nvec < 0");
  if (nvec == 0) return IWF_OK;
  if (!psi || !hpsi) return fail(IWF_ERR_ARG, "iwf_apply_noalloc: null vector pointer");
  if ((reinterpret_cast<uintptr_t>(psi) | reinterpret_cast<uintptr_t>(hpsi)) & 15)
    return fail(IWF_ERR_ARG, "iwf_apply_noalloc: vectors must be 16-byte aligned");
  if (p->pot_kind == 0) return fail(IWF_ERR_ARG, "iwf_apply_noalloc: no potential set");
  if (nvec > 65535) return fail(IWF_ERR_ARG, "iwf_apply_noalloc: nvec > 65535");
  if (blocks_overlap(p, precision, psi, hpsi, nvec))
    return fail(IWF_ERR_ARG, "iwf_apply_noalloc: psi and hpsi overlap");
  if (precision != IWF_PREC_F64 && precision != IWF_PREC_C64)
    return fail(IWF_ERR_ARG, "iwf_apply_noalloc: unknown precision");
  const size_t elt = precision == IWF_PREC_F64 ? 16 : 8;
  const size_t need = (size_t)p->g.N * elt;
  if (need > kStaticScratchBytes)
    return fail(IWF_ERR_UNSUPPORTED,
                "iwf_apply_noalloc: one vector needs " + std::to_string(need) +
                    " bytes of scratch, above the fixed maximum of " +
                    std::to_string(kStaticScratchBytes) + " bytes");
  void* scratch = nullptr;
  IWF_TRY(static_scratch_address(p->device, &scratch));
  IWF_TRY(init_twiddles(p->device));
  if (precision == IWF_PREC_F64)
    return apply_typed<double>(p, psi, hpsi, nvec, stream, nullptr, scratch, kStaticScratchBytes);
  return apply_typed<float>(p, psi, hpsi, nvec, stream, nullptr, scratch, kStaticScratchBytes);
}

}  // namespace iwf
