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
// Rolls are index permutations inside a pencil and cost no arithmetic. Vectors are processed
// in chunks sized so that the intermediate block stays resident in the 129 MB L2.
#include <atomic>
#include <mutex>
#include <string>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "common.cuh"
#include "dft.cuh"

namespace iwf {

namespace {

constexpr int kThreads = 256;

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

template <typename T> __device__ __forceinline__ T pot_tab(const PotDev& p, long long off);
template <> __device__ __forceinline__ double pot_tab<double>(const PotDev& p, long long off) { return p.tab64[off]; }
template <> __device__ __forceinline__ float pot_tab<float>(const PotDev& p, long long off) { return p.tab32[off]; }
template <typename T> __device__ __forceinline__ T pot_grid(const PotDev& p, long long i);
template <> __device__ __forceinline__ double pot_grid<double>(const PotDev& p, long long i) { return p.grid64[i]; }
template <> __device__ __forceinline__ float pot_grid<float>(const PotDev& p, long long i) { return p.grid32[i]; }
template <typename T> __device__ __forceinline__ T pot_const(const PotDev& p);
template <> __device__ __forceinline__ double pot_const<double>(const PotDev& p) { return p.c64; }
template <> __device__ __forceinline__ float pot_const<float>(const PotDev& p) { return p.c32; }

// KIND 0: pass A, KIND 1: pass B, KIND 2: pass C.
template <typename T, int KIND>
__global__ void __launch_bounds__(kThreads) pass_kernel(PassArgs a) {
  using V2 = typename Vec2<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
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

  for (int t = threadIdx.x; t < Ot * a.grp.ng; t += blockDim.x) {
    const int ot = t / a.grp.ng, ax = t % a.grp.ng;
    s_off[ot * IWF_MAX_N + ax] = roll_off(a, ax, o0 + ot);
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
    for (int ax = 0; ax < a.grp.ng; ++ax) {
      axis_dispatch<T, +1, true, false>(tile, a, ax, o0, s_off);
      __syncthreads();
    }
  } else if (KIND == 1) {
    for (int ax = 0; ax < a.grp.ng; ++ax) {
      axis_dispatch<T, +1, true, false>(tile, a, ax, o0, s_off);
      __syncthreads();
    }
    // multiply by V(y_l)/N: l_II from the group point, l_I from the inner index. With
    // per-axis tables V = [const + sum over k_I axes] + [sum over k_II axes]; both parts are
    // tabulated once per tile (vI over the C inner indices, vII over the M group points).
    if (a.pot.kind == 1) {
      T* vII = reinterpret_cast<T*>(smem_raw + a.tile_bytes);
      T* vI = vII + M;
      const long long tbase = (long long)prob * a.pot.tab_stride;
      for (int c = threadIdx.x; c < C; c += blockDim.x) {
        T v = pot_const<T>(a.pot);
        long long rem = c0 + c;              // inner index -> l_I coordinates (C order)
        for (int j = a.g.d - 1; j >= 0; --j) {
          const int lj = (int)(rem % a.g.lens[j]);
          rem /= a.g.lens[j];
          v += pot_tab<T>(a.pot, tbase + a.pot.tab_off[j] + lj);
        }
        vI[c] = v;
      }
      for (int g = threadIdx.x; g < M; g += blockDim.x) {
        T v = T(0);
        int gr = g;                          // group point -> l_II coordinates
        for (int ax = a.grp.ng - 1; ax >= 0; --ax) {
          const int lj = gr % a.grp.len[ax];
          gr /= a.grp.len[ax];
          v += pot_tab<T>(a.pot, tbase + a.pot.tab_off[a.g.d + ax] + lj);
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
        const T v = pot_grid<T>(a.pot, (long long)(e >> lc) * a.inner + c0 + (e & (C - 1)));
        V2 x = tile[padx(e)];
        x.x *= v; x.y *= v;
        tile[padx(e)] = x;
      }
    }
    __syncthreads();
    for (int ax = 0; ax < a.grp.ng; ++ax) {
      axis_dispatch<T, -1, false, true>(tile, a, ax, o0, s_off);
      __syncthreads();
    }
  } else {
    for (int ax = 0; ax < a.grp.ng; ++ax) {
      axis_dispatch<T, -1, false, true>(tile, a, ax, o0, s_off);
      __syncthreads();
    }
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

bool g_tw_ready[64] = {};

iwf_status init_twiddles(int device) {
  if (device >= 0 && device < 64 && g_tw_ready[device]) return IWF_OK;
  static double2 h64[kTwTotal];
  static float2 h32[kTwTotal];
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
    }
  }
  IWF_CUDA(cudaMemcpyToSymbol(c_tw64, h64, sizeof(h64)));
  IWF_CUDA(cudaMemcpyToSymbol(c_tw32, h32, sizeof(h32)));
  if (device >= 0 && device < 64) g_tw_ready[device] = true;
  return IWF_OK;
}

// Choose C (inner chunk) and Ot (outer indices) for a group pass within tile_kb of smem.
template <typename T>
void choose_tile(PassArgs& a, int tile_kb) {
  // pass B (inner > 1) also keeps its group's V table (M values) next to the tile
  long long kb = (long long)tile_kb * 1024 - (a.inner > 1 ? (long long)a.M * sizeof(T) : 0);
  if (kb < 0) kb = 0;
  const size_t budget = (size_t)kb / sizeof(typename Vec2<T>::type) * 32 / 33;
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

template <typename T, int KIND>
iwf_status launch_pass(PassArgs a, int nvec, cudaStream_t stream, PassTimer* timer, int threads) {
  const size_t elems = (size_t)a.Ot * a.M * a.C;
  const size_t tbytes = ((elems + elems / 32 + 1) * sizeof(typename Vec2<T>::type) + 15) / 16 * 16;
  a.tile_bytes = (int)tbytes;
  const size_t bytes = tbytes + (KIND == 1 ? (size_t)(a.M + a.C) * sizeof(T) : 0);
  if (bytes > 200 * 1024) return fail(IWF_ERR_UNSUPPORTED, "apply: tile exceeds shared memory");
  static bool attr_set[2][3] = {};
  const int ti = sizeof(T) == 8 ? 0 : 1;
  if (!attr_set[ti][KIND]) {
    IWF_CUDA(cudaFuncSetAttribute(pass_kernel<T, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  200 * 1024));
    attr_set[ti][KIND] = true;
  }
  const long long tiles = ((a.outer + a.Ot - 1) / a.Ot) * a.tiles_inner;
  dim3 grid((unsigned)tiles, (unsigned)nvec);
  if (timer) IWF_CUDA(cudaEventRecord(timer->ev[0], stream));
  pass_kernel<T, KIND><<<grid, threads, bytes, stream>>>(a);
  IWF_CUDA(cudaGetLastError());
  count_launch();
  if (timer) {
    IWF_CUDA(cudaEventRecord(timer->ev[1], stream));
    IWF_CUDA(cudaEventSynchronize(timer->ev[1]));
    float ms = 0.f;
    IWF_CUDA(cudaEventElapsedTime(&ms, timer->ev[0], timer->ev[1]));
    timer->ms[KIND] += ms;
    timer->launches[KIND] += 1;
  }
  return IWF_OK;
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
  choose_tile<T>(B, tile_kb);

  PassArgs Cp = A;
  Cp.lam = sizeof(T) == 8 ? (const void*)p->d_lam64 : (const void*)p->d_lam32;

  for (int v0 = 0; v0 < nvec; v0 += chunk) {
    const int nv = nvec - v0 < chunk ? nvec - v0 : chunk;
    const V2* in = reinterpret_cast<const V2*>(psi) + (size_t)v0 * g.N;
    V2* out = reinterpret_cast<V2*>(hpsi) + (size_t)v0 * g.N;
    V2* wk = reinterpret_cast<V2*>(work);
    A.vec_base = v0; B.vec_base = v0; Cp.vec_base = v0;
    A.in = in; A.out = wk;
    IWF_TRY((launch_pass<T, 0>(A, nv, stream, timer, threads)));
    B.in = wk; B.out = wk;
    IWF_TRY((launch_pass<T, 1>(B, nv, stream, timer, threads)));
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

iwf_status apply_impl(iwf_plan* p, int precision, const void* psi, void* hpsi, int nvec,
                      cudaStream_t stream, PassTimer* timer, const ApplyBatch* batch) {
  if (nvec < 0) return fail(IWF_ERR_ARG, "iwf_apply: nvec < 0");
  if (nvec == 0) return IWF_OK;
  if (!psi || !hpsi) return fail(IWF_ERR_ARG, "iwf_apply: null vector pointer");
  if ((reinterpret_cast<uintptr_t>(psi) | reinterpret_cast<uintptr_t>(hpsi)) & 15)
    return fail(IWF_ERR_ARG, "iwf_apply: vectors must be 16-byte aligned");
  if (p->pot_kind == 0 && !batch) return fail(IWF_ERR_ARG, "iwf_apply: no potential set");
  if (nvec > 65535) return fail(IWF_ERR_ARG, "iwf_apply: nvec > 65535");
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
  double best_t = 1e30;
  int bt = p->tune_threads[ti], bk = p->tune_tile_kb[ti], bc = p->tune_chunk_mb[ti];
  iwf_status st = IWF_OK;
  for (int th : threads)
    for (int tk : tiles)
      for (int ch : chunks) {
        if (st != IWF_OK) break;
        p->tune_threads[ti] = th; p->tune_tile_kb[ti] = tk; p->tune_chunk_mb[ti] = ch;
        st = apply_impl(p, precision, x, y, nvec, stream);           // warm-up (and workspace)
        if (st != IWF_OK) break;
        cudaEventRecord(e0, stream);
        for (int r = 0; r < 3 && st == IWF_OK; ++r) st = apply_impl(p, precision, x, y, nvec, stream);
        cudaEventRecord(e1, stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) { st = fail(IWF_ERR_CUDA, "autotune timing"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms / 3 < best_t) { best_t = ms / 3; bt = th; bk = tk; bc = ch; }
      }
  p->tune_threads[ti] = bt; p->tune_tile_kb[ti] = bk; p->tune_chunk_mb[ti] = bc;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(x);
  cudaFree(y);
  if (st != IWF_OK) return st;
  if (best_ms) *best_ms = best_t;
  if (best) { best[0] = bt; best[1] = bk; best[2] = bc; }
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
