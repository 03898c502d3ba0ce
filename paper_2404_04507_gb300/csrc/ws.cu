// Learned warm start: an MLP maps a potential's parameters to the lowest eigenvectors on a
// fixed core window, trained with a gauge-invariant subspace loss, and its prediction is
// embedded into a larger window as the eigensolver's start block.
//
// Layers: dense (bfloat16 weights and inputs, float32 accumulation in tensor memory by
// tcgen05.mma) with GELU between them and a linear output layer. Master weights and
// the AdamW state are float32. The loss per sample is |X X^H - Y Y^H|_F^2 / nvec, X the
// reference eigenvectors and Y the prediction on the core (flat layout (v*ncore + i)*2 + re/im).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "common.cuh"
#include "tc.cuh"

struct iwf_ws {
  int device = 0;
  int nl = 0;                       // weight layers
  int dims[16] = {};                // dims[0] input (mult. of 32) ... dims[nl] output
  long long woff[16] = {}, boff[16] = {};
  long long nparams = 0;
  float* params = nullptr;          // float32 master: per layer W (out x in) then b (out)
  float* grads = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  __nv_bfloat16* wbf = nullptr;     // bfloat16 copy of every W, same offsets as params
  __nv_bfloat16* wtbf = nullptr;    // transposed W (in x out) of one layer, scratch
  long long step = 0;
  // per-batch activations
  int cap = 0;                      // batch capacity
  __nv_bfloat16* hbf[16] = {};      // layer inputs (B x dims[l]) in bfloat16
  float* z[16] = {};                // pre-activations (B x dims[l+1])
  float* dz = nullptr;              // B x max dim
  __nv_bfloat16* dzbf = nullptr;
  __nv_bfloat16* dzt = nullptr;     // transposed dz
  __nv_bfloat16* ht = nullptr;      // transposed layer input
  float* dh = nullptr;
  float* gwork = nullptr;           // max(out x in) float32 GEMM output scratch
  float* lossbuf = nullptr;         // per-sample losses
  float* gsplit = nullptr;          // split-K partial tiles of the tensor-core GEMMs
  size_t gsplit_cap = 0;
  int* d_err = nullptr;             // set when a GEMM's bounded wait ran out
};

namespace iwf {
namespace {

// ---- dense layers on the tcgen05 tensor cores ---------------------------------------------
// C (M x N, float32, row-major) = A (M x K) . B (N x K)^T, A and B bfloat16 row-major (both
// K-major), one 128 x 128 tile of C per CTA accumulated in tensor memory. The K range of a CTA
// is [z kchunk, (z + 1) kchunk) for blockIdx.z = z; with several splits each writes its partial
// tile to C + z M N (summed by gemm_reduce). All 128 threads stage 64-deep K slices of A and B
// into a 4-stage ring with cp.async (rows past M or N and K past the end read as zeros); after
// its copies land each thread makes them visible to the tensor core and arrives on the stage's
// mbarrier; thread 0 issues the stage's four K16 MMAs and commits them to the stage's "empty"
// barrier. Every wait is bounded: one that runs out sets *err and the CTA winds down (its
// copies drained, its MMAs completed) before it releases tensor memory.
constexpr int kTM = 128, kTN = 128, kTK = 64, kGStages = 4, kGThreads = 128;
constexpr int kGTile = kTM * tc::kTileRowBytes;                 // 4 KB: 128 rows x K16
constexpr int kGStageBytes = 2 * (kTK / 16) * kGTile;           // A and B slices: 32 KB
constexpr int kGSmem = kGStages * kGStageBytes;
constexpr long long kGSpin = 1LL << 22;

__device__ __forceinline__ bool g_wait(uint32_t bar, uint32_t parity, bool sleep) {
  for (long long r = 0; r < kGSpin; ++r) {
    if (tc::bar_try_wait(bar, parity)) return true;
    if (sleep) __nanosleep(128);
  }
  return false;
}

__device__ __forceinline__ void g_cp16(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes)
               : "memory");
}

__global__ void __launch_bounds__(kGThreads, 1)
gemm_tc_kernel(const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ B,
               float* __restrict__ C, int M, int N, int K, int kchunk, int* err) {
  extern __shared__ __align__(1024) unsigned char gsm[];
  __shared__ __align__(8) unsigned long long full_bar[kGStages], empty_bar[kGStages], done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * kTN;
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  const int nst = ke > kb ? (ke - kb + kTK - 1) / kTK : 0;
  float* Cz = C + (size_t)blockIdx.z * M * N;
  if (tid == 0) {
    for (int s = 0; s < kGStages; ++s) {
      tc::bar_init(tc::smem_u32(&full_bar[s]), kGThreads);
      tc::bar_init(tc::smem_u32(&empty_bar[s]), 1);
    }
    tc::bar_init(tc::smem_u32(&done_bar), 1);
    tc::bar_init_fence();
    abort_flag = 0;
  }
  if (warp == 0) {
    tc::tmem_alloc(tc::smem_u32(&tmem_base), 128);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  volatile int* abort_v = &abort_flag;
  const uint32_t base = tc::smem_u32(gsm);

  // stage j: 2 operands x 128 rows x 8 chunks of 16 bytes (K16 step t = chunk / 2, half
  // h = chunk % 2); thread tid copies chunks tid + 128 i, i < 16
  const auto load = [&](int j) {
    const uint32_t sb = base + (uint32_t)((j % kGStages) * kGStageBytes);
    const int k0 = kb + j * kTK;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int e = tid + kGThreads * i;            // 0 .. 2047
      const int op = e >> 10, row = (e >> 3) & 127, ch = e & 7;
      const int t = ch >> 1, h = ch & 1;
      const int k = k0 + 8 * ch;
      const int grow = (op == 0 ? m0 : n0) + row;
      const bool in = grow < (op == 0 ? M : N) && k < ke;
      const __nv_bfloat16* src = (op == 0 ? A : B) + (in ? (size_t)grow * K + k : 0);
      const uint32_t dst = sb + (uint32_t)(op * (kGStageBytes / 2) + t * kGTile) +
                           tc::tile_off(row, h);
      g_cp16(dst, src, in ? 16 : 0);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  for (int j = 0; j < kGStages - 1; ++j) {
    if (j < nst) load(j);
    else asm volatile("cp.async.commit_group;" ::: "memory");
  }
  const uint32_t idesc = tc::idesc_bf16(kTM, kTN, false);
  for (int j = 0; j < nst && !*abort_v; ++j) {
    // refill the slot of stage j - 1 with stage j + kGStages - 1 once its MMAs are done
    const int jn = j + kGStages - 1;
    if (jn < nst) {
      if (j >= 1 && !g_wait(tc::smem_u32(&empty_bar[jn % kGStages]),
                            (uint32_t)(((jn / kGStages) - 1) & 1), false)) {
        atomicExch(&abort_flag, 1);
        break;
      }
      load(jn);
    } else {
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    asm volatile("cp.async.wait_group %0;" ::"n"(kGStages - 1) : "memory");
    tc::fence_async_smem();
    tc::bar_arrive(tc::smem_u32(&full_bar[j % kGStages]));
    if (tid == 0) {
      if (!g_wait(tc::smem_u32(&full_bar[j % kGStages]), (uint32_t)((j / kGStages) & 1), false)) {
        atomicExch(&abort_flag, 1);
        break;
      }
      tc::fence_after_sync();
      const uint32_t sb = base + (uint32_t)((j % kGStages) * kGStageBytes);
#pragma unroll
      for (int t = 0; t < kTK / 16; ++t)
        tc::mma_bf16(tmem, tc::sdesc(sb + t * kGTile), tc::sdesc(sb + kGStageBytes / 2 + t * kGTile),
                     idesc, j > 0 || t > 0);
      tc::mma_commit(tc::smem_u32(&empty_bar[j % kGStages]));
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  if (tid == 0) tc::mma_commit(tc::smem_u32(&done_bar));   // every MMA issued so far
  const bool ok = g_wait(tc::smem_u32(&done_bar), 0, true) && !*abort_v;
  tc::fence_after_sync();
  if (ok) {
    // row m0 + 32 warp + lane of the tile sits in tensor-memory lane 32 warp + lane
    const int row = m0 + 32 * warp + lane;
#pragma unroll 4
    for (int g = 0; g < kTN / 8; ++g) {
      float v[8];
      tc::tmem_ld8(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(8 * g), v);
      tc::tmem_wait_ld();
      const int col = n0 + 8 * g;
      if (row < M && col < N) {
        float4* dst = reinterpret_cast<float4*>(Cz + (size_t)row * N + col);
        dst[0] = make_float4(nst ? v[0] : 0.f, nst ? v[1] : 0.f, nst ? v[2] : 0.f, nst ? v[3] : 0.f);
        dst[1] = make_float4(nst ? v[4] : 0.f, nst ? v[5] : 0.f, nst ? v[6] : 0.f, nst ? v[7] : 0.f);
      }
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, 128);
  }
}

// C[i] = sum over the splits of P[z][i]
__global__ void gemm_reduce(const float* P, float* C, long long count, int splits) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += P[(size_t)z * count + i];
    C[i] = s;
  }
}

// out (C x R) = in (R x C)^T, bfloat16, through a 32 x 33 shared tile.
__global__ void transpose_bf16(const __nv_bfloat16* in, __nv_bfloat16* out, int R, int Cc) {
  __shared__ __nv_bfloat16 tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int r = by + j, c = bx + threadIdx.x;
    if (r < R && c < Cc) tile[j][threadIdx.x] = in[(size_t)r * Cc + c];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int c = bx + j, r = by + threadIdx.x;
    if (c < Cc && r < R) out[(size_t)c * R + r] = tile[threadIdx.x][j];
  }
}

__global__ void f32_to_bf16(const float* in, __nv_bfloat16* out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16_rn(in[i]);
}

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.3989422804014327f;
}

// z = c + b (kept for the backward pass); next layer input = bf16(gelu(z)), or for the
// output layer out = z.
__global__ void bias_act(const float* c, const float* b, float* z, __nv_bfloat16* hnext,
                         float* out, int B, int N, int last) {
  const long long n = (long long)B * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float v = c[i] + b[i % N];
    z[i] = v;
    if (last) out[i] = v;
    else hnext[i] = __float2bfloat16_rn(gelu_f(v));
  }
}

// dz = dh * gelu'(z)
__global__ void act_back(const float* dh, const float* z, float* dz, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dz[i] = dh[i] * gelu_grad_f(z[i]);
}

// db[j] = sum over rows of dz[r][j]
__global__ void colsum(const float* dz, float* db, int B, int N) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  float s = 0.f;
  for (int r = 0; r < B; ++r) s += dz[(size_t)r * N + j];
  db[j] = s;
}

// Subspace loss per sample (one CTA): Gram matrices X^H X, X^H Y, Y^H Y (nvec <= 16), then
// dY = (-4 X (X^H Y) + 4 Y (Y^H Y)) / (B nvec) and the sample's loss / (B nvec).
__global__ void subspace_loss_kernel(const float* Y, const float* X, int nvec, int ncore,
                                     int nout, float scale, float* dY, float* loss) {
  __shared__ float2 gxx[16][16], gxy[16][16], gyy[16][16];
  const int s = blockIdx.x;
  const float* y = Y + (size_t)s * nout;
  const float* x = X + (size_t)s * nout;
  const int a = threadIdx.x / 16, c = threadIdx.x % 16;
  if (a < nvec && c < nvec) {
    float xx_r = 0, xx_i = 0, xy_r = 0, xy_i = 0, yy_r = 0, yy_i = 0;
    for (int i = 0; i < ncore; ++i) {
      const float2 xa = *reinterpret_cast<const float2*>(&x[((size_t)a * ncore + i) * 2]);
      const float2 xc = *reinterpret_cast<const float2*>(&x[((size_t)c * ncore + i) * 2]);
      const float2 ya = *reinterpret_cast<const float2*>(&y[((size_t)a * ncore + i) * 2]);
      const float2 yc = *reinterpret_cast<const float2*>(&y[((size_t)c * ncore + i) * 2]);
      xx_r += xa.x * xc.x + xa.y * xc.y; xx_i += xa.x * xc.y - xa.y * xc.x;
      xy_r += xa.x * yc.x + xa.y * yc.y; xy_i += xa.x * yc.y - xa.y * yc.x;
      yy_r += ya.x * yc.x + ya.y * yc.y; yy_i += ya.x * yc.y - ya.y * yc.x;
    }
    gxx[a][c] = make_float2(xx_r, xx_i);
    gxy[a][c] = make_float2(xy_r, xy_i);
    gyy[a][c] = make_float2(yy_r, yy_i);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double l = 0;
    for (int i = 0; i < nvec; ++i)
      for (int j = 0; j < nvec; ++j) {
        l += (double)gxx[i][j].x * gxx[i][j].x + (double)gxx[i][j].y * gxx[i][j].y;
        l -= 2.0 * ((double)gxy[i][j].x * gxy[i][j].x + (double)gxy[i][j].y * gxy[i][j].y);
        l += (double)gyy[i][j].x * gyy[i][j].x + (double)gyy[i][j].y * gyy[i][j].y;
      }
    loss[s] = (float)(l * scale);
  }
  // dY[i][v] = scale * (-4 sum_a x[i][a] gxy[a][v] + 4 sum_a y[i][a] gyy[a][v])
  for (int e = threadIdx.x; e < ncore * nvec; e += blockDim.x) {
    const int v = e / ncore, i = e % ncore;
    float gr = 0.f, gi = 0.f;
    for (int aa = 0; aa < nvec; ++aa) {
      const float2 xa = *reinterpret_cast<const float2*>(&x[((size_t)aa * ncore + i) * 2]);
      const float2 ya = *reinterpret_cast<const float2*>(&y[((size_t)aa * ncore + i) * 2]);
      const float2 p = gxy[aa][v], q = gyy[aa][v];
      gr += -4.f * (xa.x * p.x - xa.y * p.y) + 4.f * (ya.x * q.x - ya.y * q.y);
      gi += -4.f * (xa.x * p.y + xa.y * p.x) + 4.f * (ya.x * q.y + ya.y * q.x);
    }
    dY[(size_t)s * nout + ((size_t)v * ncore + i) * 2] = gr * scale;
    dY[(size_t)s * nout + ((size_t)v * ncore + i) * 2 + 1] = gi * scale;
  }
}

// AdamW (decoupled weight decay on W, not on b) and the bfloat16 copy of W.
__global__ void adamw(float* w, const float* g, float* m, float* v, __nv_bfloat16* wbf,
                      const unsigned char* is_weight, long long n, float lr, float b1, float b2,
                      float eps, float wd, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi; v[i] = vi;
    float wi = w[i];
    if (is_weight[i]) wi -= lr * wd * wi;
    wi -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    wbf[i] = __float2bfloat16_rn(wi);
  }
}

// Gather rows idx[0..B) of a (n x width) float32 matrix.
__global__ void gather_rows(const float* src, const int* idx, float* dst, int B, int width) {
  const long long n = (long long)B * width;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / width), c = (int)(e % width);
    dst[e] = src[(size_t)idx[r] * width + c];
  }
}

// Core window -> big window by true index (zero elsewhere): out[p][v][pos(k)] = in[p][v][e].
struct EmbedArgs {
  Geom cg, bg;           // core and big geometry
  const int* clo;        // core slice bounds
  const int* blo;        // big slice bounds
  int nvec, nprob;
};

__global__ void embed_kernel(EmbedArgs a, const double2* in, double2* out, int* dropped) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= a.cg.N) return;
  int k[IWF_MAX_N];
  const long long s = e / a.cg.MI;
  long long t = e - s * a.cg.MI;
  for (int j = a.cg.d - 1; j >= 0; --j) { k[j] = a.clo[s * a.cg.d + j] + (int)(t % a.cg.lens[j]); t /= a.cg.lens[j]; }
  long long ss = s;
  for (int j = a.cg.n - 1; j >= a.cg.d; --j) { k[j] = (int)(ss % a.cg.lens[j]) - a.cg.half[j]; ss /= a.cg.lens[j]; }
  // big slice of k_II, then the k_I offsets inside it
  long long sb = 0;
  for (int j = a.bg.d; j < a.bg.n; ++j) {
    const int pj = k[j] + a.bg.half[j];
    if (pj < 0 || pj >= a.bg.lens[j]) { atomicAdd(dropped, 1); return; }
    sb = sb * a.bg.lens[j] + pj;
  }
  long long pos = 0;
  for (int j = 0; j < a.bg.d; ++j) {
    const int tj = k[j] - a.blo[sb * a.bg.d + j];
    if (tj < 0 || tj >= a.bg.lens[j]) { atomicAdd(dropped, 1); return; }
    pos = pos * a.bg.lens[j] + tj;
  }
  pos += sb * a.bg.MI;
  for (int p = 0; p < a.nprob; ++p)
    for (int v = 0; v < a.nvec; ++v)
      out[((size_t)p * a.nvec + v) * a.bg.N + pos] = in[((size_t)p * a.nvec + v) * a.cg.N + e];
}

// vecs[p][v][e] *= exp(i * sign * k(e) . phi_p), k(e) the true index of window position e.
__global__ void phase_kernel(Geom g, const int* lo, const double* phases, int nprob, int nvec,
                             int sign, double2* vecs) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= g.N) return;
  int k[IWF_MAX_N];
  const long long s = e / g.MI;
  long long t = e - s * g.MI;
  for (int j = g.d - 1; j >= 0; --j) { k[j] = lo[s * g.d + j] + (int)(t % g.lens[j]); t /= g.lens[j]; }
  long long ss = s;
  for (int j = g.n - 1; j >= g.d; --j) { k[j] = (int)(ss % g.lens[j]) - g.half[j]; ss /= g.lens[j]; }
  for (int p = 0; p < nprob; ++p) {
    double ph = 0.0;
    for (int j = 0; j < g.n; ++j) ph += (double)k[j] * phases[(size_t)p * g.n + j];
    double sn, cs;
    sincos(sign * ph, &sn, &cs);
    for (int v = 0; v < nvec; ++v) {
      double2& x = vecs[((size_t)p * nvec + v) * g.N + e];
      const double re = x.x * cs - x.y * sn;
      x.y = x.x * sn + x.y * cs;
      x.x = re;
    }
  }
}

int blocks_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 8 * 152)); }

template <typename U> iwf_status dalloc(U** p, size_t n);

// C = A B^T on the tensor cores. A grid of fewer tiles than SMs with a long K splits K across
// CTAs (partials in w->gsplit, then summed).
iwf_status gemm(iwf_ws* w, const __nv_bfloat16* A, const __nv_bfloat16* B, float* C, int M, int N,
                int K, cudaStream_t s) {
  if (M % 64 || N % 64 || K % 32) return fail(IWF_ERR_ARG, "gemm: shape not a tile multiple");
  static bool attr[64] = {};
  int dev = 0;
  IWF_CUDA(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64 && !attr[dev]) {
    IWF_CUDA(cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kGSmem));
    attr[dev] = true;
  }
  const int tm = (M + kTM - 1) / kTM, tn = (N + kTN - 1) / kTN;
  int splits = 1;
  if (tm * tn < 152 && K >= 2 * 512) splits = std::min((152 + tm * tn - 1) / (tm * tn), K / 512);
  const int kchunk = ((K + splits - 1) / splits + kTK - 1) / kTK * kTK;
  splits = (K + kchunk - 1) / kchunk;
  float* out = C;
  if (splits > 1) {
    const size_t need = (size_t)splits * M * N;
    if (need > w->gsplit_cap) {
      cudaFree(w->gsplit);
      w->gsplit = nullptr;
      w->gsplit_cap = 0;
      IWF_TRY(dalloc(&w->gsplit, need));
      w->gsplit_cap = need;
    }
    out = w->gsplit;
  }
  gemm_tc_kernel<<<dim3(tn, tm, splits), kGThreads, kGSmem, s>>>(A, B, out, M, N, K, kchunk, w->d_err);
  IWF_CUDA(cudaGetLastError());
  count_launch();
  if (splits > 1) {
    const long long cnt = (long long)M * N;
    gemm_reduce<<<(int)std::min<long long>((cnt + 255) / 256, 4 * 152), 256, 0, s>>>(out, C, cnt, splits);
    IWF_CUDA(cudaGetLastError());
    count_launch();
  }
  return IWF_OK;
}

iwf_status transpose(const __nv_bfloat16* in, __nv_bfloat16* out, int R, int Cc, cudaStream_t s) {
  transpose_bf16<<<dim3((Cc + 31) / 32, (R + 31) / 32), dim3(32, 8), 0, s>>>(in, out, R, Cc);
  IWF_CUDA(cudaGetLastError());
  count_launch();
  return IWF_OK;
}

template <typename U> iwf_status dalloc(U** p, size_t n) {
  if (cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(U)) != cudaSuccess)
    return fail(IWF_ERR_ALLOC, "warm-start allocation failed");
  return IWF_OK;
}

iwf_status ensure_batch(iwf_ws* w, int B) {
  if (B <= w->cap) return IWF_OK;
  for (int l = 0; l <= w->nl; ++l) { cudaFree(w->hbf[l]); cudaFree(w->z[l]); w->hbf[l] = nullptr; w->z[l] = nullptr; }
  cudaFree(w->dz); cudaFree(w->dzbf); cudaFree(w->dzt); cudaFree(w->ht); cudaFree(w->dh); cudaFree(w->lossbuf);
  int maxd = 0;
  for (int l = 0; l <= w->nl; ++l) maxd = std::max(maxd, w->dims[l]);
  for (int l = 0; l < w->nl; ++l) {
    IWF_TRY(dalloc(&w->hbf[l], (size_t)B * w->dims[l]));
    IWF_TRY(dalloc(&w->z[l], (size_t)B * w->dims[l + 1]));
  }
  IWF_TRY(dalloc(&w->dz, (size_t)B * maxd));
  IWF_TRY(dalloc(&w->dzbf, (size_t)B * maxd));
  IWF_TRY(dalloc(&w->dzt, (size_t)B * maxd));
  IWF_TRY(dalloc(&w->ht, (size_t)B * maxd));
  IWF_TRY(dalloc(&w->dh, (size_t)B * maxd));
  IWF_TRY(dalloc(&w->lossbuf, (size_t)B));
  long long maxw = 0;
  for (int l = 0; l < w->nl; ++l) maxw = std::max(maxw, (long long)w->dims[l] * w->dims[l + 1]);
  cudaFree(w->gwork);
  IWF_TRY(dalloc(&w->gwork, (size_t)std::max<long long>(maxw, (long long)B * maxd)));
  w->cap = B;
  return IWF_OK;
}

// The GEMMs' device error word, read at a synchronisation point of `s` (and cleared).
iwf_status check_ws_err(iwf_ws* w, cudaStream_t s) {
  int h = 0;
  IWF_CUDA(cudaMemcpyAsync(&h, w->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  IWF_CUDA(cudaStreamSynchronize(s));
  if (h) {
    IWF_CUDA(cudaMemsetAsync(w->d_err, 0, sizeof(int), s));
    IWF_CUDA(cudaStreamSynchronize(s));
    return fail(IWF_ERR_TIMEOUT, "warm start: a tensor-core GEMM gave up waiting");
  }
  return IWF_OK;
}

// Forward pass on B samples of features (device float32 B x dims[0]); output (B x dims[nl]).
iwf_status forward(iwf_ws* w, int B, const float* feat, float* out, cudaStream_t s) {
  IWF_TRY(ensure_batch(w, B));
  f32_to_bf16<<<blocks_for((long long)B * w->dims[0]), 256, 0, s>>>(feat, w->hbf[0], (long long)B * w->dims[0]);
  IWF_CUDA(cudaGetLastError());
  count_launch();
  for (int l = 0; l < w->nl; ++l) {
    const int in = w->dims[l], o = w->dims[l + 1];
    IWF_TRY(gemm(w, w->hbf[l], w->wbf + w->woff[l], w->gwork, B, o, in, s));
    const bool last = l + 1 == w->nl;
    bias_act<<<blocks_for((long long)B * o), 256, 0, s>>>(w->gwork, w->params + w->boff[l], w->z[l],
                                                          last ? nullptr : w->hbf[l + 1],
                                                          last ? out : nullptr, B, o, last ? 1 : 0);
    IWF_CUDA(cudaGetLastError());
    count_launch();
  }
  return IWF_OK;
}

// Loss and parameter gradients (into w->grads) for B samples; targets device (B x nout).
iwf_status loss_grad(iwf_ws* w, int B, const float* feat, const float* target, int nvec,
                     int ncore, float* yout, float* loss_dev, cudaStream_t s) {
  const int nout = w->dims[w->nl];
  if (2 * nvec * ncore != nout || nvec > 16) return fail(IWF_ERR_ARG, "warm start: output size != 2*nvec*ncore");
  IWF_TRY(forward(w, B, feat, yout, s));
  subspace_loss_kernel<<<B, 256, 0, s>>>(yout, target, nvec, ncore, nout, 1.f / (B * nvec),
                                         w->dz, loss_dev);
  IWF_CUDA(cudaGetLastError());
  count_launch();
  for (int l = w->nl - 1; l >= 0; --l) {
    const int in = w->dims[l], o = w->dims[l + 1];
    // dW = dz^T h  (o x in) = (dz^T) . (h^T)^T
    f32_to_bf16<<<blocks_for((long long)B * o), 256, 0, s>>>(w->dz, w->dzbf, (long long)B * o);
    count_launch();
    IWF_TRY(transpose(w->dzbf, w->dzt, B, o, s));
    IWF_TRY(transpose(w->hbf[l], w->ht, B, in, s));
    IWF_TRY(gemm(w, w->dzt, w->ht, w->grads + w->woff[l], o, in, B, s));
    colsum<<<(o + 255) / 256, 256, 0, s>>>(w->dz, w->grads + w->boff[l], B, o);
    count_launch();
    if (l > 0) {
      // dh = dz W  (B x in) = dz . (W^T)^T ; then dz_{l-1} = dh * gelu'(z_{l-1})
      IWF_TRY(transpose(w->wbf + w->woff[l], w->wtbf, o, in, s));
      IWF_TRY(gemm(w, w->dzbf, w->wtbf, w->dh, B, in, o, s));
      act_back<<<blocks_for((long long)B * in), 256, 0, s>>>(w->dh, w->z[l - 1], w->dz, (long long)B * in);
      count_launch();
    }
  }
  return IWF_OK;
}

}  // namespace
}  // namespace iwf

using namespace iwf;

extern "C" {

iwf_status iwf_ws_create(iwf_ws** out, int nlayers, const int* dims, unsigned long long seed,
                         int device) {
  clear_error();
  if (!out || !dims || nlayers < 1 || nlayers > 15) return fail(IWF_ERR_ARG, "iwf_ws_create: bad layers");
  *out = nullptr;
  for (int l = 0; l <= nlayers; ++l)
    if (dims[l] <= 0 || dims[l] % 64) return fail(IWF_ERR_ARG, "iwf_ws_create: layer sizes must be multiples of 64");
  DeviceGuard guard(device);
  iwf_ws* w = new (std::nothrow) iwf_ws();
  if (!w) return fail(IWF_ERR_ALLOC, "iwf_ws_create: host allocation");
  w->device = device;
  w->nl = nlayers;
  long long off = 0, maxw = 0;
  for (int l = 0; l <= nlayers; ++l) w->dims[l] = dims[l];
  for (int l = 0; l < nlayers; ++l) {
    w->woff[l] = off; off += (long long)dims[l] * dims[l + 1];
    w->boff[l] = off; off += dims[l + 1];
    maxw = std::max(maxw, (long long)dims[l] * dims[l + 1]);
  }
  w->nparams = off;
  // He-uniform weights from a seeded host generator, zero biases
  std::vector<float> h(off, 0.f);
  std::vector<unsigned char> isw(off, 0);   // 1 for weights (decayed), 0 for biases
  std::mt19937_64 rng(seed);
  for (int l = 0; l < nlayers; ++l) {
    const float lim = std::sqrt(6.f / (float)dims[l]) * (l + 1 == nlayers ? 0.1f : 1.f);
    std::uniform_real_distribution<float> U(-lim, lim);
    for (long long i = 0; i < (long long)dims[l] * dims[l + 1]; ++i) {
      h[w->woff[l] + i] = U(rng);
      isw[w->woff[l] + i] = 1;
    }
  }
  iwf_status st = IWF_OK;
  unsigned char* d_isw = nullptr;
  if (st == IWF_OK) st = dalloc(&w->params, off);
  if (st == IWF_OK) st = dalloc(&w->grads, off);
  if (st == IWF_OK) st = dalloc(&w->m, off);
  if (st == IWF_OK) st = dalloc(&w->v, off);
  if (st == IWF_OK) st = dalloc(&w->wbf, off);
  if (st == IWF_OK) st = dalloc(&w->wtbf, maxw);
  if (st == IWF_OK) st = dalloc(&d_isw, off);
  if (st == IWF_OK) st = dalloc(&w->d_err, 1);
  if (st != IWF_OK) { cudaFree(d_isw); iwf_ws_destroy(w); return st; }
  cudaMemset(w->d_err, 0, sizeof(int));
  cudaMemcpy(w->params, h.data(), off * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemcpy(d_isw, isw.data(), off, cudaMemcpyHostToDevice);
  cudaMemset(w->m, 0, off * sizeof(float));
  cudaMemset(w->v, 0, off * sizeof(float));
  cudaMemset(w->grads, 0, off * sizeof(float));
  f32_to_bf16<<<blocks_for(off), 256>>>(w->params, w->wbf, off);
  count_launch();
  cudaFree(d_isw);
  if (cudaDeviceSynchronize() != cudaSuccess) { iwf_ws_destroy(w); return fail(IWF_ERR_CUDA, "iwf_ws_create"); }
  *out = w;
  return IWF_OK;
}

void iwf_ws_destroy(iwf_ws* w) {
  if (!w) return;
  DeviceGuard guard(w->device);
  for (int l = 0; l <= w->nl; ++l) { cudaFree(w->hbf[l]); cudaFree(w->z[l]); }
  cudaFree(w->params); cudaFree(w->grads); cudaFree(w->m); cudaFree(w->v); cudaFree(w->wbf);
  cudaFree(w->wtbf); cudaFree(w->dz); cudaFree(w->dzbf); cudaFree(w->dzt); cudaFree(w->ht);
  cudaFree(w->dh); cudaFree(w->gwork); cudaFree(w->lossbuf); cudaFree(w->gsplit);
  cudaFree(w->d_err);
  delete w;
}

iwf_status iwf_ws_num_params(const iwf_ws* w, long long* n) {
  if (!w || !n) return fail(IWF_ERR_ARG, "iwf_ws_num_params: NULL argument");
  *n = w->nparams;
  return IWF_OK;
}

iwf_status iwf_ws_get_params(const iwf_ws* w, float* host) {
  if (!w || !host) return fail(IWF_ERR_ARG, "iwf_ws_get_params: NULL argument");
  DeviceGuard guard(w->device);
  IWF_CUDA(cudaMemcpy(host, w->params, w->nparams * sizeof(float), cudaMemcpyDeviceToHost));
  return IWF_OK;
}

iwf_status iwf_ws_set_params(iwf_ws* w, const float* host) {
  if (!w || !host) return fail(IWF_ERR_ARG, "iwf_ws_set_params: NULL argument");
  DeviceGuard guard(w->device);
  IWF_CUDA(cudaMemcpy(w->params, host, w->nparams * sizeof(float), cudaMemcpyHostToDevice));
  f32_to_bf16<<<blocks_for(w->nparams), 256>>>(w->params, w->wbf, w->nparams);
  count_launch();
  IWF_CUDA(cudaDeviceSynchronize());
  return IWF_OK;
}

iwf_status iwf_ws_predict(iwf_ws* w, int nsamples, const float* feat, float* out, void* stream) {
  if (!w || !feat || !out || nsamples < 0) return fail(IWF_ERR_ARG, "iwf_ws_predict: bad arguments");
  if (nsamples % 64) return fail(IWF_ERR_ARG, "iwf_ws_predict: nsamples must be a multiple of 64");
  DeviceGuard guard(w->device);
  IWF_TRY(forward(w, nsamples, feat, out, (cudaStream_t)stream));
  return check_ws_err(w, (cudaStream_t)stream);
}

iwf_status iwf_ws_loss_grad(iwf_ws* w, int nsamples, const float* feat, const float* target,
                            int nvec, int ncore, float* loss, float* grads_host, void* stream) {
  if (!w || !feat || !target || nsamples % 64 || nsamples <= 0)
    return fail(IWF_ERR_ARG, "iwf_ws_loss_grad: bad arguments (nsamples a positive multiple of 64)");
  DeviceGuard guard(w->device);
  cudaStream_t s = (cudaStream_t)stream;
  float* y = nullptr;
  IWF_TRY(dalloc(&y, (size_t)nsamples * w->dims[w->nl]));
  IWF_TRY(ensure_batch(w, nsamples));
  iwf_status st = loss_grad(w, nsamples, feat, target, nvec, ncore, y, w->lossbuf, s);
  if (st == IWF_OK) {
    std::vector<float> l(nsamples);
    cudaMemcpyAsync(l.data(), w->lossbuf, nsamples * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (grads_host) cudaMemcpyAsync(grads_host, w->grads, w->nparams * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) st = fail(IWF_ERR_CUDA, "iwf_ws_loss_grad");
    double t = 0;
    for (float v : l) t += v;
    if (loss) *loss = (float)t;
    if (st == IWF_OK) st = check_ws_err(w, s);
  }
  cudaFree(y);
  return st;
}

iwf_status iwf_ws_train(iwf_ws* w, int nsamples, const float* feat, const float* target,
                        int nvec, int ncore, int epochs, int batch, float lr, float wd,
                        unsigned long long seed, float* loss_hist, void* stream) {
  clear_error();
  if (!w || !feat || !target || batch <= 0 || batch % 64 || nsamples < batch || epochs < 0)
    return fail(IWF_ERR_ARG, "iwf_ws_train: bad arguments (batch a multiple of 64, <= nsamples)");
  DeviceGuard guard(w->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int nin = w->dims[0], nout = w->dims[w->nl];
  IWF_TRY(ensure_batch(w, batch));
  float *bf = nullptr, *bt = nullptr, *y = nullptr, *losses = nullptr;
  int* idx = nullptr;
  unsigned char* isw = nullptr;
  const int nb = nsamples / batch;
  iwf_status st = IWF_OK;
  if (st == IWF_OK) st = dalloc(&bf, (size_t)batch * nin);
  if (st == IWF_OK) st = dalloc(&bt, (size_t)batch * nout);
  if (st == IWF_OK) st = dalloc(&y, (size_t)batch * nout);
  if (st == IWF_OK) st = dalloc(&idx, (size_t)batch);
  if (st == IWF_OK) st = dalloc(&losses, (size_t)nb * batch);
  if (st == IWF_OK) st = dalloc(&isw, (size_t)w->nparams);
  if (st == IWF_OK) {
    std::vector<unsigned char> h(w->nparams, 0);
    for (int l = 0; l < w->nl; ++l)
      std::fill(h.begin() + w->woff[l], h.begin() + w->boff[l], (unsigned char)1);
    if (cudaMemcpy(isw, h.data(), w->nparams, cudaMemcpyHostToDevice) != cudaSuccess)
      st = fail(IWF_ERR_CUDA, "iwf_ws_train: mask upload");
  }
  std::mt19937_64 rng(seed);
  std::vector<int> perm(nsamples);
  for (int i = 0; i < nsamples; ++i) perm[i] = i;
  std::vector<float> hl((size_t)nb * batch);
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int ep = 0; ep < epochs && st == IWF_OK; ++ep) {
    std::shuffle(perm.begin(), perm.end(), rng);
    for (int k = 0; k < nb && st == IWF_OK; ++k) {
      if (cudaMemcpyAsync(idx, perm.data() + (size_t)k * batch, batch * sizeof(int),
                          cudaMemcpyHostToDevice, s) != cudaSuccess) { st = fail(IWF_ERR_CUDA, "idx"); break; }
      gather_rows<<<blocks_for((long long)batch * nin), 256, 0, s>>>(feat, idx, bf, batch, nin);
      gather_rows<<<blocks_for((long long)batch * nout), 256, 0, s>>>(target, idx, bt, batch, nout);
      count_launch(); count_launch();
      st = loss_grad(w, batch, bf, bt, nvec, ncore, y, losses + (size_t)k * batch, s);
      if (st != IWF_OK) break;
      ++w->step;
      const float c1 = 1.f - std::pow(b1, (float)w->step), c2 = 1.f - std::pow(b2, (float)w->step);
      adamw<<<blocks_for(w->nparams), 256, 0, s>>>(w->params, w->grads, w->m, w->v, w->wbf, isw,
                                                   w->nparams, lr, b1, b2, eps, wd, c1, c2);
      count_launch();
      if (cudaStreamSynchronize(s) != cudaSuccess) st = fail(IWF_ERR_CUDA, "iwf_ws_train step");
    }
    if (st == IWF_OK) st = check_ws_err(w, s);
    if (st == IWF_OK && loss_hist) {
      if (cudaMemcpy(hl.data(), losses, hl.size() * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) {
        st = fail(IWF_ERR_CUDA, "loss readback");
        break;
      }
      double t = 0;
      for (float v : hl) t += v;
      loss_hist[ep] = (float)(t / nb);
    }
  }
  cudaFree(bf); cudaFree(bt); cudaFree(y); cudaFree(idx); cudaFree(losses); cudaFree(isw);
  return st;
}

iwf_status iwf_ws_phase(const iwf_plan* plan, int nprob, int nvec, const double* phases, int sign,
                        void* vecs, void* stream) {
  if (!plan || !phases || !vecs || nprob < 1 || nvec < 1 || (sign != 1 && sign != -1))
    return fail(IWF_ERR_ARG, "iwf_ws_phase: bad arguments");
  DeviceGuard guard(plan->device);
  cudaStream_t s = (cudaStream_t)stream;
  double* d_ph = nullptr;
  IWF_TRY(dalloc(&d_ph, (size_t)nprob * plan->g.n));
  cudaMemcpyAsync(d_ph, phases, sizeof(double) * nprob * plan->g.n, cudaMemcpyHostToDevice, s);
  phase_kernel<<<(unsigned)((plan->g.N + 255) / 256), 256, 0, s>>>(
      plan->g, plan->d_lo, d_ph, nprob, nvec, sign, reinterpret_cast<double2*>(vecs));
  count_launch();
  const cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(d_ph);
  if (e != cudaSuccess) return cuda_fail(e, "iwf_ws_phase");
  return IWF_OK;
}

iwf_status iwf_ws_embed(const iwf_plan* core, const iwf_plan* big, int nprob, int nvec,
                        const void* in, void* out, void* stream) {
  if (!core || !big || !in || !out || nprob < 1 || nvec < 1) return fail(IWF_ERR_ARG, "iwf_ws_embed: bad arguments");
  if (core->g.d != big->g.d || core->g.n != big->g.n || core->device != big->device)
    return fail(IWF_ERR_ARG, "iwf_ws_embed: plans differ in shape or device");
  DeviceGuard guard(big->device);
  cudaStream_t s = (cudaStream_t)stream;
  IWF_CUDA(cudaMemsetAsync(out, 0, sizeof(double2) * big->g.N * nvec * nprob, s));
  int* dropped = nullptr;
  IWF_TRY(dalloc(&dropped, 1));
  cudaMemsetAsync(dropped, 0, sizeof(int), s);
  EmbedArgs a{core->g, big->g, core->d_lo, big->d_lo, nvec, nprob};
  embed_kernel<<<(unsigned)((core->g.N + 255) / 256), 256, 0, s>>>(
      a, reinterpret_cast<const double2*>(in), reinterpret_cast<double2*>(out), dropped);
  count_launch();
  int h = 0;
  cudaMemcpyAsync(&h, dropped, sizeof(int), cudaMemcpyDeviceToHost, s);
  const cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(dropped);
  if (e != cudaSuccess) return cuda_fail(e, "iwf_ws_embed");
  if (h) return fail(IWF_ERR_ARG, "iwf_ws_embed: the core window is not nested in the big window");
  return IWF_OK;
}

}  // extern "C"
