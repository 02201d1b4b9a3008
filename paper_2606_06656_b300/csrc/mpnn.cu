// mpnn.cu -- the learned initialiser: a 2-layer message-passing network
// (hidden 64) on the constraint-variable incidence graph, forward and
// backward, on sm_103a.  Dense layers run on tensor cores (bf16 operands,
// fp32 accumulation); aggregations are sign-aware gathers over the
// constraint-major literal list and its variable-major transpose; every
// reduction is blocked and summed in a fixed order (no atomics).
//
// Model (per node):  embed  h = relu(W_in f + b_in)
//   layer l = 1, 2:  a_c = L_c^-1/2   sum_{e in c} s_e h_v[v_e]
//                    h_c = relu(W_cl [h_c, a_c] + b_cl)
//                    a_v = deg_v^-1/2 sum_{e on v} s_e h_c[c_e]
//                    h_v = relu(W_vl [h_v, a_v] + b_vl)
//   head:            z_v = w_out . h_v + b_out,  x0[v,r] = tanh(z_v + tau u[v,r])
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/cls.h"
#include "mpnn.cuh"

namespace cls {
namespace mp {
namespace {

constexpr unsigned kFull = 0xffffffffu;

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// --------------------------------------------------------------------------
// embedding: out[i, j] = relu(sum_k W[j, k] f[i, k] + b[j]), K = 4 or 12
// --------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(256) k_embed(int N, const float* __restrict__ f,
                                               const float* __restrict__ W,
                                               const float* __restrict__ b,
                                               float* __restrict__ out) {
  const int j = threadIdx.x;                        // 0..63
  const int i = blockIdx.x * blockDim.y + threadIdx.y;
  if (i >= N) return;
  float acc = b[j];
#pragma unroll
  for (int k = 0; k < K; ++k) acc = fmaf(W[j * K + k], f[(size_t)i * K + k], acc);
  out[(size_t)i * kHid + j] = fmaxf(acc, 0.f);
}

// dW[j,k] (partial per block of nodes), db[j] partial: dpre = dh * (h > 0)
template <int K>
__global__ void __launch_bounds__(256) k_embed_bwd(int N, int chunk, const float* __restrict__ f,
                                                   const float* __restrict__ h,
                                                   const float* __restrict__ dh,
                                                   float* __restrict__ part) {
  // block: 64 threads (feature j); part[blk][j*(K+1) + k], k = K is the bias
  const int j = threadIdx.x;
  const int i0 = blockIdx.x * chunk, i1 = min(N, i0 + chunk);
  float acc[K + 1];
#pragma unroll
  for (int k = 0; k <= K; ++k) acc[k] = 0.f;
  for (int i = i0; i < i1; ++i) {
    const float hv = h[(size_t)i * kHid + j];
    const float d = hv > 0.f ? dh[(size_t)i * kHid + j] : 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = fmaf(d, f[(size_t)i * K + k], acc[k]);
    acc[K] += d;
  }
  float* o = part + (size_t)blockIdx.x * kHid * (K + 1) + j * (K + 1);
#pragma unroll
  for (int k = 0; k <= K; ++k) o[k] = acc[k];
}

// --------------------------------------------------------------------------
// sign-aware segmented gather: out[i,:] (=|+=) rs[i] * sum_{k in seg(i)}
//   sgn[k] * cs[idx[k]] * src[idx[k], :]   (rs, cs optional)
// one warp per output row; lane owns features lane and lane+32
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_seg_gather(int N, const int32_t* __restrict__ off,
                                                    const int32_t* __restrict__ idx,
                                                    const float* __restrict__ sgn,
                                                    const float* __restrict__ cs,
                                                    const float* __restrict__ rs,
                                                    const float* __restrict__ src,
                                                    float* __restrict__ out, int accumulate) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= N) return;
  float a0 = 0.f, a1 = 0.f;
  for (int k = off[i]; k < off[i + 1]; ++k) {
    const int s = idx[k];
    const float w = sgn[k] * (cs ? cs[s] : 1.f);
    a0 = fmaf(w, src[(size_t)s * kHid + lane], a0);
    a1 = fmaf(w, src[(size_t)s * kHid + lane + 32], a1);
  }
  const float r = rs ? rs[i] : 1.f;
  float* o = out + (size_t)i * kHid;
  if (accumulate) {
    o[lane] += r * a0;
    o[lane + 32] += r * a1;
  } else {
    o[lane] = r * a0;
    o[lane + 32] = r * a1;
  }
}

// --------------------------------------------------------------------------
// tensor cores: tcgen05 (5th-generation MMA, accumulator in tensor memory)
//
// Each dense product is one 128-row tile per CTA of 256 threads: the bf16
// operands are staged in shared memory in the canonical K-major layout
// without swizzle (8 x 16-byte core matrices; core matrices adjacent in K
// kLBO = 128 bytes apart, 8-row groups KT / 8 * 128 bytes apart), thread 0
// issues tcgen05.mma (kind::f16, bf16 x bf16 -> fp32) for every 16-wide K
// step into a tensor-memory accumulator of 128 lanes x N columns and commits
// them to an mbarrier; every thread waits on it (a bounded wait: past
// kTcSpin polls the kernel writes NaN instead of a result and sets
// g_tc_timeout), then warp w reads lanes 32 (w % 4) .. +31 (rows) of its
// share of the columns with tcgen05.ld for the epilogue.  D = A B^T with A [128 x K] and B [N x K],
// both K-major.
// --------------------------------------------------------------------------
constexpr uint32_t kLBO = 128;                // bytes between K-adjacent core matrices
constexpr int kTcSpin = 1 << 22;              // mbarrier polls before giving up
__device__ int g_tc_timeout = 0;

// byte offset of element (row, k) of a [rows x KT] K-major operand
template <int KT>
__device__ __forceinline__ uint32_t cm_off(int row, int k) {
  return (uint32_t)((row >> 3) * (KT / 8) * kLBO + (k >> 3) * kLBO + (row & 7) * 16 + (k & 7) * 2);
}
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// shared-memory matrix descriptor: start, leading (K) and stride (8-row)
// byte offsets >> 4, descriptor version 1, no swizzle
template <int KT>
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t saddr) {
  constexpr uint32_t sbo = (KT / 8) * kLBO;
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((kLBO >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// instruction descriptor, kind::f16: fp32 accumulator, bf16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
template <int M, int N>
__device__ __forceinline__ uint32_t tc_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void st_bf2(unsigned char* base, uint32_t off, float lo, float hi) {
  *reinterpret_cast<__nv_bfloat162*>(base + off) = __floats2bfloat162_rn(lo, hi);
}

// The shared tail of the three products: tensor-memory allocation, the
// K / 16 MMAs, the bounded wait.  Call with the operands staged (generic
// stores); returns the tensor-memory address and whether the result is in.
template <int KT, int N>
__device__ __forceinline__ bool tc_run(const unsigned char* As, const unsigned char* Bs,
                                       uint64_t* mbar, uint32_t* tmem_slot, uint32_t& tmem) {
  const int tid = threadIdx.x, warp = tid >> 5;
  constexpr uint32_t kCols = N < 32 ? 32 : N;
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar)));
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                 ::"r"(smem_u32(tmem_slot)), "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");     // staged operands
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  tmem = *tmem_slot;
  if (tid == 0) {
    const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
#pragma unroll
    for (int ks = 0; ks < KT / 16; ++ks) {
      const uint64_t ad = tc_sdesc<KT>(a0 + ks * 2 * kLBO), bd = tc_sdesc<KT>(b0 + ks * 2 * kLBO);
      const uint32_t acc = ks > 0 ? 1u : 0u;
      asm volatile(
          "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
          "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
          ::"r"(tmem), "l"(ad), "l"(bd), "r"(tc_idesc<128, N>()), "r"(acc));
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
        ::"r"(smem_u32(mbar)) : "memory");
  }
  uint32_t done = 0;
  for (int it = 0; it < kTcSpin && !done; ++it)
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done) : "r"(smem_u32(mbar)), "r"(0u) : "memory");
  if (!done && (tid & 31) == 0) atomicExch(&g_tc_timeout, 1);
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  return done != 0;
}

// 32 consecutive accumulator columns of this thread's row (lane 32w + lane)
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&f)[32]) {
  uint32_t v[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
      "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
        "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
        "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int c = 0; c < 32; ++c) f[c] = __uint_as_float(v[c]);
}

template <int N>
__device__ __forceinline__ void tc_free(uint32_t tmem) {
  constexpr uint32_t kCols = N < 32 ? 32 : N;
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(kCols));
}

constexpr int kTcRows = 128;                  // rows of a tile (the MMA's M)

// Y[N,64] = relu([H | A] W^T + b), W: 64 x 128 (fp32 master, rounded to bf16)
__global__ void __launch_bounds__(256) k_dense_fwd(int N, const float* __restrict__ H,
                                                   const float* __restrict__ A,
                                                   const float* __restrict__ W,
                                                   const float* __restrict__ b,
                                                   float* __restrict__ Y) {
  constexpr int KT = 2 * kHid;
  __shared__ __align__(1024) unsigned char As[kTcRows * KT * 2];   // X tile, 32 KB
  __shared__ __align__(1024) unsigned char Bs[kHid * KT * 2];      // W, 16 KB
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row0 = blockIdx.x * kTcRows;
  for (int q = tid; q < kTcRows * kHid; q += 256) {          // (row, column pair)
    const int r = q / kHid, col = 2 * (q % kHid);
    float lo = 0.f, hi = 0.f;
    if (row0 + r < N) {
      const float* src = col < kHid ? H + (size_t)(row0 + r) * kHid + col
                                    : A + (size_t)(row0 + r) * kHid + (col - kHid);
      lo = src[0];
      hi = src[1];
    }
    st_bf2(As, cm_off<KT>(r, col), lo, hi);
  }
  for (int q = tid; q < kHid * kHid; q += 256) {
    const int r = q / kHid, col = 2 * (q % kHid);
    st_bf2(Bs, cm_off<KT>(r, col), W[r * KT + col], W[r * KT + col + 1]);
  }
  uint32_t tmem;
  const bool ok = tc_run<KT, kHid>(As, Bs, &mbar, &tmem_slot, tmem);
  // warp w reads accumulator lanes 32 (w % 4) .. +31 (its rows), columns
  // 32 (w / 4) .. +31
  const int quad = warp & 3, half = warp >> 2;
  const int row = row0 + 32 * quad + lane;
  {
    float f[32];
    if (ok) tc_ld32(tmem + ((uint32_t)(32 * quad) << 16) + 32 * half, f);
    if (row < N)
#pragma unroll
      for (int c = 0; c < 32; ++c)
        Y[(size_t)row * kHid + 32 * half + c] = ok ? fmaxf(f[c] + b[32 * half + c], 0.f) : NAN;
  }
  tc_free<kHid>(tmem);
}

// [dH | dA] = (dY * (Y > 0)) W; dH may alias dY (each block reads its rows
// before writing them).  A = dpre [128 x 64], B = W^T [128 x 64].
__global__ void __launch_bounds__(256) k_dense_bwd_dx(int N, const float* dY,
                                                      const float* __restrict__ Y,
                                                      const float* __restrict__ W, float* dH,
                                                      float* __restrict__ dA) {
  constexpr int KT = kHid;
  __shared__ __align__(1024) unsigned char As[kTcRows * KT * 2];       // dpre, 16 KB
  __shared__ __align__(1024) unsigned char Bs[2 * kHid * KT * 2];      // W^T, 16 KB
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row0 = blockIdx.x * kTcRows;
  for (int q = tid; q < kTcRows * (kHid / 2); q += 256) {
    const int r = q / (kHid / 2), col = 2 * (q % (kHid / 2));
    float lo = 0.f, hi = 0.f;
    if (row0 + r < N) {
      const size_t o = (size_t)(row0 + r) * kHid + col;
      lo = Y[o] > 0.f ? dY[o] : 0.f;
      hi = Y[o + 1] > 0.f ? dY[o + 1] : 0.f;
    }
    st_bf2(As, cm_off<KT>(r, col), lo, hi);
  }
  for (int q = tid; q < 2 * kHid * (kHid / 2); q += 256) {   // B[n][k] = W[k][n]
    const int n = q / (kHid / 2), k = 2 * (q % (kHid / 2));
    st_bf2(Bs, cm_off<KT>(n, k), W[k * 2 * kHid + n], W[(k + 1) * 2 * kHid + n]);
  }
  uint32_t tmem;
  // every read of this tile's dY rows is staged before tc_run's barrier, so
  // the writes below may overwrite them (dH aliasing dY)
  const bool ok = tc_run<KT, 2 * kHid>(As, Bs, &mbar, &tmem_slot, tmem);
  // warp w: accumulator lanes 32 (w % 4) .. +31, column quarters 2 (w / 4)
  // and 2 (w / 4) + 1
  const int quad = warp & 3;
  const int row = row0 + 32 * quad + lane;
#pragma unroll
  for (int pp = 0; pp < 2; ++pp) {
    const int part = 2 * (warp >> 2) + pp;
    float f[32];
    if (ok) tc_ld32(tmem + ((uint32_t)(32 * quad) << 16) + 32 * part, f);
    float* dst = part < 2 ? dH : dA;
    const int c0 = (part & 1) * 32;
    if (row < N)
#pragma unroll
      for (int c = 0; c < 32; ++c) dst[(size_t)row * kHid + c0 + c] = ok ? f[c] : NAN;
  }
  tc_free<2 * kHid>(tmem);
}

// partial dW[64 x 128] over a chunk of kDwRows node rows, plus db partial:
// dW = dpre^T [H | A],  dpre = dY * (Y > 0).  Computed transposed on the
// tensor cores, dW^T [128 x 64] = [H | A]^T dpre: A = X^T [128 x rows],
// B = dpre^T [64 x rows], both K-major in the rows.
constexpr int kDwRows = 64;
__global__ void __launch_bounds__(256) k_dense_bwd_dw(int N, const float* __restrict__ dY,
                                                      const float* __restrict__ Y,
                                                      const float* __restrict__ H,
                                                      const float* __restrict__ A,
                                                      float* __restrict__ part) {
  constexpr int KT = kDwRows;
  __shared__ __align__(1024) unsigned char As[2 * kHid * KT * 2];      // X^T, 16 KB
  __shared__ __align__(1024) unsigned char Bs[kHid * KT * 2];          // dpre^T, 8 KB
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ float dbs[4][kHid];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row0 = blockIdx.x * kDwRows;
  // pairs along rows (the K dimension of this product)
  for (int q = tid; q < (kDwRows / 2) * kHid; q += 256) {
    const int rp = q / kHid, m = q % kHid;                // rows 2rp, 2rp+1; feature m
    float v[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int r = row0 + 2 * rp + u;
      v[u] = 0.f;
      if (r < N) {
        const size_t o = (size_t)r * kHid + m;
        v[u] = Y[o] > 0.f ? dY[o] : 0.f;
      }
    }
    st_bf2(Bs, cm_off<KT>(m, 2 * rp), v[0], v[1]);
  }
  for (int q = tid; q < (kDwRows / 2) * 2 * kHid; q += 256) {
    const int rp = q / (2 * kHid), n = q % (2 * kHid);
    float v[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int r = row0 + 2 * rp + u;
      v[u] = 0.f;
      if (r < N)
        v[u] = n < kHid ? H[(size_t)r * kHid + n] : A[(size_t)r * kHid + n - kHid];
    }
    st_bf2(As, cm_off<KT>(n, 2 * rp), v[0], v[1]);
  }
  // bias partial in fp32 (fixed order over the chunk's rows)
  {
    const int m = tid & 63, quarter = tid >> 6;
    float s = 0.f;
    for (int rr = quarter; rr < kDwRows; rr += 4) {
      const int r = row0 + rr;
      if (r < N) {
        const size_t o = (size_t)r * kHid + m;
        s += Y[o] > 0.f ? dY[o] : 0.f;
      }
    }
    dbs[quarter][m] = s;
  }
  uint32_t tmem;
  const bool ok = tc_run<KT, kHid>(As, Bs, &mbar, &tmem_slot, tmem);
  float* o = part + (size_t)blockIdx.x * (kHid * 2 * kHid + kHid);
  const int quad = warp & 3, half = warp >> 2;
  const int n = 32 * quad + lane;                          // input feature = accumulator lane
  {
    float f[32];
    if (ok) tc_ld32(tmem + ((uint32_t)(32 * quad) << 16) + 32 * half, f);
#pragma unroll
    for (int c = 0; c < 32; ++c) o[(32 * half + c) * 2 * kHid + n] = ok ? f[c] : NAN;
  }
  if (tid < kHid) o[kHid * 2 * kHid + tid] = (dbs[0][tid] + dbs[1][tid]) + (dbs[2][tid] + dbs[3][tid]);
  tc_free<kHid>(tmem);
}

// out[k] = sum_{b < nblk} part[b*stride + k], fixed order
__global__ void __launch_bounds__(256) k_reduce_parts(int nblk, int width, int stride,
                                                      const float* __restrict__ part,
                                                      float* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= width) return;
  float s = 0.f;
  for (int b = 0; b < nblk; ++b) s += part[(size_t)b * stride + k];
  out[k] = s;
}

// --------------------------------------------------------------------------
// head
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_head(int n, const float* __restrict__ h,
                                              const float* __restrict__ w,
                                              const float* __restrict__ b,
                                              float* __restrict__ z) {
  const int lane = threadIdx.x & 31;
  const int v = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (v >= n) return;
  float s = h[(size_t)v * kHid + lane] * w[lane] + h[(size_t)v * kHid + lane + 32] * w[lane + 32];
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(kFull, s, d);
  if (lane == 0) z[v] = s + b[0];
}

__device__ __forceinline__ void philox4x64_10(uint64_t& x0, uint64_t& x1, uint64_t& x2,
                                              uint64_t& x3, uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint64_t hi0 = __umul64hi(M0, x0), lo0 = M0 * x0;
    const uint64_t hi1 = __umul64hi(M1, x2), lo1 = M1 * x2;
    const uint64_t n0 = hi1 ^ x1 ^ k0, n2 = hi0 ^ x3 ^ k1;
    x0 = n0;
    x1 = lo1;
    x2 = n2;
    x3 = lo0;
    k0 += W0;
    k1 += W1;
  }
}

// x0[v*R + r] = tanh(z_v + tau u[v,r]), u the initialiser's U[-1,1) draws
__global__ void __launch_bounds__(256) k_points(int n, int R, uint64_t seed, int64_t r_off,
                                                float tau, const float* __restrict__ z,
                                                const uint8_t* __restrict__ fixed,
                                                const float* __restrict__ fixed_val,
                                                float* __restrict__ x0) {
  const int64_t nq = (n + 3) / 4;
  const int64_t total = nq * (int64_t)R;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx % R);
    const int64_t q = idx / R;
    uint64_t w0 = (uint64_t)(r + r_off), w1 = (uint64_t)q, w2 = 0, w3 = 0;
    philox4x64_10(w0, w1, w2, w3, seed, 0ull);
    const uint64_t w[4] = {w0, w1, w2, w3};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t v = 4 * q + j;
      if (v < n) {
        const float u = (float)(w[j] >> 40) * 0x1p-23f - 1.0f;
        float val = tanhf(fmaf(tau, u, z[v]));
        if (fixed && fixed[v]) val = fixed_val[v];
        x0[v * R + r] = val;
      }
    }
  }
}

// dz_v = sum_r gx0[v,r] (1 - x0^2) + lam/n_free * (-2 t_v) sigma(-2 t_v z_v)
// for free variables, 0 for pinned ones (sum over restarts in lane order)
__global__ void __launch_bounds__(256) k_head_grad(int n, int R, const float* __restrict__ z,
                                                   const float* __restrict__ x0,
                                                   const float* __restrict__ gx0,
                                                   const int8_t* __restrict__ target, float lam,
                                                   float inv_nfree,
                                                   const uint8_t* __restrict__ fixed,
                                                   float* __restrict__ dz) {
  const int lane = threadIdx.x & 31;
  const int v = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (v >= n) return;
  float s = 0.f;
  if (gx0) {
    for (int r = lane; r < R; r += 32) {
      const float x = x0[(size_t)v * R + r];
      s = fmaf(gx0[(size_t)v * R + r], 1.f - x * x, s);
    }
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(kFull, s, d);
  const bool free_v = !(fixed && fixed[v]);
  float g = free_v ? s : 0.f;
  if (free_v && target && lam != 0.f) {
    const float t = (float)target[v];
    const float sig = 1.f / (1.f + expf(2.f * t * z[v]));
    g += lam * inv_nfree * (-2.f * t) * sig;
  }
  if (lane == 0) dz[v] = g;
}

// dh[v,:] = dz_v w_out
__global__ void __launch_bounds__(256) k_head_dh(int n, const float* __restrict__ dz,
                                                 const float* __restrict__ w_out,
                                                 float* __restrict__ dh) {
  const int j = threadIdx.x & 63;
  const int v = blockIdx.x * (blockDim.x >> 6) + (threadIdx.x >> 6);
  if (v >= n) return;
  dh[(size_t)v * kHid + j] = dz[v] * w_out[j];
}

// [j][0..K] (K weights then the bias of output j) -> W[j][k], b[j]
template <int K>
__global__ void k_split_embed(const float* __restrict__ in, float* __restrict__ W,
                              float* __restrict__ b) {
  const int j = threadIdx.x;
#pragma unroll
  for (int k = 0; k < K; ++k) W[j * K + k] = in[j * (K + 1) + k];
  b[j] = in[j * (K + 1) + K];
}

// partial [dw_out(64), db_out(1)] over a chunk of variables
__global__ void __launch_bounds__(64) k_head_param_grad(int n, int chunk,
                                                        const float* __restrict__ h,
                                                        const float* __restrict__ dz,
                                                        float* __restrict__ part) {
  const int j = threadIdx.x;
  const int v0 = blockIdx.x * chunk, v1 = min(n, v0 + chunk);
  float s = 0.f, sb = 0.f;
  for (int v = v0; v < v1; ++v) {
    s = fmaf(dz[v], h[(size_t)v * kHid + j], s);
    sb += dz[v];
  }
  float* o = part + (size_t)blockIdx.x * (kHid + 1);
  o[j] = s;
  if (j == 0) o[kHid] = sb;
}

// Adam (Kingma & Ba): bias-corrected first/second moments
__global__ void __launch_bounds__(256) k_adam(int64_t n, float* __restrict__ p,
                                              const float* __restrict__ g, float* __restrict__ m,
                                              float* __restrict__ v, float lr, float b1, float b2,
                                              float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// parameters: weights U(-a, a), a = 1/sqrt(fan_in); ReLU biases 0.01; head bias 0
__global__ void __launch_bounds__(256) k_param_init(int64_t n, uint64_t seed,
                                                    const int32_t* __restrict__ fan_in,
                                                    float* __restrict__ p) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int fi = fan_in[i];
    if (fi <= 0) {
      p[i] = fi == 0 ? 0.01f : 0.f;
      continue;
    }
    uint64_t w0 = (uint64_t)i, w1 = 0x4d504e4eull, w2 = 0, w3 = 0;
    philox4x64_10(w0, w1, w2, w3, seed, 1ull);
    const float u = (float)(w0 >> 40) * 0x1p-23f - 1.0f;
    p[i] = u * rsqrtf((float)fi);
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
ParamLayout param_layout() {
  ParamLayout L;
  int64_t off = 0;
  auto put = [&off](int64_t& dst, int64_t size) {
    dst = off;
    off += size;
  };
  put(L.W_vin, kHid * kFv);
  put(L.b_vin, kHid);
  put(L.W_cin, kHid * kFc);
  put(L.b_cin, kHid);
  for (int l = 0; l < 2; ++l) {
    put(L.W_c[l], kHid * 2 * kHid);
    put(L.b_c[l], kHid);
    put(L.W_v[l], kHid * 2 * kHid);
    put(L.b_v[l], kHid);
  }
  put(L.w_out, kHid);
  put(L.b_out, 1);
  L.total = off;
  return L;
}

std::vector<int32_t> fan_in_table() {
  const ParamLayout L = param_layout();
  std::vector<int32_t> f((size_t)L.total, -1);   // -1: zero init
  auto fill = [&f](int64_t o, int64_t n, int32_t v) {
    for (int64_t i = 0; i < n; ++i) f[(size_t)(o + i)] = v;
  };
  fill(L.W_vin, kHid * kFv, kFv);
  fill(L.b_vin, kHid, 0);
  fill(L.W_cin, kHid * kFc, kFc);
  fill(L.b_cin, kHid, 0);
  for (int l = 0; l < 2; ++l) {
    fill(L.W_c[l], kHid * 2 * kHid, 2 * kHid);
    fill(L.b_c[l], kHid, 0);
    fill(L.W_v[l], kHid * 2 * kHid, 2 * kHid);
    fill(L.b_v[l], kHid, 0);
  }
  fill(L.w_out, kHid, kHid);
  return f;
}

ActLayout act_layout(int n, int m) {
  ActLayout A;
  size_t off = 0;
  auto take = [&off](size_t& dst, size_t floats) {
    dst = off;
    off += (floats + 63) / 64 * 64;   // 256-byte aligned
  };
  const size_t hn = (size_t)n * kHid, hm = (size_t)m * kHid;
  take(A.hv0, hn);
  take(A.hc0, hm);
  for (int l = 0; l < 2; ++l) {
    take(A.ac[l], hm);
    take(A.hc[l], hm);
    take(A.av[l], hn);
    take(A.hv[l], hn);
  }
  take(A.dhv, hn);
  take(A.dhc, hm);
  const int nodes = std::max(std::max(n, m), 1);
  take(A.dA, (size_t)nodes * kHid);
  A.n_dw_blk = ceil_div(nodes, kDwRows);
  take(A.dw_part, (size_t)A.n_dw_blk * (kHid * 2 * kHid + kHid));
  A.emb_chunk = 256;
  A.n_emb_blk = ceil_div(nodes, A.emb_chunk);
  take(A.emb_part, (size_t)A.n_emb_blk * kHid * (kFc + 1));
  take(A.emb_red, (size_t)kHid * (kFc + 1));
  take(A.head_part, (size_t)A.n_emb_blk * (kHid + 1));
  A.total_floats = off;
  return A;
}

cudaError_t forward(const Graph& G, const float* P, float* z, float* act, cudaStream_t s) {
  const ParamLayout L = param_layout();
  const ActLayout A = act_layout(G.n, G.m);
  float* hv = act + A.hv0;
  float* hc = act + A.hc0;
  if (G.n > 0)
    k_embed<kFv><<<ceil_div(G.n, 4), dim3(kHid, 4), 0, s>>>(G.n, G.fv, P + L.W_vin, P + L.b_vin,
                                                             hv);
  if (G.m > 0)
    k_embed<kFc><<<ceil_div(G.m, 4), dim3(kHid, 4), 0, s>>>(G.m, G.fc, P + L.W_cin, P + L.b_cin,
                                                             hc);
  for (int l = 0; l < 2; ++l) {
    float* ac = act + A.ac[l];
    float* hc_new = act + A.hc[l];
    float* av = act + A.av[l];
    float* hv_new = act + A.hv[l];
    if (G.m > 0) {
      k_seg_gather<<<ceil_div(G.m, 8), 256, 0, s>>>(G.m, G.con_off, G.con_var, G.con_sgn,
                                                    nullptr, G.isL, hv, ac, 0);
      k_dense_fwd<<<ceil_div(G.m, kTcRows), 256, 0, s>>>(G.m, hc, ac, P + L.W_c[l], P + L.b_c[l],
                                                          hc_new);
    }
    if (G.n > 0) {
      k_seg_gather<<<ceil_div(G.n, 8), 256, 0, s>>>(G.n, G.var_off, G.var_con, G.var_sgn,
                                                    nullptr, G.isd, hc_new, av, 0);
      k_dense_fwd<<<ceil_div(G.n, kTcRows), 256, 0, s>>>(G.n, hv, av, P + L.W_v[l], P + L.b_v[l],
                                                          hv_new);
    }
    hv = hv_new;
    hc = hc_new;
  }
  if (G.n > 0) k_head<<<ceil_div(G.n, 8), 256, 0, s>>>(G.n, hv, P + L.w_out, P + L.b_out, z);
  return cudaGetLastError();
}

cudaError_t points(const Graph& G, const float* z, int R, uint64_t seed, int64_t r_off, float tau,
                   float* x0, cudaStream_t s) {
  const int64_t total = (int64_t)((G.n + 3) / 4) * R;
  if (total == 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 148 * 16);
  k_points<<<blocks, 256, 0, s>>>(G.n, R, seed, r_off, tau, z, G.fixed, G.fixed_val, x0);
  return cudaGetLastError();
}

cudaError_t head_grad(const Graph& G, const float* z, const float* x0, const float* gx0, int R,
                      const int8_t* target, float lam, float* dz, cudaStream_t s) {
  if (G.n == 0) return cudaSuccess;
  const int nfree = G.n_free > 0 ? G.n_free : 1;
  k_head_grad<<<ceil_div(G.n, 8), 256, 0, s>>>(G.n, R, z, x0, gx0, target, lam, 1.f / nfree,
                                               G.fixed, dz);
  return cudaGetLastError();
}

namespace {
// backward of one dense layer: dY (aliased with dH) -> dW, db, dH, dA
cudaError_t dense_backward(int N, float* dY_dH, const float* Y, const float* H, const float* Aa,
                           const float* W, float* dA, float* dW, float* db, float* part,
                           int nblk_cap, cudaStream_t s) {
  const int nblk = ceil_div(N, kDwRows);
  if (nblk > nblk_cap) return cudaErrorInvalidValue;
  // dW/db read dY before dH overwrites it (same stream)
  k_dense_bwd_dw<<<nblk, 256, 0, s>>>(N, dY_dH, Y, H, Aa, part);
  const int stride = kHid * 2 * kHid + kHid;
  k_reduce_parts<<<ceil_div(kHid * 2 * kHid, 256), 256, 0, s>>>(nblk, kHid * 2 * kHid, stride,
                                                                part, dW);
  k_reduce_parts<<<1, kHid, 0, s>>>(nblk, kHid, stride, part + kHid * 2 * kHid, db);
  k_dense_bwd_dx<<<ceil_div(N, kTcRows), 256, 0, s>>>(N, dY_dH, Y, W, dY_dH, dA);
  return cudaGetLastError();
}

template <int K>
cudaError_t embed_backward(int N, int chunk, const float* f, const float* h, const float* dh,
                           float* part, float* red, float* W, float* b, cudaStream_t s) {
  const int nb = ceil_div(N, chunk);
  k_embed_bwd<K><<<nb, kHid, 0, s>>>(N, chunk, f, h, dh, part);
  k_reduce_parts<<<ceil_div(kHid * (K + 1), 256), 256, 0, s>>>(nb, kHid * (K + 1),
                                                               kHid * (K + 1), part, red);
  k_split_embed<K><<<1, kHid, 0, s>>>(red, W, b);
  return cudaGetLastError();
}
}  // namespace

cudaError_t backward(const Graph& G, const float* P, const float* dz, float* dP, float* act,
                     cudaStream_t s) {
  const ParamLayout L = param_layout();
  const ActLayout A = act_layout(G.n, G.m);
  float* dhv = act + A.dhv;
  float* dhc = act + A.dhc;
  float* dA = act + A.dA;
  float* part = act + A.dw_part;
  cudaError_t e;
  if (G.n > 0) {
    // head: dw_out, db_out (adjacent in the layout) and dh = dz w_out
    const int nb = ceil_div(G.n, A.emb_chunk);
    k_head_param_grad<<<nb, kHid, 0, s>>>(G.n, A.emb_chunk, act + A.hv[1], dz, act + A.head_part);
    k_reduce_parts<<<1, kHid + 1, 0, s>>>(nb, kHid + 1, kHid + 1, act + A.head_part,
                                          dP + L.w_out);
    k_head_dh<<<ceil_div(G.n, 4), 256, 0, s>>>(G.n, dz, P + L.w_out, dhv);
  } else {
    e = cudaMemsetAsync(dP + L.w_out, 0, sizeof(float) * (kHid + 1), s);
    if (e != cudaSuccess) return e;
  }
  if (G.m > 0) {
    e = cudaMemsetAsync(dhc, 0, sizeof(float) * (size_t)G.m * kHid, s);
    if (e != cudaSuccess) return e;
  }
  for (int l = 1; l >= 0; --l) {
    const float* hv_prev = l == 0 ? act + A.hv0 : act + A.hv[0];
    const float* hc_prev = l == 0 ? act + A.hc0 : act + A.hc[0];
    // variable update: dhv (d/d hv[l]) -> dW_v, db_v, d hv_prev (in place), d a_v
    if (G.n > 0) {
      e = dense_backward(G.n, dhv, act + A.hv[l], hv_prev, act + A.av[l], P + L.W_v[l], dA,
                         dP + L.W_v[l], dP + L.b_v[l], part, A.n_dw_blk, s);
      if (e != cudaSuccess) return e;
      // a_v = isd * sum s hc[l]:  dhc[c] += sum_{e in c} s_e isd[v_e] da_v[v_e]
      if (G.m > 0)
        k_seg_gather<<<ceil_div(G.m, 8), 256, 0, s>>>(G.m, G.con_off, G.con_var, G.con_sgn,
                                                      G.isd, nullptr, dA, dhc, 1);
    } else {
      cudaMemsetAsync(dP + L.W_v[l], 0, sizeof(float) * (kHid * 2 * kHid + kHid), s);
    }
    // constraint update: dhc (d/d hc[l]) -> dW_c, db_c, d hc_prev (in place), d a_c
    if (G.m > 0) {
      e = dense_backward(G.m, dhc, act + A.hc[l], hc_prev, act + A.ac[l], P + L.W_c[l], dA,
                         dP + L.W_c[l], dP + L.b_c[l], part, A.n_dw_blk, s);
      if (e != cudaSuccess) return e;
      // a_c = isL * sum s hv_prev:  dhv[v] += sum_{rows of v} s isL[c] da_c[c]
      if (G.n > 0)
        k_seg_gather<<<ceil_div(G.n, 8), 256, 0, s>>>(G.n, G.var_off, G.var_con, G.var_sgn,
                                                      G.isL, nullptr, dA, dhv, 1);
    } else {
      cudaMemsetAsync(dP + L.W_c[l], 0, sizeof(float) * (kHid * 2 * kHid + kHid), s);
    }
  }
  if (G.n > 0) {
    e = embed_backward<kFv>(G.n, A.emb_chunk, G.fv, act + A.hv0, dhv, act + A.emb_part,
                            act + A.emb_red, dP + L.W_vin, dP + L.b_vin, s);
    if (e != cudaSuccess) return e;
  }
  if (G.m > 0) {
    e = embed_backward<kFc>(G.m, A.emb_chunk, G.fc, act + A.hc0, dhc, act + A.emb_part,
                            act + A.emb_red, dP + L.W_cin, dP + L.b_cin, s);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t adam(int64_t n, float* p, const float* g, float* m, float* v, float lr, float b1,
                 float b2, float eps, int t, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 148 * 8);
  k_adam<<<blocks, 256, 0, s>>>(n, p, g, m, v, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t param_init(const int32_t* fan_in, int64_t n, uint64_t seed, float* p,
                       cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 148 * 8);
  k_param_init<<<blocks, 256, 0, s>>>(n, seed, fan_in, p);
  return cudaGetLastError();
}

}  // namespace mp
}  // namespace cls
