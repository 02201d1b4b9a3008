// kernels.cu -- sm_103a kernels of the CLS hot path.
//
// Layouts (see cls.h): x[v*R + r] (variable-major, restart-minor), literal
// partials P[row*Rp + r] with row = the literal's position in variable-major
// order (so the gradient of variable v is the sum of a contiguous run of
// rows), bitsets bits[v*RW + r/32] bit r%32.  A warp always spans 32
// consecutive restarts of a row, so every global access to x, P and bits is a
// coalesced 128-byte row segment or a warp-uniform broadcast.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "kernels.cuh"

namespace cls {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// read-only cached 16-byte table load
__device__ __forceinline__ float4 ldg4(const F4* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}

// Loads of data that an earlier stage of the SAME launch wrote (the
// persistent kernel) must not take the read-only path; CG = true routes them
// through L2 (ld.global.cg).
template <bool CG, typename T>
__device__ __forceinline__ T ldx(const T* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}
__device__ __forceinline__ int rec_row(int32_t dst) { return dst & 0x7fffffff; }
__device__ __forceinline__ float rec_sgn(int32_t dst) { return dst < 0 ? -1.0f : 1.0f; }

// ---------------------------------------------------------------------------
// A1 init: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// ---------------------------------------------------------------------------
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

__global__ void __launch_bounds__(256) k_init_uniform(int n, int R, uint64_t seed, int64_t r_off,
                                                      const uint8_t* __restrict__ fixed,
                                                      const float* __restrict__ fixed_val,
                                                      float* __restrict__ x) {
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
        float val = (float)(w[j] >> 40) * 0x1p-23f - 1.0f;  // exact: 24-bit integer * 2^-23
        if (fixed && fixed[v]) val = fixed_val[v];
        x[v * R + r] = val;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Per-restart convergence tracking and refills (Sec. 3.3: in a lockstep
// batch converged restarts idle; the distribution of steps to convergence).
// trk = int32[4][R]: best satisfied count, the step it was reached, steps
// since the last improvement, first step with every constraint satisfied
// (-1 = none yet).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_track_reset(int R, int32_t* __restrict__ trk) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  trk[r] = -1;
  trk[R + r] = -1;
  trk[2 * R + r] = 0;
  trk[3 * R + r] = -1;
}

__global__ void __launch_bounds__(256) k_track_step(int R, int m, int step,
                                                    const int32_t* __restrict__ nsat,
                                                    int32_t* __restrict__ trk) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const int32_t n = nsat[r];
  if (n > trk[r]) {
    trk[r] = n;
    trk[R + r] = step;
    trk[2 * R + r] = 0;
  } else {
    trk[2 * R + r] += 1;
  }
  if (n == m && trk[3 * R + r] < 0) trk[3 * R + r] = step;
}

__device__ __forceinline__ bool refill_due(int R, int r, int patience,
                                           const int32_t* __restrict__ trk) {
  return trk[3 * R + r] < 0 && trk[2 * R + r] >= patience;
}

// fresh points for the restarts due: the draw of k_init_uniform with the
// counter's third word = generation (>= 1); pinned variables untouched
__global__ void __launch_bounds__(256) k_refill(int n, int R, uint64_t seed, int64_t r_off,
                                                uint64_t gen, int patience,
                                                const uint8_t* __restrict__ fixed,
                                                const int32_t* __restrict__ trk,
                                                float* __restrict__ x) {
  const int64_t nq = (n + 3) / 4;
  const int64_t total = nq * (int64_t)R;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx % R);
    if (!refill_due(R, r, patience, trk)) continue;
    const int64_t q = idx / R;
    uint64_t w0 = (uint64_t)(r + r_off), w1 = (uint64_t)q, w2 = gen, w3 = 0;
    philox4x64_10(w0, w1, w2, w3, seed, 0ull);
    const uint64_t w[4] = {w0, w1, w2, w3};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t v = 4 * q + j;
      if (v < n && !(fixed && fixed[v])) x[v * R + r] = (float)(w[j] >> 40) * 0x1p-23f - 1.0f;
    }
  }
}

// after k_refill: the refilled restarts start their tracking again
__global__ void __launch_bounds__(256) k_refill_reset(int R, int patience,
                                                      int32_t* __restrict__ trk,
                                                      int32_t* __restrict__ count) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R || !refill_due(R, r, patience, trk)) return;
  trk[r] = -1;
  trk[R + r] = -1;
  trk[2 * R + r] = 0;
  atomicAdd(count, 1);
}

__global__ void __launch_bounds__(256) k_unsat_hist(int R, int m, const int32_t* __restrict__ nsat,
                                                    int32_t* __restrict__ hist) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const int k = m - nsat[r];
  if (k >= 0 && k <= m) atomicAdd(&hist[k], 1);
}

// per-restart movement of a step: maxdelta[r] = max_v |x[v, r] - x_prev[v, r]|
// (FP32, exact); a warp takes 32 restarts of kMoveVars consecutive
// variables, the maximum goes in by an integer atomicMax on the float's bits
// (non-negative floats order as their bit patterns), so the result does not
// depend on the order
constexpr int kMoveVars = 64;

__global__ void __launch_bounds__(256) k_move_max(int n, int R, const float* __restrict__ xp,
                                                  const float* __restrict__ x,
                                                  unsigned* __restrict__ maxdelta) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * 32 + lane;
  if (r >= R) return;
  const int64_t chunks = ((int64_t)n + kMoveVars - 1) / kMoveVars;
  float m = 0.f;
  for (int64_t ch = (int64_t)blockIdx.y * 8 + (threadIdx.x >> 5); ch < chunks;
       ch += (int64_t)gridDim.y * 8) {
    const int64_t v0 = ch * kMoveVars, v1 = min((int64_t)n, v0 + kMoveVars);
    for (int64_t v = v0; v < v1; ++v)
      m = fmaxf(m, fabsf(x[(size_t)v * R + r] - xp[(size_t)v * R + r]));
  }
  atomicMax(&maxdelta[r], __float_as_uint(m));
}

// first step at which a restart's movement is at most tol (conv[r] = -1
// until then)
__global__ void __launch_bounds__(256) k_track_conv(int R, const float* __restrict__ maxdelta,
                                                    float tol, int step,
                                                    int32_t* __restrict__ conv) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  if (conv[r] < 0 && maxdelta[r] <= tol) conv[r] = step;
}

// ---------------------------------------------------------------------------
// A2-A5, closed-form products (clause, XOR, NAE and complements) of short
// constraints: one thread per (constraint, restart), a warp = one constraint x
// 32 restarts, looping over kThreadTiles restart tiles.  The body is
// specialised on the exact length L (no guards in the unrolled loops); the
// literals' x and partial-row offsets are computed once per constraint (IDX =
// int when every offset fits in 31 bits).  FE = b0 + sum_j b'_j prod_i F_ij
// and dFE/dy_i = sum_j c'_j prod_{l!=i} F_lj with real factors F = A + y B:
// prefix products in registers, suffix products carried backwards (no
// division).
// ---------------------------------------------------------------------------
// The warp's literal records {var, dst} sit in shared memory (trec, one per
// literal, written by load_trec); addresses are formed with one 32x32->64
// multiply-add each, so a thread holds only its tile's values and prefixes.
__device__ __forceinline__ void load_trec(const FeItem& it, const LitRec* __restrict__ lit,
                                          int2* trec, int lane) {
  if (lane < it.L) {
    const LitRec rc = lit[it.lit0 + lane];
    trec[lane] = make_int2(rc.var, rc.dst);
  }
  __syncwarp();
}

template <int L, bool CG = false>
__device__ __forceinline__ void thread_body(const FeItem& it, const F4* __restrict__ root,
                                            const F4* __restrict__ coef, const int2* trec,
                                            const float* __restrict__ x, int R, int Rp, int RT,
                                            int tile0, int lane, float* __restrict__ P,
                                            float* __restrict__ fe_con, int ldf) {
  const float4 rt0 = ldg4(&root[it.root_off]), cf0 = ldg4(&coef[it.coef_off]);
  const bool two = it.J == 2;
  const float4 rt1 = two ? ldg4(&root[it.root_off + 1]) : make_float4(1.f, 0.f, 0.f, 0.f);
  const float4 cf1 = two ? ldg4(&coef[it.coef_off + 1]) : make_float4(0.f, 0.f, 0.f, 0.f);
  const unsigned xs = (unsigned)R, ps = (unsigned)Rp;
  for (int tt = 0; tt < kThreadTiles; ++tt) {
    const int tile = tile0 + tt;
    if (tile >= RT) break;
    const int r = tile * 32 + lane;
    if (r >= R) continue;
    const float* xr = x + r;
    float y[L], g[L], pre[L];
#pragma unroll
    for (int i = 0; i < L; ++i) {
      const int2 q = trec[i];
      y[i] = rec_sgn(q.y) * ldx<CG>(xr + (size_t)(unsigned)q.x * xs);
    }
    float run = 1.f;
#pragma unroll
    for (int i = 0; i < L; ++i) {
      pre[i] = run;
      run *= fmaf(y[i], rt0.y, rt0.x);
    }
    float val = fmaf(cf0.x, run, it.b0);
    float suf = cf0.z;
#pragma unroll
    for (int i = L - 1; i >= 0; --i) {
      g[i] = pre[i] * suf;
      suf *= fmaf(y[i], rt0.y, rt0.x);
    }
    if (two) {
      run = 1.f;
#pragma unroll
      for (int i = 0; i < L; ++i) {
        pre[i] = run;
        run *= fmaf(y[i], rt1.y, rt1.x);
      }
      val = fmaf(cf1.x, run, val);
      suf = cf1.z;
#pragma unroll
      for (int i = L - 1; i >= 0; --i) {
        g[i] = fmaf(pre[i], suf, g[i]);
        suf *= fmaf(y[i], rt1.y, rt1.x);
      }
    }
    float* pr = P + r;
#pragma unroll
    for (int i = 0; i < L; ++i) {
      const int2 q = trec[i];
      st_partial(&pr[(size_t)(unsigned)rec_row(q.y) * ps], it.w * rec_sgn(q.y) * g[i]);
    }
    if (fe_con) fe_con[(size_t)it.c * ldf + r] = val;
  }
}

// Restart tiles (of 32) per warp of k_fe_thread<LO, HI>: 8 up to 8
// literals, 4 beyond (the staging buffer stays at 64 KB per block).
template <int HI>
struct AsyncTiles {
  static constexpr int value = HI <= 8 ? 8 : 4;
};

// thread_body with the gathers of all NT tiles issued up front as
// cp.async copies into the warp's shared buffer (slot (tile, literal) at
// xb[(tt * L + i) * 32 + lane]), so that NT * L loads per thread
// are in flight without holding registers; each literal record is read from
// shared memory once (its variable for the copies, its destination kept in a
// register for the tiles when L <= 8; longer constraints read it again per
// tile).  Each thread reads back only what it copied itself.  Not for data written earlier in the same launch (the copies go
// through L1).
template <int L, int NT>
__device__ __forceinline__ void thread_body_async(const FeItem& it, const F4* __restrict__ root,
                                                  const F4* __restrict__ coef, const int2* trec,
                                                  const float* __restrict__ x, int R, int Rp,
                                                  int tile0, int lane, float* __restrict__ P,
                                                  float* __restrict__ fe_con, int ldf,
                                                  float* xb) {
  const unsigned xs = (unsigned)R, ps = (unsigned)Rp;
  constexpr bool kHold = L <= 8;
  int32_t dst[L];
#pragma unroll
  for (int i = 0; i < L; ++i) {
    const int2 q = trec[i];
    dst[i] = q.y;
    const float* xv = x + (size_t)(unsigned)q.x * xs;
#pragma unroll
    for (int tt = 0; tt < NT; ++tt) {
      const int r = (tile0 + tt) * 32 + lane;
      if (r < R) cp_async4(&xb[(tt * L + i) * 32 + lane], xv + r);
    }
  }
  cp_async_commit();
  const float4 rt0 = ldg4(&root[it.root_off]), cf0 = ldg4(&coef[it.coef_off]);
  const bool two = it.J == 2;
  const float4 rt1 = two ? ldg4(&root[it.root_off + 1]) : make_float4(1.f, 0.f, 0.f, 0.f);
  const float4 cf1 = two ? ldg4(&coef[it.coef_off + 1]) : make_float4(0.f, 0.f, 0.f, 0.f);
  cp_async_wait<0>();
#pragma unroll 1
  for (int tt = 0; tt < NT; ++tt) {
    const int r = (tile0 + tt) * 32 + lane;
    if (r >= R) break;
    float y[L], g[L], pre[L];
#pragma unroll
    for (int i = 0; i < L; ++i) {
      if constexpr (!kHold) dst[i] = trec[i].y;   // re-read per tile, fewer registers
      y[i] = rec_sgn(dst[i]) * xb[(tt * L + i) * 32 + lane];
    }
    float run = 1.f;
#pragma unroll
    for (int i = 0; i < L; ++i) {
      pre[i] = run;
      run *= fmaf(y[i], rt0.y, rt0.x);
    }
    float val = fmaf(cf0.x, run, it.b0);
    float suf = cf0.z;
#pragma unroll
    for (int i = L - 1; i >= 0; --i) {
      g[i] = pre[i] * suf;
      suf *= fmaf(y[i], rt0.y, rt0.x);
    }
    if (two) {
      run = 1.f;
#pragma unroll
      for (int i = 0; i < L; ++i) {
        pre[i] = run;
        run *= fmaf(y[i], rt1.y, rt1.x);
      }
      val = fmaf(cf1.x, run, val);
      suf = cf1.z;
#pragma unroll
      for (int i = L - 1; i >= 0; --i) {
        g[i] = fmaf(pre[i], suf, g[i]);
        suf *= fmaf(y[i], rt1.y, rt1.x);
      }
    }
    float* pr = P + r;
#pragma unroll
    for (int i = 0; i < L; ++i) {
      const int32_t d = kHold ? dst[i] : trec[i].y;
      st_partial(&pr[(size_t)(unsigned)rec_row(d) * ps], it.w * rec_sgn(d) * g[i]);
    }
    if (fe_con) fe_con[(size_t)it.c * ldf + r] = val;
  }
}

template <int LO, int HI, int NT>
__device__ __forceinline__ void thread_dispatch_async(int L, const FeItem& it, const F4* root,
                                                      const F4* coef, const int2* trec,
                                                      const float* x, int R, int Rp, int tile0,
                                                      int lane, float* P, float* fe_con, int ldf,
                                                      float* xb) {
  if constexpr (LO <= HI) {
    if (L == LO)
      thread_body_async<LO, NT>(it, root, coef, trec, x, R, Rp, tile0, lane, P, fe_con, ldf, xb);
    else
      thread_dispatch_async<LO + 1, HI, NT>(L, it, root, coef, trec, x, R, Rp, tile0, lane, P,
                                        fe_con, ldf, xb);
  }
}

template <int LO, int HI, bool CG = false>
__device__ __forceinline__ void thread_dispatch(int L, const FeItem& it, const F4* root,
                                                const F4* coef, const int2* trec,
                                                const float* x, int R, int Rp, int RT, int tile0,
                                                int lane, float* P, float* fe_con, int ldf) {
  if constexpr (LO <= HI) {
    if (L == LO)
      thread_body<LO, CG>(it, root, coef, trec, x, R, Rp, RT, tile0, lane, P, fe_con, ldf);
    else
      thread_dispatch<LO + 1, HI, CG>(L, it, root, coef, trec, x, R, Rp, RT, tile0, lane, P,
                                      fe_con, ldf);
  }
}

// Dynamic shared memory: 8 warps x AsyncTiles<HI>::value x HI x 32 floats (the
// staged literal values).
template <int LO, int HI>
__global__ void __launch_bounds__(256) k_fe_thread(
    const FeItem* __restrict__ items, int count, const F4* __restrict__ root,
    const F4* __restrict__ coef, const LitRec* __restrict__ lit, const float* __restrict__ x,
    int R, int Rp, int RT, float* __restrict__ P, float* __restrict__ fe_con, int ldf) {
  __shared__ int2 trec_s[8][HI];
  extern __shared__ float thread_xbuf[];
  const int lane = threadIdx.x;
  int2* trec = trec_s[threadIdx.y];
  constexpr int NT = AsyncTiles<HI>::value;
  float* xb = thread_xbuf + (size_t)threadIdx.y * NT * HI * 32;
  // blockIdx.x (fastest in launch order) walks the constraints, blockIdx.y
  // the restart groups: the blocks in flight share one group's slice of x
  // (n * NT * 128 B), which stays in L2 while the partial writes stream past
  for (int ci = blockIdx.x * blockDim.y + threadIdx.y; ci < count; ci += gridDim.x * blockDim.y) {
    const FeItem it = items[ci];
    __syncwarp();
    load_trec(it, lit, trec, lane);
    thread_dispatch_async<LO, HI, NT>(it.L, it, root, coef, trec, x, R, Rp,
                                      blockIdx.y * NT, lane, P, fe_con, ldf, xb);
  }
}

template <int HI>
constexpr size_t thread_xbuf_bytes() {
  return (size_t)8 * AsyncTiles<HI>::value * HI * 32 * sizeof(float);
}

// ---------------------------------------------------------------------------
// A2-A5, closed-form products (OR, XOR, NAE, ...) of any length: one thread
// per (constraint, restart).  A block takes one constraint and 8 tiles of 32
// restarts (a warp per tile).  The block first writes one record per literal
// to shared memory -- {variable, partial row, s*B_0, w*s} and, for two real
// roots, s*B_1 -- so that the inner loops do one broadcast shared load, one
// 32-bit multiply-add for the address and one coalesced load per literal
// (A_j is the same for every literal).  Literals past L (up to a multiple of
// the checkpoint interval CI) read x[0] and take the factor 1 by a select.
// The forward pass keeps every CI-th prefix product in shared memory; the
// backward pass walks the literal blocks from the end, recomputes a block's
// prefix products from its checkpoint in registers (the block's values are
// loaded again, L2 hits) and combines them with the running suffix product.
// Dynamic shared memory: 16 B x NJ x LCAP records + 8 warps x NJ x nck x 32
// floats.
// ---------------------------------------------------------------------------
template <int NJ, int CI>
__global__ void __launch_bounds__(256) k_fe_thread_ckpt(
    const int32_t* __restrict__ list, const FeItem* __restrict__ fe,
    const F4* __restrict__ root, const F4* __restrict__ coef, const LitRec* __restrict__ lit,
    const float* __restrict__ x, int R, int Rp, int RT, int nck, float* __restrict__ P,
    float* __restrict__ fe_con, int ldf) {
  extern __shared__ float4 ck_smem[];
  const int LCAP = nck * CI;
  float4* reca = ck_smem;                    // [LCAP] {var, row, s*B_0, w*s}
  float* recb = reinterpret_cast<float*>(ck_smem + LCAP);   // [LCAP] s*B_1 (NJ = 2)
  const int lane = threadIdx.x, w = threadIdx.y;
  float* ck = reinterpret_cast<float*>(ck_smem + LCAP) + (NJ > 1 ? LCAP : 0) +
              (size_t)w * NJ * nck * 32;
  const FeItem it = fe[list[blockIdx.x]];
  const int L = it.L;
  float4 rt[NJ], cf[NJ];
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    rt[j] = ldg4(&root[it.root_off + min(j, it.J - 1)]);
    cf[j] = ldg4(&coef[it.coef_off + min(j, it.J - 1)]);
    if (j >= it.J) {                 // a one-root constraint in a two-root launch
      rt[j] = make_float4(1.f, 0.f, 0.f, 0.f);
      cf[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  for (int i = w * 32 + lane; i < LCAP; i += 256) {
    if (i < L) {
      const LitRec rc = lit[it.lit0 + i];
      const float sg = rec_sgn(rc.dst);
      reca[i] = make_float4(__int_as_float(rc.var), __int_as_float(rec_row(rc.dst)),
                            sg * rt[0].y, it.w * sg);
      if (NJ > 1) recb[i] = sg * rt[NJ - 1].y;
    } else {
      reca[i] = make_float4(__int_as_float(0), __int_as_float(0), 0.f, 0.f);
      if (NJ > 1) recb[i] = 0.f;
    }
  }
  __syncthreads();
  const int tile = blockIdx.y * 8 + w;
  if (tile >= RT) return;
  const int r = tile * 32 + lane;
  const bool act = r < R;
  const float* xr = x + (act ? r : R - 1);
  const unsigned xstride = (unsigned)R * 4u, pstride = (unsigned)Rp * 4u;
  auto xval = [&](const float4& q) -> float {
    return *reinterpret_cast<const float*>(reinterpret_cast<const char*>(xr) +
                                           (size_t)(unsigned)__float_as_int(q.x) * xstride);
  };
  const float A0 = rt[0].x, A1 = rt[NJ - 1].x;
  const int nb = (L + CI - 1) / CI;
  // forward: running products, checkpoint at each block start
  float run[NJ];
#pragma unroll
  for (int j = 0; j < NJ; ++j) run[j] = 1.f;
  for (int b = 0; b < nb; ++b) {
#pragma unroll
    for (int j = 0; j < NJ; ++j) ck[(j * nck + b) * 32 + lane] = run[j];
    const int lim = L - b * CI;
    float xv[CI];
#pragma unroll
    for (int t = 0; t < CI; ++t) xv[t] = xval(reca[b * CI + t]);
#pragma unroll
    for (int t = 0; t < CI; ++t) {
      const float4 q = reca[b * CI + t];
      run[0] *= t < lim ? fmaf(xv[t], q.z, A0) : 1.f;
      if constexpr (NJ > 1) run[1] *= t < lim ? fmaf(xv[t], recb[b * CI + t], A1) : 1.f;
    }
  }
  float val = it.b0;
#pragma unroll
  for (int j = 0; j < NJ; ++j) val = fmaf(cf[j].x, run[j], val);
  // backward: suffix products with c'_j folded in
  float suf[NJ];
#pragma unroll
  for (int j = 0; j < NJ; ++j) suf[j] = cf[j].z;
  for (int b = nb - 1; b >= 0; --b) {
    float xv[CI], pre[NJ][CI], p[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) p[j] = ck[(j * nck + b) * 32 + lane];
    const int lim = L - b * CI;
#pragma unroll
    for (int t = 0; t < CI; ++t) {
      const float v = xval(reca[b * CI + t]);
      xv[t] = t < lim ? v : 0.f;
    }
#pragma unroll
    for (int t = 0; t < CI; ++t) {
      const float4 q = reca[b * CI + t];
      pre[0][t] = p[0];
      p[0] *= t < lim ? fmaf(xv[t], q.z, A0) : 1.f;
      if constexpr (NJ > 1) {
        pre[1][t] = p[1];
        p[1] *= t < lim ? fmaf(xv[t], recb[b * CI + t], A1) : 1.f;
      }
    }
#pragma unroll
    for (int t = CI - 1; t >= 0; --t) {
      const float4 q = reca[b * CI + t];
      float g = pre[0][t] * suf[0];
      suf[0] *= t < lim ? fmaf(xv[t], q.z, A0) : 1.f;
      if constexpr (NJ > 1) {
        g = fmaf(pre[1][t], suf[1], g);
        suf[1] *= t < lim ? fmaf(xv[t], recb[b * CI + t], A1) : 1.f;
      }
      if (act && t < lim)
        st_partial(reinterpret_cast<float*>(reinterpret_cast<char*>(P + r) +
                                            (size_t)(unsigned)__float_as_int(q.y) * pstride),
                   q.w * g);
    }
  }
  if (fe_con && act) fe_con[(size_t)it.c * ldf + r] = val;
}

// ---------------------------------------------------------------------------
// A2-A5 lane-group kernel: G lanes share one (constraint, restart); lane lam
// holds literals lam, lam+G, ..., (Q slots).  One block = one constraint x a
// tile of 32 restarts; literal values are staged in shared memory as
// ys[i*LDR + rr] with LDR = 32 + 32/G, which makes both the coalesced staging
// stores (lanes over rr) and the group reads (lanes over lam, groups over rr)
// bank-conflict free.  Slots beyond L are staged as y = 1.
//
// Per root j: factors F_ij, lane-local exclusive prefix products, then a
// butterfly over the G lanes that yields both the total G_j = prod_i F_ij and
// the product of the OTHER lanes' chunks (leave-one-lane-out, O).  The
// gradient uses prod_{l!=i} F_lj = O * prefix_i * suffix_i with the suffix
// carried backwards and c'_j O folded into it: no division by a factor, so
// nothing breaks where a factor vanishes.  For DFT roots y = 1 gives a factor
// of exactly 1 (A + B == 1, C - C == 0), so padding needs no masking; real
// roots mask padding explicitly (beta(1) = 0).  YS re-reads y from shared
// memory in both passes instead of holding Q registers.
// ---------------------------------------------------------------------------
template <int G>
struct GroupGeom {
  static constexpr int LDR = 32 + 32 / G;
  static constexpr int GPW = 32 / G;         // groups per warp
  static constexpr int GPB = 8 * GPW;        // groups per block (256 threads)
  static constexpr int PASSES = 32 / GPB;    // to cover 32 restarts
};

template <int G, int Q, bool CPLX, bool YS>
__global__ void __launch_bounds__(256) k_fe_group(
    const int32_t* __restrict__ list, const FeItem* __restrict__ fe,
    const F4* __restrict__ root, const F4* __restrict__ coef, const LitRec* __restrict__ lit,
    const float* __restrict__ x, int R, int Rp, float* __restrict__ P,
    float* __restrict__ fe_con, int ldf, const uint8_t* __restrict__ done, int RT,
    unsigned long long* __restrict__ flops) {
  using Geo = GroupGeom<G>;
  constexpr int LS = G * Q;          // staged literal slots
  extern __shared__ float smem[];
  float* ys = smem;                  // [LS][LDR]
  __shared__ float fe_s[32];
  const FeItem it = fe[list[blockIdx.x]];
  // the one-thread corner pass finished this tile (partials and FE written)
  if (done && done[(size_t)it.c * RT + blockIdx.y] == kTileDone) return;
  const int L = it.L;
  const int r0 = blockIdx.y * 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // the constraint's literal records once per block (one coalesced read),
  // then the literal values y = s * x (coalesced rows of 32 restarts), four
  // rows in flight per warp
  __shared__ LitRec lrec_s[LS];
  for (int i = threadIdx.x; i < L; i += 256) lrec_s[i] = lit[it.lit0 + i];
  __syncthreads();
#pragma unroll 4
  for (int i = warp; i < LS; i += 8) {
    float v = 1.0f;
    if (i < L) {
      const LitRec rc = lrec_s[i];
      const int r = r0 + lane;
      if (r < R) v = rec_sgn(rc.dst) * x[(size_t)rc.var * R + r];
    }
    ys[i * Geo::LDR + lane] = v;
  }
  __syncthreads();

  const int lam = lane % G;
  const int gi = lane / G;
#pragma unroll 1
  for (int pass = 0; pass < Geo::PASSES; ++pass) {
    const int rr = pass * Geo::GPB + warp * Geo::GPW + gi;
    const float* ycol = ys + lam * Geo::LDR + rr;   // slot s at ycol[s * G * LDR]
    float yreg[YS ? 1 : Q], acc[Q];
#pragma unroll
    for (int s = 0; s < Q; ++s) {
      if constexpr (!YS) yreg[s] = ycol[s * G * Geo::LDR];
      acc[s] = 0.f;
    }
    auto Y = [&](int s) -> float {
      if constexpr (YS) return ycol[s * G * Geo::LDR];
      else return yreg[s];
    };
    float val = 0.f;
#pragma unroll 1
    for (int j = 0; j < it.J; ++j) {
      const float4 rt = ldg4(&root[it.root_off + j]);
      const float4 cf = ldg4(&coef[it.coef_off + j]);
      if constexpr (CPLX) {
        float pr[Q], pim[Q];
        float qr, qi;
        {
          const float y0 = Y(0);
          qr = fmaf(y0, rt.y, rt.x);
          qi = fmaf(-y0, rt.z, rt.z);
        }
        pr[0] = 1.f;
        pim[0] = 0.f;
#pragma unroll
        for (int s = 1; s < Q; ++s) {
          pr[s] = qr;
          pim[s] = qi;
          const float ys_ = Y(s);
          const float fr = fmaf(ys_, rt.y, rt.x), fi = fmaf(-ys_, rt.z, rt.z);
          const float nr = qr * fr - qi * fi;
          const float ni = qr * fi + qi * fr;
          qr = nr;
          qi = ni;
        }
        // butterfly over the G lanes: Pt = total, O = product of the others
        float Ptr = qr, Pti = qi, Or = 1.f, Oi = 0.f;
#pragma unroll
        for (int d = 1; d < G; d <<= 1) {
          const float tr = __shfl_xor_sync(kFull, Ptr, d);
          const float ti = __shfl_xor_sync(kFull, Pti, d);
          if (d == 1) {
            Or = tr;
            Oi = ti;
          } else {
            const float a = Or * tr - Oi * ti, b = Or * ti + Oi * tr;
            Or = a;
            Oi = b;
          }
          const float a = Ptr * tr - Pti * ti, b = Ptr * ti + Pti * tr;
          Ptr = a;
          Pti = b;
        }
        val = fmaf(cf.x, Ptr, val);
        val = fmaf(-cf.y, Pti, val);
        float hr = cf.z * Or - cf.w * Oi, hi = cf.z * Oi + cf.w * Or;
#pragma unroll
        for (int s = Q - 1; s >= 0; --s) {
          acc[s] = fmaf(pr[s], hr, acc[s]);
          acc[s] = fmaf(-pim[s], hi, acc[s]);
          if (s > 0) {
            const float ys_ = Y(s);
            const float fr = fmaf(ys_, rt.y, rt.x), fi = fmaf(-ys_, rt.z, rt.z);
            const float a = hr * fr - hi * fi, b = hr * fi + hi * fr;
            hr = a;
            hi = b;
          }
        }
      } else {
        // real roots (closed forms): padding slots must contribute factor 1
        float pr[Q];
        float q = 1.f;
#pragma unroll
        for (int s = 0; s < Q; ++s) {
          pr[s] = q;
          const bool live = lam + G * s < L;
          q *= live ? fmaf(Y(s), rt.y, rt.x) : 1.f;
        }
        float Pt = q, O = 1.f;
#pragma unroll
        for (int d = 1; d < G; d <<= 1) {
          const float t = __shfl_xor_sync(kFull, Pt, d);
          O = (d == 1) ? t : O * t;
          Pt *= t;
        }
        val = fmaf(cf.x, Pt, val);
        float h = cf.z * O;
#pragma unroll
        for (int s = Q - 1; s >= 0; --s) {
          acc[s] = fmaf(pr[s], h, acc[s]);
          const bool live = lam + G * s < L;
          h *= live ? fmaf(Y(s), rt.y, rt.x) : 1.f;
        }
      }
    }
    // partials back into the staging slots (each slot is owned by one lane)
#pragma unroll
    for (int s = 0; s < Q; ++s) {
      const int i = lam + G * s;
      if (i < L) ys[i * Geo::LDR + rr] = acc[s];
    }
    if (lam == 0) fe_s[rr] = it.b0 + val;
  }
  __syncthreads();
  // write partials w * s_e * dFE/dy_e to their variable-major rows
#pragma unroll 4
  for (int i = warp; i < L; i += 8) {
    const LitRec rc = lrec_s[i];
    const int r = r0 + lane;
    if (r < R)
      st_partial(&P[(size_t)rec_row(rc.dst) * Rp + r], it.w * rec_sgn(rc.dst) * ys[i * Geo::LDR + lane]);
  }
  // DFT roots: 20 flops per (literal, root) of every restart (all J roots)
  if constexpr (CPLX)
    if (flops && threadIdx.x == 0)
      atomicAdd(flops, 20ull * (unsigned long long)L * (unsigned long long)it.J *
                           (unsigned long long)min(32, R - r0));
  if (fe_con && warp == 0 && r0 + lane < R) fe_con[(size_t)it.c * ldf + r0 + lane] = fe_s[lane];
}

// ---------------------------------------------------------------------------
// A6-A8: gradient accumulation through the variable-major transpose (a
// contiguous run of rows per variable, summed in row order: deterministic, no
// atomics), projected step, rounding to a bitset by warp ballot.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float pgd_project(float xv, float g, float lr) {
  // x' = min(max(fl(x - fl(lr*g)), -1), 1): two explicit roundings, no FMA
  const float t = __fmul_rn(lr, g);
  return fminf(fmaxf(__fsub_rn(xv, t), -1.0f), 1.0f);
}

// one (variable, 32-restart tile): called by whole warps
template <bool CG = false>
__device__ __forceinline__ void accum_one(int v, int tile, int lane, int R, int Rp, int RW,
                                          const int32_t* __restrict__ voff,
                                          const float* __restrict__ P, float* __restrict__ x,
                                          float lr, int do_step, const uint8_t* __restrict__ fixed,
                                          float* __restrict__ grad_out,
                                          uint32_t* __restrict__ bits) {
  const int r = tile * 32 + lane;
  const bool act = r < R;
  {
    const int k0 = voff[v], k1 = voff[v + 1];
    float g = 0.f;
    if (act) {
      const float* p = P + (size_t)k0 * Rp + r;
      int k = k0;
      for (; k + 4 <= k1; k += 4, p += 4 * (size_t)Rp) {
        const float a0 = ldx<CG>(p), a1 = ldx<CG>(p + (size_t)Rp);
        const float a2 = ldx<CG>(p + 2 * (size_t)Rp), a3 = ldx<CG>(p + 3 * (size_t)Rp);
        g += a0;
        g += a1;
        g += a2;
        g += a3;
      }
      for (; k < k1; ++k, p += Rp) g += ldx<CG>(p);
    }
    if (grad_out && act) grad_out[(size_t)v * R + r] = g;
    if (do_step) {
      float xv = 0.f;
      if (act) {
        xv = ldx<CG>(&x[(size_t)v * R + r]);
        if (!(fixed && fixed[v])) {
          xv = pgd_project(xv, g, lr);
          x[(size_t)v * R + r] = xv;
        }
      }
      const uint32_t b = __ballot_sync(kFull, act && xv < 0.0f);
      if (bits && lane == 0) bits[(size_t)v * RW + tile] = b;
    }
  }
}

__global__ void __launch_bounds__(256) k_accum_step(int n, int R, int Rp, int RW,
                                                    const int32_t* __restrict__ voff,
                                                    const float* __restrict__ P,
                                                    float* __restrict__ x, float lr, int do_step,
                                                    const uint8_t* __restrict__ fixed,
                                                    float* __restrict__ grad_out,
                                                    uint32_t* __restrict__ bits) {
  for (int v = blockIdx.y * blockDim.y + threadIdx.y; v < n; v += gridDim.y * blockDim.y)
    accum_one(v, blockIdx.x, threadIdx.x, R, Rp, RW, voff, P, x, lr, do_step, fixed, grad_out,
              bits);
}

// accum_one for NT consecutive restart tiles of one variable per warp: the
// rows' loads of all NT tiles in flight together (NT x 128 contiguous bytes
// per row), each tile's sum in row order as in accum_one, so the results are
// the same bit for bit.  For variables with few rows (short clauses, many
// restarts), where a warp per (variable, tile) spends more on its fixed
// work than on its loads.
template <int NT>
__global__ void __launch_bounds__(256) k_accum_step_nt(int n, int R, int Rp, int RW,
                                                       const int32_t* __restrict__ voff,
                                                       const float* __restrict__ P,
                                                       float* __restrict__ x, float lr,
                                                       int do_step,
                                                       const uint8_t* __restrict__ fixed,
                                                       float* __restrict__ grad_out,
                                                       uint32_t* __restrict__ bits) {
  const int lane = threadIdx.x;
  const int tile0 = blockIdx.x * NT;
  for (int v = blockIdx.y * blockDim.y + threadIdx.y; v < n; v += gridDim.y * blockDim.y) {
    const int k0 = voff[v], k1 = voff[v + 1];
    float g[NT];
    bool act[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      g[t] = 0.f;
      act[t] = tile0 + t < RW && (tile0 + t) * 32 + lane < R;
    }
    const float* p = P + (size_t)k0 * Rp + (size_t)tile0 * 32 + lane;
    int k = k0;
    for (; k + 2 <= k1; k += 2, p += 2 * (size_t)Rp) {
      float a[NT], b[NT];
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        a[t] = act[t] ? p[t * 32] : 0.f;
        b[t] = act[t] ? p[(size_t)Rp + t * 32] : 0.f;
      }
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        g[t] += a[t];
        g[t] += b[t];
      }
    }
    for (; k < k1; ++k, p += Rp) {
#pragma unroll
      for (int t = 0; t < NT; ++t)
        if (act[t]) g[t] += p[t * 32];
    }
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int tile = tile0 + t;
      if (tile >= RW) break;
      const int r = tile * 32 + lane;
      if (grad_out && act[t]) grad_out[(size_t)v * R + r] = g[t];
      if (do_step) {
        float xv = 0.f;
        if (act[t]) {
          xv = x[(size_t)v * R + r];
          if (!(fixed && fixed[v])) {
            xv = pgd_project(xv, g[t], lr);
            x[(size_t)v * R + r] = xv;
          }
        }
        const uint32_t bw = __ballot_sync(kFull, act[t] && xv < 0.0f);
        if (bits && lane == 0) bits[(size_t)v * RW + tile] = bw;
      }
    }
  }
}

// tiles per warp of the accumulate kernel: four when the variables have few
// partial rows on average and there are tiles enough to fill the GPU
inline int accum_tiles_per_warp(const DevPlan& d, int RT) {
  return (d.nnz_fe < (int64_t)16 * d.n && RT >= 4 * 148) ? 4 : 1;
}

__global__ void __launch_bounds__(256) k_pgd(int n, int R, int RW, float* __restrict__ x,
                                             const float* __restrict__ grad, float lr,
                                             int do_step, const uint8_t* __restrict__ fixed,
                                             uint32_t* __restrict__ bits) {
  const int lane = threadIdx.x;
  const int r = blockIdx.x * 32 + lane;
  const bool act = r < R;
  for (int v = blockIdx.y * blockDim.y + threadIdx.y; v < n; v += gridDim.y * blockDim.y) {
    float xv = 0.f;
    if (act) {
      xv = x[(size_t)v * R + r];
      if (do_step && !(fixed && fixed[v])) {
        xv = pgd_project(xv, grad[(size_t)v * R + r], lr);
        x[(size_t)v * R + r] = xv;
      }
    }
    const uint32_t b = __ballot_sync(kFull, act && xv < 0.0f);
    if (bits && lane == 0) bits[(size_t)v * RW + blockIdx.x] = b;
  }
}

// ---------------------------------------------------------------------------
// A9: exact satisfaction counts.  A warp owns a range of consecutive
// constraints and one tile of 32 restarts.  It walks the range's literals in
// chunks of 32: lane i fetches literal i's bitset word (bit r = its variable
// is true at restart r), inverted for a negated literal, so bit r = "literal
// true at restart r".  A 5-step shuffle butterfly transposes the 32x32 bit
// matrix, after which lane r holds, for its restart, one bit per literal of
// the chunk; each constraint's count t is a popcount of its bit segment
// (carried across chunks for long constraints).  Per-warp counts are reduced
// over the block's warps in a fixed order into per-chunk partials.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
  const uint32_t masks[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int j = 16 >> k;
    const uint32_t m = masks[k];
    const uint32_t y = __shfl_xor_sync(kFull, x, j);
    x = (lane & j) ? ((x & ~m) | ((y >> j) & m)) : ((x & m) | ((y << j) & ~m));
  }
  return x;
}

__device__ __forceinline__ bool sat_of(const ScoreItem& s, int t,
                                       const uint32_t* __restrict__ satbits) {
  if (s.mode == 0) return t >= s.lo && t <= s.hi;
  if (s.mode == 1) return (t & 1) != 0;
  return ((satbits[(s.lo + t) >> 5] >> ((s.lo + t) & 31)) & 1u) != 0;
}

// one range of constraints for one tile of 32 restarts (whole warp); returns
// the lane's satisfied count and satisfied weight (UNIT: all weights are 1,
// the weight is the count -- the same FP64 value, without FP64 adds)
template <bool CG = false, bool UNIT = false>
__device__ __forceinline__ void score_range(int rg, int tile, int lane, int RW,
                                            const int32_t* __restrict__ ranges,
                                            const ScoreItem* __restrict__ sc,
                                            const LitRec* __restrict__ lit,
                                            const uint32_t* __restrict__ satbits,
                                            const uint32_t* __restrict__ bits, int* cnt_out,
                                            double* ws_out) {
  int cnt = 0;
  double ws = 0.0;
  int c = ranges[rg];
  const int c_end = ranges[rg + 1];
  ScoreItem s = sc[c];
  int e = s.lit0;
  const ScoreItem last = sc[c_end - 1];
  const int e_end = last.lit0 + last.L;
  int run = 0;
  while (e < e_end) {
    uint32_t word = 0;
    if (e + lane < e_end) {
      const LitRec rc = lit[e + lane];
      word = ldx<CG>(&bits[(size_t)rc.var * RW + tile]);
      if (rc.dst < 0) word = ~word;
    }
    const uint32_t col = transpose32(word, lane);
    const int chunk_end = e + 32;
    // constraints ending inside this chunk
    while (c < c_end && s.lit0 + s.L <= chunk_end) {
      const int lo = max(s.lit0, e) - e;
      const int hi = s.lit0 + s.L - e;
      const uint32_t mask = (hi >= 32 ? kFull : ((1u << hi) - 1u)) & (kFull << lo);
      const int t = run + __popc(col & mask);
      run = 0;
      const bool sat = sat_of(s, t, satbits);
      cnt += sat ? 1 : 0;
      if constexpr (!UNIT) ws += sat ? (double)s.w : 0.0;
      ++c;
      if (c < c_end) s = sc[c];
    }
    // a constraint straddling into the next chunk
    if (c < c_end && s.lit0 < chunk_end) {
      const int lo = max(s.lit0, e) - e;
      run += __popc(col & (kFull << lo));
    }
    e = chunk_end;
  }
  *cnt_out = cnt;
  *ws_out = UNIT ? (double)cnt : ws;
}

// ---------------------------------------------------------------------------
// Adaptive constraint weighting (Sec. 3.1 suggests weights informed by the
// constraints' gradient magnitudes).  Per constraint c, over the R restarts:
//   gnorm[c] = sum_r || dFE_c/dy (x_r) ||_2  over the literals entering FE,
//              from the partials P (= w_c s_e dFE_c/dy_e) of the last
//              evaluation, divided by |w_c| (0 where w_c = 0);
//   unsat[c] = # restarts whose rounded point (bitset) violates c.
// Pass 1: one warp per (constraint, tile of 32 restarts), pairs in
// constraint-major order over a grid-stride loop (long and short
// constraints balance out); each lane's norm in FP32, the warp's 32 norms
// added in a fixed FP32 tree, written with the tile's violation count to
// scratch [m][RW].  Pass 2: one warp per constraint adds its RW tile sums
// in FP64 in a fixed order.
// ---------------------------------------------------------------------------
constexpr int kStatWarps = 8;
constexpr int kStatTiles = 8;   // restart tiles per warp work item (loads in flight)

__global__ void __launch_bounds__(256) k_con_stats_tile(int m, int RW, int R, int Rp,
                                                        const FeItem* __restrict__ fe,
                                                        const ScoreItem* __restrict__ sc,
                                                        const LitRec* __restrict__ fe_lit,
                                                        const LitRec* __restrict__ lit,
                                                        const uint32_t* __restrict__ satbits,
                                                        const uint32_t* __restrict__ bits,
                                                        const float* __restrict__ P,
                                                        const int32_t* __restrict__ order,
                                                        float* __restrict__ tg,
                                                        int32_t* __restrict__ tu) {
  const int lane = threadIdx.x & 31;
  const int TG = (RW + kStatTiles - 1) / kStatTiles;   // tile groups per constraint
  const int64_t total = (int64_t)m * TG;
  const int64_t nw = (int64_t)gridDim.x * kStatWarps;
  for (int64_t item = (int64_t)blockIdx.x * kStatWarps + (threadIdx.x >> 5); item < total;
       item += nw) {
    // constraints longest first, so that the long items start early
    const int oc = (int)(item / TG);
    const int c = order[oc];
    const int tile0 = (int)(item - (int64_t)oc * TG) * kStatTiles;
    const int nt = min(kStatTiles, RW - tile0);
    const FeItem it = fe[c];
    const ScoreItem s = sc[c];
    // sum of squared partials per (tile, lane): 32 literals at a time, lane k
    // fetches literal k's partial row, then every row is read for the
    // item's tiles (independent 128-byte loads)
    float q[kStatTiles];
#pragma unroll
    for (int tt = 0; tt < kStatTiles; ++tt) q[tt] = 0.f;
    const LitRec* fl = fe_lit + it.lit0;
    for (int k0 = 0; k0 < it.L; k0 += 32) {
      const int nk = min(32, it.L - k0);
      const int myrow = lane < nk ? rec_row(fl[k0 + lane].dst) : 0;
      int k = 0;
      for (; k + 2 <= nk; k += 2) {   // two rows' loads issued before their FMAs
        const float* ra = P + (size_t)__shfl_sync(kFull, myrow, k) * Rp + tile0 * 32 + lane;
        const float* rb = P + (size_t)__shfl_sync(kFull, myrow, k + 1) * Rp + tile0 * 32 + lane;
        float va[kStatTiles], vb[kStatTiles];
#pragma unroll
        for (int tt = 0; tt < kStatTiles; ++tt) {
          va[tt] = tt < nt ? ra[tt * 32] : 0.f;
          vb[tt] = tt < nt ? rb[tt * 32] : 0.f;
        }
#pragma unroll
        for (int tt = 0; tt < kStatTiles; ++tt) q[tt] = fmaf(vb[tt], vb[tt], fmaf(va[tt], va[tt], q[tt]));
      }
      if (k < nk) {
        const float* ra = P + (size_t)__shfl_sync(kFull, myrow, k) * Rp + tile0 * 32 + lane;
#pragma unroll
        for (int tt = 0; tt < kStatTiles; ++tt)
          if (tt < nt) q[tt] = fmaf(ra[tt * 32], ra[tt * 32], q[tt]);
      }
    }
    // true-literal counts: lane k fetches literal k's bitset words, a 32x32
    // bit transpose gives each lane (restart) its literals' bits
    int t[kStatTiles];
#pragma unroll
    for (int tt = 0; tt < kStatTiles; ++tt) t[tt] = 0;
    for (int k0 = 0; k0 < s.L; k0 += 32) {
      uint32_t word[kStatTiles];
      const bool mine = k0 + lane < s.L;
      LitRec rc{0, 0};
      if (mine) rc = lit[s.lit0 + k0 + lane];
#pragma unroll
      for (int tt = 0; tt < kStatTiles; ++tt) {
        word[tt] = 0;
        if (mine && tt < nt) {
          word[tt] = bits[(size_t)rc.var * RW + tile0 + tt];
          if (rc.dst < 0) word[tt] = ~word[tt];
        }
      }
#pragma unroll
      for (int tt = 0; tt < kStatTiles; ++tt) t[tt] += __popc(transpose32(word[tt], lane));
    }
    const float inv_w = it.w != 0.f ? 1.0f / fabsf(it.w) : 0.f;
#pragma unroll
    for (int tt = 0; tt < kStatTiles; ++tt) {
      if (tt >= nt) break;
      const int r = (tile0 + tt) * 32 + lane;
      const bool act = r < R;
      float g = act ? sqrtf(q[tt]) * inv_w : 0.f;
      const unsigned viol = __ballot_sync(kFull, act && !sat_of(s, t[tt], satbits));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(kFull, g, o);
      if (lane == 0) {
        tg[(size_t)c * RW + tile0 + tt] = g;
        tu[(size_t)c * RW + tile0 + tt] = __popc(viol);
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_con_stats_reduce(int m, int RW,
                                                          const float* __restrict__ tg,
                                                          const int32_t* __restrict__ tu,
                                                          double* __restrict__ gnorm,
                                                          int32_t* __restrict__ unsat) {
  const int c = blockIdx.x * kStatWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= m) return;
  double a = 0.0;
  int u = 0;
  for (int j = lane; j < RW; j += 32) {
    a += (double)tg[(size_t)c * RW + j];
    u += tu[(size_t)c * RW + j];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(kFull, a, o);
    u += __shfl_xor_sync(kFull, u, o);
  }
  if (lane == 0) {
    gnorm[c] = a;
    unsat[c] = u;
  }
}

// mean per-restart gradient norm over the constraints with FE work:
// gbar = (sum_{c: L_fe > 0} gnorm[c] / R) / #{c: L_fe > 0}; one block, fixed order
__global__ void __launch_bounds__(1024) k_rw_mean(int m, int R, const FeItem* __restrict__ fe,
                                                  const double* __restrict__ gnorm,
                                                  double* __restrict__ gbar) {
  __shared__ double sa[1024];
  __shared__ int sn[1024];
  double a = 0.0;
  int n = 0;
  for (int c = threadIdx.x; c < m; c += 1024) {
    if (fe[c].L > 0) {
      a += gnorm[c] / (double)R;
      ++n;
    }
  }
  sa[threadIdx.x] = a;
  sn[threadIdx.x] = n;
  __syncthreads();
  for (int h = 512; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      sa[threadIdx.x] += sa[threadIdx.x + h];
      sn[threadIdx.x] += sn[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *gbar = sn[0] > 0 ? sa[0] / (double)sn[0] : 0.0;
}

// w'_c = min(w_max, w_c (1 + eta u_c rho_c)), u_c = unsat[c] / R,
// rho_c = kappa if g_c kappa <= gbar else gbar / g_c, g_c = gnorm[c] / R (FP64)
__global__ void __launch_bounds__(256) k_rw_update(int m, int R, const FeItem* __restrict__ fe,
                                                   const double* __restrict__ gnorm,
                                                   const int32_t* __restrict__ unsat,
                                                   const double* __restrict__ gbar, double eta,
                                                   double kappa, double w_max,
                                                   float* __restrict__ w_out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m) return;
  const double gb = *gbar;
  const double u = (double)unsat[c] / (double)R;
  const double g = gnorm[c] / (double)R;
  const double rho = g * kappa <= gb ? kappa : gb / g;
  const double w = (double)fe[c].w * (1.0 + eta * u * rho);
  w_out[c] = (float)fmin(w_max, w);
}

// new weights into every device copy the kernels read: the FE items in
// constraint order, the score items, and the short closed-form classes'
// items (in launch order, located by their constraint index)
__global__ void __launch_bounds__(256) k_set_weights(int m, const float* __restrict__ w,
                                                     FeItem* __restrict__ fe,
                                                     ScoreItem* __restrict__ sc, FeItem* t0,
                                                     int n0, FeItem* t1, int n1, FeItem* t2,
                                                     int n2) {
  const int total = m + n0 + n1 + n2;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    if (i < m) {
      fe[i].w = w[i];
      sc[i].w = w[i];
    } else if (i < m + n0) {
      t0[i - m].w = w[t0[i - m].c];
    } else if (i < m + n0 + n1) {
      t1[i - m - n0].w = w[t1[i - m - n0].c];
    } else {
      t2[i - m - n0 - n1].w = w[t2[i - m - n0 - n1].c];
    }
  }
}

// score_range for NT consecutive restart tiles at once (the k_score path):
// one literal-record load, one constraint walk and one mask per chunk serve
// every tile; each tile has its own bitset words, transpose and counts
template <bool UNIT, int NT>
__device__ __forceinline__ void score_range_tiles(int rg, int tile0, int lane, int RW,
                                                  const int32_t* __restrict__ ranges,
                                                  const ScoreItem* __restrict__ sc,
                                                  const LitRec* __restrict__ lit,
                                                  const uint32_t* __restrict__ satbits,
                                                  const uint32_t* __restrict__ bits,
                                                  int (&cnt)[NT], double (&ws)[NT]) {
  int run[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    cnt[t] = 0;
    ws[t] = 0.0;
    run[t] = 0;
  }
  int c = ranges[rg];
  const int c_end = ranges[rg + 1];
  ScoreItem s = sc[c];
  int e = s.lit0;
  const ScoreItem last = sc[c_end - 1];
  const int e_end = last.lit0 + last.L;
  while (e < e_end) {
    uint32_t col[NT];
    {
      uint32_t word[NT];
      LitRec rc{0, 0};
      const bool has = e + lane < e_end;
      if (has) rc = lit[e + lane];
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        word[t] = 0;
        if (has && tile0 + t < RW) {
          word[t] = bits[(size_t)rc.var * RW + tile0 + t];
          if (rc.dst < 0) word[t] = ~word[t];
        }
      }
#pragma unroll
      for (int t = 0; t < NT; ++t) col[t] = transpose32(word[t], lane);
    }
    const int chunk_end = e + 32;
    while (c < c_end && s.lit0 + s.L <= chunk_end) {
      const int lo = max(s.lit0, e) - e;
      const int hi = s.lit0 + s.L - e;
      const uint32_t mask = (hi >= 32 ? kFull : ((1u << hi) - 1u)) & (kFull << lo);
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const bool sat = sat_of(s, run[t] + __popc(col[t] & mask), satbits);
        run[t] = 0;
        cnt[t] += sat ? 1 : 0;
        if constexpr (!UNIT) ws[t] += sat ? (double)s.w : 0.0;
      }
      ++c;
      if (c < c_end) s = sc[c];
    }
    if (c < c_end && s.lit0 < chunk_end) {
      const int lo = max(s.lit0, e) - e;
#pragma unroll
      for (int t = 0; t < NT; ++t) run[t] += __popc(col[t] & (kFull << lo));
    }
    e = chunk_end;
  }
  if constexpr (UNIT) {
#pragma unroll
    for (int t = 0; t < NT; ++t) ws[t] = (double)cnt[t];
  }
}

// restart tiles per warp of k_score
constexpr int kScoreTiles = 4;

template <bool UNIT>
__global__ void __launch_bounds__(256) k_score(int RW, int Rp, int n_ranges,
                                               const int32_t* __restrict__ ranges,
                                               const ScoreItem* __restrict__ sc,
                                               const LitRec* __restrict__ lit,
                                               const uint32_t* __restrict__ satbits,
                                               const uint32_t* __restrict__ bits,
                                               int32_t* __restrict__ nsat_part,
                                               double* __restrict__ wsat_part) {
  __shared__ int32_t cnt_s[kScoreTiles][kScoreWarps][32];
  __shared__ double w_s[UNIT ? 1 : kScoreTiles][kScoreWarps][32];
  const int lane = threadIdx.x, ty = threadIdx.y;
  const int tile0 = blockIdx.x * kScoreTiles;
  const int rg = blockIdx.y * kScoreWarps + ty;
  int cnt[kScoreTiles];
  double ws[kScoreTiles];
#pragma unroll
  for (int t = 0; t < kScoreTiles; ++t) {
    cnt[t] = 0;
    ws[t] = 0.0;
  }
  if (rg < n_ranges)
    score_range_tiles<UNIT, kScoreTiles>(rg, tile0, lane, RW, ranges, sc, lit, satbits, bits,
                                         cnt, ws);
#pragma unroll
  for (int t = 0; t < kScoreTiles; ++t) {
    cnt_s[t][ty][lane] = cnt[t];
    if constexpr (!UNIT) w_s[t][ty][lane] = ws[t];
  }
  __syncthreads();
  // warp t < kScoreTiles adds tile t's counts over the block's warps
  if (ty < kScoreTiles && tile0 + ty < RW) {
    int a = 0;
    double b = 0.0;
#pragma unroll
    for (int k = 0; k < kScoreWarps; ++k) {
      a += cnt_s[ty][k][lane];
      if constexpr (!UNIT) b += w_s[ty][k][lane];
    }
    const int r = (tile0 + ty) * 32 + lane;
    nsat_part[(size_t)blockIdx.y * Rp + r] = a;
    if constexpr (!UNIT) wsat_part[(size_t)blockIdx.y * Rp + r] = b;   // UNIT: wsat = nsat
  }
}

// all weights 1: wsat = nsat, an integer sum in any order; 8 threads per
// restart take every 8th chunk and add their sums in a fixed order
__global__ void __launch_bounds__(256) k_score_final_unit(int R, int Rp, int nch,
                                                          const int32_t* __restrict__ nsat_part,
                                                          int32_t* __restrict__ nsat,
                                                          double* __restrict__ wsat) {
  __shared__ int32_t part_s[8][32];
  const int r = blockIdx.x * 32 + threadIdx.x;
  int a = 0;
  if (r < R)
    for (int ch = threadIdx.y; ch < nch; ch += 8) a += nsat_part[(size_t)ch * Rp + r];
  part_s[threadIdx.y][threadIdx.x] = a;
  __syncthreads();
  if (threadIdx.y == 0 && r < R) {
    int t = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += part_s[k][threadIdx.x];
    if (nsat) nsat[r] = t;
    if (wsat) wsat[r] = (double)t;
  }
}

__global__ void k_score_final(int R, int Rp, int nch, const int32_t* __restrict__ nsat_part,
                              const double* __restrict__ wsat_part, int32_t* __restrict__ nsat,
                              double* __restrict__ wsat) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  int a = 0;
  double b = 0.0;
  for (int ch = 0; ch < nch; ++ch) {
    a += nsat_part[(size_t)ch * Rp + r];
    b += wsat_part[(size_t)ch * Rp + r];
  }
  if (nsat) nsat[r] = a;
  if (wsat) wsat[r] = b;
}

// obj[r] = sum_c w_c FE_c, FP64 in constraint order within a chunk, chunks in order
__global__ void __launch_bounds__(256) k_obj_part(int m, int R, int Rp, int chunk,
                                                  const ScoreItem* __restrict__ sc,
                                                  const float* __restrict__ fe_con, int ldf,
                                                  double* __restrict__ part) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const int c0 = blockIdx.y * chunk;
  const int c1 = min(m, c0 + chunk);
  double a = 0.0;
  for (int c = c0; c < c1; ++c) a += (double)sc[c].w * (double)fe_con[(size_t)c * ldf + r];
  part[(size_t)blockIdx.y * Rp + r] = a;
}

__global__ void k_obj_final(int R, int Rp, int nch, const double* __restrict__ part,
                            float* __restrict__ obj) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  double a = 0.0;
  for (int ch = 0; ch < nch; ++ch) a += part[(size_t)ch * Rp + r];
  obj[r] = (float)a;
}

// constant expansions (no literals enter FE): fe_con[c, r] = b0
__global__ void __launch_bounds__(256) k_fe_const(const int32_t* __restrict__ list, int count,
                                                  const FeItem* __restrict__ fe, int R,
                                                  float* __restrict__ fe_con, int ldf) {
  const int64_t total = (int64_t)count * R;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const FeItem it = fe[list[i / R]];
    fe_con[(size_t)it.c * ldf + (i % R)] = it.b0;
  }
}

// vector-Jacobian product of the per-restart objective: out[v,r] = s[r] g[v,r]
__global__ void __launch_bounds__(256) k_restart_scale(int64_t total, int R,
                                                       const float* __restrict__ g,
                                                       const float* __restrict__ sc,
                                                       float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = sc[i % R] * g[i];
}

// ---------------------------------------------------------------------------
// A10 as one persistent launch (problems whose FE work is all on the short
// closed-form path, e.g. random k-SAT): a cooperative kernel runs the whole
// step loop, its warps taking work items of each stage in turn, with a grid
// barrier between stages.  The barrier spins at most ~2^22 polls; on time-out
// it raises *err and every block returns (no hang).
// ---------------------------------------------------------------------------
struct PersistArgs {
  int R, Rp, RT, n_steps;
  float lr;
  float* x;
  float* P;
  uint32_t* bits;
  int32_t* rpart_n;     // [range][Rp]
  double* rpart_w;
  int32_t* nsat;
  double* wsat;
  unsigned* bar;        // [0] arrivals, [1] generation
  int* err;
  unsigned spin_limit;  // polls before a barrier gives up
};

constexpr unsigned kBarrierSpinLimit = 1u << 22;

// Grid barrier for a cooperative launch: arrival counter + generation word.
// Thread (0,0) of each block arrives and polls the generation with
// __nanosleep between polls; after spin_limit polls (or when another block
// already gave up) it raises *err and the call returns false; the caller then
// returns from the kernel.  nblocks is the number of arrivals that releases
// the barrier (gridDim.x in normal use).
__device__ __forceinline__ bool grid_sync(unsigned* bar, int* err, unsigned nblocks,
                                          unsigned spin_limit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    ok = 1;
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned spins = 0;
      while (*gen == g) {
        if (++spins > spin_limit || *((volatile int*)err)) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*((volatile int*)err)) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

__global__ void __launch_bounds__(256) k_persistent(DevPlan d, PersistArgs a) {
  const int lane = threadIdx.x;
  const int gw = blockIdx.x * blockDim.y + threadIdx.y;
  const int nw = gridDim.x * blockDim.y;
  const int tgroups = (a.RT + kThreadTiles - 1) / kThreadTiles;
  const int n0 = d.thread_count[0], n1 = d.thread_count[1];
  __shared__ int2 trec_s[8][16];
  int2* trec = trec_s[threadIdx.y];
  for (int step = 0; step < a.n_steps; ++step) {
    // FE + literal partials (short closed forms): items (constraint, 4 tiles)
    const int fe_items = (n0 + n1) * tgroups;
    for (int item = gw; item < fe_items; item += nw) {
      const int ci = item / tgroups, tg = item % tgroups;
      const bool c0 = ci < n0;
      const FeItem it = c0 ? d.thread_items[0][ci] : d.thread_items[1][ci - n0];
      __syncwarp();
      load_trec(it, d.fe_lit, trec, lane);
      if (c0)
        thread_dispatch<1, 8, true>(it.L, it, d.root_tab, d.coef_tab, trec, a.x, a.R, a.Rp, a.RT,
                                    tg * kThreadTiles, lane, a.P, nullptr, 0);
      else
        thread_dispatch<9, 16, true>(it.L, it, d.root_tab, d.coef_tab, trec, a.x, a.R, a.Rp, a.RT,
                                     tg * kThreadTiles, lane, a.P, nullptr, 0);
    }
    if (!grid_sync(a.bar, a.err, gridDim.x, a.spin_limit)) return;
    // accumulate + projected step + rounding: items (variable, tile)
    const int acc_items = d.n * a.RT;
    for (int item = gw; item < acc_items; item += nw)
      accum_one<true>(item / a.RT, item % a.RT, lane, a.R, a.Rp, a.RT, d.fe_voff, a.P, a.x, a.lr, 1,
                d.fixed, nullptr, a.bits);
    if (!grid_sync(a.bar, a.err, gridDim.x, a.spin_limit)) return;
    // score: items (range, tile) -> per-range partials
    const int sc_items = d.n_ranges * a.RT;
    for (int item = gw; item < sc_items; item += nw) {
      const int rg = item / a.RT, tile = item % a.RT;
      int cnt;
      double ws;
      score_range<true>(rg, tile, lane, a.RT, d.score_ranges, d.score, d.lit, d.satbits, a.bits, &cnt,
                  &ws);
      a.rpart_n[(size_t)rg * a.Rp + tile * 32 + lane] = cnt;
      a.rpart_w[(size_t)rg * a.Rp + tile * 32 + lane] = ws;
    }
    if (!grid_sync(a.bar, a.err, gridDim.x, a.spin_limit)) return;
    // totals per restart, summed in the same order as k_score + k_score_final
    // (groups of kScoreWarps ranges, then over groups), so both paths agree
    // bit for bit
    for (int r = blockIdx.x * blockDim.x * blockDim.y + threadIdx.y * blockDim.x + lane; r < a.R;
         r += gridDim.x * blockDim.x * blockDim.y) {
      int cnt = 0;
      double ws = 0.0;
      for (int rg0 = 0; rg0 < d.n_ranges; rg0 += kScoreWarps) {
        int bc = 0;
        double bw = 0.0;
        for (int rg = rg0; rg < min(rg0 + kScoreWarps, d.n_ranges); ++rg) {
          bc += __ldcg(&a.rpart_n[(size_t)rg * a.Rp + r]);
          bw += __ldcg(&a.rpart_w[(size_t)rg * a.Rp + r]);
        }
        cnt += bc;
        ws += bw;
      }
      if (a.nsat) a.nsat[r] = cnt;
      if (a.wsat) a.wsat[r] = ws;
    }
  }
}

// ---------------------------------------------------------------------------
// The step loop with one CTA per tile of 32 restarts (A10; the restarts of
// the lockstep batch are independent, Sec. 3.3).  The CTA keeps its tile of
// x, every literal partial row of the tile and the tile's bitset in shared
// memory for the whole n-step loop, with __syncthreads between the phases:
// no grid barrier, one launch.  For problems whose FE work is all short
// closed forms (L <= 16) and whose tile fits in shared memory.  Per step:
// the literal partials of every constraint (the same FP32 operations as
// thread_body), then per variable the rows summed in row order, the
// projected step and the ballot (as accum_one); after the last step the
// bitset and x go back to global memory and the score is taken there (the
// ranges as score_range, the totals in k_score_final's order), so x, the
// bitset and the counts equal cls_step's bit for bit.
// Shared memory: see tile_smem_layout.
// ---------------------------------------------------------------------------
struct TileArgs {
  int R, Rp, RT, n_steps;
  float lr;
  float* x;
  uint32_t* bits;
  int32_t* rpart_n;     // [range][Rp]
  double* rpart_w;
  int32_t* nsat;
  double* wsat;
};

constexpr int kTileWarps = 32;          // warps of a k_tile_loop CTA
constexpr int kTileRoots = 3;           // the real-root table entries (plan.h)
constexpr int kTileCoefs = 7;           // the closed-form coefficient entries

template <int L>
__device__ __forceinline__ void tile_fe_body(const FeItem& it, const float4* rt, const float4* cf,
                                             const int2* rec, const float* xs, float* ps,
                                             int lane) {
  const float4 rt0 = rt[it.root_off], cf0 = cf[it.coef_off];
  const bool two = it.J == 2;
  const float4 rt1 = two ? rt[it.root_off + 1] : make_float4(1.f, 0.f, 0.f, 0.f);
  const float4 cf1 = two ? cf[it.coef_off + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
  float y[L], g[L], pre[L];
#pragma unroll
  for (int i = 0; i < L; ++i) y[i] = rec_sgn(rec[i].y) * xs[rec[i].x * 32 + lane];
  float run = 1.f;
#pragma unroll
  for (int i = 0; i < L; ++i) {
    pre[i] = run;
    run *= fmaf(y[i], rt0.y, rt0.x);
  }
  float suf = cf0.z;
#pragma unroll
  for (int i = L - 1; i >= 0; --i) {
    g[i] = pre[i] * suf;
    suf *= fmaf(y[i], rt0.y, rt0.x);
  }
  if (two) {
    run = 1.f;
#pragma unroll
    for (int i = 0; i < L; ++i) {
      pre[i] = run;
      run *= fmaf(y[i], rt1.y, rt1.x);
    }
    suf = cf1.z;
#pragma unroll
    for (int i = L - 1; i >= 0; --i) {
      g[i] = fmaf(pre[i], suf, g[i]);
      suf *= fmaf(y[i], rt1.y, rt1.x);
    }
  }
#pragma unroll
  for (int i = 0; i < L; ++i)
    ps[rec_row(rec[i].y) * 32 + lane] = it.w * rec_sgn(rec[i].y) * g[i];
}

template <int LO, int HI>
__device__ __forceinline__ void tile_fe_dispatch(int L, const FeItem& it, const float4* rt,
                                                 const float4* cf, const int2* rec,
                                                 const float* xs, float* ps, int lane) {
  if constexpr (LO <= HI) {
    if (L == LO)
      tile_fe_body<LO>(it, rt, cf, rec, xs, ps, lane);
    else
      tile_fe_dispatch<LO + 1, HI>(L, it, rt, cf, rec, xs, ps, lane);
  }
}

// Shared memory of k_tile_loop (16-byte entries first): the real-root and
// coefficient tables, the items, then x [n][32], the partial rows
// [nnz_fe][32], the literal records, the row offsets and the bitset.
struct TileSmem {
  size_t items, xs, ps, recs, voff, bs, total;
};

__host__ __device__ inline TileSmem tile_smem_layout(int n, int64_t nnz_fe, int n_items) {
  TileSmem t;
  size_t off = (size_t)(kTileRoots + kTileCoefs) * 16;
  t.items = off;
  off += (size_t)n_items * sizeof(FeItem);
  t.xs = off;
  off += (size_t)n * 32 * sizeof(float);
  t.ps = off;
  off += (size_t)nnz_fe * 32 * sizeof(float);
  t.recs = off;
  off += (size_t)nnz_fe * sizeof(int2);
  t.voff = off;
  off += (size_t)(n + 1) * sizeof(int32_t);
  t.bs = off;
  off += (size_t)n * sizeof(uint32_t);
  t.total = off;
  return t;
}

__global__ void __launch_bounds__(32 * kTileWarps) k_tile_loop(DevPlan d, TileArgs a) {
  extern __shared__ float4 tl_smem4[];
  char* base = reinterpret_cast<char*>(tl_smem4);
  const int n = d.n, n0 = d.thread_count[0], n1 = d.thread_count[1];
  const TileSmem lay = tile_smem_layout(n, d.nnz_fe, n0 + n1);
  float4* rt = tl_smem4;                                    // [kTileRoots]
  float4* cf = tl_smem4 + kTileRoots;                       // [kTileCoefs]
  FeItem* items = reinterpret_cast<FeItem*>(base + lay.items);
  float* xs = reinterpret_cast<float*>(base + lay.xs);
  float* ps = reinterpret_cast<float*>(base + lay.ps);
  int2* recs = reinterpret_cast<int2*>(base + lay.recs);
  int32_t* voff = reinterpret_cast<int32_t*>(base + lay.voff);
  uint32_t* bs = reinterpret_cast<uint32_t*>(base + lay.bs);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tile = blockIdx.x;
  const int r = tile * 32 + lane;
  const bool act = r < a.R;
  // the problem's short-class data, read once for the whole loop
  for (int i = threadIdx.x; i < kTileRoots; i += blockDim.x) rt[i] = ldg4(&d.root_tab[i]);
  for (int i = threadIdx.x; i < kTileCoefs; i += blockDim.x) cf[i] = ldg4(&d.coef_tab[i]);
  for (int i = threadIdx.x; i < n0 + n1; i += blockDim.x)
    items[i] = i < n0 ? d.thread_items[0][i] : d.thread_items[1][i - n0];
  for (int64_t e = threadIdx.x; e < d.nnz_fe; e += blockDim.x)
    recs[e] = make_int2(d.fe_lit[e].var, d.fe_lit[e].dst);
  for (int v = threadIdx.x; v <= n; v += blockDim.x) voff[v] = d.fe_voff[v];
  for (int v = warp; v < n; v += kTileWarps)
    xs[v * 32 + lane] = act ? a.x[(size_t)v * a.R + r] : 0.f;
  for (int step = 0; step < a.n_steps; ++step) {
    __syncthreads();                                    // x of the previous step in place
    for (int ci = warp; ci < n0 + n1; ci += kTileWarps) {
      const FeItem it = items[ci];
      if (it.L <= 8)
        tile_fe_dispatch<1, 8>(it.L, it, rt, cf, recs + it.lit0, xs, ps, lane);
      else
        tile_fe_dispatch<9, 16>(it.L, it, rt, cf, recs + it.lit0, xs, ps, lane);
    }
    __syncthreads();                                    // every partial row written
    for (int v = warp; v < n; v += kTileWarps) {
      float g = 0.f;
      for (int k = voff[v]; k < voff[v + 1]; ++k) g += ps[k * 32 + lane];
      float xv = xs[v * 32 + lane];
      if (act && !(d.fixed && d.fixed[v])) {
        xv = pgd_project(xv, g, a.lr);
        xs[v * 32 + lane] = xv;
      }
      const uint32_t b = __ballot_sync(kFull, act && xv < 0.0f);
      if (lane == 0) bs[v] = b;
    }
  }
  __syncthreads();
  for (int v = warp; v < n; v += kTileWarps) {
    if (act) a.x[(size_t)v * a.R + r] = xs[v * 32 + lane];
    if (lane == 0) a.bits[(size_t)v * a.RT + tile] = bs[v];
  }
  __syncthreads();                                      // the tile's bitset in global memory
  // score of the final bitset: ranges over the warps, then the totals per
  // restart in the order of k_score + k_score_final
  for (int rg = warp; rg < d.n_ranges; rg += kTileWarps) {
    int cnt;
    double ws;
    score_range<true>(rg, tile, lane, a.RT, d.score_ranges, d.score, d.lit, d.satbits, a.bits,
                      &cnt, &ws);
    a.rpart_n[(size_t)rg * a.Rp + tile * 32 + lane] = cnt;
    a.rpart_w[(size_t)rg * a.Rp + tile * 32 + lane] = ws;
  }
  __syncthreads();
  if (warp == 0 && act) {
    int cnt = 0;
    double ws = 0.0;
    for (int rg0 = 0; rg0 < d.n_ranges; rg0 += kScoreWarps) {
      int bc = 0;
      double bw = 0.0;
      for (int rg = rg0; rg < min(rg0 + kScoreWarps, d.n_ranges); ++rg) {
        bc += __ldcg(&a.rpart_n[(size_t)rg * a.Rp + r]);
        bw += __ldcg(&a.rpart_w[(size_t)rg * a.Rp + r]);
      }
      cnt += bc;
      ws += bw;
    }
    if (a.nsat) a.nsat[r] = cnt;
    if (a.wsat) a.wsat[r] = ws;
  }
}

size_t tile_loop_smem(const DevPlan& d) {
  return tile_smem_layout(d.n, d.nnz_fe, d.thread_count[0] + d.thread_count[1]).total;
}

// Barrier check: `rounds` grid barriers that release after gridDim.x + extra
// arrivals; with extra > 0 none can release, so every block must time out,
// raise *err and return.  Block 0 records how many barriers it passed.
__global__ void __launch_bounds__(32) k_barrier_check(unsigned* bar, int* err, int rounds,
                                                      unsigned extra, unsigned spin_limit,
                                                      int* passed) {
  int k = 0;
  for (; k < rounds; ++k)
    if (!grid_sync(bar, err, gridDim.x + extra, spin_limit)) break;
  if (blockIdx.x == 0 && threadIdx.x == 0) *passed = k;
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

struct HookScope {
  LaunchHook* h;
  int kc;
  cudaStream_t s;
  HookScope(LaunchHook* h_, int kc_, cudaStream_t s_) : h(h_), kc(kc_), s(s_) {
    if (h) h->before(kc, s);
  }
  ~HookScope() {
    if (h) h->after(kc, s);
  }
};

// records (16 B, plus 4 B for a second root, per literal slot) + checkpoints
// (8 warps x NJ x nck x 32 floats)
inline size_t ckpt_smem(int maxL, int nj, int ci) {
  const int nck = std::max(1, (maxL + ci - 1) / ci);
  return (size_t)nck * ci * (nj > 1 ? 20 : 16) + (size_t)8 * nj * nck * 32 * sizeof(float);
}
// constraints up to this length use checkpoints every 8 literals (fewer
// registers); longer ones every kCkptInterval (less shared memory)
constexpr int kCkptShortMax = 512;

template <int G, int Q>
constexpr size_t group_smem() {
  return (size_t)G * Q * GroupGeom<G>::LDR * sizeof(float);
}

}  // namespace

size_t group_smem_bytes(int cfg) {
  if (cfg >= 0 && cfg < kNumGroupCfg && kGroupCfg[cfg].cplx == 3) return fr_smem_bytes(cfg);
  if (cfg >= 0 && cfg < kNumGroupCfg && kGroupCfg[cfg].cplx == 2)
    return (size_t)kGroupCfg[cfg].G * kGroupCfg[cfg].Q * (32 + 32 / kGroupCfg[cfg].G) *
           sizeof(float);
  switch (cfg) {
#define CLS_SMEM_CASE(id, G, Q, C, Y) \
  case id: return group_smem<G, Q>();
    CLS_GROUP_CONFIGS(CLS_SMEM_CASE)
#undef CLS_SMEM_CASE
    default: return 0;
  }
}

cudaError_t set_kernel_attributes() {
  cudaError_t err = cudaSuccess;
#define CLS_SET_ATTR(id, G, Q, C, Y)                                                     \
  if (err == cudaSuccess)                                                                \
    err = cudaFuncSetAttribute(k_fe_group<G, Q, (C != 0), (Y != 0)>,                     \
                               cudaFuncAttributeMaxDynamicSharedMemorySize,              \
                               (int)group_smem<G, Q>());
  CLS_GROUP_CONFIGS(CLS_SET_ATTR)
#undef CLS_SET_ATTR
  if (err == cudaSuccess) err = set_p2_attributes();
  if (err == cudaSuccess) err = set_fr_attributes();
  if (err == cudaSuccess) err = set_corner_attributes();
  if (err == cudaSuccess) err = set_series_attributes();
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute(k_fe_thread<1, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)thread_xbuf_bytes<8>());
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute(k_fe_thread<9, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)thread_xbuf_bytes<16>());
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute(k_fe_thread<17, 24>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)thread_xbuf_bytes<24>());
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute(k_tile_loop, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kTileLoopMaxSmem);
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute(k_fe_thread_ckpt<1, 16>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)ckpt_smem(1024, 1, 16));
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute(k_fe_thread_ckpt<2, 16>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)ckpt_smem(1024, 2, 16));
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute(k_fe_thread_ckpt<1, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)ckpt_smem(kCkptShortMax, 1, 8));
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute(k_fe_thread_ckpt<2, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)ckpt_smem(kCkptShortMax, 2, 8));
  return err;
}

cudaError_t launch_init(const DevPlan& d, int R, uint64_t seed, int64_t r_off, float* x,
                        cudaStream_t s, LaunchHook* h) {
  if (d.n == 0 || R == 0) return cudaSuccess;
  const int64_t total = (int64_t)((d.n + 3) / 4) * R;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 148 * 16);
  HookScope hs(h, KC_INIT, s);
  k_init_uniform<<<blocks, 256, 0, s>>>(d.n, R, seed, r_off, d.fixed, d.fixed_val, x);
  return cudaGetLastError();
}

cudaError_t launch_track_reset(int R, int32_t* trk, cudaStream_t s) {
  if (R == 0) return cudaSuccess;
  k_track_reset<<<(R + 255) / 256, 256, 0, s>>>(R, trk);
  return cudaGetLastError();
}

cudaError_t launch_track_step(const DevPlan& d, int R, int step, const int32_t* nsat,
                              int32_t* trk, cudaStream_t s) {
  if (R == 0) return cudaSuccess;
  k_track_step<<<(R + 255) / 256, 256, 0, s>>>(R, d.m, step, nsat, trk);
  return cudaGetLastError();
}

cudaError_t launch_refill(const DevPlan& d, int R, uint64_t seed, int64_t r_off, uint64_t gen,
                          int patience, int32_t* trk, float* x, int32_t* count, cudaStream_t s) {
  if (R == 0) return cudaSuccess;
  if (d.n > 0) {
    const int64_t total = (int64_t)((d.n + 3) / 4) * R;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 148 * 16);
    k_refill<<<blocks, 256, 0, s>>>(d.n, R, seed, r_off, gen, patience, d.fixed, trk, x);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_refill_reset<<<(R + 255) / 256, 256, 0, s>>>(R, patience, trk, count);
  return cudaGetLastError();
}

cudaError_t launch_unsat_hist(const DevPlan& d, int R, const int32_t* nsat, int32_t* hist,
                              cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int32_t) * ((size_t)d.m + 1), s);
  if (e != cudaSuccess || R == 0) return e;
  k_unsat_hist<<<(R + 255) / 256, 256, 0, s>>>(R, d.m, nsat, hist);
  return cudaGetLastError();
}

cudaError_t launch_movement(const DevPlan& d, int R, const float* xp, const float* x,
                            float* maxdelta, cudaStream_t s) {
  if (R == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(maxdelta, 0, sizeof(float) * (size_t)R, s);
  if (e != cudaSuccess || d.n == 0) return e;
  const int chunks = ceil_div(d.n, kMoveVars);
  const dim3 grid(ceil_div(R, 32), std::min(ceil_div(chunks, 8), 65535));
  k_move_max<<<grid, 256, 0, s>>>(d.n, R, xp, x, reinterpret_cast<unsigned*>(maxdelta));
  return cudaGetLastError();
}

cudaError_t launch_track_conv(int R, const float* maxdelta, float tol, int step, int32_t* conv,
                              cudaStream_t s) {
  if (R == 0) return cudaSuccess;
  k_track_conv<<<(R + 255) / 256, 256, 0, s>>>(R, maxdelta, tol, step, conv);
  return cudaGetLastError();
}

cudaError_t launch_con_stats(const DevPlan& d, int R, int Rp, const uint32_t* bits,
                             const float* P, float* scratch, double* gnorm, int32_t* unsat,
                             cudaStream_t s) {
  if (d.m == 0) return cudaSuccess;
  const int RW = (R + 31) / 32;
  const int64_t pairs = (int64_t)d.m * RW;
  float* tg = scratch;
  int32_t* tu = reinterpret_cast<int32_t*>(scratch + pairs);
  const int64_t items = (int64_t)d.m * ((RW + kStatTiles - 1) / kStatTiles);
  const int blocks = (int)std::min<int64_t>((items + kStatWarps - 1) / kStatWarps, 148 * 8);
  k_con_stats_tile<<<blocks, 32 * kStatWarps, 0, s>>>(d.m, RW, R, Rp, d.fe, d.score, d.fe_lit,
                                                      d.lit, d.satbits, bits, P, d.stat_order,
                                                      tg, tu);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_con_stats_reduce<<<(d.m + kStatWarps - 1) / kStatWarps, 32 * kStatWarps, 0, s>>>(
      d.m, RW, tg, tu, gnorm, unsat);
  return cudaGetLastError();
}

cudaError_t launch_set_weights(const DevPlan& d, const float* w, cudaStream_t s) {
  const int total = d.m + d.thread_count[0] + d.thread_count[1] + d.thread_count[2];
  if (total == 0) return cudaSuccess;
  const int blocks = std::min((total + 255) / 256, 148 * 8);
  k_set_weights<<<blocks, 256, 0, s>>>(d.m, w, d.fe, d.score, d.thread_items[0],
                                       d.thread_count[0], d.thread_items[1], d.thread_count[1],
                                       d.thread_items[2], d.thread_count[2]);
  return cudaGetLastError();
}

cudaError_t launch_reweight(const DevPlan& d, int R, const double* gnorm, const int32_t* unsat,
                            double eta, double kappa, double w_max, float* w_out, double* gbar,
                            cudaStream_t s) {
  if (d.m == 0) return cudaSuccess;
  k_rw_mean<<<1, 1024, 0, s>>>(d.m, R, d.fe, gnorm, gbar);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_rw_update<<<(d.m + 255) / 256, 256, 0, s>>>(d.m, R, d.fe, gnorm, unsat, gbar, eta, kappa,
                                                w_max, w_out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_set_weights(d, w_out, s);
}

cudaError_t launch_group(int cfg, const DevPlan& d, const int32_t* list, int count, int maxL, int maxJ,
                         int R, int Rp, const float* x, float* P, float* fe_con, int ldf,
                         uint8_t* done, cudaStream_t s) {
  if (count == 0 || R == 0) return cudaSuccess;
  if (cfg == kCkptCfg) {
    const int RT = ceil_div(R, 32);
    const int ci = maxL <= kCkptShortMax ? 8 : kCkptInterval;
    const int nck = std::max(1, ceil_div(maxL, ci));
    const dim3 g2(count, ceil_div(RT, 8)), b2(32, 8);
    const size_t sm = ckpt_smem(maxL, maxJ <= 1 ? 1 : 2, ci);
#define CLS_CKPT_LAUNCH(NJ, CI)                                                                 \
  k_fe_thread_ckpt<NJ, CI><<<g2, b2, sm, s>>>(list, d.fe, d.root_tab, d.coef_tab, d.fe_lit, x, \
                                              R, Rp, RT, nck, P, fe_con, ldf)
    if (maxJ <= 1) {
      if (ci == 8) CLS_CKPT_LAUNCH(1, 8);
      else CLS_CKPT_LAUNCH(1, kCkptInterval);
    } else {
      if (ci == 8) CLS_CKPT_LAUNCH(2, 8);
      else CLS_CKPT_LAUNCH(2, kCkptInterval);
    }
#undef CLS_CKPT_LAUNCH
    return cudaGetLastError();
  }
  if (cfg >= 0 && cfg < kNumGroupCfg && kGroupCfg[cfg].cplx == 2)
    return launch_group_p2(cfg, d, list, count, R, Rp, x, P, fe_con, ldf, s);
  if (cfg >= 0 && cfg < kNumGroupCfg && kGroupCfg[cfg].cplx == 3)
  {
    // factored configurations of kCornerMinSlots slots or more: the corner
    // passes first (they flag the tiles they finished), then the power-sum
    // pass on long constraints, then the dense kernel on what is left
    const bool corner = done && kGroupCfg[cfg].G * kGroupCfg[cfg].Q >= kCornerMinSlots;
    if (corner) {
      cudaError_t e = launch_dft_corner(d, list, count, maxL, R, Rp, x, P, fe_con, ldf, done, s);
      if (e == cudaSuccess)
        e = launch_dft_series(d, list, count, maxL, R, Rp, x, P, fe_con, ldf, done, s);
      if (e != cudaSuccess) return e;
    }
    return launch_group_fr(cfg, d, list, count, R, Rp, x, P, fe_con, ldf, corner ? done : nullptr,
                           s);
  }
  const dim3 grid(count, ceil_div(R, 32)), block(256);
  // direct-form DFT: the one-thread corner pass first on buckets longer than
  // its capacity; the direct kernel then skips the tiles it finished
  const bool dcorner = done && cfg >= 0 && cfg < kNumGroupCfg && kGroupCfg[cfg].cplx == 1 &&
                       maxL >= kDirectCornerMinL;
  if (dcorner) {
    cudaError_t e = launch_dft_corner(d, list, count, maxL, R, Rp, x, P, fe_con, ldf, done, s,
                                      false);
    if (e != cudaSuccess) return e;
  }
  const uint8_t* dflags = dcorner ? done : nullptr;
  const int RTg = ceil_div(R, 32);
  switch (cfg) {
#define CLS_LAUNCH_CASE(id, G, Q, C, Y)                                                      \
  case id:                                                                                   \
    k_fe_group<G, Q, (C != 0), (Y != 0)><<<grid, block, group_smem<G, Q>(), s>>>(            \
        list, d.fe, d.root_tab, d.coef_tab, d.fe_lit, x, R, Rp, P, fe_con, ldf, dflags, RTg,  \
        d.dft_flops);                                                                        \
    break;
    CLS_GROUP_CONFIGS(CLS_LAUNCH_CASE)
#undef CLS_LAUNCH_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_fe_unit(const DevPlan& d, int unit, int R, int Rp, const float* x, float* P,
                           float* fe_con, int ldf, uint8_t* done, cudaStream_t s, LaunchHook* h) {
  if (R == 0) return cudaSuccess;
  const int RT = ceil_div(R, 32);
  if (unit < kNumThreadCls) {
    const int t = unit;
    const int cnt = d.thread_count[t];
    if (cnt == 0) return cudaSuccess;
    const int nt = t == 0 ? AsyncTiles<8>::value : AsyncTiles<16>::value;   // 24: as 16
    const dim3 grid(std::min(ceil_div(cnt, 8), 1 << 30), ceil_div(RT, nt)), block(32, 8);
    HookScope hs(h, KC_THREAD, s);
    const FeItem* items = d.thread_items[t];
#define CLS_THREAD_LAUNCH(LO, HI)                                                          \
  k_fe_thread<LO, HI><<<grid, block, thread_xbuf_bytes<HI>(), s>>>(                       \
      items, cnt, d.root_tab, d.coef_tab, d.fe_lit, x, R,                                 \
                                             Rp, RT, P, fe_con, ldf);
    if (t == 0) {
      CLS_THREAD_LAUNCH(1, 8)
    } else if (t == 1) {
      CLS_THREAD_LAUNCH(9, 16)
    } else {
      CLS_THREAD_LAUNCH(17, 24)
    }
#undef CLS_THREAD_LAUNCH
    return cudaGetLastError();
  }
  const int b = unit - kNumThreadCls;
  if (b >= kNumBuckets || d.bucket_count[b] == 0) return cudaSuccess;
  HookScope hs(h, b < kNumDftBuckets ? KC_GROUP_DFT : KC_GROUP_REAL, s);
  return launch_group(d.bucket_cfg[b], d, d.bucket_list[b], d.bucket_count[b], d.bucket_maxL[b],
                      d.bucket_maxJ[b], R, Rp, x, P, fe_con, ldf, done, s);
}

bool fe_unit_active(const DevPlan& d, int unit) {
  if (unit < kNumThreadCls) return d.thread_count[unit] > 0;
  const int b = unit - kNumThreadCls;
  return b < kNumBuckets && d.bucket_count[b] > 0;
}

cudaError_t launch_fe(const DevPlan& d, int R, int Rp, const float* x, float* P, float* fe_con,
                      int ldf, uint8_t* done, cudaStream_t s, LaunchHook* h) {
  for (int u = 0; u < kNumFeUnits; ++u) {
    cudaError_t e = launch_fe_unit(d, u, R, Rp, x, P, fe_con, ldf, done, s, h);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_accum_step(const DevPlan& d, int R, int Rp, const float* P, float* x,
                              float lr, bool do_step, float* grad_out, uint32_t* bits,
                              cudaStream_t s, LaunchHook* h) {
  if (d.n == 0 || R == 0) return cudaSuccess;
  const int RT = ceil_div(R, 32);
  HookScope hs(h, KC_ACCUM, s);
  if (accum_tiles_per_warp(d, RT) == 4) {
    dim3 grid(ceil_div(RT, 4), std::min(ceil_div(d.n, 8), 65535)), block(32, 8);
    k_accum_step_nt<4><<<grid, block, 0, s>>>(d.n, R, Rp, RT, d.fe_voff, P, x, lr,
                                              do_step ? 1 : 0, d.fixed, grad_out, bits);
    return cudaGetLastError();
  }
  dim3 grid(RT, std::min(ceil_div(d.n, 8), 65535)), block(32, 8);
  k_accum_step<<<grid, block, 0, s>>>(d.n, R, Rp, RT, d.fe_voff, P, x, lr, do_step ? 1 : 0,
                                      d.fixed, grad_out, bits);
  return cudaGetLastError();
}

cudaError_t launch_pgd(const DevPlan& d, int R, float* x, const float* grad, float lr,
                       uint32_t* bits, cudaStream_t s, LaunchHook* h) {
  if (d.n == 0 || R == 0) return cudaSuccess;
  const int RT = ceil_div(R, 32);
  dim3 grid(RT, std::min(ceil_div(d.n, 8), 65535)), block(32, 8);
  HookScope hs(h, KC_ACCUM, s);
  k_pgd<<<grid, block, 0, s>>>(d.n, R, RT, x, grad, lr, 1, d.fixed, bits);
  return cudaGetLastError();
}

cudaError_t launch_round(const DevPlan& d, int R, const float* x, uint32_t* bits,
                         cudaStream_t s, LaunchHook* h) {
  if (d.n == 0 || R == 0) return cudaSuccess;
  const int RT = ceil_div(R, 32);
  dim3 grid(RT, std::min(ceil_div(d.n, 8), 65535)), block(32, 8);
  HookScope hs(h, KC_ACCUM, s);
  k_pgd<<<grid, block, 0, s>>>(d.n, R, RT, const_cast<float*>(x), nullptr, 0.f, 0, d.fixed,
                               bits);
  return cudaGetLastError();
}

cudaError_t launch_score(const DevPlan& d, int R, int Rp, const uint32_t* bits,
                         int32_t* nsat_part, double* wsat_part, int32_t* nsat, double* wsat,
                         cudaStream_t s, LaunchHook* h) {
  if (R == 0) return cudaSuccess;
  const int RT = ceil_div(R, 32);
  if (d.m == 0) {
    if (nsat) {
      cudaError_t e = cudaMemsetAsync(nsat, 0, sizeof(int32_t) * R, s);
      if (e != cudaSuccess) return e;
    }
    if (wsat) return cudaMemsetAsync(wsat, 0, sizeof(double) * R, s);
    return cudaSuccess;
  }
  const int nch = score_chunks(d.n_ranges);
  {
    HookScope hs(h, KC_SCORE, s);
    if (d.unit_weights)
      k_score<true><<<dim3(ceil_div(RT, kScoreTiles), nch), dim3(32, kScoreWarps), 0, s>>>(
          RT, Rp, d.n_ranges, d.score_ranges, d.score, d.lit, d.satbits, bits, nsat_part,
          wsat_part);
    else
      k_score<false><<<dim3(ceil_div(RT, kScoreTiles), nch), dim3(32, kScoreWarps), 0, s>>>(
          RT, Rp, d.n_ranges, d.score_ranges, d.score, d.lit, d.satbits, bits, nsat_part,
          wsat_part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  HookScope hs(h, KC_REDUCE, s);
  if (d.unit_weights)
    k_score_final_unit<<<ceil_div(R, 32), dim3(32, 8), 0, s>>>(R, Rp, nch, nsat_part, nsat, wsat);
  else
    k_score_final<<<ceil_div(R, 256), 256, 0, s>>>(R, Rp, nch, nsat_part, wsat_part, nsat, wsat);
  return cudaGetLastError();
}

bool persistent_eligible(const DevPlan& d) {
  for (int b = 0; b < kNumBuckets; ++b)
    if (d.bucket_count[b] > 0) return false;
  for (int t = 2; t < kNumThreadCls; ++t)   // the loop's body covers <= 16 literals
    if (d.thread_count[t] > 0) return false;
  return d.m > 0 && d.n > 0;
}

cudaError_t launch_persistent(const DevPlan& d, int R, int Rp, float* x, float lr, int n_steps,
                              float* P, uint32_t* bits, int32_t* rpart_n, double* rpart_w,
                              int32_t* nsat, double* wsat, unsigned* bar, int* err,
                              cudaStream_t s) {
  if (n_steps == 0 || R == 0) return cudaSuccess;
  // a tile that fits in shared memory: one CTA per tile, no grid barrier
  if (tile_loop_smem(d) <= kTileLoopMaxSmem) {
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    TileArgs ta{R, Rp, ceil_div(R, 32), n_steps, lr, x, bits, rpart_n, rpart_w, nsat, wsat};
    k_tile_loop<<<ceil_div(R, 32), 32 * kTileWarps, tile_loop_smem(d), s>>>(d, ta);
    return cudaGetLastError();
  }
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persistent, 256, 0);
  if (e != cudaSuccess) return e;
  if (!coop || per_sm < 1) return cudaErrorNotSupported;
  e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  PersistArgs a{R,       Rp,      ceil_div(R, 32), n_steps, lr,  x,   P,
                bits,    rpart_n, rpart_w,         nsat,    wsat, bar, err, kBarrierSpinLimit};
  DevPlan dd = d;
  void* args[] = {&dd, &a};
  return cudaLaunchCooperativeKernel((const void*)k_persistent, dim3(sms * per_sm),
                                     dim3(32, 8), args, 0, s);
}

cudaError_t launch_barrier_check(int rounds, unsigned extra, unsigned spin_limit, unsigned* bar,
                                 int* err, int* passed, cudaStream_t s) {
  int dev = 0, sms = 0, coop = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (e != cudaSuccess) return e;
  if (!coop) return cudaErrorNotSupported;
  e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  void* args[] = {&bar, &err, &rounds, &extra, &spin_limit, &passed};
  return cudaLaunchCooperativeKernel((const void*)k_barrier_check, dim3(sms), dim3(32), args, 0,
                                     s);
}

cudaError_t launch_fe_const(const DevPlan& d, int R, float* fe_con, int ldf, cudaStream_t s) {
  const int64_t total = (int64_t)d.const_count * R;
  if (total == 0 || !fe_con) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 148 * 8);
  k_fe_const<<<blocks, 256, 0, s>>>(d.const_list, d.const_count, d.fe, R, fe_con, ldf);
  return cudaGetLastError();
}

cudaError_t launch_restart_scale(int n, int R, const float* g, const float* sc, float* out,
                                 cudaStream_t s, LaunchHook* h) {
  const int64_t total = (int64_t)n * R;
  if (total == 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 148 * 16);
  HookScope hs(h, KC_REDUCE, s);
  k_restart_scale<<<blocks, 256, 0, s>>>(total, R, g, sc, out);
  return cudaGetLastError();
}

cudaError_t launch_obj(const DevPlan& d, int R, int Rp, int nch, int chunk, const float* fe_con,
                       int ldf, double* part, float* obj, cudaStream_t s, LaunchHook* h) {
  if (R == 0) return cudaSuccess;
  if (d.m == 0) return cudaMemsetAsync(obj, 0, sizeof(float) * R, s);
  HookScope hs(h, KC_REDUCE, s);
  k_obj_part<<<dim3(ceil_div(R, 256), nch), 256, 0, s>>>(d.m, R, Rp, chunk, d.score, fe_con,
                                                        ldf, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_obj_final<<<ceil_div(R, 256), 256, 0, s>>>(R, Rp, nch, part, obj);
  return cudaGetLastError();
}

}  // namespace cls
