// kernels.cu -- sm_103a kernels of the CLS hot path.
//
// Layouts (see cls.h): x[v*R + r] (variable-major, restart-minor), literal
// partials P[row*Rp + r] with row = lit_dst[e] (variable-major order, so the
// gradient of variable v is the sum of a contiguous run of rows), bitsets
// bits[v*RW + r/32] bit r%32.  Warps always span 32 consecutive restarts of
// one row, so every global access to x, P and bits is a coalesced 128-byte
// row segment or a warp-uniform broadcast.
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

// ---------------------------------------------------------------------------
// A1 init: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x64_10(uint64_t& x0, uint64_t& x1, uint64_t& x2,
                                              uint64_t& x3, uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    uint64_t hi0 = __umul64hi(M0, x0), lo0 = M0 * x0;
    uint64_t hi1 = __umul64hi(M1, x2), lo1 = M1 * x2;
    uint64_t n0 = hi1 ^ x1 ^ k0, n2 = hi0 ^ x3 ^ k1;
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
// A2-A5, closed-form products (OR, XOR, NAE) with L <= MAXL:
// one thread per (constraint, restart); lanes span restarts.
// FE = b0 + sum_j b'_j prod_i F_ij, dFE/dy_i = sum_j c'_j prod_{l!=i} F_lj with
// real factors F = A + y B; prefix products kept in registers, suffix products
// carried backwards -- no division.
// ---------------------------------------------------------------------------
template <int MAXL>
__global__ void __launch_bounds__(256) k_fe_thread(
    const int32_t* __restrict__ list, int count, const FeItem* __restrict__ fe,
    const F4* __restrict__ root, const F4* __restrict__ coef, const int32_t* __restrict__ lit_var,
    const float* __restrict__ lit_sgn, const int32_t* __restrict__ lit_dst,
    const float* __restrict__ x, int R, int Rp, float* __restrict__ P, float* __restrict__ fe_con,
    int ldf) {
  const int r = blockIdx.x * 32 + threadIdx.x;
  if (r >= R) return;
  for (int ci = blockIdx.y * blockDim.y + threadIdx.y; ci < count; ci += gridDim.y * blockDim.y) {
    const FeItem it = fe[list[ci]];
    const int L = it.L;
    float y[MAXL], g[MAXL], pre[MAXL];
#pragma unroll
    for (int i = 0; i < MAXL; ++i) {
      g[i] = 0.f;
      y[i] = 1.f;
      if (i < L) {
        const int e = it.lit0 + i;
        y[i] = lit_sgn[e] * x[(size_t)lit_var[e] * R + r];
      }
    }
    float val = it.b0;
    for (int j = 0; j < it.J; ++j) {
      const F4 rt = root[it.root_off + j];
      const F4 cf = coef[it.coef_off + j];
      float run = 1.f;
#pragma unroll
      for (int i = 0; i < MAXL; ++i) {
        if (i < L) {
          pre[i] = run;
          run *= fmaf(y[i], rt.y, rt.x);
        }
      }
      val = fmaf(cf.x, run, val);
      float suf = cf.z;  // c'_j folded into the suffix product
#pragma unroll
      for (int i = MAXL - 1; i >= 0; --i) {
        if (i < L) {
          g[i] = fmaf(pre[i], suf, g[i]);
          suf *= fmaf(y[i], rt.y, rt.x);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < MAXL; ++i) {
      if (i < L) {
        const int e = it.lit0 + i;
        P[(size_t)lit_dst[e] * Rp + r] = it.w * lit_sgn[e] * g[i];
      }
    }
    if (fe_con) fe_con[(size_t)it.c * ldf + r] = val;
  }
}

// ---------------------------------------------------------------------------
// A2-A5 lane-group kernel: G lanes share one (constraint, restart); lane lam
// holds literals lam, lam+G, ..., (at most Q).  One block = one constraint x
// a tile of 32 restarts; literal values are staged in shared memory as
// ys[i*LDR + rr] with LDR = 32 + 32/G, which makes both the coalesced staging
// stores (lanes over rr) and the group reads (lanes over lam, groups over rr)
// bank-conflict free.
//
// Per root j: factors F_ij, lane-local exclusive prefix products, then a
// butterfly over the G lanes that yields both the total G_j = prod_i F_ij and
// the product of the OTHER lanes' chunks (leave-one-lane-out, O).  The
// gradient uses prod_{l!=i} F_lj = O * prefix_i * suffix_i with the suffix
// carried backwards and c'_j O folded into it: no division by a factor, so
// nothing breaks where a factor vanishes.  Padding literal slots hold y = 1,
// for which every root's factor is exactly 1 (A + B == 1, C - C == 0).
// ---------------------------------------------------------------------------
template <int G>
struct GroupGeom {
  static constexpr int LDR = 32 + 32 / G;
  static constexpr int GPW = 32 / G;         // groups per warp
  static constexpr int GPB = 8 * GPW;        // groups per block (256 threads)
  static constexpr int PASSES = 32 / GPB;    // to cover 32 restarts
};

template <int G, int Q, bool CPLX>
__global__ void __launch_bounds__(256) k_fe_group(
    const int32_t* __restrict__ list, const FeItem* __restrict__ fe,
    const F4* __restrict__ root, const F4* __restrict__ coef, const int32_t* __restrict__ lit_var,
    const float* __restrict__ lit_sgn, const int32_t* __restrict__ lit_dst,
    const float* __restrict__ x, int R, int Rp, float* __restrict__ P, float* __restrict__ fe_con,
    int ldf) {
  using Geo = GroupGeom<G>;
  extern __shared__ float smem[];
  float* ys = smem;                  // [L][LDR]
  __shared__ float fe_s[32];
  const FeItem it = fe[list[blockIdx.x]];
  const int L = it.L;
  const int r0 = blockIdx.y * 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // stage literal values y = s * x (coalesced rows of 32 restarts)
  for (int i = warp; i < L; i += 8) {
    const int e = it.lit0 + i;
    const int r = r0 + lane;
    ys[i * Geo::LDR + lane] = (r < R) ? lit_sgn[e] * x[(size_t)lit_var[e] * R + r] : 1.0f;
  }
  __syncthreads();

  const int lam = lane % G;
  const int gi = lane / G;
#pragma unroll 1
  for (int pass = 0; pass < Geo::PASSES; ++pass) {
    const int rr = pass * Geo::GPB + warp * Geo::GPW + gi;
    float y[Q], acc[Q];
#pragma unroll
    for (int s = 0; s < Q; ++s) {
      const int i = lam + G * s;
      y[s] = (i < L) ? ys[i * Geo::LDR + rr] : 1.0f;
      acc[s] = 0.f;
    }
    float val = 0.f;
#pragma unroll 1
    for (int j = 0; j < it.J; ++j) {
      const float4 rt = ldg4(&root[it.root_off + j]);
      const float4 cf = ldg4(&coef[it.coef_off + j]);
      if constexpr (CPLX) {
        float pr[Q], pim[Q];
        float qr = fmaf(y[0], rt.y, rt.x), qi = fmaf(-y[0], rt.z, rt.z);
        pr[0] = 1.f;
        pim[0] = 0.f;
#pragma unroll
        for (int s = 1; s < Q; ++s) {
          pr[s] = qr;
          pim[s] = qi;
          const float fr = fmaf(y[s], rt.y, rt.x), fi = fmaf(-y[s], rt.z, rt.z);
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
            const float fr = fmaf(y[s], rt.y, rt.x), fi = fmaf(-y[s], rt.z, rt.z);
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
          q *= live ? fmaf(y[s], rt.y, rt.x) : 1.f;
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
          h *= live ? fmaf(y[s], rt.y, rt.x) : 1.f;
        }
      }
    }
    // partials back into the staging slots (each lane owns its slots)
#pragma unroll
    for (int s = 0; s < Q; ++s) {
      const int i = lam + G * s;
      if (i < L) ys[i * Geo::LDR + rr] = acc[s];
    }
    if (lam == 0) fe_s[rr] = it.b0 + val;
  }
  __syncthreads();
  // write partials w * s_e * dFE/dy_e to their variable-major rows
  for (int i = warp; i < L; i += 8) {
    const int e = it.lit0 + i;
    const int r = r0 + lane;
    if (r < R) P[(size_t)lit_dst[e] * Rp + r] = it.w * lit_sgn[e] * ys[i * Geo::LDR + lane];
  }
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

__global__ void __launch_bounds__(256) k_accum_step(int n, int R, int Rp, int RW,
                                                    const int32_t* __restrict__ voff,
                                                    const float* __restrict__ P,
                                                    float* __restrict__ x, float lr, int do_step,
                                                    const uint8_t* __restrict__ fixed,
                                                    float* __restrict__ grad_out,
                                                    uint32_t* __restrict__ bits) {
  const int lane = threadIdx.x;
  const int r = blockIdx.x * 32 + lane;
  const bool act = r < R;
  for (int v = blockIdx.y * blockDim.y + threadIdx.y; v < n; v += gridDim.y * blockDim.y) {
    const int k0 = voff[v], k1 = voff[v + 1];
    float g = 0.f;
    if (act) {
      const float* p = P + (size_t)k0 * Rp + r;
      int k = k0;
      for (; k + 4 <= k1; k += 4, p += 4 * (size_t)Rp) {
        const float a0 = p[0], a1 = p[(size_t)Rp], a2 = p[2 * (size_t)Rp], a3 = p[3 * (size_t)Rp];
        g += a0;
        g += a1;
        g += a2;
        g += a3;
      }
      for (; k < k1; ++k, p += Rp) g += p[0];
    }
    if (grad_out && act) grad_out[(size_t)v * R + r] = g;
    if (do_step) {
      float xv = 0.f;
      if (act) {
        xv = x[(size_t)v * R + r];
        if (!(fixed && fixed[v])) {
          xv = pgd_project(xv, g, lr);
          x[(size_t)v * R + r] = xv;
        }
      }
      const uint32_t b = __ballot_sync(kFull, act && xv < 0.0f);
      if (bits && lane == 0) bits[(size_t)v * RW + blockIdx.x] = b;
    }
  }
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
// A9: exact satisfaction counts.  A literal is true iff its variable's bit
// XOR (sign < 0).  The bitset word of a variable is a warp-uniform load; lane
// r extracts its own bit.  Per block: a chunk of constraints x 32 restarts,
// reduced over the 8 warps in a fixed order into per-chunk partials.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_score(int m, int R, int Rp, int RW, int chunk,
                                               const ScoreItem* __restrict__ sc,
                                               const int32_t* __restrict__ lit_var,
                                               const float* __restrict__ lit_sgn,
                                               const uint32_t* __restrict__ satbits,
                                               const uint32_t* __restrict__ bits,
                                               int32_t* __restrict__ nsat_part,
                                               double* __restrict__ wsat_part) {
  __shared__ int32_t cnt_s[8][32];
  __shared__ double w_s[8][32];
  const int lane = threadIdx.x, ty = threadIdx.y;
  const int tile = blockIdx.x;
  const int c0 = blockIdx.y * chunk;
  const int c1 = min(m, c0 + chunk);
  int cnt = 0;
  double ws = 0.0;
  for (int c = c0 + ty; c < c1; c += blockDim.y) {
    const ScoreItem s = sc[c];
    int t = 0;
    for (int i = 0; i < s.L; ++i) {
      const int e = s.lit0 + i;
      const uint32_t wd = bits[(size_t)lit_var[e] * RW + tile];
      t += (int)((wd >> lane) & 1u) ^ (int)(lit_sgn[e] < 0.f);
    }
    bool sat;
    if (s.mode == 0)
      sat = (t >= s.lo) && (t <= s.hi);
    else if (s.mode == 1)
      sat = (t & 1) != 0;
    else
      sat = ((satbits[(s.lo + t) >> 5] >> ((s.lo + t) & 31)) & 1u) != 0;
    cnt += sat ? 1 : 0;
    ws += sat ? (double)s.w : 0.0;
  }
  cnt_s[ty][lane] = cnt;
  w_s[ty][lane] = ws;
  __syncthreads();
  if (ty == 0) {
    int a = 0;
    double b = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      a += cnt_s[k][lane];
      b += w_s[k][lane];
    }
    const int r = tile * 32 + lane;
    nsat_part[(size_t)blockIdx.y * Rp + r] = a;
    wsat_part[(size_t)blockIdx.y * Rp + r] = b;
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

template <int G, int Q, int C>
size_t group_smem(int maxL) {
  return (size_t)maxL * GroupGeom<G>::LDR * sizeof(float);
}

}  // namespace

cudaError_t set_kernel_attributes() {
  cudaError_t err = cudaSuccess;
#define CLS_SET_ATTR(id, G, Q, C)                                                        \
  if (err == cudaSuccess)                                                                \
    err = cudaFuncSetAttribute(k_fe_group<G, Q, (C != 0)>,                               \
                               cudaFuncAttributeMaxDynamicSharedMemorySize,              \
                               (int)group_smem<G, Q, C>(G * Q));
  CLS_GROUP_CONFIGS(CLS_SET_ATTR)
#undef CLS_SET_ATTR
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

cudaError_t launch_fe(const DevPlan& d, int R, int Rp, const float* x, float* P, float* fe_con,
                      int ldf, cudaStream_t s, LaunchHook* h) {
  const int RT = ceil_div(R, 32);
  if (R == 0) return cudaSuccess;
  for (int t = 0; t < 2; ++t) {
    const int cnt = d.thread_count[t];
    if (cnt == 0) continue;
    dim3 grid(RT, std::min(ceil_div(cnt, 8), 65535)), block(32, 8);
    HookScope hs(h, KC_THREAD, s);
    if (t == 0)
      k_fe_thread<kThreadMaxL0><<<grid, block, 0, s>>>(d.thread_list[t], cnt, d.fe, d.root_tab,
                                                       d.coef_tab, d.lit_var, d.lit_sgn,
                                                       d.lit_dst, x, R, Rp, P, fe_con, ldf);
    else
      k_fe_thread<kThreadMaxL1><<<grid, block, 0, s>>>(d.thread_list[t], cnt, d.fe, d.root_tab,
                                                       d.coef_tab, d.lit_var, d.lit_sgn,
                                                       d.lit_dst, x, R, Rp, P, fe_con, ldf);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
#define CLS_LAUNCH_GROUP(id, G, Q, C)                                                        \
  if (d.group_count[id] > 0) {                                                               \
    dim3 grid(d.group_count[id], RT), block(256);                                            \
    HookScope hs(h, C ? KC_GROUP_DFT : KC_GROUP_REAL, s);                                    \
    k_fe_group<G, Q, (C != 0)><<<grid, block, group_smem<G, Q, C>(d.group_maxL[id]), s>>>(   \
        d.group_list[id], d.fe, d.root_tab, d.coef_tab, d.lit_var, d.lit_sgn, d.lit_dst, x, \
        R, Rp, P, fe_con, ldf);                                                              \
    cudaError_t e = cudaGetLastError();                                                      \
    if (e != cudaSuccess) return e;                                                          \
  }
  CLS_GROUP_CONFIGS(CLS_LAUNCH_GROUP)
#undef CLS_LAUNCH_GROUP
  return cudaSuccess;
}

cudaError_t launch_accum_step(const DevPlan& d, int R, int Rp, const float* P, float* x,
                              float lr, bool do_step, float* grad_out, uint32_t* bits,
                              cudaStream_t s, LaunchHook* h) {
  if (d.n == 0 || R == 0) return cudaSuccess;
  const int RT = ceil_div(R, 32);
  dim3 grid(RT, std::min(ceil_div(d.n, 8), 65535)), block(32, 8);
  HookScope hs(h, KC_ACCUM, s);
  k_accum_step<<<grid, block, 0, s>>>(d.n, R, Rp, RT, d.voff, P, x, lr, do_step ? 1 : 0,
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

cudaError_t launch_score(const DevPlan& d, int R, int Rp, int nch, int chunk,
                         const uint32_t* bits, int32_t* nsat_part, double* wsat_part,
                         int32_t* nsat, double* wsat, cudaStream_t s, LaunchHook* h) {
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
  {
    HookScope hs(h, KC_SCORE, s);
    k_score<<<dim3(RT, nch), dim3(32, 8), 0, s>>>(d.m, R, Rp, RT, chunk, d.score, d.lit_var,
                                                  d.lit_sgn, d.satbits, bits, nsat_part,
                                                  wsat_part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  HookScope hs(h, KC_REDUCE, s);
  k_score_final<<<ceil_div(R, 256), 256, 0, s>>>(R, Rp, nch, nsat_part, wsat_part, nsat, wsat);
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
