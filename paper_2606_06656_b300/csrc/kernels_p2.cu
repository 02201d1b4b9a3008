// kernels_p2.cu -- the lane-group DFT FE+gradient kernel with roots taken in
// pairs (j, j+1) and carried in packed FP32x2 registers (sm_100+ FFMA2/FMUL2).
//
// Same mathematics, data layout and staging as k_fe_group (kernels.cu): G
// lanes share one (constraint, restart), lane lam holds literals lam,
// lam+G, ...; per root, the factors F_ij = (A + y B) + i (C - y C), lane-local
// exclusive prefix products, a butterfly over the G lanes giving the total
// product G_j and the product of the other lanes' chunks O, and a backward
// sweep carrying c'_j O times the suffix product.  Here every complex
// quantity holds the two roots of a pair in the .x/.y halves of float2
// values, so each packed instruction advances both roots: half the
// instructions and two independent dependency chains per thread.  Imaginary
// parts are kept negated where a product needs them (nfi = y C - C, nhi =
// -Im h), so no packed negation is ever required.  An odd last root is paired
// with a dummy root of factor exactly 1 and coefficient 0.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "kernels.cuh"

namespace cls {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float4 ldg4(const F4* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ int rec_row(int32_t dst) { return dst & 0x7fffffff; }
__device__ __forceinline__ float rec_sgn(int32_t dst) { return dst < 0 ? -1.0f : 1.0f; }

__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 dup(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 shfl2(float2 v, int d) {
  return make_float2(__shfl_xor_sync(kFull, v.x, d), __shfl_xor_sync(kFull, v.y, d));
}

template <int G>
struct Geo2 {
  static constexpr int LDR = 32 + 32 / G;
  static constexpr int GPW = 32 / G;
  static constexpr int GPB = 8 * GPW;
  static constexpr int PASSES = 32 / GPB;
};

template <int G, int Q, bool YS>
__global__ void __launch_bounds__(256) k_fe_group_p2(
    const int32_t* __restrict__ list, const FeItem* __restrict__ fe,
    const F4* __restrict__ root, const F4* __restrict__ coef, const LitRec* __restrict__ lit,
    const float* __restrict__ x, int R, int Rp, float* __restrict__ P,
    float* __restrict__ fe_con, int ldf, unsigned long long* __restrict__ flops) {
  using Geo = Geo2<G>;
  constexpr int LS = G * Q;
  extern __shared__ float smem[];
  float* ys = smem;                  // [LS][LDR]
  __shared__ float fe_s[32];
  const FeItem it = fe[list[blockIdx.x]];
  const int L = it.L;
  const int r0 = blockIdx.y * 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  for (int i = warp; i < LS; i += 8) {
    float v = 1.0f;
    if (i < L) {
      const LitRec rc = lit[it.lit0 + i];
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
    const float* ycol = ys + lam * Geo::LDR + rr;
    float yreg[YS ? 1 : Q];
    float2 acc[Q];
#pragma unroll
    for (int s = 0; s < Q; ++s) {
      if constexpr (!YS) yreg[s] = ycol[s * G * Geo::LDR];
      acc[s] = make_float2(0.f, 0.f);
    }
    auto Y = [&](int s) -> float {
      if constexpr (YS) return ycol[s * G * Geo::LDR];
      else return yreg[s];
    };
    float val = 0.f;
#pragma unroll 1
    for (int j = 0; j < it.J; j += 2) {
      const bool two = j + 1 < it.J;
      const float4 ra = ldg4(&root[it.root_off + j]);
      const float4 ca = ldg4(&coef[it.coef_off + j]);
      const float4 rb = two ? ldg4(&root[it.root_off + j + 1]) : make_float4(1.f, 0.f, 0.f, 0.f);
      const float4 cb = two ? ldg4(&coef[it.coef_off + j + 1]) : make_float4(0.f, 0.f, 0.f, 0.f);
      const float2 A2 = make_float2(ra.x, rb.x), B2 = make_float2(ra.y, rb.y);
      const float2 C2 = make_float2(ra.z, rb.z), nC2 = make_float2(-ra.z, -rb.z);
      // forward: exclusive prefix products q = qr + i qi of both roots
      float2 pr[Q], pim[Q];
      float2 qr, qi;
      {
        const float2 y2 = dup(Y(0));
        qr = fma2(y2, B2, A2);
        qi = fma2(y2, nC2, C2);
      }
      pr[0] = make_float2(1.f, 1.f);
      pim[0] = make_float2(0.f, 0.f);
#pragma unroll
      for (int s = 1; s < Q; ++s) {
        pr[s] = qr;
        pim[s] = qi;
        const float2 y2 = dup(Y(s));
        const float2 fr = fma2(y2, B2, A2);
        const float2 fi = fma2(y2, nC2, C2);
        const float2 nfi = fma2(y2, C2, nC2);
        const float2 nr = fma2(qi, nfi, mul2(qr, fr));   // qr fr - qi fi
        const float2 ni = fma2(qi, fr, mul2(qr, fi));    // qr fi + qi fr
        qr = nr;
        qi = ni;
      }
      // butterfly over the G lanes: Pt = total, O = product of the others
      float2 Ptr = qr, Pti = qi, Or = make_float2(1.f, 1.f), Oi = make_float2(0.f, 0.f);
#pragma unroll
      for (int d = 1; d < G; d <<= 1) {
        const float2 tr = shfl2(Ptr, d), ti = shfl2(Pti, d);
        const float2 nti = make_float2(-ti.x, -ti.y);
        if (d == 1) {
          Or = tr;
          Oi = ti;
        } else {
          const float2 a = fma2(Oi, nti, mul2(Or, tr)), b = fma2(Oi, tr, mul2(Or, ti));
          Or = a;
          Oi = b;
        }
        const float2 a = fma2(Pti, nti, mul2(Ptr, tr)), b = fma2(Pti, tr, mul2(Ptr, ti));
        Ptr = a;
        Pti = b;
      }
      // FE += Re(b'_j G_j) for both roots
      val = fmaf(ca.x, Ptr.x, val);
      val = fmaf(-ca.y, Pti.x, val);
      val = fmaf(cb.x, Ptr.y, val);
      val = fmaf(-cb.y, Pti.y, val);
      // h = c' O, kept as (hr, nhi = -Im h)
      const float2 cre = make_float2(ca.z, cb.z), ncim = make_float2(-ca.w, -cb.w);
      const float2 ncre = make_float2(-ca.z, -cb.z);
      float2 hr = fma2(ncim, Oi, mul2(cre, Or));      // c.re Or - c.im Oi
      float2 nhi = fma2(ncre, Oi, mul2(ncim, Or));    // -(c.re Oi + c.im Or)
#pragma unroll
      for (int s = Q - 1; s >= 0; --s) {
        // acc += Re(prefix * h) = pr hr - pi hi = pr hr + pi nhi
        acc[s] = fma2(pr[s], hr, acc[s]);
        acc[s] = fma2(pim[s], nhi, acc[s]);
        if (s > 0) {
          const float2 y2 = dup(Y(s));
          const float2 fr = fma2(y2, B2, A2);
          const float2 fi = fma2(y2, nC2, C2);
          const float2 nfi = fma2(y2, C2, nC2);
          const float2 a = fma2(nhi, fi, mul2(hr, fr));    // hr fr - hi fi
          const float2 b = fma2(hr, nfi, mul2(nhi, fr));   // -(hr fi + hi fr)
          hr = a;
          nhi = b;
        }
      }
    }
#pragma unroll
    for (int s = 0; s < Q; ++s) {
      const int i = lam + G * s;
      if (i < L) ys[i * Geo::LDR + rr] = acc[s].x + acc[s].y;
    }
    if (lam == 0) fe_s[rr] = it.b0 + val;
  }
  __syncthreads();
  for (int i = warp; i < L; i += 8) {
    const LitRec rc = lit[it.lit0 + i];
    const int r = r0 + lane;
    if (r < R)
      st_partial(&P[(size_t)rec_row(rc.dst) * Rp + r], it.w * rec_sgn(rc.dst) * ys[i * Geo::LDR + lane]);
  }
  // 20 flops per (literal, root) of every restart, as the direct form
  if (flops && threadIdx.x == 0)
    atomicAdd(flops, 20ull * (unsigned long long)L * (unsigned long long)it.J *
                         (unsigned long long)min(32, R - r0));
  if (fe_con && warp == 0 && r0 + lane < R) fe_con[(size_t)it.c * ldf + r0 + lane] = fe_s[lane];
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

template <int G, int Q>
constexpr size_t p2_smem() {
  return (size_t)G * Q * Geo2<G>::LDR * sizeof(float);
}

}  // namespace

cudaError_t set_p2_attributes() {
  cudaError_t err = cudaSuccess;
#define CLS_P2_ATTR(id, G, Q, C, Y)                                                           \
  if (err == cudaSuccess)                                                                     \
    err = cudaFuncSetAttribute(k_fe_group_p2<G, Q, (Y != 0)>,                                 \
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p2_smem<G, Q>());
  CLS_P2_CONFIGS(CLS_P2_ATTR)
#undef CLS_P2_ATTR
  return err;
}

cudaError_t launch_group_p2(int cfg, const DevPlan& d, const int32_t* list, int count, int R,
                            int Rp, const float* x, float* P, float* fe_con, int ldf,
                            cudaStream_t s) {
  if (count == 0 || R == 0) return cudaSuccess;
  const dim3 grid(count, ceil_div(R, 32)), block(256);
  switch (cfg) {
#define CLS_P2_CASE(id, G, Q, C, Y)                                                        \
  case id:                                                                                 \
    k_fe_group_p2<G, Q, (Y != 0)><<<grid, block, p2_smem<G, Q>(), s>>>(                    \
        list, d.fe, d.root_tab, d.coef_tab, d.fe_lit, x, R, Rp, P, fe_con, ldf,            \
        d.dft_flops);                                                                      \
    break;
    CLS_P2_CONFIGS(CLS_P2_CASE)
#undef CLS_P2_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace cls
