// kernels_fr.cu -- the lane-group DFT FE+gradient kernel on factored roots.
//
// Same work split, staging and output as k_fe_group (kernels.cu): a block
// takes one constraint and 32 restarts, G lanes share one (constraint,
// restart), lane lam holds literal slots lam, lam+G, ... (Q of them; slots
// beyond L are staged as y = 1).  What changes is the arithmetic per root.
//
// With phi = pi j/(L+1) (half the root's angle), the Poisson-binomial factor
// of Sec. 2.3's characteristic function is
//     alpha + beta w^j = e^{i phi} (cos phi - i y sin phi) = z_j u_j(y),
//     phi <= pi/4:           z = 1/(1 - i t), u = 1 - i y t,  t = tan phi,
//     pi/4 < phi <= 0.42 pi: z = 1/(t + i),   u = y t + i,    t = tan phi,
//     phi > 0.42 pi:         z = 1/(1 + i t), u = y + i t,    t = cot phi,
// so |u| <= 4.02 and a padding slot (y = 1) has z u = 1 exactly.  A lane's
// product of its Q factors is carried in u alone (3 FP32 operations per
// complex product in the first two forms, 4 in the third, against 6 for the
// factor alpha + beta w^j itself) and scaled once by z^Q; the products over
// all lanes then equal G_j = prod_i (alpha_i + beta_i w^j), and the
// leave-one-out product for literal i is O * z^(Q-1) * (the lane's
// u-products before and after i), O the other lanes' scaled products.
// Products of up to 32 factors of modulus <= 4.02 stay far inside the FP32
// range (and z^Q far above its underflow).  z is defined from the FP32-rounded
// t itself (z = 1/u(1)), so padding is neutral up to one rounding of z^Q;
// z^Q and z^(Q-1) come from an FP64 host table, c'_j z^(Q-1) is formed per
// block in a prologue.  No division in the kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "kernels.cuh"

namespace cls {
namespace {

constexpr unsigned kFull = 0xffffffffu;
// bound on the sum of the skipped tail terms: kTailEps = 2^-30 (the
// threshold uses ln(1 / kTailEps) = 30 ln 2, rounded up)
constexpr float kTailLogInvEps = 20.80f;

__device__ __forceinline__ float4 ldg4(const F4* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ int rec_row(int32_t dst) { return dst & 0x7fffffff; }
__device__ __forceinline__ float rec_sgn(int32_t dst) { return dst < 0 ? -1.0f : 1.0f; }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// index of Q in kFrQ (compile time)
template <int Q>
struct FrQIndex {
  static constexpr int value = Q == 1    ? 0
                               : Q == 2  ? 1
                               : Q == 4  ? 2
                               : Q == 6  ? 3
                               : Q == 8  ? 4
                               : Q == 10 ? 5
                               : Q == 12 ? 6
                               : Q == 14 ? 7
                               : Q == 16 ? 8
                               : Q == 18 ? 9
                               : Q == 20 ? 10
                               : Q == 24 ? 11
                               : Q == 28 ? 12
                               : Q == 32 ? 13
                                         : -1;
  static_assert(value >= 0, "slot count without a root-power table");
};

template <int G>
struct FrGeom {
  static constexpr int LDR = 32 + 32 / G;
  static constexpr int GPW = 32 / G;
  static constexpr int GPB = 8 * GPW;
  static constexpr int PASSES = 32 / GPB;
};

// One root for one lane: forward u-products, scale by z^Q, butterfly over
// the G lanes, FE term, backward sweep of the leave-one-out products into
// acc.  F selects the factored form (kernels.cuh).  rt = {t, z^Q},
// cf = {b'_j, c'_j z^(Q-1)}.  Returns Re(b'_j G_j).
template <int G, int Q, bool YS, int F>
__device__ __forceinline__ float fr_root(const float4 rt, const float4 cf,
                                         const float (&yreg)[YS ? 1 : Q], const float* ycol,
                                         float (&acc)[Q]) {
  constexpr int YST = G * FrGeom<G>::LDR;
  auto Y = [&](int s) -> float {
    if constexpr (YS) return ycol[s * YST];
    else return yreg[s];
  };
  const float tk = rt.x;
  float pr[Q], pim[Q];
  float qr, qi;
  fr_uinit<F>(qr, qi, Y(0), tk);
#pragma unroll
  for (int s = 1; s < Q; ++s) {
    pr[s] = qr;
    pim[s] = qi;
    fr_umul<F>(qr, qi, Y(s), tk);
  }
  // the lane's chunk times z^Q, then total (Pt) and others' product (O)
  float Ptr = qr * rt.y - qi * rt.z, Pti = qr * rt.z + qi * rt.y;
  float Or = 1.f, Oi = 0.f;
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
  const float val = cf.x * Ptr - cf.y * Pti;
  float hr = cf.z * Or - cf.w * Oi, hi = cf.z * Oi + cf.w * Or;
#pragma unroll
  for (int s = Q - 1; s >= 1; --s) {
    acc[s] = fmaf(pr[s], hr, acc[s]);
    acc[s] = fmaf(-pim[s], hi, acc[s]);
    fr_umul<F>(hr, hi, Y(s), tk);
  }
  acc[0] += hr;
  return val;
}

template <int G, int Q>
struct FrCap {
  static constexpr int JC = (G * Q + 1) / 2;   // most roots of a constraint that fits
};

template <int G, int Q>
constexpr size_t fr_smem() {
  return (size_t)2 * FrCap<G, Q>::JC * sizeof(float4) +
         (size_t)G * Q * FrGeom<G>::LDR * sizeof(float);
}

template <int G, int Q, bool YS>
__global__ void __launch_bounds__(256) k_fe_group_fr(
    const int32_t* __restrict__ list, const FeItem* __restrict__ fe,
    const F4* __restrict__ root, const F4* __restrict__ zpow, const F4* __restrict__ coef,
    const LitRec* __restrict__ lit,
    const float* __restrict__ x, int R, int Rp, float* __restrict__ P,
    float* __restrict__ fe_con, int ldf, const uint8_t* __restrict__ done,
    const SerInfo* __restrict__ ser_info, const float* __restrict__ ser_d,
    unsigned long long* __restrict__ flops) {
  using Geo = FrGeom<G>;
  constexpr int LS = G * Q;
  constexpr int JC = FrCap<G, Q>::JC;
  extern __shared__ float4 smem4[];
  float4* rs = smem4;                                        // [JC]
  float4* cs = smem4 + JC;                                   // [JC]
  float* ys = reinterpret_cast<float*>(smem4 + 2 * JC);     // [LS][LDR]
  __shared__ float fe_s[32];
  // a tile the corner pass has finished (kernels_corner.cu); the flag is
  // indexed by the constraint id, which is also the FE item's index
  const int ci = list[blockIdx.x];
  const uint8_t tflag = done ? done[(size_t)ci * gridDim.y + blockIdx.y] : kTileOpen;
  if (tflag == kTileDone) return;
  // a tile whose low roots the Chebyshev pass evaluated: start after them
  // and add its saved terms (D_k, FE - b0 per restart) to the partials and FE
  const bool low = tflag == kTileLow;
  const int j0 = low ? ser_info[ci].js1 : 0;
  __shared__ float sD[(kSeriesK1 + 1) * 32];
  const FeItem it = fe[ci];
  const int L = it.L, J = it.J;
  const int r0 = blockIdx.y * 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // per-root constants for this Q
  for (int j = threadIdx.x; j < J; j += 256) {
    const float4 rt = ldg4(&root[it.root_off + j]);
    const float4 zp = ldg4(&zpow[(size_t)(it.root_off + j) * kNumFrQ + FrQIndex<Q>::value]);
    const float4 cf = ldg4(&coef[it.coef_off + j]);
    const float2 cz = cmul(make_float2(cf.z, cf.w), make_float2(zp.z, zp.w));
    rs[j] = make_float4(rt.w, zp.x, zp.y, 0.f);
    cs[j] = make_float4(cf.x, cf.y, cz.x, cz.y);
  }
  // the constraint's literal records once per block (one coalesced read),
  // then the literal values y = s * x (coalesced rows of 32 restarts), four
  // rows in flight per warp
  __shared__ LitRec lrec_s[LS];
  for (int i = threadIdx.x; i < L; i += 256) lrec_s[i] = lit[it.lit0 + i];
  if (low) {
    const float* sdg = ser_d + (size_t)ser_info[ci].slot * (kSeriesK1 + 1) * Rp + r0;
    for (int e = threadIdx.x; e < (kSeriesK1 + 1) * 32; e += 256)
      sD[e] = (r0 + (e & 31) < R) ? sdg[(size_t)(e >> 5) * Rp + (e & 31)] : 0.f;
  }
  __syncthreads();
  // rows of x go to shared memory as asynchronous 4-byte copies (all of a
  // thread's rows in flight at once); the signs are applied afterwards
  {
    const int r = r0 + lane;
    for (int i = warp; i < LS; i += 8) {
      float* dst = &ys[i * Geo::LDR + lane];
      if (i < L && r < R) cp_async4(dst, &x[(size_t)lrec_s[i].var * R + r]);
      else *dst = 1.0f;
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    if (r < R)
      for (int i = warp; i < L; i += 8)
        if (lrec_s[i].dst < 0) ys[i * Geo::LDR + lane] = -ys[i * Geo::LDR + lane];
  }
  __syncthreads();

  const int lam = lane % G;
  const int gi = lane / G;
  const int nA = fr_roots_form0(L), nB = fr_roots_form01(L);   // root forms 0 | 1 | 2
  const float tailT = logf(2.f * (float)J) + kTailLogInvEps;
#pragma unroll 1
  for (int pass = 0; pass < Geo::PASSES; ++pass) {
    const int rr = pass * Geo::GPB + warp * Geo::GPW + gi;
    const float* ycol = ys + lam * Geo::LDR + rr;
    float yreg[YS ? 1 : Q], acc[Q];
#pragma unroll
    for (int s = 0; s < Q; ++s) {
      if constexpr (!YS) yreg[s] = ycol[s * G * Geo::LDR];
      acc[s] = 0.f;
    }
    // Tail cutoff.  |alpha + beta w^j|^2 = 1 - 2 alpha beta (1 - cos theta_j),
    // so with S = sum_i alpha_i beta_i = sum_i (1 - y_i^2)/4 every product
    // over all or all-but-one factors has modulus <= exp(-(S - 1/4)(1 - cos
    // theta_j)), and |b'_j|, |c'_j| <= 2.  Roots with 2 sin^2(phi_j)(S - 1/4)
    // >= T = ln(2J / kTailEps) therefore add at most kTailEps in total to FE
    // and to every partial; they are skipped.  The warp runs to the largest
    // cutoff of its groups (extra roots are exact terms).
    float S = 0.f;
#pragma unroll
    for (int s = 0; s < Q; ++s) {
      const float y = YS ? ycol[s * G * Geo::LDR] : yreg[s];
      S = fmaf(-0.25f * y, y, S + 0.25f);
    }
#pragma unroll
    for (int d = 1; d < G; d <<= 1) S += __shfl_xor_sync(kFull, S, d);
    int jc = J;
    const float S1 = S - 0.25f;
    if (S1 > 0.f) {
      const float q = tailT / (2.f * S1);
      if (q < 1.f)
        jc = min(J, (int)ceilf(asinf(sqrtf(q)) * (float)(L + 1) * 0.318309886f) + 1);
    }
    const int jw = __reduce_max_sync(kFull, jc);
    if (flops) {
      // algorithmic work of the roots each restart needs: 14 / 16 flops per
      // (literal, root) in the two factored forms (counted once per group)
      // (per group <= 1024 * 16 * 512 < 2^24, so the warp sum fits 32 bits)
      const int jl = min(jc, j0);   // roots the power-sum pass took
      const unsigned f = lam == 0 ? (unsigned)L * (14u * (min(nB, jc) - min(nB, jl)) +
                                                   16u * (max(0, jc - nB) - max(0, jl - nB)) +
                                                   (low ? 4u * kSeriesK1 : 0u))
                                  : 0u;
      const unsigned tot = __reduce_add_sync(kFull, f);
      if (lane == 0) atomicAdd(flops, (unsigned long long)tot);
    }
    float val = 0.f;
#pragma unroll 1
    for (int j = j0; j < min(nA, jw); ++j)
      val += fr_root<G, Q, YS, 0>(rs[j], cs[j], yreg, ycol, acc);
#pragma unroll 1
    for (int j = max(nA, j0); j < min(nB, jw); ++j)
      val += fr_root<G, Q, YS, 1>(rs[j], cs[j], yreg, ycol, acc);
#pragma unroll 1
    for (int j = max(nB, j0); j < jw; ++j)
      val += fr_root<G, Q, YS, 2>(rs[j], cs[j], yreg, ycol, acc);
    if (low) {
      // the low roots' share of each partial, sum_k D_k U_k(y) (Clenshaw)
#pragma unroll
      for (int s = 0; s < Q; ++s) {
        const float y = YS ? ycol[s * G * Geo::LDR] : yreg[s], y2 = y + y;
        float b1 = 0.f, b2 = 0.f;
#pragma unroll
        for (int k = kSeriesK1 - 1; k >= 0; --k) {
          const float b0 = fmaf(y2, b1, sD[k * 32 + rr] - b2);
          b2 = b1;
          b1 = b0;
        }
        acc[s] += b1;
      }
      val += sD[kSeriesK1 * 32 + rr];
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
  if (fe_con && warp == 0 && r0 + lane < R) fe_con[(size_t)it.c * ldf + r0 + lane] = fe_s[lane];
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace

size_t fr_smem_bytes(int cfg) {
  switch (cfg) {
#define CLS_FR_SMEM(id, G, Q, C, Y) \
  case id: return fr_smem<G, Q>();
    CLS_FR_CONFIGS(CLS_FR_SMEM)
#undef CLS_FR_SMEM
    default: return 0;
  }
}

cudaError_t set_fr_attributes() {
  cudaError_t err = cudaSuccess;
#define CLS_FR_ATTR(id, G, Q, C, Y)                                                \
  if (err == cudaSuccess)                                                          \
    err = cudaFuncSetAttribute(k_fe_group_fr<G, Q, (Y != 0)>,                      \
                               cudaFuncAttributeMaxDynamicSharedMemorySize,        \
                               (int)fr_smem<G, Q>());
  CLS_FR_CONFIGS(CLS_FR_ATTR)
#undef CLS_FR_ATTR
  return err;
}

cudaError_t launch_group_fr(int cfg, const DevPlan& d, const int32_t* list, int count, int R,
                            int Rp, const float* x, float* P, float* fe_con, int ldf,
                            uint8_t* done, cudaStream_t s) {
  if (count == 0 || R == 0) return cudaSuccess;
  const dim3 grid(count, ceil_div(R, 32)), block(256);
  switch (cfg) {
#define CLS_FR_CASE(id, G, Q, C, Y)                                                       \
  case id:                                                                                \
    k_fe_group_fr<G, Q, (Y != 0)><<<grid, block, fr_smem<G, Q>(), s>>>(                   \
        list, d.fe, d.root_tab, d.zpow_tab, d.coef_tab, d.fe_lit, x, R, Rp, P, fe_con, ldf,  \
        done, d.ser_info, done ? ser_terms(d, done, ceil_div(R, 32)) : nullptr,           \
        d.dft_flops);                                                                     \
    break;
    CLS_FR_CONFIGS(CLS_FR_CASE)
#undef CLS_FR_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace cls
