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
#include <type_traits>

#include "kernels.cuh"

namespace cls {
namespace {

constexpr unsigned kFull = 0xffffffffu;
// The root cutoff (kernels.cuh, tail_roots) bounds the skipped tail terms by
// 2^-24 in total, the FP32 unit roundoff: they change FE and each partial by
// no more than one rounding of a term of modulus 1.

__device__ __forceinline__ float4 ldg4(const F4* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ int rec_row(int32_t dst) { return dst & 0x7fffffff; }
__device__ __forceinline__ float rec_sgn(int32_t dst) { return dst < 0 ? -1.0f : 1.0f; }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// The low roots' share of a low tile's partials: acc[s] += sum_k D_k U_k(y_s)
// by Clenshaw's recurrence, D_k = d[k * 32] (the Chebyshev pass's saved
// coefficients of this restart).  Slots go four at a time, two per packed
// FP32x2 instruction, each D_k read once per group of four.  yv(s) = y_s.
template <int S, typename YF>
__device__ __forceinline__ void clenshaw_low(const float* d, YF&& yv, float (&acc)[S]) {
  constexpr int C = 4;
#pragma unroll
  for (int s0 = 0; s0 < S; s0 += C) {
    constexpr int NP = C / 2;
    float2 y2[NP], b1[NP], b2[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const int sa = s0 + 2 * p, sb = sa + 1;
      const float ya = sa < S ? yv(sa) : 0.f, yb = sb < S ? yv(sb) : 0.f;
      y2[p] = make_float2(ya + ya, yb + yb);
      b1[p] = make_float2(0.f, 0.f);
      b2[p] = b1[p];
    }
#pragma unroll
    for (int k = kSeriesK1 - 1; k >= 0; --k) {
      const float dk = d[k * 32];
      const float2 dd = make_float2(dk, dk);
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        if (s0 + 2 * p < S) {
          const float2 b0 =
              __ffma2_rn(y2[p], b1[p], __fadd2_rn(dd, make_float2(-b2[p].x, -b2[p].y)));
          b2[p] = b1[p];
          b1[p] = b0;
        }
      }
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const int sa = s0 + 2 * p, sb = sa + 1;
      if (sa < S) acc[sa] += b1[p].x;
      if (sb < S) acc[sb] += b1[p].y;
    }
  }
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

// ---------------------------------------------------------------------------
// Packed interior slots.
//
// Along a run, projected steps put coordinates exactly on +-1, and a literal
// at a corner has the factor 1 (false, y = 1) or w^j (true, y = -1).  For a
// restart with t true corners
//     G_j = w^(j t) prod_{interior i} F_ij,
// a false corner's leave-one-out product is G_j and a true corner's
// w^(-j) G_j, so every corner literal of the restart shares one of two
// partials, Re sum_j c'_j G_j or Re sum_j c'_j w^(-j) G_j (the identity the
// corner passes use).  After staging, the kernel records per literal and
// restart a 2-bit code (true corner, interior); when the tile's largest
// interior count fits in qw <= QC slots per lane with qw at most half of Q,
// each restart's interior values are packed into the first slots of a
// second buffer and the root loop runs over G * qw slots instead of G * Q.
// In the later middle of a run, when the tiles that reach this kernel have
// more than half of their literals at corners, that cuts the root products
// per restart in proportion.  Same results up to FP32 rounding.
template <int G, int Q>
struct FrcLayout {
  static constexpr int LS = G * Q;                     // staged literal slots
  // packed slots per lane, at most: half of Q rounded down to an even count
  // (a tabulated slot count), at most 12
  static constexpr int QC = ((Q / 2) & ~1) < 12 ? ((Q / 2) & ~1) : 12;
  static constexpr int LC = G * QC;                    // packed slots per restart
  static constexpr int JC = FrCap<G, Q>::JC;
  static constexpr int NWD = (LS + 15) / 16;          // 2-bit code words per restart
  static constexpr int LDR = FrGeom<G>::LDR;
  // float4 tables rs, cs, gs [JC]; float2 ws [LS + 1] (w^q, q = 0..L, padded
  // to a float4 boundary); staging ys [LS][LDR] and packed yc [LC][LDR]
  // floats; codes and word bases [NWD][32] ints
  static constexpr int WS4 = (LS + 2) / 2;             // float4 units of ws
  static constexpr size_t bytes = (size_t)(3 * JC + WS4) * 16 + (size_t)(LS + LC) * LDR * 4 +
                                  (size_t)2 * NWD * 32 * 4;
};
// A tile is packed when its packed slots are at most kPackDen / kPackNum of
// the full ones: below that the per-tile work of the codes, the packing and
// the write-out (a few dozen integer operations per literal) and the corner
// factor of every root outweigh the shorter products (measured on the mixed
// workload's middle steps, where only a few dozen roots follow the
// power-sum pass's low ones).
constexpr int kPackNum = 2, kPackDen = 1;

// Configurations with the packed path: those the corner passes serve (32
// slots or more) with 14 <= Q <= 24 and at most 320 slots, where the packed
// buffers leave room for two blocks per SM.  Their full path already takes
// about 128 registers; with fewer slots the packed path's registers would
// lower the occupancy, and with the occupancy held (64 or 80 registers) the
// 8..12-slot configurations measured slower packed than full.
template <int G, int Q>
struct FrcFits {
  static constexpr bool value =
      G * Q >= kCornerMinSlots && FrcLayout<G, Q>::bytes <= 110 * 1024 && Q >= 14 &&
      Q <= 24 && G * Q <= 320;
};
template <int G, int Q>
constexpr size_t fr_dyn_smem() {
  return FrcFits<G, Q>::value ? FrcLayout<G, Q>::bytes : fr_smem<G, Q>();
}

// One root for one lane over its QW packed slots (values in registers): as
// fr_root, with the corner factor W = w^(j t) multiplied into the first
// factor of the group's lane 0, so that it enters G_j and every
// leave-one-out product exactly once (lane 0's prefixes carry it, the other
// lanes get it through O), and the two corner partials accumulated.
// rt = {t, z^QW}, cf = {b'_j, c'_j z^(QW-1)}, gc = {c'_j, c'_j w^-j}.
template <int G, int QW, int F>
__device__ __forceinline__ void frc_root(const float4 rt, const float4 cf, const float4 gc,
                                         const float2 W, const float (&y)[QW],
                                         float (&acc)[QW], float& val, float& gF, float& gT) {
  const float tk = rt.x;
  float pr[QW], pim[QW];
  float ur, ui;
  fr_uinit<F>(ur, ui, y[0], tk);
  float qr = W.x * ur - W.y * ui, qi = W.x * ui + W.y * ur;
#pragma unroll
  for (int s = 1; s < QW; ++s) {
    pr[s] = qr;
    pim[s] = qi;
    fr_umul<F>(qr, qi, y[s], tk);
  }
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
  val = fmaf(cf.x, Ptr, fmaf(-cf.y, Pti, val));
  gF = fmaf(gc.x, Ptr, fmaf(-gc.y, Pti, gF));
  gT = fmaf(gc.z, Ptr, fmaf(-gc.w, Pti, gT));
  float hr = cf.z * Or - cf.w * Oi, hi = cf.z * Oi + cf.w * Or;
#pragma unroll
  for (int s = QW - 1; s >= 1; --s) {
    acc[s] = fmaf(pr[s], hr, acc[s]);
    acc[s] = fmaf(-pim[s], hi, acc[s]);
    fr_umul<F>(hr, hi, y[s], tk);
  }
  // slot 0: the suffix times W (lane 0's W sits in its prefixes only)
  acc[0] = fmaf(W.x, hr, fmaf(-W.y, hi, acc[0]));
}

// Two roots at once (j and j + 1, same factored form): the same arithmetic
// as two frc_root calls, written as two independent chains so that their
// forward products and butterflies overlap.
template <int G, int QW, int F>
__device__ __forceinline__ void frc_root2(const float4 rtA, const float4 cfA, const float4 gcA,
                                          const float2 WA, const float4 rtB, const float4 cfB,
                                          const float4 gcB, const float2 WB,
                                          const float (&y)[QW], float (&acc)[QW], float& val,
                                          float& gF, float& gT) {
  const float ta = rtA.x, tb = rtB.x;
  float pra[QW], pia[QW], prb[QW], pib[QW];
  float ur, ui, vr, vi;
  fr_uinit<F>(ur, ui, y[0], ta);
  fr_uinit<F>(vr, vi, y[0], tb);
  float qar = WA.x * ur - WA.y * ui, qai = WA.x * ui + WA.y * ur;
  float qbr = WB.x * vr - WB.y * vi, qbi = WB.x * vi + WB.y * vr;
#pragma unroll
  for (int s = 1; s < QW; ++s) {
    pra[s] = qar;
    pia[s] = qai;
    prb[s] = qbr;
    pib[s] = qbi;
    fr_umul<F>(qar, qai, y[s], ta);
    fr_umul<F>(qbr, qbi, y[s], tb);
  }
  float Par = qar * rtA.y - qai * rtA.z, Pai = qar * rtA.z + qai * rtA.y;
  float Pbr = qbr * rtB.y - qbi * rtB.z, Pbi = qbr * rtB.z + qbi * rtB.y;
  float Oar = 1.f, Oai = 0.f, Obr = 1.f, Obi = 0.f;
#pragma unroll
  for (int d = 1; d < G; d <<= 1) {
    const float tar = __shfl_xor_sync(kFull, Par, d);
    const float tai = __shfl_xor_sync(kFull, Pai, d);
    const float tbr = __shfl_xor_sync(kFull, Pbr, d);
    const float tbi = __shfl_xor_sync(kFull, Pbi, d);
    if (d == 1) {
      Oar = tar;
      Oai = tai;
      Obr = tbr;
      Obi = tbi;
    } else {
      const float a = Oar * tar - Oai * tai, b = Oar * tai + Oai * tar;
      Oar = a;
      Oai = b;
      const float c = Obr * tbr - Obi * tbi, e = Obr * tbi + Obi * tbr;
      Obr = c;
      Obi = e;
    }
    const float a = Par * tar - Pai * tai, b = Par * tai + Pai * tar;
    Par = a;
    Pai = b;
    const float c = Pbr * tbr - Pbi * tbi, e = Pbr * tbi + Pbi * tbr;
    Pbr = c;
    Pbi = e;
  }
  val = fmaf(cfA.x, Par, fmaf(-cfA.y, Pai, val));
  val = fmaf(cfB.x, Pbr, fmaf(-cfB.y, Pbi, val));
  gF = fmaf(gcA.x, Par, fmaf(-gcA.y, Pai, gF));
  gF = fmaf(gcB.x, Pbr, fmaf(-gcB.y, Pbi, gF));
  gT = fmaf(gcA.z, Par, fmaf(-gcA.w, Pai, gT));
  gT = fmaf(gcB.z, Pbr, fmaf(-gcB.w, Pbi, gT));
  float har = cfA.z * Oar - cfA.w * Oai, hai = cfA.z * Oai + cfA.w * Oar;
  float hbr = cfB.z * Obr - cfB.w * Obi, hbi = cfB.z * Obi + cfB.w * Obr;
#pragma unroll
  for (int s = QW - 1; s >= 1; --s) {
    acc[s] = fmaf(pra[s], har, acc[s]);
    acc[s] = fmaf(-pia[s], hai, acc[s]);
    acc[s] = fmaf(prb[s], hbr, acc[s]);
    acc[s] = fmaf(-pib[s], hbi, acc[s]);
    fr_umul<F>(har, hai, y[s], ta);
    fr_umul<F>(hbr, hbi, y[s], tb);
  }
  acc[0] = fmaf(WA.x, har, fmaf(-WA.y, hai, acc[0]));
  acc[0] = fmaf(WB.x, hbr, fmaf(-WB.y, hbi, acc[0]));
}

// The packed tile, after staging (ys) and the codes: packs, evaluates over
// QW slots per lane and writes the partials of every literal.
// Block-uniform; ends with the partials written.
template <int G, int Q, int QW>
__device__ __forceinline__ void frc_tile(
    const FeItem& it, int j0, bool low, const F4* __restrict__ root,
    const F4* __restrict__ zpow, const F4* __restrict__ coef, const LitRec* lrec_s,
    const float* sD, float4* rs, float4* cs, float4* gs, float2* ws, const float* ys, float* yc,
    const uint32_t* codes, const int32_t* wbase, const int* q_s, const int* t_s, float* fe_s,
    float* gF_s, float* gT_s, int R, int Rp, int r0, float* __restrict__ P,
    float* __restrict__ fe_con, int ldf, unsigned long long* __restrict__ flops) {
  using Geo = FrGeom<G>;
  constexpr int LDR = Geo::LDR;
  static_assert(QW <= FrcLayout<G, Q>::QC, "packed slots beyond the packed buffer");
  const int L = it.L, J = it.J, N = L + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwd = (L + 15) >> 4;
  // pack each restart's interior values; pad its slots up to G * QW with 1
  for (int wd = warp; wd < nwd; wd += 8) {
    const uint32_t code = codes[wd * 32 + lane];
    int k = wbase[wd * 32 + lane];
#pragma unroll
    for (int u = 0; u < 16; ++u)
      if ((code >> (2 * u)) & 2u) yc[(k++) * LDR + lane] = ys[(wd * 16 + u) * LDR + lane];
  }
  for (int k = q_s[lane] + warp; k < G * QW; k += 8) yc[k * LDR + lane] = 1.0f;
  // per-root constants for QW slots; w^q for the corner factor
  for (int j = threadIdx.x; j < J; j += 256) {
    const float4 rt = ldg4(&root[it.root_off + j]);
    const float4 zp = ldg4(&zpow[(size_t)(it.root_off + j) * kNumFrQ + FrQIndex<QW>::value]);
    const float4 cf = ldg4(&coef[it.coef_off + j]);
    const float2 cz = cmul(make_float2(cf.z, cf.w), make_float2(zp.z, zp.w));
    const float wr = 1.f - 2.f * rt.y, wi = 2.f * rt.z;       // w^(j+1)
    const float2 cw = cmul(make_float2(cf.z, cf.w), make_float2(wr, -wi));
    rs[j] = make_float4(rt.w, zp.x, zp.y, 0.f);
    cs[j] = make_float4(cf.x, cf.y, cz.x, cz.y);
    gs[j] = make_float4(cf.z, cf.w, cw.x, cw.y);
    ws[j + 1] = make_float2(wr, wi);
    if (j + 1 < N - (j + 1)) ws[N - (j + 1)] = make_float2(wr, -wi);   // w^(N-q) = conj w^q
  }
  if (threadIdx.x == 0) ws[0] = make_float2(1.f, 0.f);
  __syncthreads();

  const int lam = lane % G;
  const int gi = lane / G;
  const int nA = fr_roots_form0(L), nB = fr_roots_form01(L);
  const float tailT = logf(2.f * (float)J) + kTailLogInvEps;
#pragma unroll 1
  for (int pass = 0; pass < Geo::PASSES; ++pass) {
    const int rr = pass * Geo::GPB + warp * Geo::GPW + gi;
    const float* ycol = yc + lam * LDR + rr;
    float y[QW], acc[QW];
#pragma unroll
    for (int s = 0; s < QW; ++s) {
      y[s] = ycol[s * G * LDR];
      acc[s] = 0.f;
    }
    // tail cutoff over the interior slots (corners and padding add nothing)
    TailSums ts;
#pragma unroll
    for (int s = 0; s < QW; ++s) ts.add(y[s]);
    ts.group_reduce(G);
    const int jc = tail_roots(ts, L, J, tailT);
    const int jw = __reduce_max_sync(kFull, jc);
    const int qn = q_s[rr], tn = t_s[rr];
    if (flops) {
      // 14 / 16 flops per (interior literal, root) in the two factored
      // forms for the roots each restart needs (counted once per group)
      const int jl = min(jc, j0);
      const unsigned f = lam == 0 ? (unsigned)qn * (14u * (min(nB, jc) - min(nB, jl)) +
                                                    16u * (max(0, jc - nB) - max(0, jl - nB)) +
                                                    (low ? 4u * kSeriesK1 : 0u))
                                  : 0u;
      const unsigned tot = __reduce_add_sync(kFull, f);
      if (lane == 0) atomicAdd(flops, (unsigned long long)tot);
    }
    // root number (j + 1) times t, mod N, indexes w^((j+1) t); only the
    // group's lane 0 carries the corner factor
    const int dq = tn % N;
    int qq = (int)(((int64_t)(j0 + 1) * tn) % N);
    const bool lam0 = lam == 0;
    auto Wnext = [&]() -> float2 {
      const float2 w = ws[qq];
      qq += dq;
      qq -= qq >= N ? N : 0;
      return lam0 ? w : make_float2(1.f, 0.f);
    };
    float val = 0.f, gF = 0.f, gT = 0.f;
    // the roots of one factored form in pairs, then the odd one
    auto run = [&](auto form, int ja, int jb) {
      constexpr int F = decltype(form)::value;
      int j = ja;
#pragma unroll 1
      for (; j + 1 < jb; j += 2) {
        const float2 WA = Wnext(), WB = Wnext();
        frc_root2<G, QW, F>(rs[j], cs[j], gs[j], WA, rs[j + 1], cs[j + 1], gs[j + 1], WB, y,
                            acc, val, gF, gT);
      }
      if (j < jb) frc_root<G, QW, F>(rs[j], cs[j], gs[j], Wnext(), y, acc, val, gF, gT);
    };
    run(std::integral_constant<int, 0>(), j0, min(nA, jw));
    run(std::integral_constant<int, 1>(), max(nA, j0), min(nB, jw));
    run(std::integral_constant<int, 2>(), max(nB, j0), jw);
    if (low) {
      // the low roots' share, sum_k D_k U_k(y) (Clenshaw) for the interior
      // slots; U_k(1) = k + 1 and U_k(-1) = (-1)^k (k + 1) for the corners
      clenshaw_low<QW>(sD + rr, [&](int s) { return y[s]; }, acc);
#pragma unroll
      for (int k = 0; k < kSeriesK1; ++k) {
        const float dk = sD[k * 32 + rr] * (float)(k + 1);
        gF += dk;
        gT += (k & 1) ? -dk : dk;
      }
      val += sD[kSeriesK1 * 32 + rr];
    }
    // interior partials back into the packed slots (each owned by one lane)
#pragma unroll
    for (int s = 0; s < QW; ++s) {
      const int k = lam + G * s;
      if (k < qn) yc[k * LDR + rr] = acc[s];
    }
    if (lam == 0) {
      fe_s[rr] = it.b0 + val;
      gF_s[rr] = gF;
      gT_s[rr] = gT;
    }
  }
  __syncthreads();
  // partials w * s_e * dFE/dy_e of every literal to their variable-major rows
  const int r = r0 + lane;
  const float gFw = it.w * gF_s[lane], gTw = it.w * gT_s[lane];
#pragma unroll 4
  for (int i = warp; i < L; i += 8) {
    const LitRec rc = lrec_s[i];
    const int wd = i >> 4, u = i & 15;
    const uint32_t code = codes[wd * 32 + lane];
    const uint32_t c2 = (code >> (2 * u)) & 3u;
    float v;
    if (c2 & 2u) {
      const int k = wbase[wd * 32 + lane] + __popc(code & 0xAAAAAAAAu & ((1u << (2 * u)) - 1u));
      v = it.w * yc[k * LDR + lane];
    } else {
      v = (c2 & 1u) ? gTw : gFw;
    }
    if (r < R) st_partial(&P[(size_t)rec_row(rc.dst) * Rp + r], rec_sgn(rc.dst) * v);
  }
  if (fe_con && warp == 0 && r < R) fe_con[(size_t)it.c * ldf + r] = fe_s[lane];
}

// Blocks per SM the packed configurations keep (that of their full path).
template <int G, int Q>
struct FrMinBlocks {
  static constexpr int value = FrcFits<G, Q>::value ? 2 : 0;
};

template <int G, int Q, bool YS>
__global__ void __launch_bounds__(256, FrMinBlocks<G, Q>::value) k_fe_group_fr(
    const int32_t* __restrict__ list, const FeItem* __restrict__ fe,
    const F4* __restrict__ root, const F4* __restrict__ zpow, const F4* __restrict__ coef,
    const LitRec* __restrict__ lit,
    const float* __restrict__ x, int R, int Rp, float* __restrict__ P,
    float* __restrict__ fe_con, int ldf, const uint8_t* __restrict__ done,
    const SerInfo* __restrict__ ser_info, const float* __restrict__ ser_d,
    unsigned long long* __restrict__ flops) {
  using Geo = FrGeom<G>;
  using Lay = FrcLayout<G, Q>;
  constexpr int LS = G * Q;
  constexpr int JC = FrCap<G, Q>::JC;
  constexpr bool CP = FrcFits<G, Q>::value;
  extern __shared__ float4 smem4[];
  float4* rs = smem4;                                        // [JC]
  float4* cs = smem4 + JC;                                   // [JC]
  // the packed path's tables sit between cs and the staging buffer
  float4* gs = smem4 + 2 * JC;                               // [JC]      (CP)
  float2* ws = reinterpret_cast<float2*>(smem4 + 3 * JC);    // [J + 1]   (CP)
  float* ys = reinterpret_cast<float*>(smem4 + (CP ? 3 * JC + Lay::WS4 : 2 * JC));  // [LS][LDR]
  float* yc = ys + LS * Geo::LDR;                                         // [LC][LDR] (CP)
  uint32_t* codes = reinterpret_cast<uint32_t*>(yc + Lay::LC * Geo::LDR); // [NWD][32] (CP)
  int32_t* wbase = reinterpret_cast<int32_t*>(codes + Lay::NWD * 32);     // [NWD][32] (CP)
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

  if constexpr (!CP) {
    // per-root constants for this Q
    for (int j = threadIdx.x; j < J; j += 256) {
      const float4 rt = ldg4(&root[it.root_off + j]);
      const float4 zp = ldg4(&zpow[(size_t)(it.root_off + j) * kNumFrQ + FrQIndex<Q>::value]);
      const float4 cf = ldg4(&coef[it.coef_off + j]);
      const float2 cz = cmul(make_float2(cf.z, cf.w), make_float2(zp.z, zp.w));
      rs[j] = make_float4(rt.w, zp.x, zp.y, 0.f);
      cs[j] = make_float4(cf.x, cf.y, cz.x, cz.y);
    }
  }
  // the constraint's literal records once per block (one coalesced read),
  // then the literal values y = s * x (coalesced rows of 32 restarts)
  __shared__ LitRec lrec_s[LS];
  for (int i = threadIdx.x; i < L; i += 256) lrec_s[i] = lit[it.lit0 + i];
  if (low) {
    const float* sdg = ser_d + (size_t)ser_info[ci].slot * (kSeriesK1 + 1) * Rp + r0;
    for (int e = threadIdx.x; e < (kSeriesK1 + 1) * 32; e += 256)
      sD[e] = (r0 + (e & 31) < R) ? sdg[(size_t)(e >> 5) * Rp + (e & 31)] : 0.f;
  }
  __syncthreads();
  // rows of x go to shared memory as asynchronous 4-byte copies (all of a
  // thread's rows in flight at once); the signs are applied afterwards.
  // With the packed path, warp w stages the 16-literal words w, w + 8, ...
  // and, reading back only its own copies, applies the signs and records per
  // literal and restart a 2-bit code (bit 0 true corner, bit 1 interior).
  bool packed_try = false;
  if constexpr (CP) packed_try = done != nullptr;
  {
    const int r = r0 + lane;
    if (packed_try) {
      constexpr int NWA = (LS + 15) / 16;
      for (int wd = warp; wd < NWA; wd += 8)
#pragma unroll 4
        for (int u = 0; u < 16; ++u) {
          const int i = wd * 16 + u;
          if (i >= LS) break;
          float* dst = &ys[i * Geo::LDR + lane];
          if (i < L && r < R) cp_async4(dst, &x[(size_t)lrec_s[i].var * R + r]);
          else *dst = 1.0f;
        }
      cp_async_commit();
      cp_async_wait<0>();
      const int nwd = (L + 15) >> 4;
      for (int wd = warp; wd < nwd; wd += 8) {
        uint32_t code = 0;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int i = wd * 16 + u;
          if (i < L) {
            float y = ys[i * Geo::LDR + lane];
            if (r < R && lrec_s[i].dst < 0) {
              y = -y;
              ys[i * Geo::LDR + lane] = y;
            }
            code |= (y == -1.f ? 1u : 0u) << (2 * u);
            code |= (fabsf(y) != 1.f ? 2u : 0u) << (2 * u);
          }
        }
        codes[wd * 32 + lane] = code;
      }
    } else {
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
  }
  __syncthreads();

  if constexpr (CP) {
    // per restart the interior count q and the true-corner count t; pack
    // when the tile's largest q fits in qw <= QC slots per lane with
    // kPackNum qw <= kPackDen Q
    __shared__ int q_s[32], t_s[32], qw_s;
    __shared__ float gF_s[32], gT_s[32];
    if (packed_try) {
      const int nwd = (L + 15) >> 4;
      if (warp == 0) {
        int run = 0, tt = 0;
        for (int wd = 0; wd < nwd; ++wd) {
          const uint32_t code = codes[wd * 32 + lane];
          wbase[wd * 32 + lane] = run;
          run += __popc(code & 0xAAAAAAAAu);
          tt += __popc(code & 0x55555555u);
        }
        q_s[lane] = run;
        t_s[lane] = tt;
        const int qmax = __reduce_max_sync(kFull, run);
        if (lane == 0) {
          // packed slots per lane: 4, 6, 8, 10 or 12 (the smallest that
          // holds the tile's largest interior count), if it halves the slots
          const int need = max(4, (qmax + G - 1) / G + ((qmax + G - 1) / G & 1));
          qw_s = (need <= Lay::QC && kPackNum * need <= kPackDen * Q) ? need : 0;
        }
      }
      __syncthreads();
      const int qw = qw_s;
      if (qw > 0) {
#define CLS_FRC_TILE(QW)                                                                     \
  frc_tile<G, Q, (QW <= Lay::QC ? QW : Lay::QC)>(it, j0, low, root, zpow, coef, lrec_s, sD, rs, \
                                                 cs, gs, ws, ys, yc, codes, wbase, q_s, t_s,  \
                                                 fe_s, gF_s, gT_s, R, Rp, r0, P, fe_con, ldf, \
                                                 flops)
        if (qw <= 4 || Lay::QC < 6) CLS_FRC_TILE(4);
        else if (qw <= 6 || Lay::QC < 8) CLS_FRC_TILE(6);
        else if (qw <= 8) CLS_FRC_TILE(8);
        else if (qw <= 10) CLS_FRC_TILE(10);
        else CLS_FRC_TILE(12);
#undef CLS_FRC_TILE
        return;
      }
    }
  }

  if constexpr (CP) {
    // per-root constants for this Q (the packed path fills its own)
    for (int j = threadIdx.x; j < J; j += 256) {
      const float4 rt = ldg4(&root[it.root_off + j]);
      const float4 zp = ldg4(&zpow[(size_t)(it.root_off + j) * kNumFrQ + FrQIndex<Q>::value]);
      const float4 cf = ldg4(&coef[it.coef_off + j]);
      const float2 cz = cmul(make_float2(cf.z, cf.w), make_float2(zp.z, zp.w));
      rs[j] = make_float4(rt.w, zp.x, zp.y, 0.f);
      cs[j] = make_float4(cf.x, cf.y, cz.x, cz.y);
    }
    __syncthreads();
  }

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
    // Tail cutoff (kernels.cuh, tail_roots): the roots whose products over
    // all or all-but-one factors are provably below 2^-24 / (2J) are
    // skipped.  The warp runs to the largest cutoff of its groups (extra
    // roots are exact terms).
    TailSums ts;
#pragma unroll
    for (int s = 0; s < Q; ++s) ts.add(YS ? ycol[s * G * Geo::LDR] : yreg[s]);
    ts.group_reduce(G);
    const int jc = tail_roots(ts, L, J, tailT);
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
      clenshaw_low<Q>(sD + rr, [&](int s) { return YS ? ycol[s * G * Geo::LDR] : yreg[s]; },
                      acc);
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
  case id: return fr_dyn_smem<G, Q>();
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
                               (int)fr_dyn_smem<G, Q>());
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
    k_fe_group_fr<G, Q, (Y != 0)><<<grid, block, fr_dyn_smem<G, Q>(), s>>>(               \
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
