// kernels_corner.cu -- the corner pass of the factored DFT path.
//
// Projected gradient steps pin coordinates to the faces of the cube: after a
// few dozen steps almost every x_v is exactly +-1.  A literal at a corner has
// alpha, beta in {0, 1}, so its Poisson-binomial factor is 1 (false literal,
// y = 1) or w^j (true literal, y = -1), and for a restart with t true-corner
// literals
//     G_j = w^(j t) * prod_{non-corner i} F_ij,
//     prod_{l != i} F_lj = G_j            (i a false corner)
//                        = w^(-j) G_j     (i a true corner)
//                        = w^(j t) prod_{non-corner l != i} F_lj  (otherwise).
// Every corner literal of a restart therefore shares one of two partials,
// and the products run over the few non-corner literals only.
//
// One thread per (constraint, restart), a warp per tile of 32 restarts, a
// block per constraint and 8 tiles.  Pass 1 reads the restart's literal
// values (eight loads in flight), counts the true corners, collects the
// non-corner values (at most kCornerQS; a warp that finds more in any lane
// gives the tile to the dense kernel by clearing its flag) and keeps the
// tile's classification of every literal as two ballots in shared memory.
// Pass 2, decided per warp from the largest interior count q: q <= 8, an
// exact small Poisson-binomial DP over the interior literals that keeps its
// prefix distributions (corner_dp); q <= 16 (and q <= 32 in the 4-lane
// pass), the same DP without them, each literal's factor divided back out of
// the distribution in the stable direction (corner_dpx), where that costs
// less than the roots; otherwise every root over 16 slots (padding y = 1,
// exactly neutral in the factored form, as in kernels_fr.cu), with w^(j t)
// read from the root table.  Pass 3 writes the partials of all literals and
// sets the tile's flag, which tells the dense factored kernel launched next
// on the stream to skip the tile.  Exact up to FP32 rounding.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "kernels.cuh"

namespace cls {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kCornerQS = 16;   // non-corner slots per lane
constexpr int kCornerGroup = 4; // lanes per restart in the second pass
constexpr int kCornerDpx = 32;  // interior literals of the second pass's root-free DP
constexpr int kCornerChebMin = 24; // fewest low roots worth the 4-lane pass's Chebyshev sums

__device__ __forceinline__ float4 ldg4(const F4* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ int rec_row(int32_t dst) { return dst & 0x7fffffff; }
__device__ __forceinline__ float rec_sgn(int32_t dst) { return dst < 0 ? -1.0f : 1.0f; }
// v * rec_sgn(dst) as one sign-bit flip
__device__ __forceinline__ float apply_sgn(float v, int32_t dst) {
  return __int_as_float(__float_as_int(v) ^ (dst & (int32_t)0x80000000));
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// index of the 16-slot root powers in kFrQ
constexpr int kCornerZq = 8;

// One root for one restart: u-products over the QS non-corner slots (form F
// of the factored roots, kernels.cuh), scaled by z^QS; G_j = W times that.
// Adds Re(b' G_j) to fe, Re(c' G_j) to gF, Re(c' w^-j G_j) to gT and the
// non-corner partials Re(c' W z^(QS-1) prod_{s' != s} u_s') to acc.
// rt = {A, B, C, t} (w^j = (1 - 2B) + i 2C), zp = {z^QS, z^(QS-1)},
// cf = {b', c'}.
template <int QS, int F>
__device__ __forceinline__ void corner_root(const float4 rt, const float4 zp, const float4 cf,
                                            const float2 W, const float (&y)[QS],
                                            float (&acc)[QS], float& fe, float& gF, float& gT) {
  const float tk = rt.w;
  float pr[QS], pim[QS];
  float qr, qi;
  fr_uinit<F>(qr, qi, y[0], tk);
#pragma unroll
  for (int s = 1; s < QS; ++s) {
    pr[s] = qr;
    pim[s] = qi;
    fr_umul<F>(qr, qi, y[s], tk);
  }
  const float2 Gj = cmul(W, cmul(make_float2(qr, qi), make_float2(zp.x, zp.y)));
  fe = fmaf(cf.x, Gj.x, fmaf(-cf.y, Gj.y, fe));
  gF = fmaf(cf.z, Gj.x, fmaf(-cf.w, Gj.y, gF));
  const float2 cw = cmul(make_float2(cf.z, cf.w), make_float2(1.f - 2.f * rt.y, -2.f * rt.z));
  gT = fmaf(cw.x, Gj.x, fmaf(-cw.y, Gj.y, gT));
  const float2 h0 = cmul(cmul(make_float2(cf.z, cf.w), make_float2(zp.z, zp.w)), W);
  float hr = h0.x, hi = h0.y;
#pragma unroll
  for (int s = QS - 1; s >= 1; --s) {
    acc[s] = fmaf(pr[s], hr, acc[s]);
    acc[s] = fmaf(-pim[s], hi, acc[s]);
    fr_umul<F>(hr, hi, y[s], tk);
  }
  acc[0] += hr;
}

// Pass 2 for one restart: all roots; the non-corner partials go back into the
// restart's slots of ncy (slot s at my[s * 32]).
template <int QS>
__device__ __forceinline__ void corner_roots(int L, int J, int nnc, int t, const float4* rtab,
                                             const float4* ctab, const float4* ztab, float* my,
                                             float& fe, float& gF, float& gT) {
  const int N = L + 1, nA = fr_roots_form0(L), nB = fr_roots_form01(L);
  float y[QS], acc[QS];
#pragma unroll
  for (int s = 0; s < QS; ++s) {
    y[s] = s < nnc ? my[s * 32] : 1.f;
    acc[s] = 0.f;
  }
  fe = gF = gT = 0.f;
  const int dq = t % N;
  int q = dq;                               // (root number) * t mod N, root 1 first
#pragma unroll 1
  for (int j = 0; j < J; ++j) {
    float2 W = make_float2(1.f, 0.f);
    if (q != 0) {
      const bool low = q <= J;
      const float4 e = rtab[(low ? q : N - q) - 1];
      W = make_float2(1.f - 2.f * e.y, low ? 2.f * e.z : -2.f * e.z);
    }
    const float4 rt = rtab[j], cf = ctab[j], zp = ztab[j];
    if (j < nA) corner_root<QS, 0>(rt, zp, cf, W, y, acc, fe, gF, gT);
    else if (j < nB) corner_root<QS, 1>(rt, zp, cf, W, y, acc, fe, gF, gT);
    else corner_root<QS, 2>(rt, zp, cf, W, y, acc, fe, gF, gT);
    q += dq;
    if (q >= N) q -= N;
  }
#pragma unroll
  for (int s = 0; s < QS; ++s) my[s * 32] = acc[s];
}

// Pass 2 without roots, for at most QS <= 8 interior literals: with t true
// corners T = t + T_int, and the restart's FE and partials are expectations
// over the small Poisson-binomial distribution of the interior literals,
//   FE = E[sp_T],  dFE/dy_i = E[d_{T_{-i}}],  d_s = (sp_s - sp_{s+1}) / 2,
// a false corner's T_{-i} = t + T_int, a true corner's t - 1 + T_int.  The
// prefix distributions are kept and an adjoint sweep gives the interior
// partials (no division); padding slots are literals false with
// probability 1.  Exact up to FP32 rounding of nonnegative terms.
template <int QS>
__device__ __forceinline__ void corner_dp(int L, int t, const int8_t* __restrict__ sp,
                                          float* my, int nnc, float& fe, float& gF, float& gT) {
  float al[QS], be[QS];
#pragma unroll
  for (int s = 0; s < QS; ++s) {
    const float y = s < nnc ? my[s * 32] : 1.f;
    al[s] = fmaf(0.5f, y, 0.5f);
    be[s] = fmaf(-0.5f, y, 0.5f);
  }
  // spectrum values sp_{t-1 .. t+QS+1} (gF reads d_{t+QS}); outside 0..L
  // they never meet a nonzero probability except through d, which is 0 there
  float sv[QS + 3];
  bool ok[QS + 3];
#pragma unroll
  for (int a = 0; a < QS + 3; ++a) {
    const int idx = t - 1 + a;
    ok[a] = idx >= 0 && idx <= L;
    sv[a] = ok[a] ? (float)sp[idx] : 0.f;
  }
  auto dv = [&](int a) -> float {       // d_{t - 1 + a}
    return (ok[a] && ok[a + 1]) ? 0.5f * (sv[a] - sv[a + 1]) : 0.f;
  };
  // forward: pre[k] = distribution of interior literals 0..k-1 (support 0..k)
  float pre[QS][QS], cur[QS + 1];
  cur[0] = 1.f;
#pragma unroll
  for (int a = 1; a <= QS; ++a) cur[a] = 0.f;
#pragma unroll
  for (int k = 0; k < QS; ++k) {
#pragma unroll
    for (int a = 0; a <= k; ++a) pre[k][a] = cur[a];
#pragma unroll
    for (int a = k + 1; a >= 1; --a) cur[a] = fmaf(be[k], cur[a - 1], al[k] * cur[a]);
    cur[0] *= al[k];
  }
  fe = 0.f;
  gF = 0.f;
  gT = 0.f;
#pragma unroll
  for (int a = 0; a <= QS; ++a) {
    fe = fmaf(sv[a + 1], cur[a], fe);
    gF = fmaf(dv(a + 1), cur[a], gF);
    gT = fmaf(dv(a), cur[a], gT);
  }
  // adjoint: D(a) = E[d_{t + a + T_{k..}}], starting after the last literal
  float D[QS];
#pragma unroll
  for (int a = 0; a < QS; ++a) D[a] = dv(a + 1);
#pragma unroll
  for (int k = QS - 1; k >= 0; --k) {
    float g = 0.f;
#pragma unroll
    for (int a = 0; a <= k; ++a) g = fmaf(pre[k][a], D[a], g);
    my[k * 32] = g;                     // the interior partial of slot k
#pragma unroll
    for (int a = 0; a < k; ++a) D[a] = fmaf(be[k], D[a + 1], al[k] * D[a]);
  }
}

// Pass 2 without roots for up to NI interior literals, without keeping the
// prefix distributions: P = the distribution of T_int over all interior
// slots (padding literals are false with probability 1, so P vanishes above
// nnc), FE and the corner partials as in corner_dp, and the leave-one-out
// distribution of slot k by dividing its factor (alpha + beta z) back out of
// P.  The division runs upwards, x_a = (P_a - beta x_{a-1}) / alpha, when
// alpha >= beta, and downwards from the top, x_{a-1} = (P_a - alpha x_a) /
// beta, otherwise: the ratio that multiplies a carried error is then at most
// 1, so rounding errors add up over the NI cells instead of growing.  Both
// start exactly (x_{-1} = 0, x_NI = 0).  qmax = the warp's largest nnc.
template <int NI>
__device__ __forceinline__ void corner_dpx(int L, int t, int qmax, const int8_t* __restrict__ sp,
                                           float* my, int nnc, float& fe, float& gF, float& gT) {
  float P[NI + 1];
  P[0] = 1.f;
#pragma unroll
  for (int a = 1; a <= NI; ++a) P[a] = 0.f;
#pragma unroll
  for (int k = 0; k < NI; ++k) {
    if (k >= qmax) break;
    const float y = k < nnc ? my[k * 32] : 1.f;
    const float al = fmaf(0.5f, y, 0.5f), be = fmaf(-0.5f, y, 0.5f);
#pragma unroll
    for (int a = k + 1; a >= 1; --a) P[a] = fmaf(be, P[a - 1], al * P[a]);
    P[0] *= al;
  }
  // D[a] = d_{t-1+a}, a = 0..NI+1 (0 where the index leaves 0..L-1)
  float D[NI + 2];
  {
    float sprev = t >= 1 ? (float)sp[t - 1] : 0.f;
#pragma unroll
    for (int a = 0; a <= NI + 1; ++a) {
      const int i = t + a;                     // index of the upper spectrum value
      const float snext = i <= L ? (float)sp[i] : 0.f;
      D[a] = (i >= 1 && i <= L) ? 0.5f * (sprev - snext) : 0.f;
      sprev = snext;
    }
  }
  fe = 0.f;
  gF = 0.f;
  gT = 0.f;
#pragma unroll
  for (int a = 0; a <= NI; ++a) {
    const int i = t + a;
    fe = fmaf(i <= L ? (float)sp[i] : 0.f, P[a], fe);
    gF = fmaf(D[a + 1], P[a], gF);
    gT = fmaf(D[a], P[a], gT);
  }
#pragma unroll 1
  for (int k = 0; k < qmax; ++k) {
    const float y = k < nnc ? my[k * 32] : 1.f;
    const float al = fmaf(0.5f, y, 0.5f), be = fmaf(-0.5f, y, 0.5f);
    float g = 0.f;
    if (al >= be) {
      const float ia = 1.f / al, r = -be * ia;
      float xv = 0.f;
#pragma unroll
      for (int a = 0; a < NI; ++a) {
        xv = fmaf(r, xv, P[a] * ia);           // x_a
        g = fmaf(D[a + 1], xv, g);
      }
    } else {
      const float ib = 1.f / be, r = -al * ib;
      float xv = 0.f;
#pragma unroll
      for (int a = NI; a >= 1; --a) {
        xv = fmaf(r, xv, P[a] * ib);           // x_{a-1}
        g = fmaf(D[a], xv, g);
      }
    }
    if (k < nnc) my[k * 32] = g;
  }
}

// Whether the root-free pass costs less than the roots: about NI (NI + 1) * 7
// operations per restart against J roots over the pass's slots at 8 each.
__device__ __forceinline__ bool dp_pays(int J, int ni, int slots) {
  return ni * (ni + 1) * 7 <= J * slots * 8;
}

// One root for a group of G lanes sharing a restart (lane lam holds the
// restart's non-corner slots lam, lam + G, ...; QS per lane): u-products,
// z^QS scaling, butterfly over the G lanes for the total and the other
// lanes' product O, then as corner_root with W = w^(j t).  czq = c' z^(QS-1).
template <int G, int QS, int F>
__device__ __forceinline__ void group_root(const float4 rt, const float4 zp, const float4 cf,
                                           const float2 W, const float (&y)[QS],
                                           float (&acc)[QS], float& fe, float& gF, float& gT) {
  const float tk = rt.w;
  float pr[QS], pim[QS];
  float qr, qi;
  fr_uinit<F>(qr, qi, y[0], tk);
#pragma unroll
  for (int s = 1; s < QS; ++s) {
    pr[s] = qr;
    pim[s] = qi;
    fr_umul<F>(qr, qi, y[s], tk);
  }
  float2 Pt = cmul(make_float2(qr, qi), make_float2(zp.x, zp.y));
  float2 O = make_float2(1.f, 0.f);
#pragma unroll
  for (int d = 1; d < G; d <<= 1) {
    const float2 o = make_float2(__shfl_xor_sync(kFull, Pt.x, d), __shfl_xor_sync(kFull, Pt.y, d));
    O = (d == 1) ? o : cmul(O, o);
    Pt = cmul(Pt, o);
  }
  const float2 Gj = cmul(W, Pt);
  fe = fmaf(cf.x, Gj.x, fmaf(-cf.y, Gj.y, fe));
  gF = fmaf(cf.z, Gj.x, fmaf(-cf.w, Gj.y, gF));
  const float2 cw = cmul(make_float2(cf.z, cf.w), make_float2(1.f - 2.f * rt.y, -2.f * rt.z));
  gT = fmaf(cw.x, Gj.x, fmaf(-cw.y, Gj.y, gT));
  const float2 h0 = cmul(cmul(cmul(make_float2(cf.z, cf.w), make_float2(zp.z, zp.w)), W), O);
  float hr = h0.x, hi = h0.y;
#pragma unroll
  for (int s = QS - 1; s >= 1; --s) {
    acc[s] = fmaf(pr[s], hr, acc[s]);
    acc[s] = fmaf(-pim[s], hi, acc[s]);
    fr_umul<F>(hr, hi, y[s], tk);
  }
  acc[0] += hr;
}

// The low roots 1..jlo of one restart by Chebyshev sums over its interior
// slots (the expansions of kernels_series.cu; corner literals exact: log 1
// and i theta_j), spread over the restart's G lanes: each lane sums its own
// slots and evaluates the roots j = lam, lam + G, ...; butterflies combine
// the sums, FE and the coefficients D_k.  Sets fe and, in each lane, the
// partials of its slots (acc) and of the two kinds of corner literal
// (gF = sum_k D_k U_k(1), gT = sum_k D_k U_k(-1)).  ser = the length's rows.
template <int G, int QS>
__device__ __forceinline__ void group_low_cheb(int jlo, int nnc, int t, int lam,
                                               const float (&y)[QS], const F4* __restrict__ ser,
                                               const float4* ctab, float (&acc)[QS], float& fe,
                                               float& gF, float& gT) {
  constexpr int K = kSeriesK1;
  float M[K];
#pragma unroll
  for (int k = 0; k < K; ++k) M[k] = 0.f;
#pragma unroll
  for (int s = 0; s < QS; ++s) {
    const float m = lam + G * s < nnc ? 1.f : 0.f, y2 = y[s] + y[s];
    float tp = 1.f, tt = y[s];
    M[0] = fmaf(m, tt, M[0]);
#pragma unroll
    for (int k = 1; k < K; ++k) {
      const float tn = fmaf(y2, tt, -tp);
      tp = tt;
      tt = tn;
      M[k] = fmaf(m, tt, M[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int d = 1; d < G; d <<= 1) M[k] += __shfl_xor_sync(kFull, M[k], d);
    M[k] *= 1.0f / (float)(k + 1);
  }
  float D[K];
#pragma unroll
  for (int k = 0; k < K; ++k) D[k] = 0.f;
  float fl = 0.f;
#pragma unroll 1
  for (int j = lam; j < jlo; j += G) {
    const float4* row = reinterpret_cast<const float4*>(ser + (size_t)j * kSerRow);
    const float4 h = __ldg(row);
    const uint32_t turns = (uint32_t)nnc * __float_as_uint(h.y) + (uint32_t)t * __float_as_uint(h.z);
    float lr = (float)nnc * h.x, li = 0.f;
#pragma unroll
    for (int m = 0; m < K / 2; ++m) {
      const float4 e = __ldg(row + 1 + m);   // Re E_2m, Re E_2m+1, Im E_2m, Im E_2m+1
      lr = fmaf(e.x, M[2 * m], lr);
      li = fmaf(e.z, M[2 * m], li);
      lr = fmaf(e.y, M[2 * m + 1], lr);
      li = fmaf(e.w, M[2 * m + 1], li);
    }
    float sn, cs;
    sincosf(fmaf((float)(int32_t)turns, 1.4629180792671596e-9f, li), &sn, &cs);
    const float mag = expf(lr);
    const float4 b = ctab[j];
    const float gr = mag * cs, gi = mag * sn;
    const float wr = fmaf(b.x, gr, -b.y * gi), wi = fmaf(b.x, gi, b.y * gr);
    fl += wr;
#pragma unroll
    for (int m = 0; m < K / 2; ++m) {
      const float4 e = __ldg(row + 1 + m);
      D[2 * m] = fmaf(e.x, wr, fmaf(-e.z, wi, D[2 * m]));
      D[2 * m + 1] = fmaf(e.y, wr, fmaf(-e.w, wi, D[2 * m + 1]));
    }
  }
#pragma unroll
  for (int d = 1; d < G; d <<= 1) fl += __shfl_xor_sync(kFull, fl, d);
  fe = fl;
  gF = 0.f;
  gT = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int d = 1; d < G; d <<= 1) D[k] += __shfl_xor_sync(kFull, D[k], d);
    gF = fmaf((float)(k + 1), D[k], gF);
    gT = fmaf((k & 1) ? -(float)(k + 1) : (float)(k + 1), D[k], gT);
  }
#pragma unroll
  for (int s = 0; s < QS; ++s) {
    const float y2 = y[s] + y[s];
    float b1 = 0.f, b2 = 0.f;
#pragma unroll
    for (int k = K - 1; k >= 0; --k) {
      const float b0 = fmaf(y2, b1, D[k] - b2);
      b2 = b1;
      b1 = b0;
    }
    acc[s] = b1;
  }
}

// Pass 2 with G lanes per restart: G rounds over the tile's 32 restarts, 32/G
// restarts per round.  ncw = the warp's slots (slot k of restart r at
// ncw[k * 32 + r]); the restart's values are replaced by its partials; fe,
// gF, gT of restart r go to vals[0..2][r].
// With jlo > 0 the roots 1..jlo come from group_low_cheb (ser = the
// length's Chebyshev rows) and the root loop starts after them.
template <int G>
__device__ __forceinline__ void group_roots(int L, int J, int nnc_own, int t_own, int lane,
                                            const float4* rtab, const float4* ctab,
                                            const float4* ztab, float* ncw, float* vals, int jlo,
                                            const F4* __restrict__ ser) {
  constexpr int QS = kCornerQS;
  const int N = L + 1, nA = fr_roots_form0(L), nB = fr_roots_form01(L);
  const int lam = lane % G;
#pragma unroll 1
  for (int round = 0; round < G; ++round) {
    const int rr = round * (32 / G) + lane / G;
    const int nnc = __shfl_sync(kFull, nnc_own, rr), t = __shfl_sync(kFull, t_own, rr);
    float y[QS], acc[QS];
#pragma unroll
    for (int s = 0; s < QS; ++s) {
      const int k = lam + G * s;
      y[s] = k < nnc ? ncw[k * 32 + rr] : 1.f;
      acc[s] = 0.f;
    }
    float fe = 0.f, gF = 0.f, gT = 0.f;
    if (jlo > 0) group_low_cheb<G, QS>(jlo, nnc, t, lam, y, ser, ctab, acc, fe, gF, gT);
    const int dq = t % N;
    int q = (int)(((int64_t)(jlo + 1) * t) % N);   // (root number) * t mod N
#pragma unroll 1
    for (int j = jlo; j < J; ++j) {
      float2 W = make_float2(1.f, 0.f);
      if (q != 0) {
        const bool low = q <= J;
        const float4 e = rtab[(low ? q : N - q) - 1];
        W = make_float2(1.f - 2.f * e.y, low ? 2.f * e.z : -2.f * e.z);
      }
      const float4 rt = rtab[j], cf = ctab[j], zp = ztab[j];
      if (j < nA) group_root<G, QS, 0>(rt, zp, cf, W, y, acc, fe, gF, gT);
      else if (j < nB) group_root<G, QS, 1>(rt, zp, cf, W, y, acc, fe, gF, gT);
      else group_root<G, QS, 2>(rt, zp, cf, W, y, acc, fe, gF, gT);
      q += dq;
      if (q >= N) q -= N;
    }
    __syncwarp();
#pragma unroll
    for (int s = 0; s < QS; ++s) {
      const int k = lam + G * s;
      if (k < nnc) ncw[k * 32 + rr] = acc[s];
    }
    if (lam == 0) {
      vals[rr] = fe;
      vals[32 + rr] = gF;
      vals[64 + rr] = gT;
    }
    __syncwarp();
  }
}

// GC = 1: one thread per restart, at most kCornerQS non-corner literals;
// GC > 1: GC lanes per restart, at most GC * kCornerQS, for the tiles the
// GC = 1 pass left (GC > 1 only reads the flags; GC = 1 writes every flag).
template <int GC>
__global__ void __launch_bounds__(256, GC == 1 ? 3 : 2) k_fe_dft_corner(
    const int32_t* __restrict__ list, const FeItem* __restrict__ fe,
    const F4* __restrict__ root, const F4* __restrict__ zpow, const F4* __restrict__ coef,
    const LitRec* __restrict__ lit, const float* __restrict__ x, int R, int Rp, int RT,
    int maxL, float* __restrict__ P, float* __restrict__ fe_con, int ldf,
    uint8_t* __restrict__ done, const int8_t* __restrict__ spec_tab,
    const int32_t* __restrict__ spec_off, const SerInfo* __restrict__ ser_info,
    const F4* __restrict__ ser_tab) {
  extern __shared__ float4 cs4[];
  const FeItem it = fe[list[blockIdx.x]];
  const int L = it.L, J = it.J;
  const int JC = (maxL + 1) / 2;
  float4* rtab = cs4;                                         // [JC] {A, B, C, t}
  float4* ctab = rtab + JC;                                   // [JC] {b', c'}
  float4* ztab = ctab + JC;                                   // [JC] {z^16, z^15}
  constexpr int CAP = GC * kCornerQS;                          // non-corner literals
  float* ncy = reinterpret_cast<float*>(ztab + JC);          // [8][CAP][32]
  float* vals = ncy + 8 * CAP * 32;                           // [8][3][32] fe, gF, gT
  LitRec* recs = reinterpret_cast<LitRec*>(vals + 8 * 3 * 32);          // [maxL]
  const int FLW = (maxL + 15) / 16;
  uint32_t* flags = reinterpret_cast<uint32_t*>(recs + maxL);            // [8][FLW][32]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if constexpr (GC > 1) {
    // nothing to do unless one of the block's tiles is still open
    const int tl = blockIdx.y * 8 + (threadIdx.x & 7);
    const bool open = (threadIdx.x < 8) && tl < RT && done[(size_t)it.c * RT + tl] == kTileOpen;
    if (!__syncthreads_or(open)) return;
  }
  for (int i = threadIdx.x; i < L; i += 256) recs[i] = lit[it.lit0 + i];
  __syncthreads();
  const int tile = blockIdx.y * 8 + warp;
  const bool live = tile < RT;
  const int r = (live ? tile : RT - 1) * 32 + lane;
  const bool act = r < R;
  const float* xr = x + (act ? r : R - 1);
  float* my = ncy + warp * CAP * 32 + lane;
  // pass 1: true corners and the non-corner values, in literal order; each
  // lane keeps its restart's classification of every literal as a 2-bit code
  // (bit 0 true corner, bit 1 non-corner), 16 literals per word in its own
  // column of shared memory, so that pass 3 need not read x again
  uint32_t* fl = flags + (size_t)warp * FLW * 32 + lane;
  int nnc = 0, t = 0;
  // GC > 1: tiles the one-thread pass finished are left alone
  const bool skip = GC > 1 && live && done[(size_t)it.c * RT + tile] != kTileOpen;
  bool over = !live || skip;
  int i_over = L;
  for (int i0 = 0; i0 < L && !over; i0 += 16) {
    const int i1 = min(L, i0 + 16);
    uint32_t code = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int b = i0 + 8 * h;
      if (b >= i1) break;
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const LitRec rc = recs[min(b + u, L - 1)];
        v[u] = apply_sgn(xr[(size_t)rc.var * R], rc.dst);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (b + u < i1) {
          const float y = act ? v[u] : 1.f;
          const bool tc = y == -1.f, nc = fabsf(y) != 1.f;
          code |= (tc ? 1u : 0u) << (16 * h + 2 * u);
          code |= (nc ? 2u : 0u) << (16 * h + 2 * u);
          if (nc) {
            if (nnc < CAP) my[nnc * 32] = y;
            ++nnc;
          }
        }
      }
    }
    fl[(i0 >> 4) * 32] = code;
    t += __popc(code & 0x55555555u);
    if (__any_sync(kFull, nnc > CAP)) {
      over = true;
      i_over = i1;
      break;
    }
  }
  // the root tables only if some tile of the block stays here
  // GC = 1 marks a tile whose non-corner density projects past the second
  // pass's capacity (more than 5/4 of it over L literals) as dense outright
  const uint8_t gave_up =
      (GC == 1 && (int64_t)(CAP + 1) * L > (int64_t)i_over * (kCornerGroup * kCornerQS * 5 / 4))
          ? kTileDense
          : kTileOpen;
  if (!__syncthreads_or(!over)) {
    if (GC == 1 && live && lane == 0) done[(size_t)it.c * RT + tile] = gave_up;
    return;
  }
  for (int j = threadIdx.x; j < J; j += 256) {
    rtab[j] = ldg4(&root[it.root_off + j]);
    ctab[j] = ldg4(&coef[it.coef_off + j]);
    ztab[j] = ldg4(&zpow[(size_t)(it.root_off + j) * kNumFrQ + kCornerZq]);
  }
  __syncthreads();
  if (over) {
    if (GC == 1 && live && lane == 0) done[(size_t)it.c * RT + tile] = gave_up;
    return;
  }
  // pass 2
  float fev, gF, gT;
  if constexpr (GC == 1) {
    const int qmax = __reduce_max_sync(kFull, nnc);
    const int8_t* sp = spec_tab + spec_off[it.c];
    // the DPs give FE itself; the write-out below adds the constant term
    if (qmax <= 8) {
      if (qmax <= 4) corner_dp<4>(L, t, sp, my, nnc, fev, gF, gT);
      else corner_dp<8>(L, t, sp, my, nnc, fev, gF, gT);
      fev -= it.b0;
    } else if (dp_pays(J, kCornerQS, kCornerQS)) {
      corner_dpx<kCornerQS>(L, t, qmax, sp, my, nnc, fev, gF, gT);
      fev -= it.b0;
    } else {
      corner_roots<kCornerQS>(L, J, nnc, t, rtab, ctab, ztab, my, fev, gF, gT);
    }
  } else {
    const int qmax = __reduce_max_sync(kFull, nnc);
    if (qmax <= kCornerDpx && dp_pays(J, kCornerDpx, CAP)) {
      corner_dpx<kCornerDpx>(L, t, qmax, spec_tab + spec_off[it.c], my, nnc, fev, gF, gT);
      fev -= it.b0;
    } else {
      float* vw = vals + warp * 96;
      // long constraints: the low roots by Chebyshev sums over the interior
      const SerInfo si = ser_info[it.c];
      const int jlo = (si.off >= 0 && si.js1 >= kCornerChebMin) ? si.js1 : 0;
      group_roots<GC>(L, J, nnc, t, lane, rtab, ctab, ztab, ncy + warp * CAP * 32, vw, jlo,
                      ser_tab + (si.off >= 0 ? si.off : 0));
      fev = vw[lane];
      gF = vw[32 + lane];
      gT = vw[64 + lane];
    }
  }
  // pass 3: partials w * s_e * dFE/dy_e of every literal
  int k = 0;
  const float wgF = it.w * gF, wgT = it.w * gT;
  for (int i0 = 0; i0 < L; i0 += 16) {
    const uint32_t code = fl[(i0 >> 4) * 32];
    const int n = min(16, L - i0);
#pragma unroll 4
    for (int u = 0; u < n; ++u) {
      const LitRec rc = recs[i0 + u];
      const uint32_t cu = code >> (2 * u);
      float val = (cu & 1u) ? wgT : wgF;
      if (cu & 2u) {
        val = it.w * my[k * 32];
        ++k;
      }
      if (act) st_partial(&P[(size_t)rec_row(rc.dst) * Rp + r], apply_sgn(val, rc.dst));
    }
  }
  if (fe_con && act) fe_con[(size_t)it.c * ldf + r] = it.b0 + fev;
  __syncwarp();
  if (lane == 0) done[(size_t)it.c * RT + tile] = kTileDone;
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace

size_t corner_smem_bytes(int maxL, int gc) {
  const int JC = (maxL + 1) / 2;
  return (size_t)3 * JC * sizeof(float4) + (size_t)8 * gc * kCornerQS * 32 * sizeof(float) +
         (size_t)8 * 3 * 32 * sizeof(float) + (size_t)maxL * sizeof(LitRec) +
         (size_t)8 * ((maxL + 15) / 16) * 32 * sizeof(uint32_t);
}

cudaError_t set_corner_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_fe_dft_corner<1>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)corner_smem_bytes(1024, 1));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fe_dft_corner<kCornerGroup>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)corner_smem_bytes(1024, kCornerGroup));
  return e;
}

cudaError_t launch_dft_corner(const DevPlan& d, const int32_t* list, int count, int maxL, int R,
                              int Rp, const float* x, float* P, float* fe_con, int ldf,
                              uint8_t* done, cudaStream_t s, bool group) {
  if (count == 0 || R == 0) return cudaSuccess;
  const int RT = ceil_div(R, 32);
  const dim3 grid(count, ceil_div(RT, 8)), block(256);
  k_fe_dft_corner<1><<<grid, block, corner_smem_bytes(maxL, 1), s>>>(
      list, d.fe, d.root_tab, d.zpow_tab, d.coef_tab, d.fe_lit, x, R, Rp, RT, maxL, P, fe_con,
      ldf, done, d.spec_tab, d.spec_off, d.ser_info, d.ser_tab);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !group) return e;
  k_fe_dft_corner<kCornerGroup><<<grid, block, corner_smem_bytes(maxL, kCornerGroup), s>>>(
      list, d.fe, d.root_tab, d.zpow_tab, d.coef_tab, d.fe_lit, x, R, Rp, RT, maxL, P, fe_con,
      ldf, done, d.spec_tab, d.spec_off, d.ser_info, d.ser_tab);
  return cudaGetLastError();
}

}  // namespace cls
