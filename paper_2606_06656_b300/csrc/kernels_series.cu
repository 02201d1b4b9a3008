// kernels_series.cu -- the low roots of long DFT constraints by Chebyshev sums.
//
// FE = b0 + sum_j Re(b'_j G_j) and dFE/dy_i = sum_j Re(b'_j G_j dlog F_ij /
// dy_i) (the Fourier form of the expansion, Sec. 2.3), G_j = prod_i F_ij,
// F_ij = alpha_i + beta_i w^j = h_j (1 + q_j y_i).  With r_j as in plan.h
// (|r_j| = tan(phi_j / 2)) the Chebyshev generating function gives, on all
// of [-1, 1],
//   log F_j(y)       = C_j + sum_{k>=1} E_{k-1} T_k(y) / k,
//   dlog F_j(y) / dy = sum_{k>=0} E_k U_k(y),          E_k = -2 r_j^(k+1),
// so with the Chebyshev sums M_k = sum_{interior i} T_k(y_i) (interior:
// |y| < 1; a literal at a corner contributes log 1 = 0 or log w^j =
// i theta_j exactly)
//   log G_j = n_int C_j + i theta_j n_true + sum_k E_{k-1} M_k / k,
// and every literal's partial is a Chebyshev-U series in its own value:
//   dFE/dy_i = sum_k D_k U_k(y_i),   D_k = Re sum_j b'_j G_j E_k,
// evaluated by Clenshaw's recurrence.  The host keeps, per length, the roots
// whose truncation after K terms is bounded by 2^-24 (plan.cpp,
// series_roots).  Per restart the work is about 4K per literal and 4K per
// root instead of 7 per (literal, root).
//
// One thread per (constraint, restart), a warp per tile of 32 restarts, a
// block per constraint and 8 tiles.  Pass A computes the tail cutoff of
// kernels.cuh (tail_roots, from the sums of a^m, a = 1 - y^2, m = 1..4); a
// tile whose largest cutoff lies in the range of 12..26 terms is finished
// here with the fewest that suffice (flag done).  A tile that
// needs more roots gets the terms of the roots 1..js1 (26 terms) here when
// that saves enough root products (flag low: the dense factored kernel adds
// the rest); any other is left to the dense kernel.  Pass B forms the
// Chebyshev sums, the root loop G_j and the coefficients D_k, pass C the
// partials.  Phases: arg of e^{C_j} and theta_j are tabulated as uint32
// fractions of a turn, so n arg mod 2 pi is an exact integer product (error
// <= n/2 2^-32 turns); sincosf only sees that plus the series' part.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "kernels.cuh"

namespace cls {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kTwoPiOver2p32 = 1.4629180792671596e-9f;

__device__ __forceinline__ int rec_row(int32_t dst) { return dst & 0x7fffffff; }
// a table row entry from shared memory, loaded where it is used (volatile, so
// that the compiler does not keep a root's K entries live across both loops)
__device__ __forceinline__ float4 lds4(const float4* p) {
  float4 v;
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(a));
  return v;
}
__device__ __forceinline__ float rec_sgn(int32_t dst) { return dst < 0 ? -1.0f : 1.0f; }

// Literal values reach the passes as cp.async copies in chunks of kSerChunk
// literals, double-buffered per warp (stw = the warp's stage[2][kSerChunk][32]).
// With vec (R a multiple of 4 and x 16-byte aligned) lane l copies 16 bytes,
// restarts 4 (l % 8) .. +3 of chunk literals l / 8, l / 8 + 4, ...: four
// copies per lane per chunk instead of sixteen; otherwise every lane copies
// its own 4-byte values.  Each lane reads back its own restart's values
// after the warp has synchronised.  f2(i, y_i, y_{i+1}) takes two consecutive
// literals, with y = s x when SGN (the signs as a bitmask, sgn bit i =
// literal i negated; the sign bit is flipped in place) and y = x otherwise;
// a full chunk runs unrolled, so the sign bits are compile-time positions.
// f1(i, y_i) takes the last literal of an odd tail.  No copy ever targets an
// inactive lane's column; the kernel fills those with 1 once
// (stage_fill_inactive), so every lane reads without a test.
// [y^n] U_k: (-1)^m C(k - m, m) 2^(k - 2m) for n = k - 2m, else 0; every
// value for k < 26 is an integer times a power of 2 with at most 15
// significant bits, so the float is exact.
__host__ __device__ constexpr float umono(int k, int n) {
  if (n > k || ((k - n) & 1)) return 0.f;
  const int m = (k - n) / 2;
  double bin = 1.0;
  for (int i = 0; i < m; ++i) bin = bin * (double)(k - m - i) / (double)(i + 1);
  double p = 1.0;
  for (int i = 0; i < k - 2 * m; ++i) p *= 2.0;
  return (float)((m & 1 ? -1.0 : 1.0) * bin * p);
}
// sum of |[y^n] U_k| over n: the Pell number P_(k+1) (P_1 = 1, P_2 = 2,
// P_n = 2 P_(n-1) + P_(n-2))
__host__ __device__ constexpr float upell(int k) {
  double a = 0.0, b = 1.0;   // P_0, P_1
  for (int i = 0; i < k; ++i) {
    const double c = 2.0 * b + a;
    a = b;
    b = c;
  }
  return (float)b;
}
static_assert(umono(3, 1) == -4.f && umono(4, 0) == 1.f && upell(3) == 12.f, "U_k tables");

constexpr int kSerChunk = 16;
__device__ __forceinline__ void stage_fill_inactive(float* stw, int lane, bool act) {
  if (!act)
#pragma unroll
    for (int u = 0; u < 2 * kSerChunk; ++u) stw[u * 32 + lane] = 1.f;
}
template <bool SGN, typename F2, typename F1>
__device__ __forceinline__ void staged_scan(int L, const LitRec* recs, const uint32_t* sgn,
                                            const float* __restrict__ x, int R, int r0, int lane,
                                            bool vec, float* stw, F2&& f2, F1&& f1) {
  static_assert(kSerChunk == 16, "one 16-bit half of a sign word per chunk");
  const int nch = (L + kSerChunk - 1) / kSerChunk;
  const bool act = r0 + lane < R;
  auto issue = [&](int c) {
    float* dst = stw + (c & 1) * kSerChunk * 32;
    const int b0 = c * kSerChunk;
    if (vec) {
      const int q = lane & 7, u0 = lane >> 3;
      if (r0 + 4 * q < R) {                 // the whole quad: R is a multiple of 4
#pragma unroll
        for (int v = 0; v < kSerChunk / 4; ++v) {
          const int u = u0 + 4 * v;
          if (b0 + u < L)
            cp_async16(dst + u * 32 + 4 * q, x + (size_t)recs[b0 + u].var * R + r0 + 4 * q);
        }
      }
    } else if (act) {
#pragma unroll 8
      for (int u = 0; u < kSerChunk; ++u)
        if (b0 + u < L) cp_async4(dst + u * 32 + lane, x + (size_t)recs[b0 + u].var * R + r0 + lane);
    }
    cp_async_commit();
  };
  __syncwarp();                              // the previous scan's reads of buffer 0 are done
  issue(0);
  for (int c = 0; c < nch; ++c) {
    __syncwarp();                            // every lane is done with the buffer refilled next
    if (c + 1 < nch) issue(c + 1);
    else cp_async_commit();                  // an empty group keeps the count
    cp_async_wait<1>();
    __syncwarp();                            // chunk c is in place for every lane
    const float* src = stw + (c & 1) * kSerChunk * 32 + lane;
    const int b0 = c * kSerChunk, n = min(kSerChunk, L - b0);
    const uint32_t sb = SGN ? (sgn[b0 >> 5] >> (b0 & 31)) : 0u;
    auto val = [&](int u) -> float {
      const float v = src[u * 32];
      return SGN ? __uint_as_float(__float_as_uint(v) ^ ((sb << (31 - u)) & 0x80000000u)) : v;
    };
    if (n == kSerChunk) {
#pragma unroll
      for (int u = 0; u < kSerChunk; u += 2) f2(b0 + u, val(u), val(u + 1));
    } else {
      int u = 0;
#pragma unroll 1
      for (; u + 2 <= n; u += 2) f2(b0 + u, val(u), val(u + 1));
      if (u < n) f1(b0 + u, val(u));
    }
  }
  cp_async_wait<0>();
}

// The tail sums of kernels.cuh for two literals per packed instruction.
struct TailSums2 {
  float2 a1 = {0.f, 0.f}, a2 = {0.f, 0.f}, a3 = {0.f, 0.f}, a4 = {0.f, 0.f};
  float amax = 0.f;
  __device__ __forceinline__ void add2(float x0, float x1) {
    const float2 xv = make_float2(x0, x1);
    const float2 a = __ffma2_rn(make_float2(-x0, -x1), xv, make_float2(1.f, 1.f));
    const float2 b = __fmul2_rn(a, a);
    a1 = __fadd2_rn(a1, a);
    a2 = __fadd2_rn(a2, b);
    a3 = __ffma2_rn(b, a, a3);
    a4 = __ffma2_rn(b, b, a4);
    amax = fmaxf(amax, fmaxf(a.x, a.y));
  }
  __device__ __forceinline__ TailSums fold() const {
    TailSums t;
    t.a1 = a1.x + a1.y;
    t.a2 = a2.x + a2.y;
    t.a3 = a3.x + a3.y;
    t.a4 = a4.x + a4.y;
    t.amax = amax;
    return t;
  }
};

// one restart's K-term pass: Chebyshev sums, the root loop over jw roots, the
// partials of all L literals (written to P) and FE - b0 (returned).  With sd
// (a low tile) the pass stops after the roots and saves D_0..D_{K-1} and
// FE - b0 at sd[k * Rp] instead; the dense factored kernel adds them.
template <int K>
__device__ __forceinline__ float series_restart(int L, int jw, const LitRec* recs,
                                                const uint32_t* sgn, const float* x, int R,
                                                int r0, int lane, bool vec,
                                                const float4* tab, const float2* bsm,
                                                float* __restrict__ P, int Rp, float wgt,
                                                float* stw, float* sd, bool& horner) {
  const int r = r0 + lane;
  const bool act = r < R;
  static_assert(K % 2 == 0, "table rows hold pairs of terms");
  // pass B: M[k-1] = sum over interior literals of T_k(y); two literals per
  // packed FP32x2 instruction (float2 sums, folded afterwards)
  float2 M2[K];
#pragma unroll
  for (int k = 0; k < K; ++k) M2[k] = make_float2(0.f, 0.f);
  uint32_t ni = 0, nt = 0;
  auto cls1 = [&](int, float yv, float& y, float& m) {
    y = yv;
    const bool corner = fabsf(y) == 1.f;
    nt += (y == -1.f) ? 1u : 0u;
    ni += corner ? 0u : 1u;
    m = corner ? 0.f : 1.f;
  };
  auto sums = [&](float2 y, float2 m) {
    const float2 y2 = __fadd2_rn(y, y);
    float2 tp = make_float2(1.f, 1.f), t = y;          // T_0, T_1
    M2[0] = __ffma2_rn(m, t, M2[0]);
#pragma unroll
    for (int k = 1; k < K; ++k) {
      const float2 tn = __ffma2_rn(y2, t, make_float2(-tp.x, -tp.y));
      tp = t;
      t = tn;
      M2[k] = __ffma2_rn(m, t, M2[k]);
    }
  };
  staged_scan<true>(
      L, recs, sgn, x, R, r0, lane, vec, stw,
      [&](int i, float x0, float x1) {
        float ya, yb, ma, mb;
        cls1(i, x0, ya, ma);
        cls1(i + 1, x1, yb, mb);
        sums(make_float2(ya, yb), make_float2(ma, mb));
      },
      [&](int i, float x0) {
        float ya, ma;
        cls1(i, x0, ya, ma);
        sums(make_float2(ya, 0.f), make_float2(ma, 0.f));
      });
  // the sums of terms 2m and 2m + 1 side by side (the table's pairs)
  float2 Mp[K / 2];
#pragma unroll
  for (int m = 0; m < K / 2; ++m)
    Mp[m] = make_float2((M2[2 * m].x + M2[2 * m].y) * (1.0f / (float)(2 * m + 1)),
                        (M2[2 * m + 1].x + M2[2 * m + 1].y) * (1.0f / (float)(2 * m + 2)));
  // roots: log G_j, G_j, w = b'_j G_j, FE and D_k, two terms per packed
  // instruction (Dp[m] = {D_2m, D_2m+1})
  float2 Dp[K / 2];
#pragma unroll
  for (int m = 0; m < K / 2; ++m) Dp[m] = make_float2(0.f, 0.f);
  float fe = 0.f;
  const float fni = (float)ni;
#pragma unroll 1
  for (int j = 0; j < jw; ++j) {
    const float4* row = tab + j * kSerRow;
    const float4 h = row[0];
    const uint32_t turns = ni * __float_as_uint(h.y) + nt * __float_as_uint(h.z);
    float2 lr2 = make_float2(fni * h.x, 0.f), li2 = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 0; m < K / 2; ++m) {
      const float4 e = lds4(row + 1 + m);     // Re E_2m, Re E_2m+1, Im E_2m, Im E_2m+1
      lr2 = __ffma2_rn(make_float2(e.x, e.y), Mp[m], lr2);
      li2 = __ffma2_rn(make_float2(e.z, e.w), Mp[m], li2);
    }
    const float lr = lr2.x + lr2.y, li = li2.x + li2.y;
    float sn, cs;
    sincosf(fmaf((float)(int32_t)turns, kTwoPiOver2p32, li), &sn, &cs);
    const float mag = expf(lr);
    const float2 b = bsm[j];
    const float gr = mag * cs, gi = mag * sn;
    const float wr = fmaf(b.x, gr, -b.y * gi), wi = fmaf(b.x, gi, b.y * gr);
    fe += wr;
    const float2 wr2 = make_float2(wr, wr), nwi2 = make_float2(-wi, -wi);
#pragma unroll
    for (int m = 0; m < K / 2; ++m) {
      const float4 e = lds4(row + 1 + m);
      Dp[m] = __ffma2_rn(make_float2(e.x, e.y), wr2,
                         __ffma2_rn(make_float2(e.z, e.w), nwi2, Dp[m]));
    }
  }
  float D[K];
#pragma unroll
  for (int m = 0; m < K / 2; ++m) {
    D[2 * m] = Dp[m].x;
    D[2 * m + 1] = Dp[m].y;
  }
  if (sd) {
    if (act) {
#pragma unroll
      for (int k = 0; k < K; ++k) sd[(size_t)k * Rp] = D[k];
      sd[(size_t)K * Rp] = fe;
    }
    return fe;
  }
  // pass C: partials, p(y) = sum_k D_k U_k(y), two literals per packed
  // instruction.  Horner's rule on the monomial coefficients c_n takes one
  // operation per term, Clenshaw's recurrence two.  In FP32 (unit roundoff
  // u = 2^-24), converting D to c (K products per coefficient) and
  // evaluating by Horner (|y| <= 1) err by at most about 3K u sum_k |D_k|
  // P_(k+1), P_(k+1) = sum over n of |[y^n] U_k| (a Pell number, ~2.41^k).
  // The warp takes Horner's rule only when for every restart that bound is
  // at most 2^-17 sum_k (k+1) |D_k|, 2^-17 of the largest value |p| can
  // take on [-1, 1] and below the a-priori bound of the recurrence itself
  // (of order K^2 u of the same scale).  That holds when D_k decays fast,
  // as it does while only the first roots matter (points far from the
  // corners); otherwise the warp keeps Clenshaw's recurrence.
  float sP = 0.f, sM = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float a = fabsf(D[k]);
    sP = fmaf(upell(k), a, sP);
    sM = fmaf((float)(k + 1), a, sM);
  }
  horner = __all_sync(0xffffffffu, !act || 3.f * (float)K * sP <= 128.f * sM);
  auto clenshaw = [&](float2 y) -> float2 {
    const float2 y2 = __fadd2_rn(y, y);
    float2 b1 = make_float2(0.f, 0.f), b2 = b1;
#pragma unroll
    for (int k = K - 1; k >= 0; --k) {
      const float2 b0 = __ffma2_rn(y2, b1, __fadd2_rn(make_float2(D[k], D[k]),
                                                      make_float2(-b2.x, -b2.y)));
      b2 = b1;
      b1 = b0;
    }
    return b1;
  };
  auto put = [&](int i, float g) {
    const int32_t dst = recs[i].dst;
    if (act) st_partial(&P[(size_t)rec_row(dst) * Rp + r], wgt * rec_sgn(dst) * g);
  };
  if (horner) {
    float c[K];                      // c_n = sum_k [y^n] U_k D_k
#pragma unroll
    for (int n = 0; n < K; ++n) c[n] = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
      for (int n = k & 1; n <= k; n += 2) c[n] = fmaf(umono(k, n), D[k], c[n]);
    }
    auto horner_eval = [&](float2 y) -> float2 {
      float2 h = make_float2(c[K - 1], c[K - 1]);
#pragma unroll
      for (int n = K - 2; n >= 0; --n) h = __ffma2_rn(h, y, make_float2(c[n], c[n]));
      return h;
    };
    staged_scan<true>(
        L, recs, sgn, x, R, r0, lane, vec, stw,
        [&](int i, float y0, float y1) {
          const float2 g = horner_eval(make_float2(y0, y1));
          put(i, g.x);
          put(i + 1, g.y);
        },
        [&](int i, float y0) { put(i, horner_eval(make_float2(y0, 0.f)).x); });
  } else {
    staged_scan<true>(
        L, recs, sgn, x, R, r0, lane, vec, stw,
        [&](int i, float y0, float y1) {
          const float2 g = clenshaw(make_float2(y0, y1));
          put(i, g.x);
          put(i + 1, g.y);
        },
        [&](int i, float y0) { put(i, clenshaw(make_float2(y0, 0.f)).x); });
  }
  return fe;
}

// Dynamic shared memory: kSeriesMaxRoots * kSerRow float4 (rows), as many
// float2 (b'_j), the staging buffers (8 warps x 2 x kSerChunk x 32 floats),
// maxL LitRec, the sign bits of maxL literals.
__global__ void __launch_bounds__(256, 3) k_fe_series(
    const int32_t* __restrict__ list, const FeItem* __restrict__ fe,
    const F4* __restrict__ coef, const F4* __restrict__ ser_tab,
    const SerInfo* __restrict__ ser_info, const LitRec* __restrict__ lit,
    const float* __restrict__ x, int R, int Rp, int RT, int maxL, int vec,
    float* __restrict__ P, float* __restrict__ fe_con, int ldf, uint8_t* __restrict__ done,
    float* __restrict__ ser_d, unsigned long long* __restrict__ flops) {
  extern __shared__ float4 ss4[];
  float4* tab = ss4;                                                  // [96][kSerRow]
  float2* bsm = reinterpret_cast<float2*>(tab + kSeriesMaxRoots * kSerRow);  // [96]
  float* stage = reinterpret_cast<float*>(bsm + kSeriesMaxRoots);     // [8][2][chunk][32]
  LitRec* recs = reinterpret_cast<LitRec*>(stage + 8 * 2 * kSerChunk * 32);   // [maxL]
  uint32_t* sgn = reinterpret_cast<uint32_t*>(recs + maxL);           // [(maxL + 31) / 32]
  __shared__ int jneed_s[8];
  const int ci = list[blockIdx.x];
  const SerInfo si = ser_info[ci];
  if (si.off < 0) return;
  const FeItem it = fe[ci];
  const int L = it.L, J = it.J;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = blockIdx.y * 8 + warp;
  const bool live = tile < RT;
  const bool mine = live && done[(size_t)ci * RT + tile] != kTileDone;
  if (!__syncthreads_or(mine)) return;
  for (int i = threadIdx.x; i < L; i += 256) recs[i] = lit[it.lit0 + i];
  for (int w = threadIdx.x; w < (L + 31) / 32; w += 256) {
    uint32_t bits = 0;
    for (int b = 0; b < 32 && 32 * w + b < L; ++b)
      bits |= (lit[it.lit0 + 32 * w + b].dst < 0 ? 1u : 0u) << b;
    sgn[w] = bits;
  }
  __syncthreads();
  const int r0 = (live ? tile : RT - 1) * 32;
  const int r = r0 + lane;
  const bool act = r < R;
  float* stw = stage + (size_t)warp * 2 * kSerChunk * 32;
  stage_fill_inactive(stw, lane, act);
  // pass A: the tail cutoff (as in kernels_fr.cu) and the terms it needs
  int jw = 0, K = 0;
  bool part = false;
  if (mine) {
    TailSums2 ts;   // (1 - x^2 does not depend on the literal's sign)
    staged_scan<false>(L, recs, sgn, x, R, r0, lane, vec, stw,
                       [&](int, float x0, float x1) { ts.add2(x0, x1); },
                       [&](int, float x0) { ts.add2(x0, 1.f); });
    const int jc = act ? tail_roots(ts.fold(), L, J, logf(2.f * (float)J) + kTailLogInvEps) : 0;
    jw = __reduce_max_sync(kFull, act ? jc : 0);
    // the fewest terms whose range holds the tile's roots: 12, 14, 16, 18,
    // 22 or 26
    K = jw <= si.jsx[0]   ? 12
        : jw <= si.jsx[1] ? 14
        : jw <= si.jsx[2] ? 16
        : jw <= si.js0    ? kSeriesK0
        : jw <= si.jsx[3] ? 22
        : jw <= si.js1    ? kSeriesK1
                          : 0;
    // beyond the range: the low roots 1..js1 here, the others in the dense
    // kernel, when the root products saved (14 flops per literal and root)
    // outweigh the cost of this pass and of the Clenshaw share
    if (K == 0 && 14 * (int64_t)L * si.js1 >
                      (int64_t)L * (4 + 8 * kSeriesK1) + (int64_t)si.js1 * (8 * kSeriesK1 + 40)) {
      K = kSeriesK1;
      part = true;
      jw = si.js1;
    }
  }
  if (lane == 0) jneed_s[warp] = K ? jw : 0;
  __syncthreads();
  int jb = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) jb = max(jb, jneed_s[w]);
  if (jb == 0) return;
  for (int e = threadIdx.x; e < jb * kSerRow; e += 256)
    tab[e] = *reinterpret_cast<const float4*>(&ser_tab[si.off + e]);
  for (int j = threadIdx.x; j < jb; j += 256) {
    const F4 cf = coef[it.coef_off + j];
    bsm[j] = make_float2(cf.x, cf.y);
  }
  __syncthreads();
  if (K == 0) return;
  float fev;
  bool horner = false;
  float* sd = part ? ser_d + (size_t)si.slot * (kSeriesK1 + 1) * Rp + r : nullptr;
  static_assert(kSeriesK0 == 18 && kSeriesK1 == 26 && kSeriesKx[0] == 12 &&
                    kSeriesKx[1] == 14 && kSeriesKx[2] == 16 && kSeriesKx[3] == 22,
                "term counts of the dispatch below");
#define CLS_SERIES(KK) \
  series_restart<KK>(L, jw, recs, sgn, x, R, r0, lane, vec, tab, bsm, P, Rp, it.w, stw, sd, horner)
  switch (K) {
    case 12: fev = CLS_SERIES(12); break;
    case 14: fev = CLS_SERIES(14); break;
    case 16: fev = CLS_SERIES(16); break;
    case 18: fev = CLS_SERIES(18); break;
    case 22: fev = CLS_SERIES(22); break;
    default: fev = CLS_SERIES(26); break;
  }
#undef CLS_SERIES
  if (fe_con && act && !part) fe_con[(size_t)it.c * ldf + r] = it.b0 + fev;
  // (K is uniform over the warp, so every lane is here)
  const unsigned nact = (unsigned)__popc(__ballot_sync(kFull, act));
  if (flops && lane == 0) {
    // per restart: L (4 + 8K) for the passes with Clenshaw's partials,
    // L (4 + 6K) + K^2 with Horner's (L (4 + 4K) on a low tile, whose
    // Clenshaw pass the dense kernel counts), jw (8K + 40) for the roots
    const unsigned long long per =
        (unsigned long long)L * (4 + (part ? 4 : horner ? 6 : 8) * K) +
        (horner ? (unsigned long long)(K * K) : 0ull) + (unsigned long long)jw * (8 * K + 40);
    atomicAdd(flops, per * (unsigned long long)nact);
  }
  __syncwarp();
  if (lane == 0) done[(size_t)ci * RT + tile] = part ? kTileLow : kTileDone;
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

size_t series_smem_bytes(int maxL) {
  return (size_t)kSeriesMaxRoots * kSerRow * sizeof(float4) +
         (size_t)kSeriesMaxRoots * sizeof(float2) +
         (size_t)8 * 2 * kSerChunk * 32 * sizeof(float) + (size_t)maxL * sizeof(LitRec) +
         (size_t)((maxL + 31) / 32) * sizeof(uint32_t);
}

}  // namespace

cudaError_t set_series_attributes() {
  return cudaFuncSetAttribute(k_fe_series, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)series_smem_bytes(1024));
}

cudaError_t launch_dft_series(const DevPlan& d, const int32_t* list, int count, int maxL, int R,
                              int Rp, const float* x, float* P, float* fe_con, int ldf,
                              uint8_t* done, cudaStream_t s) {
  if (count == 0 || R == 0 || maxL < kSeriesMinL || !d.ser_info) return cudaSuccess;
  const int RT = ceil_div(R, 32);
  const dim3 grid(count, ceil_div(RT, 8)), block(256);
  // 16-byte staging copies need every x row and the restart tiles on 16-byte
  // boundaries
  const int vec = (R % 4 == 0 && reinterpret_cast<uintptr_t>(x) % 16 == 0) ? 1 : 0;
  k_fe_series<<<grid, block, series_smem_bytes(maxL), s>>>(
      list, d.fe, d.coef_tab, d.ser_tab, d.ser_info, d.fe_lit, x, R, Rp, RT, maxL, vec, P,
      fe_con, ldf, done, ser_terms(d, done, RT), d.dft_flops);
  return cudaGetLastError();
}

}  // namespace cls
