// kernels.cuh -- launchers of the sm_103a kernels (kernels.cu), called by the
// C ABI layer (api.cu).  All launches are asynchronous on the given stream.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "plan.h"

namespace cls {

constexpr int kNumBuckets = kNumDftBuckets + kNumRealBuckets;

// Device copy of a HostPlan.
struct DevPlan {
  int32_t n = 0, m = 0;
  int64_t nnz = 0, nnz_fe = 0;
  LitRec* lit = nullptr;        // all literals (score, learned initialiser)
  int32_t* voff = nullptr;
  LitRec* fe_lit = nullptr;     // literals entering FE; dst = partial-buffer row
  int32_t* fe_voff = nullptr;   // n+1 partial-buffer rows per variable
  int32_t* const_list = nullptr;
  int32_t const_count = 0;
  FeItem* fe = nullptr;
  FeItem* thread_items[kNumThreadCls] = {};
  int32_t thread_count[kNumThreadCls] = {};
  int32_t* bucket_list[kNumBuckets] = {};
  int32_t bucket_count[kNumBuckets] = {};
  int32_t bucket_cfg[kNumBuckets] = {};
  int32_t bucket_maxL[kNumBuckets] = {};
  int32_t bucket_maxJ[kNumBuckets] = {};
  ScoreItem* score = nullptr;        // constraint order
  int32_t* score_ranges = nullptr;   // n_ranges+1 constraint boundaries
  int32_t n_ranges = 0;
  int32_t unit_weights = 0;          // every constraint weight is exactly 1
  unsigned long long* dft_flops = nullptr;   // flops of the evaluated DFT roots
  double* rw_gbar = nullptr;         // scratch of the weight update (mean gradient norm)
  int32_t* stat_order = nullptr;     // constraints by FE length, longest first
  int8_t* spec_tab = nullptr;        // spectra of the DFT constraints (+-1, t = 0..L)
  int32_t* spec_off = nullptr;       // per constraint, -1 if not a DFT constraint
  F4* ser_tab = nullptr;             // power-sum tables (plan.h, kSeriesK0)
  SerInfo* ser_info = nullptr;       // per constraint
  uint32_t* satbits = nullptr;
  F4* root_tab = nullptr;
  F4* zpow_tab = nullptr;
  F4* coef_tab = nullptr;
  uint8_t* fixed = nullptr;
  float* fixed_val = nullptr;
};

// Warps (score ranges) per score block; partial rows = ceil(n_ranges / this).
constexpr int kScoreWarps = 8;
inline int score_chunks(int n_ranges) { return (n_ranges + kScoreWarps - 1) / kScoreWarps; }

// Kernel classes for profiling (cls_profile_read).
enum KernelClass { KC_THREAD = 0, KC_GROUP_REAL, KC_GROUP_DFT, KC_ACCUM, KC_SCORE,
                   KC_REDUCE, KC_INIT, KC_COUNT };

// Called around each launch when profiling is on.
struct LaunchHook {
  virtual void before(int kc, cudaStream_t s) = 0;
  virtual void after(int kc, cudaStream_t s) = 0;
  virtual ~LaunchHook() {}
};

cudaError_t set_kernel_attributes();
cudaError_t set_p2_attributes();   // kernels_p2.cu
cudaError_t set_fr_attributes();   // kernels_fr.cu
cudaError_t launch_group_fr(int cfg, const DevPlan& d, const int32_t* list, int count, int R,
                            int Rp, const float* x, float* P, float* fe_con, int ldf,
                            uint8_t* done, cudaStream_t s);
size_t fr_smem_bytes(int cfg);

// Factored root forms (kernels_fr.cu, kernels_corner.cu).  With phi = pi j/N,
// N = L + 1, a root j = 1..J uses
//   form 0 (4j <= N):            u = 1 - i y t,  t = tan phi
//   form 1 (N < 4j, 50j <= 21N):  u = y t + i,   t = tan phi  (t <= 3.9)
//   form 2 (otherwise):           u = y + i t,   t = cot phi
// (3 FP32 operations per complex product in forms 0 and 1, 4 in form 2).
__host__ __device__ inline int fr_roots_form0(int L) { return (L + 1) / 4; }
__host__ __device__ inline int fr_roots_form01(int L) {
  const int J = (L + 1) / 2, n = 21 * (L + 1) / 50;
  return n < J ? n : J;
}
// Tail cutoff of the DFT root sums (Sec. 2.3's expansion evaluated at the
// roots w^j, j = 1..J).  With a = 1 - y^2 a literal's factor has
// |alpha + beta w^j|^2 = 1 - a s_j, s_j = sin^2(pi j / (L + 1)).  Since
// -ln(1 - x) >= x + x^2/2 + x^3/3 + x^4/4 on [0, 1], a product over all
// literals, or over all but one, has modulus at most exp(-B(s_j)) with
//   B(s) = 1/2 sum_{m=1..4} s^m (A_m - a_max^m) / m,   A_m = sum_i a_i^m
// (leaving out one literal removes at most the terms of the largest a, and
// literals at +-1 have a = 0).  The DFT coefficients of a +-1 spectrum and
// their derivative versions are at most 2 in modulus, so the roots with
// B(s_j) >= T = ln(2J / 2^-24) add at most 2^-24 in total to FE and to
// every partial; they are skipped.  (The first version used only the m = 1
// term with a_max <= 1: 1 - x <= e^-x.)
constexpr float kTailLogInvEps = 16.64f;   // >= 24 ln 2
struct TailSums {
  float a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f, amax = 0.f;
  __device__ __forceinline__ void add(float y) {
    const float a = fmaf(-y, y, 1.f), b = a * a;
    a1 += a;
    a2 += b;
    a3 = fmaf(b, a, a3);
    a4 = fmaf(b, b, a4);
    amax = fmaxf(amax, a);
  }
  // combine the sums of the lanes of an aligned group of G lanes (xor tree)
  __device__ __forceinline__ void group_reduce(int G) {
    for (int d = 1; d < G; d <<= 1) {
      a1 += __shfl_xor_sync(0xffffffffu, a1, d);
      a2 += __shfl_xor_sync(0xffffffffu, a2, d);
      a3 += __shfl_xor_sync(0xffffffffu, a3, d);
      a4 += __shfl_xor_sync(0xffffffffu, a4, d);
      amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, d));
    }
  }
};
// Roots 1..jc to evaluate (jc <= J).  The FP32 sums of up to 1024 terms are
// within 2^-14 relative, covered by shrinking each A_m by 2^-13.  B is
// increasing and convex on [0, 1], so Newton's method started right of the
// root s* of B(s) = T (at the root of the m = 1 term, or at 1) stays right of
// it; the result is widened by 2^-12 against rounding, and the index by one.
__device__ __forceinline__ int tail_roots(const TailSums& t, int L, int J, float T) {
  const float sh = 1.f - 0x1p-13f;
  const float am = t.amax, am2 = am * am;
  const float b0 = 0.5f * fmaxf(0.f, fmaf(t.a1, sh, -am));
  const float b1 = 0.25f * fmaxf(0.f, fmaf(t.a2, sh, -am2));
  const float b2 = (1.f / 6.f) * fmaxf(0.f, fmaf(t.a3, sh, -am2 * am));
  const float b3 = 0.125f * fmaxf(0.f, fmaf(t.a4, sh, -am2 * am2));
  auto B = [&](float s) { return s * fmaf(s, fmaf(s, fmaf(s, b3, b2), b1), b0); };
  auto dB = [&](float s) {
    return fmaf(s, fmaf(s, fmaf(s, 4.f * b3, 3.f * b2), 2.f * b1), b0);
  };
  if (!(b0 > 0.f) || B(1.f) < T) return J;
  float s = fminf(1.f, T / b0);
#pragma unroll
  for (int it = 0; it < 3; ++it) s -= (B(s) - T) / dB(s);
  s = fminf(1.f, s * (1.f + 0x1p-12f));
  return min(J, (int)ceilf(asinf(sqrtf(s)) * (float)(L + 1) * 0.318309886f) + 1);
}

// A partial row entry: written once per step and read once, by the
// accumulate kernel; evict-first (st.global.cs) so that the partials do not
// push the point array x, which the FE kernels gather, out of L2.
__device__ __forceinline__ void st_partial(float* p, float v) { __stcs(p, v); }

// Asynchronous global -> shared copies of 4 bytes (no register round trip):
// issue, close a group, wait until at most N groups are pending.  A thread
// sees its own copies after the wait.
__device__ __forceinline__ void cp_async4(float* smem, const float* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
// 16 bytes; both addresses 16-byte aligned
__device__ __forceinline__ void cp_async16(float* smem, const float* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int F>
__device__ __forceinline__ void fr_uinit(float& qr, float& qi, float y, float t) {
  if constexpr (F == 0) {
    qr = 1.f;
    qi = -y * t;
  } else if constexpr (F == 1) {
    qr = y * t;
    qi = 1.f;
  } else {
    qr = y;
    qi = t;
  }
}
// (qr + i qi) *= u_F(y)
template <int F>
__device__ __forceinline__ void fr_umul(float& qr, float& qi, float y, float t) {
  if constexpr (F == 0) {
    const float w = y * t;
    const float nr = fmaf(qi, w, qr), ni = fmaf(-qr, w, qi);
    qr = nr;
    qi = ni;
  } else if constexpr (F == 1) {
    const float w = y * t;
    const float nr = fmaf(qr, w, -qi), ni = fmaf(qi, w, qr);
    qr = nr;
    qi = ni;
  } else {
    const float nr = fmaf(qr, y, -qi * t), ni = fmaf(qi, y, qr * t);
    qr = nr;
    qi = ni;
  }
}
// The corner pass (kernels_corner.cu): runs before the dense factored kernel
// of buckets whose configuration has >= kCornerMinSlots slots.
constexpr int kCornerMinSlots = 32;
// per-(constraint, tile) flag values: open (the next pass may try), done
// (partials written; later passes and the dense kernel skip it), dense
// (left to the dense kernel), low (the power-sum pass wrote the terms of the
// roots 1..js1 of kernels_series.cu; the dense kernel adds the others)
constexpr uint8_t kTileOpen = 0, kTileDone = 1, kTileDense = 2, kTileLow = 3;
// In the workspace the flags (max(1, m) x RT bytes) are followed, 256-byte
// aligned, by the Chebyshev pass's terms of the low tiles: per constraint
// slot (SerInfo::slot) kSeriesK1 + 1 rows of Rp floats, D_0 .. D_{K1-1} and
// then FE - b0 of the low roots, which the dense factored kernel adds.
inline float* ser_terms(const DevPlan& d, uint8_t* done, int RT) {
  uintptr_t a = reinterpret_cast<uintptr_t>(done) + (size_t)(d.m > 1 ? d.m : 1) * RT;
  a = (a + 255) & ~(uintptr_t)255;
  return reinterpret_cast<float*>(a);
}
cudaError_t set_corner_attributes();
size_t corner_smem_bytes(int maxL, int gc);
// group = false: only the one-thread pass (before the direct-form kernel)
cudaError_t launch_dft_corner(const DevPlan& d, const int32_t* list, int count, int maxL, int R,
                              int Rp, const float* x, float* P, float* fe_con, int ldf,
                              uint8_t* done, cudaStream_t s, bool group = true);
// The direct-form DFT kernel runs after the one-thread corner pass for
// buckets longer than the pass's capacity (kDirectCornerMinL), skipping the
// tiles it finished; shorter buckets go to the direct kernel alone.
constexpr int kDirectCornerMinL = 17;
// The power-sum pass (kernels_series.cu): after the corner passes, on the
// tiles they left, for constraints of kSeriesMinL literals or more.
cudaError_t set_series_attributes();
cudaError_t launch_dft_series(const DevPlan& d, const int32_t* list, int count, int maxL, int R,
                              int Rp, const float* x, float* P, float* fe_con, int ldf,
                              uint8_t* done, cudaStream_t s);
cudaError_t launch_group_p2(int cfg, const DevPlan& d, const int32_t* list, int count, int R,
                            int Rp, const float* x, float* P, float* fe_con, int ldf,
                            cudaStream_t s);
size_t group_smem_bytes(int cfg);

cudaError_t launch_init(const DevPlan& d, int R, uint64_t seed, int64_t r_off, float* x,
                        cudaStream_t s, LaunchHook* h);
// per-restart convergence tracking and refills (kernels.cu)
cudaError_t launch_track_reset(int R, int32_t* trk, cudaStream_t s);
cudaError_t launch_track_step(const DevPlan& d, int R, int step, const int32_t* nsat,
                              int32_t* trk, cudaStream_t s);
cudaError_t launch_refill(const DevPlan& d, int R, uint64_t seed, int64_t r_off, uint64_t gen,
                          int patience, int32_t* trk, float* x, int32_t* count, cudaStream_t s);
cudaError_t launch_unsat_hist(const DevPlan& d, int R, const int32_t* nsat, int32_t* hist,
                              cudaStream_t s);
// per-restart movement of a step and the first step it fell to tol
cudaError_t launch_movement(const DevPlan& d, int R, const float* xp, const float* x,
                            float* maxdelta, cudaStream_t s);
cudaError_t launch_track_conv(int R, const float* maxdelta, float tol, int step, int32_t* conv,
                              cudaStream_t s);

// adaptive constraint weighting (kernels.cu): per-constraint statistics over
// the restarts, the weight update, and writing weights into the plan's items
// scratch: at least m * ceil(R/32) * 8 bytes, 4-byte aligned
cudaError_t launch_con_stats(const DevPlan& d, int R, int Rp, const uint32_t* bits,
                             const float* P, float* scratch, double* gnorm, int32_t* unsat,
                             cudaStream_t s);
cudaError_t launch_set_weights(const DevPlan& d, const float* w, cudaStream_t s);
cudaError_t launch_reweight(const DevPlan& d, int R, const double* gnorm, const int32_t* unsat,
                            double eta, double kappa, double w_max, float* w_out, double* gbar,
                            cudaStream_t s);

// FE + literal partials: P[row * Rp + r] = w_c s_e dFE_c/dy_e (row = the
// literal's variable-major row), and (if fe_con) fe_con[c * ldf + r] = FE_c.
// done: workspace flags [m][ceil(R/32)], one per (constraint, restart tile),
// set by the corner pass of the factored DFT kernels (see launch_group).
cudaError_t launch_fe(const DevPlan& d, int R, int Rp, const float* x, float* P, float* fe_con,
                      int ldf, uint8_t* done, cudaStream_t s, LaunchHook* h);

// The FE stage as independent units (thread-path classes, then lane-group
// buckets); units write disjoint partial rows and may run concurrently.
constexpr int kNumFeUnits = kNumThreadCls + kNumBuckets;
bool fe_unit_active(const DevPlan& d, int unit);
cudaError_t launch_fe_unit(const DevPlan& d, int unit, int R, int Rp, const float* x, float* P,
                           float* fe_con, int ldf, uint8_t* done, cudaStream_t s, LaunchHook* h);

// The whole step loop as one launch; only for problems whose FE work is all
// on the short closed-form path.  When a restart tile's x, partial rows and
// bitset fit in kTileLoopMaxSmem bytes of shared memory, one CTA per tile
// runs the loop with no grid barrier (k_tile_loop); otherwise one
// cooperative launch over all items with bounded grid barriers.
bool persistent_eligible(const DevPlan& d);
constexpr size_t kTileLoopMaxSmem = 220 * 1024;
cudaError_t launch_persistent(const DevPlan& d, int R, int Rp, float* x, float lr, int n_steps,
                              float* P, uint32_t* bits, int32_t* rpart_n, double* rpart_w,
                              int32_t* nsat, double* wsat, unsigned* bar, int* err,
                              cudaStream_t s);

// The grid barrier alone (see cls_grid_barrier_check).
cudaError_t launch_barrier_check(int rounds, unsigned extra, unsigned spin_limit, unsigned* bar,
                                 int* err, int* passed, cudaStream_t s);

// fe_con[c * ldf + r] = b0 for constraints whose expansion is constant.
cudaError_t launch_fe_const(const DevPlan& d, int R, float* fe_con, int ldf, cudaStream_t s);

// One lane-group launch over an explicit constraint list (the autotuner).
cudaError_t launch_group(int cfg, const DevPlan& d, const int32_t* list, int count, int maxL, int maxJ,
                         int R, int Rp, const float* x, float* P, float* fe_con, int ldf,
                         uint8_t* done, cudaStream_t s);

// g[v,r] = sum of rows voff[v]..voff[v+1]-1 of P; optional grad output;
// optional projected step of x in place and bitset of the new x.
cudaError_t launch_accum_step(const DevPlan& d, int R, int Rp, const float* P, float* x,
                              float lr, bool do_step, float* grad_out, uint32_t* bits,
                              cudaStream_t s, LaunchHook* h);

// x <- clamp(x - lr*grad) for free variables, optional bitset.
cudaError_t launch_pgd(const DevPlan& d, int R, float* x, const float* grad, float lr,
                       uint32_t* bits, cudaStream_t s, LaunchHook* h);

// bitset of x (x < 0).
cudaError_t launch_round(const DevPlan& d, int R, const float* x, uint32_t* bits,
                         cudaStream_t s, LaunchHook* h);

// Exact satisfaction counts from the bitset, two-stage (chunks, then order).
cudaError_t launch_score(const DevPlan& d, int R, int Rp, const uint32_t* bits,
                         int32_t* nsat_part, double* wsat_part, int32_t* nsat, double* wsat,
                         cudaStream_t s, LaunchHook* h);

// out[v*R + r] = sc[r] * g[v*R + r] (vector-Jacobian product of obj[r]).
cudaError_t launch_restart_scale(int n, int R, const float* g, const float* sc, float* out,
                                 cudaStream_t s, LaunchHook* h);

// obj[r] = sum_c w_c fe_con[c*ldf + r] in FP64 (fixed order), rounded to FP32.
cudaError_t launch_obj(const DevPlan& d, int R, int Rp, int nch, int chunk, const float* fe_con,
                       int ldf, double* part, float* obj, cudaStream_t s, LaunchHook* h);

}  // namespace cls
