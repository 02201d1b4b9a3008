// plan.h -- data layout shared by the host problem builder (plan.cpp) and
// the sm_103a kernels (kernels.cu).  Plain structs only; no CUDA types.
#pragma once
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

namespace cls {

// 16-byte table entry (matches CUDA float4 layout).
struct F4 {
  float x, y, z, w;
};

// One literal: its variable and its row in variable-major order; the top bit
// of `dst` is set when the literal is negated (sign -1).
struct LitRec {
  int32_t var;
  int32_t dst;
};
constexpr int32_t kNegBit = int32_t(0x80000000u);

// FE+gradient work description of one constraint.
//   Literal values y_i = s_i x_{v_i} enter each "root" j as the factor
//     F_ij = (A_j + y_i B_j) + i (C_j - y_i C_j)
//   root table entry (A, B, C, 0).  For a DFT root (Sec. 2.3: evaluation at
//   the L+1 roots of unity w^j) A = (1+cos)/2, B = (1-cos)/2, C = sin/2 of
//   2 pi j/(L+1), with A rounded as 1 - B in FP32 so that A + B == 1 exactly;
//   i.e. F = alpha_i + beta_i w^j with alpha = (1+y)/2 = P[literal false],
//   beta = (1-y)/2 = P[literal true]; every factor has modulus <= 1.  Real
//   roots (C = 0) give the closed-form products of OR/XOR/NAE: alpha
//   (A=B=1/2), beta (A=1/2, B=-1/2), y (A=0, B=1).
//   coefficient entry (b'.re, b'.im, c'.re, c'.im):
//     FE       = b0 + Re sum_j b'_j prod_i F_ij
//     dFE/dy_i =      Re sum_j c'_j prod_{l != i} F_lj,   c'_j = b'_j (B_j - i C_j)
struct FeItem {
  int32_t lit0;      // first literal (constraint order)
  int32_t L;         // number of literals
  int32_t J;         // number of roots
  int32_t root_off;  // first root-table entry
  int32_t coef_off;  // first coefficient-table entry
  float b0;          // constant term
  float w;           // constraint weight
  int32_t c;         // constraint index
};

// Satisfaction test of one constraint on t = # true literals.
//   mode 0: lo <= t <= hi;  mode 1: t odd;  mode 2: table bit (satbits[lo + t])
struct ScoreItem {
  int32_t lit0;
  int32_t L;
  int32_t mode;
  int32_t lo;
  int32_t hi;
  float w;
  int32_t c;
  int32_t pad;
};

// Lane-group kernel configurations: G lanes share one (constraint, restart),
// each lane holds up to Q literals (L <= G*Q); CPLX = DFT roots vs real
// roots; YS = literal values re-read from shared memory instead of kept in
// registers (fewer registers, more resident warps).  The same list is
// instantiated in kernels.cu.  X(id, G, Q, CPLX, YS)
#define CLS_GROUP_CONFIGS(X) \
  X(0, 8, 1, 1, 0)           \
  X(1, 8, 2, 1, 0)           \
  X(2, 8, 4, 1, 0)           \
  X(3, 8, 6, 1, 0)           \
  X(4, 8, 8, 1, 0)           \
  X(5, 8, 12, 1, 0)          \
  X(6, 8, 16, 1, 0)          \
  X(7, 16, 4, 1, 0)          \
  X(8, 16, 6, 1, 0)          \
  X(9, 16, 8, 1, 0)          \
  X(10, 16, 10, 1, 0)        \
  X(11, 16, 12, 1, 0)        \
  X(12, 16, 16, 1, 0)        \
  X(13, 16, 20, 1, 0)        \
  X(14, 32, 8, 1, 0)         \
  X(15, 32, 10, 1, 0)        \
  X(16, 32, 12, 1, 0)        \
  X(17, 32, 16, 1, 0)        \
  X(18, 32, 24, 1, 0)        \
  X(19, 32, 32, 1, 0)        \
  X(20, 8, 8, 1, 1)          \
  X(21, 8, 12, 1, 1)         \
  X(22, 8, 16, 1, 1)         \
  X(23, 16, 8, 1, 1)         \
  X(24, 16, 10, 1, 1)        \
  X(25, 16, 12, 1, 1)        \
  X(26, 16, 14, 1, 1)        \
  X(27, 16, 16, 1, 1)        \
  X(28, 16, 18, 1, 1)        \
  X(29, 16, 20, 1, 1)        \
  X(30, 16, 24, 1, 1)        \
  X(31, 32, 10, 1, 1)        \
  X(32, 32, 12, 1, 1)        \
  X(33, 32, 14, 1, 1)        \
  X(34, 32, 16, 1, 1)        \
  X(35, 32, 20, 1, 1)        \
  X(36, 32, 24, 1, 1)        \
  X(37, 32, 32, 1, 1)        \
  X(38, 8, 24, 1, 1)         \
  X(39, 8, 32, 1, 1)         \
  X(40, 8, 40, 1, 1)         \
  X(41, 32, 2, 0, 0)         \
  X(42, 32, 4, 0, 0)         \
  X(43, 32, 8, 0, 0)         \
  X(44, 32, 16, 0, 0)        \
  X(45, 32, 32, 0, 0)        \
  X(46, 16, 4, 0, 0)         \
  X(47, 16, 8, 0, 0)         \
  X(48, 16, 16, 0, 0)
// DFT roots processed in pairs with packed FP32x2 arithmetic (CPLX = 2),
// instantiated in kernels_p2.cu.
#define CLS_P2_CONFIGS(X) \
  X(49, 8, 4, 2, 0)   \
  X(50, 8, 8, 2, 0)   \
  X(51, 8, 8, 2, 1)   \
  X(52, 8, 16, 2, 1)  \
  X(53, 16, 4, 2, 0)  \
  X(54, 16, 8, 2, 0)  \
  X(55, 16, 8, 2, 1)  \
  X(56, 16, 10, 2, 1) \
  X(57, 16, 12, 2, 1) \
  X(58, 16, 14, 2, 1) \
  X(59, 16, 16, 2, 1) \
  X(60, 16, 18, 2, 1) \
  X(61, 16, 20, 2, 1) \
  X(62, 32, 8, 2, 1)  \
  X(63, 32, 10, 2, 1) \
  X(64, 32, 12, 2, 1) \
  X(65, 32, 14, 2, 1) \
  X(66, 32, 16, 2, 1) \
  X(67, 32, 20, 2, 1) \
  X(68, 8, 2, 2, 0)   \
  X(69, 8, 1, 2, 0)
// DFT roots in factored form (CPLX = 3), instantiated in kernels_fr.cu: per
// root the factor alpha + beta w^j is written z_j u_j(y) with a root constant
// z_j and u = 1 - i y tan(phi) (phi = pi j/(L+1) <= pi/4) or u = y + i cot(phi)
// (phi > pi/4): 3 or 4 FP32 operations per complex product instead of 6.
#define CLS_FR_CONFIGS(X) \
  X(70, 8, 1, 3, 0)   \
  X(71, 8, 2, 3, 0)   \
  X(72, 8, 4, 3, 0)   \
  X(73, 8, 6, 3, 0)   \
  X(74, 8, 8, 3, 0)   \
  X(75, 8, 12, 3, 0)  \
  X(76, 8, 16, 3, 0)  \
  X(77, 16, 8, 3, 0)  \
  X(78, 16, 10, 3, 0) \
  X(79, 16, 12, 3, 0) \
  X(80, 16, 14, 3, 0) \
  X(81, 16, 16, 3, 0) \
  X(82, 16, 18, 3, 0) \
  X(83, 16, 20, 3, 0) \
  X(84, 8, 20, 3, 0)  \
  X(85, 8, 24, 3, 0)  \
  X(86, 16, 24, 3, 1) \
  X(87, 16, 16, 3, 1) \
  X(88, 16, 20, 3, 1) \
  X(89, 32, 12, 3, 0) \
  X(90, 32, 14, 3, 1) \
  X(91, 32, 16, 3, 1) \
  X(92, 32, 20, 3, 1) \
  X(93, 32, 24, 3, 1) \
  X(94, 32, 32, 3, 1) \
  X(95, 8, 32, 3, 1)  \
  X(96, 16, 28, 3, 1) \
  X(97, 32, 16, 3, 0) \
  X(98, 16, 12, 3, 1)
constexpr int kNumGroupCfg = 99;
// Slot counts Q used by the factored configurations.  For a DFT root the
// root table's 4th entry holds t = tan(phi) (phi <= pi/4) or t = cot(phi),
// rounded to FP32, and z' = 1/(1 - i t) or 1/(1 + i t) is the root constant
// that makes a padding slot (y = 1) exactly neutral for that rounded t; its
// powers are formed in FP64 and rounded once.
// Power-sum (series) pass for the low roots of long DFT constraints.  With
// phi = pi j / (L + 1), every factor is alpha + beta w^j = h_j (1 + q_j y),
// h_j = (1 + w^j)/2, q_j = -i tan phi, and with r_j = -q_j / (1 + sqrt(1 -
// q_j^2)), |r_j| = tan(phi/2), the Chebyshev generating function gives on
// all of [-1, 1]
//   log(1 + q y) = -log(1 + r^2) - 2 sum_{k>=1} r^k T_k(y) / k,
//   d/dy log(1 + q y) = sum_{k>=0} E_k U_k(y),   E_k = -2 r^(k+1).
// A root is in the range of K terms when both truncation bounds (the log
// series over L literals, the derivative series relative to |dlog F/dy| >=
// sin phi) are at most 2^-24.  Per length L the table holds, for root j =
// 1..js1, kSerRow float4: {Re C_j, Im C_j and theta_j as uint32 fractions of
// a turn, 0} with C_j = log h_j - log(1 + r_j^2), then {Re E_2m, Re E_2m+1,
// Im E_2m, Im E_2m+1} for m = 0..K1/2 - 1 (real and imaginary parts of a
// pair of terms side by side, for packed FP32x2 products).
constexpr int kSeriesK0 = 18, kSeriesK1 = 26;
constexpr int kSeriesMaxRoots = 96;   // rows a block stages
constexpr int kSeriesMinL = 64;       // shorter constraints keep the root products
constexpr int kSerRow = 1 + kSeriesK1 / 2;
// Shorter term counts the pass may take when a tile's roots fit their range
// (js of 12, 14, 16 and 22 terms, below and between kSeriesK0 and kSeriesK1).
constexpr int kNumSeriesKx = 4;
constexpr int kSeriesKx[kNumSeriesKx] = {12, 14, 16, 22};
struct SerInfo {
  int32_t off;    // first row in ser_tab, -1 if the constraint has none
  int32_t js0;    // roots in range of kSeriesK0 terms
  int32_t js1;    // roots in range of kSeriesK1 terms
  int32_t slot;   // this constraint's rows of saved low-root terms (workspace)
  int16_t jsx[kNumSeriesKx];   // roots in range of kSeriesKx[i] terms
};

// roots in range of the power-sum pass with K terms (plan.cpp)
int series_roots(int L, int K);

constexpr int kNumFrQ = 14;
constexpr int kFrQ[kNumFrQ] = {1, 2, 4, 6, 8, 10, 12, 14, 16, 18, 20, 24, 28, 32};
// Configuration id of the restart-parallel checkpointed kernel for real-root
// (closed-form) constraints of any length; valid only for real buckets.
constexpr int kCkptCfg = 100;
constexpr int kCkptInterval = 16;   // literals between stored prefix products
struct GroupCfg {
  int G, Q, cplx, ys;
};
extern const GroupCfg kGroupCfg[kNumGroupCfg];

// Thread-path (one thread per (constraint, restart)) length classes.
constexpr int kNumThreadCls = 3;
constexpr int kThreadMaxL[kNumThreadCls] = {8, 16, 24};
constexpr int kThreadTiles = 4;   // restart tiles (of 32) per warp

// Score path: consecutive constraints are grouped into ranges of about this
// many literals; one warp scores one range for 32 restarts.
constexpr int kScoreRangeLits = 256;

// Fixed entries of the root table (real roots).
constexpr int kRootAlpha = 0;  // alpha, then beta at 1 (NAE uses both)
constexpr int kRootBeta = 1;
constexpr int kRootY = 2;
constexpr int kCoefOr = 0;     // (2, 0, 1, 0)
constexpr int kCoefXor = 1;    // (1, 0, 1, 0)
constexpr int kCoefNae = 2;    // (2, 0, 1, 0), (2, 0, -1, 0); the second alone: not all true
constexpr int kCoefXnor = 4;   // (-1, 0, -1, 0): FE = -prod y
constexpr int kCoefNor = 5;    // (-2, 0, -1, 0): FE = 1 - 2 prod alpha (no literal true)
constexpr int kCoefAllTrue = 6;  // (-2, 0, 1, 0): FE = 1 - 2 prod beta (every literal true)

// Problem build flags.
constexpr uint32_t kFlagSimplifyFixed = 1;   // fold pinned variables into the spectra

// Length buckets of the lane-group paths: one launch per non-empty bucket;
// the tuning maps each bucket to a configuration.
constexpr int kNumDftBuckets = 19;
constexpr int kDftBucketMax[kNumDftBuckets] = {8,   16,  32,  48,  64,  96,  128,
                                               160, 192, 224, 256, 288, 320, 384,
                                               448, 512, 640, 768, 1024};
constexpr int kNumRealBuckets = 6;
constexpr int kRealBucketMax[kNumRealBuckets] = {32, 64, 128, 256, 512, 1024};

struct Tuning {
  int dft[kNumDftBuckets];
  int real[kNumRealBuckets];
};
Tuning default_tuning();
bool tuning_valid(const Tuning& t, std::string* msg);

struct HostPlan {
  int32_t n = 0, m = 0;
  int64_t nnz = 0;
  uint32_t flags = 0;
  std::vector<LitRec> lit;        // all literals, constraint order; dst = row among all
  std::vector<int32_t> voff;      // n+1: rows of variable v among all literals
  std::vector<LitRec> fe_lit;     // literals entering FE (all, or the free ones)
  std::vector<int32_t> fe_voff;   // n+1: rows of variable v in the partial buffer
  int64_t nnz_fe = 0;
  std::vector<FeItem> fe;         // m (constraint order)
  std::vector<ScoreItem> score;          // constraint order
  std::vector<int32_t> score_ranges;     // constraint boundaries of the ranges
  std::vector<uint32_t> satbits;  // truth tables of SPECTRUM constraints
  std::vector<F4> root_tab, coef_tab;
  // factored DFT roots: per root-table entry r and per slot count Q of the
  // factored configurations (kFrQ[q]), zpow_tab[r * kNumFrQ + q] =
  // {z'^Q, z'^(Q-1)} (see kFrQ)
  std::vector<F4> zpow_tab;
  // spectra of the DFT constraints (after folding), +-1 per t = 0..L, at
  // spec_off[c] (-1 for the others); the corner passes' exact small DP
  std::vector<int8_t> spec_tab;
  std::vector<int32_t> spec_off;
  // power-sum tables of the DFT constraints (see kSeriesK0), per constraint
  std::vector<F4> ser_tab;
  std::vector<SerInfo> ser_info;
  int32_t n_ser_slots = 0;        // constraints with a power-sum table
  std::vector<FeItem> thread_items[kNumThreadCls];   // items in launch order
  // lane-group buckets: [0, kNumDftBuckets) DFT, then real
  std::vector<int32_t> bucket_list[kNumDftBuckets + kNumRealBuckets];
  int bucket_cfg[kNumDftBuckets + kNumRealBuckets] = {};
  std::vector<int32_t> ctype, kthr;   // per constraint: type and threshold (0 if none)
  std::vector<float> weight;          // per constraint
  std::vector<int32_t> const_list;    // constraints whose expansion is a constant
  std::vector<uint8_t> fixed;     // n (empty = none)
  std::vector<float> fixed_val;   // n
  Tuning tuning;
  int64_t dft_roots = 0, dft_lroots = 0;
  int64_t n_thread = 0, n_group_real = 0, n_group_dft = 0;
};

// Validates and builds the plan. Returns 0 or -1 (msg set).
int build_plan(int32_t n, int32_t m, const int32_t* offsets, const int32_t* lit_var,
               const int8_t* lit_sign, const int32_t* type, const int32_t* k,
               const float* weight, const int8_t* spectra, const uint8_t* fixed,
               const float* fixed_val, uint32_t flags, bool validate_only, HostPlan* out,
               std::string* msg);

// (Re)split the FE work lists for a tuning.
void assign_groups(HostPlan* plan, const Tuning& tun);

}  // namespace cls
