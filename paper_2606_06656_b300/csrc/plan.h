// plan.h -- data layout shared by the host problem builder (plan.cpp) and
// the sm_103a kernels (kernels.cu).  Plain structs only; no CUDA types.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace cls {

// 16-byte table entry (matches CUDA float4 layout).
struct F4 {
  float x, y, z, w;
};

// FE+gradient work description of one constraint.
//   Literal values y_i = s_i x_{v_i} enter each "root" j as the factor
//     F_ij = (A_j + y_i B_j) + i (C_j - y_i C_j)
//   root table entry (A, B, C, 0).  For a DFT root (Sec. 2.3: evaluation at
//   the L+1 roots of unity w^j) A = (1+cos)/2, B = (1-cos)/2, C = sin/2 of
//   2 pi j/(L+1) (A rounded as 1 - B in FP32, so A + B == 1 exactly), i.e. F = alpha_i + beta_i w^j with alpha = (1+y)/2 =
//   P[literal false], beta = (1-y)/2 = P[literal true]; every factor has
//   modulus <= 1.  Real roots (C = 0) give the closed-form products of
//   OR/XOR/NAE: alpha (A=B=1/2), beta (A=1/2, B=-1/2), y (A=0, B=1).
//   coefficient entry (b'.re, b'.im, c'.re, c'.im):
//     FE      = b0 + Re sum_j b'_j prod_i F_ij
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
  int32_t pad0, pad1;
};

// Lane-group kernel configurations: G lanes share one (constraint, restart),
// each lane holds up to Q literals (L <= G*Q); CPLX = DFT roots vs real roots.
// The same list is instantiated in kernels.cu.
#define CLS_GROUP_CONFIGS(X) \
  X(0, 8, 1, 1)              \
  X(1, 8, 2, 1)              \
  X(2, 8, 4, 1)              \
  X(3, 8, 8, 1)              \
  X(4, 16, 4, 1)             \
  X(5, 16, 8, 1)             \
  X(6, 16, 12, 1)            \
  X(7, 16, 16, 1)            \
  X(8, 32, 4, 1)             \
  X(9, 32, 8, 1)             \
  X(10, 32, 12, 1)           \
  X(11, 32, 16, 1)           \
  X(12, 32, 24, 1)           \
  X(13, 32, 32, 1)           \
  X(14, 32, 2, 0)            \
  X(15, 32, 4, 0)            \
  X(16, 32, 8, 0)            \
  X(17, 32, 16, 0)           \
  X(18, 32, 32, 0)           \
  X(19, 8, 16, 1)            \
  X(20, 16, 20, 1)
constexpr int kNumGroupCfg = 21;
struct GroupCfg {
  int G, Q, cplx;
};
extern const GroupCfg kGroupCfg[kNumGroupCfg];

// Thread-path (one thread per (constraint, restart)) length classes.
constexpr int kThreadMaxL0 = 8;
constexpr int kThreadMaxL1 = 32;

// Fixed entries of the root table (real roots).
constexpr int kRootAlpha = 0;  // alpha, then beta at 1 (NAE uses both)
constexpr int kRootBeta = 1;
constexpr int kRootY = 2;
constexpr int kCoefOr = 0;     // (2, 0, 1, 0)
constexpr int kCoefXor = 1;    // (1, 0, 1, 0)
constexpr int kCoefNae = 2;    // (2, 0, 1, 0), (2, 0, -1, 0)

struct HostPlan {
  int32_t n = 0, m = 0;
  int64_t nnz = 0;
  std::vector<int32_t> lit_var;   // constraint order
  std::vector<float> lit_sgn;     // +-1
  std::vector<int32_t> lit_dst;   // row of the literal in variable-major order
  std::vector<int32_t> voff;      // n+1: rows of variable v
  std::vector<FeItem> fe;         // m
  std::vector<ScoreItem> score;   // m
  std::vector<uint32_t> satbits;  // truth tables of SPECTRUM constraints
  std::vector<F4> root_tab, coef_tab;
  std::vector<int32_t> thread_list[2];             // MAXL 8 / 32
  std::vector<int32_t> group_list[kNumGroupCfg];   // per config, L descending
  std::vector<uint8_t> fixed;     // n (empty = none)
  std::vector<float> fixed_val;   // n
  int64_t dft_roots = 0, dft_lroots = 0;
  int64_t n_thread = 0, n_group_real = 0, n_group_dft = 0;
};

// Length -> group configuration map (index into kGroupCfg), per kind.
struct Tuning {
  // upper length bounds and config ids, ascending bounds
  std::vector<std::pair<int, int>> dft, real;
};
Tuning default_tuning();

// Validates and builds the plan. Returns 0 or -1 (msg set).
int build_plan(int32_t n, int32_t m, const int32_t* offsets, const int32_t* lit_var,
               const int8_t* lit_sign, const int32_t* type, const int32_t* k,
               const float* weight, const int8_t* spectra, const uint8_t* fixed,
               const float* fixed_val, const Tuning& tun, bool validate_only,
               HostPlan* out, std::string* msg);

// Re-split the FE work lists for a different tuning (same plan).
void assign_groups(HostPlan* plan, const Tuning& tun);

}  // namespace cls
