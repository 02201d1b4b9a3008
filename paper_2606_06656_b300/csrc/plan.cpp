// plan.cpp -- host-side problem build: validation, spectra, Fourier tables
// in FP64, the variable-major transpose of the literal list and the kernel
// work lists.  Runs once per problem (cls_problem_create).
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <numeric>

namespace cls {

const GroupCfg kGroupCfg[kNumGroupCfg] = {
#define CLS_CFG_ENTRY(id, G, Q, C, Y) {G, Q, C, Y},
    CLS_GROUP_CONFIGS(CLS_CFG_ENTRY) CLS_P2_CONFIGS(CLS_CFG_ENTRY) CLS_FR_CONFIGS(CLS_CFG_ENTRY)
#undef CLS_CFG_ENTRY
};

Tuning default_tuning() {
  Tuning t;
  // measured on a B300 (autotuner, mixed and long cardinality workloads):
  // the factored-root kernel from 17 literals up
  const int dft[kNumDftBuckets] = {0,  1,  72, 73, 74, 75, 76, 84, 85, 80,
                                   87, 82, 83, 86, 96, 91, 92, 93, 94};
  const int real[kNumRealBuckets] = {46, kCkptCfg, kCkptCfg, kCkptCfg, kCkptCfg, kCkptCfg};
  for (int b = 0; b < kNumDftBuckets; ++b) t.dft[b] = dft[b];
  for (int b = 0; b < kNumRealBuckets; ++b) t.real[b] = real[b];
  return t;
}

bool tuning_valid(const Tuning& t, std::string* msg) {
  for (int b = 0; b < kNumDftBuckets + kNumRealBuckets; ++b) {
    const bool dft = b < kNumDftBuckets;
    const int id = dft ? t.dft[b] : t.real[b - kNumDftBuckets];
    const int maxL = dft ? kDftBucketMax[b] : kRealBucketMax[b - kNumDftBuckets];
    if (!dft && id == kCkptCfg) continue;
    if (id < 0 || id >= kNumGroupCfg) {
      if (msg) *msg = "configuration id out of range";
      return false;
    }
    const GroupCfg& g = kGroupCfg[id];
    if ((g.cplx != 0) != dft || g.G * g.Q < maxL) {
      if (msg)
        *msg = "configuration " + std::to_string(id) + " cannot serve bucket " +
               std::to_string(b) + " (max length " + std::to_string(maxL) + ")";
      return false;
    }
  }
  return true;
}

namespace {

enum { T_OR = 0, T_XOR, T_CARD_GE, T_CARD_LE, T_NAE, T_EO, T_EK, T_AMO, T_SPECTRUM };

// Does constraint (type, L, k) hold with t true literals (Sec. 2.2; Table 2)?
bool holds(int type, int L, int k, int t, const int8_t* spec) {
  switch (type) {
    case T_OR: return t >= 1;
    case T_XOR: return (t & 1) == 1;
    case T_CARD_GE: return t >= k;
    case T_CARD_LE: return t <= k;
    case T_NAE: return t > 0 && t < L;
    case T_EO: return t == 1;
    case T_EK: return t == k;
    case T_AMO: return t <= 1;
    default: return spec[t] == -1;
  }
}

int bucket_of(const int* maxes, int nb, int L) {
  for (int b = 0; b < nb; ++b)
    if (L <= maxes[b]) return b;
  return nb - 1;
}

}  // namespace

void assign_groups(HostPlan* P, const Tuning& tun) {
  for (auto& v : P->thread_items) v.clear();
  for (auto& v : P->bucket_list) v.clear();
  P->const_list.clear();
  P->tuning = tun;
  for (int b = 0; b < kNumDftBuckets; ++b) P->bucket_cfg[b] = tun.dft[b];
  for (int b = 0; b < kNumRealBuckets; ++b) P->bucket_cfg[kNumDftBuckets + b] = tun.real[b];
  P->n_thread = P->n_group_real = P->n_group_dft = 0;
  std::vector<int32_t> thread_c[kNumThreadCls];
  for (int32_t c = 0; c < P->m; ++c) {
    const FeItem& it = P->fe[c];
    if (it.L == 0) {              // constant expansion: no FE work, no partials
      P->const_list.push_back(c);
      continue;
    }
    bool real = it.root_off < 3;  // real roots live at the start of the table
    if (real && it.L <= kThreadMaxL[kNumThreadCls - 1]) {
      int t = 0;
      while (it.L > kThreadMaxL[t]) ++t;
      thread_c[t].push_back(c);
      P->n_thread++;
    } else if (real) {
      P->bucket_list[kNumDftBuckets + bucket_of(kRealBucketMax, kNumRealBuckets, it.L)]
          .push_back(c);
      P->n_group_real++;
    } else {
      P->bucket_list[bucket_of(kDftBucketMax, kNumDftBuckets, it.L)].push_back(c);
      P->n_group_dft++;
    }
  }
  // longest first: expensive blocks are scheduled early (LPT order)
  auto byL = [P](int32_t a, int32_t b) {
    return P->fe[a].L != P->fe[b].L ? P->fe[a].L > P->fe[b].L : a < b;
  };
  for (int t = 0; t < kNumThreadCls; ++t) {
    std::stable_sort(thread_c[t].begin(), thread_c[t].end(), byL);
    for (int32_t c : thread_c[t]) P->thread_items[t].push_back(P->fe[c]);
  }
  for (auto& v : P->bucket_list) std::stable_sort(v.begin(), v.end(), byL);
}

// Roots in range of the power-sum pass with K terms (see kSeriesK0): the
// largest js such that for every root j <= js, with rho = tan(phi/2),
//   L 2 rho^(K+1) / ((K+1)(1 - rho))                          <= 2^-24
//     (the log series summed over L literals, |T_k| <= 1), and
//   2 rho^(K+1) ((K+1)/(1 - rho) + rho/(1 - rho)^2) / sin phi <= 2^-24
//     (the derivative series, |U_k| <= k + 1, relative to its smallest
//     modulus sin phi on [-1, 1]); rho grows with j below the middle root.
int series_roots(int L, int K) {
  const int N = L + 1;
  const double eps = std::ldexp(1.0, -24);
  int js = 0;
  for (int j = 1; 2 * j < N && j <= kSeriesMaxRoots; ++j) {
    const double phi = M_PI * (double)j / (double)N;
    const double rho = std::tan(0.5 * phi);
    const double pk = std::pow(rho, K + 1);
    const double tl = (double)L * 2.0 * pk / ((double)(K + 1) * (1.0 - rho));
    const double td = 2.0 * pk * ((double)(K + 1) / (1.0 - rho) + rho / ((1.0 - rho) * (1.0 - rho))) /
                      std::sin(phi);
    if (tl > eps || td > eps) break;
    js = j;
  }
  return js;
}

// a fraction of a turn as a uint32 (mod 2^32), stored in a float's bits
static float turn_bits(double turns) {
  double f = turns - std::floor(turns);
  uint64_t q = (uint64_t)std::llround(f * 4294967296.0);
  uint32_t u = (uint32_t)(q & 0xffffffffull);
  float out;
  std::memcpy(&out, &u, sizeof(out));
  return out;
}

// Appends the power-sum rows of length L (root j = 1..js1, see kSeriesK0).
static SerInfo series_table(int L, std::vector<F4>& tab) {
  SerInfo si{-1, series_roots(L, kSeriesK0), series_roots(L, kSeriesK1), 0, {0, 0, 0, 0}};
  if (si.js1 == 0) return SerInfo{-1, 0, 0, 0, {0, 0, 0, 0}};
  for (int i = 0; i < kNumSeriesKx; ++i) si.jsx[i] = (int16_t)series_roots(L, kSeriesKx[i]);
  si.off = (int32_t)tab.size();
  const int N = L + 1;
  for (int j = 1; j <= si.js1; ++j) {
    const double th = 2.0 * M_PI * (double)j / (double)N;
    const std::complex<double> w(std::cos(th), std::sin(th));
    const std::complex<double> h = (1.0 + w) / 2.0, q = (1.0 - w) / (1.0 + w);
    const std::complex<double> r = -q / (1.0 + std::sqrt(1.0 - q * q));
    const std::complex<double> Cj = std::log(h) - std::log(1.0 + r * r);
    tab.push_back({(float)Cj.real(), turn_bits(Cj.imag() / (2.0 * M_PI)),
                   turn_bits((double)j / (double)N), 0.f});
    std::complex<double> e = -2.0 * r;                      // E_0
    for (int k = 0; k < kSeriesK1; k += 2) {
      const std::complex<double> e1 = e * r;
      tab.push_back({(float)e.real(), (float)e1.real(), (float)e.imag(), (float)e1.imag()});
      e = e1 * r;
    }
  }
  return si;
}

int build_plan(int32_t n, int32_t m, const int32_t* offsets, const int32_t* lit_var,
               const int8_t* lit_sign, const int32_t* type, const int32_t* kk,
               const float* weight, const int8_t* spectra, const uint8_t* fixed,
               const float* fixed_val, uint32_t flags, bool validate_only, HostPlan* out,
               std::string* msg) {
  auto fail = [msg](const std::string& s) {
    if (msg) *msg = s;
    return -1;
  };
  if (n < 0 || m < 0) return fail("n_vars and n_cons must be >= 0");
  if (m > 0 && (!offsets || !lit_var || !lit_sign || !type))
    return fail("offsets, lit_var, lit_sign and type are required when n_cons > 0");
  if (m > 0 && offsets[0] != 0) return fail("offsets[0] must be 0");
  int64_t nnz = m > 0 ? offsets[m] : 0;
  std::vector<int32_t> seen(n > 0 ? n : 1, -1);
  int64_t spec_need = 0;
  for (int32_t c = 0; c < m; ++c) {
    int64_t L = (int64_t)offsets[c + 1] - offsets[c];
    if (L < 1 || L > 1024)
      return fail("constraint " + std::to_string(c) + ": length " + std::to_string(L) +
                  " outside 1..1024 (or offsets not increasing)");
    int t = type[c];
    if (t < T_OR || t > T_SPECTRUM)
      return fail("constraint " + std::to_string(c) + ": unknown type " + std::to_string(t));
    if (t == T_CARD_GE || t == T_CARD_LE || t == T_EK) {
      if (!kk) return fail("k is required for CARD_GE/CARD_LE/EK constraints");
      if (kk[c] < 0 || kk[c] > L)
        return fail("constraint " + std::to_string(c) + ": k=" + std::to_string(kk[c]) +
                    " outside 0..L");
    }
    if (t == T_SPECTRUM) spec_need += L + 1;
    if (weight && !std::isfinite(weight[c]))
      return fail("constraint " + std::to_string(c) + ": weight is not finite");
    for (int64_t e = offsets[c]; e < offsets[c + 1]; ++e) {
      int32_t v = lit_var[e];
      if (v < 0 || v >= n)
        return fail("literal " + std::to_string(e) + ": variable " + std::to_string(v) +
                    " out of range");
      if (lit_sign[e] != 1 && lit_sign[e] != -1)
        return fail("literal " + std::to_string(e) + ": sign must be +1 or -1");
      if (seen[v] == c)
        return fail("constraint " + std::to_string(c) + ": variable " + std::to_string(v) +
                    " appears twice");
      seen[v] = c;
    }
  }
  if (spec_need > 0 && !spectra) return fail("spectra are required for SPECTRUM constraints");
  for (int64_t i = 0; i < spec_need; ++i)
    if (spectra[i] != 1 && spectra[i] != -1) return fail("spectra entries must be +1 or -1");
  if (fixed) {
    if (!fixed_val) return fail("fixed_val is required when fixed is given");
    for (int32_t v = 0; v < n; ++v) {
      if (fixed[v] > 1) return fail("fixed entries must be 0 or 1");
      if (fixed[v] && fixed_val[v] != 1.0f && fixed_val[v] != -1.0f)
        return fail("variable " + std::to_string(v) + ": fixed value must be +1 or -1");
    }
  }
  if (validate_only) return 0;

  HostPlan& P = *out;
  P = HostPlan();
  P.n = n;
  P.m = m;
  P.nnz = nnz;

  // variable-major transpose: rows of variable v are voff[v]..voff[v+1]-1,
  // literals in increasing constraint order (a fixed summation order)
  P.flags = flags;
  P.voff.assign(n + 1, 0);
  for (int64_t e = 0; e < nnz; ++e) P.voff[lit_var[e] + 1]++;
  for (int32_t v = 0; v < n; ++v) P.voff[v + 1] += P.voff[v];
  std::vector<int32_t> cur(P.voff.begin(), P.voff.end() - 1);
  P.lit.resize(nnz);
  for (int64_t e = 0; e < nnz; ++e) {
    int32_t dst = cur[lit_var[e]]++;
    P.lit[e].var = lit_var[e];
    P.lit[e].dst = dst | (lit_sign[e] < 0 ? kNegBit : 0);
  }

  // fixed real roots and their coefficients
  P.root_tab = {{0.5f, 0.5f, 0.f, 0.f}, {0.5f, -0.5f, 0.f, 0.f}, {0.f, 1.f, 0.f, 0.f}};
  P.zpow_tab.assign(P.root_tab.size() * kNumFrQ, F4{0.f, 0.f, 0.f, 0.f});
  P.spec_tab.clear();
  P.spec_off.assign(m, -1);
  P.ser_tab.clear();
  P.ser_info.assign(m, SerInfo{-1, 0, 0, 0, {0, 0, 0, 0}});
  P.n_ser_slots = 0;
  P.coef_tab = {{2.f, 0.f, 1.f, 0.f},  {1.f, 0.f, 1.f, 0.f},   {2.f, 0.f, 1.f, 0.f},
                {2.f, 0.f, -1.f, 0.f}, {-1.f, 0.f, -1.f, 0.f}, {-2.f, 0.f, -1.f, 0.f},
                {-2.f, 0.f, 1.f, 0.f}};
  const bool simplify = (flags & kFlagSimplifyFixed) && fixed;
  std::vector<LitRec> fe_lit_tmp;      // FE literals: var, sign bit (rows later)
  fe_lit_tmp.reserve(nnz);
  std::map<int, int> root_of_len;
  std::map<int, SerInfo> ser_of_len;
  std::map<std::pair<int, std::string>, int> coef_of_spec;

  P.fe.resize(m);
  P.ctype.assign(type, type + m);
  P.kthr.assign(m, 0);
  P.weight.assign(m, 1.0f);
  int64_t soff = 0;
  std::vector<int8_t> sp;
  for (int32_t c = 0; c < m; ++c) {
    int L = offsets[c + 1] - offsets[c];
    int t = type[c];
    int k = (t == T_CARD_GE || t == T_CARD_LE || t == T_EK) ? kk[c] : 0;
    const int8_t* spec = nullptr;
    if (t == T_SPECTRUM) {
      spec = spectra + soff;
      soff += L + 1;
    }
    float w = weight ? weight[c] : 1.0f;
    P.kthr[c] = k;
    P.weight[c] = w;
    // spectrum sp_t (Eq. 3): -1 where the constraint holds
    sp.assign(L + 1, 1);
    for (int tt = 0; tt <= L; ++tt) sp[tt] = holds(t, L, k, tt, spec) ? -1 : 1;

    // score predicate
    ScoreItem s = ScoreItem{offsets[c], L, 0, 0, 0, w, c, 0};
    switch (t) {
      case T_OR: s.lo = 1; s.hi = L; break;
      case T_XOR: s.mode = 1; break;
      case T_CARD_GE: s.lo = k; s.hi = L; break;
      case T_CARD_LE: s.lo = 0; s.hi = k; break;
      case T_NAE: s.lo = 1; s.hi = L - 1; break;
      case T_EO: s.lo = 1; s.hi = 1; break;
      case T_EK: s.lo = k; s.hi = k; break;
      case T_AMO: s.lo = 0; s.hi = 1; break;
      default: {
        s.mode = 2;
        s.lo = (int32_t)(P.satbits.size() * 32);
        P.satbits.resize(P.satbits.size() + (L + 1 + 31) / 32 + 1, 0u);
        for (int tt = 0; tt <= L; ++tt)
          if (sp[tt] == -1) P.satbits[(s.lo + tt) >> 5] |= 1u << ((s.lo + tt) & 31);
      }
    }
    P.score.push_back(s);

    // literals that enter FE: all of them, or only the free ones when pinned
    // variables are folded into a shifted spectrum sp'_t = sp_{t + f}, f =
    // number of pinned literals that are true (a pinned literal's factor is
    // exactly 1 or w^j, Sec. 3.2's partial assignment).
    int f_true = 0, Lf = 0;
    const size_t fe0 = fe_lit_tmp.size();
    for (int e = offsets[c]; e < offsets[c + 1]; ++e) {
      const int v = lit_var[e];
      if (simplify && fixed[v]) {
        if ((float)lit_sign[e] * fixed_val[v] == -1.0f) ++f_true;
        continue;
      }
      fe_lit_tmp.push_back({v, lit_sign[e] < 0 ? kNegBit : 0});
      ++Lf;
    }
    std::vector<int8_t> spf(sp.begin() + f_true, sp.begin() + f_true + Lf + 1);
    FeItem& it = P.fe[c];
    it.lit0 = (int32_t)fe0;
    it.L = Lf;
    it.w = w;
    it.c = c;
    // classify the (shifted) spectrum: constant, a closed-form product of one
    // or two real roots (Appendix A's OR, XOR, NAE and their complements),
    // or the generic DFT
    bool all_same = true;
    for (int tt = 1; tt <= Lf; ++tt) all_same &= spf[tt] == spf[0];
    auto is_pattern = [&](auto fn) {
      for (int tt = 0; tt <= Lf; ++tt)
        if (spf[tt] != fn(tt)) return false;
      return true;
    };
    auto set_real = [&](int J, int root, int coef, float b0v) {
      it.J = J;
      it.root_off = root;
      it.coef_off = coef;
      it.b0 = b0v;
    };
    if (Lf == 0 || all_same) {           // FE constant, no gradient
      fe_lit_tmp.resize(fe0);
      it.L = 0;
      set_real(0, kRootAlpha, kCoefOr, (float)spf[0]);
      continue;
    }
    if (is_pattern([](int tt) { return tt == 0 ? 1 : -1; })) {            // OR
      set_real(1, kRootAlpha, kCoefOr, -1.f);
      continue;
    }
    if (is_pattern([](int tt) { return tt == 0 ? -1 : 1; })) {            // none true
      set_real(1, kRootAlpha, kCoefNor, 1.f);
      continue;
    }
    if (is_pattern([Lf](int tt) { return tt == Lf ? -1 : 1; })) {         // all true
      set_real(1, kRootBeta, kCoefAllTrue, 1.f);
      continue;
    }
    if (is_pattern([Lf](int tt) { return tt == Lf ? 1 : -1; })) {         // not all true
      set_real(1, kRootBeta, kCoefNae + 1, -1.f);
      continue;
    }
    if (is_pattern([](int tt) { return (tt & 1) ? -1 : 1; })) {           // XOR
      set_real(1, kRootY, kCoefXor, 0.f);
      continue;
    }
    if (is_pattern([](int tt) { return (tt & 1) ? 1 : -1; })) {           // XNOR
      set_real(1, kRootY, kCoefXnor, 0.f);
      continue;
    }
    if (Lf >= 2 && is_pattern([Lf](int tt) { return (tt == 0 || tt == Lf) ? 1 : -1; })) {
      set_real(2, kRootAlpha, kCoefNae, -1.f);                             // NAE
      continue;
    }
    sp.swap(spf);   // the DFT below works on sp with L = Lf
    L = Lf;
    P.spec_off[c] = (int32_t)P.spec_tab.size();
    for (int tt = 0; tt <= L; ++tt) P.spec_tab.push_back((int8_t)sp[tt]);
    // DFT of the spectrum at the L+1 roots of unity, FP64 (Sec. 2.3):
    //   b_j = 1/(L+1) sum_t sp_t w^(-jt),  FE = sum_{j=0}^{L} b_j G_j with
    //   G_j = prod_i (alpha_i + beta_i w^j) (G_0 = 1).  b_{L+1-j} =
    //   conj(b_j) and G_{L+1-j} = conj(G_j), so only j = 1..ceil(L/2) are
    //   kept, pairs with weight 2, the self-conjugate middle root (L odd)
    //   with weight 1.
    const int N = L + 1;
    const int J = (L + 1) / 2;
    std::vector<double> cs(N), sn(N);
    for (int q = 0; q < N; ++q) {
      if (2 * q == N) { cs[q] = -1.0; sn[q] = 0.0; continue; }
      if (q == 0) { cs[q] = 1.0; sn[q] = 0.0; continue; }
      double a = 2.0 * M_PI * (double)q / (double)N;
      cs[q] = std::cos(a);
      sn[q] = std::sin(a);
    }
    double b0 = 0.0;
    for (int tt = 0; tt <= L; ++tt) b0 += sp[tt];
    it.b0 = (float)(b0 / N);
    it.J = J;
    auto rit = root_of_len.find(L);
    if (rit == root_of_len.end()) {
      int off = (int)P.root_tab.size();
      for (int j = 1; j <= J; ++j) {
        float B = (float)((1.0 - cs[j]) * 0.5);
        float A = 1.0f - B;
        float C = (float)(sn[j] * 0.5);
        // factored form, phi = theta_j / 2: alpha + beta w = e^{i phi}
        // (cos phi - i y sin phi) = z u(y) with
        //   phi <= pi/4:         z = 1/(1 - i t),  u = 1 - i y t,  t = tan phi
        //   pi/4 < phi <= 0.42pi: z = 1/(t + i),   u = y t + i,    t = tan phi
        //   phi > 0.42 pi:       z = 1/(1 + i t),  u = y + i t,    t = cot phi
        // (|u| <= 4.02 in the middle form, sqrt 2 in the others).  z is taken
        // from the FP32-rounded t, so that z u(1) = 1 for the value the
        // kernel multiplies by.
        const double ph = M_PI * (double)j / (double)N;
        const double c = (2 * j == N) ? 0.0 : std::cos(ph), s = std::sin(ph);
        // forms 0 / 1 / 2 (see the device helpers): t = tan phi, tan phi,
        // cot phi; z = 1/u(1) = 1/(1 - i t), 1/(t + i), 1/(1 + i t)
        const int form = (4 * j <= N) ? 0 : (50 * j <= 21 * N) ? 1 : 2;
        const float t32 = (float)(form < 2 ? s / c : c / s);
        const double t = t32, den = 1.0 + t * t;
        const double zr = form == 1 ? t / den : 1.0 / den;
        const double zi = form == 0 ? t / den : -(form == 1 ? 1.0 : t) / den;
        P.root_tab.push_back({A, B, C, t32});
        double pr = 1.0, pi = 0.0;   // z^k, k = 0, 1, ...
        double prev_r = 1.0, prev_i = 0.0;
        int k = 0;
        for (int q = 0; q < kNumFrQ; ++q) {
          while (k < kFrQ[q]) {
            prev_r = pr;
            prev_i = pi;
            const double nr = pr * zr - pi * zi, ni = pr * zi + pi * zr;
            pr = nr;
            pi = ni;
            ++k;
          }
          P.zpow_tab.push_back({(float)pr, (float)pi, (float)prev_r, (float)prev_i});
        }
      }
      rit = root_of_len.emplace(L, off).first;
    }
    it.root_off = rit->second;
    std::string key(reinterpret_cast<const char*>(sp.data()), sp.size());
    auto cit = coef_of_spec.find({L, key});
    if (cit == coef_of_spec.end()) {
      int off = (int)P.coef_tab.size();
      for (int j = 1; j <= J; ++j) {
        double re = 0.0, im = 0.0;
        for (int tt = 0; tt <= L; ++tt) {
          int q = (int)(((int64_t)j * tt) % N);
          re += sp[tt] * cs[q];
          im -= sp[tt] * sn[q];
        }
        re /= N;
        im /= N;
        double mult = (2 * j == N) ? 1.0 : 2.0;
        re *= mult;
        im *= mult;
        double B = (1.0 - cs[j]) * 0.5, C = sn[j] * 0.5;
        // c' = b' * dF/dy = b' * (B - i C)
        double cre = re * B + im * C;
        double cim = im * B - re * C;
        P.coef_tab.push_back({(float)re, (float)im, (float)cre, (float)cim});
      }
      cit = coef_of_spec.emplace(std::make_pair(L, key), off).first;
    }
    it.coef_off = cit->second;
    if (L >= kSeriesMinL) {
      auto sit = ser_of_len.find(L);
      if (sit == ser_of_len.end()) sit = ser_of_len.emplace(L, series_table(L, P.ser_tab)).first;
      P.ser_info[c] = sit->second;
      if (P.ser_info[c].off >= 0) P.ser_info[c].slot = P.n_ser_slots++;
    }
    P.dft_roots += J;
    P.dft_lroots += (int64_t)J * L;
  }
  // variable-major rows of the FE literals (the partial buffer): rows of
  // variable v are fe_voff[v]..fe_voff[v+1]-1, in constraint order
  P.nnz_fe = (int64_t)fe_lit_tmp.size();
  P.fe_voff.assign(n + 1, 0);
  for (const LitRec& r : fe_lit_tmp) P.fe_voff[r.var + 1]++;
  for (int32_t v = 0; v < n; ++v) P.fe_voff[v + 1] += P.fe_voff[v];
  {
    std::vector<int32_t> fcur(P.fe_voff.begin(), P.fe_voff.end() - 1);
    P.fe_lit = fe_lit_tmp;
    for (LitRec& r : P.fe_lit) r.dst |= fcur[r.var]++;
  }
  // score ranges: consecutive constraints, about kScoreRangeLits literals each
  // (fewer for small problems, so that their scoring still spreads over
  // many warps)
  const int64_t range_lits =
      std::min<int64_t>(kScoreRangeLits, std::max<int64_t>(32, nnz / 1024));
  P.score_ranges.push_back(0);
  int64_t acc = 0;
  for (int32_t c = 0; c < m; ++c) {
    acc += P.score[c].L;
    if (acc >= range_lits || c == m - 1) {
      P.score_ranges.push_back(c + 1);
      acc = 0;
    }
  }
  if (fixed) {
    P.fixed.assign(fixed, fixed + n);
    P.fixed_val.assign(fixed_val, fixed_val + n);
  }
  assign_groups(&P, default_tuning());
  return 0;
}

}  // namespace cls
