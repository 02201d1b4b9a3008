// api.cu -- the extern "C" boundary (include/cls.h): argument checks, device
// residency of the problem, workspace carving and the per-call kernel
// sequences.  No exceptions or aborts cross the boundary.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/cls.h"
#include "kernels.cuh"
#include "mpnn.cuh"
#include "plan.h"

namespace {

thread_local std::string g_last_error;

int set_err(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_err(cudaError_t e, const char* where) {
  return set_err(CLS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CLS_CUDA_TRY(expr, where)          \
  do {                                     \
    cudaError_t e_ = (expr);               \
    if (e_ != cudaSuccess) {               \
      (void)cudaGetLastError();            \
      return cuda_err(e_, where);          \
    }                                      \
  } while (0)

struct EventHook : cls::LaunchHook {
  struct Rec {
    int kc;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t pending = nullptr;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void before(int, cudaStream_t s) override {
    pending = get();
    cudaEventRecord(pending, s);
  }
  void after(int kc, cudaStream_t s) override {
    cudaEvent_t b = get();
    cudaEventRecord(b, s);
    recs.push_back({kc, pending, b});
    pending = nullptr;
  }
  void reset() {
    for (auto& r : recs) {
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    recs.clear();
  }
  ~EventHook() override {
    for (auto& r : recs) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

}  // namespace

struct cls_problem {
  int device = 0;
  cls::HostPlan host;
  cls::DevPlan dev;
  std::vector<void*> allocations;
  EventHook* hook = nullptr;  // non-null while profiling
  EventHook events;
  bool weights_dirty = false;  // device weights changed since the host plan's copy
  int64_t list_epoch = 0;      // bumped whenever the work lists are uploaded again
  // cls_solve_host's recorded step chunk, reused while its workspace, R, lr,
  // work lists and weight mode stay the same (a cache: mutable)
  mutable cls_graph* solve_graph = nullptr;
  mutable const void* sg_ws = nullptr;
  mutable int sg_R = 0;
  mutable float sg_lr = 0.f;
  mutable int64_t sg_epoch = -1;
  mutable int sg_unit = -1;
};

namespace {

template <typename T>
int upload(cls_problem* p, const std::vector<T>& v, T** out) {
  *out = nullptr;
  if (v.empty()) return CLS_OK;
  void* ptr = nullptr;
  cudaError_t e = cudaMalloc(&ptr, v.size() * sizeof(T));
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return set_err(e == cudaErrorMemoryAllocation ? CLS_ERR_NOMEM : CLS_ERR_CUDA,
                   std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  p->allocations.push_back(ptr);
  CLS_CUDA_TRY(cudaMemcpy(ptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice),
               "cudaMemcpy");
  *out = static_cast<T*>(ptr);
  return CLS_OK;
}

void free_problem(cls_problem* p) {
  for (void* a : p->allocations) cudaFree(a);
  p->allocations.clear();
}

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Workspace layout for R restarts.
struct Layout {
  int R = 0, Rp = 0, RT = 0;
  int nch = 1, chunk = 1;
  size_t P = 0, fe = 0, bits = 0, nsat_part = 0, wsat_part = 0, obj_part = 0, nsat = 0,
         rpart_n = 0, rpart_w = 0, bar = 0, done = 0, ser = 0, total = 0;
};

Layout layout_for(const cls_problem* p, int R) {
  Layout L;
  L.R = R;
  L.RT = (R + 31) / 32;
  L.Rp = L.RT * 32;
  const int m = p->host.m;
  // enough (restart tile x chunk) blocks to fill the GPU in the reductions
  int want = std::max(1, (148 * 4 + L.RT - 1) / std::max(1, L.RT));
  want = std::min(want, std::max(1, (m + 7) / 8));
  L.chunk = std::max(1, (m + want - 1) / want);
  L.nch = std::max(1, (m + L.chunk - 1) / L.chunk);
  size_t off = 0;
  auto take = [&off](size_t bytes) {
    size_t at = off;
    off = align_up(off + bytes);
    return at;
  };
  const int nsc = std::max(1, cls::score_chunks(p->dev.n_ranges));
  L.P = take((size_t)p->host.nnz_fe * L.Rp * sizeof(float));
  L.fe = take((size_t)m * L.Rp * sizeof(float));
  L.bits = take((size_t)p->host.n * L.RT * sizeof(uint32_t));
  L.nsat_part = take((size_t)nsc * L.Rp * sizeof(int32_t));
  L.wsat_part = take((size_t)nsc * L.Rp * sizeof(double));
  L.obj_part = take((size_t)L.nch * L.Rp * sizeof(double));
  L.nsat = take((size_t)L.Rp * sizeof(int32_t));
  // corner-pass flags of the factored DFT kernels, one per (constraint, tile)
  L.done = take((size_t)std::max(1, m) * L.RT);
  // directly after the flags (cls::ser_terms locates it from them): the
  // Chebyshev pass's saved low-root terms, kSeriesK1 + 1 rows per slot
  L.ser = take((size_t)p->host.n_ser_slots * (cls::kSeriesK1 + 1) * L.Rp * sizeof(float));
  // persistent loop: per-range score partials and the grid barrier words
  const size_t nr = (size_t)std::max(1, p->dev.n_ranges);
  L.rpart_n = take(nr * L.Rp * sizeof(int32_t));
  L.rpart_w = take(nr * L.Rp * sizeof(double));
  L.bar = take(4 * sizeof(int32_t));
  L.total = off;
  return L;
}

int check_ws(const Layout& L, void* ws, size_t ws_bytes) {
  if (L.total == 0) return CLS_OK;
  if (!ws) return set_err(CLS_ERR_WORKSPACE, "workspace pointer is NULL");
  if (reinterpret_cast<uintptr_t>(ws) % kAlign != 0)
    return set_err(CLS_ERR_WORKSPACE, "workspace is not 256-byte aligned");
  if (ws_bytes < L.total)
    return set_err(CLS_ERR_WORKSPACE, "workspace too small: need " + std::to_string(L.total) +
                                          " bytes, got " + std::to_string(ws_bytes));
  return CLS_OK;
}

template <typename T>
T* at(void* ws, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(ws) + off);
}

int check_device(cls_problem* p) {
  int dev = 0;
  CLS_CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
  cudaDeviceProp prop;
  CLS_CUDA_TRY(cudaGetDeviceProperties(&prop, dev), "cudaGetDeviceProperties");
  if (!(prop.major == 10 && prop.minor == 3))
    return set_err(CLS_ERR_UNSUPPORTED, std::string("device ") + prop.name + " is sm_" +
                                            std::to_string(prop.major) +
                                            std::to_string(prop.minor) +
                                            "; this library is built for sm_103a (B300)");
  p->device = dev;
  return CLS_OK;
}

int check_R(const cls_problem* p, int32_t R) {
  if (!p) return set_err(CLS_ERR_INVALID, "problem is NULL");
  if (R < 0) return set_err(CLS_ERR_INVALID, "R must be >= 0");
  if (R > 65535 * 32) return set_err(CLS_ERR_INVALID, "R must be <= 2097120");
  if ((int64_t)R * std::max<int64_t>(1, p->host.n) > (int64_t)1 << 40)
    return set_err(CLS_ERR_INVALID, "R * n too large");
  return CLS_OK;
}

cls::LaunchHook* hook_of(const cls_problem* p) { return p->hook; }

// (Re)upload the FE work lists of the current tuning.  Old list buffers stay
// allocated until the problem is destroyed (tuning changes are rare).
int upload_lists(cls_problem* p) {
  const cls::HostPlan& H = p->host;
  cls::DevPlan& D = p->dev;
  ++p->list_epoch;
  for (int t = 0; t < cls::kNumThreadCls; ++t) {
    int rc = upload(p, H.thread_items[t], &D.thread_items[t]);
    if (rc != CLS_OK) return rc;
    D.thread_count[t] = (int32_t)H.thread_items[t].size();
  }
  {
    int rc = upload(p, H.const_list, &D.const_list);
    if (rc != CLS_OK) return rc;
    D.const_count = (int32_t)H.const_list.size();
  }
  for (int b = 0; b < cls::kNumBuckets; ++b) {
    int rc = upload(p, H.bucket_list[b], &D.bucket_list[b]);
    if (rc != CLS_OK) return rc;
    D.bucket_count[b] = (int32_t)H.bucket_list[b].size();
    D.bucket_cfg[b] = H.bucket_cfg[b];
    D.bucket_maxL[b] = H.bucket_list[b].empty() ? 0 : H.fe[H.bucket_list[b][0]].L;
    D.bucket_maxJ[b] = 0;
    for (int32_t c : H.bucket_list[b]) D.bucket_maxJ[b] = std::max(D.bucket_maxJ[b], H.fe[c].J);
  }
  return CLS_OK;
}

// Weights changed on the device (cls_set_weights, cls_reweight) back into the
// host plan, whose items the short-class lists are rebuilt from on retuning.
int pull_weights(cls_problem* p) {
  if (!p->weights_dirty) return CLS_OK;
  cls::HostPlan& H = p->host;
  CLS_CUDA_TRY(cudaDeviceSynchronize(), "synchronize before reading weights");
  if (H.m > 0)
    CLS_CUDA_TRY(cudaMemcpy(H.fe.data(), p->dev.fe, sizeof(cls::FeItem) * (size_t)H.m,
                            cudaMemcpyDeviceToHost),
                 "copy weights");
  for (int32_t c = 0; c < H.m; ++c) {
    H.weight[c] = H.fe[c].w;
    H.score[c].w = H.fe[c].w;
  }
  p->weights_dirty = false;
  return CLS_OK;
}

// One full CLS step: FE + partials, accumulate + step + round, score.
int run_step(const cls_problem* p, const Layout& L, float* x, float lr, uint32_t* bits,
             int32_t* nsat, double* wsat, void* ws, cudaStream_t s, bool score) {
  float* P = at<float>(ws, L.P);
  CLS_CUDA_TRY(cls::launch_fe(p->dev, L.R, L.Rp, x, P, nullptr, 0, at<uint8_t>(ws, L.done), s,
                              hook_of(p)),
               "fe kernels");
  CLS_CUDA_TRY(cls::launch_accum_step(p->dev, L.R, L.Rp, P, x, lr, true, nullptr, bits, s,
                                      hook_of(p)),
               "accumulate/step kernel");
  if (score)
    CLS_CUDA_TRY(cls::launch_score(p->dev, L.R, L.Rp, bits, at<int32_t>(ws, L.nsat_part),
                                   at<double>(ws, L.wsat_part), nsat, wsat, s, hook_of(p)),
                 "score kernels");
  return CLS_OK;
}

}  // namespace

namespace cls {
// Helpers for other translation units of the library (noalloc.cu).
int set_error(int code, const std::string& msg) { return set_err(code, msg); }
bool profiling_enabled(const cls_problem* p) { return p && p->hook != nullptr; }
int problem_device(const cls_problem* p) { return p ? p->device : -1; }
}  // namespace cls

extern "C" {

int cls_problem_check(int32_t n, int32_t m, const int32_t* offsets, const int32_t* lit_var,
                      const int8_t* lit_sign, const int32_t* type, const int32_t* k,
                      const float* weight, const int8_t* spectra, const uint8_t* fixed,
                      const float* fixed_val) {
  std::string msg;
  int rc = cls::build_plan(n, m, offsets, lit_var, lit_sign, type, k, weight, spectra, fixed,
                           fixed_val, 0u, true, nullptr, &msg);
  if (rc != 0) return set_err(CLS_ERR_INVALID, msg);
  return CLS_OK;
}

int cls_problem_create(int32_t n, int32_t m, const int32_t* offsets, const int32_t* lit_var,
                       const int8_t* lit_sign, const int32_t* type, const int32_t* k,
                       const float* weight, const int8_t* spectra, const uint8_t* fixed,
                       const float* fixed_val, cls_problem** out) {
  return cls_problem_create_ex(n, m, offsets, lit_var, lit_sign, type, k, weight, spectra, fixed,
                               fixed_val, 0u, out);
}

int cls_problem_create_ex(int32_t n, int32_t m, const int32_t* offsets, const int32_t* lit_var,
                          const int8_t* lit_sign, const int32_t* type, const int32_t* k,
                          const float* weight, const int8_t* spectra, const uint8_t* fixed,
                          const float* fixed_val, uint32_t flags, cls_problem** out) {
  if (!out) return set_err(CLS_ERR_INVALID, "out is NULL");
  if (flags & ~(uint32_t)CLS_SIMPLIFY_FIXED) return set_err(CLS_ERR_INVALID, "unknown flags");
  *out = nullptr;
  cls_problem* p = new (std::nothrow) cls_problem();
  if (!p) return set_err(CLS_ERR_NOMEM, "host allocation failed");
  std::string msg;
  int rc;
  try {
    rc = cls::build_plan(n, m, offsets, lit_var, lit_sign, type, k, weight, spectra, fixed,
                         fixed_val, flags, false, &p->host, &msg);
  } catch (const std::bad_alloc&) {
    delete p;
    return set_err(CLS_ERR_NOMEM, "host allocation failed while building the problem");
  }
  if (rc != 0) {
    delete p;
    return set_err(CLS_ERR_INVALID, msg);
  }
  rc = check_device(p);
  if (rc != CLS_OK) {
    delete p;
    return rc;
  }
  static bool attrs_set = false;
  if (!attrs_set) {
    cudaError_t e = cls::set_kernel_attributes();
    if (e != cudaSuccess) {
      delete p;
      (void)cudaGetLastError();
      return cuda_err(e, "cudaFuncSetAttribute");
    }
    attrs_set = true;
  }
  const cls::HostPlan& H = p->host;
  cls::DevPlan& D = p->dev;
  D.n = H.n;
  D.m = H.m;
  D.nnz = H.nnz;
  D.nnz_fe = H.nnz_fe;
  int r2 = CLS_OK;
  auto up = [&](auto& vec, auto** dst) {
    if (r2 == CLS_OK) r2 = upload(p, vec, dst);
  };
  up(H.lit, &D.lit);
  up(H.voff, &D.voff);
  up(H.fe_lit, &D.fe_lit);
  up(H.fe_voff, &D.fe_voff);
  up(H.fe, &D.fe);
  up(H.score, &D.score);
  up(H.score_ranges, &D.score_ranges);
  D.n_ranges = H.score_ranges.empty() ? 0 : (int32_t)H.score_ranges.size() - 1;
  D.unit_weights = 1;
  for (float w : H.weight)
    if (w != 1.0f) D.unit_weights = 0;
  up(H.satbits, &D.satbits);
  up(H.root_tab, &D.root_tab);
  up(H.zpow_tab, &D.zpow_tab);
  up(H.coef_tab, &D.coef_tab);
  up(H.fixed, &D.fixed);
  up(H.fixed_val, &D.fixed_val);
  up(H.spec_tab, &D.spec_tab);
  up(H.spec_off, &D.spec_off);
  up(H.ser_tab, &D.ser_tab);
  up(H.ser_info, &D.ser_info);
  {
    // statistics: flops of the DFT roots the dense factored kernel evaluated
    const std::vector<unsigned long long> zero(1, 0ull);
    up(zero, &D.dft_flops);
    const std::vector<double> zd(1, 0.0);
    up(zd, &D.rw_gbar);
    // work order of the constraint statistics pass
    std::vector<int32_t> order(H.m);
    for (int32_t c = 0; c < H.m; ++c) order[c] = c;
    std::stable_sort(order.begin(), order.end(),
                     [&H](int32_t a, int32_t b) { return H.fe[a].L > H.fe[b].L; });
    up(order, &D.stat_order);
  }
  if (r2 == CLS_OK) r2 = upload_lists(p);
  if (r2 != CLS_OK) {
    free_problem(p);
    delete p;
    return r2;
  }
  *out = p;
  return CLS_OK;
}

int cls_problem_destroy(cls_problem* p) {
  if (!p) return CLS_OK;
  cudaDeviceSynchronize();
  if (p->solve_graph) cls_graph_destroy(p->solve_graph);
  p->solve_graph = nullptr;
  free_problem(p);
  delete p;
  return CLS_OK;
}

int cls_problem_info(const cls_problem* p, int64_t* info) {
  if (!p || !info) return set_err(CLS_ERR_INVALID, "NULL argument");
  const cls::HostPlan& H = p->host;
  info[0] = H.n;
  info[1] = H.m;
  info[2] = H.nnz;
  info[3] = H.n_thread;
  info[4] = H.n_group_real;
  info[5] = H.n_group_dft;
  info[6] = H.dft_roots;
  info[7] = H.dft_lroots;
  info[8] = H.nnz_fe;
  info[9] = (int64_t)H.const_list.size();
  return CLS_OK;
}

int cls_dft_work(const cls_problem* p, int64_t* out) {
  if (!p || !out) return set_err(CLS_ERR_INVALID, "NULL argument");
  const cls::HostPlan& H = p->host;
  int64_t flops = 0, lroots = 0;
  for (int b = 0; b < cls::kNumDftBuckets; ++b) {
    const int cfg = H.bucket_cfg[b];
    const bool fr = cfg >= 0 && cfg < cls::kNumGroupCfg && cls::kGroupCfg[cfg].cplx == 3;
    for (int32_t c : H.bucket_list[b]) {
      const cls::FeItem& it = H.fe[c];
      const int64_t L = it.L, J = it.J, nA = cls::fr_roots_form01(it.L);
      lroots += L * J;
      // factored roots: 14 flops per (literal, root) in forms 0 and 1 and 16
      // in form 2; the direct factor alpha + beta w^j: 20
      flops += fr ? L * (14 * nA + 16 * (J - nA)) : 20 * L * J;
    }
  }
  out[0] = flops;
  out[1] = lroots;
  return CLS_OK;
}

int cls_dft_flops_counter(cls_problem* p, int64_t* flops, int32_t reset) {
  if (!p || !flops) return set_err(CLS_ERR_INVALID, "NULL argument");
  unsigned long long v = 0;
  CLS_CUDA_TRY(cudaDeviceSynchronize(), "synchronize");
  CLS_CUDA_TRY(cudaMemcpy(&v, p->dev.dft_flops, sizeof(v), cudaMemcpyDeviceToHost), "copy");
  *flops = (int64_t)v;
  if (reset) CLS_CUDA_TRY(cudaMemset(p->dev.dft_flops, 0, sizeof(v)), "memset");
  return CLS_OK;
}

int cls_series_range(int32_t L, int32_t K) {
  if (L < 1 || K < 1) return set_err(CLS_ERR_INVALID, "L and K must be >= 1");
  return cls::series_roots(L, K);
}

int cls_workspace_size(const cls_problem* p, int32_t R, size_t* bytes) {
  int rc = check_R(p, R);
  if (rc != CLS_OK) return rc;
  if (!bytes) return set_err(CLS_ERR_INVALID, "bytes is NULL");
  *bytes = layout_for(p, R).total;
  return CLS_OK;
}

int cls_init_uniform(const cls_problem* p, int32_t R, uint64_t seed, int64_t r_offset, float* x,
                     void* stream) {
  int rc = check_R(p, R);
  if (rc != CLS_OK) return rc;
  if (!x && R > 0 && p->host.n > 0) return set_err(CLS_ERR_INVALID, "x is NULL");
  if (r_offset < 0) return set_err(CLS_ERR_INVALID, "r_offset must be >= 0");
  CLS_CUDA_TRY(cls::launch_init(p->dev, R, seed, r_offset, x, (cudaStream_t)stream, hook_of(p)),
               "init kernel");
  return CLS_OK;
}

int cls_track_reset(const cls_problem* p, int32_t R, int32_t* trk, void* stream) {
  int rc = check_R(p, R);
  if (rc != CLS_OK) return rc;
  if (!trk && R > 0) return set_err(CLS_ERR_INVALID, "trk is NULL");
  CLS_CUDA_TRY(cls::launch_track_reset(R, trk, (cudaStream_t)stream), "track reset kernel");
  return CLS_OK;
}

int cls_track_step(const cls_problem* p, int32_t R, const int32_t* nsat, int32_t step,
                   int32_t* trk, void* stream) {
  int rc = check_R(p, R);
  if (rc != CLS_OK) return rc;
  if (step < 0) return set_err(CLS_ERR_INVALID, "step must be >= 0");
  if (R > 0 && (!nsat || !trk)) return set_err(CLS_ERR_INVALID, "nsat or trk is NULL");
  CLS_CUDA_TRY(cls::launch_track_step(p->dev, R, step, nsat, trk, (cudaStream_t)stream),
               "track kernel");
  return CLS_OK;
}

int cls_refill(const cls_problem* p, int32_t R, float* x, int32_t* trk, int32_t patience,
               uint64_t seed, int64_t r_offset, int32_t generation, int32_t* count,
               void* stream) {
  int rc = check_R(p, R);
  if (rc != CLS_OK) return rc;
  if (patience < 1) return set_err(CLS_ERR_INVALID, "patience must be >= 1");
  if (generation < 1) return set_err(CLS_ERR_INVALID, "generation must be >= 1");
  if (r_offset < 0) return set_err(CLS_ERR_INVALID, "r_offset must be >= 0");
  if (R > 0 && (!trk || !count || (!x && p->host.n > 0)))
    return set_err(CLS_ERR_INVALID, "x, trk or count is NULL");
  CLS_CUDA_TRY(cls::launch_refill(p->dev, R, seed, r_offset, (uint64_t)generation, patience, trk,
                                  x, count, (cudaStream_t)stream),
               "refill kernels");
  return CLS_OK;
}

int cls_unsat_histogram(const cls_problem* p, int32_t R, const int32_t* nsat, int32_t* hist,
                        void* stream) {
  int rc = check_R(p, R);
  if (rc != CLS_OK) return rc;
  if (!hist || (R > 0 && !nsat)) return set_err(CLS_ERR_INVALID, "nsat or hist is NULL");
  CLS_CUDA_TRY(cls::launch_unsat_hist(p->dev, R, nsat, hist, (cudaStream_t)stream),
               "histogram kernel");
  return CLS_OK;
}

int cls_movement(const cls_problem* p, int32_t R, const float* x_prev, const float* x,
                 float* maxdelta, void* stream) {
  int rc = check_R(p, R);
  if (rc != CLS_OK) return rc;
  if (R > 0 && (!maxdelta || (p->host.n > 0 && (!x_prev || !x))))
    return set_err(CLS_ERR_INVALID, "x_prev, x or maxdelta is NULL");
  CLS_CUDA_TRY(cls::launch_movement(p->dev, R, x_prev, x, maxdelta, (cudaStream_t)stream),
               "movement kernel");
  return CLS_OK;
}

int cls_track_converged(const cls_problem* p, int32_t R, const float* maxdelta, float tol,
                        int32_t step, int32_t* conv, void* stream) {
  int rc = check_R(p, R);
  if (rc != CLS_OK) return rc;
  if (step < 0 || !(tol >= 0.f)) return set_err(CLS_ERR_INVALID, "need step >= 0 and tol >= 0");
  if (R > 0 && (!maxdelta || !conv)) return set_err(CLS_ERR_INVALID, "maxdelta or conv is NULL");
  CLS_CUDA_TRY(cls::launch_track_conv(R, maxdelta, tol, step, conv, (cudaStream_t)stream),
               "convergence kernel");
  return CLS_OK;
}

int cls_constraint_stats(const cls_problem* p, int32_t R, const uint32_t* bits, void* ws,
                         size_t ws_bytes, double* gnorm, int32_t* unsat, void* stream) {
  int rc = check_R(p, R);
  if (rc != CLS_OK) return rc;
  if (p->host.m > 0 && (!gnorm || !unsat)) return set_err(CLS_ERR_INVALID, "gnorm or unsat is NULL");
  if (R > 0 && p->host.n > 0 && !bits) return set_err(CLS_ERR_INVALID, "bits is NULL");
  if (R == 0) return set_err(CLS_ERR_INVALID, "R must be >= 1");
  Layout L = layout_for(p, R);
  rc = check_ws(L, ws, ws_bytes);
  if (rc != CLS_OK) return rc;
  const float* P = at<float>(ws, L.P);
  // the objective's FE scratch (m x Rp floats) holds the per-tile sums
  float* scratch = at<float>(ws, L.fe);
  CLS_CUDA_TRY(cls::launch_con_stats(p->dev, R, L.Rp, bits, P, scratch, gnorm, unsat,
                                     (cudaStream_t)stream),
               "constraint statistics kernels");
  return CLS_OK;
}

int cls_set_weights(cls_problem* p, const float* w, void* stream) {
  if (!p) return set_err(CLS_ERR_INVALID, "problem is NULL");
  if (p->host.m > 0 && !w) return set_err(CLS_ERR_INVALID, "w is NULL");
  CLS_CUDA_TRY(cls::launch_set_weights(p->dev, w, (cudaStream_t)stream), "weights kernel");
  p->dev.unit_weights = 0;
  p->weights_dirty = true;
  return CLS_OK;
}

int cls_reweight(cls_problem* p, int32_t R, const double* gnorm, const int32_t* unsat, double eta,
                 double kappa, double w_max, float* w_out, void* stream) {
  int rc = check_R(p, R);
  if (rc != CLS_OK) return rc;
  if (R == 0) return set_err(CLS_ERR_INVALID, "R must be >= 1");
  if (!(eta >= 0.0 && eta < 1e30) || !(kappa > 0.0 && kappa < 1e30) ||
      !(w_max > 0.0 && w_max <= 3.0e38))
    return set_err(CLS_ERR_INVALID, "need 0 <= eta, 0 < kappa, 0 < w_max <= FLT_MAX, all finite");
  if (p->host.m > 0 && (!gnorm || !unsat || !w_out))
    return set_err(CLS_ERR_INVALID, "gnorm, unsat or w_out is NULL");
  CLS_CUDA_TRY(cls::launch_reweight(p->dev, R, gnorm, unsat, eta, kappa, w_max, w_out,
                                    p->dev.rw_gbar, (cudaStream_t)stream),
               "reweight kernels");
  p->dev.unit_weights = 0;
  p->weights_dirty = true;
  return CLS_OK;
}

int cls_eval(const cls_problem* p, int32_t R, const float* x, float* obj, float* grad,
             float* fe_con, void* ws, size_t ws_bytes, void* stream) {
  int rc = check_R(p, R);
  if (rc != CLS_OK) return rc;
  if (R == 0) return CLS_OK;
  if (!x && p->host.n > 0) return set_err(CLS_ERR_INVALID, "x is NULL");
  Layout L = layout_for(p, R);
  rc = check_ws(L, ws, ws_bytes);
  if (rc != CLS_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  float* P = at<float>(ws, L.P);
  float* fe = fe_con;
  int ldf = R;
  if (!fe && obj) {
    fe = at<float>(ws, L.fe);
    ldf = L.Rp;
  }
  CLS_CUDA_TRY(cls::launch_fe(p->dev, R, L.Rp, x, P, fe, ldf, at<uint8_t>(ws, L.done), s,
                              hook_of(p)),
               "fe kernels");
  CLS_CUDA_TRY(cls::launch_fe_const(p->dev, R, fe, ldf, s), "constant expansions");
  if (grad)
    CLS_CUDA_TRY(cls::launch_accum_step(p->dev, R, L.Rp, P, nullptr, 0.f, false, grad, nullptr,
                                        s, hook_of(p)),
                 "accumulate kernel");
  if (obj)
    CLS_CUDA_TRY(cls::launch_obj(p->dev, R, L.Rp, L.nch, L.chunk, fe, ldf,
                                 at<double>(ws, L.obj_part), obj, s, hook_of(p)),
                 "objective reduction");
  return CLS_OK;
}

int cls_restart_scale(const cls_problem* p, int32_t R, const float* g, const float* scale,
                      float* out, void* stream) {
  int rc = check_R(p, R);
  if (rc != CLS_OK) return rc;
  if (R == 0 || p->host.n == 0) return CLS_OK;
  if (!g || !scale || !out) return set_err(CLS_ERR_INVALID, "g, scale and out are required");
  CLS_CUDA_TRY(cls::launch_restart_scale(p->host.n, R, g, scale, out, (cudaStream_t)stream,
                                         hook_of(p)),
               "scale kernel");
  return CLS_OK;
}

int cls_pgd_update(const cls_problem* p, int32_t R, float* x, const float* grad, float lr,
                   uint32_t* bits, void* stream) {
  int rc = check_R(p, R);
  if (rc != CLS_OK) return rc;
  if (R == 0 || p->host.n == 0) return CLS_OK;
  if (!x || !grad) return set_err(CLS_ERR_INVALID, "x and grad are required");
  CLS_CUDA_TRY(cls::launch_pgd(p->dev, R, x, grad, lr, bits, (cudaStream_t)stream, hook_of(p)),
               "step kernel");
  return CLS_OK;
}

int cls_round_score(const cls_problem* p, int32_t R, const float* x, uint32_t* bits,
                    int32_t* nsat, double* wsat, void* ws, size_t ws_bytes, void* stream) {
  int rc = check_R(p, R);
  if (rc != CLS_OK) return rc;
  if (R == 0) return CLS_OK;
  if (!x && p->host.n > 0) return set_err(CLS_ERR_INVALID, "x is NULL");
  Layout L = layout_for(p, R);
  rc = check_ws(L, ws, ws_bytes);
  if (rc != CLS_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t* b = bits ? bits : at<uint32_t>(ws, L.bits);
  CLS_CUDA_TRY(cls::launch_round(p->dev, R, x, b, s, hook_of(p)), "round kernel");
  CLS_CUDA_TRY(cls::launch_score(p->dev, R, L.Rp, b, at<int32_t>(ws, L.nsat_part),
                                 at<double>(ws, L.wsat_part), nsat, wsat, s, hook_of(p)),
               "score kernels");
  return CLS_OK;
}

int cls_step(const cls_problem* p, int32_t R, float* x, float lr, int32_t n_steps,
             uint32_t* bits, int32_t* nsat, double* wsat, void* ws, size_t ws_bytes,
             void* stream) {
  int rc = check_R(p, R);
  if (rc != CLS_OK) return rc;
  if (n_steps < 0) return set_err(CLS_ERR_INVALID, "n_steps must be >= 0");
  if (R == 0) return CLS_OK;
  if (!x && p->host.n > 0) return set_err(CLS_ERR_INVALID, "x is NULL");
  Layout L = layout_for(p, R);
  rc = check_ws(L, ws, ws_bytes);
  if (rc != CLS_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t* b = bits ? bits : at<uint32_t>(ws, L.bits);
  if (n_steps == 0) {
    if (!bits && !nsat && !wsat) return CLS_OK;
    return cls_round_score(p, R, x, b, nsat, wsat, ws, ws_bytes, stream);
  }
  const bool want_score = nsat || wsat;
  for (int st = 0; st < n_steps; ++st) {
    rc = run_step(p, L, x, lr, b, nsat, wsat, ws, s, want_score);
    if (rc != CLS_OK) return rc;
  }
  return CLS_OK;
}

int cls_step_persistent(const cls_problem* p, int32_t R, float* x, float lr, int32_t n_steps,
                        uint32_t* bits, int32_t* nsat, double* wsat, void* ws, size_t ws_bytes,
                        void* stream) {
  int rc = check_R(p, R);
  if (rc != CLS_OK) return rc;
  if (n_steps < 0) return set_err(CLS_ERR_INVALID, "n_steps must be >= 0");
  if (R == 0 || n_steps == 0) return CLS_OK;
  if (!x) return set_err(CLS_ERR_INVALID, "x is NULL");
  if (!cls::persistent_eligible(p->dev))
    return set_err(CLS_ERR_UNSUPPORTED,
                   "the persistent loop needs every FE constraint on the short closed-form path "
                   "(<= 16 literals); use cls_step or a graph");
  const Layout L = layout_for(p, R);
  rc = check_ws(L, ws, ws_bytes);
  if (rc != CLS_OK) return rc;
  uint32_t* b = bits ? bits : at<uint32_t>(ws, L.bits);
  unsigned* bar = at<unsigned>(ws, L.bar);
  cudaError_t e = cls::launch_persistent(p->dev, R, L.Rp, x, lr, n_steps, at<float>(ws, L.P), b,
                                         at<int32_t>(ws, L.rpart_n), at<double>(ws, L.rpart_w),
                                         nsat, wsat, bar, reinterpret_cast<int*>(bar + 2),
                                         (cudaStream_t)stream);
  if (e == cudaErrorNotSupported)
    return set_err(CLS_ERR_UNSUPPORTED, "cooperative launch not available on this device");
  CLS_CUDA_TRY(e, "persistent kernel");
  return CLS_OK;
}

int cls_persistent_status(const cls_problem* p, int32_t R, const void* ws, size_t ws_bytes,
                          int32_t* status) {
  int rc = check_R(p, R);
  if (rc != CLS_OK) return rc;
  if (!status) return set_err(CLS_ERR_INVALID, "status is NULL");
  const Layout L = layout_for(p, R);
  rc = check_ws(L, const_cast<void*>(ws), ws_bytes);
  if (rc != CLS_OK) return rc;
  int v = 0;
  CLS_CUDA_TRY(cudaMemcpy(&v, static_cast<const char*>(ws) + L.bar + 2 * sizeof(unsigned),
                          sizeof(int), cudaMemcpyDeviceToHost),
               "status copy");
  *status = v;
  return CLS_OK;
}

int cls_grid_barrier_check(int32_t rounds, int32_t extra, uint32_t spin_limit, void* scratch,
                           size_t scratch_bytes, int32_t* status, int32_t* passed) {
  if (rounds < 0 || extra < 0 || spin_limit == 0 || spin_limit > (1u << 24))
    return set_err(CLS_ERR_INVALID, "rounds/extra must be >= 0 and 0 < spin_limit <= 2^24");
  if (!scratch || scratch_bytes < 16) return set_err(CLS_ERR_INVALID, "scratch < 16 bytes");
  if (!status || !passed) return set_err(CLS_ERR_INVALID, "status/passed is NULL");
  unsigned* bar = static_cast<unsigned*>(scratch);
  cudaError_t e = cls::launch_barrier_check(rounds, (unsigned)extra, spin_limit, bar,
                                            reinterpret_cast<int*>(bar + 2),
                                            reinterpret_cast<int*>(bar + 3), nullptr);
  if (e == cudaErrorNotSupported)
    return set_err(CLS_ERR_UNSUPPORTED, "cooperative launch not available on this device");
  CLS_CUDA_TRY(e, "barrier check");
  CLS_CUDA_TRY(cudaStreamSynchronize(nullptr), "barrier check");
  int32_t v[2] = {0, 0};
  CLS_CUDA_TRY(cudaMemcpy(v, bar + 2, sizeof(v), cudaMemcpyDeviceToHost), "barrier check copy");
  *status = v[0];
  *passed = v[1];
  return CLS_OK;
}

int cls_solve_host_workspace_size(const cls_problem* p, int32_t R, size_t* bytes) {
  int rc = check_R(p, R);
  if (rc != CLS_OK) return rc;
  if (!bytes) return set_err(CLS_ERR_INVALID, "bytes is NULL");
  const Layout L = layout_for(p, R);
  *bytes = L.total + align_up((size_t)p->host.n * R * sizeof(float)) +
           align_up((size_t)R * sizeof(int32_t));
  return CLS_OK;
}

int cls_solve_host(const cls_problem* p, int32_t R, const float* x0_host, float lr,
                   int32_t n_steps, int32_t* nsat_host, float* x_host, void* ws,
                   size_t ws_bytes, void* stream) {
  int rc = check_R(p, R);
  if (rc != CLS_OK) return rc;
  if (n_steps < 0) return set_err(CLS_ERR_INVALID, "n_steps must be >= 0");
  if (R == 0) return CLS_OK;
  if ((!x0_host && p->host.n > 0) || !nsat_host)
    return set_err(CLS_ERR_INVALID, "x0_host and nsat_host are required");
  size_t need = 0;
  cls_solve_host_workspace_size(p, R, &need);
  if (!ws || reinterpret_cast<uintptr_t>(ws) % kAlign != 0 || ws_bytes < need)
    return set_err(CLS_ERR_WORKSPACE, "workspace missing, unaligned or smaller than " +
                                          std::to_string(need) + " bytes");
  const Layout L = layout_for(p, R);
  float* xd = at<float>(ws, L.total);
  int32_t* nd = at<int32_t>(ws, L.total + align_up((size_t)p->host.n * R * sizeof(float)));
  cudaStream_t s = (cudaStream_t)stream;
  const size_t xbytes = (size_t)p->host.n * R * sizeof(float);
  if (xbytes) CLS_CUDA_TRY(cudaMemcpyAsync(xd, x0_host, xbytes, cudaMemcpyHostToDevice, s), "H2D x0");
  // whole chunks of kSolveChunk steps through a recorded graph (the length
  // classes' FE launches run concurrently, each step's score overlaps the
  // next step's FE); the remaining steps as cls_step.  Same results.
  constexpr int kSolveChunk = 10;
  int32_t done_steps = 0;
  if (n_steps >= kSolveChunk && !p->hook) {
    const cls_problem* mp = p;
    if (!(mp->solve_graph && mp->sg_ws == ws && mp->sg_R == R && mp->sg_lr == lr &&
          mp->sg_epoch == p->list_epoch && mp->sg_unit == p->dev.unit_weights)) {
      if (mp->solve_graph) cls_graph_destroy(mp->solve_graph);
      mp->solve_graph = nullptr;
      cls_graph* g = nullptr;
      rc = cls_graph_create(p, R, xd, lr, kSolveChunk, nullptr, nd, nullptr, ws, L.total, &g);
      if (rc != CLS_OK) return rc;
      mp->solve_graph = g;
      mp->sg_ws = ws;
      mp->sg_R = R;
      mp->sg_lr = lr;
      mp->sg_epoch = p->list_epoch;
      mp->sg_unit = p->dev.unit_weights;
    }
    for (; done_steps + kSolveChunk <= n_steps; done_steps += kSolveChunk) {
      rc = cls_graph_launch(mp->solve_graph, stream);
      if (rc != CLS_OK) return rc;
    }
  }
  if (n_steps - done_steps > 0 || n_steps == 0) {
    rc = cls_step(p, R, xd, lr, n_steps - done_steps, nullptr, nd, nullptr, ws, L.total, stream);
    if (rc != CLS_OK) return rc;
  }
  if (n_steps == 0) {
    rc = cls_round_score(p, R, xd, nullptr, nd, nullptr, ws, L.total, stream);
    if (rc != CLS_OK) return rc;
  }
  CLS_CUDA_TRY(cudaMemcpyAsync(nsat_host, nd, (size_t)R * sizeof(int32_t), cudaMemcpyDeviceToHost, s),
               "D2H nsat");
  if (x_host && xbytes)
    CLS_CUDA_TRY(cudaMemcpyAsync(x_host, xd, xbytes, cudaMemcpyDeviceToHost, s), "D2H x");
  CLS_CUDA_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  return CLS_OK;
}

int cls_tuning_get(const cls_problem* p, int32_t* cfg, int32_t n) {
  if (!p || !cfg) return set_err(CLS_ERR_INVALID, "NULL argument");
  if (n != cls::kNumBuckets)
    return set_err(CLS_ERR_INVALID, "tuning has " + std::to_string(cls::kNumBuckets) + " entries");
  for (int b = 0; b < cls::kNumBuckets; ++b) cfg[b] = p->host.bucket_cfg[b];
  return CLS_OK;
}

int cls_tuning_set(cls_problem* p, const int32_t* cfg, int32_t n) {
  if (!p || !cfg) return set_err(CLS_ERR_INVALID, "NULL argument");
  if (n != cls::kNumBuckets)
    return set_err(CLS_ERR_INVALID, "tuning has " + std::to_string(cls::kNumBuckets) + " entries");
  cls::Tuning t;
  for (int b = 0; b < cls::kNumDftBuckets; ++b) t.dft[b] = cfg[b];
  for (int b = 0; b < cls::kNumRealBuckets; ++b) t.real[b] = cfg[cls::kNumDftBuckets + b];
  std::string msg;
  if (!cls::tuning_valid(t, &msg)) return set_err(CLS_ERR_INVALID, msg);
  int rc = pull_weights(p);
  if (rc != CLS_OK) return rc;
  cls::assign_groups(&p->host, t);
  return upload_lists(p);
}

int cls_config_info(int32_t id, int32_t* out) {
  if (!out) return set_err(CLS_ERR_INVALID, "NULL argument");
  if (id == cls::kCkptCfg) {   // checkpointed restart-parallel kernel, real roots
    out[0] = 1;
    out[1] = 1024;
    out[2] = 0;
    out[3] = 0;
    return CLS_OK;
  }
  if (id >= 0 && id < cls::kNumGroupCfg) {
    const cls::GroupCfg& g = cls::kGroupCfg[id];
    out[0] = g.G;
    out[1] = g.Q;
    out[2] = g.cplx;
    out[3] = g.ys;
    return CLS_OK;
  }
  const int b = id - 1000;   // 1000 + bucket: bucket kind and maximum length
  if (b >= 0 && b < cls::kNumBuckets) {
    out[0] = b < cls::kNumDftBuckets ? 1 : 0;
    out[1] = b < cls::kNumDftBuckets ? cls::kDftBucketMax[b]
                                     : cls::kRealBucketMax[b - cls::kNumDftBuckets];
    out[2] = 0;
    out[3] = 0;
    return CLS_OK;
  }
  return set_err(CLS_ERR_INVALID, "unknown configuration id");
}

int cls_autotune(cls_problem* p, int32_t R, const float* x, int32_t reps, void* ws,
                 size_t ws_bytes, void* stream) {
  int rc = check_R(p, R);
  if (rc != CLS_OK) return rc;
  if (R == 0 || p->host.m == 0) return CLS_OK;
  if (!x) return set_err(CLS_ERR_INVALID, "x is NULL");
  if (reps < 1) return set_err(CLS_ERR_INVALID, "reps must be >= 1");
  const Layout L = layout_for(p, R);
  rc = check_ws(L, ws, ws_bytes);
  if (rc != CLS_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  float* P = at<float>(ws, L.P);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CLS_CUDA_TRY(cudaEventCreate(&e0), "cudaEventCreate");
  CLS_CUDA_TRY(cudaEventCreate(&e1), "cudaEventCreate");
  const cls::DevPlan& D = p->dev;
  int chosen[cls::kNumBuckets];
  for (int b = 0; b < cls::kNumBuckets; ++b) chosen[b] = p->host.bucket_cfg[b];
  int result = CLS_OK;
  for (int b = 0; b < cls::kNumBuckets && result == CLS_OK; ++b) {
    if (D.bucket_count[b] == 0) continue;
    const bool dft = b < cls::kNumDftBuckets;
    const int bmax = dft ? cls::kDftBucketMax[b] : cls::kRealBucketMax[b - cls::kNumDftBuckets];
    float best = 1e30f;
    for (int id = 0; id <= cls::kNumGroupCfg && result == CLS_OK; ++id) {
      if (id == cls::kNumGroupCfg) {
        if (dft) break;
        id = cls::kCkptCfg;          // the checkpointed thread kernel (real buckets)
      } else {
        const cls::GroupCfg& g = cls::kGroupCfg[id];
        // candidates: right kind, able to hold the bucket's longest
        // constraint, at most twice the slots needed
        if ((g.cplx != 0) != dft || g.G * g.Q < bmax || g.G * g.Q > 2 * std::max(bmax, 32))
          continue;
      }
      cudaError_t e = cls::launch_group(id, D, D.bucket_list[b], D.bucket_count[b],
                                        D.bucket_maxL[b], D.bucket_maxJ[b], R, L.Rp, x, P, nullptr, 0,
                                        at<uint8_t>(ws, L.done), s);
      if (e == cudaSuccess) e = cudaEventRecord(e0, s);
      for (int k = 0; k < reps && e == cudaSuccess; ++k)
        e = cls::launch_group(id, D, D.bucket_list[b], D.bucket_count[b], D.bucket_maxL[b],
                              D.bucket_maxJ[b], R, L.Rp, x, P, nullptr, 0,
                              at<uint8_t>(ws, L.done), s);
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        (void)cudaGetLastError();
        result = cuda_err(e, "autotune");
        break;
      }
      if (ms < best) {
        best = ms;
        chosen[b] = id;
      }
      if (id == cls::kCkptCfg) break;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (result != CLS_OK) return result;
  return cls_tuning_set(p, chosen, cls::kNumBuckets);
}

}  // extern "C"

struct cls_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
  std::vector<cudaStream_t> streams;   // every stream created for the capture
  std::vector<cudaEvent_t> events;     // every event created for the capture
  int64_t launches = 0;
  // problems whose score was recorded with the all-weights-one kernel
  std::vector<const cls_problem*> unit_score;
};

namespace {

void graph_release(cls_graph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  for (auto e : g->events) cudaEventDestroy(e);
  for (auto s : g->streams) cudaStreamDestroy(s);
  if (g->cap) cudaStreamDestroy(g->cap);
  delete g;
}


// Streams and events of one problem's branch of a captured graph.
struct Branch {
  cudaStream_t main = nullptr;
  std::vector<cudaStream_t> side;   // FE side streams, then the score stream last
  std::vector<cudaEvent_t> ev;      // fork, score-done, then one join event per side
};

// Records the n-step loop of one problem into br.main (which must already be
// part of the capture).  FE units fork onto side streams (they write disjoint
// partial rows); step k's score runs on its own stream, concurrently with
// step k+1's FE, and step k+1's accumulate (which rewrites the bitset) waits
// for it.
int record_steps(const cls_problem* p, const Layout& L, const Branch& br, int64_t* launches,
                 float* x, float lr, int n_steps, uint32_t* bits, int32_t* nsat, double* wsat,
                 void* ws, bool score) {
  const cls::DevPlan& D = p->dev;
  float* P = at<float>(ws, L.P);
  // capture order: the DFT buckets longest first (the Chebyshev pass and
  // the dense kernels of the long constraints are the longest branches),
  // then the short closed forms, then the closed-form lane-group buckets
  std::vector<int> units;
  for (int b = cls::kNumDftBuckets - 1; b >= 0; --b)
    if (cls::fe_unit_active(D, cls::kNumThreadCls + b)) units.push_back(cls::kNumThreadCls + b);
  for (int u = 0; u < cls::kNumThreadCls; ++u)
    if (cls::fe_unit_active(D, u)) units.push_back(u);
  for (int u = cls::kNumThreadCls + cls::kNumDftBuckets; u < cls::kNumFeUnits; ++u)
    if (cls::fe_unit_active(D, u)) units.push_back(u);
  const int nside = (int)br.side.size();
  cudaEvent_t ev_fork = br.ev[0], ev_score = br.ev[1];
  cudaStream_t s_score = br.side[nside - 1];
  bool have_score = false;
  for (int st = 0; st < n_steps; ++st) {
    CLS_CUDA_TRY(cudaEventRecord(ev_fork, br.main), "fork");
    for (size_t i = 0; i < units.size(); ++i) {
      cudaStream_t s = br.side[i % (nside - 1)];
      CLS_CUDA_TRY(cudaStreamWaitEvent(s, ev_fork, 0), "fork wait");
      CLS_CUDA_TRY(cls::launch_fe_unit(D, units[i], L.R, L.Rp, x, P, nullptr, 0,
                                       at<uint8_t>(ws, L.done), s, nullptr),
                   "fe unit");
      (*launches)++;
    }
    for (int k = 0; k + 1 < nside && k < (int)units.size(); ++k) {
      CLS_CUDA_TRY(cudaEventRecord(br.ev[2 + k], br.side[k]), "join");
      CLS_CUDA_TRY(cudaStreamWaitEvent(br.main, br.ev[2 + k], 0), "join wait");
    }
    if (have_score) CLS_CUDA_TRY(cudaStreamWaitEvent(br.main, ev_score, 0), "score wait");
    CLS_CUDA_TRY(cls::launch_accum_step(D, L.R, L.Rp, P, x, lr, true, nullptr, bits, br.main,
                                        nullptr),
                 "accumulate/step kernel");
    (*launches)++;
    if (score) {
      CLS_CUDA_TRY(cudaEventRecord(ev_fork, br.main), "score fork");
      CLS_CUDA_TRY(cudaStreamWaitEvent(s_score, ev_fork, 0), "score fork wait");
      CLS_CUDA_TRY(cls::launch_score(D, L.R, L.Rp, bits, at<int32_t>(ws, L.nsat_part),
                                     at<double>(ws, L.wsat_part), nsat, wsat, s_score, nullptr),
                   "score kernels");
      *launches += D.m > 0 ? 2 : 0;
      CLS_CUDA_TRY(cudaEventRecord(ev_score, s_score), "score done");
      have_score = true;
    }
  }
  if (have_score) CLS_CUDA_TRY(cudaStreamWaitEvent(br.main, ev_score, 0), "final join");
  return CLS_OK;
}

// One side stream per FE unit and one score stream: every unit of a step is
// its own branch of the graph, so no unit waits on another that merely
// shared its stream (against 6 shared side streams: 4.26 -> 4.22 ms per
// step over the first 60 steps of the mixed workload).
constexpr int kSideStreams = cls::kNumFeUnits + 1;
// Side streams 0..kHighPrioStreams-1 (the longest units in capture order)
// carry the device's greatest stream priority; their kernel nodes keep it
// (the graph is instantiated with node priorities), so when SMs free up the
// long branches get them first.
constexpr int kHighPrioStreams = 8;

cudaError_t make_branch(Branch* br, bool own_main) {
  cudaError_t e = cudaSuccess;
  if (own_main) e = cudaStreamCreateWithFlags(&br->main, cudaStreamNonBlocking);
  int least = 0, greatest = 0;
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
  for (int i = 0; i < kSideStreams && e == cudaSuccess; ++i) {
    cudaStream_t s = nullptr;
    e = cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking,
                                     i < kHighPrioStreams ? greatest : least);
    if (e == cudaSuccess) br->side.push_back(s);
  }
  for (int i = 0; i < kSideStreams + 2 && e == cudaSuccess; ++i) {
    cudaEvent_t ev = nullptr;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) br->ev.push_back(ev);
  }
  return e;
}

void adopt(cls_graph* g, const Branch& br) {
  if (br.main) g->streams.push_back(br.main);
  for (auto s : br.side) g->streams.push_back(s);
  for (auto e : br.ev) g->events.push_back(e);
}

}  // namespace

extern "C" {

int cls_graph_create(const cls_problem* p, int32_t R, float* x, float lr, int32_t n_steps,
                     uint32_t* bits, int32_t* nsat, double* wsat, void* ws, size_t ws_bytes,
                     cls_graph** out) {
  if (!out) return set_err(CLS_ERR_INVALID, "out is NULL");
  *out = nullptr;
  int rc = check_R(p, R);
  if (rc != CLS_OK) return rc;
  if (R == 0 || (!x && p->host.n > 0)) return set_err(CLS_ERR_INVALID, "x is NULL or R == 0");
  return cls_batch_graph_create(1, &p, &R, &x, lr, n_steps, &bits, &nsat, &wsat, &ws, &ws_bytes,
                                out);
}

int cls_batch_graph_create(int32_t count, const cls_problem* const* ps, const int32_t* Rs,
                           float* const* xs, float lr, int32_t n_steps, uint32_t* const* bits,
                           int32_t* const* nsats, double* const* wsats, void* const* wss,
                           const size_t* ws_bytes, cls_graph** out) {
  if (!out) return set_err(CLS_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (count < 1 || !ps || !Rs || !xs || !wss || !ws_bytes)
    return set_err(CLS_ERR_INVALID, "count >= 1 and the per-problem arrays are required");
  if (n_steps < 1) return set_err(CLS_ERR_INVALID, "n_steps must be >= 1");
  std::vector<Layout> lays;
  for (int i = 0; i < count; ++i) {
    int rc = check_R(ps[i], Rs[i]);
    if (rc != CLS_OK) return rc;
    if (Rs[i] == 0 || (!xs[i] && ps[i]->host.n > 0))
      return set_err(CLS_ERR_INVALID, "x is NULL or R == 0 for problem " + std::to_string(i));
    if (ps[i]->hook) return set_err(CLS_ERR_INVALID, "disable profiling before capturing a graph");
    lays.push_back(layout_for(ps[i], Rs[i]));
    rc = check_ws(lays.back(), wss[i], ws_bytes[i]);
    if (rc != CLS_OK) return rc;
  }
  cls_graph* g = new (std::nothrow) cls_graph();
  if (!g) return set_err(CLS_ERR_NOMEM, "host allocation failed");
  cudaError_t e = cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking);
  std::vector<Branch> branches(count);
  cudaEvent_t ev_start = nullptr;
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_start, cudaEventDisableTiming);
  if (ev_start) g->events.push_back(ev_start);
  for (int i = 0; i < count && e == cudaSuccess; ++i) {
    // one problem alone records straight into the capture stream
    Branch& br = branches[i];
    if (count == 1) br.main = g->cap;
    e = make_branch(&br, count > 1);
    if (count == 1) br.main = nullptr, adopt(g, br), br.main = g->cap;
    else adopt(g, br);
  }
  if (e != cudaSuccess) {
    graph_release(g);
    (void)cudaGetLastError();
    return cuda_err(e, "graph resources");
  }
  e = cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    graph_release(g);
    (void)cudaGetLastError();
    return cuda_err(e, "cudaStreamBeginCapture");
  }
  int rc = CLS_OK;
  if (count > 1) {
    e = cudaEventRecord(ev_start, g->cap);
    for (int i = 0; i < count && e == cudaSuccess; ++i)
      e = cudaStreamWaitEvent(branches[i].main, ev_start, 0);
    if (e != cudaSuccess) rc = cuda_err(e, "batch fork");
  }
  for (int i = 0; i < count && rc == CLS_OK; ++i) {
    const cls_problem* p = ps[i];
    uint32_t* b = (bits && bits[i]) ? bits[i] : at<uint32_t>(wss[i], lays[i].bits);
    int32_t* ns = nsats ? nsats[i] : nullptr;
    double* wsv = wsats ? wsats[i] : nullptr;
    rc = record_steps(p, lays[i], branches[i], &g->launches, xs[i], lr, n_steps, b, ns, wsv,
                      wss[i], ns || wsv);
  }
  if (rc == CLS_OK && count > 1) {
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
      e = cudaEventRecord(branches[i].ev[1], branches[i].main);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(g->cap, branches[i].ev[1], 0);
    }
    if (e != cudaSuccess) rc = cuda_err(e, "batch join");
  }
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(g->cap, &graph);
  g->graph = graph;
  if (rc != CLS_OK || e != cudaSuccess) {
    graph_release(g);
    (void)cudaGetLastError();
    return rc != CLS_OK ? rc : cuda_err(e, "cudaStreamEndCapture");
  }
  // the kernel launches one graph launch performs: its kernel nodes (the
  // recording counted units, some of which launch several kernels)
  {
    size_t nn = 0;
    e = cudaGraphGetNodes(g->graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (e == cudaSuccess && nn) e = cudaGraphGetNodes(g->graph, nodes.data(), &nn);
    int64_t kernels = 0;
    for (size_t i = 0; i < nn && e == cudaSuccess; ++i) {
      cudaGraphNodeType ty;
      e = cudaGraphNodeGetType(nodes[i], &ty);
      if (e == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++kernels;
    }
    if (e != cudaSuccess) {
      graph_release(g);
      (void)cudaGetLastError();
      return cuda_err(e, "graph node count");
    }
    g->launches = kernels;
  }
  e = cudaGraphInstantiate(&g->exec, g->graph, cudaGraphInstantiateFlagUseNodePriority);
  if (e != cudaSuccess) {
    graph_release(g);
    (void)cudaGetLastError();
    return cuda_err(e, "cudaGraphInstantiate");
  }
  for (int i = 0; i < count; ++i)
    if (ps[i]->dev.unit_weights) g->unit_score.push_back(ps[i]);
  *out = g;
  return CLS_OK;
}

int cls_graph_launch(cls_graph* g, void* stream) {
  if (!g || !g->exec) return set_err(CLS_ERR_INVALID, "graph is NULL");
  for (const cls_problem* p : g->unit_score)
    if (!p->dev.unit_weights)
      return set_err(CLS_ERR_INVALID,
                     "weights changed after the graph was created with all weights 1; "
                     "create it again");
  CLS_CUDA_TRY(cudaGraphLaunch(g->exec, (cudaStream_t)stream), "cudaGraphLaunch");
  return CLS_OK;
}

int cls_graph_kernel_count(const cls_graph* g, int64_t* n) {
  if (!g || !n) return set_err(CLS_ERR_INVALID, "NULL argument");
  *n = g->launches;
  return CLS_OK;
}

int cls_graph_destroy(cls_graph* g) {
  graph_release(g);
  return CLS_OK;
}

}  // extern "C"

struct cls_mpnn {
  const cls_problem* p = nullptr;
  cls::mp::Graph G;
  std::vector<void*> allocations;
  int32_t* fan_in = nullptr;
  int64_t n_params = 0;
  size_t act_bytes = 0;
};

namespace {
template <typename T>
int upload_to(std::vector<void*>& allocs, const std::vector<T>& v, const T** out) {
  *out = nullptr;
  if (v.empty()) return CLS_OK;
  void* ptr = nullptr;
  cudaError_t e = cudaMalloc(&ptr, v.size() * sizeof(T));
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return set_err(e == cudaErrorMemoryAllocation ? CLS_ERR_NOMEM : CLS_ERR_CUDA,
                   std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  allocs.push_back(ptr);
  CLS_CUDA_TRY(cudaMemcpy(ptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice),
               "cudaMemcpy");
  *out = static_cast<const T*>(ptr);
  return CLS_OK;
}

void mpnn_free(cls_mpnn* g) {
  if (!g) return;
  for (void* a : g->allocations) cudaFree(a);
  delete g;
}

int check_act(const cls_mpnn* g, void* act, size_t act_bytes) {
  if (!act) return set_err(CLS_ERR_WORKSPACE, "activation workspace is NULL");
  if (reinterpret_cast<uintptr_t>(act) % kAlign != 0)
    return set_err(CLS_ERR_WORKSPACE, "activation workspace is not 256-byte aligned");
  if (act_bytes < g->act_bytes)
    return set_err(CLS_ERR_WORKSPACE, "activation workspace too small: need " +
                                          std::to_string(g->act_bytes) + " bytes");
  return CLS_OK;
}
}  // namespace

extern "C" {

int cls_mpnn_create(const cls_problem* p, cls_mpnn** out) {
  if (!p || !out) return set_err(CLS_ERR_INVALID, "NULL argument");
  *out = nullptr;
  const cls::HostPlan& H = p->host;
  const int n = H.n, m = H.m;
  std::vector<int32_t> con_off(m + 1, 0), con_var(H.nnz), var_con(H.nnz);
  std::vector<float> con_sgn(H.nnz), var_sgn(H.nnz), isL(m), isd(n);
  std::vector<float> fv((size_t)n * cls::mp::kFv), fc((size_t)m * cls::mp::kFc, 0.f);
  std::vector<int32_t> deg(n, 0), pos(n, 0);
  for (int c = 0; c < m; ++c) {
    const int lit0 = H.score[c].lit0, Lc = H.score[c].L;
    con_off[c + 1] = lit0 + Lc;
    isL[c] = 1.0f / std::sqrt((float)Lc);
    for (int e = lit0; e < lit0 + Lc; ++e) {
      const cls::LitRec& rc = H.lit[e];
      const float sg = rc.dst < 0 ? -1.f : 1.f;
      con_var[e] = rc.var;
      con_sgn[e] = sg;
      const int row = rc.dst & 0x7fffffff;
      var_con[row] = c;
      var_sgn[row] = sg;
      deg[rc.var]++;
      if (sg > 0) pos[rc.var]++;
    }
    // f_c = [onehot(type, 9), L/64, k/L, w]
    float* f = &fc[(size_t)c * cls::mp::kFc];
    f[H.ctype[c]] = 1.f;
    f[9] = (float)Lc / 64.f;
    f[10] = (float)H.kthr[c] / (float)Lc;
    f[11] = H.weight[c];
  }
  int n_free = n;
  for (int v = 0; v < n; ++v) {
    const float d1 = (float)std::max(deg[v], 1);
    isd[v] = 1.0f / std::sqrt(d1);
    float* f = &fv[(size_t)v * cls::mp::kFv];
    f[0] = 1.f;
    f[1] = (float)deg[v] / 16.f;
    f[2] = (float)pos[v] / d1;
    f[3] = (float)(deg[v] - pos[v]) / d1;
    if (!H.fixed.empty() && H.fixed[v]) n_free--;
  }
  cls_mpnn* g = new (std::nothrow) cls_mpnn();
  if (!g) return set_err(CLS_ERR_NOMEM, "host allocation failed");
  g->p = p;
  cls::mp::Graph& G = g->G;
  G.n = n;
  G.m = m;
  G.n_free = n_free;
  int rc = CLS_OK;
  auto up = [&](auto& vec, auto** dst) {
    if (rc == CLS_OK) rc = upload_to(g->allocations, vec, dst);
  };
  up(con_off, &G.con_off);
  up(con_var, &G.con_var);
  up(con_sgn, &G.con_sgn);
  up(H.voff, &G.var_off);
  up(var_con, &G.var_con);
  up(var_sgn, &G.var_sgn);
  up(isL, &G.isL);
  up(isd, &G.isd);
  up(fv, &G.fv);
  up(fc, &G.fc);
  std::vector<int32_t> fan = cls::mp::fan_in_table();
  const int32_t* fan_dev = nullptr;
  up(fan, &fan_dev);
  if (rc != CLS_OK) {
    mpnn_free(g);
    return rc;
  }
  g->fan_in = const_cast<int32_t*>(fan_dev);
  G.fixed = p->dev.fixed;
  G.fixed_val = p->dev.fixed_val;
  g->n_params = cls::mp::param_layout().total;
  g->act_bytes = cls::mp::act_layout(n, m).total_floats * sizeof(float);
  *out = g;
  return CLS_OK;
}

int cls_mpnn_destroy(cls_mpnn* g) {
  mpnn_free(g);
  return CLS_OK;
}

int cls_mpnn_sizes(const cls_mpnn* g, int64_t* n_params, size_t* act_bytes) {
  if (!g || !n_params || !act_bytes) return set_err(CLS_ERR_INVALID, "NULL argument");
  *n_params = g->n_params;
  *act_bytes = g->act_bytes;
  return CLS_OK;
}

int cls_mpnn_param_init(const cls_mpnn* g, uint64_t seed, float* params, void* stream) {
  if (!g || !params) return set_err(CLS_ERR_INVALID, "NULL argument");
  CLS_CUDA_TRY(cls::mp::param_init(g->fan_in, g->n_params, seed, params, (cudaStream_t)stream),
               "param init kernel");
  return CLS_OK;
}

int cls_mpnn_forward(const cls_mpnn* g, const float* params, float* z, void* act,
                     size_t act_bytes, void* stream) {
  if (!g || !params || (!z && g->G.n > 0)) return set_err(CLS_ERR_INVALID, "NULL argument");
  int rc = check_act(g, act, act_bytes);
  if (rc != CLS_OK) return rc;
  CLS_CUDA_TRY(cls::mp::forward(g->G, params, z, static_cast<float*>(act), (cudaStream_t)stream),
               "mpnn forward");
  return CLS_OK;
}

int cls_mpnn_points(const cls_mpnn* g, const float* z, int32_t R, uint64_t seed, int64_t r_offset,
                    float tau, float* x0, void* stream) {
  if (!g) return set_err(CLS_ERR_INVALID, "NULL argument");
  int rc = check_R(g->p, R);
  if (rc != CLS_OK) return rc;
  if (R == 0 || g->G.n == 0) return CLS_OK;
  if (!z || !x0) return set_err(CLS_ERR_INVALID, "z and x0 are required");
  if (r_offset < 0) return set_err(CLS_ERR_INVALID, "r_offset must be >= 0");
  CLS_CUDA_TRY(cls::mp::points(g->G, z, R, seed, r_offset, tau, x0, (cudaStream_t)stream),
               "points kernel");
  return CLS_OK;
}

int cls_mpnn_head_grad(const cls_mpnn* g, const float* z, const float* x0, const float* gx0,
                       int32_t R, const int8_t* target, float lam, float* dz, void* stream) {
  if (!g) return set_err(CLS_ERR_INVALID, "NULL argument");
  int rc = check_R(g->p, R);
  if (rc != CLS_OK) return rc;
  if (g->G.n == 0) return CLS_OK;
  if (!z || !dz || (gx0 && !x0)) return set_err(CLS_ERR_INVALID, "z, dz (and x0 with gx0) required");
  CLS_CUDA_TRY(cls::mp::head_grad(g->G, z, x0, gx0, R, target, lam, dz, (cudaStream_t)stream),
               "head gradient kernel");
  return CLS_OK;
}

int cls_mpnn_backward(const cls_mpnn* g, const float* params, const float* dz, float* dparams,
                      void* act, size_t act_bytes, void* stream) {
  if (!g || !params || !dparams || (!dz && g->G.n > 0))
    return set_err(CLS_ERR_INVALID, "NULL argument");
  int rc = check_act(g, act, act_bytes);
  if (rc != CLS_OK) return rc;
  CLS_CUDA_TRY(cls::mp::backward(g->G, params, dz, dparams, static_cast<float*>(act),
                                 (cudaStream_t)stream),
               "mpnn backward");
  return CLS_OK;
}

int cls_adam_step(int64_t n, float* params, const float* grads, float* m, float* v, float lr,
                  float beta1, float beta2, float eps, int32_t t, void* stream) {
  if (n < 0 || (n > 0 && (!params || !grads || !m || !v)) || t < 1)
    return set_err(CLS_ERR_INVALID, "bad Adam arguments");
  CLS_CUDA_TRY(cls::mp::adam(n, params, grads, m, v, lr, beta1, beta2, eps, t,
                             (cudaStream_t)stream),
               "adam kernel");
  return CLS_OK;
}

int cls_profile_enable(cls_problem* p, int on) {
  if (!p) return set_err(CLS_ERR_INVALID, "problem is NULL");
  p->hook = on ? &p->events : nullptr;
  return CLS_OK;
}

int cls_profile_reset(cls_problem* p) {
  if (!p) return set_err(CLS_ERR_INVALID, "problem is NULL");
  p->events.reset();
  return CLS_OK;
}

int cls_profile_read(cls_problem* p, int kc, int64_t* launches, double* total_ms) {
  if (!p || !launches || !total_ms) return set_err(CLS_ERR_INVALID, "NULL argument");
  if (kc < 0 || kc >= cls::KC_COUNT) return set_err(CLS_ERR_INVALID, "unknown kernel class");
  int64_t n = 0;
  double ms = 0.0;
  for (auto& r : p->events.recs) {
    if (r.kc != kc) continue;
    CLS_CUDA_TRY(cudaEventSynchronize(r.b), "cudaEventSynchronize");
    float t = 0.f;
    CLS_CUDA_TRY(cudaEventElapsedTime(&t, r.a, r.b), "cudaEventElapsedTime");
    ms += t;
    n++;
  }
  *launches = n;
  *total_ms = ms;
  return CLS_OK;
}

const char* cls_strerror(int code) {
  switch (code) {
    case CLS_OK: return "ok";
    case CLS_ERR_INVALID: return "invalid argument";
    case CLS_ERR_CUDA: return "CUDA error";
    case CLS_ERR_NOMEM: return "out of memory";
    case CLS_ERR_UNSUPPORTED: return "unsupported device";
    case CLS_ERR_WORKSPACE: return "bad workspace";
    default: return "unknown error";
  }
}

const char* cls_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
