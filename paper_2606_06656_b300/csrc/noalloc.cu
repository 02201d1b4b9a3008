// noalloc.cu -- a CLS step entry point that allocates no memory.
//
// Some callers cannot allocate device memory once they are running: a
// real-time loop that must not call into the allocator after start-up, code
// living under another runtime's fixed device-memory budget, or a host
// language with no way to reach cudaMalloc.  For them the scratch that
// cls_step normally takes from a caller-supplied workspace (literal partials,
// the rounded bitset, per-chunk score partials) lives in one file-scope
// device array of fixed size instead.  Every GPU that loads this library
// holds that array until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/cls.h"

namespace cls {
int set_error(int code, const std::string& msg);   // api.cu
bool profiling_enabled(const cls_problem* p);       // api.cu
int problem_device(const cls_problem* p);           // api.cu
}  // namespace cls

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;   // 32 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch per device.  In host code the array's
// name is only a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress, once per device, with that device current.  A
// cudaDeviceReset (or any teardown of the device's primary context) makes the
// cached address stale; such a process must not call cls_step_noalloc again.
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

int scratch_for_current_device(int want_dev, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return cls::set_error(CLS_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  }
  // The problem's tables live on the device it was created on; the scratch
  // must be that device's copy of the array, so the caller's current device
  // has to match.
  if (dev != want_dev)
    return cls::set_error(CLS_ERR_INVALID,
                          "cls_step_noalloc: current device " + std::to_string(dev) +
                              " is not the problem's device " + std::to_string(want_dev));
  if (dev < 0 || dev >= kMaxDevices)
    return cls::set_error(CLS_ERR_UNSUPPORTED, "device index beyond the static scratch table");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess || !ptr) {
      (void)cudaGetLastError();
      return cls::set_error(CLS_ERR_CUDA, std::string("cudaGetSymbolAddress: ") +
                                              cudaGetErrorString(e));
    }
    g_scratch_addr[dev] = ptr;
  }
  *out = g_scratch_addr[dev];
  return CLS_OK;
}

}  // namespace

extern "C" int cls_step_noalloc(const cls_problem* p, int32_t R, float* x, float lr,
                                int32_t n_steps, uint32_t* bits, int32_t* nsat, double* wsat,
                                void* stream) {
  if (!p) return cls::set_error(CLS_ERR_INVALID, "problem is NULL");
  if (cls::profiling_enabled(p))
    return cls::set_error(CLS_ERR_INVALID,
                          "cls_step_noalloc: profiling creates CUDA events; disable it first");
  size_t need = 0;
  int rc = cls_workspace_size(p, R, &need);
  if (rc != CLS_OK) return rc;
  if (need > kStaticScratchBytes)
    return cls::set_error(CLS_ERR_WORKSPACE,
                          "cls_step_noalloc: this problem needs " + std::to_string(need) +
                              " bytes of scratch for R=" + std::to_string(R) +
                              ", more than the static limit of " +
                              std::to_string(kStaticScratchBytes) + " bytes (use cls_step)");
  void* scratch = nullptr;
  rc = scratch_for_current_device(cls::problem_device(p), &scratch);
  if (rc != CLS_OK) return rc;
  // Nothing in the step reads scratch before writing it in the same call, so
  // the array needs no clearing between calls.
  return cls_step(p, R, x, lr, n_steps, bits, nsat, wsat, scratch, kStaticScratchBytes, stream);
}
