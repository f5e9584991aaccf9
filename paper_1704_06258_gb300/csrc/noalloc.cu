// FP64 rescoring that allocates nothing: the per-block partial sums of the
// rescoring kernels live in a fixed array compiled into the library instead
// of a cudaMalloc'ed buffer.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>
#include <string>

#include "usaphmp.h"
#include "common.cuh"
#include "kernels.cuh"

namespace usaphmp {
namespace {

// Scratch for usaphmp_rescore_fp64_noalloc: fp64 partial sums, one per
// (chromosome, row block).  1 MiB on every device that loads the library.
constexpr size_t kNoAllocScratchDoubles = 131072;
__device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

constexpr int kMaxDevices = 256;

// The scratch array's device address on each device, with the id of the
// CUDA context it was looked up in.  Host code only sees a stand-in symbol,
// not a device address, so the address is looked up (cudaGetSymbolAddress)
// with the device current, once per context: when the device's context is
// destroyed (cudaDeviceReset) and made again, the module is loaded again,
// possibly elsewhere, and the next call looks the address up anew.
struct ScratchSite {
  unsigned long long ctx_id = 0;
  bool valid = false;
  double* addr = nullptr;
};
std::mutex g_scratch_mu;
ScratchSite g_scratch[kMaxDevices];

// Driver entry points that name the current context (fetched once; null
// when the driver lacks them, and the address is then looked up on every call).
struct CtxApi {
  PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
  PFN_cuCtxGetId_v12000 get_id = nullptr;
};

const CtxApi& ctx_api() {
  static const CtxApi api = [] {
    CtxApi a;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      a.get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(fn);
    fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      a.get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(fn);
    return a;
  }();
  return api;
}

// Id of the calling thread's current context; false when there is none yet
// or the driver cannot say.
bool current_ctx_id(unsigned long long* id) {
  const CtxApi& api = ctx_api();
  if (!api.get_current || !api.get_id) return false;
  CUcontext ctx = nullptr;
  if (api.get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
  return api.get_id(ctx, id) == CUDA_SUCCESS;
}

int scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return report_error(USAPHMP_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return report_error(USAPHMP_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  ScratchSite& site = g_scratch[dev];
  unsigned long long id = 0;
  const bool known = current_ctx_id(&id);
  if (known && site.valid && site.ctx_id == id) {
    *out = site.addr;
    return USAPHMP_OK;
  }
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    return report_error(USAPHMP_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  // the lookup makes the device's context current if no runtime call had yet
  site.valid = current_ctx_id(&site.ctx_id);
  site.addr = static_cast<double*>(p);
  *out = site.addr;
  return USAPHMP_OK;
}

}  // namespace
}  // namespace usaphmp

extern "C" int usaphmp_rescore_fp64_noalloc(int32_t n, int32_t p, int32_t B, const float* W, const float* C,
                                            double chi, double alpha, double delta, const int32_t* hubs,
                                            const uint8_t* slot, double* cost, void* stream) {
  using namespace usaphmp;
  if (!W || !C || !hubs || !slot || !cost) return report_error(USAPHMP_EINVAL, "NULL argument");
  if (n < 2 || n > kMaxN) return report_error(USAPHMP_EINVAL, "n must be in [2, 16384]");
  if (p < 1 || p > n || p > kMaxP) return report_error(USAPHMP_EINVAL, "p must be in [1, min(n, 255)]");
  if (B < 0) return report_error(USAPHMP_EINVAL, "B < 0");
  if (B == 0) return USAPHMP_OK;
  const size_t need = (size_t)B * (size_t)rescore_parts(n);
  if (need > kNoAllocScratchDoubles)
    return report_error(USAPHMP_EINVAL, "usaphmp_rescore_fp64_noalloc: B * min(n, 128) = " + std::to_string(need) +
                                            " exceeds the fixed scratch of " + std::to_string(kNoAllocScratchDoubles) +
                                            " partial sums");
  double* scratch = nullptr;
  const int r = scratch_address(&scratch);
  if (r != USAPHMP_OK) return r;
  DevInst in{};
  in.n = n; in.p = p; in.ldw = n; in.ns = n; in.nw = (n + 31) / 32; in.symmetric = 0;
  in.chi = (float)chi; in.alpha = (float)alpha; in.delta = (float)delta;
  in.chi_d = chi; in.alpha_d = alpha; in.delta_d = delta;
  in.W = W; in.C = C; in.CT = C;
  launch_rescore(in, B, hubs, slot, scratch, cost, static_cast<cudaStream_t>(stream));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return report_error(USAPHMP_ECUDA, std::string("rescore launch: ") + cudaGetErrorString(e));
  return USAPHMP_OK;
}
