// FP64 rescoring that allocates nothing: the per-block partial sums of the
// rescoring kernels live in a fixed array compiled into the library instead
// of a cudaMalloc'ed buffer.
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
std::mutex g_scratch_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (host code only sees a stand-in symbol, not a device address).
int scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return report_error(USAPHMP_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return report_error(USAPHMP_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return report_error(USAPHMP_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
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
