// Split-bf16 tcgen05 evaluator (placeholder until the kernel lands).
#include "common.cuh"
#include "kernels.cuh"

namespace usaphmp {

int tc_tile_rows() { return 128; }
void prepare_eval_tc() {}

__global__ void k_tc_unavailable(uint32_t* status) { atomicOr(status, kStatusBadValue); }

void launch_eval_tc(const TaskSet&, int, uint32_t* status, cudaStream_t s) {
  k_tc_unavailable<<<1, 1, 0, s>>>(status);
}

}  // namespace usaphmp
