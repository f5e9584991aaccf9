// Fitness assembly: fit_b = t12_b + alpha * T3_b, with T3_b the sum of the
// evaluator's partial transfer sums part[r][b] taken in a fixed order (r
// ascending), so a chromosome's fitness does not depend on the launch it was
// evaluated in; times the output scale of §4.3 (1, 10^-3 or 1/sum W) for
// values returned to the caller.
#include "common.cuh"
#include "kernels.cuh"

namespace usaphmp {

__global__ void k_reduce(const __grid_constant__ TaskParam tp) {
  pdl_wait();
  pdl_allow_next();
  const int t = task_of(tp.bo, blockIdx.x);
  const Task& T = task_at(tp, t);
  const int b = (blockIdx.x - tp.bo.o[t]) * blockDim.x + threadIdx.x;
  const int B = T.pop.B;
  // every kernel that can raise the status ran before this one
  if (b == 0 && T.pop.status_host) {
    T.pop.status_host[0] = *T.pop.status;
    T.pop.status_host[1] = (uint32_t)*T.pop.bad;
  }
  if (b >= B) return;
  const float s = sum_rows_in_order(T.pop.part + b, T.pop.npart, B);
  T.pop.fit[b] = (T.pop.t12[b] + T.in.alpha * s) * T.pop.out_scale;
}

void launch_reduce(const TaskSet& ts, cudaStream_t s) {
  TaskParam tp = make_param(ts);
  for (int t = 0; t < ts.count; ++t) tp.bo.o[t + 1] = tp.bo.o[t] + (ts.h[t].pop.B + 127) / 128;
  const int blocks = tp.bo.o[ts.count];
  if (blocks == 0) return;
  launch_pdl(k_reduce, blocks, 128, 0, s, tp);
}

}  // namespace usaphmp
