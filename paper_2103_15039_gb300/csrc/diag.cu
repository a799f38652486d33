// Diagnostic of the failure path of the E step's copy pipeline: the bounded
// wait (pipeline.cuh) on a barrier that nothing completes (no copy is issued)
// must give up after `budget` cycles and report the timeout in the status word,
// leaving the context usable.
#include "internal.cuh"
#include "pipeline.cuh"

namespace lsg {
namespace {

__global__ void wait_selftest_kernel(long long budget, int* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0, budget)) atomicOr(status, kStatusTimeout);
}

}  // namespace

cudaError_t launch_wait_selftest(long long budget, int* status, cudaStream_t s) {
  wait_selftest_kernel<<<1, 32, 0, s>>>(budget, status);
  return cudaGetLastError();
}

}  // namespace lsg
