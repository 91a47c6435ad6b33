// Self-check of the bounded device wait that guards every TMA pipeline of the
// step kernels: one thread waits, with a short poll limit, on an mbarrier
// whose phase nothing completes, and flags the time-out the way the step
// kernels do; the host turns the flag into FWI_ERR_TIMEOUT.  Nothing is in
// flight on the barrier (no copy, no other waiter), so giving up is safe and
// the context stays usable.
#include "fwi_plan.cuh"
#include "tma_util.cuh"

namespace fwi {

namespace {

__global__ void k_wait_check(uint32_t polls, int* flag) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tma::mbar_init(&bar, 1);
    tma::fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !tma::mbar_wait_bounded(&bar, 0u, polls)) atomicOr(flag, 2);
}

}  // namespace

}  // namespace fwi

using namespace fwi;

extern "C" fwi_status fwi_check_bounded_wait(unsigned int polls) {
  if (polls < 1 || polls > (1u << 22)) return fail(FWI_ERR_INVALID_ARG, "polls must be in [1, 2^22]");
  int* d_flag = nullptr;
  CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(&d_flag), sizeof(int)));
  int flag = 0;
  cudaError_t e = cudaMemset(d_flag, 0, sizeof(int));
  if (e == cudaSuccess) {
    k_wait_check<<<1, 32>>>(polls, d_flag);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d_flag);
  if (e != cudaSuccess) return fail(FWI_ERR_CUDA, cudaGetErrorString(e));
  if (flag & 2)
    return fail(FWI_ERR_TIMEOUT, "bounded wait gave up after " + std::to_string(polls) +
                                     " polls (self-check)");
  return fail(FWI_ERR_CUDA, "bounded wait self-check: an mbarrier phase completed with no arrival");
}
