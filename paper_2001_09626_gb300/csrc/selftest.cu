// Self-test of the failure path that every tensor-core kernel of the library
// takes when one of its mbarrier waits (TMA or MMA completion) runs out: the
// CTA holds tensor memory, polls an mbarrier a bounded number of times, gives
// up, frees the tensor memory and returns, and the host reads the outcome.
// Here nothing ever arrives on the barrier, so the wait must run out.
#include "tc.cuh"

namespace afi {

__global__ void k_selftest_wait(long long polls, long long *out) {
  using namespace tc;
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t slot;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&slot)),
               "r"(32));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = slot;
  long long used = 0;
  const bool done = wait_phase_n(&bar, 0, polls, &used);   // no arrival is ever made
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32));
  if (threadIdx.x == 0) {
    out[0] = done ? 1 : 0;
    out[1] = used;
  }
}

}  // namespace afi

extern "C" afi_status afi_selftest_bounded_wait(long long polls, long long *polls_used) {
  using namespace afi;
  if (polls < 1 || polls > (1LL << 22)) {
    set_error("afi_selftest_bounded_wait: polls must be in [1, 2^22]");
    return AFI_EINVAL;
  }
  long long *d = nullptr, h[2] = {0, 0};
  AFI_CUDA(cudaMalloc(&d, 2 * sizeof(long long)));
  launch(k_selftest_wait, 1, 32, 0, (cudaStream_t)0, polls, d);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) {
    set_error(std::string("afi_selftest_bounded_wait: ") + cudaGetErrorString(e));
    return AFI_ECUDA;
  }
  if (polls_used) *polls_used = h[1];
  return h[0] ? AFI_OK : AFI_ETIMEOUT;
}
