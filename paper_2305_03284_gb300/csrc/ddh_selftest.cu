// Self-test of the device-side bounded wait (failure detection without a fault).
//
// One thread waits on a shared-memory mbarrier that nothing ever arrives at, polling it with
// the non-blocking mbarrier.test_wait until `limit_ns` of the global timer have passed; it then
// latches kStatusTimeout in the stream's status word, exactly as the step kernel does when its
// frame copy does not complete within its poll limit, and the kernel returns.  The context stays
// usable: the host reads DDH_ETIMEOUT at its next synchronising call and may step again.  The
// loop ends on elapsed time, so it cannot hang whatever the barrier does.
#include <cstdint>

#include "ddh_device.cuh"
#include "ddh_kernels.cuh"

namespace ddh {
namespace {

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__global__ void k_wait_selftest(unsigned* status, uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);  // one expected arrival, which never comes
  const uint64_t t0 = global_ns();
  bool done = false;
  while (!done && global_ns() - t0 < limit_ns) done = mbar_test_wait(&bar, 0);
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(&bar)) : "memory");
  if (!done) atomicOr(status, kStatusTimeout);
}

}  // namespace

cudaError_t launch_wait_selftest(unsigned* status, uint64_t limit_ns, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(status, limit_ns);
  return cudaGetLastError();
}

}  // namespace ddh
