// Failure detection without a fault: the bounded-wait pattern of the
// interaction kernel's ring, run on an mbarrier that nothing arrives on
// (bldtt_wait_probe).
#include "internal.cuh"

namespace bldtt {

// The bounded-wait pattern of the interaction kernel's ring (try_wait on an
// mbarrier phase until %globaltimer passes the limit, then the error flag),
// on a barrier that nothing arrives on.
__global__ void k_wait_probe(unsigned long long limit_ns, int* __restrict__ err) {
  __shared__ __align__(8) unsigned long long bar;
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  unsigned long long t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(0u)
        : "memory");
    if (ok) return;                       // cannot happen: no arrival
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > limit_ns) {
      atomicExch(err, kDevErrTimeout);
      return;
    }
  }
}

}  // namespace bldtt

using namespace bldtt;

extern "C" int bldtt_wait_probe(int64_t limit_ns, void* cuda_stream) {
  if (limit_ns < 1000 || limit_ns > 1000000000LL) {
    set_error("wait_probe: limit_ns %lld outside [1000, 1e9]", (long long)limit_ns);
    return BLDTT_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int* err = nullptr;
  BL_TRY(dalloc_n(&err, 1, s));
  BL_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  k_wait_probe<<<1, 32, 0, s>>>((unsigned long long)limit_ns, err);
  int64_t dummy = 0;
  BL_LAUNCHED(dummy);
  int h = 0;
  BL_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  BL_CUDA(cudaStreamSynchronize(s));
  dfree(err, s);
  if (h == kDevErrTimeout) {
    set_error("wait_probe: the bounded wait gave up after %lld ns (expected)", (long long)limit_ns);
    return BLDTT_ETIMEOUT;
  }
  set_error("wait_probe: the wait completed without an arrival");
  return BLDTT_EINTERNAL;
}
