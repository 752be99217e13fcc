// Throughput of the arithmetic pipes the interaction kernel lives on, for the
// roofline's issue ceilings: one CTA of 1024 threads per SM (each CTA reserves
// more than half of an SM's shared memory, so no SM holds two) runs eight
// independent dependency chains per thread of one operation, and the SM's own
// cycle counter (clock64) times it, so the rate is in operations (lanes) per
// clock per SM whatever the clock frequency.
#include <algorithm>

#include "internal.cuh"

namespace bldtt {

constexpr int kRateThreads = 1024;

enum RateOp { kOpFfma = 0, kOpFfma2 = 1, kOpRsqrt = 2, kOpEx2 = 3, kOpDfma = 4 };

template <int OP>
__global__ void __launch_bounds__(kRateThreads) k_rate(int iters, float seed, float* __restrict__ sink,
                                                       long long* __restrict__ cycles) {
  float a[8];
  double d[8];
  unsigned long long p[4];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    a[k] = seed + 1e-3f * (float)(threadIdx.x + k);
    d[k] = (double)a[k];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) asm("mov.b64 %0, {%1, %2};" : "=l"(p[k]) : "f"(a[2 * k]), "f"(a[2 * k + 1]));
  unsigned long long c2;
  {
    const float c = 0.999f;
    asm("mov.b64 %0, {%1, %1};" : "=l"(c2) : "f"(c));
  }
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (OP == kOpFfma) a[k] = fmaf(a[k], 0.999f, 1e-4f);
      if (OP == kOpRsqrt) asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(a[k]));
      if (OP == kOpEx2)   // 2^-a: a bounded chain (a -> ~0.64)
        asm volatile("{ .reg .f32 t; neg.f32 t, %0; ex2.approx.ftz.f32 %0, t; }" : "+f"(a[k]));
      if (OP == kOpDfma) d[k] = fma(d[k], 0.999, 1e-4);
    }
    if (OP == kOpFfma2) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {   // 4 packed chains, twice: 8 packed operations = 16 lanes
        asm volatile("fma.rn.f32x2 %0, %0, %1, %1;" : "+l"(p[k]) : "l"(c2));
        asm volatile("fma.rn.f32x2 %0, %0, %1, %1;" : "+l"(p[k]) : "l"(c2));
      }
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k] + (float)d[k];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(p[k]));
    s += lo + hi;
  }
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// Dynamic shared memory the CTAs reserve (unused) so that no SM holds two.
constexpr int kRateSmem = 120 * 1024;

template <int OP>
static int rate(int sms, int iters, float* sink, long long* cycles, cudaStream_t s, double* out) {
  BL_CUDA(cudaFuncSetAttribute(k_rate<OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRateSmem));
  k_rate<OP><<<sms, kRateThreads, kRateSmem, s>>>(iters, 0.75f, sink, cycles);
  int64_t dummy = 0;
  BL_LAUNCHED(dummy);
  std::vector<long long> h(sms);
  BL_CUDA(cudaMemcpyAsync(h.data(), cycles, sms * sizeof(long long), cudaMemcpyDeviceToHost, s));
  BL_CUDA(cudaStreamSynchronize(s));
  std::sort(h.begin(), h.end());
  const double lanes = (double)kRateThreads * iters * (OP == kOpFfma2 ? 16 : 8);
  *out = lanes / (double)h[sms / 2];   // median CTA
  return BLDTT_OK;
}

}  // namespace bldtt

using namespace bldtt;

extern "C" int bldtt_pipe_rates(double* out, void* cuda_stream) {
  if (!out) {
    set_error("pipe_rates: out is NULL");
    return BLDTT_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0;
  BL_CUDA(cudaGetDevice(&dev));
  BL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  float* sink = nullptr;
  long long* cycles = nullptr;
  BL_TRY(dalloc_n(&sink, (size_t)sms * kRateThreads, s));
  BL_TRY(dalloc_n(&cycles, (size_t)sms, s));
  int rc = rate<kOpFfma>(sms, 4096, sink, cycles, s, &out[0]);
  if (rc == BLDTT_OK) rc = rate<kOpFfma2>(sms, 2048, sink, cycles, s, &out[1]);
  if (rc == BLDTT_OK) rc = rate<kOpRsqrt>(sms, 1024, sink, cycles, s, &out[2]);
  if (rc == BLDTT_OK) rc = rate<kOpEx2>(sms, 1024, sink, cycles, s, &out[3]);
  if (rc == BLDTT_OK) rc = rate<kOpDfma>(sms, 256, sink, cycles, s, &out[4]);
  dfree(sink, s);
  dfree(cycles, s);
  return rc;
}

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
