// Pipe-throughput microbenchmark behind the benchmark's issue ceilings.  It is
// measurement tooling, built into its own library (libbldtt_pipes.so) that only
// bench.py and its test load; the BLDTT library does not contain it.
//
// One CTA of 1024 threads per SM (each CTA reserves more than half of an SM's
// shared memory, so no SM holds two) runs eight independent dependency chains
// per thread of one operation, and the SM's own cycle counter (clock64) times
// it, so the rate is in operations (lanes) per clock per SM whatever the clock
// frequency.
//
// C ABI:
//   int pipes_rates(double* out, void* cuda_stream)
//     out: host, 5 doubles: lanes per clock per SM of FP32 FMA, packed FP32x2
//     FMA (two lanes per instruction), MUFU rsqrt, MUFU exp2 and FP64 FMA
//     (median CTA).  Synchronous on cuda_stream.  Returns 0, or the CUDA error
//     code of the first failing call (message from pipes_last_error()).
//   const char* pipes_last_error(void)
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <vector>

namespace {

constexpr int kRateThreads = 1024;
constexpr int kRateSmem = 120 * 1024;   // dynamic shared memory reserved, unused

enum RateOp { kOpFfma = 0, kOpFfma2 = 1, kOpRsqrt = 2, kOpEx2 = 3, kOpDfma = 4 };

char g_msg[256] = "";

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

int fail(cudaError_t e, const char* what) {
  std::snprintf(g_msg, sizeof(g_msg), "%s failed: %s", what, cudaGetErrorString(e));
  return (int)e;
}

#define PIPES_CUDA(call)                          \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return fail(e_, #call); \
  } while (0)

template <int OP>
int rate(int sms, int iters, float* sink, long long* cycles, cudaStream_t s, double* out) {
  PIPES_CUDA(cudaFuncSetAttribute(k_rate<OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRateSmem));
  k_rate<OP><<<sms, kRateThreads, kRateSmem, s>>>(iters, 0.75f, sink, cycles);
  PIPES_CUDA(cudaGetLastError());
  std::vector<long long> h(sms);
  PIPES_CUDA(cudaMemcpyAsync(h.data(), cycles, sms * sizeof(long long), cudaMemcpyDeviceToHost, s));
  PIPES_CUDA(cudaStreamSynchronize(s));
  std::sort(h.begin(), h.end());
  const double lanes = (double)kRateThreads * iters * (OP == kOpFfma2 ? 16 : 8);
  *out = lanes / (double)h[sms / 2];   // median CTA
  return 0;
}

int rates_all(int sms, float* sink, long long* cycles, cudaStream_t s, double* out) {
  int rc = rate<kOpFfma>(sms, 4096, sink, cycles, s, &out[0]);
  if (rc == 0) rc = rate<kOpFfma2>(sms, 2048, sink, cycles, s, &out[1]);
  if (rc == 0) rc = rate<kOpRsqrt>(sms, 1024, sink, cycles, s, &out[2]);
  if (rc == 0) rc = rate<kOpEx2>(sms, 1024, sink, cycles, s, &out[3]);
  if (rc == 0) rc = rate<kOpDfma>(sms, 256, sink, cycles, s, &out[4]);
  return rc;
}

}  // namespace

extern "C" int pipes_rates(double* out, void* cuda_stream) {
  if (!out) {
    std::snprintf(g_msg, sizeof(g_msg), "pipes_rates: out is NULL");
    return -1;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0;
  PIPES_CUDA(cudaGetDevice(&dev));
  PIPES_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  float* sink = nullptr;
  long long* cycles = nullptr;
  PIPES_CUDA(cudaMalloc(&sink, (size_t)sms * kRateThreads * sizeof(float)));
  cudaError_t e = cudaMalloc(&cycles, (size_t)sms * sizeof(long long));
  if (e != cudaSuccess) {
    cudaFree(sink);
    return fail(e, "cudaMalloc");
  }
  const int rc = rates_all(sms, sink, cycles, s, out);
  cudaFree(sink);
  cudaFree(cycles);
  return rc;
}

extern "C" const char* pipes_last_error(void) { return g_msg; }
