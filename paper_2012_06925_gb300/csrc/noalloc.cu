// Allocation-free variant of the bounding-box reduction that bldtt_setup
// uses to build the root cluster of a tree.
//
// bldtt_setup obtains the scratch for its per-block partial boxes from the
// stream-ordered allocator.  Some callers cannot allocate device memory at
// all: code that runs while a framework owns the whole device memory pool,
// real-time loops where allocation is forbidden, or a host that may only
// launch work into memory it was handed.  For them,
// bldtt_bounding_box_noalloc keeps its scratch in the fixed array below.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds its 56 KB until the process exits.  In host code its name is
// only a host-side stand-in, so the entry point looks up the real device
// address with cudaGetSymbolAddress once per device (on the first call made
// with that device current) and passes that address to the kernels.  That
// first call should therefore come before any stream capture.  All calls
// share the array; each call overwrites every slot it later reads, so no
// state carries over between calls, but calls that overlap on the GPU (for
// example on two streams) race on it and must be serialised by the caller.
#include <mutex>

#include "internal.cuh"

namespace bldtt {

constexpr int kBoxBlocks = 1024;          // partial boxes (one per CTA, grid-stride)
constexpr int kBoxThreads = 256;
constexpr int kBoxSlot = 7;               // lo x,y,z, hi x,y,z, non-finite flag

// 1024 x 7 doubles = 56 KB of scratch per device.
static __device__ __align__(256) double g_box_scratch[kBoxBlocks * kBoxSlot];

__device__ __forceinline__ bool is_finite_bits(double v) {
  return (__double_as_longlong(v) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}

__global__ void __launch_bounds__(kBoxThreads) k_box_partial_noalloc(const double* __restrict__ pts,
                                                                     int64_t n,
                                                                     double* __restrict__ scratch) {
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  bool ok = true;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      double v = pts[(int64_t)d * n + i];
      ok = ok && is_finite_bits(v);
      lo[d] = fmin(lo[d], v);
      hi[d] = fmax(hi[d], v);
    }
  }
  __shared__ double sm[kBoxThreads / 32][kBoxSlot];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 0; d < 3; ++d)
    for (int off = 16; off; off >>= 1) {
      lo[d] = fmin(lo[d], __shfl_down_sync(0xffffffffu, lo[d], off));
      hi[d] = fmax(hi[d], __shfl_down_sync(0xffffffffu, hi[d], off));
    }
  bool all_ok = __all_sync(0xffffffffu, ok);
  if (lane == 0) {
    for (int d = 0; d < 3; ++d) {
      sm[warp][d] = lo[d];
      sm[warp][3 + d] = hi[d];
    }
    sm[warp][6] = all_ok ? 0.0 : 1.0;
  }
  __syncthreads();
  if (threadIdx.x < kBoxSlot) {
    const int k = threadIdx.x;
    double r = sm[0][k];
    for (int w = 1; w < kBoxThreads / 32; ++w)
      r = k < 3 ? fmin(r, sm[w][k]) : fmax(r, sm[w][k]);
    scratch[(int64_t)blockIdx.x * kBoxSlot + k] = r;   // every slot read later is rewritten
  }
}

__global__ void __launch_bounds__(kBoxThreads) k_box_final_noalloc(const double* __restrict__ scratch,
                                                                   int nparts, double* __restrict__ box,
                                                                   int* __restrict__ nonfinite) {
  __shared__ double sm[kBoxThreads / 32][kBoxSlot];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double v[kBoxSlot] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY, 0.0};
  for (int b = threadIdx.x; b < nparts; b += blockDim.x)
    for (int k = 0; k < kBoxSlot; ++k) {
      double p = scratch[(int64_t)b * kBoxSlot + k];
      v[k] = k < 3 ? fmin(v[k], p) : fmax(v[k], p);
    }
  for (int k = 0; k < kBoxSlot; ++k)
    for (int off = 16; off; off >>= 1) {
      double o = __shfl_down_sync(0xffffffffu, v[k], off);
      v[k] = k < 3 ? fmin(v[k], o) : fmax(v[k], o);
    }
  if (lane == 0)
    for (int k = 0; k < kBoxSlot; ++k) sm[warp][k] = v[k];
  __syncthreads();
  if (threadIdx.x < kBoxSlot) {
    const int k = threadIdx.x;
    double r = sm[0][k];
    for (int w = 1; w < kBoxThreads / 32; ++w) r = k < 3 ? fmin(r, sm[w][k]) : fmax(r, sm[w][k]);
    if (k < 6) box[k] = r;
    else if (nonfinite) *nonfinite = r != 0.0 ? 1 : 0;
  }
}

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_box_mutex;
double* g_box_ptr[kMaxDevices] = {};

// Device address of g_box_scratch for the current device, looked up once.
int box_scratch_for_current_device(double** out) {
  int dev = 0;
  BL_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal %d beyond the %d devices this entry point tracks", dev, kMaxDevices);
    return BLDTT_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_box_mutex);
  if (!g_box_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_box_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      set_error("cudaGetSymbolAddress of the bounding-box scratch failed on device %d: %s", dev,
                cudaGetErrorString(e));
      return BLDTT_ECUDA;
    }
    g_box_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_box_ptr[dev];
  return BLDTT_OK;
}
}  // namespace

}  // namespace bldtt

extern "C" int bldtt_bounding_box_noalloc(const double* points, int64_t n, double* box,
                                          int* nonfinite, void* cuda_stream) {
  using namespace bldtt;
  if (!points || !box) {
    set_error("bounding_box_noalloc: points and box must be non-NULL device pointers");
    return BLDTT_EINVAL;
  }
  if (n < 1 || n >= (int64_t)INT32_MAX) {
    set_error("bounding_box_noalloc: n=%lld outside [1, 2^31-1), the particle counts this "
              "library accepts", (long long)n);
    return BLDTT_EINVAL;
  }
  double* scratch = nullptr;
  BL_TRY(box_scratch_for_current_device(&scratch));
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int64_t want = (n + kBoxThreads - 1) / kBoxThreads;
  int blocks = (int)(want < kBoxBlocks ? want : kBoxBlocks);
  int64_t launches = 0;
  k_box_partial_noalloc<<<blocks, kBoxThreads, 0, s>>>(points, n, scratch);
  BL_LAUNCHED(launches);
  k_box_final_noalloc<<<1, kBoxThreads, 0, s>>>(scratch, blocks, box, nonfinite);
  BL_LAUNCHED(launches);
  return BLDTT_OK;
}
