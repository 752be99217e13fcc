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
// address with cudaGetSymbolAddress (on the first call made with a device
// current, and again on later calls outside stream capture) and passes that
// address to the kernels.  The first call on a device should therefore come
// before any stream capture.  All calls
// share the array; each call overwrites every slot it later reads, so no
// state carries over between calls, but calls that overlap on the GPU (for
// example on two streams) race on it and must be serialised by the caller.
#include <mutex>

#include "internal.cuh"

namespace bldtt {

constexpr int kBoxBlocks = 1024;          // partial boxes (one per CTA, grid-stride)
constexpr int kBoxThreads = 256;
constexpr int kBoxSlot = 7;               // lo x,y,z, hi x,y,z (order keys), non-finite flag

// 1024 x 7 64-bit words = 56 KB of scratch per device.
static __device__ __align__(256) long long g_box_scratch[kBoxBlocks * kBoxSlot];

__device__ __forceinline__ bool is_finite_bits(double v) {
  return (__double_as_longlong(v) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}

// Minima and maxima run on okey, the order-preserving integer image of a
// double that bldtt_setup's box kernels use, so the result equals the root
// box of a tree bit for bit (-0.0 and +0.0 compare equal and come back as
// +0.0).  Non-finite coordinates are left out of the box and raise the flag.
__global__ void __launch_bounds__(kBoxThreads) k_box_partial_noalloc(const double* __restrict__ pts,
                                                                     int64_t n,
                                                                     long long* __restrict__ scratch) {
  long long lo[3] = {kKeyPosInf, kKeyPosInf, kKeyPosInf}, hi[3] = {kKeyNegInf, kKeyNegInf, kKeyNegInf};
  bool ok = true;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double v = pts[(int64_t)d * n + i];
      if (is_finite_bits(v)) {
        const long long k = okey(v);
        lo[d] = min(lo[d], k);
        hi[d] = max(hi[d], k);
      } else {
        ok = false;
      }
    }
  }
  __shared__ long long sm[kBoxThreads / 32][kBoxSlot];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 0; d < 3; ++d)
    for (int off = 16; off; off >>= 1) {
      lo[d] = min(lo[d], __shfl_down_sync(0xffffffffu, lo[d], off));
      hi[d] = max(hi[d], __shfl_down_sync(0xffffffffu, hi[d], off));
    }
  const bool all_ok = __all_sync(0xffffffffu, ok);
  if (lane == 0) {
    for (int d = 0; d < 3; ++d) {
      sm[warp][d] = lo[d];
      sm[warp][3 + d] = hi[d];
    }
    sm[warp][6] = all_ok ? 0 : 1;
  }
  __syncthreads();
  if (threadIdx.x < kBoxSlot) {
    const int k = threadIdx.x;
    long long r = sm[0][k];
    for (int w = 1; w < kBoxThreads / 32; ++w) r = k < 3 ? min(r, sm[w][k]) : max(r, sm[w][k]);
    scratch[(int64_t)blockIdx.x * kBoxSlot + k] = r;   // every slot read later is rewritten
  }
}

__global__ void __launch_bounds__(kBoxThreads) k_box_final_noalloc(const long long* __restrict__ scratch,
                                                                   int nparts, double* __restrict__ box,
                                                                   int* __restrict__ nonfinite) {
  __shared__ long long sm[kBoxThreads / 32][kBoxSlot];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long v[kBoxSlot] = {kKeyPosInf, kKeyPosInf, kKeyPosInf, kKeyNegInf, kKeyNegInf, kKeyNegInf, 0};
  for (int b = threadIdx.x; b < nparts; b += blockDim.x)
    for (int k = 0; k < kBoxSlot; ++k) {
      const long long p = scratch[(int64_t)b * kBoxSlot + k];
      v[k] = k < 3 ? min(v[k], p) : max(v[k], p);
    }
  for (int k = 0; k < kBoxSlot; ++k)
    for (int off = 16; off; off >>= 1) {
      const long long o = __shfl_down_sync(0xffffffffu, v[k], off);
      v[k] = k < 3 ? min(v[k], o) : max(v[k], o);
    }
  if (lane == 0)
    for (int k = 0; k < kBoxSlot; ++k) sm[warp][k] = v[k];
  __syncthreads();
  if (threadIdx.x < kBoxSlot) {
    const int k = threadIdx.x;
    long long r = sm[0][k];
    for (int w = 1; w < kBoxThreads / 32; ++w) r = k < 3 ? min(r, sm[w][k]) : max(r, sm[w][k]);
    if (k < 6) box[k] = okey_inv(r);   // no finite coordinate in a dimension: +inf / -inf
    else if (nonfinite) *nonfinite = r != 0 ? 1 : 0;
  }
}

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_box_mutex;
long long* g_box_ptr[kMaxDevices] = {};

// Device address of g_box_scratch for the current device, looked up once.
int box_scratch_for_current_device(cudaStream_t s, long long** out) {
  int dev = 0;
  BL_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal %d beyond the %d devices this entry point tracks", dev, kMaxDevices);
    return BLDTT_EINVAL;
  }
  // The address is looked up on the first call with the device current, and
  // again on any later call whose stream is not capturing, so that a context
  // re-created after cudaDeviceReset (the module reloaded, the array maybe
  // elsewhere) is never given a stale address.  Under capture the cached
  // address is used, which requires a call before the capture started.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    cudaGetLastError();
    cap = cudaStreamCaptureStatusActive;   // unknown: do not call into the runtime's lookup
  }
  std::lock_guard<std::mutex> lock(g_box_mutex);
  if (!g_box_ptr[dev] || cap == cudaStreamCaptureStatusNone) {
    if (!g_box_ptr[dev] && cap != cudaStreamCaptureStatusNone) {
      set_error("bounding_box_noalloc: first call on device %d made during stream capture; "
                "call it once before capturing", dev);
      return BLDTT_EINVAL;
    }
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_box_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      set_error("cudaGetSymbolAddress of the bounding-box scratch failed on device %d: %s", dev,
                cudaGetErrorString(e));
      return BLDTT_ECUDA;
    }
    g_box_ptr[dev] = static_cast<long long*>(p);
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
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  long long* scratch = nullptr;
  BL_TRY(box_scratch_for_current_device(s, &scratch));
  int64_t want = (n + kBoxThreads - 1) / kBoxThreads;
  int blocks = (int)(want < kBoxBlocks ? want : kBoxBlocks);
  int64_t launches = 0;
  k_box_partial_noalloc<<<blocks, kBoxThreads, 0, s>>>(points, n, scratch);
  BL_LAUNCHED(launches);
  k_box_final_noalloc<<<1, kBoxThreads, 0, s>>>(scratch, blocks, box, nonfinite);
  BL_LAUNCHED(launches);
  return BLDTT_OK;
}
