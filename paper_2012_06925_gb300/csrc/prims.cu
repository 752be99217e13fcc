// Device-wide primitives used by tree building, the traversal and work-list
// construction: exclusive scan, stable LSD radix sort of (key, value) pairs
// and a finiteness check.  Deterministic: no result
// depends on the order in which atomics land.
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "internal.cuh"

namespace bldtt {

namespace {
thread_local char g_err[512] = "";
}

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

const char* last_error() { return g_err; }

namespace {
thread_local cudaMemPool_t t_pool = nullptr;
thread_local void* t_pinned = nullptr;
}
void set_thread_context(cudaMemPool_t pool, void* pinned) {
  t_pool = pool;
  t_pinned = pinned;
}
cudaMemPool_t thread_pool() { return t_pool; }
void* thread_pinned() { return t_pinned; }

std::mutex& cooperative_launch_mutex() {
  static std::mutex mu;
  return mu;
}

bool cooperative_set_up_disabled() {
  const char* e = std::getenv("BLDTT_LEVEL_BY_LEVEL");
  return e && e[0] == '1' && e[1] == '\0';
}

int read_device(const void* dev, void* host, size_t bytes, cudaStream_t s) {
  if (t_pinned && bytes <= kPinnedSlot) {
    BL_CUDA(cudaMemcpyAsync(t_pinned, dev, bytes, cudaMemcpyDeviceToHost, s));
    BL_CUDA(cudaStreamSynchronize(s));
    std::memcpy(host, t_pinned, bytes);
  } else {
    BL_CUDA(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, s));
    BL_CUDA(cudaStreamSynchronize(s));
  }
  return BLDTT_OK;
}

int dalloc(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  cudaError_t e = t_pool ? cudaMallocFromPoolAsync(p, bytes, t_pool, s) : cudaMallocAsync(p, bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? BLDTT_ENOMEM : BLDTT_ECUDA;
  }
  return BLDTT_OK;
}

void dfree(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

template <class T>
int dgrow(T** p, size_t* cap, size_t need, size_t keep, cudaStream_t s) {
  if (need <= *cap && *p) return BLDTT_OK;
  size_t ncap = *cap ? *cap : 64;
  while (ncap < need) ncap *= 2;
  T* q = nullptr;
  BL_TRY(dalloc_n(&q, ncap, s));
  if (*p && keep) BL_CUDA(cudaMemcpyAsync(q, *p, keep * sizeof(T), cudaMemcpyDeviceToDevice, s));
  dfree(*p, s);
  *p = q;
  *cap = ncap;
  return BLDTT_OK;
}
template int dgrow<int32_t>(int32_t**, size_t*, size_t, size_t, cudaStream_t);
template int dgrow<double>(double**, size_t*, size_t, size_t, cudaStream_t);
template int dgrow<int2>(int2**, size_t*, size_t, size_t, cudaStream_t);
template int dgrow<uint8_t>(uint8_t**, size_t*, size_t, size_t, cudaStream_t);
template int dgrow<int8_t>(int8_t**, size_t*, size_t, size_t, cudaStream_t);
template int dgrow<int16_t>(int16_t**, size_t*, size_t, size_t, cudaStream_t);
template int dgrow<int4>(int4**, size_t*, size_t, size_t, cudaStream_t);
template int dgrow<long long>(long long**, size_t*, size_t, size_t, cudaStream_t);
template int dgrow<unsigned long long>(unsigned long long**, size_t*, size_t, size_t, cudaStream_t);

// ---------------------------------------------------------------------------
// Exclusive scan (reduce, scan the tile sums, apply)
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int32_t block_exclusive_sum(int32_t v, int32_t* warp_tot,
                                                       int32_t* block_total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t x = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    int32_t y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int32_t w = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += y;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = w;
  }
  __syncthreads();
  int32_t prefix = warp ? warp_tot[warp - 1] : 0;
  *block_total = warp_tot[kScanThreads / 32 - 1];
  __syncthreads();
  return prefix + x - v;
}

__global__ void k_scan_reduce(const int32_t* __restrict__ in, int64_t n,
                              int32_t* __restrict__ tile_sums) {
  __shared__ int32_t warp_tot[kScanThreads / 32];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  int32_t s = 0;
  for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
    int64_t g = base + i;
    if (g < n) s += in[g];
  }
  int32_t total;
  block_exclusive_sum(s, warp_tot, &total);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void k_scan_apply(const int32_t* __restrict__ in, int32_t* __restrict__ out, int64_t n,
                             const int32_t* __restrict__ tile_off, int32_t* __restrict__ total_out) {
  __shared__ int32_t tile[kScanTile];
  __shared__ int32_t warp_tot[kScanThreads / 32];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
    int64_t g = base + i;
    tile[i] = g < n ? in[g] : 0;
  }
  __syncthreads();
  int32_t loc[kScanItems];
  int32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    loc[k] = s;
    s += tile[threadIdx.x * kScanItems + k];
  }
  int32_t total;
  int32_t pre = block_exclusive_sum(s, warp_tot, &total);
  int32_t off = tile_off ? tile_off[blockIdx.x] : 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) tile[threadIdx.x * kScanItems + k] = off + pre + loc[k];
  __syncthreads();
  for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
    int64_t g = base + i;
    if (g < n) out[g] = tile[i];
  }
  if (total_out && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total_out = off + total;
}

static int scan_impl(const int32_t* in, int32_t* out, int64_t n, int32_t* total_dev,
                     cudaStream_t s, Counters& c) {
  int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles <= 1) {
    k_scan_apply<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr, total_dev);
    BL_LAUNCHED(c.launches);
    return BLDTT_OK;
  }
  int32_t *sums = nullptr, *offs = nullptr;
  Arena scratch;
  scratch.add(&sums, tiles);
  scratch.add(&offs, tiles);
  BL_TRY(scratch.alloc(s));
  k_scan_reduce<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sums);
  BL_LAUNCHED(c.launches);
  BL_TRY(scan_impl(sums, offs, tiles, nullptr, s, c));
  k_scan_apply<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, n, offs, total_dev);
  BL_LAUNCHED(c.launches);
  scratch.release(s);
  return BLDTT_OK;
}

int scan_exclusive(const int32_t* in, int32_t* out, int64_t n, int32_t* total_host,
                   cudaStream_t s, Counters& c) {
  if (n <= 0) {
    if (total_host) *total_host = 0;
    return BLDTT_OK;
  }
  int32_t* tot = nullptr;
  if (total_host) BL_TRY(dalloc_n(&tot, 1, s));
  BL_TRY(scan_impl(in, out, n, tot, s, c));
  if (total_host) {
    const int rc = read_device(tot, total_host, sizeof(int32_t), s);
    dfree(tot, s);
    return rc;
  }
  return BLDTT_OK;
}

int scan_exclusive_dev(const int32_t* in, int32_t* out, int64_t n, int32_t* total_dev,
                       cudaStream_t s, Counters& c) {
  if (n <= 0) {
    BL_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(int32_t), s));
    return BLDTT_OK;
  }
  return scan_impl(in, out, n, total_dev, s, c);
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort, 8-bit digits (a set-up sorts keys of 13 to 28 bits:
// two to four passes of four launches each)
// ---------------------------------------------------------------------------
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
static_assert(kRadix <= kScanThreads, "one thread per digit in the histogram and scatter kernels");

__global__ void k_radix_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                             int32_t* __restrict__ hist, int64_t tiles) {
  __shared__ int32_t cnt[kRadix];
  if (threadIdx.x < kRadix) cnt[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
    int64_t g = base + i;
    if (g < n) atomicAdd(&cnt[(keys[g] >> shift) & (kRadix - 1)], 1);
  }
  __syncthreads();
  if (threadIdx.x < kRadix) hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void k_radix_scatter(const uint32_t* __restrict__ kin, const int32_t* __restrict__ vin,
                                uint32_t* __restrict__ kout, int32_t* __restrict__ vout, int64_t n,
                                int shift, const int32_t* __restrict__ offs, int64_t tiles) {
  constexpr int W = kScanThreads / 32;
  __shared__ int32_t warp_cnt[W][kRadix + 1];
  __shared__ int32_t running[kRadix];
  __shared__ int32_t tile_off[kRadix];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < kRadix) {
    running[threadIdx.x] = 0;
    tile_off[threadIdx.x] = offs[(int64_t)threadIdx.x * tiles + blockIdx.x];
  }
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  for (int r = 0; r < kScanItems; ++r) {
    for (int i = threadIdx.x; i < W * (kRadix + 1); i += kScanThreads) (&warp_cnt[0][0])[i] = 0;
    __syncthreads();
    int64_t g = base + (int64_t)r * kScanThreads + threadIdx.x;
    bool valid = g < n;
    uint32_t key = valid ? kin[g] : 0u;
    int d = valid ? (int)((key >> shift) & (kRadix - 1)) : kRadix;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    int rank = __popc(peers & ((1u << lane) - 1u));
    if (rank == 0) warp_cnt[warp][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      int32_t pos = tile_off[d] + running[d] + rank;
      for (int w = 0; w < warp; ++w) pos += warp_cnt[w][d];
      kout[pos] = key;
      vout[pos] = vin[g];
    }
    __syncthreads();
    if (threadIdx.x < kRadix) {
      int32_t t = 0;
      for (int w = 0; w < W; ++w) t += warp_cnt[w][threadIdx.x];
      running[threadIdx.x] += t;
    }
    __syncthreads();
  }
}

int radix_sort_pairs(uint32_t* keys, int32_t* vals, int64_t n, int bits, cudaStream_t s,
                     Counters& c) {
  if (n <= 1) return BLDTT_OK;
  int passes = (bits + kRadixBits - 1) / kRadixBits;
  if (passes == 0) return BLDTT_OK;
  int64_t tiles = (n + kScanTile - 1) / kScanTile;
  uint32_t* k2 = nullptr;
  int32_t *v2 = nullptr, *hist = nullptr, *offs = nullptr;
  Arena scratch;
  scratch.add(&k2, n);
  scratch.add(&v2, n);
  scratch.add(&hist, tiles * kRadix);
  scratch.add(&offs, tiles * kRadix);
  BL_TRY(scratch.alloc(s));
  uint32_t *ka = keys, *kb = k2;
  int32_t *va = vals, *vb = v2;
  for (int p = 0; p < passes; ++p) {
    int shift = p * kRadixBits;
    k_radix_hist<<<(unsigned)tiles, kScanThreads, 0, s>>>(ka, n, shift, hist, tiles);
    BL_LAUNCHED(c.launches);
    BL_TRY(scan_impl(hist, offs, tiles * kRadix, nullptr, s, c));
    k_radix_scatter<<<(unsigned)tiles, kScanThreads, 0, s>>>(ka, va, kb, vb, n, shift, offs, tiles);
    BL_LAUNCHED(c.launches);
    uint32_t* tk = ka; ka = kb; kb = tk;
    int32_t* tv = va; va = vb; vb = tv;
  }
  if (ka != keys) {
    BL_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    BL_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  }
  scratch.release(s);
  return BLDTT_OK;
}

// ---------------------------------------------------------------------------
// Bounding box and finiteness
// ---------------------------------------------------------------------------
constexpr int kRedThreads = 256;

__device__ __forceinline__ bool finite_d(double v) {
  return (__double_as_longlong(v) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}

__global__ void k_check_finite(const double* __restrict__ v, int64_t n, int* __restrict__ bad) {
  bool ok = true;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    ok = ok && finite_d(v[i]);
  if (!__all_sync(0xffffffffu, ok) && (threadIdx.x & 31) == 0) atomicExch(bad, 1);
}

int check_finite(const double* v, int64_t n, int* bad_dev, cudaStream_t s, Counters& c) {
  int blocks = (int)((n + kRedThreads - 1) / kRedThreads);
  if (blocks > 1024) blocks = 1024;
  if (blocks < 1) blocks = 1;
  k_check_finite<<<blocks, kRedThreads, 0, s>>>(v, n, bad_dev);
  BL_LAUNCHED(c.launches);
  return BLDTT_OK;
}

}  // namespace bldtt
