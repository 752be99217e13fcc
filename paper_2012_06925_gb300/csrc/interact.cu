// PP, PC, CP and CC interactions (Sec. 2.4, Eqs. (6), (8), (12), (15)) in one
// persistent kernel.
//
// All four interaction types are "targets x sources" sums (Sec. 3.3): the
// targets are particles (PP, PC) or proxy points (CP, CC) of a target cluster,
// the sources are particles (PP, CP) or proxy points with proxy charges
// (PC, CC) of a source cluster.  A work item is a tile of up to kTile targets
// of one target cluster; its sources are the concatenation of
//   particle tiles: PP and PC entries of the leaf and of every ancestor
//                   (an entry on an ancestor applies to all its particles)
//   proxy tiles:    CP and CC entries of the cluster itself.
// Each item owns its outputs, so there are no atomics and the summation order
// is fixed.
//
// Per CTA, one producer warp grabs items from a global counter, walks their
// lists and streams the sources, kChunk at a time, from the source pool into
// a kStages-deep shared-memory ring with cp.async.bulk (TMA) copies that
// complete on mbarriers; four consumer warps evaluate G for kTargetsPerThread
// targets per thread against every staged source.
//
// FP32_BULK: pool entries are float4 (y - c, q) in the frame of the source
// segment's centre c (a leaf centre or a cluster centre), rounded once from
// the FP64 difference.  Targets keep FP64 coordinates and are moved into each
// segment's frame with the same expression, (float)(x - c), so the coordinate
// rounding error is relative to the cluster size, not to |x|, and a target
// that coincides with a source gets exactly the same FP32 coordinates (r = 0).
// Each chunk is summed in FP32 and added to an FP64 accumulator.
// FP64: pool entries are double4 (y, q) in absolute coordinates.
//
// A pair at distance 0 contributes nothing.  The fast path evaluates
// 1/sqrt(r^2) unguarded; a chunk whose FP32/FP64 partial is not finite (only
// possible when some r^2 == 0) is recomputed by the warp with the guard.
#include <type_traits>

#include "internal.cuh"

namespace bldtt {

constexpr int kThreads = (kConsumerWarps + 1) * 32;
constexpr int kConsumers = kConsumerWarps * 32;
constexpr uint64_t kWaitNs = 20ull * 1000ull * 1000ull * 1000ull;   // 20 s bound on any wait
constexpr int kFlagNewSegment = 1;

struct InteractView {
  const int4* items;
  int32_t nitems;
  int32_t* counter;
  // lists and source layout (producer)
  const int32_t* list_ptr;
  const int32_t* list_src;
  int32_t nct;
  const int32_t* t_parent;
  const int32_t* s_leaf_first;
  const int32_t* s_leaf_last;
  const int32_t* s_leaf_ids;
  const int32_t* pad_prefix;
  const double* s_center;
  int32_t np_pad;
  int64_t proxy_base;
  const void* pool;
  // targets and outputs (consumers)
  const double* tx;
  const double* ty;
  const double* tz;
  const double* t_nodes;
  int32_t P, np;
  double* phi_near;
  double* phit;
  int* err;
  double kappa;
  float neg_kappa_log2e;
};

struct StageMeta {
  int item;
  int flags;
  double c[3];   // segment centre (frame origin of the staged FP32 sources)
};

// ---- PTX helpers: mbarrier, bulk copy, timer -------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait: gives up after kWaitNs, raising the plan's error flag.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int* err) {
  if (mbar_try_wait(b, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(b, parity)) {
    if (global_ns() - t0 > kWaitNs) {
      atomicExch(err, kDevErrTimeout);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float exp2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ bool not_finite(float v) {
  return (__float_as_uint(v) & 0x7f800000u) == 0x7f800000u;
}
__device__ __forceinline__ bool not_finite(double v) {
  return (__double_as_longlong(v) & 0x7ff0000000000000LL) == 0x7ff0000000000000LL;
}

// ---- kernel functions (Sec. 4.6); d = x - y -------------------------------
template <int KERN, typename T>
__device__ __forceinline__ T poly_kernel(T dx, T dy, T dz) {
  return (T)1 + dx - (T)2 * dy + (T)3 * dz + dx * dy - dy * dz + dx * dx * dz * dz -
         (T)0.5 * dy * dy;
}

// Unguarded FP32 evaluation of q * G.
template <int KERN>
__device__ __forceinline__ float pair_f32(float dx, float dy, float dz, float q, float nk) {
  float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
  if (KERN == BLDTT_COULOMB) {
    return q * rsqrt_approx(r2);
  } else if (KERN == BLDTT_YUKAWA) {
    float ri = rsqrt_approx(r2);
    return (q * ri) * exp2_approx(r2 * ri * nk);
  } else {
    return r2 > 0.f ? q * poly_kernel<KERN, float>(dx, dy, dz) : 0.f;
  }
}
// Guarded FP32 evaluation (r^2 == 0 contributes 0).
template <int KERN>
__device__ __forceinline__ float pair_f32_guarded(float dx, float dy, float dz, float q, float nk) {
  float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
  if (!(r2 > 0.f)) return 0.f;
  return pair_f32<KERN>(dx, dy, dz, q, nk);
}
template <int KERN>
__device__ __forceinline__ double pair_f64(double dx, double dy, double dz, double q, double kappa) {
  double r2 = dx * dx + dy * dy + dz * dz;
  if (KERN == BLDTT_COULOMB) {
    return q * rsqrt(r2);
  } else if (KERN == BLDTT_YUKAWA) {
    double ri = rsqrt(r2);
    return q * ri * exp(-kappa * (r2 * ri));
  } else {
    return r2 > 0.0 ? q * poly_kernel<KERN, double>(dx, dy, dz) : 0.0;
  }
}
template <int KERN>
__device__ __forceinline__ double pair_f64_guarded(double dx, double dy, double dz, double q,
                                                   double kappa) {
  double r2 = dx * dx + dy * dy + dz * dz;
  if (!(r2 > 0.0)) return 0.0;
  return pair_f64<KERN>(dx, dy, dz, q, kappa);
}

// ---- producer: walks an item's segments ------------------------------------
template <typename Vec>
struct Producer {
  const InteractView& v;
  Vec (*buf)[kChunk];
  StageMeta* meta;
  uint64_t* full;
  uint64_t* empty;
  uint32_t it = 0;
  int cur_item = -1;

  __device__ Producer(const InteractView& v_, Vec (*b)[kChunk], StageMeta* m, uint64_t* f,
                      uint64_t* e)
      : v(v_), buf(b), meta(m), full(f), empty(e) {}

  __device__ bool acquire(int& s) {
    s = (int)(it % kStages);
    return mbar_wait(&empty[s], ((it / kStages) & 1u) ^ 1u, v.err);
  }

  // Stream one segment (pool offset, entries, centre) in kChunk pieces.
  __device__ bool segment(int64_t off, int64_t len, const double* c) {
    const double c0 = c[0], c1 = c[1], c2 = c[2];
    const Vec* src = reinterpret_cast<const Vec*>(v.pool) + off;
    for (int64_t k = 0; k < len; k += kChunk) {
      int s;
      if (!acquire(s)) return false;
      StageMeta& m = meta[s];
      m.item = cur_item;
      m.flags = k == 0 ? kFlagNewSegment : 0;
      m.c[0] = c0;
      m.c[1] = c1;
      m.c[2] = c2;
      mbar_arrive_tx(&full[s], (uint32_t)(kChunk * sizeof(Vec)));
      bulk_copy_g2s(buf[s], src + k, (uint32_t)(kChunk * sizeof(Vec)), &full[s]);
      ++it;
    }
    return true;
  }

  // Particles of every source leaf under cluster s (one segment per leaf).
  __device__ bool leaves_of(int32_t s) {
    for (int32_t lf = v.s_leaf_first[s]; lf < v.s_leaf_last[s]; ++lf) {
      int64_t o = v.pad_prefix[lf];
      int64_t len = v.pad_prefix[lf + 1] - o;
      if (!segment(o, len, v.s_center + (int64_t)v.s_leaf_ids[lf] * 3)) return false;
    }
    return true;
  }

  __device__ bool lists(int type_particles, int type_proxies, int32_t c) {
    int64_t k0 = (int64_t)type_particles * v.nct + c;
    for (int32_t e = v.list_ptr[k0]; e < v.list_ptr[k0 + 1]; ++e)
      if (!leaves_of(v.list_src[e])) return false;
    int64_t k1 = (int64_t)type_proxies * v.nct + c;
    for (int32_t e = v.list_ptr[k1]; e < v.list_ptr[k1 + 1]; ++e) {
      int32_t s = v.list_src[e];
      if (!segment(v.proxy_base + (int64_t)s * v.np_pad, v.np_pad, v.s_center + (int64_t)s * 3))
        return false;
    }
    return true;
  }

  __device__ void run() {
    bool ok = true;
    for (;;) {
      int idx = atomicAdd(v.counter, 1);
      if (idx >= v.nitems) break;
      int4 item = v.items[idx];
      cur_item = idx;
      if (item.w == kItemParticles) {
        for (int32_t a = item.x; a >= 0 && ok; a = v.t_parent[a]) ok = lists(BLDTT_PP, BLDTT_PC, a);
      } else {
        ok = lists(BLDTT_CP, BLDTT_CC, item.x);
      }
      if (!ok) break;
    }
    if (ok) {
      int s;
      if (acquire(s)) {
        meta[s].item = -1;
        meta[s].flags = 0;
        mbar_arrive(&full[s]);
        ++it;
        return;
      }
    }
    // Error path: let the copies already issued land before the CTA exits.
    uint32_t first = it > (uint32_t)kStages ? it - kStages : 0;
    for (uint32_t j = first; j < it; ++j) mbar_wait(&full[j % kStages], (j / kStages) & 1u, v.err);
  }
};

// ---- consumers --------------------------------------------------------------
template <int KERN>
__device__ __forceinline__ void chunk_f32(const float4* __restrict__ sb, const float (&xr)[kTargetsPerThread][3],
                                          float (&a)[kTargetsPerThread], float nk) {
#pragma unroll
  for (int k = 0; k < kTargetsPerThread; ++k) a[k] = 0.f;
#pragma unroll 8
  for (int j = 0; j < kChunk; ++j) {
    const float4 p = sb[j];
#pragma unroll
    for (int k = 0; k < kTargetsPerThread; ++k) {
      float dx = xr[k][0] - p.x, dy = xr[k][1] - p.y, dz = xr[k][2] - p.z;
      if (KERN == BLDTT_COULOMB) {
        float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        a[k] = fmaf(p.w, rsqrt_approx(r2), a[k]);
      } else {
        a[k] += pair_f32<KERN>(dx, dy, dz, p.w, nk);
      }
    }
  }
}

template <int KERN>
__device__ __noinline__ void chunk_f32_guarded(const float4* __restrict__ sb,
                                               const float (&xr)[kTargetsPerThread][3],
                                               float (&a)[kTargetsPerThread], float nk) {
  for (int k = 0; k < kTargetsPerThread; ++k) a[k] = 0.f;
  for (int j = 0; j < kChunk; ++j) {
    const float4 p = sb[j];
    for (int k = 0; k < kTargetsPerThread; ++k)
      a[k] += pair_f32_guarded<KERN>(xr[k][0] - p.x, xr[k][1] - p.y, xr[k][2] - p.z, p.w, nk);
  }
}

template <int KERN>
__device__ __forceinline__ void chunk_f64(const double4* __restrict__ sb,
                                          const double (&x)[kTargetsPerThread][3],
                                          double (&a)[kTargetsPerThread], double kappa) {
#pragma unroll
  for (int k = 0; k < kTargetsPerThread; ++k) a[k] = 0.0;
#pragma unroll 4
  for (int j = 0; j < kChunk; ++j) {
    const double4 p = sb[j];
#pragma unroll
    for (int k = 0; k < kTargetsPerThread; ++k)
      a[k] += pair_f64<KERN>(x[k][0] - p.x, x[k][1] - p.y, x[k][2] - p.z, p.w, kappa);
  }
}

template <int KERN>
__device__ __noinline__ void chunk_f64_guarded(const double4* __restrict__ sb,
                                               const double (&x)[kTargetsPerThread][3],
                                               double (&a)[kTargetsPerThread], double kappa) {
  for (int k = 0; k < kTargetsPerThread; ++k) a[k] = 0.0;
  for (int j = 0; j < kChunk; ++j) {
    const double4 p = sb[j];
    for (int k = 0; k < kTargetsPerThread; ++k)
      a[k] += pair_f64_guarded<KERN>(x[k][0] - p.x, x[k][1] - p.y, x[k][2] - p.z, p.w, kappa);
  }
}

// Absolute coordinates of target row r of an item (a particle or a proxy point).
__device__ __forceinline__ void target_coords(const InteractView& v, const int4& item, int r,
                                              double& X, double& Y, double& Z) {
  if (r >= item.z) {       // idle slot of a partial tile: far away, contributes nothing
    X = Y = Z = 1.0e15;
    return;
  }
  if (item.w == kItemParticles) {
    int64_t i = (int64_t)item.y + r;
    X = v.tx[i];
    Y = v.ty[i];
    Z = v.tz[i];
  } else {
    const int P = v.P;
    int l = item.y + r;
    int l1 = l / (P * P), l2 = (l / P) % P, l3 = l % P;
    const double* nd = v.t_nodes + (int64_t)item.x * 3 * P;
    X = nd[l1];
    Y = nd[P + l2];
    Z = nd[2 * P + l3];
  }
}

__device__ __forceinline__ void store_outputs(const InteractView& v, const int4& item, int ct,
                                              const double (&acc)[kTargetsPerThread]) {
#pragma unroll
  for (int k = 0; k < kTargetsPerThread; ++k) {
    int r = k * kConsumers + ct;
    if (r < item.z) {
      if (item.w == kItemParticles)
        v.phi_near[(int64_t)item.y + r] = acc[k];
      else
        v.phit[(int64_t)item.x * v.np + item.y + r] = acc[k];
    }
  }
}

template <bool F32, int KERN>
__global__ void __launch_bounds__(kThreads) k_interact(InteractView v) {
  using Vec = typename std::conditional<F32, float4, double4>::type;
  __shared__ __align__(128) Vec sbuf[kStages][kChunk];
  __shared__ StageMeta smeta[kStages];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ __align__(8) uint64_t empty[kStages];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumerWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == kConsumerWarps) {
    if (lane == 0) {
      Producer<Vec> prod(v, sbuf, smeta, full, empty);
      prod.run();
    }
    return;
  }

  const int ct = threadIdx.x;   // consumer thread 0..kConsumers-1
  int cur = -1;
  int4 item = make_int4(0, 0, 0, 0);
  double acc[kTargetsPerThread];
  double X[kTargetsPerThread][3];
  float xr[kTargetsPerThread][3];
  for (uint32_t it = 0;; ++it) {
    const int s = (int)(it % kStages);
    if (!mbar_wait(&full[s], (it / kStages) & 1u, v.err)) return;
    const int mi = smeta[s].item;
    if (mi != cur) {
      if (cur >= 0) store_outputs(v, item, ct, acc);
      if (mi < 0) return;
      cur = mi;
      item = v.items[mi];
#pragma unroll
      for (int k = 0; k < kTargetsPerThread; ++k) {
        acc[k] = 0.0;
        target_coords(v, item, k * kConsumers + ct, X[k][0], X[k][1], X[k][2]);
      }
    }
    if (F32) {
      if (smeta[s].flags & kFlagNewSegment) {
        const double c0 = smeta[s].c[0], c1 = smeta[s].c[1], c2 = smeta[s].c[2];
#pragma unroll
        for (int k = 0; k < kTargetsPerThread; ++k) {
          xr[k][0] = (float)(X[k][0] - c0);
          xr[k][1] = (float)(X[k][1] - c1);
          xr[k][2] = (float)(X[k][2] - c2);
        }
      }
      float a[kTargetsPerThread];
      const float4* sb = reinterpret_cast<const float4*>(sbuf[s]);
      chunk_f32<KERN>(sb, xr, a, v.neg_kappa_log2e);
      bool bad = false;
#pragma unroll
      for (int k = 0; k < kTargetsPerThread; ++k) bad = bad || not_finite(a[k]);
      if (__any_sync(0xffffffffu, bad)) chunk_f32_guarded<KERN>(sb, xr, a, v.neg_kappa_log2e);
#pragma unroll
      for (int k = 0; k < kTargetsPerThread; ++k) acc[k] += (double)a[k];
    } else {
      double a[kTargetsPerThread];
      const double4* sb = reinterpret_cast<const double4*>(sbuf[s]);
      chunk_f64<KERN>(sb, X, a, v.kappa);
      bool bad = false;
#pragma unroll
      for (int k = 0; k < kTargetsPerThread; ++k) bad = bad || not_finite(a[k]);
      if (__any_sync(0xffffffffu, bad)) chunk_f64_guarded<KERN>(sb, X, a, v.kappa);
#pragma unroll
      for (int k = 0; k < kTargetsPerThread; ++k) acc[k] += a[k];
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
}

template <bool F32, int KERN>
static const void* kernel_ptr() {
  return reinterpret_cast<const void*>(&k_interact<F32, KERN>);
}

static const void* select_kernel(const bldtt_plan* p) {
  bool f32 = p->precision == BLDTT_FP32_BULK;
  switch (p->kernel) {
    case BLDTT_COULOMB: return f32 ? kernel_ptr<true, BLDTT_COULOMB>() : kernel_ptr<false, BLDTT_COULOMB>();
    case BLDTT_YUKAWA: return f32 ? kernel_ptr<true, BLDTT_YUKAWA>() : kernel_ptr<false, BLDTT_YUKAWA>();
    default: return f32 ? kernel_ptr<true, BLDTT_TEST_POLY>() : kernel_ptr<false, BLDTT_TEST_POLY>();
  }
}

int interaction_grid(bldtt_plan* p, int* grid) {
  int dev = 0, sms = 0, per_sm = 0;
  BL_CUDA(cudaGetDevice(&dev));
  BL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  BL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, select_kernel(p), kThreads, 0));
  if (per_sm < 1) per_sm = 1;
  int g = sms * per_sm;
  if (p->nitems > 0 && g > p->nitems) g = p->nitems;
  *grid = g < 1 ? 1 : g;
  return BLDTT_OK;
}

int run_interactions(bldtt_plan* p, cudaStream_t s) {
  if (p->nitems == 0) return BLDTT_OK;
  const Tree& tt = p->tt;
  const Tree& st = p->st;
  InteractView v;
  v.items = p->items;
  v.nitems = p->nitems;
  v.counter = p->item_counter;
  v.list_ptr = p->list_ptr;
  v.list_src = p->list_src;
  v.nct = tt.nclusters;
  v.t_parent = tt.parent;
  v.s_leaf_first = st.leaf_first;
  v.s_leaf_last = st.leaf_last;
  v.s_leaf_ids = st.leaf_ids;
  v.pad_prefix = p->pad_prefix;
  v.s_center = st.center;
  v.np_pad = p->np_pad;
  v.proxy_base = p->pool_particles;
  v.pool = p->pool;
  v.tx = tt.x;
  v.ty = tt.y;
  v.tz = tt.z;
  v.t_nodes = tt.nodes;
  v.P = p->P;
  v.np = p->np;
  v.phi_near = p->phi_near;
  v.phit = p->phit;
  v.err = p->dev_err;
  v.kappa = p->kappa;
  v.neg_kappa_log2e = (float)(-p->kappa * 1.4426950408889634);
  BL_CUDA(cudaMemsetAsync(p->item_counter, 0, sizeof(int32_t), s));
  void* args[] = {&v};
  BL_CUDA(cudaLaunchKernel(select_kernel(p), dim3(p->interact_grid), dim3(kThreads), args, 0, s));
  BL_LAUNCHED(p->compute_counter.launches);
  return BLDTT_OK;
}

}  // namespace bldtt
