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
// complete on mbarriers; NCW consumer warps evaluate G for K targets per
// thread against every staged source (NCW * 32 * K == kTile).
//
// FP32_BULK: every chunk of kChunk pool entries has its own frame centre c, a
// float near the chunk (particles inside a source leaf are in Morton order, so
// a chunk is spatially compact).  Entries hold y - c in FP32, formed from the
// split y = hi + lo (hi = fl(y), lo = fl(y - hi)) as fl(fl(hi - c) + lo), and
// are stored as pair records {x0,x1, y0,y1, z0,z1, q0,q1} so that one target
// meets two sources in packed f32x2 arithmetic (7 packed FP32 instructions and
// 2 MUFU.RSQ per two Coulomb evaluations).  Targets keep the same split and
// are moved into each chunk's frame with the same expression, so the
// coordinate rounding error is relative to the chunk size, and a target that
// coincides with a source gets exactly the same FP32 coordinates (r = 0).
// The two halves of the packed accumulator are two interleaved partial sums;
// each chunk's sum is added into an FP64 accumulator.
// FP64: pool entries are double4 (y, q) in absolute coordinates.
// Chunks carry their real source count, so padding is neither copied nor
// evaluated.
//
// A pair at distance 0 contributes nothing.  The fast path evaluates
// 1/sqrt(r^2) unguarded; a chunk whose partial sum is not finite (only
// possible when some r^2 == 0) is recomputed by the warp with the guard.
#include <type_traits>

#include "internal.cuh"

namespace bldtt {

constexpr uint64_t kWaitNs = 20ull * 1000ull * 1000ull * 1000ull;   // 20 s bound on any wait

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
  const int32_t* pad_prefix;
  const float4* chunk_frame;   // [chunks]: frame centre x, y, z (FP32) and the real count (int bits)
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
  float prm;                   // FP32 kernel parameter (see pair_f32)
};

struct StageMeta {
  int item;
  int count;                    // real sources in the staged chunk
  unsigned long long c2[3];     // frame centre, each component duplicated (f32x2)
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

// ---- packed FP32 (f32x2) helpers: low half = first element -----------------
typedef unsigned long long f2_t;
__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b) {
  f2_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b) {
  f2_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b) {
  f2_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c) {
  f2_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2_t f2_pack(float lo, float hi) {
  f2_t d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
__device__ __forceinline__ void f2_unpack(f2_t v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

// ---- kernel functions (Sec. 4.6); d = x - y -------------------------------
template <typename T>
__device__ __forceinline__ T poly_kernel(T dx, T dy, T dz) {
  return (T)1 + dx - (T)2 * dy + (T)3 * dz + dx * dy - dy * dz + dx * dx * dz * dz -
         (T)0.5 * dy * dy;
}

// Kernels that need an explicit r = 0 guard on every pair (finite at r = 0, or
// the test kernel); they take the scalar path in FP32.
template <int KERN>
struct AlwaysGuarded {
  static constexpr bool value = KERN == BLDTT_OSCILLATORY || KERN == BLDTT_REG_COULOMB ||
                                KERN == BLDTT_TEST_POLY;
};

// q * G in FP32; GUARD makes a pair at r^2 == 0 contribute 0.  prm is the
// kernel parameter in the form the kernel uses (Yukawa: -kappa*log2(e);
// oscillatory: kappa; regularized Coulomb: kappa^2).
template <int KERN, bool GUARD>
__device__ __forceinline__ float pair_f32(float dx, float dy, float dz, float q, float prm) {
  float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
  if (KERN == BLDTT_TEST_POLY) return r2 > 0.f ? q * poly_kernel<float>(dx, dy, dz) : 0.f;
  if ((GUARD || AlwaysGuarded<KERN>::value) && !(r2 > 0.f)) return 0.f;
  if (KERN == BLDTT_REG_COULOMB) return q * rsqrt_approx(r2 + prm);
  float ri = rsqrt_approx(r2);
  if (KERN == BLDTT_COULOMB) return q * ri;
  if (KERN == BLDTT_OSCILLATORY) return (q * ri) * sinf(prm * (r2 * ri));
  return (q * ri) * exp2_approx(r2 * ri * prm);
}
template <int KERN, bool GUARD>
__device__ __forceinline__ double pair_f64(double dx, double dy, double dz, double q, double kappa) {
  double r2 = dx * dx + dy * dy + dz * dz;
  if (KERN == BLDTT_TEST_POLY) return r2 > 0.0 ? q * poly_kernel<double>(dx, dy, dz) : 0.0;
  if ((GUARD || AlwaysGuarded<KERN>::value) && !(r2 > 0.0)) return 0.0;
  if (KERN == BLDTT_REG_COULOMB) return q * rsqrt(r2 + kappa * kappa);
  double ri = rsqrt(r2);
  if (KERN == BLDTT_COULOMB) return q * ri;
  if (KERN == BLDTT_OSCILLATORY) return q * ri * sin(kappa * (r2 * ri));
  return q * ri * exp(-kappa * (r2 * ri));
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

  // Stream pool entries [off, off + len) in kChunk pieces (real entries only).
  __device__ bool segment(int64_t off, int64_t len) {
    for (int64_t k = 0; k < len; k += kChunk) {
      int s;
      if (!acquire(s)) return false;
      const int64_t q = (off + k) / kChunk;
      const float4 f = v.chunk_frame[q];
      const int count = __float_as_int(f.w);
      StageMeta& m = meta[s];
      m.item = cur_item;
      m.count = count;
      uint32_t bytes;
      if (std::is_same<Vec, float4>::value) {
        m.c2[0] = f2_pack(f.x, f.x);
        m.c2[1] = f2_pack(f.y, f.y);
        m.c2[2] = f2_pack(f.z, f.z);
        bytes = (uint32_t)(((count + 1) / 2) * 32);          // whole pair records
      } else {
        bytes = (uint32_t)(count * sizeof(Vec));
      }
      const char* src = reinterpret_cast<const char*>(v.pool) + (off + k) * (int64_t)sizeof(Vec);
      mbar_arrive_tx(&full[s], bytes);
      bulk_copy_g2s(buf[s], src, bytes, &full[s]);
      ++it;
    }
    return true;
  }

  // Particles of all source leaves under cluster s: one contiguous pool range,
  // because leaves under a cluster are consecutive in leaf order.
  __device__ bool leaves_of(int32_t s) {
    int64_t o = v.pad_prefix[v.s_leaf_first[s]];
    return segment(o, v.pad_prefix[v.s_leaf_last[s]] - o);
  }

  __device__ bool lists(int type_particles, int type_proxies, int32_t c) {
    int64_t k0 = (int64_t)type_particles * v.nct + c;
    for (int32_t e = v.list_ptr[k0]; e < v.list_ptr[k0 + 1]; ++e)
      if (!leaves_of(v.list_src[e])) return false;
    int64_t k1 = (int64_t)type_proxies * v.nct + c;
    for (int32_t e = v.list_ptr[k1]; e < v.list_ptr[k1 + 1]; ++e)
      if (!segment(v.proxy_base + (int64_t)v.list_src[e] * v.np_pad, v.np_pad)) return false;
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
// Packed evaluation of target k against the source pair (s0, s1):
// acc += (q0 G(x - s0), q1 G(x - s1)).
template <int KERN>
__device__ __forceinline__ f2_t pair2_f32(f2_t tx, f2_t ty, f2_t tz, const ulonglong2& a,
                                          const ulonglong2& b, f2_t acc, f2_t nk2) {
  const f2_t dx = f2_sub(tx, a.x), dy = f2_sub(ty, a.y), dz = f2_sub(tz, b.x);
  const f2_t r2 = f2_fma(dz, dz, f2_fma(dy, dy, f2_mul(dx, dx)));
  float r0, r1;
  f2_unpack(r2, r0, r1);
  const f2_t ri = f2_pack(rsqrt_approx(r0), rsqrt_approx(r1));
  if (KERN == BLDTT_COULOMB) return f2_fma(b.y, ri, acc);
  // Yukawa: q ri exp2(-kappa log2(e) r), r = r2 ri
  float e0, e1;
  f2_unpack(f2_mul(f2_mul(r2, ri), nk2), e0, e1);
  return f2_fma(f2_mul(b.y, ri), f2_pack(exp2_approx(e0), exp2_approx(e1)), acc);
}

// Sum over the staged chunk of q G for K targets; two partial sums per target.
template <int KERN, int K>
__device__ __forceinline__ void chunk_f32(const ulonglong2* __restrict__ sb, int npairs,
                                          const f2_t (&x2)[K][3], float (&a)[K], float nk) {
  f2_t acc[K];
  const f2_t nk2 = f2_pack(nk, nk);
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0ull;
  if (npairs == kChunk / 2) {
#pragma unroll 8
    for (int jp = 0; jp < kChunk / 2; ++jp) {
      const ulonglong2 A = sb[2 * jp], Bq = sb[2 * jp + 1];
#pragma unroll
      for (int k = 0; k < K; ++k) acc[k] = pair2_f32<KERN>(x2[k][0], x2[k][1], x2[k][2], A, Bq, acc[k], nk2);
    }
  } else {
    for (int jp = 0; jp < npairs; ++jp) {
      const ulonglong2 A = sb[2 * jp], Bq = sb[2 * jp + 1];
#pragma unroll
      for (int k = 0; k < K; ++k) acc[k] = pair2_f32<KERN>(x2[k][0], x2[k][1], x2[k][2], A, Bq, acc[k], nk2);
    }
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    float lo, hi;
    f2_unpack(acc[k], lo, hi);
    a[k] = lo + hi;
  }
}

// Scalar re-evaluation with the r = 0 guard (rare: only chunks that produced a
// non-finite partial sum), and the test kernel.
template <int KERN, int K>
__device__ __forceinline__ void chunk_f32_guarded(const float* __restrict__ sf, int count,
                                                  const f2_t (&x2)[K][3], float (&a)[K], float nk) {
  float xs[K][3];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    float hi;
    f2_unpack(x2[k][0], xs[k][0], hi);
    f2_unpack(x2[k][1], xs[k][1], hi);
    f2_unpack(x2[k][2], xs[k][2], hi);
    a[k] = 0.f;
  }
  for (int j = 0; j < count; ++j) {
    const float* r = sf + (j >> 1) * 8 + (j & 1);   // pair record: x0 x1 y0 y1 z0 z1 q0 q1
    const float sx = r[0], sy = r[2], sz = r[4], q = r[6];
#pragma unroll
    for (int k = 0; k < K; ++k)
      a[k] += pair_f32<KERN, true>(xs[k][0] - sx, xs[k][1] - sy, xs[k][2] - sz, q, nk);
  }
}

template <int KERN, bool GUARD, int K>
__device__ __forceinline__ void chunk_f64(const double4* __restrict__ sb, int count,
                                          const double (&x)[K][3], double (&a)[K], double kappa) {
#pragma unroll
  for (int k = 0; k < K; ++k) a[k] = 0.0;
#pragma unroll 4
  for (int j = 0; j < count; ++j) {
    const double4 p = sb[j];
#pragma unroll
    for (int k = 0; k < K; ++k)
      a[k] += pair_f64<KERN, GUARD>(x[k][0] - p.x, x[k][1] - p.y, x[k][2] - p.z, p.w, kappa);
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

__device__ __forceinline__ void store_output(const InteractView& v, const int4& item, int r,
                                             double value) {
  if (r < item.z) {
    if (item.w == kItemParticles)
      v.phi_near[(int64_t)item.y + r] = value;
    else
      v.phit[(int64_t)item.x * v.np + item.y + r] = value;
  }
}

template <bool F32, int KERN, int NCW, int K, int MINB>
__global__ void __launch_bounds__((NCW + 1) * 32, MINB) k_interact(InteractView v) {
  static_assert(NCW * 32 * K == kTile, "a CTA covers exactly one work-item tile");
  constexpr int kConsumers = NCW * 32;
  using Vec = typename std::conditional<F32, float4, double4>::type;
  __shared__ __align__(128) Vec sbuf[kStages][kChunk];
  __shared__ __align__(16) StageMeta smeta[kStages];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ __align__(8) uint64_t empty[kStages];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NCW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == NCW) {
    if (lane == 0) {
      Producer<Vec> prod(v, sbuf, smeta, full, empty);
      prod.run();
    }
    return;
  }

  const int ct = threadIdx.x;   // consumer thread 0..kConsumers-1
  int cur = -1;
  int4 item = make_int4(0, 0, 0, 0);
  double X[K][3];               // FP64 targets (FP64 path)
  f2_t xh2[K][3], xl2[K][3];    // FP32 split of the targets, each duplicated (FP32 path)
  double acc[K];
  bool warp_full = true;
  for (uint32_t it = 0;; ++it) {
    const int s = (int)(it % kStages);
    if (!mbar_wait(&full[s], (it / kStages) & 1u, v.err)) return;
    const int mi = smeta[s].item;
    if (mi != cur) {
      if (cur >= 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) store_output(v, item, k * kConsumers + ct, acc[k]);
      }
      if (mi < 0) return;
      cur = mi;
      item = v.items[mi];
      // does any row of this warp's last target slot hold a real target?
      warp_full = (K - 1) * kConsumers + (warp * 32) < item.z;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        acc[k] = 0.0;
        target_coords(v, item, k * kConsumers + ct, X[k][0], X[k][1], X[k][2]);
        if (F32) {
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const float h = (float)X[k][d];
            const float l = (float)(X[k][d] - (double)h);
            xh2[k][d] = f2_pack(h, h);
            xl2[k][d] = f2_pack(l, l);
          }
        }
      }
    }
    const int count = smeta[s].count;
    if (F32) {
      f2_t x2[K][3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const f2_t c2 = smeta[s].c2[d];
#pragma unroll
        for (int k = 0; k < K; ++k) x2[k][d] = f2_add(f2_sub(xh2[k][d], c2), xl2[k][d]);
      }
      float a[K];
      if (AlwaysGuarded<KERN>::value) {
        chunk_f32_guarded<KERN, K>(reinterpret_cast<const float*>(sbuf[s]), count, x2, a,
                                   v.prm);
      } else {
        if (K > 1 && !warp_full) {
          // the warp's last target row lies beyond a partial tile: evaluate the others only
          float a1[K > 1 ? K - 1 : 1];
          const f2_t(&x2s)[K > 1 ? K - 1 : 1][3] = *reinterpret_cast<const f2_t(*)[K > 1 ? K - 1 : 1][3]>(&x2);
          chunk_f32<KERN, (K > 1 ? K - 1 : 1)>(reinterpret_cast<const ulonglong2*>(sbuf[s]),
                                               (count + 1) / 2, x2s, a1, v.prm);
#pragma unroll
          for (int k = 0; k < K; ++k) a[k] = k < K - 1 ? a1[k < K - 1 ? k : 0] : 0.f;
        } else {
          chunk_f32<KERN, K>(reinterpret_cast<const ulonglong2*>(sbuf[s]), (count + 1) / 2, x2, a,
                             v.prm);
        }
        bool bad = false;
#pragma unroll
        for (int k = 0; k < K; ++k) bad = bad || not_finite(a[k]);
        if (__any_sync(0xffffffffu, bad))
          chunk_f32_guarded<KERN, K>(reinterpret_cast<const float*>(sbuf[s]), count, x2, a,
                                     v.prm);
      }
#pragma unroll
      for (int k = 0; k < K; ++k) acc[k] += (double)a[k];
    } else {
      const double4* sb = reinterpret_cast<const double4*>(sbuf[s]);
      double a[K];
      chunk_f64<KERN, false, K>(sb, count, X, a, v.kappa);
      if (!AlwaysGuarded<KERN>::value) {
        bool bad = false;
#pragma unroll
        for (int k = 0; k < K; ++k) bad = bad || not_finite(a[k]);
        if (__any_sync(0xffffffffu, bad)) chunk_f64<KERN, true, K>(sb, count, X, a, v.kappa);
      }
#pragma unroll
      for (int k = 0; k < K; ++k) acc[k] += a[k];
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
}

// Consumer layouts the kernel is instantiated for (NCW warps x K targets, and
// the CTAs per SM the register allocation is sized for).
struct Layout {
  int ncw, k, minb;
};
static const Layout kLayouts[] = {{4, 2, 6}, {2, 4, 6}, {4, 2, 8}};
constexpr int kNumLayouts = 3;

template <bool F32, int KERN>
static const void* kernel_for(int layout) {
  if (KERN == BLDTT_COULOMB) {   // the tuned path: every layout is instantiated
    switch (layout) {
      case 1: return reinterpret_cast<const void*>(&k_interact<F32, KERN, 2, 4, 6>);
      case 2: return reinterpret_cast<const void*>(&k_interact<F32, KERN, 4, 2, 8>);
      default: break;
    }
  }
  return reinterpret_cast<const void*>(&k_interact<F32, KERN, 4, 2, 6>);
}

static int effective_layout(const bldtt_plan* p) {
  return p->kernel == BLDTT_COULOMB ? p->interact_layout : 0;
}

static const void* select_kernel(const bldtt_plan* p, int layout) {
  bool f32 = p->precision == BLDTT_FP32_BULK;
  switch (p->kernel) {
    case BLDTT_COULOMB: return f32 ? kernel_for<true, BLDTT_COULOMB>(layout) : kernel_for<false, BLDTT_COULOMB>(layout);
    case BLDTT_YUKAWA: return f32 ? kernel_for<true, BLDTT_YUKAWA>(layout) : kernel_for<false, BLDTT_YUKAWA>(layout);
    case BLDTT_OSCILLATORY: return f32 ? kernel_for<true, BLDTT_OSCILLATORY>(layout) : kernel_for<false, BLDTT_OSCILLATORY>(layout);
    case BLDTT_REG_COULOMB: return f32 ? kernel_for<true, BLDTT_REG_COULOMB>(layout) : kernel_for<false, BLDTT_REG_COULOMB>(layout);
    default: return f32 ? kernel_for<true, BLDTT_TEST_POLY>(layout) : kernel_for<false, BLDTT_TEST_POLY>(layout);
  }
}

int interaction_grid(bldtt_plan* p, int* grid) {
  int dev = 0, sms = 0, per_sm = 0;
  p->interact_layout = effective_layout(p);
  const int threads = (kLayouts[p->interact_layout].ncw + 1) * 32;
  BL_CUDA(cudaGetDevice(&dev));
  BL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  BL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, select_kernel(p, p->interact_layout),
                                                        threads, 0));
  if (per_sm < 1) per_sm = 1;
  int g = sms * per_sm;
  if (p->nitems > 0 && g > p->nitems) g = p->nitems;
  *grid = g < 1 ? 1 : g;
  p->interact_threads = threads;
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
  v.pad_prefix = p->pad_prefix;
  v.chunk_frame = p->chunk_frame;
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
  v.prm = p->kernel == BLDTT_YUKAWA       ? (float)(-p->kappa * 1.4426950408889634)
          : p->kernel == BLDTT_REG_COULOMB ? (float)(p->kappa * p->kappa)
                                           : (float)p->kappa;
  BL_CUDA(cudaMemsetAsync(p->item_counter, 0, sizeof(int32_t), s));
  void* args[] = {&v};
  BL_CUDA(cudaLaunchKernel(select_kernel(p, p->interact_layout), dim3(p->interact_grid),
                           dim3(p->interact_threads), args, 0, s));
  BL_LAUNCHED(p->compute_counter.launches);
  return BLDTT_OK;
}

}  // namespace bldtt
