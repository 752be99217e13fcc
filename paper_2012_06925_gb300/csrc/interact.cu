// PP, PC, CP and CC interactions (Sec. 2.4, Eqs. (6), (8), (12), (15)) in one
// persistent kernel, launched once per kernel type of the plan.
//
// All four interaction types are "targets x sources" sums (Sec. 3.3): the
// targets are particles (PP, PC) or proxy points (CP, CC) of a target cluster,
// the sources are particles (PP, CP) or proxy points with proxy charges
// (PC, CC) of a source cluster.  A work item is a tile of up to kTile targets
// of one target cluster; its sources are the concatenation of
//   particle tiles: PP and PC (every degree) entries of the leaf and of every
//                   ancestor (an entry on an ancestor applies to all its
//                   particles)
//   proxy tiles:    CP and CC entries of one degree on the cluster itself
//                   (the targets are that degree's proxy points).
// Each item owns its outputs, so there are no atomics and the summation order
// is fixed.
//
// Per CTA, one producer warp grabs items from a global counter, walks their
// lists and streams the sources, kChunk at a time, from the source pool into
// a shared-memory ring (3 or 4 stages) with cp.async.bulk (TMA) copies that
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
// Close pairs (FP32_BULK): every chunk also carries its half-extents and a
// near distance tau; the producer flags the 32-target groups whose box comes
// within tau of a particle chunk and then also stages the chunk's frame
// residuals; a flagged warp adds the residuals of both points to the
// coordinate differences of its near targets (see eval_chunk_f32).
//
// A pair at distance 0 contributes nothing.  The fast path evaluates
// 1/sqrt(r^2) unguarded; a chunk whose partial sum is not finite (only
// possible when some r^2 == 0) is recomputed by the warp with the guard, in
// the same arithmetic and order, so that a target's result never depends on
// which warp or consumer layout evaluated it.
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
  const float4* chunk_frame;   // [chunks][2]: frame centre + real count (int bits), extents + tau
  const float* pool_res;       // FP32: frame residuals of the pool's particles (pair records)
  const float4* item_box;      // FP32: [items][kItemGroups][2] target group boxes (lo, hi)
  DegreeSet deg;               // degrees, proxies per cluster and pool offsets per degree
  const void* pool;
  // targets and outputs (consumers)
  const double* tx;
  const double* ty;
  const double* tz;
  const double* t_nodes[kMaxDegrees];   // target proxy nodes per degree index
  double* phi_near;
  double* phit[kMaxDegrees];            // target proxy potentials per degree index
  int* err;
  // per-problem kernel parameters (read once per work item)
  const int32_t* t_problem;    // target cluster -> problem
  const float* prob_prm;       // FP32 kernel parameter (see pair_f32)
  const double* prob_kappa;
  const int* prob_kernel;      // kernel of each problem (read per item by the fused launch)
};

struct StageMeta {
  int item;
  int count;                    // real sources in the staged chunk
  int chunk;                    // pool chunk index
  unsigned near;                // bit g: target group g may be near the chunk (residuals staged)
  unsigned long long c2[3];     // frame centre, each component duplicated (f32x2)
  float4 ext;                   // half-extents and near distance tau (-inf: proxies)
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
template <typename Vec, int RES, int STAGES>
struct Producer {
  const InteractView& v;
  Vec (*buf)[kChunk];
  float4 (*rbuf)[RES];
  StageMeta* meta;
  uint64_t* full;
  uint64_t* empty;
  uint32_t it = 0;
  int cur_item = -1;
  int cur_groups = 0;
  float* ibox;                  // [6] bounding box of the current item's targets (shared memory)

  __device__ Producer(const InteractView& v_, Vec (*b)[kChunk], float4 (*r)[RES], StageMeta* m,
                      uint64_t* f, uint64_t* e, float* box)
      : v(v_), buf(b), rbuf(r), meta(m), full(f), empty(e), ibox(box) {}

  __device__ __noinline__ void load_item_box() {
    const float4* gb = v.item_box + (int64_t)cur_item * (2 * kItemGroups);
    float b[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (int g = 0; g < cur_groups; ++g) {
      const float4 lo = gb[2 * g], hi = gb[2 * g + 1];
      b[0] = fminf(b[0], lo.x);
      b[1] = fminf(b[1], lo.y);
      b[2] = fminf(b[2], lo.z);
      b[3] = fmaxf(b[3], hi.x);
      b[4] = fmaxf(b[4], hi.y);
      b[5] = fmaxf(b[5], hi.z);
    }
    for (int d = 0; d < 6; ++d) ibox[d] = b[d];
  }

  // Target groups of the current item whose box comes within tau of the
  // particle chunk's box (c +- e): a superset of the targets the consumers'
  // own test finds near.  The item's box is tested first.
  __device__ __forceinline__ unsigned near_groups(const float4& f, const float4& ext) const {
    if (!(ext.w >= 0.f)) return 0u;       // proxy chunk
    const float gap = fmaxf(fmaxf(fmaxf(ibox[0] - (f.x + ext.x), (f.x - ext.x) - ibox[3]),
                                  fmaxf(ibox[1] - (f.y + ext.y), (f.y - ext.y) - ibox[4])),
                            fmaxf(ibox[2] - (f.z + ext.z), (f.z - ext.z) - ibox[5]));
    return gap < ext.w ? near_groups_of_item(f, ext) : 0u;
  }
  __device__ __noinline__ unsigned near_groups_of_item(const float4 f, const float4 ext) const {
    const float clo[3] = {f.x - ext.x, f.y - ext.y, f.z - ext.z};
    const float chi[3] = {f.x + ext.x, f.y + ext.y, f.z + ext.z};
    const float4* gb = v.item_box + (int64_t)cur_item * (2 * kItemGroups);
    unsigned mask = 0;
    for (int g = 0; g < cur_groups; ++g) {
      const float4 lo = gb[2 * g], hi = gb[2 * g + 1];
      const float gap = fmaxf(fmaxf(fmaxf(lo.x - chi[0], clo[0] - hi.x), fmaxf(lo.y - chi[1], clo[1] - hi.y)),
                              fmaxf(lo.z - chi[2], clo[2] - hi.z));
      if (gap < ext.w) mask |= 1u << g;
    }
    return mask;
  }

  __device__ bool acquire(int& s) {
    s = (int)(it % STAGES);
    return mbar_wait(&empty[s], ((it / STAGES) & 1u) ^ 1u, v.err);
  }

  // Stream pool entries [off, off + len) in kChunk pieces (real entries only).
  __device__ bool segment(int64_t off, int64_t len) {
    for (int64_t k = 0; k < len; k += kChunk) {
      int s;
      if (!acquire(s)) return false;
      const int64_t q = (off + k) / kChunk;
      const float4 f = v.chunk_frame[kChunkInfo * q];
      const int count = __float_as_int(f.w);
      StageMeta& m = meta[s];
      m.item = cur_item;
      m.count = count;
      m.chunk = (int)q;
      m.near = 0;
      uint32_t bytes;
      if (std::is_same<Vec, float4>::value) {
        m.c2[0] = f2_pack(f.x, f.x);
        m.c2[1] = f2_pack(f.y, f.y);
        m.c2[2] = f2_pack(f.z, f.z);
        m.ext = v.chunk_frame[kChunkInfo * q + 1];
        m.near = near_groups(f, m.ext);
        bytes = (uint32_t)(((count + 1) / 2) * 32);          // whole pair records
      } else {
        bytes = (uint32_t)(count * sizeof(Vec));
      }
      const char* src = reinterpret_cast<const char*>(v.pool) + (off + k) * (int64_t)sizeof(Vec);
      mbar_arrive_tx(&full[s], m.near ? 2 * bytes : bytes);
      bulk_copy_g2s(buf[s], src, bytes, &full[s]);
      if (RES == kChunk && m.near)     // the chunk's frame residuals, same record layout
        bulk_copy_g2s(rbuf[s], v.pool_res + q * (int64_t)(kChunk * 4), bytes, &full[s]);
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

  // Entries of list class cls of target cluster c: particles of the source
  // clusters, or their proxy blocks of degree index i (i >= 0).
  __device__ bool entries(int cls, int i, int32_t c) {
    const int64_t k = (int64_t)cls * v.nct + c;
    for (int32_t e = v.list_ptr[k]; e < v.list_ptr[k + 1]; ++e) {
      const int32_t src = v.list_src[e];
      const bool ok = i < 0 ? leaves_of(src)
                            : segment(v.deg.proxy_base[i] + (int64_t)src * v.deg.np_pad[i], v.deg.np_pad[i]);
      if (!ok) return false;
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
      cur_groups = (item.z + 31) / 32;
      if (std::is_same<Vec, float4>::value) load_item_box();
      if (item.w == kItemParticles) {   // PP and PC of every degree, leaf and ancestors
        for (int32_t a = item.x; a >= 0 && ok; a = v.t_parent[a]) {
          ok = entries(0, -1, a);
          for (int i = 0; i < v.deg.n && ok; ++i) ok = entries(class_of(BLDTT_PC, i), i, a);
        }
      } else {                          // CP and CC of one degree on the cluster itself
        const int i = item.w - kItemProxies;
        ok = entries(class_of(BLDTT_CP, i), -1, item.x) && entries(class_of(BLDTT_CC, i), i, item.x);
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
    uint32_t first = it > (uint32_t)STAGES ? it - STAGES : 0;
    for (uint32_t j = first; j < it; ++j) mbar_wait(&full[j % STAGES], (j / STAGES) & 1u, v.err);
  }
};

// ---- consumers --------------------------------------------------------------
// Packed evaluation of target k against the source pair (s0, s1):
// acc += (q0 G(x - s0), q1 G(x - s1)).
template <int KERN>
__device__ __forceinline__ f2_t pair2_eval(f2_t dx, f2_t dy, f2_t dz, f2_t q2, f2_t acc, f2_t nk2) {
  const f2_t r2 = f2_fma(dz, dz, f2_fma(dy, dy, f2_mul(dx, dx)));
  float r0, r1;
  f2_unpack(r2, r0, r1);
  const f2_t ri = f2_pack(rsqrt_approx(r0), rsqrt_approx(r1));
  if (KERN == BLDTT_COULOMB) return f2_fma(q2, ri, acc);
  // Yukawa: q ri exp2(-kappa log2(e) r), r = r2 ri
  float e0, e1;
  f2_unpack(f2_mul(f2_mul(r2, ri), nk2), e0, e1);
  return f2_fma(f2_mul(q2, ri), f2_pack(exp2_approx(e0), exp2_approx(e1)), acc);
}
template <int KERN>
__device__ __forceinline__ f2_t pair2_f32(f2_t tx, f2_t ty, f2_t tz, const ulonglong2& a,
                                          const ulonglong2& b, f2_t acc, f2_t nk2) {
  return pair2_eval<KERN>(f2_sub(tx, a.x), f2_sub(ty, a.y), f2_sub(tz, b.x), b.y, acc, nk2);
}
// Careful variant: d = fma(m, x_r - y_r, x'' - y'') with m = 1 for a target
// near the chunk (frame residuals added) and m = 0 otherwise (exactly the
// packed difference x'' - y'').
template <int KERN>
__device__ __forceinline__ f2_t pair2_careful(f2_t tx, f2_t ty, f2_t tz, f2_t rx, f2_t ry, f2_t rz,
                                              f2_t m2, const ulonglong2& a, const ulonglong2& b,
                                              const ulonglong2& ra, const ulonglong2& rb, f2_t acc,
                                              f2_t nk2) {
  return pair2_eval<KERN>(f2_fma(m2, f2_sub(rx, ra.x), f2_sub(tx, a.x)),
                          f2_fma(m2, f2_sub(ry, ra.y), f2_sub(ty, a.y)),
                          f2_fma(m2, f2_sub(rz, rb.x), f2_sub(tz, b.x)), b.y, acc, nk2);
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

// A consumer thread's targets, split v = hi + lo in FP32 (each duplicated
// f32x2), kept in shared memory rather than registers: entry (k, d) of the
// thread is h[(3k + d) * stride].
struct TargetSplit {
  const f2_t* h;
  const f2_t* l;
  int stride;
  __device__ __forceinline__ f2_t hi(int k, int d) const { return h[(3 * k + d) * stride]; }
  __device__ __forceinline__ f2_t lo(int k, int d) const { return l[(3 * k + d) * stride]; }
};

// Frame residual (frame_resid) of target slot k in the chunk's frame c2.
__device__ __forceinline__ void target_residual(const TargetSplit& ts, const f2_t* c2, int k,
                                                float (&xr)[3]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    float c, h, l, hi;
    f2_unpack(c2[d], c, hi);
    f2_unpack(ts.hi(k, d), h, hi);
    f2_unpack(ts.lo(k, d), l, hi);
    xr[d] = frame_resid(h, l, c);
  }
}

// Careful packed sum over the staged chunk (sr: its frame residual records).
template <int KERN, int K>
__device__ __forceinline__ void chunk_f32_careful(const ulonglong2* __restrict__ sb,
                                                  const ulonglong2* __restrict__ sr, int npairs,
                                                  const f2_t (&x2)[K][3], const TargetSplit& ts,
                                                  const f2_t* c2, unsigned near, float (&a)[K],
                                                  float nk) {
  const f2_t nk2 = f2_pack(nk, nk);
  f2_t acc[K], m2[K], r2x[K][3];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float m = ((near >> k) & 1u) ? 1.f : 0.f;
    m2[k] = f2_pack(m, m);
    float xr[3];
    target_residual(ts, c2, k, xr);
#pragma unroll
    for (int d = 0; d < 3; ++d) r2x[k][d] = f2_pack(xr[d], xr[d]);
    acc[k] = 0ull;
  }
#pragma unroll 2
  for (int jp = 0; jp < npairs; ++jp) {
    const ulonglong2 A = sb[2 * jp], Bq = sb[2 * jp + 1], RA = sr[2 * jp], RB = sr[2 * jp + 1];
#pragma unroll
    for (int k = 0; k < K; ++k)
      acc[k] = pair2_careful<KERN>(x2[k][0], x2[k][1], x2[k][2], r2x[k][0], r2x[k][1], r2x[k][2],
                                   m2[k], A, Bq, RA, RB, acc[k], nk2);
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    float lo, hi;
    f2_unpack(acc[k], lo, hi);
    a[k] = lo + hi;
  }
}

// One pair in the fast path's scalar arithmetic (the packed path computes
// exactly this per lane), with the r = 0 guard: acc + q G(d).
template <int KERN>
__device__ __forceinline__ float pair_acc_f32(float dx, float dy, float dz, float q, float prm,
                                              float acc) {
  const float r2 = fmaf(dz, dz, fmaf(dy, dy, __fmul_rn(dx, dx)));
  if (!(r2 > 0.f)) return acc;
  if (KERN == BLDTT_COULOMB) return fmaf(q, rsqrt_approx(r2), acc);
  if (KERN == BLDTT_YUKAWA) {
    const float ri = rsqrt_approx(r2);
    return fmaf(__fmul_rn(q, ri), exp2_approx(__fmul_rn(__fmul_rn(r2, ri), prm)), acc);
  }
  return __fadd_rn(acc, pair_f32<KERN, true>(dx, dy, dz, q, prm));
}

// Scalar evaluation of a staged chunk: the same two partial sums (even and
// odd entries) and the same arithmetic as the packed path, with the r = 0
// guard.  Targets whose bit is set in `near` use the corrected difference
//   d = fl(fl(x'' - y'') + fl(x_r - y_r))
// of the frame coordinates x'', y'' and frame residuals x_r, y_r, which is
// within a few u |d| of the exact x - y however small |d| is.  Every other
// target gets bit for bit what the packed path gives it (when that is
// finite), so a target's result does not depend on its warp.
template <int KERN, int K>
__device__ __forceinline__ void chunk_f32_slow(const float* __restrict__ sf, const float* __restrict__ res,
                                               int count, const float (&xs)[K][3],
                                               const TargetSplit& ts, const f2_t* c2, unsigned near,
                                               float prm, float (&a)[K]) {
  // one target slot at a time: few live registers on this rare path
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const bool nr = (near >> k) & 1u;
    float xr[3] = {0.f, 0.f, 0.f};
    if (nr) target_residual(ts, c2, k, xr);
    float acc0 = 0.f, acc1 = 0.f;
    for (int jp = 0; jp < (count + 1) / 2; ++jp) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = 2 * jp + h;
        if (j < count) {
          const float* r = sf + jp * 8 + h;   // pair record: x0 x1 y0 y1 z0 z1 q0 q1
          float dx = __fsub_rn(xs[k][0], r[0]), dy = __fsub_rn(xs[k][1], r[2]),
                dz = __fsub_rn(xs[k][2], r[4]);
          if (nr) {
            const float* e = res + jp * 8 + h;
            dx = __fadd_rn(dx, __fsub_rn(xr[0], e[0]));
            dy = __fadd_rn(dy, __fsub_rn(xr[1], e[2]));
            dz = __fadd_rn(dz, __fsub_rn(xr[2], e[4]));
          }
          if (h == 0)
            acc0 = pair_acc_f32<KERN>(dx, dy, dz, r[6], prm, acc0);
          else
            acc1 = pair_acc_f32<KERN>(dx, dy, dz, r[6], prm, acc1);
        }
      }
    }
    a[k] = acc0 + acc1;
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
    const int i = item.w - kItemProxies;
    const int P = v.deg.d[i] + 1;
    int l = item.y + r;
    int l1 = l / (P * P), l2 = (l / P) % P, l3 = l % P;
    const double* nd = v.t_nodes[i] + (int64_t)item.x * 3 * P;
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
      v.phit[item.w - kItemProxies][(int64_t)item.x * v.deg.np[item.w - kItemProxies] + item.y + r] = value;
  }
}

// Out-of-line entries to the rare paths of the packed kernels, so that their
// registers do not burden the packed loop: they rebuild the targets' frame
// coordinates from the shared-memory split (the same rounding as the packed
// path) and return the K partial sums.
template <int K>
struct PartialSums {
  float v[K];
};
template <int K>
__device__ __forceinline__ void frame_targets(const TargetSplit& ts, const f2_t* c2, f2_t (&x2)[K][3]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const f2_t c = c2[d];
#pragma unroll
    for (int k = 0; k < K; ++k) x2[k][d] = f2_add(f2_sub(ts.hi(k, d), c), ts.lo(k, d));
  }
}
template <int KERN, int K>
__device__ __noinline__ PartialSums<K> slow_sums(const float* sf, const float* res, int count,
                                                 const TargetSplit ts, const f2_t* c2, unsigned near,
                                                 float prm) {
  f2_t x2[K][3];
  frame_targets<K>(ts, c2, x2);
  float xs[K][3];
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      float hi;
      f2_unpack(x2[k][d], xs[k][d], hi);
    }
  PartialSums<K> out;
  chunk_f32_slow<KERN, K>(sf, res, count, xs, ts, c2, near, prm, out.v);
  return out;
}
// One staged chunk in FP32 for K targets (partial sums in a[]).  ts holds
// the targets' FP32 splits and c2 the chunk's frame centre (duplicated
// f32x2), x2 the targets' frame coordinates, ext the chunk's half-extents and
// near distance tau, res its staged frame residuals, and bit k of `slot` says
// that the producer found target slot k's group near the chunk.  A target
// with max_d (|x''_d| - e_d) < tau is near: the warp then takes the careful
// packed path, which adds the frame residuals for near targets only.
// Otherwise the plain packed path runs.  A chunk whose packed sum is not
// finite (some r = 0) is redone in the scalar path with the r = 0 guard.
template <int KERN, int K>
__device__ __forceinline__ void eval_chunk_f32(const void* buf, const float4* rbuf, int count,
                                               const f2_t (&x2)[K][3], const TargetSplit& ts,
                                               const f2_t* c2, const float4* ext_p, unsigned slot, bool warp_full,
                                               float prm, float (&a)[K]) {
  const float* sf = reinterpret_cast<const float*>(buf);
  const float* res = reinterpret_cast<const float*>(rbuf);
  float xs[K][3];
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      float hi;
      f2_unpack(x2[k][d], xs[k][d], hi);
    }
  unsigned near = 0;
  bool any_near = false;
  if (slot) {                                   // warp-uniform
    const float4 ext = *ext_p;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float m = fmaxf(fmaxf(fabsf(xs[k][0]) - ext.x, fabsf(xs[k][1]) - ext.y),
                            fabsf(xs[k][2]) - ext.z);
      if (((slot >> k) & 1u) && m < ext.w) near |= 1u << k;
    }
    any_near = __any_sync(0xffffffffu, near != 0);
  }
  if (AlwaysGuarded<KERN>::value) {
    chunk_f32_slow<KERN, K>(sf, res, count, xs, ts, c2, near, prm, a);
    return;
  }
  const ulonglong2* sb = reinterpret_cast<const ulonglong2*>(buf);
  if (any_near) {
    chunk_f32_careful<KERN, K>(sb, reinterpret_cast<const ulonglong2*>(rbuf), (count + 1) / 2, x2, ts,
                               c2, near, a, prm);
  } else if (K > 1 && !warp_full) {
    // the warp's last target row lies beyond a partial tile: evaluate the others only
    constexpr int K1 = K > 1 ? K - 1 : 1;
    float a1[K1];
    const f2_t(&x2s)[K1][3] = *reinterpret_cast<const f2_t(*)[K1][3]>(&x2);
    chunk_f32<KERN, K1>(sb, (count + 1) / 2, x2s, a1, prm);
#pragma unroll
    for (int k = 0; k < K; ++k) a[k] = k < K1 ? a1[k < K1 ? k : 0] : 0.f;
  } else {
    chunk_f32<KERN, K>(sb, (count + 1) / 2, x2, a, prm);
  }
  bool bad = false;
#pragma unroll
  for (int k = 0; k < K; ++k) bad = bad || not_finite(a[k]);
  if (__any_sync(0xffffffffu, bad)) {
    const PartialSums<K> r = slow_sums<KERN, K>(sf, res, count, ts, c2, near, prm);
#pragma unroll
    for (int k = 0; k < K; ++k) a[k] = r.v[k];
  }
}

// One staged chunk in FP64 for K targets.
template <int KERN, int K>
__device__ __forceinline__ void eval_chunk_f64(const void* buf, int count, const double (&X)[K][3],
                                               double kappa, double (&a)[K]) {
  const double4* sb = reinterpret_cast<const double4*>(buf);
  chunk_f64<KERN, false, K>(sb, count, X, a, kappa);
  if (!AlwaysGuarded<KERN>::value) {
    bool bad = false;
#pragma unroll
    for (int k = 0; k < K; ++k) bad = bad || not_finite(a[k]);
    if (__any_sync(0xffffffffu, bad)) chunk_f64<KERN, true, K>(sb, count, X, a, kappa);
  }
}

// The parameter block is taken by value: device functions that read it by
// reference make each thread keep a private copy on its stack (0.5 KB; 70 MB
// of local writes per launch at 1E6, cached in L1).  Passing it as a
// __grid_constant__ parameter instead removes those writes but ran slower,
// 32.30 against 32.09 ms at 1E6 and 154-179 against 90 ms on the unequal-set
// Yukawa workload (1E7 targets, 5E6 Plummer sources), also when only the
// producer kept a private copy.  A pointer to per-segment blocks in device
// memory ran slower too: 32.3 against 32.1 ms and 143 against 90 ms.
template <bool F32, int KERN, int NCW, int K, int MINB, int STAGES, bool SKIP>
__global__ void __launch_bounds__((NCW + 1) * 32, MINB) k_interact(InteractView v) {
  static_assert(NCW * 32 * K == kTile, "a CTA covers exactly one work-item tile");
  constexpr int kConsumers = NCW * 32;
  using Vec = typename std::conditional<F32, float4, double4>::type;
  __shared__ __align__(128) Vec sbuf[STAGES][kChunk];
  constexpr int kRes = F32 ? kChunk : 1;     // frame residual records (FP32 only)
  __shared__ __align__(128) float4 sres[STAGES][kRes];
  __shared__ __align__(16) StageMeta smeta[STAGES];
  __shared__ __align__(8) uint64_t full[STAGES];
  __shared__ __align__(8) uint64_t empty[STAGES];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NCW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == NCW) {
    if (lane == 0) {
      __shared__ float s_ibox[6];
      Producer<Vec, kRes, STAGES> prod(v, sbuf, sres, smeta, full, empty, s_ibox);
      prod.run();
    }
    return;
  }

  const int ct = threadIdx.x;   // consumer thread 0..kConsumers-1
  int cur = -1;
  int4 item = make_int4(0, 0, 0, 0);
  double X[K][3];               // FP64 targets (FP64 path)
  // FP32 split of this thread's targets (FP32 path), in shared memory
  constexpr int kSplit = F32 ? K * 3 * kConsumers : 1;
  __shared__ __align__(16) f2_t s_th[kSplit], s_tl[kSplit];
  const TargetSplit ts{s_th + ct, s_tl + ct, kConsumers};
  double acc[K];
  bool warp_full = true;
  bool warp_active = true;
  float prm = 0.f;              // its FP32 parameter
  double kappa = 0.0;           // its FP64 parameter
  bool yukawa = KERN == BLDTT_YUKAWA;   // the fused Coulomb/Yukawa launch: this item's kernel
  for (uint32_t it = 0;; ++it) {
    const int s = (int)(it % STAGES);
    if (!mbar_wait(&full[s], (it / STAGES) & 1u, v.err)) return;
    const int mi = smeta[s].item;
    if (mi != cur) {
      if (cur >= 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) store_output(v, item, k * kConsumers + ct, acc[k]);
      }
      if (mi < 0) return;
      cur = mi;
      item = v.items[mi];
      const int pid = v.t_problem[item.x];
      prm = v.prob_prm[pid];
      kappa = v.prob_kappa[pid];
      if (KERN == kKernCoulombYukawa) yukawa = v.prob_kernel[pid] == BLDTT_YUKAWA;
      // does any row of this warp's last target slot hold a real target?
      warp_full = (K - 1) * kConsumers + (warp * 32) < item.z;
      // does any row of its first slot?  (if not, the warp only keeps the ring
      // going; layouts for plans with many small items skip such warps' work)
      if (SKIP) warp_active = warp * 32 < item.z;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        acc[k] = 0.0;
        target_coords(v, item, k * kConsumers + ct, X[k][0], X[k][1], X[k][2]);
        if (F32) {
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const float h = (float)X[k][d];
            const float l = (float)(X[k][d] - (double)h);
            s_th[(3 * k + d) * kConsumers + ct] = f2_pack(h, h);
            s_tl[(3 * k + d) * kConsumers + ct] = f2_pack(l, l);
          }
        }
      }
    }
    const int count = smeta[s].count;
    if (SKIP && !warp_active) {
      // no real target in this warp's rows: nothing to evaluate
    } else if constexpr (F32) {
      f2_t x2[K][3];
      const f2_t* c2 = smeta[s].c2;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const f2_t c = c2[d];
#pragma unroll
        for (int k = 0; k < K; ++k) x2[k][d] = f2_add(f2_sub(ts.hi(k, d), c), ts.lo(k, d));
      }
      const float4* ext = &smeta[s].ext;
      const unsigned gm = smeta[s].near;
      unsigned slot = 0;
      if (gm) {
#pragma unroll
        for (int k = 0; k < K; ++k) slot |= ((gm >> (k * NCW + warp)) & 1u) << k;
      }
      float a[K];
      if (KERN != kKernCoulombYukawa)
        eval_chunk_f32<KERN, K>(sbuf[s], sres[s], count, x2, ts, c2, ext, slot, warp_full, prm, a);
      else if (yukawa)
        eval_chunk_f32<BLDTT_YUKAWA, K>(sbuf[s], sres[s], count, x2, ts, c2, ext, slot, warp_full, prm, a);
      else
        eval_chunk_f32<BLDTT_COULOMB, K>(sbuf[s], sres[s], count, x2, ts, c2, ext, slot, warp_full, prm, a);
#pragma unroll
      for (int k = 0; k < K; ++k) acc[k] += (double)a[k];
    } else {
      double a[K];
      if (KERN != kKernCoulombYukawa)
        eval_chunk_f64<KERN, K>(sbuf[s], count, X, kappa, a);
      else if (yukawa)
        eval_chunk_f64<BLDTT_YUKAWA, K>(sbuf[s], count, X, kappa, a);
      else
        eval_chunk_f64<BLDTT_COULOMB, K>(sbuf[s], count, X, kappa, a);
#pragma unroll
      for (int k = 0; k < K; ++k) acc[k] += a[k];
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
}

// Consumer layouts the kernel is instantiated for: NCW warps x K targets, the
// CTAs per SM the register allocation is sized for, the depth of the
// shared-memory ring (3 stages let six CTAs share an SM; 4 stages at five
// CTAs hide the producer's list walks better on short items), and whether
// warps whose rows hold no real target skip their work (worth it when many
// items are smaller than a tile; a cost of about 1 % otherwise).  Layouts
// kLayoutSkip + i are layout i with skipping.
struct Layout {
  int ncw, k, minb, stages;
};
static const Layout kLayouts[kLayoutSkip] = {{4, 2, 6, 3}, {2, 4, 6, 3}, {4, 2, 5, 4}};

template <bool F32, int KERN, bool SKIP>
static const void* kernel_for_skip(int base) {
  if constexpr (KERN == BLDTT_COULOMB || KERN == kKernCoulombYukawa) {
    if (base == 1) return reinterpret_cast<const void*>(&k_interact<F32, KERN, 2, 4, 6, 3, SKIP>);
    if (base == 2) return reinterpret_cast<const void*>(&k_interact<F32, KERN, 4, 2, 5, 4, SKIP>);
  }
  return reinterpret_cast<const void*>(&k_interact<F32, KERN, 4, 2, 6, 3, SKIP>);
}

template <bool F32, int KERN>
static const void* kernel_for(int layout) {
  if constexpr (F32) {
    if (layout >= kLayoutSkip) return kernel_for_skip<F32, KERN, true>(layout - kLayoutSkip);
  }
  // FP64: the skipping instances are not built (the FP64 path's cost is its
  // arithmetic, not idle rows); a skipping layout runs its base layout.
  return kernel_for_skip<F32, KERN, false>(layout % kLayoutSkip);
}

// Layouts instantiated for a kernel (the autotuner tries these).
int layouts_available(int kernel, int* out) {
  const int nbase = (kernel == BLDTT_COULOMB || kernel == kKernCoulombYukawa) ? kLayoutSkip : 1;
  int n = 0;
  for (int i = 0; i < nbase; ++i) out[n++] = i;
  for (int i = 0; i < nbase; ++i) out[n++] = kLayoutSkip + i;
  return n;
}

int layout_threads(int layout) { return (kLayouts[layout % kLayoutSkip].ncw + 1) * 32; }

static const void* select_kernel(int kernel, bool f32, int layout) {
  switch (kernel) {
    case BLDTT_COULOMB: return f32 ? kernel_for<true, BLDTT_COULOMB>(layout) : kernel_for<false, BLDTT_COULOMB>(layout);
    case BLDTT_YUKAWA: return f32 ? kernel_for<true, BLDTT_YUKAWA>(layout) : kernel_for<false, BLDTT_YUKAWA>(layout);
    case kKernCoulombYukawa:
      return f32 ? kernel_for<true, kKernCoulombYukawa>(layout) : kernel_for<false, kKernCoulombYukawa>(layout);
    case BLDTT_OSCILLATORY: return f32 ? kernel_for<true, BLDTT_OSCILLATORY>(layout) : kernel_for<false, BLDTT_OSCILLATORY>(layout);
    case BLDTT_REG_COULOMB: return f32 ? kernel_for<true, BLDTT_REG_COULOMB>(layout) : kernel_for<false, BLDTT_REG_COULOMB>(layout);
    default: return f32 ? kernel_for<true, BLDTT_TEST_POLY>(layout) : kernel_for<false, BLDTT_TEST_POLY>(layout);
  }
}

// Persistent grid of every segment: all CTAs that fit on the device at once
// (never more than the segment's items).
int interaction_grids(bldtt_plan* p) {
  int dev = 0, sms = 0;
  BL_CUDA(cudaGetDevice(&dev));
  BL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const bool f32 = p->precision == BLDTT_FP32_BULK;
  for (auto& seg : p->segments) {
    int per_sm = 0;
    seg.threads = layout_threads(seg.layout);
    BL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, select_kernel(seg.kernel, f32, seg.layout), seg.threads, 0));
    if (per_sm < 1) per_sm = 1;
    const int g = sms * per_sm;
    seg.grid = g > seg.count ? seg.count : g;
    if (seg.grid < 1) seg.grid = 1;
  }
  return BLDTT_OK;
}

static InteractView make_view(const bldtt_plan* p) {
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
  v.pool_res = p->pool_res;
  v.item_box = p->item_box;
  v.deg = p->deg;
  v.pool = p->pool;
  v.tx = tt.x;
  v.ty = tt.y;
  v.tz = tt.z;
  for (int i = 0; i < kMaxDegrees; ++i) {
    v.t_nodes[i] = i < p->deg.n ? p->nodes_t[i] : nullptr;
    v.phit[i] = i < p->deg.n ? p->phit_d[i] : nullptr;
  }
  v.phi_near = p->phi_near;
  v.err = p->dev_err;
  v.t_problem = tt.problem;
  v.prob_prm = p->prob_prm;
  v.prob_kappa = p->prob_kappa;
  v.prob_kernel = p->prob_kernel;
  return v;
}

// One segment's persistent launch over items [first, first + count).
static int launch_segment(const bldtt_plan* p, const InteractView& base, int g, cudaStream_t s) {
  const auto& seg = p->segments[g];
  InteractView v = base;
  v.items = p->items + seg.first;
  v.nitems = seg.count;
  v.counter = p->item_counter + g;
  if (v.item_box) v.item_box = p->item_box + (int64_t)seg.first * (2 * kItemGroups);
  void* args[] = {&v};
  BL_CUDA(cudaLaunchKernel(select_kernel(seg.kernel, p->precision == BLDTT_FP32_BULK, seg.layout),
                           dim3(seg.grid), dim3(seg.threads), args, 0, s));
  return BLDTT_OK;
}

int run_segment(bldtt_plan* p, int g, cudaStream_t s) {
  BL_CUDA(cudaMemsetAsync(p->item_counter + g, 0, sizeof(int32_t), s));
  BL_TRY(launch_segment(p, make_view(p), g, s));
  BL_LAUNCHED(p->compute_counter.launches);
  return BLDTT_OK;
}

int run_interactions(bldtt_plan* p, cudaStream_t s) {
  if (p->nitems == 0 || p->segments.empty()) return BLDTT_OK;
  const InteractView v = make_view(p);
  BL_CUDA(cudaMemsetAsync(p->item_counter, 0, p->segments.size() * sizeof(int32_t), s));
  for (int g = 0; g < (int)p->segments.size(); ++g) {
    BL_TRY(launch_segment(p, v, g, s));
    BL_LAUNCHED(p->compute_counter.launches);
  }
  return BLDTT_OK;
}

}  // namespace bldtt
