// Tensor-core (tcgen05) forms of the two leaf contractions of FP32_BULK mode:
//
//   upward, Eq. (9):    qhat[k1,k2,k3] = sum_j L_k1(y_j1) L_k2(y_j2) L_k3(y_j3) q_j
//   downward, Eq. (21): phi(x_i)       = sum_k L_k1(x_i1) L_k2(x_i2) L_k3(x_i3) phi_t[k]
//
// Both are tensor-product contractions with one dense matrix product inside:
//   upward:   D[u][k1] = sum_j W[u][j] L1[k1][j],  W[u][j] = (L2[k2][j] q_j) L3[k3][j],
//             u = k2 P + k3 (M = P^2 rows padded to 128, N = P padded to 16,
//             K = the leaf's particles, 32 per chunk);
//   downward: T[i][u]  = sum_k1 L1[i][k1] phi_t[k1][u] (M = 128 particles per
//             tile, N = P^2 padded to a multiple of 16, K = P padded to 16),
//             then phi(x_i) = sum_k2 L2[i][k2] (sum_k3 L3[i][k3] T[i][k2 P + k3]).
// The basis values are the FP32_BULK ones of the SIMT kernels (float pairs of
// the points and nodes, exact weights, the coincident-point guard).
//
// Precision: the MMA runs kind::tf32 on operands split into two TF32 parts,
// a = a_h + a_l (a_h = tf32(a), a_l = tf32(a - a_h), so a_h + a_l holds a to
// about 2^-22), as all four products A_l B_l + A_h B_l + A_l B_h + A_h B_h
// (smallest first; dropping A_l B_l cost 10 % more error at 1E6 for no time)
// accumulated in FP32 in tensor memory.  The upward sum restarts every chunk
// of 32 particles and the chunks' results are added by TwoSum into a float
// pair per output (as the SIMT kernel folds its runs); the downward outer
// sums are compensated as in the SIMT kernel.
//
// Layout: operands are K-major in shared memory without swizzling: 8-row x
// 16-byte core matrices stored contiguously, core matrices adjacent in K 128
// bytes apart (leading byte offset) and 8-row groups KG*128 bytes apart
// (stride byte offset).  One thread issues the MMAs; tcgen05.commit signals an
// mbarrier whose wait is bounded (the plan's error flag on timeout); every
// warp reads its 32 rows of the accumulator with tcgen05.ld.
#include "basis.cuh"
#include "internal.cuh"

namespace bldtt {
namespace {

constexpr int kTcThreads = 128;
constexpr uint64_t kTcWaitNs = 5ull * 1000ull * 1000ull * 1000ull;   // 5 s bound on an MMA wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Element (r, k) of a K-major operand with KG core matrices along K, in floats.
__device__ __forceinline__ int kmaj(int r, int k, int KG) {
  return ((r >> 3) * KG + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | ((uint64_t)1 << 46);
}

// D in F32 (bits 4-5), A and B in TF32 (bits 7-9, 10-12), both K-major, N/8
// at bits 17-22, M/16 at bits 24-28.
constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Generic-proxy stores to shared memory made visible to the tensor core.
__device__ __forceinline__ void fence_smem_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ float to_tf32(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}

// Bounded wait for phase `parity` of an mbarrier (false after kTcWaitNs).
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  uint64_t t0 = 0;
  for (int spin = 0;; ++spin) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (spin == 0) t0 = t;
    else if (t - t0 > kTcWaitNs) return false;
  }
}

// 16 consecutive accumulator columns of this warp's 32 rows (one row per thread).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
      "[%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

template <int NCOLS>
__device__ __forceinline__ void tmem_alloc(uint32_t* slot) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "n"(NCOLS)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
template <int NCOLS>
__device__ __forceinline__ void tmem_free(uint32_t taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "n"(NCOLS) : "memory");
}

__device__ __forceinline__ void mbar_init1(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Upward leaf contraction, Eq. (9)
// ---------------------------------------------------------------------------
constexpr int kUpKC = 32;           // particles per MMA chunk: 4 K steps of 8
constexpr int kUpKG = kUpKC / 4;    // core matrices along K
constexpr int kUpGroup = 1;         // chunks accumulated in tensor memory per fold

template <int P>
__global__ void __launch_bounds__(kTcThreads) k_up_leaf_tc(
    const int32_t* __restrict__ leaf_ids, const int32_t* __restrict__ begin,
    const int32_t* __restrict__ end, const double* __restrict__ x, const double* __restrict__ y,
    const double* __restrict__ z, const double* __restrict__ q, const double* __restrict__ nodes,
    double* __restrict__ qhat, int* __restrict__ err) {
  constexpr int P2 = P * P, NP = P2 * P;
  static_assert(P2 <= 128 && P <= 16, "grid too large for one 128 x 16 accumulator");
  constexpr uint32_t kIdesc = idesc_tf32(128, 16);
  __shared__ __align__(1024) float sAh[128 * kUpKC], sAl[128 * kUpKC];
  __shared__ __align__(1024) float sBh[16 * kUpKC], sBl[16 * kUpKC];
  __shared__ float s2[P][kUpKC + 1], s3[P][kUpKC + 1];
  __shared__ float shl[3][2 * kMaxP];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int c = leaf_ids[blockIdx.x];
  const int32_t b = begin[c], e = end[c];
  // padding rows (u >= P^2 of A, k1 >= P of B) stay zero for the whole leaf
  for (int i = tid; i < 128 * kUpKC; i += kTcThreads) sAh[i] = sAl[i] = 0.f;
  for (int i = tid; i < 16 * kUpKC; i += kTcThreads) sBh[i] = sBl[i] = 0.f;
  if (tid < 3 * P) {
    float h, l;
    split_f64(nodes[(int64_t)c * 3 * P + tid], h, l);
    shl[tid / P][tid % P] = h;
    shl[tid / P][kMaxP + tid % P] = l;
  }
  if (tid == 0) mbar_init1(&bar);
  if (warp == 0) tmem_alloc<32>(&tmem_slot);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;
  float hi[P], lo[P];                 // each row's outputs as float pairs (TwoSum of the folds)
#pragma unroll
  for (int k = 0; k < P; ++k) hi[k] = lo[k] = 0.f;
  uint32_t phase = 0;
  bool ok = true;
  int ci = 0;
  for (int32_t base = b; base < e && ok; base += kUpKC, ++ci) {
    const int cnt = min(kUpKC, e - base);
    if (tid < 3 * kUpKC) {          // the chunk's basis values, one (dimension, particle) per thread
      const int d = tid / kUpKC, j = tid % kUpKC;
      float L[P];
      if (j < cnt) {
        const double* cd = d == 0 ? x : (d == 1 ? y : z);
        basis_f32_fixed<P>(cd[base + j], shl[d], L);
      } else {
#pragma unroll
        for (int k = 0; k < P; ++k) L[k] = 0.f;
      }
      if (d == 0) {
#pragma unroll
        for (int k = 0; k < P; ++k) {
          const float h = to_tf32(L[k]);
          sBh[kmaj(k, j, kUpKG)] = h;
          sBl[kmaj(k, j, kUpKG)] = to_tf32(L[k] - h);
        }
      } else if (d == 1) {
        const float qj = j < cnt ? (float)q[base + j] : 0.f;
#pragma unroll
        for (int k = 0; k < P; ++k) s2[k][j] = L[k] * qj;
      } else {
#pragma unroll
        for (int k = 0; k < P; ++k) s3[k][j] = L[k];
      }
    }
    __syncthreads();
    // W[u][j], the Khatri-Rao operand, walked in storage order (consecutive
    // threads write consecutive words: idx == kmaj(u, j, kUpKG))
    constexpr int kRowGroups = (P2 + 7) / 8;
    for (int idx = tid; idx < kRowGroups * 32 * kUpKG; idx += kTcThreads) {
      const int u = (idx / (32 * kUpKG)) * 8 + ((idx >> 2) & 7);
      const int j = ((idx >> 5) % kUpKG) * 4 + (idx & 3);
      if (u < P2) {
        const float w = s2[u / P][j] * s3[u % P][j];
        const float h = to_tf32(w);
        sAh[idx] = h;
        sAl[idx] = to_tf32(w - h);
      }
    }
    fence_smem_async();
    fence_before();
    __syncthreads();
    fence_after();
    if (tid == 0) {
      const uint32_t ah = smem_u32(sAh), al = smem_u32(sAl), bh = smem_u32(sBh), bl = smem_u32(sBl);
      const uint32_t sbo = kUpKG * 128;
      const bool restart = ci % kUpGroup == 0;
#pragma unroll
      for (int s = 0; s < kUpKC / 8; ++s) {
        const uint32_t o = s * 256;             // two core matrices along K per step
        // the small products first, the large one last
        mma_tf32(tmem, smem_desc(al + o, 128, sbo), smem_desc(bl + o, 128, sbo), kIdesc,
                 (restart && s == 0) ? 0u : 1u);
        mma_tf32(tmem, smem_desc(ah + o, 128, sbo), smem_desc(bl + o, 128, sbo), kIdesc, 1u);
        mma_tf32(tmem, smem_desc(al + o, 128, sbo), smem_desc(bh + o, 128, sbo), kIdesc, 1u);
        mma_tf32(tmem, smem_desc(ah + o, 128, sbo), smem_desc(bh + o, 128, sbo), kIdesc, 1u);
      }
      mma_commit(&bar);
    }
    const bool done = wait_phase(&bar, phase);
    phase ^= 1u;                          // the phase of the next commit
    ok = __syncthreads_and(done);
    fence_after();
    if (ok && (ci % kUpGroup == kUpGroup - 1 || base + kUpKC >= e)) {   // fold the group
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16), v);
      if (tid < P2) {
#pragma unroll
        for (int k = 0; k < P; ++k) {
          const float t = __fadd_rn(hi[k], v[k]);
          lo[k] = __fadd_rn(lo[k], two_sum_err(hi[k], v[k], t));
          hi[k] = t;
        }
      }
    }
    fence_before();
  }
  if (!ok) {
    if (tid == 0) atomicExch(err, kDevErrTimeout);
    wait_phase(&bar, phase ^ 1u);       // let the MMAs in flight finish (bounded) before freeing
  } else if (tid < P2) {
#pragma unroll
    for (int k = 0; k < P; ++k) qhat[(int64_t)c * NP + k * P2 + tid] = (double)hi[k] + (double)lo[k];
  }
  __syncthreads();
  fence_after();
  if (warp == 0) tmem_free<32>(tmem);
}

// ---------------------------------------------------------------------------
// Downward leaf contraction, Eq. (21)
// ---------------------------------------------------------------------------
constexpr int kDownKD = 16;                 // K = P padded to 16 (two K steps of 8)
constexpr int kDownKG = kDownKD / 4;
constexpr int kDownTcSplit = 2;             // CTAs per leaf (tiles interleaved)
// Dynamic shared memory reserved so that CTAs whose accumulators take 128
// (64) columns share an SM at most 4 (8) at a time: they then fit the SM's 512
// columns of tensor memory and no CTA waits in its allocation.
constexpr int kDownTcPadSmem = 24 * 1024;

template <int P>
__global__ void __launch_bounds__(kTcThreads) k_down_leaf_tc(
    const int32_t* __restrict__ leaf_ids, const int32_t* __restrict__ begin,
    const int32_t* __restrict__ end, const double* __restrict__ x, const double* __restrict__ y,
    const double* __restrict__ z, const int32_t* __restrict__ perm, const double* __restrict__ nodes,
    const double* __restrict__ phit, const double* __restrict__ phi_near,
    double* __restrict__ phi_user, int* __restrict__ err) {
  constexpr int P2 = P * P, NP = P2 * P;
  constexpr int NB = (P2 + 15) / 16 * 16;   // MMA N
  constexpr int NCOLS = NB <= 32 ? 32 : (NB <= 64 ? 64 : 128);
  static_assert(P <= kDownKD && NB <= 128, "grid too large for one 128-column accumulator");
  constexpr uint32_t kIdesc = idesc_tf32(128, NB);
  __shared__ __align__(1024) float sAh[128 * kDownKD], sAl[128 * kDownKD];
  __shared__ __align__(1024) float sBh[NB * kDownKD], sBl[NB * kDownKD];
  __shared__ float shl[3][2 * kMaxP];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int c = leaf_ids[blockIdx.x];
  const int32_t b = begin[c], e = end[c];
  for (int i = tid; i < 128 * kDownKD; i += kTcThreads) sAh[i] = sAl[i] = 0.f;
  // B[u][k1] = phi_t[k1][u] (zero padding for u >= P^2, k1 >= P), split once per leaf
  for (int i = tid; i < NB * kDownKD; i += kTcThreads) {
    const int u = i / kDownKD, k = i % kDownKD;
    const float v = (u < P2 && k < P) ? (float)phit[(int64_t)c * NP + k * P2 + u] : 0.f;
    const float h = to_tf32(v);
    sBh[kmaj(u, k, kDownKG)] = h;
    sBl[kmaj(u, k, kDownKG)] = to_tf32(v - h);
  }
  if (tid < 3 * P) {
    float h, l;
    split_f64(nodes[(int64_t)c * 3 * P + tid], h, l);
    shl[tid / P][tid % P] = h;
    shl[tid / P][kMaxP + tid % P] = l;
  }
  if (tid == 0) mbar_init1(&bar);
  if (warp == 0) tmem_alloc<NCOLS>(&tmem_slot);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t row_addr = tmem + ((uint32_t)(warp * 32) << 16);
  uint32_t phase = 0;
  bool ok = true;
  for (int32_t base = b + blockIdx.y * 128; base < e && ok; base += kDownTcSplit * 128) {
    const int32_t i = base + tid;
    const bool valid = i < e;
    float L1[P], L2[P], L3[P];
    if (valid) {
      basis_f32_fixed<P>(x[i], shl[0], L1);
      basis_f32_fixed<P>(y[i], shl[1], L2);
      basis_f32_fixed<P>(z[i], shl[2], L3);
    } else {
#pragma unroll
      for (int k = 0; k < P; ++k) L1[k] = L2[k] = L3[k] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < P; ++k) {
      const float h = to_tf32(L1[k]);
      sAh[kmaj(tid, k, kDownKG)] = h;
      sAl[kmaj(tid, k, kDownKG)] = to_tf32(L1[k] - h);
    }
    fence_smem_async();
    fence_before();
    __syncthreads();
    fence_after();
    if (tid == 0) {
      const uint32_t ah = smem_u32(sAh), al = smem_u32(sAl), bh = smem_u32(sBh), bl = smem_u32(sBl);
      const uint32_t sbo = kDownKG * 128;
#pragma unroll
      for (int s = 0; s < kDownKD / 8; ++s) {
        const uint32_t o = s * 256;
        // the small products first, the large one last (less rounding of the small terms)
        mma_tf32(tmem, smem_desc(al + o, 128, sbo), smem_desc(bl + o, 128, sbo), kIdesc, s > 0 ? 1u : 0u);
        mma_tf32(tmem, smem_desc(ah + o, 128, sbo), smem_desc(bl + o, 128, sbo), kIdesc, 1u);
        mma_tf32(tmem, smem_desc(al + o, 128, sbo), smem_desc(bh + o, 128, sbo), kIdesc, 1u);
        mma_tf32(tmem, smem_desc(ah + o, 128, sbo), smem_desc(bh + o, 128, sbo), kIdesc, 1u);
      }
      mma_commit(&bar);
    }
    const bool done = wait_phase(&bar, phase);
    phase ^= 1u;                          // the phase of the next commit
    ok = __syncthreads_and(done);
    fence_after();
    if (!ok) break;
    // phi(x_i) = sum_k2 L2[k2] (sum_k3 L3[k3] T[k2 P + k3]); the k2 sum compensated
    CompSum a;
    float s2 = 0.f;
#pragma unroll
    for (int c0 = 0; c0 < NB; c0 += 16) {
      float v[16];
      tmem_ld16(row_addr + (uint32_t)c0, v);
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        const int u = c0 + jj;
        if (u < P2) {
          s2 = fmaf(L3[u % P], v[jj], s2);
          if (u % P == P - 1) {
            a.add_prod(L2[u / P], s2);
            s2 = 0.f;
          }
        }
      }
    }
    if (valid) phi_user[perm[i]] = phi_near[i] + ((double)a.s + (double)a.c);
    fence_before();
  }
  if (!ok) {
    if (tid == 0) atomicExch(err, kDevErrTimeout);
    wait_phase(&bar, phase ^ 1u);       // the commit that timed out, bounded again
  }
  __syncthreads();
  fence_after();
  if (warp == 0) tmem_free<NCOLS>(tmem);
}

}  // namespace

// Grids the tensor-core leaf kernels take: P^2 <= 121 (one accumulator).
bool leaf_tc_supported(int P) { return P >= 2 && P <= 11; }

int configure_tc_kernels() {
#define BL_TC_ATTR(PP)                                                                         \
  BL_CUDA(cudaFuncSetAttribute(k_down_leaf_tc<PP>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                               kDownTcPadSmem));
  BL_TC_ATTR(2) BL_TC_ATTR(3) BL_TC_ATTR(4) BL_TC_ATTR(5) BL_TC_ATTR(6)
  BL_TC_ATTR(7) BL_TC_ATTR(8) BL_TC_ATTR(9) BL_TC_ATTR(10) BL_TC_ATTR(11)
#undef BL_TC_ATTR
  return BLDTT_OK;
}

int up_leaf_tc(bldtt_plan* p, cudaStream_t s) {
  const Tree& T = p->st;
  if (T.nleaves == 0) return BLDTT_OK;
  switch (p->P) {
#define BL_UP_TC(PP)                                                                              \
  case PP:                                                                                        \
    k_up_leaf_tc<PP><<<T.nleaves, kTcThreads, 0, s>>>(T.leaf_ids, T.begin, T.end, T.x, T.y, T.z,  \
                                                      p->q_tree, T.nodes, p->qhat, p->dev_err);   \
    break;
    BL_UP_TC(2) BL_UP_TC(3) BL_UP_TC(4) BL_UP_TC(5) BL_UP_TC(6)
    BL_UP_TC(7) BL_UP_TC(8) BL_UP_TC(9) BL_UP_TC(10) BL_UP_TC(11)
#undef BL_UP_TC
    default:
      set_error("tensor-core upward leaf pass: grid of %d points not supported", p->P);
      return BLDTT_EINVAL;
  }
  BL_LAUNCHED(p->compute_counter.launches);
  return BLDTT_OK;
}

int down_leaf_tc(bldtt_plan* p, const int32_t* leaf_ids, int32_t nleaves, double* phi_user,
                 cudaStream_t s) {
  const Tree& T = p->tt;
  if (nleaves <= 0) return BLDTT_OK;
  const dim3 grid(nleaves, kDownTcSplit);
  switch (p->P) {
#define BL_DOWN_TC(PP)                                                                            \
  case PP:                                                                                        \
    k_down_leaf_tc<PP><<<grid, kTcThreads, kDownTcPadSmem, s>>>(leaf_ids, T.begin, T.end, T.x, T.y, \
                                                                T.z, T.perm, T.nodes, p->phit,     \
                                                                p->phi_near, phi_user, p->dev_err); \
    break;
    BL_DOWN_TC(2) BL_DOWN_TC(3) BL_DOWN_TC(4) BL_DOWN_TC(5) BL_DOWN_TC(6)
    BL_DOWN_TC(7) BL_DOWN_TC(8) BL_DOWN_TC(9) BL_DOWN_TC(10) BL_DOWN_TC(11)
#undef BL_DOWN_TC
    default:
      set_error("tensor-core downward leaf pass: grid of %d points not supported", p->P);
      return BLDTT_EINVAL;
  }
  BL_LAUNCHED(p->compute_counter.launches);
  return BLDTT_OK;
}

}  // namespace bldtt
