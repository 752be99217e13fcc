// Dual tree traversal (Sec. 2.6, Algorithm 2) as a breadth-first pair
// frontier, the four interaction lists of every target cluster (Sec. 3.1),
// and the work items the interaction kernel drains.
//
// One pass classifies every (C_t, C_s) pair of the frontier: well separated
// pairs (r_t + r_s < theta R) become a CC, CP, PC or PP list entry according
// to |C_t|, |C_s| versus n_p; non-separated leaf pairs become PP entries; the
// rest are replaced by the pairs of the split side's children (Alg. 2,
// lines 11-17).  Compaction uses prefix sums, so the entry order, and hence
// every later summation order, is deterministic.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace bldtt {

struct TreeView {
  const int32_t *begin, *end, *nchild, *first_child;
  const double *center, *radius;
};

static TreeView view(const Tree& T) {
  return TreeView{T.begin, T.end, T.nchild, T.first_child, T.center, T.radius};
}

// Action of a frontier pair: an entry of list class 0..kMaxClasses-1, or a split.
constexpr int8_t kActSplitT = 100, kActSplitS = 101;

// Alg. 2's decision for the pair (t, s): an entry of list class 0..kMaxClasses-1
// or a split (kActSplitT / kActSplitS, with the number of child pairs in
// *kids).  ch is the learned selector's decision for the pair, or
// kChoiceFallback for the MAC at the highest degree (index imax).
__device__ __forceinline__ int8_t classify_pair(int t, int s, const TreeView& tt, const TreeView& st,
                                                int64_t np, int imax, double theta, int variant,
                                                int16_t ch, int32_t* kids) {
  const int64_t cnt_t = tt.end[t] - tt.begin[t], cnt_s = st.end[s] - st.begin[s];
  int8_t a = -1;
  *kids = 0;
  if (ch >= 0) {
    a = (int8_t)ch;
  } else if (ch == kChoiceFallback) {
    const double* ct = tt.center + (int64_t)t * 3;
    const double* cs = st.center + (int64_t)s * 3;
    double dx = __dsub_rn(ct[0], cs[0]), dy = __dsub_rn(ct[1], cs[1]), dz = __dsub_rn(ct[2], cs[2]);
    double R = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
    bool sep = __dadd_rn(tt.radius[t], st.radius[s]) < __dmul_rn(theta, R);
    if (sep) {
      bool big_t = cnt_t > np, big_s = cnt_s > np;
      int type = big_t ? (big_s ? BLDTT_CC : BLDTT_CP) : (big_s ? BLDTT_PC : BLDTT_PP);
      if (variant == BLDTT_VARIANT_CC_PP_ONLY && type != BLDTT_CC) type = BLDTT_PP;   // Sec. 4.3 ablation
      a = (int8_t)class_of(type, imax);
    }
  }
  if (a < 0) {
    bool leaf_t = tt.nchild[t] == 0, leaf_s = st.nchild[s] == 0;
    if (leaf_t && leaf_s) a = 0;   // PP
    else if (leaf_s) a = kActSplitT;
    else if (leaf_t) a = kActSplitS;
    else a = cnt_s < cnt_t ? kActSplitT : kActSplitS;
    if (a == kActSplitT) *kids = tt.nchild[t];
    if (a == kActSplitS) *kids = st.nchild[s];
  }
  return a;
}

// choice (may be NULL): the learned selector's decision per pair; NULL or
// kChoiceFallback applies Alg. 2's MAC at the highest degree (index imax).
__global__ void k_dtt_classify(const int2* __restrict__ pairs, int32_t F, TreeView tt, TreeView st,
                               int64_t np, int imax, double theta, int variant,
                               const int16_t* __restrict__ choice, int32_t* __restrict__ nkids,
                               int32_t* __restrict__ isentry, int8_t* __restrict__ action) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= F) return;
  int32_t kids = 0;
  const int8_t a = classify_pair(pairs[i].x, pairs[i].y, tt, st, np, imax, theta, variant,
                                 choice ? choice[i] : kChoiceFallback, &kids);
  action[i] = a;
  nkids[i] = kids;
  isentry[i] = a < kActSplitT ? 1 : 0;
}

__global__ void k_dtt_emit(const int2* __restrict__ pairs, int32_t F, const int8_t* __restrict__ action,
                           const int32_t* __restrict__ koff, const int32_t* __restrict__ eoff,
                           TreeView tt, TreeView st, int2* __restrict__ next, int32_t* __restrict__ ent_t,
                           int32_t* __restrict__ ent_s, uint32_t* __restrict__ ent_key, int64_t ebase,
                           int32_t nct) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= F) return;
  int t = pairs[i].x, s = pairs[i].y;
  int8_t a = action[i];
  if (a < kActSplitT) {
    int64_t e = ebase + eoff[i];
    ent_t[e] = t;
    ent_s[e] = s;
    ent_key[e] = (uint32_t)a * (uint32_t)nct + (uint32_t)t;
  } else if (a == kActSplitT) {
    int32_t fc = tt.first_child[t], k = tt.nchild[t];
    for (int j = 0; j < k; ++j) next[koff[i] + j] = make_int2(fc + j, s);
  } else {
    int32_t fc = st.first_child[s], k = st.nchild[s];
    for (int j = 0; j < k; ++j) next[koff[i] + j] = make_int2(t, fc + j);
  }
}

// ---------------------------------------------------------------------------
// The whole fixed-rule traversal in one cooperative launch
// ---------------------------------------------------------------------------
// Every level of the frontier loop above in one kernel, with no host round
// trip between levels: each block takes a contiguous range of the frontier,
// classifies its pairs and scans their child and entry counts; after a grid
// barrier every block reads all blocks' totals (so every block knows its
// offsets and the level's totals), checks the buffer capacities (the same
// decision in every block), emits its entries and child pairs at those
// offsets, and a second barrier ends the level.  Ranges and offsets follow the
// frontier order, so entries and next frontiers are exactly those of the
// level-by-level loop.  Data written by other blocks is read with L2 loads
// (ld.global.cg).  Barriers wait at most kDttWaitNs, then report and return.
constexpr int kDttThreads = 256;
constexpr uint64_t kDttWaitNs = 5ull * 1000ull * 1000ull * 1000ull;

struct DttGrid {
  unsigned int count;   // blocks arrived at the current barrier
  unsigned int gen;     // barrier generation
  int32_t F0;           // size of the first frontier (set by the host)
  int32_t status;       // 0 done, 1 a buffer would overflow, 2 a barrier gave up
  long long E;          // entries written
  int32_t levels;
};

__device__ __forceinline__ uint64_t dtt_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded grid barrier of the cooperative launch (all blocks co-resident).
__device__ bool dtt_grid_sync(DttGrid* g, unsigned nblocks) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* vgen = &g->gen;
    const unsigned gen0 = *vgen;
    __threadfence();
    if (atomicAdd(&g->count, 1u) == nblocks - 1u) {
      atomicExch(&g->count, 0u);
      __threadfence();
      atomicAdd(&g->gen, 1u);
    } else {
      const uint64_t t0 = dtt_ns();
      while (*vgen == gen0) {
        if (dtt_ns() - t0 > kDttWaitNs) {
          ok = 0;
          atomicExch(&g->status, 2);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Block-wide exclusive scan of two counts; totals in *tk, *te.
__device__ __forceinline__ void block_scan2(int32_t k, int32_t e, int32_t* xk, int32_t* xe, int32_t* tk,
                                            int32_t* te) {
  __shared__ int32_t wk[kDttThreads / 32], we[kDttThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t ik = k, ie = e;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t a = __shfl_up_sync(0xffffffffu, ik, o), c = __shfl_up_sync(0xffffffffu, ie, o);
    if (lane >= o) {
      ik += a;
      ie += c;
    }
  }
  if (lane == 31) {
    wk[warp] = ik;
    we[warp] = ie;
  }
  __syncthreads();
  int32_t pk = 0, pe = 0, sk = 0, se = 0;
  for (int w = 0; w < kDttThreads / 32; ++w) {
    if (w < warp) {
      pk += wk[w];
      pe += we[w];
    }
    sk += wk[w];
    se += we[w];
  }
  *xk = pk + ik - k;
  *xe = pe + ie - e;
  *tk = sk;
  *te = se;
  __syncthreads();
}

__global__ void __launch_bounds__(kDttThreads) k_dtt_all(
    TreeView tt, TreeView st, int64_t np, int imax, double theta, int variant, int32_t nct,
    int2* __restrict__ buf0, int2* __restrict__ buf1, int32_t fcap, int32_t* __restrict__ ent_t,
    int32_t* __restrict__ ent_s, uint32_t* __restrict__ ent_key, int64_t ecap,
    int32_t* __restrict__ koff, int32_t* __restrict__ eoff, int8_t* __restrict__ action,
    int2* __restrict__ part, DttGrid* __restrict__ g) {
  __shared__ int32_t red[4][kDttThreads / 32];
  const unsigned G = gridDim.x, b = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int2* front = buf0;
  int2* next = buf1;
  int32_t F = g->F0;
  int64_t E = 0;
  int level = 0;
  for (; F > 0; ++level) {
    const int32_t lo = (int32_t)((int64_t)F * b / G), hi = (int32_t)((int64_t)F * (b + 1) / G);
    int32_t run_k = 0, run_e = 0;
    for (int32_t base = lo; base < hi; base += kDttThreads) {   // block-uniform trip count
      const int32_t i = base + threadIdx.x;
      int32_t kids = 0, ent = 0;
      if (i < hi) {
        const int2 pr = __ldcg(front + i);
        const int8_t a = classify_pair(pr.x, pr.y, tt, st, np, imax, theta, variant, kChoiceFallback, &kids);
        action[i] = a;
        ent = a < kActSplitT ? 1 : 0;
      }
      int32_t xk, xe, tk, te;
      block_scan2(kids, ent, &xk, &xe, &tk, &te);
      if (i < hi) {
        koff[i] = run_k + xk;
        eoff[i] = run_e + xe;
      }
      run_k += tk;
      run_e += te;
    }
    if (threadIdx.x == 0) part[b] = make_int2(run_k, run_e);
    if (!dtt_grid_sync(g, G)) return;
    // this block's offsets and the level's totals, from every block's counts
    int32_t pk = 0, pe = 0, sk = 0, se = 0;
    for (unsigned j = threadIdx.x; j < G; j += kDttThreads) {
      const int2 v = __ldcg(part + j);
      if (j < b) {
        pk += v.x;
        pe += v.y;
      }
      sk += v.x;
      se += v.y;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      pk += __shfl_xor_sync(0xffffffffu, pk, o);
      pe += __shfl_xor_sync(0xffffffffu, pe, o);
      sk += __shfl_xor_sync(0xffffffffu, sk, o);
      se += __shfl_xor_sync(0xffffffffu, se, o);
    }
    if (lane == 0) {
      red[0][warp] = pk;
      red[1][warp] = pe;
      red[2][warp] = sk;
      red[3][warp] = se;
    }
    __syncthreads();
    int32_t off_k = 0, off_e = 0, K = 0, En = 0;
    for (int w = 0; w < kDttThreads / 32; ++w) {
      off_k += red[0][w];
      off_e += red[1][w];
      K += red[2][w];
      En += red[3][w];
    }
    __syncthreads();
    if (K > fcap || E + En > ecap) {          // the same decision in every block
      if (b == 0 && threadIdx.x == 0) atomicExch(&g->status, 1);
      return;
    }
    for (int32_t i = lo + threadIdx.x; i < hi; i += kDttThreads) {
      const int2 pr = __ldcg(front + i);
      const int8_t a = action[i];
      if (a < kActSplitT) {
        const int64_t e = E + off_e + eoff[i];
        ent_t[e] = pr.x;
        ent_s[e] = pr.y;
        ent_key[e] = (uint32_t)a * (uint32_t)nct + (uint32_t)pr.x;
      } else if (a == kActSplitT) {
        const int32_t fc = tt.first_child[pr.x], k = tt.nchild[pr.x], o = off_k + koff[i];
        for (int j = 0; j < k; ++j) next[o + j] = make_int2(fc + j, pr.y);
      } else {
        const int32_t fc = st.first_child[pr.y], k = st.nchild[pr.y], o = off_k + koff[i];
        for (int j = 0; j < k; ++j) next[o + j] = make_int2(pr.x, fc + j);
      }
    }
    if (!dtt_grid_sync(g, G)) return;
    int2* tmp = front;
    front = next;
    next = tmp;
    E += En;
    F = K;
  }
  if (b == 0 && threadIdx.x == 0) {
    g->E = E;
    g->levels = level;
  }
}

// Root pair (r, r) of every problem r.
__global__ void k_root_pairs(int2* __restrict__ front, int32_t P) {
  const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < P) front[r] = make_int2(r, r);
}

__global__ void k_iota(int32_t* v, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = (int32_t)i;
}

__global__ void k_gather_i32(const int32_t* __restrict__ src, const int32_t* __restrict__ idx,
                             int32_t* __restrict__ dst, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[idx[i]];
}

__global__ void k_key_hist(const uint32_t* __restrict__ keys, int64_t n, int32_t* __restrict__ cnt) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(&cnt[keys[i]], 1);
}

// Kernel evaluations per list class (Eqs. (6), (8), (12), (15)); integer sums,
// exact.  Each CTA sums its entries per class in shared memory first, so the
// global counters see one atomic per class and CTA.
__global__ void k_count_evals(const int32_t* __restrict__ et, const int32_t* __restrict__ es,
                              const uint32_t* __restrict__ key, int64_t n, int32_t nct,
                              TreeView tt, TreeView st, DegreeSet deg,
                              unsigned long long* __restrict__ out) {
  __shared__ unsigned long long part[kMaxClasses];
  if (threadIdx.x < kMaxClasses) part[threadIdx.x] = 0ull;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const int c = (int)(key[i] / (uint32_t)nct);
    const int type = class_type(c);
    const int64_t np = deg.np[class_degree(c)];
    int64_t ct = tt.end[et[i]] - tt.begin[et[i]], cs = st.end[es[i]] - st.begin[es[i]];
    int64_t v = type == BLDTT_PP ? ct * cs : type == BLDTT_PC ? ct * np : type == BLDTT_CP ? np * cs : np * np;
    atomicAdd(&part[c], (unsigned long long)v);
  }
  __syncthreads();
  if (threadIdx.x < kMaxClasses && part[threadIdx.x]) atomicAdd(&out[threadIdx.x], part[threadIdx.x]);
}

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Offsets list_ptr[k * nct], k = 0..nclass, written as int32 after the
// kMaxClasses evaluation counters of `out`.
__global__ void k_class_bounds(const int32_t* __restrict__ list_ptr, int32_t nct, int nclass,
                               unsigned long long* __restrict__ out) {
  int32_t* o = reinterpret_cast<int32_t*>(out + kMaxClasses);
  for (int k = threadIdx.x; k <= nclass; k += blockDim.x) o[k] = list_ptr[(int64_t)k * nct];
}

// The fixed-rule traversal from the P root pairs in `roots` by one cooperative
// launch (k_dtt_all).  On success *E receives the entry count, the three entry
// arrays are allocated here and *done is set; when a buffer would overflow the
// capacity is doubled and the launch repeated (twice at most), after which
// *done stays false and the caller runs the level-by-level loop.
static int traverse_cooperative(bldtt_plan* p, const TreeView& tt, const TreeView& st, const int2* roots,
                                int32_t P, int32_t** ent_t, int32_t** ent_s, uint32_t** ent_key,
                                int64_t* E, bool* done, cudaStream_t s) {
  *done = false;
  if (cooperative_set_up_disabled()) return BLDTT_OK;
  int dev = 0, sms = 0, coop = 0, per_sm = 0;
  BL_CUDA(cudaGetDevice(&dev));
  BL_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return BLDTT_OK;
  BL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  BL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dtt_all, kDttThreads, 0));
  if (per_sm < 1) return BLDTT_OK;
  const unsigned G = (unsigned)(sms * (per_sm < 2 ? per_sm : 2));
  const int32_t imax = p->deg.n - 1;
  int64_t cap = 64 * ((int64_t)p->tt.nclusters + (int64_t)p->st.nclusters);
  if (cap < 32768) cap = 32768;
  if (const char* e = std::getenv("BLDTT_TRAVERSAL_CAPACITY"))   // a smaller start exercises the relaunches
    cap = std::max<int64_t>(std::strtoll(e, nullptr, 10), (int64_t)P);
  for (int attempt = 0; attempt < 3 && !*done; ++attempt, cap *= 2) {
    if (cap >= (int64_t)INT32_MAX) break;
    int2 *b0 = nullptr, *b1 = nullptr, *part = nullptr;
    int32_t *koff = nullptr, *eoff = nullptr, *et = nullptr, *es = nullptr;
    uint32_t* ek = nullptr;
    int8_t* act = nullptr;
    DttGrid* g = nullptr;
    Arena scratch;
    scratch.add(&b0, cap);
    scratch.add(&b1, cap);
    scratch.add(&koff, cap);
    scratch.add(&eoff, cap);
    scratch.add(&act, cap);
    scratch.add(&part, G);
    scratch.add(&g, 1);
    BL_TRY(scratch.alloc(s));
    BL_TRY(dalloc_n(&et, cap, s));
    BL_TRY(dalloc_n(&es, cap, s));
    BL_TRY(dalloc_n(&ek, cap, s));
    BL_CUDA(cudaMemsetAsync(g, 0, sizeof(DttGrid), s));
    BL_CUDA(cudaMemcpyAsync(b0, roots, (size_t)P * sizeof(int2), cudaMemcpyDeviceToDevice, s));
    BL_CUDA(cudaMemcpyAsync(&g->F0, &P, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    int64_t np = p->deg.np[imax];
    double theta = p->theta;
    int variant = p->variant;
    int32_t nct = p->tt.nclusters;
    int32_t fcap = (int32_t)cap;
    int64_t ecap = cap;
    TreeView a = tt, c = st;
    int imx = imax;
    void* args[] = {&a, &c, &np, &imx, &theta, &variant, &nct, &b0, &b1, &fcap, &et, &es, &ek, &ecap,
                    &koff, &eoff, &act, &part, &g};
    DttGrid h{};
    {
      std::lock_guard<std::mutex> lock(cooperative_launch_mutex());
      BL_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(&k_dtt_all), dim3(G),
                                          dim3(kDttThreads), args, 0, s));
      BL_LAUNCHED(p->setup_counter.launches);
      BL_TRY(read_device(g, &h, sizeof(h), s));
    }
    scratch.release(s);
    if (h.status == 2) {
      dfree(et, s); dfree(es, s); dfree(ek, s);
      set_error("a grid barrier of the cooperative traversal gave up after %llu ns",
                (unsigned long long)kDttWaitNs);
      return BLDTT_ETIMEOUT;
    }
    if (h.status == 0) {
      *ent_t = et;
      *ent_s = es;
      *ent_key = ek;
      *E = h.E;
      *done = true;
    } else {
      dfree(et, s); dfree(es, s); dfree(ek, s);
    }
  }
  return BLDTT_OK;
}

int build_lists(bldtt_plan* p, cudaStream_t s) {
  bldtt::Counters& cnt = p->setup_counter;
  const TreeView tt = view(p->tt), st = view(p->st);
  const int32_t nct = p->tt.nclusters;
  size_t fcap = 1024, ncap = 1024, ecap = 4096;
  int2 *front = nullptr, *next = nullptr;
  int32_t *ent_t = nullptr, *ent_s = nullptr;
  uint32_t* ent_key = nullptr;
  // One root pair per problem (Alg. 2 starts from the two roots of each problem).
  const int32_t P = p->tt.nroots;
  fcap = std::max(fcap, (size_t)P);
  BL_TRY(dalloc_n(&front, fcap, s));
  k_root_pairs<<<nblk(P, 256), 256, 0, s>>>(front, P);
  BL_LAUNCHED(cnt.launches);
  int32_t F = P;
  int64_t E = 0;
  const int imax = p->deg.n - 1;
  // The fixed rule runs as one cooperative launch; the learned selector (a
  // network inference per frontier level) and an overflowing estimate of the
  // buffers take the level-by-level loop below.
  if (!p->learned) {
    bool done = false;
    int32_t *ct = nullptr, *cs = nullptr;
    uint32_t* ck = nullptr;
    BL_TRY(traverse_cooperative(p, tt, st, front, P, &ct, &cs, &ck, &E, &done, s));
    if (done) {
      ent_t = ct;
      ent_s = cs;
      ent_key = ck;
      F = 0;                                   // the loop below has nothing left to do
    }
  }
  if (F > 0) {   // the level-by-level loop's buffers
    BL_TRY(dalloc_n(&next, ncap, s));
    BL_TRY(dalloc_n(&ent_t, ecap, s));
    BL_TRY(dalloc_n(&ent_s, ecap, s));
    BL_TRY(dalloc_n(&ent_key, ecap, s));
  }
  // per-level scratch, grown as the front grows; the two totals of a level
  // come back to the host in one read
  size_t cap_k = 0, cap_i = 0, cap_o = 0, cap_e = 0, cap_a = 0, cap_c = 0;
  int32_t *nkids = nullptr, *isentry = nullptr, *koff = nullptr, *eoff = nullptr, *tot2 = nullptr;
  int8_t* action = nullptr;
  int16_t* choice = nullptr;
  if (F > 0) BL_TRY(dalloc_n(&tot2, 2, s));
  while (F > 0) {
    BL_TRY(dgrow(&nkids, &cap_k, (size_t)F, 0, s));
    BL_TRY(dgrow(&isentry, &cap_i, (size_t)F, 0, s));
    BL_TRY(dgrow(&koff, &cap_o, (size_t)F, 0, s));
    BL_TRY(dgrow(&eoff, &cap_e, (size_t)F, 0, s));
    BL_TRY(dgrow(&action, &cap_a, (size_t)F, 0, s));
    if (p->learned) {
      BL_TRY(dgrow(&choice, &cap_c, (size_t)F, 0, s));
      BL_TRY(select_pairs(p, front, F, choice, s));
    }
    k_dtt_classify<<<nblk(F, 256), 256, 0, s>>>(front, F, tt, st, p->deg.np[imax], imax, p->theta,
                                                p->variant, p->learned ? choice : nullptr, nkids,
                                                isentry, action);
    BL_LAUNCHED(cnt.launches);
    BL_TRY(scan_exclusive_dev(nkids, koff, F, tot2, s, cnt));
    BL_TRY(scan_exclusive_dev(isentry, eoff, F, tot2 + 1, s, cnt));
    int32_t h2[2];
    BL_TRY(read_device(tot2, h2, sizeof(h2), s));
    const int32_t K = h2[0], En = h2[1];
    if ((size_t)K > ncap) {
      size_t c = ncap;
      BL_TRY(dgrow(&next, &c, (size_t)K, 0, s));
      ncap = c;
    }
    if ((size_t)(E + En) > ecap) {
      size_t c1 = ecap, c2 = ecap, c3 = ecap;
      BL_TRY(dgrow(&ent_t, &c1, (size_t)(E + En), (size_t)E, s));
      BL_TRY(dgrow(&ent_s, &c2, (size_t)(E + En), (size_t)E, s));
      int32_t* kk = reinterpret_cast<int32_t*>(ent_key);
      BL_TRY(dgrow(&kk, &c3, (size_t)(E + En), (size_t)E, s));
      ent_key = reinterpret_cast<uint32_t*>(kk);
      ecap = c1;
    }
    k_dtt_emit<<<nblk(F, 256), 256, 0, s>>>(front, F, action, koff, eoff, tt, st, next, ent_t, ent_s,
                                            ent_key, E, nct);
    BL_LAUNCHED(cnt.launches);
    E += En;
    int2* tmp = front; front = next; next = tmp;
    size_t tc = fcap; fcap = ncap; ncap = tc;
    F = K;
  }
  dfree(nkids, s); dfree(isentry, s); dfree(koff, s); dfree(eoff, s); dfree(tot2, s);
  dfree(action, s); dfree(choice, s);
  dfree(front, s);
  dfree(next, s);

  // Sort entries by (type, target cluster); the traversal order breaks ties.
  p->nentries = E;
  const int nclass = p->nclass;
  int key_bits = 1;
  while ((1ull << key_bits) < (unsigned long long)nclass * (unsigned long long)nct) ++key_bits;
  int32_t* order = nullptr;
  BL_TRY(dalloc_n(&order, E, s));
  if (E > 0) {
    k_iota<<<nblk(E, 256), 256, 0, s>>>(order, E);
    BL_LAUNCHED(cnt.launches);
  }
  BL_TRY(radix_sort_pairs(ent_key, order, E, key_bits, s, cnt));
  BL_TRY(dalloc_n(&p->list_src, E, s));
  BL_TRY(dalloc_n(&p->list_tgt, E, s));
  if (E > 0) {
    k_gather_i32<<<nblk(E, 256), 256, 0, s>>>(ent_s, order, p->list_src, E);
    BL_LAUNCHED(cnt.launches);
    k_gather_i32<<<nblk(E, 256), 256, 0, s>>>(ent_t, order, p->list_tgt, E);
    BL_LAUNCHED(cnt.launches);
  }
  int64_t nkeys = (int64_t)nclass * nct;
  int32_t* hist = nullptr;
  BL_TRY(dalloc_n(&hist, nkeys, s));
  BL_TRY(dalloc_n(&p->list_ptr, nkeys + 1, s));
  BL_CUDA(cudaMemsetAsync(hist, 0, nkeys * sizeof(int32_t), s));
  if (E > 0) {
    k_key_hist<<<nblk(E, 256), 256, 0, s>>>(ent_key, E, hist);
    BL_LAUNCHED(cnt.launches);
  }
  BL_TRY(scan_exclusive_dev(hist, p->list_ptr, nkeys, p->list_ptr + nkeys, s, cnt));   // total last

  // evals: kMaxClasses counters, then room for the nclass + 1 class offsets
  constexpr int kRead = kMaxClasses + (kMaxClasses + 2) / 2;
  unsigned long long* evals = nullptr;
  BL_TRY(dalloc_n(&evals, kRead, s));
  BL_CUDA(cudaMemsetAsync(evals, 0, kRead * sizeof(unsigned long long), s));
  if (E > 0) {
    k_count_evals<<<nblk(E, 256), 256, 0, s>>>(p->list_tgt, p->list_src, ent_key, E, nct, tt, st,
                                               p->deg, evals);
    BL_LAUNCHED(cnt.launches);
  }
  // class boundaries of the CSR and the evaluation counts, in one read
  unsigned long long h_read[kMaxClasses + (kMaxClasses + 2) / 2];
  k_class_bounds<<<1, 32, 0, s>>>(p->list_ptr, nct, nclass, evals);
  BL_LAUNCHED(cnt.launches);
  BL_TRY(read_device(evals, h_read, sizeof(h_read), s));
  const unsigned long long* h_evals = h_read;
  const int32_t* h_ptr = reinterpret_cast<const int32_t*>(h_read + kMaxClasses);
  p->class_count.assign(nclass, 0);
  p->class_evals.assign(nclass, 0.0);
  for (int k = 0; k < 4; ++k) {
    p->list_count[k] = 0;
    p->interactions[k] = 0.0;
  }
  for (int i = 0; i < kMaxDegrees; ++i) p->deg_used[i] = i == p->deg.n - 1;   // the highest always
  for (int c = 0; c < nclass; ++c) {
    p->class_count[c] = h_ptr[c + 1] - h_ptr[c];
    if (c > 0 && p->class_count[c] > 0) p->deg_used[class_degree(c)] = true;
    p->class_evals[c] = (double)h_evals[c];
    p->list_count[class_type(c)] += p->class_count[c];
    p->interactions[class_type(c)] += p->class_evals[c];
  }
  if (h_ptr[nclass] != E) {
    set_error("interaction list CSR holds %d entries, traversal produced %lld", h_ptr[nclass], (long long)E);
    return BLDTT_EINTERNAL;
  }
  dfree(evals, s); dfree(hist, s); dfree(order, s);
  dfree(ent_t, s); dfree(ent_s, s); dfree(ent_key, s);
  return BLDTT_OK;
}

// ---------------------------------------------------------------------------
// Work items
// ---------------------------------------------------------------------------

__global__ void k_leaf_padded(int32_t nleaves, const int32_t* __restrict__ leaf_ids,
                              const int32_t* __restrict__ begin, const int32_t* __restrict__ end,
                              int32_t* __restrict__ padded) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nleaves) return;
  int c = leaf_ids[i];
  int32_t m = end[c] - begin[c];
  padded[i] = (m + kChunk - 1) / kChunk * kChunk;
}

struct ListView {
  const int32_t *ptr, *src;
  int32_t nct;
  const int32_t *s_leaf_first, *s_leaf_last, *pad_prefix;
  DegreeSet deg;
};

// Real sources (no padding) and pool chunks that the entries of list class
// `cls` of target cluster c contribute: particles of source clusters
// (particles = true) or proxies of degree index i.
__device__ __forceinline__ void class_work(const ListView& L, const int32_t* s_begin, const int32_t* s_end,
                                           int cls, bool particles, int i, int32_t c, int64_t& sources,
                                           int64_t& chunks) {
  const int64_t k = (int64_t)cls * L.nct + c;
  const int32_t e0 = L.ptr[k], e1 = L.ptr[k + 1];
  if (particles) {
    for (int32_t e = e0; e < e1; ++e) {
      const int32_t s = L.src[e];
      sources += s_end[s] - s_begin[s];
      chunks += (L.pad_prefix[L.s_leaf_last[s]] - L.pad_prefix[L.s_leaf_first[s]]) / kChunk;
    }
  } else {
    sources += (int64_t)(e1 - e0) * L.deg.np[i];
    chunks += (int64_t)(e1 - e0) * (L.deg.np_pad[i] / kChunk);
  }
}

// Target rows the interaction kernel evaluates in its default consumer layout
// (4 warps x 2 rows of 32) for m targets cut into tiles of kTile: with idle
// warps skipping, every 32-row group that holds a real target (its idle rows
// included); without, a partial tile of at most 128 targets costs all four
// warps' first rows.
__device__ __forceinline__ int64_t executed_rows_skip(int64_t m) { return (m + 31) / 32 * 32; }
__device__ __forceinline__ int64_t executed_rows_noskip(int64_t m) {
  const int64_t r = m % kTile;
  return m - r + (r == 0 ? 0 : (r <= kTile / 2 ? kTile / 2 : (r + 31) / 32 * 32));
}

// Items of target cluster c: tiles of its particles (a leaf: PP and PC of every
// degree, on the leaf and on each ancestor), and tiles of its proxy points of
// degree i (CP and CC of degree i on the cluster itself).  cost_prox is
// [nct][kMaxDegrees].
__global__ void k_item_count(int32_t nct, ListView L, const int32_t* __restrict__ parent,
                             const int32_t* __restrict__ nchild, const int32_t* __restrict__ begin,
                             const int32_t* __restrict__ end, const int32_t* __restrict__ s_begin,
                             const int32_t* __restrict__ s_end, int32_t* __restrict__ nitems,
                             int64_t* __restrict__ cost_part, int64_t* __restrict__ cost_prox,
                             unsigned long long* __restrict__ executed,   // [2]: skip, no skip
                             int64_t* __restrict__ eval_part, int64_t* __restrict__ eval_prox) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nct) return;
  int64_t cp = 0, sp = 0;
  if (nchild[c] == 0)   // PP + PC of the leaf and of all its ancestors (Sec. 2.7 chain)
    for (int32_t a = c; a >= 0; a = parent[a]) {
      class_work(L, s_begin, s_end, 0, true, 0, a, sp, cp);
      for (int i = 0; i < L.deg.n; ++i)
        class_work(L, s_begin, s_end, class_of(BLDTT_PC, i), false, i, a, sp, cp);
    }
  const int32_t tp = cp > 0 ? (end[c] - begin[c] + kTile - 1) / kTile : 0;
  int32_t items = tp;
  unsigned long long ex = cp > 0 ? (unsigned long long)executed_rows_skip(end[c] - begin[c]) * sp : 0ull;
  unsigned long long ex_ns = cp > 0 ? (unsigned long long)executed_rows_noskip(end[c] - begin[c]) * sp : 0ull;
  eval_part[c] = cp > 0 ? (int64_t)(end[c] - begin[c]) * sp : 0;   // real evaluations (no padding)
  int64_t evq = 0;
  for (int i = 0; i < L.deg.n; ++i) {   // CP + CC of degree i on the cluster itself
    int64_t cq = 0, sq = 0;
    class_work(L, s_begin, s_end, class_of(BLDTT_CP, i), true, i, c, sq, cq);
    class_work(L, s_begin, s_end, class_of(BLDTT_CC, i), false, i, c, sq, cq);
    const int32_t tq = cq > 0 ? (L.deg.np[i] + kTile - 1) / kTile : 0;
    items += tq;
    cost_prox[(int64_t)c * kMaxDegrees + i] = cq;
    if (cq > 0) {
      ex += (unsigned long long)executed_rows_skip(L.deg.np[i]) * sq;
      ex_ns += (unsigned long long)executed_rows_noskip(L.deg.np[i]) * sq;
    }
    if (cq > 0) evq += (int64_t)L.deg.np[i] * sq;
  }
  eval_prox[c] = evq;
  nitems[c] = items;
  cost_part[c] = cp;
  // evaluations the kernel performs: every target slot of every tile meets every real source
  if (ex) atomicAdd(executed, ex);
  if (ex_ns) atomicAdd(executed + 1, ex_ns);
}

// Sort key of an item: the segment (kernel group) of its problem in the high
// bits, then (in the shared Coulomb/Yukawa launch) its kernel, then decreasing
// cost.  Kernel-major order keeps one kernel's code hot on all SMs at a time:
// items of the two kernels interleaved by cost ran 44 % slower.
struct SegmentMap {
  int n;
  int kernel[8];
};

__global__ void k_item_fill(int32_t nct, const int32_t* __restrict__ off,
                            const int64_t* __restrict__ cost_part, const int64_t* __restrict__ cost_prox,
                            const int32_t* __restrict__ begin, const int32_t* __restrict__ end,
                            const int32_t* __restrict__ problem, const int* __restrict__ prob_kernel,
                            SegmentMap segmap, DegreeSet deg, int4* __restrict__ items,
                            uint32_t* __restrict__ keys, int32_t* __restrict__ vals) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nct) return;
  int32_t o = off[c];
  const uint32_t kKeyMax = (1u << 24) - 1u;
  uint32_t seg = 0;
  uint32_t sub = 0;          // the shared Coulomb/Yukawa launch: Coulomb items first
  const int kern = prob_kernel[problem[c]];
  for (int i = 0; i < segmap.n; ++i)
    if (segmap.kernel[i] == kern ||
        (segmap.kernel[i] == kKernCoulombYukawa && (kern == BLDTT_COULOMB || kern == BLDTT_YUKAWA))) {
      seg = (uint32_t)i;
      sub = segmap.kernel[i] == kKernCoulombYukawa && kern == BLDTT_YUKAWA ? 1u : 0u;
    }
  if (cost_part[c] > 0) {
    uint32_t k = (seg << 25) | (sub << 24) | (kKeyMax - (uint32_t)min((int64_t)kKeyMax, cost_part[c]));
    for (int32_t r = begin[c]; r < end[c]; r += kTile) {
      items[o] = make_int4(c, r, min(kTile, end[c] - r), kItemParticles);
      keys[o] = k;
      vals[o] = o;
      ++o;
    }
  }
  for (int i = 0; i < deg.n; ++i) {
    const int64_t cq = cost_prox[(int64_t)c * kMaxDegrees + i];
    if (cq <= 0) continue;
    const int32_t np = deg.np[i];
    uint32_t k = (seg << 25) | (sub << 24) | (kKeyMax - (uint32_t)min((int64_t)kKeyMax, cq));
    for (int32_t r = 0; r < np; r += kTile) {
      items[o] = make_int4(c, r, min(kTile, np - r), kItemProxies + i);
      keys[o] = k;
      vals[o] = o;
      ++o;
    }
  }
}

// First item of every segment (keys sorted): first[seg] = i where the segment starts.
__global__ void k_segment_starts(const uint32_t* __restrict__ keys, int32_t n, int32_t* __restrict__ first) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t sg = keys[i] >> 25;
  if (i == 0 || (keys[i - 1] >> 25) != sg) first[sg] = i;
}

__global__ void k_gather_items(const int4* __restrict__ src, const int32_t* __restrict__ idx,
                               int4* __restrict__ dst, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[idx[i]];
}

// Bounding box of every 32-row group of every work item (the targets one warp
// evaluates together in any consumer layout), rounded outward to floats; an
// empty group gets an empty box.  One warp per group.
struct NodeSet {
  const double* nodes[kMaxDegrees];   // [C][3][d+1] per degree index
};

__global__ void k_item_boxes(int32_t nitems, const int4* __restrict__ items, const double* __restrict__ x,
                             const double* __restrict__ y, const double* __restrict__ z, NodeSet ns,
                             DegreeSet deg, float4* __restrict__ box) {
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= (int64_t)nitems * kItemGroups) return;
  const int4 it = items[w / kItemGroups];
  const int r = (int)(w % kItemGroups) * 32 + lane;
  // float bounds (rounded outward) first: min/max commute with the monotone
  // roundings, and float min/max avoid the FP64 pipe
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  if (r < it.z) {
    double v[3];
    if (it.w == kItemParticles) {
      const int64_t i = (int64_t)it.y + r;
      v[0] = x[i];
      v[1] = y[i];
      v[2] = z[i];
    } else {
      const int l = it.y + r;
      const int P = deg.d[it.w - kItemProxies] + 1;
      const double* nd = ns.nodes[it.w - kItemProxies] + (int64_t)it.x * 3 * P;
      v[0] = nd[l / (P * P)];
      v[1] = nd[P + (l / P) % P];
      v[2] = nd[2 * P + l % P];
    }
    for (int d = 0; d < 3; ++d) {
      lo[d] = __double2float_rd(v[d]);
      hi[d] = __double2float_ru(v[d]);
    }
  }
  for (int d = 0; d < 3; ++d)
    for (int o = 16; o; o >>= 1) {
      lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
      hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
    }
  if (lane == 0) {
    box[2 * w] = make_float4(lo[0], lo[1], lo[2], 0.f);
    box[2 * w + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
  }
}

int build_work_items(bldtt_plan* p, cudaStream_t s) {
  bldtt::Counters& cnt = p->setup_counter;
  const Tree& st = p->st;
  const Tree& tt = p->tt;
  // Source pool layout: padded leaves (leaf order), then padded proxy blocks.
  int32_t* padded = nullptr;
  BL_TRY(dalloc_n(&padded, st.nleaves, s));
  BL_TRY(dalloc_n(&p->pad_prefix, (size_t)st.nleaves + 1, s));
  k_leaf_padded<<<nblk(st.nleaves, 256), 256, 0, s>>>(st.nleaves, st.leaf_ids, st.begin, st.end,
                                                      padded);
  BL_LAUNCHED(cnt.launches);
  int64_t bound = (int64_t)st.n + (int64_t)st.nleaves * kChunk;
  if (bound >= (int64_t)INT32_MAX) {
    set_error("source pool of %lld entries exceeds the int32 index range", (long long)bound);
    return BLDTT_EINVAL;
  }
  // the padded total lands at pad_prefix[nleaves]; it comes back to the host
  // with the item count, in one read
  BL_TRY(scan_exclusive_dev(padded, p->pad_prefix, st.nleaves, p->pad_prefix + st.nleaves, s, cnt));
  dfree(padded, s);

  const int32_t nct = tt.nclusters;
  ListView L{p->list_ptr, p->list_src, nct, st.leaf_first, st.leaf_last, p->pad_prefix, p->deg};
  int32_t *nitems = nullptr, *off = nullptr;
  int64_t *cost_part = nullptr, *cost_prox = nullptr;
  BL_TRY(dalloc_n(&nitems, nct, s));
  BL_TRY(dalloc_n(&off, nct, s));
  BL_TRY(dalloc_n(&cost_part, nct, s));
  BL_TRY(dalloc_n(&cost_prox, (size_t)nct * kMaxDegrees, s));
  unsigned long long* summary = nullptr;   // [0, 2): executed counters; [2, 6): segment starts
  BL_TRY(dalloc_n(&summary, 6, s));
  BL_CUDA(cudaMemsetAsync(summary, 0, 2 * sizeof(unsigned long long), s));
  unsigned long long* executed = summary;
  dfree_ptr(p->eval_part, s);
  dfree_ptr(p->eval_prox, s);
  BL_TRY(dalloc_n(&p->eval_part, nct, s));
  BL_TRY(dalloc_n(&p->eval_prox, nct, s));
  k_item_count<<<nblk(nct, 128), 128, 0, s>>>(nct, L, tt.parent, tt.nchild, tt.begin, tt.end,
                                              st.begin, st.end, nitems, cost_part, cost_prox,
                                              executed, p->eval_part, p->eval_prox);
  BL_LAUNCHED(cnt.launches);
  int32_t* totals = nullptr;   // [0] items, [1] padded pool particles
  BL_TRY(dalloc_n(&totals, 2, s));
  BL_TRY(scan_exclusive_dev(nitems, off, nct, totals, s, cnt));
  BL_CUDA(cudaMemcpyAsync(totals + 1, p->pad_prefix + st.nleaves, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  int32_t h_tot[2];
  BL_TRY(read_device(totals, h_tot, sizeof(h_tot), s));
  dfree(totals, s);
  const int32_t ni = h_tot[0];
  p->nitems = ni;
  p->pool_particles = h_tot[1];
  p->pool_len = h_tot[1];
  for (int i = 0; i < p->deg.n; ++i) {   // proxy blocks of every source cluster, per degree
    p->deg.proxy_base[i] = p->pool_len;
    p->pool_len += (int64_t)st.nclusters * p->deg.np_pad[i];
  }
  p->np_pad = p->deg.np_pad[p->deg.n - 1];
  int4* items = nullptr;
  uint32_t* keys = nullptr;
  int32_t* vals = nullptr;
  BL_TRY(dalloc_n(&items, ni, s));
  BL_TRY(dalloc_n(&keys, ni, s));
  BL_TRY(dalloc_n(&vals, ni, s));
  BL_TRY(dalloc_n(&p->items, ni, s));
  SegmentMap segmap{};
  segmap.n = (int)p->segment_kernels.size();
  for (int i = 0; i < segmap.n; ++i) segmap.kernel[i] = p->segment_kernels[i];
  k_item_fill<<<nblk(nct, 128), 128, 0, s>>>(nct, off, cost_part, cost_prox, tt.begin, tt.end,
                                             tt.problem, p->prob_kernel, segmap, p->deg, items, keys,
                                             vals);
  BL_LAUNCHED(cnt.launches);
  // Grouped by kernel, longest items first within a group (stable), so that
  // each persistent launch's tail is short.
  int seg_bits = 0;
  while ((1 << seg_bits) < segmap.n) ++seg_bits;
  bool fused = false;   // a shared Coulomb/Yukawa segment sets the kernel bit (bit 24)
  for (int i = 0; i < segmap.n; ++i) fused |= segmap.kernel[i] == kKernCoulombYukawa;
  const int key_bits = seg_bits > 0 ? 25 + seg_bits : (fused ? 25 : 24);
  BL_TRY(radix_sort_pairs(keys, vals, ni, key_bits, s, cnt));
  // segment starts (8 int32) and the two executed-evaluation counters come
  // back to the host in one read
  int32_t* seg_first = reinterpret_cast<int32_t*>(summary + 2);
  BL_CUDA(cudaMemsetAsync(seg_first, 0xff, 8 * sizeof(int32_t), s));
  if (ni > 0) {
    k_segment_starts<<<nblk(ni, 256), 256, 0, s>>>(keys, ni, seg_first);
    BL_LAUNCHED(cnt.launches);
  }
  int32_t h_first[8];
  if (ni > 0) {
    k_gather_items<<<nblk(ni, 256), 256, 0, s>>>(items, vals, p->items, ni);
    BL_LAUNCHED(cnt.launches);
  }
  if (p->precision == BLDTT_FP32_BULK && ni > 0) {
    BL_TRY(dalloc_n(&p->item_box, (size_t)ni * kItemGroups * 2, s));
    NodeSet ns{};
    for (int i = 0; i < p->deg.n; ++i) ns.nodes[i] = p->nodes_t[i];
    k_item_boxes<<<nblk((int64_t)ni * kItemGroups, 8), 256, 0, s>>>(ni, p->items, tt.x, tt.y, tt.z, ns,
                                                                    p->deg, p->item_box);
    BL_LAUNCHED(cnt.launches);
  }
  unsigned long long h_sum[6];
  BL_TRY(read_device(summary, h_sum, sizeof(h_sum), s));
  const unsigned long long h_exec[2] = {h_sum[0], h_sum[1]};
  std::memcpy(h_first, h_sum + 2, sizeof(h_first));
  p->executed_skip = (double)h_exec[0];
  p->executed_noskip = (double)h_exec[1];
  p->skip_saved_evaluations = p->executed_noskip - p->executed_skip;
  p->executed_evaluations = p->executed_noskip;
  dfree(summary, s);
  p->segments.clear();
  for (int i = 0; i < segmap.n; ++i) {
    if (h_first[i] < 0) continue;                    // no items for this kernel
    int32_t end = ni;
    for (int j = i + 1; j < segmap.n; ++j)
      if (h_first[j] >= 0) {
        end = h_first[j];
        break;
      }
    p->segments.push_back({segmap.kernel[i], h_first[i], end - h_first[i], 0, 0, 0});
  }
  dfree(items, s); dfree(keys, s); dfree(vals, s);
  dfree(nitems, s); dfree(off, s); dfree(cost_part, s); dfree(cost_prox, s);
  return BLDTT_OK;
}

}  // namespace bldtt
