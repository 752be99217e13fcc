// Internal declarations of the GB300 BLDTT library.
//
// Layout summary (all device memory, one plan per problem):
//  - Each tree stores its particles permuted into tree order (FP64 x, y, z
//    arrays and perm[] back to input order) so every cluster is a contiguous
//    range [begin, end).  Clusters are numbered level by level; the children
//    of a cluster are consecutive.  Boxes are 6 doubles per cluster
//    (lo x,y,z, hi x,y,z); proxy points are kept as three 1D arrays of n+1
//    Chebyshev points per cluster (Sec. 2.1: the 3D grid is their tensor
//    product).
//  - The four interaction lists (Sec. 3.1) are one CSR keyed by
//    type * num_target_clusters + target cluster.
//  - The "source pool" is what the interaction kernel streams: every source
//    leaf's particles followed by every source cluster's proxy points, each
//    segment padded to a multiple of kChunk entries (charge 0) so that every
//    chunk is one aligned bulk copy.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/bldtt.h"

namespace bldtt {

constexpr int kMaxDegree = 16;                 // n <= 16  ->  P = n + 1 <= 17
constexpr int kMaxP = kMaxDegree + 1;
constexpr int kChunk = 256;                    // sources per staged chunk (one coordinate frame)
constexpr int kTile = 256;                     // targets per work item of the interaction kernel
constexpr int kChunkInfo = 2;                  // float4 per pool chunk description
constexpr int kItemGroups = kTile / 32;        // 32-row target groups per work item
constexpr int kMaxDegrees = 8;                 // interpolation degrees of one plan
// Segment kernel id of a persistent launch that drains the Coulomb and the
// Yukawa problems of a batch together (the kernel is chosen per work item).
constexpr int kKernCoulombYukawa = 1000;
// Interaction-kernel layouts: kLayoutSkip base layouts, and the same again
// (ids kLayoutSkip..2*kLayoutSkip-1) with idle warps skipping their work.
constexpr int kLayoutSkip = 3;
constexpr int kMaxLayouts = 2 * kLayoutSkip;
constexpr int kMaxClasses = 1 + 3 * kMaxDegrees;
constexpr int kHidden = 64;                    // selector network width
constexpr int kFeatures = 6;                   // selector network inputs

// Degree set of a plan (one degree, n, unless a learned selector picks a
// degree per pair).  Interaction-list classes: 0 = PP, 1 + 3 i + t with
// t = 0 PC, 1 CP, 2 CC at degree d[i]; with one degree the classes are
// PP, PC, CP, CC = 0, 1, 2, 3.
struct DegreeSet {
  int n = 1;
  int d[kMaxDegrees] = {};
  int np[kMaxDegrees] = {};
  int np_pad[kMaxDegrees] = {};
  int64_t proxy_base[kMaxDegrees] = {};   // source-pool offset of degree i's proxy blocks
};
// Chebyshev point of the 2nd kind s_k = cos(pi k / n) on [-1, 1], symmetrised
// (s_{n-k} = -s_k, s_{n/2} = 0) as the proxy points of Sec. 2.2.
__device__ __forceinline__ double cheb_point(int k, int n) {
  if (2 * k == n) return 0.0;
  if (2 * k < n) return cos(__ddiv_rn(__dmul_rn(M_PI, (double)k), (double)n));
  return -cos(__ddiv_rn(__dmul_rn(M_PI, (double)(n - k)), (double)n));
}
__host__ __device__ inline int class_type(int c) { return c == 0 ? BLDTT_PP : 1 + (c - 1) % 3; }
__host__ __device__ inline int class_degree(int c) { return c == 0 ? 0 : (c - 1) / 3; }
__host__ __device__ inline int class_of(int type, int i) { return type == BLDTT_PP ? 0 : 1 + 3 * i + (type - 1); }

// ---- FP32 frame coordinates ------------------------------------------------
// A coordinate v (FP64) is carried in FP32 relative to a frame centre c (a
// float) by the split v = hi + lo, hi = fl(v), lo = fl(v - hi):
//   main  = fl(fl(hi - c) + lo)
//   resid = the exact rounding errors of both additions (TwoSum), summed,
// so that hi - c + lo = main + resid to within u^2 |v|.  The same expressions
// serve the source pool and the targets, so that equal FP64 points get equal
// FP32 parts.
__device__ __forceinline__ float frame_main(float hi, float lo, float c) {
  return __fadd_rn(__fsub_rn(hi, c), lo);
}
__device__ __forceinline__ float two_sum_err(float a, float b, float s) {
  const float bb = __fsub_rn(s, a);
  return __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ float frame_resid(float hi, float lo, float c) {
  const float d = __fsub_rn(hi, c);
  return __fadd_rn(two_sum_err(hi, -c, d), two_sum_err(d, lo, __fadd_rn(d, lo)));
}
// Order-preserving integer image of a finite double: for finite a and b,
// a < b exactly when okey(a) < okey(b), and okey(-0.0) == okey(+0.0).  The
// set-up's coordinate comparisons, minima and maxima run on the integer pipe
// with the results the FP64 operations give: on GB300 FP64 instructions issue
// at about 1/64 of the FP32 rate.  okey_inv maps a key back (-0.0 as +0.0).
__device__ __forceinline__ long long okey(double v) {
  long long k = __double_as_longlong(v);
  k = k == (long long)0x8000000000000000ULL ? 0LL : k;
  return k ^ ((k >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double okey_inv(long long k) {
  return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}
constexpr long long kKeyPosInf = 0x7ff0000000000000LL;                 // okey(+inf)
constexpr long long kKeyNegInf = (long long)0x800fffffffffffffULL;     // okey(-inf)

__device__ __forceinline__ void split_f64(double v, float& hi, float& lo) {
  hi = __double2float_rn(v);
  lo = __double2float_rn(__dsub_rn(v, (double)hi));
}

// Work-item kinds: particle targets, or the proxy points of degree index
// (kind - kItemProxies) of a target cluster.
enum ItemKind { kItemParticles = 0, kItemProxies = 1 };

// Error flag codes written by kernels into plan->dev_err.
enum DevErr { kDevErrNone = 0, kDevErrTimeout = 1, kDevErrBounds = 2 };

void set_error(const char* fmt, ...);

#define BL_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      ::bldtt::set_error("%s:%d: %s failed: %s", __FILE__, __LINE__, #call,                \
                         cudaGetErrorString(e_));                                          \
      return e_ == cudaErrorMemoryAllocation ? BLDTT_ENOMEM : BLDTT_ECUDA;                 \
    }                                                                                      \
  } while (0)

#define BL_LAUNCHED(counter)                                                               \
  do {                                                                                     \
    cudaError_t e_ = cudaGetLastError();                                                   \
    if (e_ != cudaSuccess) {                                                               \
      ::bldtt::set_error("%s:%d: kernel launch failed: %s", __FILE__, __LINE__,            \
                         cudaGetErrorString(e_));                                          \
      return BLDTT_ECUDA;                                                                  \
    }                                                                                      \
    ++(counter);                                                                           \
  } while (0)

#define BL_TRY(expr)                                                                       \
  do {                                                                                     \
    int s_ = (expr);                                                                       \
    if (s_ != BLDTT_OK) return s_;                                                         \
  } while (0)

// Stream-ordered device allocation helpers.  Allocations come from the memory
// pool set for the calling thread (the library's shared pool of the device
// while a plan is set up or a host solve runs), else from the device's
// default pool.  The shared pool keeps freed memory for reuse (up to an
// eighth of the device's memory between set-ups), where the default pool
// hands it back to the driver at every host synchronisation.
int dalloc(void** p, size_t bytes, cudaStream_t s);
// Per-thread context of the plan being set up: its memory pool and a pinned
// host slot of kPinnedSlot bytes for small device-to-host reads.
constexpr size_t kPinnedSlot = 1024;
void set_thread_context(cudaMemPool_t pool, void* pinned);
cudaMemPool_t thread_pool();
void* thread_pinned();
struct PlanScope {
  cudaMemPool_t prev_pool;
  void* prev_pinned;
  PlanScope(cudaMemPool_t pool, void* pinned) : prev_pool(thread_pool()), prev_pinned(thread_pinned()) {
    set_thread_context(pool, pinned);
  }
  ~PlanScope() { set_thread_context(prev_pool, prev_pinned); }
  PlanScope(const PlanScope&) = delete;
  PlanScope& operator=(const PlanScope&) = delete;
};
template <class T>
inline int dalloc_n(T** p, size_t n, cudaStream_t s) {
  return dalloc(reinterpret_cast<void**>(p), n * sizeof(T) + (n == 0 ? sizeof(T) : 0), s);
}
void dfree(void* p, cudaStream_t s);
template <class T>
inline void dfree_ptr(T*& p, cudaStream_t s) {
  dfree(reinterpret_cast<void*>(p), s);
  p = nullptr;
}
// Grow a device array to hold at least `need` elements, keeping `keep` of them.
template <class T>
int dgrow(T** p, size_t* cap, size_t need, size_t keep, cudaStream_t s);
// Several scratch arrays carved from one device allocation (256-byte aligned
// each): one pool call instead of one per array.  add() records where each
// array's pointer goes; alloc() allocates and sets them all; the block is
// freed (stream-ordered) by release() or when the arena goes out of scope,
// so an early error return does not leak it.
class Arena {
 public:
  Arena() = default;
  Arena(const Arena&) = delete;
  Arena& operator=(const Arena&) = delete;
  Arena(Arena&& o) noexcept { take(o); }
  Arena& operator=(Arena&& o) noexcept {
    if (this != &o) {
      release(stream_);
      take(o);
    }
    return *this;
  }
  ~Arena() { release(stream_); }
  template <class T>
  void add(T** p, size_t n) {
    parts_.push_back({reinterpret_cast<void**>(p), n * sizeof(T)});
  }
  int alloc(cudaStream_t s) {
    size_t total = 0;
    for (const auto& pr : parts_) total += round(pr.second);
    stream_ = s;
    BL_TRY(dalloc(&block_, total > 0 ? total : 256, s));
    char* c = static_cast<char*>(block_);
    for (const auto& pr : parts_) {
      *pr.first = c;
      c += round(pr.second);
    }
    return BLDTT_OK;
  }
  void release(cudaStream_t s) {
    if (block_) dfree(block_, s);
    block_ = nullptr;
  }

 private:
  static size_t round(size_t b) { return (b + 255) & ~size_t(255); }
  void take(Arena& o) {
    parts_ = std::move(o.parts_);
    block_ = o.block_;
    stream_ = o.stream_;
    o.block_ = nullptr;
  }
  std::vector<std::pair<void**, size_t>> parts_;
  void* block_ = nullptr;
  cudaStream_t stream_ = nullptr;
};

struct Tree {
  int32_t n = 0;                      // particles
  int32_t nclusters = 0, nlevels = 0, nleaves = 0;
  size_t cap = 0;                     // allocated cluster capacity
  double *x = nullptr, *y = nullptr, *z = nullptr;   // tree order
  int32_t* perm = nullptr;            // tree position -> input index
  double *sx = nullptr, *sy = nullptr, *sz = nullptr;   // spare buffers of the build (or null),
  int32_t* sperm = nullptr;                             // taken by the Morton pass
  int32_t *begin = nullptr, *end = nullptr, *parent = nullptr;
  int32_t *first_child = nullptr, *nchild = nullptr, *level = nullptr;
  int32_t* problem = nullptr;         // [C] problem (root) the cluster belongs to
  int32_t nroots = 1;                 // problems: clusters 0..nroots-1 are the roots
  double* box = nullptr;              // [C][6]: lo x,y,z, hi x,y,z
  double* center = nullptr;           // [C][3]
  double* radius = nullptr;           // [C]
  double* nodes = nullptr;            // [C][3][P], P = n + 1 of the plan's highest degree
  double* xfer_u = nullptr;           // [C][3][P][P]: parent's basis at the cluster's nodes
  int32_t* leaf_ids = nullptr;        // leaf order (by begin) -> cluster
  int32_t *leaf_first = nullptr, *leaf_last = nullptr;   // per cluster: leaf-order range
  std::vector<int32_t> level_start;   // host: level l holds clusters [ls[l], ls[l+1])
  std::vector<int32_t> h_nchild;      // host copy (used to pick upward/downward clusters)
};

struct Counters {
  int64_t launches = 0;
};

}  // namespace bldtt

struct bldtt_plan {
  int64_t M = 0, N = 0;
  int kernel = 0;
  double kappa = 0.0;
  int n = 0, P = 0, np = 0;
  double theta = 0.0;
  int N0 = 0, M0 = 0;
  int precision = 0;
  int variant = 0;                    // enum bldtt_variant
  int device = 0;

  // Problems of a batch (one for bldtt_setup): particle offsets of each
  // problem's targets and sources, and each problem's kernel and parameter.
  int32_t nprob = 1;
  std::vector<int32_t> t_off, s_off;  // host, nprob + 1 entries
  std::vector<int> prob_kernel_h;     // host copies
  std::vector<double> prob_kappa_h;
  std::vector<float> prob_prm_h;      // host copy of prob_prm
  int* prob_kernel = nullptr;         // device [nprob]
  double* prob_kappa = nullptr;       // device [nprob]
  float* prob_prm = nullptr;          // device [nprob] FP32 form of the parameter
  std::vector<int> kernels_present;   // distinct kernel ids of the batch, ascending
  // Kernel id of each persistent interaction launch: one per kernel present,
  // except that Coulomb and Yukawa problems share one (kKernCoulombYukawa).
  std::vector<int> segment_kernels;
  cudaStream_t stream = nullptr;      // stream of the last call (for synchronisation)

  bldtt::Tree tt, st;                 // target and source trees
  bool shared_tree = false;           // st aliases tt (targets are the sources)
  // Degrees (bldtt::DegreeSet); n above is the highest.  Per degree index i
  // below the highest: proxy nodes of both trees [C][3][d+1], the proxy
  // charges and potentials [C][np], and the (d+1) x (n+1) matrix
  // A[k][k'] = L^(d)_k(s^(n)_k') of Chebyshev points on [-1, 1].
  bldtt::DegreeSet deg;
  int nclass = 4;
  bool deg_used[bldtt::kMaxDegrees] = {};   // some list entry has this degree (set by build_lists)
  double* nodes_t[bldtt::kMaxDegrees] = {};
  double* nodes_s[bldtt::kMaxDegrees] = {};
  double* qhat_d[bldtt::kMaxDegrees] = {};
  double* phit_d[bldtt::kMaxDegrees] = {};
  double* xfer[bldtt::kMaxDegrees] = {};
  // Learned selector (bldtt_setup_learned): bf16 weights W1..W4, float
  // biases, the training box of the features and the per-pair budget.
  bool learned = false;
  bool selector_net = false;          // false: the MAC fallback decides every pair
  void* sel_w = nullptr;              // __nv_bfloat16 [64*6 + 64*64*2 + nout*64]
  float* sel_b = nullptr;             // [64*3 + nout]
  int sel_nout = 0;
  float sel_lo[bldtt::kFeatures] = {}, sel_hi[bldtt::kFeatures] = {};
  float sel_log_eps = 0.f;
  double* q_tree = nullptr;           // [N] charges, source tree order

  // Interaction lists: CSR over key = type * nct + t.
  int32_t* list_ptr = nullptr;        // [4*nct + 1]
  int32_t* list_src = nullptr;        // [E]
  int32_t* list_tgt = nullptr;        // [E]
  int64_t nentries = 0;
  int64_t list_count[4] = {0, 0, 0, 0};        // entries per type (all degrees)
  double interactions[4] = {0, 0, 0, 0};
  std::vector<int64_t> class_count;             // entries per class
  std::vector<double> class_evals;              // kernel evaluations per class

  // Source pool.
  int np_pad = 0;                     // proxies per cluster rounded up to kChunk
  int32_t* pad_prefix = nullptr;      // [nleaves_s + 1] pool offset of each source leaf
  int64_t pool_particles = 0, pool_len = 0;
  void* pool = nullptr;               // float4 (FP32_BULK) or double4 (FP64) entries

  // Work items of the interaction kernel, sorted by decreasing cost.
  int4* items = nullptr;              // {cluster, row_begin, row_count, kind}
  int32_t nitems = 0;
  int32_t* item_counter = nullptr;    // one per segment
  double executed_evaluations = 0.0;
  // Evaluations the interaction kernel performs with and without idle warps
  // skipping their work (rows of 32-target groups holding no real target).
  double executed_skip = 0.0, executed_noskip = 0.0, skip_saved_evaluations = 0.0;
  // Items are grouped by the kernel of their problem; each group is one
  // persistent launch of the interaction kernel specialised for that kernel.
  struct Segment {
    int kernel;                       // BLDTT_COULOMB, ...
    int32_t first, count;             // items [first, first + count)
    int layout, grid, threads;        // consumer layout and launch shape
  };
  std::vector<Segment> segments;
  struct TuneRow {
    int launch, kernel, layout;
    float ms;
  };
  std::vector<TuneRow> tune_table;    // what the last bldtt_autotune searched
  bool tuned = false;
  int interact_layout = 0;            // requested layout: 0 = 4 warps x 2 targets, 1 = 2 x 4, 2 = 4 x 2 at 5 CTAs/SM, 4 stages; +kLayoutSkip: idle warps skip
  // Real kernel evaluations per target cluster: its particle items (leaves)
  // and its proxy items (all degrees); the costs behind target-leaf sharding.
  int64_t* eval_part = nullptr;       // [Ct]
  int64_t* eval_prox = nullptr;       // [Ct]
  // Target-leaf sharding (bldtt_compute_shard): the leaf-order ranges of the
  // last partition, and the work items of the last shard computed.
  int32_t shard_parts = 0;            // shards of the cached partition (0: none)
  std::vector<int32_t> shard_begin;   // [shard_parts + 1] first leaf (leaf order) of each shard
  int32_t shard_cached = -1;          // shard whose items are below
  std::vector<int64_t> h_eval_part, h_eval_prox;     // host copies for the shard's count
  std::vector<int32_t> h_leaf_first, h_leaf_last;
  double sh_evals = 0.0;              // evaluations of the cached shard's items
  double computed_evals = 0.0;        // evaluations of the last compute's items
  int4* sh_items = nullptr;
  float4* sh_item_box = nullptr;
  int32_t sh_nitems = 0;
  std::vector<Segment> sh_segments;
  // Engines of the FP32_BULK leaf contractions, Eq. (9) (upward) and Eq. (21)
  // (downward): BLDTT_PASS_SIMT or BLDTT_PASS_TENSOR (tcgen05).  The set-up
  // picks the downward default by the target leaves' mean size.
  int up_engine = BLDTT_PASS_SIMT;
  int down_engine = BLDTT_PASS_TENSOR;
  // Leaves (leaf order) the downward leaf pass writes: [down_lo, down_hi);
  // down_hi < 0 means all leaves.
  int32_t down_lo = 0, down_hi = -1;
  float4* chunk_frame = nullptr;      // [pool chunks][kChunkInfo]: frame centre + count, extents + tau
  float4* item_box = nullptr;         // FP32_BULK: [items][kItemGroups][2] target group boxes (lo, hi)
  float* pool_res = nullptr;          // FP32_BULK: frame residuals of the pool's particles (pair records)

  // Compute-phase arrays.
  double* qhat = nullptr;             // [Cs][np] proxy charges
  double* phit = nullptr;             // [Ct][np] proxy potentials
  double* phi_near = nullptr;         // [M] PP + PC part of phi, target tree order
  int* dev_err = nullptr;

  // Statistics.
  bldtt::Counters setup_counter, compute_counter;
  float ms_tree = 0.f, ms_lists = 0.f;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  bool have_compute_events = false;

  // Captured compute phase (bldtt_compute_graph).
  cudaGraphExec_t graph_exec = nullptr;
  cudaMemPool_t mempool = nullptr;    // the device's pool, shared by the process's plans (see dalloc)
  void* h_pinned = nullptr;           // two pinned read slots (set-up thread, source-tree thread),
                                      // recycled between plans
  double* graph_phi = nullptr;
};

namespace bldtt {

// ---- primitives (prims.cu) ----
// Exclusive prefix sum of n int32 values; *total_host (if not NULL) receives
// the sum (the call then synchronises the stream).
int scan_exclusive(const int32_t* in, int32_t* out, int64_t n, int32_t* total_host,
                   cudaStream_t s, Counters& c);
// The same with the sum left in device memory (*total_dev; 0 when n == 0).
int scan_exclusive_dev(const int32_t* in, int32_t* out, int64_t n, int32_t* total_dev,
                       cudaStream_t s, Counters& c);
// Copy `bytes` of device memory to the host after the stream's prior work, then
// synchronise it: through the calling thread's pinned slot when it has one
// (a pinned copy costs ~1 us against ~9 us for a pageable one).
int read_device(const void* dev, void* host, size_t bytes, cudaStream_t s);
// Stable ascending sort of (key, value) pairs on the low `bits` bits of key.
int radix_sort_pairs(uint32_t* keys, int32_t* vals, int64_t n, int bits, cudaStream_t s,
                     Counters& c);
// Raise *bad_dev if any of n doubles is not finite.
int check_finite(const double* v, int64_t n, int* bad_dev, cudaStream_t s, Counters& c);

// ---- trees (tree.cu) ----
// roots: host offsets (nroots + 1 entries) of the problems' particle ranges.
// The coordinates must be finite (the set-up checks them first).
int build_tree(Tree& T, const double* coords_user, int32_t n, const std::vector<int32_t>& roots,
               int32_t max_leaf, int degree, cudaStream_t s, Counters& c);
// Reorder the particles inside every leaf along a Morton curve of the leaf's box.
// build_tree by one cooperative launch where the device has them, else level
// by level; non-finite coordinates or charges (charges may be null) give
// BLDTT_EINVAL before any cluster splits.
int build_tree_checked(Tree& T, const double* coords, int32_t n, const std::vector<int32_t>& roots,
                       int32_t max_leaf, int degree, const double* charges, int64_t ncharges,
                       cudaStream_t s, Counters& cnt);
bool tree_build_cooperative();
// The environment variable BLDTT_LEVEL_BY_LEVEL=1 turns the cooperative tree
// build and traversal off (the level-by-level loops run instead; same results).
bool cooperative_set_up_disabled();
// Held from a cooperative launch until its result is read, so that set-ups on
// several host threads run their grid-synchronised launches one at a time.
std::mutex& cooperative_launch_mutex();
int morton_order_leaves(Tree& T, int32_t max_leaf, cudaStream_t s, Counters& c);
void free_tree(Tree& T, cudaStream_t s);

// ---- traversal, lists and work items (dtt.cu) ----
int build_lists(bldtt_plan* p, cudaStream_t s);
int build_work_items(bldtt_plan* p, cudaStream_t s);

// ---- passes (passes.cu) ----
int permute_charges(bldtt_plan* p, const double* charges_user, cudaStream_t s);
int upward_pass(bldtt_plan* p, cudaStream_t s);
int build_pool(bldtt_plan* p, cudaStream_t s);
// Proxy nodes and degree-transfer matrices of the degrees below the highest.
int setup_degrees(bldtt_plan* p, cudaStream_t s);
int build_chunk_frames(bldtt_plan* p, cudaStream_t s);
int downward_pass(bldtt_plan* p, double* phi_user, cudaStream_t s);
int configure_pass_kernels();

// ---- interactions (interact.cu) ----
int layouts_available(int kernel, int* out);
int interaction_grids(bldtt_plan* p);                 // launch shape of every segment
int run_segment(bldtt_plan* p, int seg, cudaStream_t s);
int run_interactions(bldtt_plan* p, cudaStream_t s);

// ---- tensor-core leaf passes (passes_tc.cu) ----
bool leaf_tc_supported(int P);
int configure_tc_kernels();
int up_leaf_tc(bldtt_plan* p, cudaStream_t s);
int down_leaf_tc(bldtt_plan* p, const int32_t* leaf_ids, int32_t nleaves, double* phi_user,
                 cudaStream_t s);

// ---- compute phase (capi.cu) ----
// Upward pass, pool, interactions of the plan's current work items, downward
// pass (leaves [down_lo, down_hi) only).
int compute_body(bldtt_plan* p, double* phi, cudaStream_t s);

// ---- learned selector (learned.cu) ----
// Class decision of every frontier pair (class >= 0, kChoiceNoApprox, or
// kChoiceFallback for the MAC of Alg. 2).
constexpr int16_t kChoiceNoApprox = -2;
constexpr int16_t kChoiceFallback = -1;
int select_pairs(bldtt_plan* p, const int2* pairs, int32_t F, int16_t* choice, cudaStream_t s);

// ---- direct sum (direct.cu) ----
int direct_sum(const double* targets, int64_t M, const double* sources, int64_t N,
               const double* charges, int kernel, double kappa, double* phi, cudaStream_t s);

}  // namespace bldtt
