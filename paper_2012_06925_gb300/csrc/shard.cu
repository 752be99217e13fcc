// Target-leaf sharding of the compute phase, for one process per GPU.
//
// The paper distributes its method over MPI ranks by partitioning both
// particle sets and exchanging locally essential trees (Sec. 3.2).  Here the
// sources stay whole on every GPU: each rank builds the same plan (trees and
// lists are deterministic), runs the whole upward pass, and then computes the
// potentials of one contiguous range of target leaves only:
//   - the particle work items (PP and PC) of its leaves;
//   - the proxy work items (CP and CC) of every target cluster whose subtree
//     holds one of its leaves (an ancestor shared by two ranks is computed by
//     both, with the same result);
//   - the downward pass, whose leaf step writes only its leaves' targets.
// Every work item owns its outputs and runs the same arithmetic whichever
// items run beside it, so the union of the shards' potentials equals the
// one-rank result bit for bit; the caller gathers them (each shard leaves the
// other entries of phi untouched, so a sum over ranks of zero-filled buffers
// is exact).
//
// The leaves (in leaf order, i.e. tree order) are split into contiguous
// ranges of equal cost: a leaf costs its particle items' kernel evaluations
// plus, for every cluster on its path to the root, that cluster's proxy-item
// evaluations divided evenly among the leaves under it.
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace bldtt {

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__global__ void k_leaf_costs(int32_t nleaves, const int32_t* __restrict__ leaf_ids,
                             const int32_t* __restrict__ parent, const int32_t* __restrict__ leaf_first,
                             const int32_t* __restrict__ leaf_last, const int64_t* __restrict__ eval_part,
                             const int64_t* __restrict__ eval_prox, double* __restrict__ cost) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nleaves) return;
  const int32_t c = leaf_ids[i];
  double v = (double)eval_part[c];
  for (int32_t a = c; a >= 0; a = parent[a])
    v += (double)eval_prox[a] / (double)(leaf_last[a] - leaf_first[a]);
  cost[i] = v;
}

// 1 if work item i belongs to the shard of leaves [lo, hi) (leaf order).
__global__ void k_shard_flags(int32_t nitems, const int4* __restrict__ items,
                              const int32_t* __restrict__ leaf_first, const int32_t* __restrict__ leaf_last,
                              int32_t lo, int32_t hi, int32_t* __restrict__ flag) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nitems) return;
  const int4 it = items[i];
  const int32_t f = leaf_first[it.x], l = leaf_last[it.x];
  const bool keep = it.w == kItemParticles ? (f >= lo && f < hi) : (f < hi && l > lo);
  flag[i] = keep ? 1 : 0;
}

__global__ void k_shard_gather(int32_t nitems, const int4* __restrict__ items,
                               const float4* __restrict__ box, const int32_t* __restrict__ flag,
                               const int32_t* __restrict__ pos, int4* __restrict__ out_items,
                               float4* __restrict__ out_box) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = t / (2 * kItemGroups + 1);
  const int r = (int)(t % (2 * kItemGroups + 1));
  if (i >= nitems || !flag[i]) return;
  if (r == 2 * kItemGroups)
    out_items[pos[i]] = items[i];
  else if (box)
    out_box[(int64_t)pos[i] * 2 * kItemGroups + r] = box[i * 2 * kItemGroups + r];
}

// Leaf-order ranges of a partition into nshards (cached in the plan).
static int shard_partition(bldtt_plan* p, int nshards, cudaStream_t s) {
  if (p->shard_parts == nshards) return BLDTT_OK;
  const Tree& T = p->tt;
  std::vector<double> cost(T.nleaves);
  if (T.nleaves > 0) {
    double* d_cost = nullptr;
    BL_TRY(dalloc_n(&d_cost, T.nleaves, s));
    k_leaf_costs<<<nblk(T.nleaves, 256), 256, 0, s>>>(T.nleaves, T.leaf_ids, T.parent, T.leaf_first,
                                                      T.leaf_last, p->eval_part, p->eval_prox, d_cost);
    BL_LAUNCHED(p->compute_counter.launches);
    BL_CUDA(cudaMemcpyAsync(cost.data(), d_cost, sizeof(double) * T.nleaves, cudaMemcpyDeviceToHost, s));
    const size_t nc = (size_t)T.nclusters;
    p->h_eval_part.resize(nc);
    p->h_eval_prox.resize(nc);
    p->h_leaf_first.resize(nc);
    p->h_leaf_last.resize(nc);
    BL_CUDA(cudaMemcpyAsync(p->h_eval_part.data(), p->eval_part, nc * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    BL_CUDA(cudaMemcpyAsync(p->h_eval_prox.data(), p->eval_prox, nc * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    BL_CUDA(cudaMemcpyAsync(p->h_leaf_first.data(), T.leaf_first, nc * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    BL_CUDA(cudaMemcpyAsync(p->h_leaf_last.data(), T.leaf_last, nc * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    BL_CUDA(cudaStreamSynchronize(s));
    dfree(d_cost, s);
  }
  std::vector<int32_t> begin(nshards + 1);
  BL_TRY(bldtt_partition_leaves(cost.data(), T.nleaves, nshards, begin.data()));
  p->shard_begin = begin;
  p->shard_parts = nshards;
  p->shard_cached = -1;
  return BLDTT_OK;
}

// Work items (and, in FP32_BULK, their target-group boxes) of one shard, in
// the plan's order, with the per-kernel segments recounted.
static int shard_items(bldtt_plan* p, int shard, cudaStream_t s) {
  if (p->shard_cached == shard) return BLDTT_OK;
  const int32_t lo = p->shard_begin[shard], hi = p->shard_begin[shard + 1];
  dfree_ptr(p->sh_items, s);
  dfree_ptr(p->sh_item_box, s);
  p->sh_nitems = 0;
  p->sh_segments.clear();
  const int32_t ni = p->nitems;
  if (ni > 0 && hi > lo) {
    int32_t *flag = nullptr, *pos = nullptr;
    BL_TRY(dalloc_n(&flag, ni, s));
    BL_TRY(dalloc_n(&pos, (size_t)ni + 1, s));
    k_shard_flags<<<nblk(ni, 256), 256, 0, s>>>(ni, p->items, p->tt.leaf_first, p->tt.leaf_last, lo, hi,
                                                flag);
    BL_LAUNCHED(p->compute_counter.launches);
    BL_TRY(scan_exclusive_dev(flag, pos, ni, pos + ni, s, p->compute_counter));
    std::vector<int32_t> h_pos(ni + 1);
    BL_CUDA(cudaMemcpyAsync(h_pos.data(), pos, sizeof(int32_t) * (ni + 1), cudaMemcpyDeviceToHost, s));
    BL_CUDA(cudaStreamSynchronize(s));
    const int32_t kept = h_pos[ni];
    if (kept > 0) {
      BL_TRY(dalloc_n(&p->sh_items, kept, s));
      if (p->item_box) BL_TRY(dalloc_n(&p->sh_item_box, (size_t)kept * 2 * kItemGroups, s));
      const int64_t threads = (int64_t)ni * (2 * kItemGroups + 1);
      k_shard_gather<<<nblk(threads, 256), 256, 0, s>>>(ni, p->items, p->item_box, flag, pos, p->sh_items,
                                                        p->sh_item_box);
      BL_LAUNCHED(p->compute_counter.launches);
    }
    for (const auto& seg : p->segments) {
      const int32_t f = h_pos[seg.first], c = h_pos[seg.first + seg.count] - f;
      if (c > 0) {
        auto sg = seg;
        sg.first = f;
        sg.count = c;
        p->sh_segments.push_back(sg);
      }
    }
    p->sh_nitems = kept;
    dfree(flag, s);
    dfree(pos, s);
  }
  // Evaluations of the shard's items: its leaves' particle items and the proxy
  // items of every cluster whose leaves meet the shard.
  double ev = 0.0;
  for (size_t c = 0; c < p->h_eval_part.size(); ++c) {
    const int32_t f = p->h_leaf_first[c], l = p->h_leaf_last[c];
    if (f >= lo && f < hi) ev += (double)p->h_eval_part[c];
    if (f < hi && l > lo) ev += (double)p->h_eval_prox[c];
  }
  p->sh_evals = ev;
  p->shard_cached = shard;
  return BLDTT_OK;
}

// The plan's full work set, swapped for one shard's during a compute.
struct WorkSwap {
  bldtt_plan* p;
  int4* items;
  float4* box;
  int32_t nitems;
  std::vector<bldtt_plan::Segment> segments;
  explicit WorkSwap(bldtt_plan* plan) : p(plan), items(plan->items), box(plan->item_box),
                                        nitems(plan->nitems), segments(plan->segments) {
    p->items = p->sh_items;
    p->item_box = p->sh_item_box;
    p->nitems = p->sh_nitems;
    p->segments = p->sh_segments;
  }
  ~WorkSwap() {
    p->items = items;
    p->item_box = box;
    p->nitems = nitems;
    p->segments = segments;
    p->down_lo = 0;
    p->down_hi = -1;
  }
};

int compute_shard(bldtt_plan* p, int shard, int nshards, double* phi, cudaStream_t s) {
  BL_TRY(shard_partition(p, nshards, s));
  BL_TRY(shard_items(p, shard, s));
  for (auto& sg : p->sh_segments)          // the plan's current (possibly autotuned) layouts
    for (const auto& seg : p->segments)
      if (seg.kernel == sg.kernel) sg.layout = seg.layout;
  WorkSwap swap(p);
  BL_TRY(interaction_grids(p));
  p->down_lo = p->shard_begin[shard];
  p->down_hi = p->shard_begin[shard + 1];
  p->computed_evals = p->sh_evals;
  const int rc = compute_body(p, phi, s);
  return rc;
}

}  // namespace bldtt

using namespace bldtt;

extern "C" int bldtt_partition_leaves(const double* leaf_cost, int32_t nleaves, int32_t nshards,
                                      int32_t* leaf_begin) {
  if (nshards < 1 || nleaves < 0 || !leaf_begin || (nleaves > 0 && !leaf_cost)) {
    set_error("partition_leaves: need nshards >= 1, nleaves >= 0, leaf_begin and leaf_cost");
    return BLDTT_EINVAL;
  }
  std::vector<double> prefix(nleaves + 1, 0.0);
  for (int32_t i = 0; i < nleaves; ++i) {
    const double c = leaf_cost[i];
    if (!std::isfinite(c) || c < 0.0) {
      set_error("partition_leaves: cost of leaf %d is negative or not finite", i);
      return BLDTT_EINVAL;
    }
    prefix[i + 1] = prefix[i] + c;
  }
  if (!(prefix[nleaves] > 0.0))             // no cost at all: equal leaf counts
    for (int32_t i = 0; i <= nleaves; ++i) prefix[i] = (double)i;
  const double total = prefix[nleaves];
  leaf_begin[0] = 0;
  int32_t b = 0;
  for (int32_t k = 1; k < nshards; ++k) {
    const double target = total * (double)k / (double)nshards;
    while (b < nleaves && prefix[b + 1] <= target) ++b;       // prefix[b] <= target < prefix[b + 1]
    int32_t cut = b;
    if (b < nleaves && prefix[b + 1] - target < target - prefix[b]) cut = b + 1;   // the nearer boundary
    if (cut < leaf_begin[k - 1]) cut = leaf_begin[k - 1];
    leaf_begin[k] = cut;
  }
  leaf_begin[nshards] = nleaves;
  return BLDTT_OK;
}

extern "C" int bldtt_compute_shard(bldtt_plan* p, int shard, int nshards, double* phi, void* cuda_stream) {
  if (!p || !phi) {
    set_error("plan and phi must be non-NULL");
    return BLDTT_EINVAL;
  }
  if (nshards < 1 || shard < 0 || shard >= nshards) {
    set_error("compute_shard: shard %d outside [0, %d)", shard, nshards);
    return BLDTT_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  p->stream = s;
  p->compute_counter.launches = 0;
  if (nshards == 1) {
    p->computed_evals = p->interactions[0] + p->interactions[1] + p->interactions[2] + p->interactions[3];
    return compute_body(p, phi, s);
  }
  return compute_shard(p, shard, nshards, phi, s);
}
