// Tree building (Sec. 2.3), level by level on the device.
//
// Each level: decide the split of every cluster of the level (count rule and
// sqrt(2) aspect rule, midpoint of the shrunk box), cut every splitting
// cluster's particle range into fixed chunks, count the 8 child codes per
// chunk, turn the counts into stable destinations, scatter the particles
// (a stable 8-way partition, so particles keep input order inside each
// cluster), create the non-empty children and shrink each to the bounding
// box of its particles.  All geometric decisions are made in FP64 with
// explicitly rounded operations (no FMA contraction) so that they are the
// decisions a plain FP64 evaluation of the same expressions makes.
//
// The build works on a forest: level 0 holds one root per problem (a
// contiguous range of the particle array), and every level is processed for
// all problems at once, so a batch of independent problems costs one set of
// launches per level.
#include <algorithm>
#include <cstdlib>
#include <utility>

#include "internal.cuh"

namespace bldtt {

constexpr int kTreeChunk = 2048;
constexpr int kTreeThreads = 256;
static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Chebyshev point of the 2nd kind, s_k = cos(pi k / n), symmetrised so that
// s_0 = 1, s_n = -1, s_{n-k} = -s_k and s_{n/2} = 0 (Sec. 2.1, Eq. (4)).
__global__ void k_tree_init(const double* __restrict__ coords, int32_t n, double* __restrict__ x,
                            double* __restrict__ y, double* __restrict__ z,
                            int32_t* __restrict__ perm) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  x[i] = coords[i];
  y[i] = coords[(int64_t)n + i];
  z[i] = coords[2 * (int64_t)n + i];
  perm[i] = (int32_t)i;
}

// One root per problem: cluster p holds particles [offsets[p], offsets[p+1]).
__global__ void k_tree_roots(int32_t nroots, const int32_t* __restrict__ offsets,
                             int32_t* __restrict__ begin, int32_t* __restrict__ end,
                             int32_t* __restrict__ parent, int32_t* __restrict__ level,
                             int32_t* __restrict__ problem) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nroots) return;
  begin[p] = offsets[p];
  end[p] = offsets[p + 1];
  parent[p] = -1;
  level[p] = 0;
  problem[p] = p;
}

// Split decision of one cluster of cnt particles in box b (reading: leaf iff
// |C| <= M0 or all extents zero; up to 1/2/3 dims by the count rule; eligible
// iff L_d*L_d*2 >= L_max*L_max; longest eligible first, ties to the lower
// axis).  Returns the split mask (bit 4 >> d for dimension d) and the box
// midpoint.
__device__ __forceinline__ uint8_t decide_split(int64_t cnt, const double* b, int32_t max_leaf,
                                                double mid[3]) {
  double ext[3];
  for (int d = 0; d < 3; ++d) ext[d] = __dsub_rn(b[3 + d], b[d]);
  uint8_t mask = 0;
  if (cnt > (int64_t)max_leaf) {
    double lmax = fmax(fmax(ext[0], ext[1]), ext[2]);
    if (lmax > 0.0) {
      int cap = cnt <= 2 * (int64_t)max_leaf ? 1 : (cnt <= 4 * (int64_t)max_leaf ? 2 : 3);
      double lm2 = __dmul_rn(lmax, lmax);
      int o[3] = {0, 1, 2};
      for (int i = 0; i < 3; ++i)
        for (int k = i + 1; k < 3; ++k)
          if (ext[o[k]] > ext[o[i]] || (ext[o[k]] == ext[o[i]] && o[k] < o[i])) {
            int t = o[i]; o[i] = o[k]; o[k] = t;
          }
      int taken = 0;
      for (int i = 0; i < 3; ++i) {
        int d = o[i];
        bool eligible = __dmul_rn(__dmul_rn(ext[d], ext[d]), 2.0) >= lm2;
        if (eligible && taken < cap) {
          mask |= (uint8_t)(4 >> d);
          ++taken;
        }
      }
    }
  }
  for (int d = 0; d < 3; ++d) mid[d] = __dmul_rn(__dadd_rn(b[d], b[3 + d]), 0.5);
  return mask;
}

// Split decision of each cluster of the level.
__global__ void k_tree_decide(int32_t ls, int32_t nl, const int32_t* __restrict__ begin,
                              const int32_t* __restrict__ end, const double* __restrict__ box,
                              int32_t max_leaf, uint8_t* __restrict__ splitmask,
                              double* __restrict__ mid, int32_t* __restrict__ nchunks,
                              int32_t* __restrict__ first_child, int32_t* __restrict__ nchild,
                              int32_t* __restrict__ nsplit) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nl) return;
  int c = ls + j;
  int64_t cnt = (int64_t)end[c] - begin[c];
  first_child[c] = -1;
  nchild[c] = 0;
  double m[3];
  const uint8_t mask = decide_split(cnt, box + (int64_t)c * 6, max_leaf, m);
  splitmask[j] = mask;
  for (int d = 0; d < 3; ++d) mid[(int64_t)j * 3 + d] = m[d];
  // every cluster of the level is streamed: split ones are scattered to their
  // children, the others (leaves) copied to the same place of the other buffer
  nchunks[j] = (int32_t)((cnt + kTreeChunk - 1) / kTreeChunk);
  if (mask) atomicAdd(nsplit, 1);
}

__global__ void k_tree_chunks(int32_t nl, int32_t ls, const int32_t* __restrict__ chunk_off,
                              int32_t tc, const int32_t* __restrict__ begin,
                              int32_t* __restrict__ chunk_cluster, int32_t* __restrict__ chunk_start) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= tc) return;
  int lo = 0, hi = nl;   // first j with chunk_off[j] > q, minus one
  while (lo < hi) {
    int m = (lo + hi) >> 1;
    if (chunk_off[m] <= q) lo = m + 1; else hi = m;
  }
  int j = lo - 1;
  chunk_cluster[q] = j;
  chunk_start[q] = begin[ls + j] + (q - chunk_off[j]) * kTreeChunk;
}

// Child code of a particle: bit (4 >> d) set when coordinate d is at or above
// the midpoint (a plain FP64 comparison, done on the order-preserving keys).
__device__ __forceinline__ int child_code(double px, double py, double pz, uint8_t mask,
                                          const long long* mk) {
  int code = 0;
  if ((mask & 4) && okey(px) >= mk[0]) code |= 4;
  if ((mask & 2) && okey(py) >= mk[1]) code |= 2;
  if ((mask & 1) && okey(pz) >= mk[2]) code |= 1;
  return code;
}

__global__ void k_tree_count(int32_t ls, const int32_t* __restrict__ chunk_cluster,
                             const int32_t* __restrict__ chunk_start, const int32_t* __restrict__ end,
                             const double* __restrict__ x, const double* __restrict__ y,
                             const double* __restrict__ z, const uint8_t* __restrict__ splitmask,
                             const double* __restrict__ mid, uint8_t* __restrict__ code,
                             int32_t* __restrict__ counts) {
  __shared__ int32_t cnt[8];
  int q = blockIdx.x;
  int j = chunk_cluster[q];
  uint8_t mask = splitmask[j];
  if (!mask) return;   // a leaf's chunk: copied, not counted
  if (threadIdx.x < 8) cnt[threadIdx.x] = 0;
  __syncthreads();
  int32_t s0 = chunk_start[q];
  int32_t s1 = min(s0 + kTreeChunk, end[ls + j]);
  const long long mk[3] = {okey(mid[(int64_t)j * 3]), okey(mid[(int64_t)j * 3 + 1]),
                           okey(mid[(int64_t)j * 3 + 2])};
  const int lane = threadIdx.x & 31;
  for (int32_t i0 = s0; i0 < s1; i0 += blockDim.x) {   // warp-uniform trip count
    const int32_t i = i0 + threadIdx.x;
    const bool valid = i < s1;
    const int c = valid ? child_code(x[i], y[i], z[i], mask, mk) : 8;
    if (valid) code[i] = (uint8_t)c;
    const unsigned peers = __match_any_sync(0xffffffffu, c);
    if (valid && (peers & ((1u << lane) - 1u)) == 0) atomicAdd(&cnt[c], __popc(peers));
  }
  __syncthreads();
  if (threadIdx.x < 8) counts[(int64_t)q * 8 + threadIdx.x] = cnt[threadIdx.x];
}

// One CTA per splitting cluster: totals per child code, then stable
// destinations of every chunk's particles (exclusive scan over the chunks).
constexpr int kCombineThreads = 256;

__device__ __forceinline__ void block_scan8(const int32_t (&v)[8], int32_t (&ex)[8],
                                            int32_t (&tot)[8], int32_t (*warp_sums)[8]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t inc[8];
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    int32_t x = v[b];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, x, off);
      if (lane >= off) x += y;
    }
    inc[b] = x;
  }
  if (lane == 31)
    for (int b = 0; b < 8; ++b) warp_sums[warp][b] = inc[b];
  __syncthreads();
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    int32_t pre = 0, all = 0;
    for (int w = 0; w < kCombineThreads / 32; ++w) {
      int32_t ws = warp_sums[w][b];
      if (w < warp) pre += ws;
      all += ws;
    }
    ex[b] = pre + inc[b] - v[b];
    tot[b] = all;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kCombineThreads) k_tree_combine(
    int32_t ls, const uint8_t* __restrict__ splitmask, const int32_t* __restrict__ chunk_off,
    const int32_t* __restrict__ nchunks, const int32_t* __restrict__ counts,
    int32_t* __restrict__ chunk_base, int32_t* __restrict__ child_cnt, int32_t* __restrict__ nch,
    const int32_t* __restrict__ begin) {
  __shared__ int32_t warp_sums[kCombineThreads / 32][8];
  const int j = blockIdx.x;
  if (!splitmask[j]) {
    if (threadIdx.x == 0) nch[j] = 0;
    return;
  }
  const int32_t q0 = chunk_off[j], nq = nchunks[j];
  int32_t v[8], ex[8], tot[8], cb[8], run[8];
  // totals per code
  for (int b = 0; b < 8; ++b) v[b] = 0;
  for (int32_t t = threadIdx.x; t < nq; t += kCombineThreads)
    for (int b = 0; b < 8; ++b) v[b] += counts[(int64_t)(q0 + t) * 8 + b];
  block_scan8(v, ex, tot, warp_sums);
  int32_t pos = begin[ls + j];
  int k = 0;
  for (int b = 0; b < 8; ++b) {
    cb[b] = pos;
    pos += tot[b];
    run[b] = 0;
    k += tot[b] > 0;
  }
  if (threadIdx.x < 8) child_cnt[(int64_t)j * 8 + threadIdx.x] = tot[threadIdx.x];
  if (threadIdx.x == 0) nch[j] = k;
  // stable destinations: chunk-order exclusive scan per code
  for (int32_t base = 0; base < nq; base += kCombineThreads) {
    const int32_t t = base + threadIdx.x;
    for (int b = 0; b < 8; ++b) v[b] = t < nq ? counts[(int64_t)(q0 + t) * 8 + b] : 0;
    int32_t tile[8];
    block_scan8(v, ex, tile, warp_sums);
    if (t < nq)
      for (int b = 0; b < 8; ++b) chunk_base[(int64_t)(q0 + t) * 8 + b] = cb[b] + run[b] + ex[b];
    for (int b = 0; b < 8; ++b) run[b] += tile[b];
  }
}

__global__ void k_tree_children(int32_t nl, int32_t ls, int32_t le, int32_t lvl,
                                const uint8_t* __restrict__ splitmask,
                                const int32_t* __restrict__ child_off,
                                const int32_t* __restrict__ child_cnt, int32_t* __restrict__ begin,
                                int32_t* __restrict__ end, int32_t* __restrict__ parent,
                                int32_t* __restrict__ level, int32_t* __restrict__ first_child,
                                int32_t* __restrict__ nchild, int32_t* __restrict__ problem) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nl || !splitmask[j]) return;
  int c = ls + j;
  int32_t fc = le + child_off[j];
  int32_t pos = begin[c];
  int k = 0;
  for (int b = 0; b < 8; ++b) {
    int32_t cnt = child_cnt[(int64_t)j * 8 + b];
    if (cnt == 0) continue;
    int32_t id = fc + k++;
    begin[id] = pos;
    end[id] = pos + cnt;
    parent[id] = c;
    level[id] = lvl + 1;
    problem[id] = problem[c];
    pos += cnt;
  }
  first_child[c] = fc;
  nchild[c] = k;
}

// Stable scatter of the splitting chunk [s0, s1) by child code: particle i
// goes to base[code] + (its rank among the chunk's particles of that code).
// warp_cnt, running and base are shared arrays of the block; base[0..8) holds
// the chunk's destinations on entry.  Every thread of the block calls this.
template <typename Ld>
__device__ __forceinline__ void scatter_chunk(int32_t s0, int32_t s1, const uint8_t* __restrict__ code,
                                              const double* __restrict__ x, const double* __restrict__ y,
                                              const double* __restrict__ z, const int32_t* __restrict__ perm,
                                              double* __restrict__ x2, double* __restrict__ y2,
                                              double* __restrict__ z2, int32_t* __restrict__ perm2,
                                              int32_t (*warp_cnt)[9], int32_t* running, const int32_t* base,
                                              Ld ld) {
  constexpr int W = kTreeThreads / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // each step's particle is loaded one step ahead, so that its loads overlap
  // the block barriers of the step before
  int32_t i = s0 + threadIdx.x;
  bool valid = i < s1;
  double px = 0.0, py = 0.0, pz = 0.0;
  int32_t pp = 0;
  int d = 8;
  if (valid) {
    px = ld(x + i);
    py = ld(y + i);
    pz = ld(z + i);
    pp = ld(perm + i);
    d = code[i];
  }
  for (int r = 0; r < kTreeChunk / kTreeThreads; ++r) {
    const int32_t in = i + kTreeThreads;
    const bool vn = in < s1;
    double nx = 0.0, ny = 0.0, nz = 0.0;
    int32_t np = 0;
    int dn = 8;
    if (vn) {
      nx = ld(x + in);
      ny = ld(y + in);
      nz = ld(z + in);
      np = ld(perm + in);
      dn = code[in];
    }
    for (int k = threadIdx.x; k < W * 9; k += kTreeThreads) (&warp_cnt[0][0])[k] = 0;
    __syncthreads();
    unsigned peers = __match_any_sync(0xffffffffu, d);
    int rank = __popc(peers & ((1u << lane) - 1u));
    if (rank == 0) warp_cnt[warp][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      int32_t dst = base[d] + running[d] + rank;
      for (int w = 0; w < warp; ++w) dst += warp_cnt[w][d];
      x2[dst] = px;
      y2[dst] = py;
      z2[dst] = pz;
      perm2[dst] = pp;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
      int32_t t = 0;
      for (int w = 0; w < W; ++w) t += warp_cnt[w][threadIdx.x];
      running[threadIdx.x] += t;
    }
    __syncthreads();
    i = in;
    valid = vn;
    px = nx;
    py = ny;
    pz = nz;
    pp = np;
    d = dn;
  }
}

struct LdPlain {
  template <typename T>
  __device__ T operator()(const T* p) const { return *p; }
};
struct LdCg {   // bypasses L1: data written by other blocks of the same launch
  template <typename T>
  __device__ T operator()(const T* p) const { return __ldcg(p); }
};

__global__ void k_tree_scatter(int32_t ls, const int32_t* __restrict__ chunk_cluster,
                               const int32_t* __restrict__ chunk_start,
                               const int32_t* __restrict__ end, const uint8_t* __restrict__ splitmask,
                               const uint8_t* __restrict__ code,
                               const int32_t* __restrict__ chunk_base, const double* __restrict__ x,
                               const double* __restrict__ y, const double* __restrict__ z,
                               const int32_t* __restrict__ perm, double* __restrict__ x2,
                               double* __restrict__ y2, double* __restrict__ z2,
                               int32_t* __restrict__ perm2) {
  constexpr int W = kTreeThreads / 32;
  __shared__ int32_t warp_cnt[W][9];
  __shared__ int32_t running[8];
  __shared__ int32_t base[8];
  int q = blockIdx.x;
  int32_t s0 = chunk_start[q];
  int32_t s1 = min(s0 + kTreeChunk, end[ls + chunk_cluster[q]]);
  if (!splitmask[chunk_cluster[q]]) {   // a leaf: same positions in the other buffer
    for (int32_t i = s0 + threadIdx.x; i < s1; i += blockDim.x) {
      x2[i] = x[i];
      y2[i] = y[i];
      z2[i] = z[i];
      perm2[i] = perm[i];
    }
    return;
  }
  if (threadIdx.x < 8) {
    running[threadIdx.x] = 0;
    base[threadIdx.x] = chunk_base[(int64_t)q * 8 + threadIdx.x];
  }
  scatter_chunk(s0, s1, code, x, y, z, perm, x2, y2, z2, perm2, warp_cnt, running, base, LdPlain());
}

// Shrink every new cluster to the bounding box of its particles (Sec. 2.3):
// every cluster is cut into slices of kBoxSlice particles (at least one), one
// CTA per slice (the slice's cluster found by binary search in the prefix of
// slice counts, which stays on the device), then one warp per cluster
// combines its slices.  Min/max are exact, so the result does not depend on
// the cut.  Slices per cluster follow its own size, so one very populous
// cluster (a Plummer core) still spreads over many CTAs.
constexpr int kBoxSlice = 8192;

__global__ void k_box_slices(int32_t first, int32_t nc, const int32_t* __restrict__ begin,
                             const int32_t* __restrict__ end, int32_t* __restrict__ nslice) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nc) return;
  const int32_t cnt = end[first + j] - begin[first + j];
  nslice[j] = cnt > kBoxSlice ? (cnt + kBoxSlice - 1) / kBoxSlice : 1;
}

__global__ void k_tree_child_bbox(int32_t first, int32_t nc, const int32_t* __restrict__ slice_off,
                                  const int32_t* __restrict__ nslice, const int32_t* __restrict__ begin,
                                  const int32_t* __restrict__ end, const double* __restrict__ x,
                                  const double* __restrict__ y, const double* __restrict__ z,
                                  double* __restrict__ part) {
  const int32_t b = blockIdx.x;
  if (b >= slice_off[nc - 1] + nslice[nc - 1]) return;
  int lo_j = 0, hi_j = nc;   // last cluster whose first slice is <= b
  while (hi_j - lo_j > 1) {
    const int m = (lo_j + hi_j) >> 1;
    if (slice_off[m] <= b) lo_j = m; else hi_j = m;
  }
  const int c = first + lo_j;
  const int32_t s0 = begin[c] + (b - slice_off[lo_j]) * kBoxSlice;
  const int32_t s1 = min(end[c], s0 + kBoxSlice);
  // exact minima and maxima, on the order-preserving keys
  long long lo[3] = {kKeyPosInf, kKeyPosInf, kKeyPosInf}, hi[3] = {kKeyNegInf, kKeyNegInf, kKeyNegInf};
  for (int32_t i = s0 + threadIdx.x; i < s1; i += blockDim.x) {
    const long long v[3] = {okey(x[i]), okey(y[i]), okey(z[i])};
    for (int d = 0; d < 3; ++d) {
      lo[d] = min(lo[d], v[d]);
      hi[d] = max(hi[d], v[d]);
    }
  }
  __shared__ long long sm[kTreeThreads / 32][6];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = 0; d < 3; ++d)
    for (int off = 16; off; off >>= 1) {
      lo[d] = min(lo[d], __shfl_down_sync(0xffffffffu, lo[d], off));
      hi[d] = max(hi[d], __shfl_down_sync(0xffffffffu, hi[d], off));
    }
  if (lane == 0)
    for (int d = 0; d < 3; ++d) {
      sm[warp][d] = lo[d];
      sm[warp][3 + d] = hi[d];
    }
  __syncthreads();
  if (threadIdx.x < 6) {
    long long r = sm[0][threadIdx.x];
    for (int w = 1; w < kTreeThreads / 32; ++w)
      r = threadIdx.x < 3 ? min(r, sm[w][threadIdx.x]) : max(r, sm[w][threadIdx.x]);
    part[(int64_t)b * 6 + threadIdx.x] = okey_inv(r);
  }
}

__global__ void k_tree_child_bbox_combine(int32_t first, int32_t nc, const int32_t* __restrict__ slice_off,
                                          const int32_t* __restrict__ nslice,
                                          const double* __restrict__ part, double* __restrict__ box) {
  const int j = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= nc) return;
  const int32_t p0 = slice_off[j], ns = nslice[j];
  for (int k = 0; k < 6; ++k) {
    double r = k < 3 ? INFINITY : -INFINITY;
    for (int32_t t = lane; t < ns; t += 32) {
      const double v = part[(int64_t)(p0 + t) * 6 + k];
      r = k < 3 ? fmin(r, v) : fmax(r, v);
    }
    for (int off = 16; off; off >>= 1) {
      double o = __shfl_down_sync(0xffffffffu, r, off);
      r = k < 3 ? fmin(r, o) : fmax(r, o);
    }
    if (lane == 0) box[(int64_t)(first + j) * 6 + k] = r;
  }
}

// Bounding boxes of the nc clusters [first, first + nc) of a tree of n particles.
static int cluster_boxes(Tree& T, int32_t first, int32_t nc, int32_t n, cudaStream_t s, Counters& cnt) {
  int32_t *nslice = nullptr, *slice_off = nullptr;
  double* part = nullptr;
  const int64_t bound = (int64_t)n / kBoxSlice + nc + 1;   // slices <= n / kBoxSlice + nc
  BL_TRY(dalloc_n(&nslice, nc, s));
  BL_TRY(dalloc_n(&slice_off, nc, s));
  BL_TRY(dalloc_n(&part, (size_t)bound * 6, s));
  k_box_slices<<<nblk(nc, 128), 128, 0, s>>>(first, nc, T.begin, T.end, nslice);
  BL_LAUNCHED(cnt.launches);
  BL_TRY(scan_exclusive(nslice, slice_off, nc, nullptr, s, cnt));
  k_tree_child_bbox<<<(unsigned)bound, kTreeThreads, 0, s>>>(first, nc, slice_off, nslice, T.begin, T.end,
                                                             T.x, T.y, T.z, part);
  BL_LAUNCHED(cnt.launches);
  k_tree_child_bbox_combine<<<nblk(nc, 4), 128, 0, s>>>(first, nc, slice_off, nslice, part, T.box);
  BL_LAUNCHED(cnt.launches);
  dfree(part, s);
  dfree(slice_off, s);
  dfree(nslice, s);
  return BLDTT_OK;
}

// Centre = box centre, radius = half the diagonal, proxy points c + h s_k.
__global__ void k_tree_geometry(int32_t C, int degree, const double* __restrict__ box,
                                double* __restrict__ center, double* __restrict__ radius,
                                double* __restrict__ nodes) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  const int P = degree + 1;
  const double* b = box + (int64_t)c * 6;
  double e[3];
  for (int d = 0; d < 3; ++d) {
    double lo = b[d], hi = b[3 + d];
    double cc = __dmul_rn(__dadd_rn(lo, hi), 0.5);
    double h = __dmul_rn(__dsub_rn(hi, lo), 0.5);
    e[d] = __dsub_rn(hi, lo);
    center[(int64_t)c * 3 + d] = cc;
    for (int k = 0; k < P; ++k)
      nodes[((int64_t)c * 3 + d) * P + k] = __dadd_rn(cc, __dmul_rn(h, cheb_point(k, degree)));
  }
  double s2 = __dadd_rn(__dadd_rn(__dmul_rn(e[0], e[0]), __dmul_rn(e[1], e[1])), __dmul_rn(e[2], e[2]));
  radius[c] = __dmul_rn(__dsqrt_rn(s2), 0.5);
}

__global__ void k_tree_leaf_flags(int32_t C, const int32_t* __restrict__ nchild,
                                  const int32_t* __restrict__ begin, int32_t* __restrict__ flag) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < C && nchild[c] == 0) flag[begin[c]] = 1;
}

__global__ void k_tree_leaf_order(int32_t C, int32_t n, int32_t nleaves,
                                  const int32_t* __restrict__ nchild,
                                  const int32_t* __restrict__ begin, const int32_t* __restrict__ end,
                                  const int32_t* __restrict__ excl, int32_t* __restrict__ leaf_ids,
                                  int32_t* __restrict__ leaf_first, int32_t* __restrict__ leaf_last) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  leaf_first[c] = excl[begin[c]];
  leaf_last[c] = end[c] < n ? excl[end[c]] : nleaves;
  if (nchild[c] == 0) leaf_ids[excl[begin[c]]] = c;
}

static int grow_clusters(Tree& T, size_t need, size_t keep, cudaStream_t s) {
  if (need <= T.cap && T.begin) return BLDTT_OK;
  size_t ncap = T.cap ? T.cap : 64;
  while (ncap < need) ncap *= 2;
  int32_t** iarr[7] = {&T.begin, &T.end, &T.parent, &T.first_child, &T.nchild, &T.level,
                       &T.problem};
  for (auto a : iarr) {
    size_t c = T.cap;
    BL_TRY(dgrow(a, &c, ncap, keep, s));
  }
  size_t c6 = T.cap * 6;
  BL_TRY(dgrow(&T.box, &c6, ncap * 6, keep * 6, s));
  T.cap = ncap;
  return BLDTT_OK;
}


// Levels past this many mean a cluster that the midpoint rule cannot
// separate (e.g. more than max_leaf points on two adjacent doubles whose
// midpoint rounds to the lower one); the build stops with an error.
constexpr int kMaxTreeLevels = 2048;

int build_tree(Tree& T, const double* coords, int32_t n, const std::vector<int32_t>& roots,
               int32_t max_leaf, int degree, cudaStream_t s, Counters& cnt) {
  T.n = n;
  double *x2 = nullptr, *y2 = nullptr, *z2 = nullptr;
  int32_t* perm2 = nullptr;
  uint8_t* code = nullptr;
  BL_TRY(dalloc_n(&T.x, n, s));
  BL_TRY(dalloc_n(&T.y, n, s));
  BL_TRY(dalloc_n(&T.z, n, s));
  BL_TRY(dalloc_n(&T.perm, n, s));
  BL_TRY(dalloc_n(&x2, n, s));
  BL_TRY(dalloc_n(&y2, n, s));
  BL_TRY(dalloc_n(&z2, n, s));
  BL_TRY(dalloc_n(&perm2, n, s));
  BL_TRY(dalloc_n(&code, n, s));
  k_tree_init<<<nblk(n, 256), 256, 0, s>>>(coords, n, T.x, T.y, T.z, T.perm);
  BL_LAUNCHED(cnt.launches);
  const int32_t nroots = (int32_t)roots.size() - 1;
  BL_TRY(grow_clusters(T, std::max<size_t>(1024, 2 * (size_t)nroots), 0, s));
  {
    int32_t* d_roots = nullptr;
    BL_TRY(dalloc_n(&d_roots, roots.size(), s));
    BL_CUDA(cudaMemcpyAsync(d_roots, roots.data(), roots.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice, s));
    k_tree_roots<<<nblk(nroots, 128), 128, 0, s>>>(nroots, d_roots, T.begin, T.end, T.parent,
                                                   T.level, T.problem);
    BL_LAUNCHED(cnt.launches);
    // root boxes: the minimal bounding box of each problem's particles (Sec. 2.3)
    BL_TRY(cluster_boxes(T, 0, nroots, n, s, cnt));
    dfree(d_roots, s);
  }

  T.level_start.assign({0, nroots});
  T.nroots = nroots;
  // per-level scratch, grown with the level (nl clusters, tc particle chunks)
  uint8_t* splitmask = nullptr;
  double* mid = nullptr;
  int32_t *nchunks = nullptr, *chunk_off = nullptr, *chunk_cluster = nullptr, *chunk_start = nullptr,
          *counts = nullptr, *chunk_base = nullptr, *child_cnt = nullptr, *nch = nullptr,
          *child_off = nullptr;
  size_t c_sm = 0, c_mid = 0, c_nq = 0, c_qo = 0, c_qc = 0, c_qs = 0, c_cnt = 0, c_cb = 0, c_cc = 0,
         c_nch = 0, c_co = 0;
  int32_t* tot2 = nullptr;   // [0] chunks of the level, [1] clusters that split
  BL_TRY(dalloc_n(&tot2, 2, s));
  // Particles of a cluster that stays a leaf are copied into the other buffer
  // at its level, so both buffers hold them from then on and later levels only
  // touch the clusters they split.
  int status = BLDTT_OK;
  for (int lvl = 0;; ++lvl) {
    if (lvl >= kMaxTreeLevels) {   // only clusters that no midpoint split separates get here
      set_error("tree deeper than %d levels: some cluster is not separated by its midpoints",
                kMaxTreeLevels);
      status = BLDTT_EINTERNAL;
      break;
    }
    int32_t ls = T.level_start[lvl], le = T.level_start[lvl + 1], nl = le - ls;
    BL_TRY(dgrow(&splitmask, &c_sm, (size_t)nl, 0, s));
    BL_TRY(dgrow(&mid, &c_mid, (size_t)nl * 3, 0, s));
    BL_TRY(dgrow(&nchunks, &c_nq, (size_t)nl, 0, s));
    BL_TRY(dgrow(&chunk_off, &c_qo, (size_t)nl, 0, s));
    BL_CUDA(cudaMemsetAsync(tot2 + 1, 0, sizeof(int32_t), s));
    k_tree_decide<<<nblk(nl, 128), 128, 0, s>>>(ls, nl, T.begin, T.end, T.box, max_leaf, splitmask,
                                                mid, nchunks, T.first_child, T.nchild, tot2 + 1);
    BL_LAUNCHED(cnt.launches);
    BL_TRY(scan_exclusive_dev(nchunks, chunk_off, nl, tot2, s, cnt));
    int32_t h2[2];
    BL_TRY(read_device(tot2, h2, sizeof(h2), s));
    const int32_t tc = h2[0];
    if (h2[1] == 0) break;   // no cluster of this level splits
    BL_TRY(dgrow(&chunk_cluster, &c_qc, (size_t)tc, 0, s));
    BL_TRY(dgrow(&chunk_start, &c_qs, (size_t)tc, 0, s));
    BL_TRY(dgrow(&counts, &c_cnt, (size_t)tc * 8, 0, s));
    BL_TRY(dgrow(&chunk_base, &c_cb, (size_t)tc * 8, 0, s));
    BL_TRY(dgrow(&child_cnt, &c_cc, (size_t)nl * 8, 0, s));
    BL_TRY(dgrow(&nch, &c_nch, (size_t)nl, 0, s));
    BL_TRY(dgrow(&child_off, &c_co, (size_t)nl, 0, s));
    k_tree_chunks<<<nblk(tc, 256), 256, 0, s>>>(nl, ls, chunk_off, tc, T.begin, chunk_cluster,
                                                chunk_start);
    BL_LAUNCHED(cnt.launches);
    k_tree_count<<<tc, kTreeThreads, 0, s>>>(ls, chunk_cluster, chunk_start, T.end, T.x, T.y, T.z,
                                             splitmask, mid, code, counts);
    BL_LAUNCHED(cnt.launches);
    k_tree_combine<<<nl, kCombineThreads, 0, s>>>(ls, splitmask, chunk_off, nchunks, counts,
                                                  chunk_base, child_cnt, nch, T.begin);
    BL_LAUNCHED(cnt.launches);
    int32_t nc = 0;
    BL_TRY(scan_exclusive(nch, child_off, nl, &nc, s, cnt));
    BL_TRY(grow_clusters(T, (size_t)le + nc, (size_t)le, s));
    k_tree_children<<<nblk(nl, 128), 128, 0, s>>>(nl, ls, le, lvl, splitmask, child_off, child_cnt,
                                                  T.begin, T.end, T.parent, T.level, T.first_child,
                                                  T.nchild, T.problem);
    BL_LAUNCHED(cnt.launches);
    k_tree_scatter<<<tc, kTreeThreads, 0, s>>>(ls, chunk_cluster, chunk_start, T.end, splitmask, code,
                                               chunk_base, T.x, T.y, T.z, T.perm, x2, y2, z2, perm2);
    BL_LAUNCHED(cnt.launches);
    { double* t = T.x; T.x = x2; x2 = t; }
    { double* t = T.y; T.y = y2; y2 = t; }
    { double* t = T.z; T.z = z2; z2 = t; }
    { int32_t* t = T.perm; T.perm = perm2; perm2 = t; }
    BL_TRY(cluster_boxes(T, le, nc, n, s, cnt));
    T.level_start.push_back(le + nc);
  }
  dfree(splitmask, s); dfree(mid, s); dfree(nchunks, s); dfree(chunk_off, s);
  dfree(chunk_cluster, s); dfree(chunk_start, s); dfree(counts, s); dfree(chunk_base, s);
  dfree(child_cnt, s); dfree(nch, s); dfree(child_off, s); dfree(tot2, s);
  if (status != BLDTT_OK) {
    dfree(x2, s); dfree(y2, s); dfree(z2, s); dfree(perm2, s); dfree(code, s);
    return status;
  }
  dfree(x2, s); dfree(y2, s); dfree(z2, s); dfree(perm2, s); dfree(code, s);

  T.nclusters = T.level_start.back();
  T.nlevels = (int32_t)T.level_start.size() - 1;
  const int C = T.nclusters;
  BL_TRY(dalloc_n(&T.center, (size_t)C * 3, s));
  BL_TRY(dalloc_n(&T.radius, (size_t)C, s));
  BL_TRY(dalloc_n(&T.nodes, (size_t)C * 3 * (degree + 1), s));
  k_tree_geometry<<<nblk(C, 128), 128, 0, s>>>(C, degree, T.box, T.center, T.radius, T.nodes);
  BL_LAUNCHED(cnt.launches);

  int32_t *flag = nullptr, *excl = nullptr;
  BL_TRY(dalloc_n(&flag, n, s));
  BL_TRY(dalloc_n(&excl, n, s));
  BL_CUDA(cudaMemsetAsync(flag, 0, (size_t)n * 4, s));
  k_tree_leaf_flags<<<nblk(C, 128), 128, 0, s>>>(C, T.nchild, T.begin, flag);
  BL_LAUNCHED(cnt.launches);
  int32_t nleaves = 0;
  BL_TRY(scan_exclusive(flag, excl, n, &nleaves, s, cnt));
  T.nleaves = nleaves;
  BL_TRY(dalloc_n(&T.leaf_ids, nleaves, s));
  BL_TRY(dalloc_n(&T.leaf_first, C, s));
  BL_TRY(dalloc_n(&T.leaf_last, C, s));
  k_tree_leaf_order<<<nblk(C, 128), 128, 0, s>>>(C, n, nleaves, T.nchild, T.begin, T.end, excl,
                                                 T.leaf_ids, T.leaf_first, T.leaf_last);
  BL_LAUNCHED(cnt.launches);
  dfree(flag, s);
  dfree(excl, s);
  return BLDTT_OK;
}

// ---------------------------------------------------------------------------
// The whole build in one cooperative launch
// ---------------------------------------------------------------------------
// k_tree_all runs the build above without returning to the host: the roots'
// boxes, then every level (split decisions, child counts, stable scatter),
// then the leaf order, separated by grid barriers (all blocks are co-resident
// in a cooperative launch; every barrier wait is bounded).  The decisions,
// the scatter and hence the tree are those of the level-by-level kernels:
// the same device functions make them.  Two things differ in how, not what:
// the children's boxes are reduced per chunk of the scattered order (each
// chunk holds whole runs of children; exact minima and maxima of the
// order-preserving keys, folded together by atomics), and the leaf order
// comes from subtree leaf counts instead of a scan over particles.
//
// Key boxes: entry e holds 6 unsigned words, the complements of the flipped
// keys of the minima (x, y, z) and the flipped keys of the maxima, so that
// every update is an atomicMax and zero is the empty box.
constexpr int kTreeCoopThreads = kTreeThreads;
constexpr int kTreeMaxBlocks = 1024;
constexpr uint64_t kTreeWaitNs = 5000000000ull;   // bound on one grid barrier wait (5 s)
constexpr int kTreeHeadLevels = 232;              // level starts carried in the result header
constexpr int kWideCombine = 64;                  // clusters of more chunks are combined block-wide

struct TreeGrid {
  unsigned count, gen;   // barrier
  int32_t status;        // -1 running, 0 done, 1 clusters would exceed the capacity, 2 a barrier
                         // gave up, 3 deeper than kMaxTreeLevels, 4 a non-finite input value
  int32_t level;         // resume: the level to (re)process; done: the last level
  int32_t parity;        // coordinate buffer holding that level's order
  int32_t need;          // status 1: clusters needed
  int32_t nleaves;
  int32_t bad;           // set by any block that met a non-finite value
  int32_t level_start[kTreeHeadLevels];   // first kTreeHeadLevels level starts
};
static_assert(sizeof(TreeGrid) <= kPinnedSlot, "the result header is read through one pinned slot");

struct TreeCoop {
  int32_t *begin, *end, *parent, *first_child, *nchild, *level, *problem;
  double* box;
  int32_t cap;                                   // cluster capacity of every per-cluster array
  const double* coords;                          // input, SoA [3][n]
  int32_t n;
  double *x0, *y0, *z0, *x1, *y1, *z1;
  int32_t *perm0, *perm1;
  uint8_t* code;
  const int32_t* roots;                          // [nroots + 1] particle offsets
  int32_t nroots;
  const double* charges;                         // checked for finite values (may be null)
  int64_t ncharges;
  int32_t max_leaf;
  uint8_t* mask;                                 // per cluster of the level, [cap]
  long long* midk;                               // [cap][3] midpoint keys
  int32_t *coff, *nchk, *child_cnt, *nch, *chof;   // chunk offsets (block-local), chunks, [cap][8], children
  int32_t *chunk_cluster, *chunk_start, *counts, *chunk_base;   // per chunk, [qcap], [qcap][8]
  int32_t qcap;
  unsigned long long *kbox0, *kbox1;             // [8 cap][6] key boxes (by level parity)
  int32_t* bsrc;                                 // [cap] cluster -> its key box entry
  int32_t *nsub, *leaf_ids, *leaf_first, *leaf_last;
  int2* part;                                    // [grid] per-block chunk and split counts
  int32_t* part2;                                // [grid] per-block child counts
  int32_t* level_start;                          // [kMaxTreeLevels + 2]
  TreeGrid* g;
};

__device__ __forceinline__ uint64_t tree_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ bool tree_grid_sync(TreeGrid* g, unsigned nblocks) {
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
      const uint64_t t0 = tree_ns();
      while (*vgen == gen0) {
        if (tree_ns() - t0 > kTreeWaitNs) {
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

__device__ __forceinline__ unsigned long long flip_key(double v) {
  return (unsigned long long)okey(v) ^ 0x8000000000000000ull;
}
__device__ __forceinline__ double unflip_key(unsigned long long u) {
  return okey_inv((long long)(u ^ 0x8000000000000000ull));
}

// Block-wide exclusive scan of two counts; totals in *ta, *tb.
__device__ __forceinline__ void tree_block_scan2(int32_t a, int32_t b, int32_t* xa, int32_t* xb,
                                                 int32_t* ta, int32_t* tb) {
  __shared__ int32_t wa[kTreeCoopThreads / 32], wb[kTreeCoopThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t ia = a, ib = b;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t u = __shfl_up_sync(0xffffffffu, ia, o), v = __shfl_up_sync(0xffffffffu, ib, o);
    if (lane >= o) {
      ia += u;
      ib += v;
    }
  }
  if (lane == 31) {
    wa[warp] = ia;
    wb[warp] = ib;
  }
  __syncthreads();
  int32_t pa = 0, pb = 0, sa = 0, sb = 0;
  for (int w = 0; w < kTreeCoopThreads / 32; ++w) {
    if (w < warp) {
      pa += wa[w];
      pb += wb[w];
    }
    sa += wa[w];
    sb += wb[w];
  }
  *xa = pa + ia - a;
  *xb = pb + ib - b;
  *ta = sa;
  *tb = sb;
  __syncthreads();
}

// pre[0..G] = exclusive prefix of v(0..G-1) (per-block counts), in shared memory.
template <typename F>
__device__ __forceinline__ void block_prefix(unsigned G, int32_t* pre, F v) {
  int32_t run = 0;
  for (unsigned base = 0; base < G; base += kTreeCoopThreads) {
    const unsigned i = base + threadIdx.x;
    const int32_t x = i < G ? v(i) : 0;
    int32_t xa, xb, ta, tb;
    tree_block_scan2(x, 0, &xa, &xb, &ta, &tb);
    if (i < G) pre[i] = run + xa;
    run += ta;
  }
  if (threadIdx.x == 0) pre[G] = run;
  __syncthreads();
}

// Last index k in [lo, hi) with key(k) <= q (key non-decreasing, key(lo) <= q).
template <typename F>
__device__ __forceinline__ int32_t last_le(int32_t lo, int32_t hi, int64_t q, F key) {
  while (hi - lo > 1) {
    const int32_t m = (lo + hi) >> 1;
    if (key(m) <= q) lo = m; else hi = m;
  }
  return lo;
}

// Exact box of particles [a, b) folded into key box kb (flipped keys; the
// block's threads all call this and thread 0 issues the atomics).
__device__ void box_keys_of_range(int32_t a, int32_t b, const double* __restrict__ x,
                                  const double* __restrict__ y, const double* __restrict__ z,
                                  unsigned long long* __restrict__ kb) {
  __shared__ unsigned long long sm[kTreeCoopThreads / 32][6];
  unsigned long long m[6] = {0, 0, 0, 0, 0, 0};
  for (int32_t i = a + threadIdx.x; i < b; i += kTreeCoopThreads) {
    const unsigned long long u[3] = {flip_key(__ldcg(x + i)), flip_key(__ldcg(y + i)), flip_key(__ldcg(z + i))};
    for (int d = 0; d < 3; ++d) {
      m[d] = max(m[d], ~u[d]);
      m[3 + d] = max(m[3 + d], u[d]);
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < 6; ++k)
    for (int o = 16; o; o >>= 1) m[k] = max(m[k], __shfl_down_sync(0xffffffffu, m[k], o));
  if (lane == 0)
    for (int k = 0; k < 6; ++k) sm[warp][k] = m[k];
  __syncthreads();
  if (threadIdx.x < 6) {
    unsigned long long r = 0;
    for (int w = 0; w < kTreeCoopThreads / 32; ++w) r = max(r, sm[w][threadIdx.x]);
    if (b > a) atomicMax(kb + threadIdx.x, r);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kTreeCoopThreads, 4) k_tree_all(TreeCoop p) {
  __shared__ int32_t pq[kTreeMaxBlocks + 1];   // per-block chunk prefix of the level
  __shared__ int32_t pc[kTreeMaxBlocks + 1];   // per-block child prefix of the level
  __shared__ int32_t s_cnt[8];
  __shared__ int32_t s_ws[kTreeCoopThreads / 32][8];   // block_scan8 workspace
  __shared__ int32_t warp_cnt[kTreeThreads / 32][9];
  __shared__ int32_t running[8], s_base[8];
  const unsigned G = gridDim.x, b = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  TreeGrid* g = p.g;
  int L = __ldcg(&g->level);
  int par = __ldcg(&g->parity);
  const int64_t gthreads = (int64_t)G * kTreeCoopThreads;
  const int64_t gtid = (int64_t)b * kTreeCoopThreads + threadIdx.x;

  if (L == 0 && par == 0) {
    // ---- prologue: particles into buffer 0, the roots and their boxes ----
    bool bad = false;
    for (int64_t i = gtid; i < p.n; i += gthreads) {
      const double vx = p.coords[i], vy = p.coords[(int64_t)p.n + i], vz = p.coords[2 * (int64_t)p.n + i];
      bad |= !isfinite(vx) || !isfinite(vy) || !isfinite(vz);
      p.x0[i] = vx;
      p.y0[i] = vy;
      p.z0[i] = vz;
      p.perm0[i] = (int32_t)i;
    }
    for (int64_t i = gtid; i < p.ncharges; i += gthreads) bad |= !isfinite(p.charges[i]);
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicExch(&g->bad, 1);
    for (int64_t r = gtid; r < p.nroots; r += gthreads) {
      p.begin[r] = p.roots[r];
      p.end[r] = p.roots[r + 1];
      p.parent[r] = -1;
      p.level[r] = 0;
      p.problem[r] = (int32_t)r;
      p.bsrc[r] = (int32_t)r * 8;
    }
    if (b == 0 && threadIdx.x == 0) {
      p.level_start[0] = g->level_start[0] = 0;
      p.level_start[1] = g->level_start[1] = p.nroots;
    }
    // root boxes: chunks of the particle array, each folded into the roots it overlaps
    const int64_t nq = ((int64_t)p.n + kTreeChunk - 1) / kTreeChunk;
    for (int64_t q = b; q < nq; q += G) {
      const int32_t s0 = (int32_t)(q * kTreeChunk), s1 = (int32_t)min((int64_t)p.n, (q + 1) * kTreeChunk);
      int32_t r = last_le(0, p.nroots, s0, [&](int32_t k) { return (int64_t)p.roots[k]; });
      for (; r < p.nroots && p.roots[r] < s1; ++r) {
        const int32_t a = max(s0, p.roots[r]), e = min(s1, p.roots[r + 1]);
        box_keys_of_range(a, e, p.coords, p.coords + p.n, p.coords + 2 * (int64_t)p.n,
                          p.kbox0 + (int64_t)r * 8 * 6);
      }
    }
    if (!tree_grid_sync(g, G)) return;
    if (__ldcg(&g->bad)) {
      if (b == 0 && threadIdx.x == 0) atomicExch(&g->status, 4);
      return;
    }
  }

  for (;; ++L, par ^= 1) {
    const int32_t ls = __ldcg(p.level_start + L), le = __ldcg(p.level_start + L + 1), nl = le - ls;
    const double* x = par ? p.x1 : p.x0;
    const double* y = par ? p.y1 : p.y0;
    const double* z = par ? p.z1 : p.z0;
    const int32_t* perm = par ? p.perm1 : p.perm0;
    double* x2 = par ? p.x0 : p.x1;
    double* y2 = par ? p.y0 : p.y1;
    double* z2 = par ? p.z0 : p.z1;
    int32_t* perm2 = par ? p.perm0 : p.perm1;
    const unsigned long long* kcur = (L & 1) ? p.kbox1 : p.kbox0;
    unsigned long long* knext = (L & 1) ? p.kbox0 : p.kbox1;
    const int32_t jlo = (int32_t)((int64_t)nl * b / G), jhi = (int32_t)((int64_t)nl * (b + 1) / G);

    // ---- 1. boxes of the level's clusters, split decisions, chunk counts ----
    int32_t run_q = 0, run_s = 0;
    for (int32_t base = jlo; base < jhi; base += kTreeCoopThreads) {   // block-uniform trip count
      const int32_t j = base + threadIdx.x;
      int32_t nq = 0, sp = 0;
      if (j < jhi) {
        const int32_t c = ls + j;
        const unsigned long long* kb = kcur + (int64_t)__ldcg(p.bsrc + c) * 6;
        double bx[6];
        for (int d = 0; d < 3; ++d) {
          bx[d] = unflip_key(~__ldcg(kb + d));
          bx[3 + d] = unflip_key(__ldcg(kb + 3 + d));
        }
        for (int k = 0; k < 6; ++k) p.box[(int64_t)c * 6 + k] = bx[k];
        const int64_t cnt = (int64_t)__ldcg(p.end + c) - __ldcg(p.begin + c);
        double mid[3];
        const uint8_t mask = decide_split(cnt, bx, p.max_leaf, mid);
        p.mask[j] = mask;
        for (int d = 0; d < 3; ++d) p.midk[(int64_t)j * 3 + d] = okey(mid[d]);
        p.first_child[c] = -1;
        p.nchild[c] = 0;
        nq = (int32_t)((cnt + kTreeChunk - 1) / kTreeChunk);
        p.nchk[j] = nq;
        sp = mask ? 1 : 0;
        if (mask)
          for (int k = 0; k < 48; ++k) knext[(int64_t)j * 48 + k] = 0ull;
      }
      int32_t xq, xs, tq, ts;
      tree_block_scan2(nq, sp, &xq, &xs, &tq, &ts);
      if (j < jhi) p.coff[j] = run_q + xq;
      run_q += tq;
      run_s += ts;
    }
    if (threadIdx.x == 0) p.part[b] = make_int2(run_q, run_s);
    if (!tree_grid_sync(g, G)) return;
    block_prefix(G, pq, [&](unsigned i) { return __ldcg(&p.part[i].x); });
    {
      int32_t splits = 0;
      for (unsigned i = threadIdx.x; i < G; i += kTreeCoopThreads) splits += __ldcg(&p.part[i].y);
      splits = __syncthreads_or(splits != 0);
      if (!splits) break;                     // no cluster of this level splits
    }
    const int32_t TC = pq[G];
    if (TC > p.qcap) {                        // cannot happen: qcap >= n / kTreeChunk + cap
      if (b == 0 && threadIdx.x == 0) atomicExch(&g->status, 1);
      return;
    }
    // cluster j of chunk q: the block whose chunk range holds q, then its cluster
    auto cluster_of = [&](int32_t q, int32_t* qstart) {
      const int32_t bb = last_le(0, (int32_t)G, q, [&](int32_t k) { return (int64_t)pq[k]; });
      // blocks with no chunks share pq with their successor: take the last block at or below q
      const int32_t blo = (int32_t)((int64_t)nl * bb / G), bhi = (int32_t)((int64_t)nl * (bb + 1) / G);
      const int32_t j = last_le(blo, bhi, q, [&](int32_t k) { return (int64_t)pq[bb] + __ldcg(p.coff + k); });
      *qstart = pq[bb] + __ldcg(p.coff + j);
      return j;
    };

    // ---- 2. child codes and counts per chunk (two particles per thread and step) ----
    for (int32_t q = b; q < TC; q += G) {
      int32_t q0;
      const int32_t j = cluster_of(q, &q0);
      const int32_t c = ls + j;
      const int32_t s0 = __ldcg(p.begin + c) + (q - q0) * kTreeChunk;
      const int32_t s1 = min(s0 + kTreeChunk, __ldcg(p.end + c));
      if (threadIdx.x == 0) {
        p.chunk_cluster[q] = j;
        p.chunk_start[q] = s0;
      }
      const uint8_t mask = __ldcg(p.mask + j);
      if (!mask) continue;                    // a leaf's chunk: copied, not counted
      if (threadIdx.x < 8) s_cnt[threadIdx.x] = 0;
      __syncthreads();
      const long long mk[3] = {__ldcg(p.midk + (int64_t)j * 3), __ldcg(p.midk + (int64_t)j * 3 + 1),
                               __ldcg(p.midk + (int64_t)j * 3 + 2)};
      for (int32_t i0 = s0; i0 < s1; i0 += 2 * kTreeCoopThreads) {   // warp-uniform trip count
        const int32_t ia = i0 + threadIdx.x, ib = ia + kTreeCoopThreads;
        const bool va = ia < s1, vb = ib < s1;
        double ax = 0.0, ay = 0.0, az = 0.0, bx = 0.0, by = 0.0, bz = 0.0;
        if (va) {
          ax = __ldcg(x + ia);
          ay = __ldcg(y + ia);
          az = __ldcg(z + ia);
        }
        if (vb) {
          bx = __ldcg(x + ib);
          by = __ldcg(y + ib);
          bz = __ldcg(z + ib);
        }
        const int ca = va ? child_code(ax, ay, az, mask, mk) : 8;
        const int cb = vb ? child_code(bx, by, bz, mask, mk) : 8;
        if (va) p.code[ia] = (uint8_t)ca;
        if (vb) p.code[ib] = (uint8_t)cb;
        const unsigned pa = __match_any_sync(0xffffffffu, ca), pb = __match_any_sync(0xffffffffu, cb);
        if (va && (pa & ((1u << lane) - 1u)) == 0) atomicAdd(&s_cnt[ca], __popc(pa));
        if (vb && (pb & ((1u << lane) - 1u)) == 0) atomicAdd(&s_cnt[cb], __popc(pb));
      }
      __syncthreads();
      if (threadIdx.x < 8) p.counts[(int64_t)q * 8 + threadIdx.x] = s_cnt[threadIdx.x];
      __syncthreads();
    }
    if (!tree_grid_sync(g, G)) return;

    // ---- 3. per splitting cluster: child counts and the chunks' destinations ----
    // Clusters of many chunks take the whole block, one after the other; the
    // rest take one warp each.
    for (int32_t j = jlo; j < jhi; ++j) {     // block-uniform
      const int32_t nq = __ldcg(p.nchk + j);
      if (nq <= kWideCombine || !__ldcg(p.mask + j)) continue;
      const int32_t q0 = pq[b] + __ldcg(p.coff + j);
      int32_t v[8], ex[8], tot[8], cb[8], run[8];
      for (int d = 0; d < 8; ++d) v[d] = 0;
      for (int32_t t = threadIdx.x; t < nq; t += kTreeCoopThreads)
        for (int d = 0; d < 8; ++d) v[d] += __ldcg(p.counts + (int64_t)(q0 + t) * 8 + d);
      block_scan8(v, ex, tot, s_ws);
      int32_t pos = __ldcg(p.begin + ls + j), k = 0;
      for (int d = 0; d < 8; ++d) {
        cb[d] = pos;
        pos += tot[d];
        run[d] = 0;
        k += tot[d] > 0;
      }
      if (threadIdx.x < 8) p.child_cnt[(int64_t)j * 8 + threadIdx.x] = tot[threadIdx.x];
      if (threadIdx.x == 0) p.nch[j] = k;
      for (int32_t base = 0; base < nq; base += kTreeCoopThreads) {
        const int32_t t = base + threadIdx.x;
        for (int d = 0; d < 8; ++d) v[d] = t < nq ? __ldcg(p.counts + (int64_t)(q0 + t) * 8 + d) : 0;
        int32_t tile[8];
        block_scan8(v, ex, tile, s_ws);
        if (t < nq)
          for (int d = 0; d < 8; ++d) p.chunk_base[(int64_t)(q0 + t) * 8 + d] = cb[d] + run[d] + ex[d];
        for (int d = 0; d < 8; ++d) run[d] += tile[d];
      }
    }
    for (int32_t j = jlo + warp; j < jhi; j += kTreeCoopThreads / 32) {
      const uint8_t mask = __ldcg(p.mask + j);
      const int32_t nq = __ldcg(p.nchk + j);
      if (!mask) {
        if (lane == 0) p.nch[j] = 0;
        continue;
      }
      if (nq > kWideCombine) continue;        // done above
      const int32_t q0 = pq[b] + __ldcg(p.coff + j);
      int32_t tot[8];
      for (int d = 0; d < 8; ++d) tot[d] = 0;
      for (int32_t t = lane; t < nq; t += 32)
        for (int d = 0; d < 8; ++d) tot[d] += __ldcg(p.counts + (int64_t)(q0 + t) * 8 + d);
      for (int d = 0; d < 8; ++d)
        for (int o = 16; o; o >>= 1) tot[d] += __shfl_xor_sync(0xffffffffu, tot[d], o);
      int32_t cb[8], k = 0;
      int32_t pos = __ldcg(p.begin + ls + j);
      for (int d = 0; d < 8; ++d) {
        cb[d] = pos;
        pos += tot[d];
        k += tot[d] > 0;
      }
      if (lane < 8) p.child_cnt[(int64_t)j * 8 + lane] = tot[lane];
      if (lane == 0) p.nch[j] = k;
      for (int32_t t0 = 0; t0 < nq; t0 += 32) {   // chunk-order exclusive scan per code
        const int32_t t = t0 + lane;
        for (int d = 0; d < 8; ++d) {
          const int32_t v = t < nq ? __ldcg(p.counts + (int64_t)(q0 + t) * 8 + d) : 0;
          int32_t inc = v;
          for (int o = 1; o < 32; o <<= 1) {
            const int32_t w = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += w;
          }
          if (t < nq) p.chunk_base[(int64_t)(q0 + t) * 8 + d] = cb[d] + inc - v;
          cb[d] += __shfl_sync(0xffffffffu, inc, 31);
        }
      }
    }
    __threadfence();
    __syncthreads();
    {
      int32_t run_c = 0;
      for (int32_t base = jlo; base < jhi; base += kTreeCoopThreads) {
        const int32_t j = base + threadIdx.x;
        const int32_t v = j < jhi ? __ldcg(p.nch + j) : 0;
        int32_t xa, xb, ta, tb;
        tree_block_scan2(v, 0, &xa, &xb, &ta, &tb);
        if (j < jhi) p.chof[j] = run_c + xa;
        run_c += ta;
      }
      if (threadIdx.x == 0) p.part2[b] = run_c;
    }
    if (!tree_grid_sync(g, G)) return;
    block_prefix(G, pc, [&](unsigned i) { return __ldcg(p.part2 + i); });
    const int32_t NC = pc[G];
    if ((int64_t)le + NC > (int64_t)p.cap || L + 1 >= kMaxTreeLevels) {   // the same decision in every block
      if (b == 0 && threadIdx.x == 0) {
        g->level = L;
        g->parity = par;
        g->need = le + NC;
        atomicExch(&g->status, L + 1 >= kMaxTreeLevels ? 3 : 1);
      }
      return;
    }

    // ---- 4. the children, and the stable scatter into the other buffer ----
    for (int32_t j = jlo + threadIdx.x; j < jhi; j += kTreeCoopThreads) {
      if (!__ldcg(p.mask + j)) continue;
      const int32_t c = ls + j;
      const int32_t fc = le + pc[b] + __ldcg(p.chof + j);
      int32_t pos = __ldcg(p.begin + c), k = 0;
      const int32_t prob = __ldcg(p.problem + c);
      for (int d = 0; d < 8; ++d) {
        const int32_t cnt = __ldcg(p.child_cnt + (int64_t)j * 8 + d);
        if (cnt == 0) continue;
        const int32_t id = fc + k++;
        p.begin[id] = pos;
        p.end[id] = pos + cnt;
        p.parent[id] = c;
        p.level[id] = L + 1;
        p.problem[id] = prob;
        p.bsrc[id] = j * 8 + d;
        pos += cnt;
      }
      p.first_child[c] = fc;
      p.nchild[c] = k;
    }
    for (int32_t q = b; q < TC; q += G) {
      const int32_t j = __ldcg(p.chunk_cluster + q);
      const int32_t s0 = __ldcg(p.chunk_start + q);
      const int32_t s1 = min(s0 + kTreeChunk, __ldcg(p.end + ls + j));
      if (!__ldcg(p.mask + j)) {              // a leaf: same positions in the other buffer
        for (int32_t i = s0 + threadIdx.x; i < s1; i += kTreeCoopThreads) {
          x2[i] = __ldcg(x + i);
          y2[i] = __ldcg(y + i);
          z2[i] = __ldcg(z + i);
          perm2[i] = __ldcg(perm + i);
        }
        continue;
      }
      if (threadIdx.x < 8) {
        running[threadIdx.x] = 0;
        s_base[threadIdx.x] = __ldcg(p.chunk_base + (int64_t)q * 8 + threadIdx.x);
      }
      scatter_chunk(s0, s1, p.code, x, y, z, perm, x2, y2, z2, perm2, warp_cnt, running, s_base, LdCg());
    }
    if (b == 0 && threadIdx.x == 0) {
      p.level_start[L + 2] = le + NC;
      if (L + 2 < kTreeHeadLevels) g->level_start[L + 2] = le + NC;   // the host reads these
    }
    if (!tree_grid_sync(g, G)) return;

    // ---- 5. the children's boxes: each chunk's positions now hold whole runs of children ----
    for (int32_t q = b; q < TC; q += G) {
      const int32_t j = __ldcg(p.chunk_cluster + q);
      if (!__ldcg(p.mask + j)) continue;
      const int32_t s0 = __ldcg(p.chunk_start + q);
      const int32_t s1 = min(s0 + kTreeChunk, __ldcg(p.end + ls + j));
      int32_t pos = __ldcg(p.begin + ls + j);
      for (int d = 0; d < 8 && pos < s1; ++d) {   // block-uniform
        const int32_t e = pos + __ldcg(p.child_cnt + (int64_t)j * 8 + d);
        if (e > s0 && e > pos)
          box_keys_of_range(max(pos, s0), min(e, s1), x2, y2, z2, knext + ((int64_t)j * 8 + d) * 6);
        pos = e;
      }
    }
    if (!tree_grid_sync(g, G)) return;
  }

  // ---- leaf order: leaves under every cluster, then each cluster's first leaf ----
  const int32_t C = __ldcg(p.level_start + L + 1);
  for (int64_t c = gtid; c < C; c += gthreads) p.nsub[c] = 0;
  if (!tree_grid_sync(g, G)) return;
  for (int64_t c = gtid; c < C; c += gthreads)   // every leaf counts itself in each ancestor
    if (__ldcg(p.nchild + c) == 0)
      for (int32_t a = (int32_t)c; a >= 0; a = __ldcg(p.parent + a)) atomicAdd(p.nsub + a, 1);
  if (!tree_grid_sync(g, G)) return;
  if (b == 0) {   // roots in particle order
    int32_t run = 0;
    for (int32_t base = 0; base < p.nroots; base += kTreeCoopThreads) {
      const int32_t r = base + threadIdx.x;
      const int32_t v = r < p.nroots ? __ldcg(p.nsub + r) : 0;
      int32_t xa, xb, ta, tb;
      tree_block_scan2(v, 0, &xa, &xb, &ta, &tb);
      if (r < p.nroots) p.leaf_first[r] = run + xa;
      run += ta;
    }
    if (threadIdx.x == 0) g->nleaves = run;
  }
  if (!tree_grid_sync(g, G)) return;
  // first leaf of c: its root's first leaf plus the leaves under the earlier
  // siblings of c and of each of its ancestors (children are in particle order)
  for (int64_t c = gtid; c < C; c += gthreads) {
    int32_t f = 0, a = (int32_t)c;
    for (int32_t up = __ldcg(p.parent + a); up >= 0; a = up, up = __ldcg(p.parent + a))
      for (int32_t sib = __ldcg(p.first_child + up); sib < a; ++sib) f += __ldcg(p.nsub + sib);
    f += __ldcg(p.leaf_first + a);   // a is the root
    const int32_t n_c = __ldcg(p.nsub + c);
    if (c >= p.nroots) p.leaf_first[c] = f;
    p.leaf_last[c] = f + n_c;
    if (__ldcg(p.nchild + c) == 0) p.leaf_ids[f] = (int32_t)c;
  }
  if (b == 0 && threadIdx.x == 0) {
    g->level = L;
    g->parity = par;
    atomicCAS(&g->status, -1, 0);            // unless a block met an error
  }
}

static bool coop_tree_available(int* blocks) {
  if (cooperative_set_up_disabled()) return false;
  int dev = 0, sms = 0, coop = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tree_all, kTreeCoopThreads, 0) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (!coop || per_sm < 1) return false;
  *blocks = std::min(kTreeMaxBlocks, sms * std::min(per_sm, 4));
  return true;
}

// The build by one cooperative launch (k_tree_all), relaunched from the level
// it stopped at when the cluster arrays must grow.  *done stays false when the
// device has no cooperative launch; the caller then runs build_tree.
static int build_tree_coop(Tree& T, const double* coords, int32_t n, const std::vector<int32_t>& roots,
                           int32_t max_leaf, int degree, const double* charges, int64_t ncharges,
                           cudaStream_t s, Counters& cnt, bool* done) {
  *done = false;
  int G = 0;
  if (!coop_tree_available(&G)) return BLDTT_OK;
  T.n = n;
  const int32_t nroots = (int32_t)roots.size() - 1;
  TreeCoop p{};
  p.n = n;
  p.coords = coords;
  p.nroots = nroots;
  p.charges = charges;
  p.ncharges = charges ? ncharges : 0;
  p.max_leaf = max_leaf;
  BL_TRY(dalloc_n(&T.x, n, s));
  BL_TRY(dalloc_n(&T.y, n, s));
  BL_TRY(dalloc_n(&T.z, n, s));
  BL_TRY(dalloc_n(&T.perm, n, s));
  BL_TRY(dalloc_n(&T.sx, n, s));   // the other coordinate buffer, held by the tree from here on
  BL_TRY(dalloc_n(&T.sy, n, s));   // (the Morton pass writes into it; free_tree frees it)
  BL_TRY(dalloc_n(&T.sz, n, s));
  BL_TRY(dalloc_n(&T.sperm, n, s));
  p.x1 = T.sx;
  p.y1 = T.sy;
  p.z1 = T.sz;
  p.perm1 = T.sperm;
  p.x0 = T.x;
  p.y0 = T.y;
  p.z0 = T.z;
  p.perm0 = T.perm;
  int32_t* d_roots = nullptr;
  Arena fixed;   // scratch of the whole build
  fixed.add(&p.code, n);
  fixed.add(&d_roots, roots.size());
  fixed.add(&p.part, G);
  fixed.add(&p.part2, G);
  fixed.add(&p.level_start, kMaxTreeLevels + 2);
  fixed.add(&p.g, 1);
  BL_TRY(fixed.alloc(s));
  BL_CUDA(cudaMemcpyAsync(d_roots, roots.data(), roots.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  p.roots = d_roots;
  BL_CUDA(cudaMemsetAsync(p.g, 0, sizeof(TreeGrid), s));
  // cluster capacity: grown (and the launch resumed) when a level needs more
  size_t cap = std::max<size_t>(1024, 2 * (size_t)nroots + 4 * ((size_t)n / std::max(1, max_leaf) + 1));
  if (const char* e = std::getenv("BLDTT_TREE_CAPACITY"))   // a smaller start exercises the regrowth
    cap = std::max<size_t>((size_t)std::strtoull(e, nullptr, 10), (size_t)nroots);
  size_t c_lid = 0, c_lf = 0, c_ll = 0, old_cap = 0;
  Arena per_cap;   // scratch sized by the cluster capacity
  int status = BLDTT_OK;
  TreeGrid h{};
  bool first = true;
  for (;;) {
    const size_t keep = first ? 0 : (size_t)T.level_start.back();   // clusters made so far
    BL_TRY(grow_clusters(T, cap, keep, s));
    cap = T.cap;
    const size_t qcap = (size_t)n / kTreeChunk + cap + 1;
    Arena grown;
    TreeCoop q = p;   // the new capacity's arrays, then what must carry over
    grown.add(&q.kbox0, cap * 48);
    grown.add(&q.kbox1, cap * 48);
    grown.add(&q.bsrc, cap);
    grown.add(&q.mask, cap);
    grown.add(&q.midk, cap * 3);
    grown.add(&q.coff, cap);
    grown.add(&q.nchk, cap);
    grown.add(&q.child_cnt, cap * 8);
    grown.add(&q.nch, cap);
    grown.add(&q.chof, cap);
    grown.add(&q.nsub, cap);
    grown.add(&q.chunk_cluster, qcap);
    grown.add(&q.chunk_start, qcap);
    grown.add(&q.counts, qcap * 8);
    grown.add(&q.chunk_base, qcap * 8);
    BL_TRY(grown.alloc(s));
    if (first) {   // the roots' key boxes start empty (zero)
      BL_CUDA(cudaMemsetAsync(q.kbox0, 0, (size_t)nroots * 48 * sizeof(unsigned long long), s));
    } else {       // the key boxes of the level to resume, and the clusters' box entries
      BL_CUDA(cudaMemcpyAsync(q.kbox0, p.kbox0, old_cap * 48 * sizeof(unsigned long long),
                              cudaMemcpyDeviceToDevice, s));
      BL_CUDA(cudaMemcpyAsync(q.kbox1, p.kbox1, old_cap * 48 * sizeof(unsigned long long),
                              cudaMemcpyDeviceToDevice, s));
      BL_CUDA(cudaMemcpyAsync(q.bsrc, p.bsrc, keep * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    }
    per_cap.release(s);
    per_cap = std::move(grown);
    p = q;
    old_cap = cap;
    BL_TRY(dgrow(&T.leaf_ids, &c_lid, cap, 0, s));
    BL_TRY(dgrow(&T.leaf_first, &c_lf, cap, 0, s));
    BL_TRY(dgrow(&T.leaf_last, &c_ll, cap, 0, s));
    BL_CUDA(cudaMemsetAsync(p.g, 0, 2 * sizeof(unsigned), s));           // barrier
    BL_CUDA(cudaMemsetAsync(&p.g->status, 0xff, sizeof(int32_t), s));    // -1: running
    p.begin = T.begin;
    p.end = T.end;
    p.parent = T.parent;
    p.first_child = T.first_child;
    p.nchild = T.nchild;
    p.level = T.level;
    p.problem = T.problem;
    p.box = T.box;
    p.cap = (int32_t)std::min<size_t>(cap, INT32_MAX);
    p.qcap = (int32_t)std::min<size_t>(qcap, INT32_MAX);
    p.leaf_ids = T.leaf_ids;
    p.leaf_first = T.leaf_first;
    p.leaf_last = T.leaf_last;
    void* args[] = {&p};
    {
      std::lock_guard<std::mutex> lock(cooperative_launch_mutex());
      BL_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(&k_tree_all), dim3(G),
                                          dim3(kTreeCoopThreads), args, 0, s));
      BL_LAUNCHED(cnt.launches);
      BL_TRY(read_device(p.g, &h, sizeof(h), s));
    }
    first = false;
    if (h.status != 1) break;
    // clusters so far: the levels up to the one that stopped
    T.level_start.assign(h.level_start, h.level_start + std::min(h.level + 2, kTreeHeadLevels));
    if (h.level + 2 > kTreeHeadLevels) {
      T.level_start.resize(h.level + 2);
      BL_TRY(read_device(p.level_start, T.level_start.data(), T.level_start.size() * sizeof(int32_t), s));
    }
    cap = std::max<size_t>(2 * cap, (size_t)h.need);
  }
  if (h.status == 0) {
    const int L = h.level;
    T.level_start.assign(h.level_start, h.level_start + std::min(L + 2, kTreeHeadLevels));
    if (L + 2 > kTreeHeadLevels) {
      T.level_start.resize(L + 2);
      BL_TRY(read_device(p.level_start, T.level_start.data(), T.level_start.size() * sizeof(int32_t), s));
    }
    T.nlevels = L + 1;
    T.nclusters = T.level_start.back();
    T.nroots = nroots;
    T.nleaves = h.nleaves;
    if (h.parity) {   // the final order is in buffer 1
      std::swap(T.x, T.sx);
      std::swap(T.y, T.sy);
      std::swap(T.z, T.sz);
      std::swap(T.perm, T.sperm);
    }
  } else if (h.status == 2) {
    set_error("a grid barrier of the tree build gave up after %llu ns", (unsigned long long)kTreeWaitNs);
    status = BLDTT_ETIMEOUT;
  } else if (h.status == 3) {
    set_error("tree deeper than %d levels: some cluster is not separated by its midpoints", kMaxTreeLevels);
    status = BLDTT_EINTERNAL;
  } else if (h.status == 4) {
    set_error("a target, source or charge value is not finite");
    status = BLDTT_EINVAL;
  } else {
    set_error("the tree build ended with status %d", h.status);
    status = BLDTT_EINTERNAL;
  }
  fixed.release(s);
  per_cap.release(s);
  if (status != BLDTT_OK) return status;
  const int C = T.nclusters;
  BL_TRY(dalloc_n(&T.center, (size_t)C * 3, s));
  BL_TRY(dalloc_n(&T.radius, (size_t)C, s));
  BL_TRY(dalloc_n(&T.nodes, (size_t)C * 3 * (degree + 1), s));
  k_tree_geometry<<<nblk(C, 128), 128, 0, s>>>(C, degree, T.box, T.center, T.radius, T.nodes);
  BL_LAUNCHED(cnt.launches);
  *done = true;
  return BLDTT_OK;
}

bool tree_build_cooperative() {
  int G = 0;
  return coop_tree_available(&G);
}

int build_tree_checked(Tree& T, const double* coords, int32_t n, const std::vector<int32_t>& roots,
                       int32_t max_leaf, int degree, const double* charges, int64_t ncharges,
                       cudaStream_t s, Counters& cnt) {
  bool done = false;
  BL_TRY(build_tree_coop(T, coords, n, roots, max_leaf, degree, charges, ncharges, s, cnt, &done));
  if (done) return BLDTT_OK;
  // level by level: reject non-finite input first (an infinite box is split without end)
  int* bad = nullptr;
  BL_TRY(dalloc_n(&bad, 1, s));
  BL_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
  BL_TRY(check_finite(coords, 3 * (int64_t)n, bad, s, cnt));
  if (charges) BL_TRY(check_finite(charges, ncharges, bad, s, cnt));
  int h_bad = 0;
  BL_TRY(read_device(bad, &h_bad, sizeof(int), s));
  dfree(bad, s);
  if (h_bad) {
    set_error("a target, source or charge value is not finite");
    return BLDTT_EINVAL;
  }
  return build_tree(T, coords, n, roots, max_leaf, degree, s, cnt);
}

// ---------------------------------------------------------------------------
// Morton order inside leaves
// ---------------------------------------------------------------------------
// The order of particles inside a leaf is not part of the method; putting
// them along a Morton curve of the leaf box makes every run of kChunk
// consecutive sources spatially compact, which the FP32 interaction path
// exploits (its coordinate frames are per run of kChunk).  A leaf is sorted by one CTA (bitonic
// network in shared memory, one compare-exchange per thread and step); leaves
// above the power of two covering max_leaf (only degenerate ones, whose
// particles share a point) or above kMortonMax particles keep their order.
constexpr int kMortonMax = 4096;
constexpr int kMortonThreads = 256;

__device__ __forceinline__ uint32_t spread10(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// Cell of a coordinate in [lo, lo + cells / scale), 0..cells-1: an ordering
// key only, so FP32 suffices (scale = 0 for a zero-width box).
__device__ __forceinline__ uint32_t quantize(double v, float lo, float scale, int cells) {
  const int q = (int)(__fsub_rn((float)v, lo) * scale);
  return (uint32_t)(q < 0 ? 0 : (q >= cells ? cells - 1 : q));
}

// Sort keys: the Morton code of the point's cell above its position in the
// leaf (unique keys, ties by position).  32-bit keys (7 bits per dimension,
// 11 position bits) for leaves of up to 2048 points, 64-bit keys (10 bits per
// dimension) above: the sort is bound by shared-memory traffic.
template <typename Key>
struct MortonKey;
template <>
struct MortonKey<uint32_t> {
  static constexpr int kBits = 7, kMaxPoints = 2048;
  __device__ static uint32_t make(uint32_t code, int i) { return (code << 11) | (uint32_t)i; }
  __device__ static int index(uint32_t k) { return (int)(k & 0x7ffu); }
  __device__ static uint32_t none() { return ~0u; }
};
template <>
struct MortonKey<unsigned long long> {
  static constexpr int kBits = 10, kMaxPoints = 1 << 30;
  __device__ static unsigned long long make(uint32_t code, int i) {
    return ((unsigned long long)code << 32) | (unsigned)i;
  }
  __device__ static int index(unsigned long long k) { return (int)(k & 0xffffffffu); }
  __device__ static unsigned long long none() { return ~0ull; }
};

template <typename Key>
__global__ void __launch_bounds__(kMortonThreads) k_leaf_morton(
    const int32_t* __restrict__ leaf_ids, const int32_t* __restrict__ begin,
    const int32_t* __restrict__ end, const double* __restrict__ box, const double* __restrict__ x,
    const double* __restrict__ y, const double* __restrict__ z, const int32_t* __restrict__ perm,
    double* __restrict__ x2, double* __restrict__ y2, double* __restrict__ z2,
    int32_t* __restrict__ perm2, int cap) {
  using MK = MortonKey<Key>;
  extern __shared__ __align__(16) unsigned char kraw[];
  Key* key = reinterpret_cast<Key*>(kraw);   // [cap], cap a power of two
  const int c = leaf_ids[blockIdx.x];
  const int32_t b = begin[c];
  const int m = end[c] - b;
  if (m > cap || m < 2) {   // keep the order
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      x2[b + i] = x[b + i];
      y2[b + i] = y[b + i];
      z2[b + i] = z[b + i];
      perm2[b + i] = perm[b + i];
    }
    return;
  }
  int n2 = 1;
  while (n2 < m) n2 <<= 1;
  const double* bx = box + (int64_t)c * 6;
  constexpr int kCells = 1 << MK::kBits;
  float lo[3], sc[3];
  for (int d = 0; d < 3; ++d) {
    lo[d] = (float)bx[d];
    const float e = (float)bx[3 + d] - lo[d];
    sc[d] = e > 0.f ? (float)kCells / e : 0.f;
  }
  for (int i = threadIdx.x; i < n2; i += blockDim.x) {
    if (i < m) {
      const uint32_t code = (spread10(quantize(x[b + i], lo[0], sc[0], kCells)) << 2) |
                            (spread10(quantize(y[b + i], lo[1], sc[1], kCells)) << 1) |
                            spread10(quantize(z[b + i], lo[2], sc[2], kCells));
      key[i] = MK::make(code, i);
    } else {
      key[i] = MK::none();
    }
  }
  __syncthreads();
  for (int k = 2; k <= n2; k <<= 1) {        // bitonic sort, ascending
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < (n2 >> 1); t += blockDim.x) {   // one compare-exchange each
        const int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));          // lower index of pair t
        const int ixj = i | j;
        const Key a = key[i], bb = key[ixj];
        const bool up = (i & k) == 0;
        if ((a > bb) == up) {
          key[i] = bb;
          key[ixj] = a;
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const int src = b + MK::index(key[i]);
    x2[b + i] = x[src];
    y2[b + i] = y[src];
    z2[b + i] = z[src];
    perm2[b + i] = perm[src];
  }
}

int morton_order_leaves(Tree& T, int32_t max_leaf, cudaStream_t s, Counters& cnt) {
  double *x2 = T.sx, *y2 = T.sy, *z2 = T.sz;   // the build's spare buffers, else new ones
  int32_t* perm2 = T.sperm;
  T.sx = T.sy = T.sz = nullptr;
  T.sperm = nullptr;
  if (T.nleaves == 0) {
    dfree(x2, s); dfree(y2, s); dfree(z2, s); dfree(perm2, s);
    return BLDTT_OK;
  }
  if (!x2) BL_TRY(dalloc_n(&x2, T.n, s));
  if (!y2) BL_TRY(dalloc_n(&y2, T.n, s));
  if (!z2) BL_TRY(dalloc_n(&z2, T.n, s));
  if (!perm2) BL_TRY(dalloc_n(&perm2, T.n, s));
  // keys of the largest sorted leaf (leaves hold at most max_leaf particles)
  int n2max = 2;
  while (n2max < max_leaf && n2max < kMortonMax) n2max <<= 1;
  if (n2max <= MortonKey<uint32_t>::kMaxPoints) {
    const size_t smem = sizeof(uint32_t) * (size_t)n2max;
    BL_CUDA(cudaFuncSetAttribute(k_leaf_morton<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    k_leaf_morton<uint32_t><<<T.nleaves, kMortonThreads, smem, s>>>(
        T.leaf_ids, T.begin, T.end, T.box, T.x, T.y, T.z, T.perm, x2, y2, z2, perm2, n2max);
  } else {
    const size_t smem = sizeof(unsigned long long) * (size_t)n2max;
    BL_CUDA(cudaFuncSetAttribute(k_leaf_morton<unsigned long long>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_leaf_morton<unsigned long long><<<T.nleaves, kMortonThreads, smem, s>>>(
        T.leaf_ids, T.begin, T.end, T.box, T.x, T.y, T.z, T.perm, x2, y2, z2, perm2, n2max);
  }
  BL_LAUNCHED(cnt.launches);
  std::swap(T.x, x2);
  std::swap(T.y, y2);
  std::swap(T.z, z2);
  std::swap(T.perm, perm2);
  dfree(x2, s);
  dfree(y2, s);
  dfree(z2, s);
  dfree(perm2, s);
  return BLDTT_OK;
}

void free_tree(Tree& T, cudaStream_t s) {
  dfree_ptr(T.x, s); dfree_ptr(T.y, s); dfree_ptr(T.z, s); dfree_ptr(T.perm, s);
  dfree_ptr(T.sx, s); dfree_ptr(T.sy, s); dfree_ptr(T.sz, s); dfree_ptr(T.sperm, s);
  dfree_ptr(T.begin, s); dfree_ptr(T.end, s); dfree_ptr(T.parent, s);
  dfree_ptr(T.first_child, s); dfree_ptr(T.nchild, s); dfree_ptr(T.level, s);
  dfree_ptr(T.problem, s);
  dfree_ptr(T.box, s); dfree_ptr(T.center, s); dfree_ptr(T.radius, s); dfree_ptr(T.nodes, s);
  dfree_ptr(T.xfer_u, s);
  dfree_ptr(T.leaf_ids, s); dfree_ptr(T.leaf_first, s); dfree_ptr(T.leaf_last, s);
  T.cap = 0;
  T.nclusters = T.nlevels = T.nleaves = 0;
  T.level_start.clear();
}

}  // namespace bldtt
