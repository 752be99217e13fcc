// Upward pass (Sec. 2.5, App. B), source-pool construction, and downward
// pass (Sec. 2.7, App. C).
//
// The Lagrange basis is always evaluated in FP64 with the coincident-point
// guard of the second barycentric form (Sec. 2.1, Eq. (3)); in FP32_BULK mode
// the contractions that follow (leaf proxy charges and the leaf interpolation
// to particles) run in FP32 over short runs that are summed in FP64.
#include <cmath>
#include <type_traits>
#include <vector>

#include "basis.cuh"
#include "internal.cuh"

namespace bldtt {

// ---------------------------------------------------------------------------
// Charges into source tree order
// ---------------------------------------------------------------------------
__global__ void k_permute(const double* __restrict__ src, const int32_t* __restrict__ perm, int64_t n,
                          double* __restrict__ dst) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[perm[i]];
}

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

int permute_charges(bldtt_plan* p, const double* charges, cudaStream_t s) {
  k_permute<<<nblk(p->N, 256), 256, 0, s>>>(charges, p->st.perm, p->N, p->q_tree);
  BL_LAUNCHED(p->setup_counter.launches);
  return BLDTT_OK;
}

// ---------------------------------------------------------------------------
// Upward pass
// ---------------------------------------------------------------------------
constexpr int kUpThreads = 256;
constexpr int kUpChunk = 64;
constexpr int kUpStride = kUpChunk + 1;        // odd row stride: no bank conflicts
constexpr int kMaxOutPerThread = (kMaxP * kMaxP * kMaxP + kUpThreads - 1) / kUpThreads;

// Eq. (9) for every source leaf: qhat_k = sum_j L_k1(y_j1) L_k2(y_j2) L_k3(y_j3) q_j.
template <bool F32>
__global__ void __launch_bounds__(kUpThreads) k_up_leaf(
    const int32_t* __restrict__ leaf_ids, const int32_t* __restrict__ begin,
    const int32_t* __restrict__ end, const double* __restrict__ x, const double* __restrict__ y,
    const double* __restrict__ z, const double* __restrict__ q, const double* __restrict__ nodes,
    int n, double* __restrict__ qhat) {
  using T = typename std::conditional<F32, float, double>::type;
  __shared__ double snodes[3][kMaxP];
  __shared__ float shl[3][2 * kMaxP];          // FP32_BULK: float split of the nodes
  __shared__ T sB[3][kMaxP][kUpStride];
  __shared__ T sq[kUpChunk];
  const int P = n + 1, np = P * P * P;
  const int c = leaf_ids[blockIdx.x];
  const int32_t b = begin[c], e = end[c];
  if (threadIdx.x < 3 * P) {
    const double v = nodes[(int64_t)c * 3 * P + threadIdx.x];
    snodes[threadIdx.x / P][threadIdx.x % P] = v;
    float h, l;
    split_f64(v, h, l);
    shl[threadIdx.x / P][threadIdx.x % P] = h;
    shl[threadIdx.x / P][kMaxP + threadIdx.x % P] = l;
  }
  double acc[kMaxOutPerThread];
#pragma unroll
  for (int r = 0; r < kMaxOutPerThread; ++r) acc[r] = 0.0;
  const double* coord[3] = {x, y, z};
  __syncthreads();
  for (int32_t base = b; base < e; base += kUpChunk) {
    const int cnt = min(kUpChunk, e - base);
    for (int task = threadIdx.x; task < 3 * kUpChunk; task += kUpThreads) {
      int d = task / kUpChunk, j = task % kUpChunk;
      if (j < cnt) {
        if constexpr (F32)
          basis_1d_f32(coord[d][base + j], shl[d], n, &sB[d][0][j], kUpStride);
        else
          basis_1d<T>(coord[d][base + j], snodes[d], n, &sB[d][0][j], kUpStride);
      } else {
        for (int k = 0; k < P; ++k) sB[d][k][j] = (T)0;
      }
    }
    if (threadIdx.x < kUpChunk) sq[threadIdx.x] = threadIdx.x < cnt ? (T)q[base + threadIdx.x] : (T)0;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kMaxOutPerThread; ++r) {
      int o = threadIdx.x + r * kUpThreads;
      if (o < np) {
        int k1 = o / (P * P), k2 = (o / P) % P, k3 = o % P;
        T sacc = (T)0;
        for (int j = 0; j < cnt; ++j) sacc += sB[0][k1][j] * sB[1][k2][j] * (sB[2][k3][j] * sq[j]);
        acc[r] += (double)sacc;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < kMaxOutPerThread; ++r) {
    int o = threadIdx.x + r * kUpThreads;
    if (o < np) qhat[(int64_t)c * np + o] = acc[r];
  }
}

// FP32_BULK form of Eq. (9) for a grid of P points fixed at compile time
// (P <= 16).  Thread (g, k2, k3) of a P^2 x G layout owns the P outputs
// (k1, k2, k3), k1 = 0..P-1, over the particles of group g (every G-th
// particle of a chunk): per particle it forms w = (L_k2(y2) q) L_k3(y3) once
// and adds L_k1(y1) w to its P outputs, reading the k1 row as float4
// broadcasts, so every basis value loaded serves P products.  Each output's
// float run over one chunk (RUN terms) is added to a float pair by TwoSum; the
// groups' pairs are summed in FP64 at the end (fixed order).
template <int P>
struct UpLeafShape {
  static constexpr int P2 = P * P;
  static constexpr int G = kUpThreads / P2;            // particle groups
  static constexpr int RUN = 512 / G < 32 ? 512 / G : 32;   // particles of a group per chunk
  static constexpr int CH = G * RUN;                   // particles per chunk
  static constexpr int RS = (P + 3) / 4 * 4;           // k1-row stride (float4 aligned)
  static constexpr int LS = CH + 1;                    // odd stride of the k2 and k3 rows
};

template <int P>
__global__ void __launch_bounds__(kUpThreads) k_up_leaf_f32(
    const int32_t* __restrict__ leaf_ids, const int32_t* __restrict__ begin,
    const int32_t* __restrict__ end, const double* __restrict__ x, const double* __restrict__ y,
    const double* __restrict__ z, const double* __restrict__ q, const double* __restrict__ nodes,
    double* __restrict__ qhat) {
  using S = UpLeafShape<P>;
  static_assert(S::G >= 1, "P^2 must not exceed the block size");
  constexpr int NP = P * P * P;
  __shared__ float shl[3][2 * kMaxP];
  __shared__ __align__(16) float s1[S::CH][S::RS];     // L_k1(y1), one row per particle
  __shared__ float s2[P][S::LS];                        // L_k2(y2) q
  __shared__ float s3[P][S::LS];                        // L_k3(y3)
  __shared__ double sred[S::G][NP];
  const int tid = threadIdx.x;
  const int c = leaf_ids[blockIdx.x];
  const int32_t b = begin[c], e = end[c];
  if (tid < 3 * P) {
    float h, l;
    split_f64(nodes[(int64_t)c * 3 * P + tid], h, l);
    shl[tid / P][tid % P] = h;
    shl[tid / P][kMaxP + tid % P] = l;
  }
  const bool active = tid < S::P2 * S::G;
  const int g = tid / S::P2, u = tid % S::P2, k2 = u / P, k3 = u % P;
  float hi[P], lo[P];
#pragma unroll
  for (int k = 0; k < P; ++k) hi[k] = lo[k] = 0.f;
  __syncthreads();
  for (int32_t base = b; base < e; base += S::CH) {
    const int cnt = min(S::CH, e - base);
    for (int task = tid; task < 3 * S::CH; task += kUpThreads) {
      const int d = task / S::CH, j = task % S::CH;
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
        for (int k = 0; k < S::RS; ++k) s1[j][k] = k < P ? L[k < P ? k : 0] : 0.f;
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
    if (active) {
      float part[P];
#pragma unroll
      for (int k = 0; k < P; ++k) part[k] = 0.f;
      for (int i = 0; i < S::RUN; ++i) {
        const int j = g + S::G * i;
        if (j >= cnt) break;
        const float w = s2[k2][j] * s3[k3][j];
        float l1[S::RS];
        const float4* row = reinterpret_cast<const float4*>(s1[j]);
#pragma unroll
        for (int v = 0; v < S::RS / 4; ++v) {
          const float4 t = row[v];
          l1[4 * v] = t.x;
          l1[4 * v + 1] = t.y;
          l1[4 * v + 2] = t.z;
          l1[4 * v + 3] = t.w;
        }
#pragma unroll
        for (int k = 0; k < P; ++k) part[k] = fmaf(l1[k], w, part[k]);
      }
#pragma unroll
      for (int k = 0; k < P; ++k) {
        const float t = __fadd_rn(hi[k], part[k]);
        lo[k] = __fadd_rn(lo[k], two_sum_err(hi[k], part[k], t));
        hi[k] = t;
      }
    }
    __syncthreads();
  }
  if (active) {
#pragma unroll
    for (int k = 0; k < P; ++k) sred[g][k * S::P2 + u] = (double)hi[k] + (double)lo[k];
  }
  __syncthreads();
  for (int o = tid; o < NP; o += kUpThreads) {
    double v = 0.0;
    for (int gg = 0; gg < S::G; ++gg) v += sred[gg][o];
    qhat[(int64_t)c * NP + o] = v;
  }
}

// Grids of 2..9 points take the specialised FP32_BULK leaf kernels.
constexpr int kFixedPMin = 2, kFixedPMax = 9;

// Transfer matrices of Eqs. (16) and (20): U[c][d][k][k'] = L^par_k(t^c_k'),
// the parent's 1D basis (Eq. (3)) at the cluster's own proxy coordinates, for
// every non-root cluster c (one thread per (c, d, k')).  They depend on the
// tree alone, so the set-up computes them once for the upward and downward
// passes of every compute call.
__global__ void k_transfer_matrices(int32_t C, const int32_t* __restrict__ parent,
                                    const double* __restrict__ nodes, int n, double* __restrict__ U) {
  const int P = n + 1;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)C * 3 * P) return;
  const int c = (int)(t / (3 * P)), dk = (int)(t % (3 * P)), d = dk / P, kp = dk % P;
  const int par = parent[c];
  if (par < 0) return;
  basis_1d<double>(nodes[(int64_t)c * 3 * P + dk], nodes + (int64_t)par * 3 * P + d * P, n,
                   U + ((int64_t)c * 3 + d) * P * P + kp, P);
}

constexpr int kXferThreads = 128;

// Eq. (16) as three mode products with the children's U_d, one CTA per
// (parent, k1): qhat^par[k1][k2][k3] = sum over children (in child order) of
// sum_c U3[k3][c] sum_b U2[k2][b] sum_a U1[k1][a] qhat^child[a][b][c].  The P
// slices of a parent run on P SMs, which matters on levels with few clusters
// because FP64 issues at a small fraction of the FP32 rate.
__global__ void __launch_bounds__(kXferThreads) k_up_parent(int32_t ls, const int32_t* __restrict__ nchild,
                                                           const int32_t* __restrict__ first_child,
                                                           const double* __restrict__ U, int n,
                                                           double* __restrict__ qhat) {
  __shared__ double T1[kMaxP * kMaxP], T2[kMaxP * kMaxP], out[kMaxP * kMaxP];
  const int P = n + 1, P2 = P * P, np = P2 * P;
  const int c = ls + blockIdx.x, k1 = blockIdx.y;
  if (nchild[c] == 0) return;
  for (int o = threadIdx.x; o < P2; o += blockDim.x) out[o] = 0.0;
  for (int ci = 0; ci < nchild[c]; ++ci) {
    const int ch = first_child[c] + ci;
    const double* Uc = U + (int64_t)ch * 3 * P2;
    const double* A = qhat + (int64_t)ch * np;
    for (int o = threadIdx.x; o < P2; o += blockDim.x) {     // (b, c)
      double v = 0.0;
      for (int a = 0; a < P; ++a) v += Uc[k1 * P + a] * A[a * P2 + o];
      T1[o] = v;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < P2; o += blockDim.x) {     // (k2, c)
      const int k2 = o / P, cc = o % P;
      double v = 0.0;
      for (int b = 0; b < P; ++b) v += Uc[P2 + k2 * P + b] * T1[b * P + cc];
      T2[o] = v;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < P2; o += blockDim.x) {     // (k2, k3)
      const int k2 = o / P, k3 = o % P;
      double v = 0.0;
      for (int cc = 0; cc < P; ++cc) v += Uc[2 * P2 + k3 * P + cc] * T2[k2 * P + cc];
      out[o] += v;
    }
    __syncthreads();
  }
  for (int o = threadIdx.x; o < P2; o += blockDim.x) qhat[(int64_t)c * np + k1 * P2 + o] = out[o];
}

// Degree change on one proxy grid (same box): with A[k][k'] = L^(d)_k(s^(n)_k')
// (Chebyshev points on [-1, 1]; the barycentric basis is scale free),
//   proxy charges of degree d:   qhat^(d)_k  = sum_k' A(x)A(x)A [k][k'] qhat^(n)_k'
//   proxy potentials to degree n: phi^(n)_k' += sum_k A(x)A(x)A [k][k'] phi^(d)_k
// Both are exact in exact arithmetic: L^(d)_k is a polynomial of degree
// d <= n, reproduced by the degree-n interpolation (App. A).
// y[a][b][c] (+)= sum M[a][a'] M[b][b'] M[c][c'] x[a'][b'][c'], M = Pout x Pin,
// element (r, k) at M[r * ms_r + k * ms_k].  One block per cluster.
__global__ void k_mode3(int32_t C, const double* __restrict__ M, int ms_r, int ms_k, int Pin, int Pout,
                        const double* __restrict__ in, double* __restrict__ out, int accumulate) {
  extern __shared__ double smem[];
  const int c = blockIdx.x;
  if (c >= C) return;
  double* Ms = smem;                         // [Pout][Pin]
  double* X = Ms + Pout * Pin;               // [Pin^3]
  double* T1 = X + Pin * Pin * Pin;          // [Pout][Pin][Pin]
  double* T2 = T1 + Pout * Pin * Pin;        // [Pout][Pout][Pin]
  const int nin = Pin * Pin * Pin, nout = Pout * Pout * Pout;
  for (int t = threadIdx.x; t < Pout * Pin; t += blockDim.x)
    Ms[t] = M[(t / Pin) * ms_r + (t % Pin) * ms_k];
  for (int t = threadIdx.x; t < nin; t += blockDim.x) X[t] = in[(int64_t)c * nin + t];
  __syncthreads();
  for (int t = threadIdx.x; t < Pout * Pin * Pin; t += blockDim.x) {
    const int a = t / (Pin * Pin), rest = t % (Pin * Pin);
    double v = 0.0;
    for (int k = 0; k < Pin; ++k) v += Ms[a * Pin + k] * X[k * Pin * Pin + rest];
    T1[t] = v;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < Pout * Pout * Pin; t += blockDim.x) {
    const int a = t / (Pout * Pin), b = (t / Pin) % Pout, cc = t % Pin;
    double v = 0.0;
    for (int k = 0; k < Pin; ++k) v += Ms[b * Pin + k] * T1[(a * Pin + k) * Pin + cc];
    T2[t] = v;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nout; t += blockDim.x) {
    const int ab = t / Pout, cc = t % Pout;
    double v = 0.0;
    for (int k = 0; k < Pin; ++k) v += Ms[cc * Pin + k] * T2[ab * Pin + k];
    if (accumulate)
      out[(int64_t)c * nout + t] += v;
    else
      out[(int64_t)c * nout + t] = v;
  }
}

static size_t mode3_smem_bytes(int Pin, int Pout) {
  return sizeof(double) * (size_t)(Pout * Pin + Pin * Pin * Pin + Pout * Pin * Pin + Pout * Pout * Pin);
}

int upward_pass(bldtt_plan* p, cudaStream_t s) {
  Counters& cnt = p->compute_counter;
  const Tree& T = p->st;
  const bool f32 = p->precision == BLDTT_FP32_BULK;
  if (f32 && p->up_engine == BLDTT_PASS_TENSOR && leaf_tc_supported(p->P)) {
    BL_TRY(up_leaf_tc(p, s));          // counts its launch
  } else {
  if (f32 && p->P >= kFixedPMin && p->P <= kFixedPMax) {
    switch (p->P) {
#define BL_UP_LEAF(PP)                                                                          \
  case PP:                                                                                      \
    k_up_leaf_f32<PP><<<T.nleaves, kUpThreads, 0, s>>>(T.leaf_ids, T.begin, T.end, T.x, T.y, T.z, \
                                                       p->q_tree, T.nodes, p->qhat);            \
    break;
      BL_UP_LEAF(2) BL_UP_LEAF(3) BL_UP_LEAF(4) BL_UP_LEAF(5)
      BL_UP_LEAF(6) BL_UP_LEAF(7) BL_UP_LEAF(8) BL_UP_LEAF(9)
#undef BL_UP_LEAF
    }
  } else if (f32)
    k_up_leaf<true><<<T.nleaves, kUpThreads, 0, s>>>(T.leaf_ids, T.begin, T.end, T.x, T.y, T.z,
                                                      p->q_tree, T.nodes, p->n, p->qhat);
  else
    k_up_leaf<false><<<T.nleaves, kUpThreads, 0, s>>>(T.leaf_ids, T.begin, T.end, T.x, T.y, T.z,
                                                       p->q_tree, T.nodes, p->n, p->qhat);
  BL_LAUNCHED(cnt.launches);
  }
  for (int lvl = T.nlevels - 2; lvl >= 0; --lvl) {
    int32_t ls = T.level_start[lvl], nl = T.level_start[lvl + 1] - ls;
    k_up_parent<<<dim3(nl, p->P), kXferThreads, 0, s>>>(ls, T.nchild, T.first_child, T.xfer_u, p->n,
                                                         p->qhat);
    BL_LAUNCHED(cnt.launches);
  }
  // Proxy charges of the lower degrees from those of the highest.
  const int Pm = p->P;
  for (int i = 0; i + 1 < p->deg.n; ++i) {
    if (!p->deg_used[i]) continue;   // no entry reads these proxy charges
    const int Pi = p->deg.d[i] + 1;
    k_mode3<<<T.nclusters, kUpThreads, mode3_smem_bytes(Pm, Pi), s>>>(T.nclusters, p->xfer[i], Pm, 1,
                                                                      Pm, Pi, p->qhat, p->qhat_d[i], 0);
    BL_LAUNCHED(cnt.launches);
  }
  return BLDTT_OK;
}

// ---------------------------------------------------------------------------
// Source pool: leaf particles then proxy points, each block padded to kChunk
// ---------------------------------------------------------------------------
// FP32_BULK pool entries are the frame coordinates (frame_main) of their
// point relative to the frame centre c (a float) of their chunk of kChunk
// entries; the interaction kernel moves its targets into each chunk's frame
// with the same expression.  A chunk is stored as 32 pair records
// {x0,x1, y0,y1, z0,z1, q0,q1}.
__device__ __forceinline__ float frame_coord(double v, float c) {
  float hi, lo;
  split_f64(v, hi, lo);
  return frame_main(hi, lo, c);
}

__device__ __forceinline__ void put(float4* pool, const float4* frame, int64_t i, double x, double y,
                                    double z, double q) {
  const float4 f = frame[kChunkInfo * (i / kChunk)];
  const int64_t j = i % kChunk;
  float* r = reinterpret_cast<float*>(pool) + ((i / kChunk) * (kChunk / 2) + j / 2) * 8 + (j & 1);
  r[0] = frame_coord(x, f.x);
  r[2] = frame_coord(y, f.y);
  r[4] = frame_coord(z, f.z);
  r[6] = (float)q;
}
__device__ __forceinline__ void put(double4* pool, const float4*, int64_t i, double x, double y,
                                    double z, double q) {
  pool[i] = make_double4(x, y, z, q);
}

template <typename Vec>
__global__ void k_pool_particles(const int32_t* __restrict__ leaf_ids, const int32_t* __restrict__ begin,
                                 const int32_t* __restrict__ end, const int32_t* __restrict__ pad_prefix,
                                 const float4* __restrict__ frame, const double* __restrict__ x,
                                 const double* __restrict__ y, const double* __restrict__ z,
                                 const double* __restrict__ q, Vec* __restrict__ pool) {
  const int lf = blockIdx.x;
  const int c = leaf_ids[lf];
  const int64_t o = pad_prefix[lf];
  for (int32_t i = begin[c] + threadIdx.x; i < end[c]; i += blockDim.x)
    put(pool, frame, o + (i - begin[c]), x[i], y[i], z[i], q[i]);
}

template <typename Vec>
__global__ void k_pool_proxies(int n, int np_pad, int64_t base, const double* __restrict__ nodes,
                               const float4* __restrict__ frame, const double* __restrict__ qhat,
                               Vec* __restrict__ pool) {
  const int c = blockIdx.x;
  const int P = n + 1, np = P * P * P;
  const double* nd = nodes + (int64_t)c * 3 * P;
  for (int k = threadIdx.x; k < np; k += blockDim.x) {
    int k1 = k / (P * P), k2 = (k / P) % P, k3 = k % P;
    put(pool, frame, base + (int64_t)c * np_pad + k, nd[k1], nd[P + k2], nd[2 * P + k3],
        qhat[(int64_t)c * np + k]);
  }
}

int build_pool(bldtt_plan* p, cudaStream_t s) {
  Counters& cnt = p->compute_counter;
  const Tree& T = p->st;
  const bool f32 = p->precision == BLDTT_FP32_BULK;
  size_t esz = f32 ? sizeof(float4) : sizeof(double4);
  BL_CUDA(cudaMemsetAsync(p->pool, 0, (size_t)p->pool_len * esz, s));
  if (f32) {
    k_pool_particles<float4><<<T.nleaves, 256, 0, s>>>(T.leaf_ids, T.begin, T.end, p->pad_prefix,
                                                       p->chunk_frame, T.x, T.y, T.z, p->q_tree,
                                                       (float4*)p->pool);
    BL_LAUNCHED(cnt.launches);
    for (int i = 0; i < p->deg.n; ++i) {
      if (!p->deg_used[i]) continue;
      k_pool_proxies<float4><<<T.nclusters, 256, 0, s>>>(p->deg.d[i], p->deg.np_pad[i],
                                                         p->deg.proxy_base[i], p->nodes_s[i],
                                                         p->chunk_frame, p->qhat_d[i],
                                                         (float4*)p->pool);
      if (i + 1 < p->deg.n) BL_LAUNCHED(cnt.launches);
    }
  } else {
    k_pool_particles<double4><<<T.nleaves, 256, 0, s>>>(T.leaf_ids, T.begin, T.end, p->pad_prefix,
                                                        p->chunk_frame, T.x, T.y, T.z, p->q_tree,
                                                        (double4*)p->pool);
    BL_LAUNCHED(cnt.launches);
    for (int i = 0; i < p->deg.n; ++i) {
      if (!p->deg_used[i]) continue;
      k_pool_proxies<double4><<<T.nclusters, 256, 0, s>>>(p->deg.d[i], p->deg.np_pad[i],
                                                          p->deg.proxy_base[i], p->nodes_s[i],
                                                          p->chunk_frame, p->qhat_d[i],
                                                          (double4*)p->pool);
      if (i + 1 < p->deg.n) BL_LAUNCHED(cnt.launches);
    }
  }
  BL_LAUNCHED(cnt.launches);
  return BLDTT_OK;
}

// Description of every pool chunk (kChunkInfo float4 per chunk):
//  [0] frame centre c (floats: the rounded centre of the chunk's bounding box
//      for particles, the rounded cluster centre for proxies), real entries;
//  [1] half-extents e of the chunk's entries around c (rounded up) and the
//      near distance tau = 0.3 |e| (particle chunks; -inf for proxy chunks).
// A target whose frame coordinates x'' satisfy max_d (|x''_d| - e_d) >= tau is
// at distance r >= tau from every entry, so the FP32 rounding of the two frame
// coordinates (at most u |x''| and u |e|, |x''| <= r + |e|) changes r by at
// most sqrt(3) u (1 + 2|e|/tau) r < 14 u r.  Nearer targets add the frame
// residuals of both points (the interaction kernel's careful path), which
// restores a relative error of a few u at any r > 0.  Proxy chunks need no
// such path: the MAC keeps every target at r > (1 - theta) R from them.
__device__ __forceinline__ void store_chunk(float4* info, int64_t q, const double* c, const double* e,
                                            int count, bool particles) {
  float cf[3], ef[3];
  double e2 = 0.0;
  for (int d = 0; d < 3; ++d) {
    cf[d] = (float)c[d];
    double ed = e[d] + fabs(c[d] - (double)cf[d]);
    ef[d] = __double2float_ru(ed);
    e2 += (double)ef[d] * (double)ef[d];
  }
  const float tau = particles ? __double2float_ru(0.3 * sqrt(e2)) : -INFINITY;
  info[kChunkInfo * q] = make_float4(cf[0], cf[1], cf[2], __int_as_float(count));
  info[kChunkInfo * q + 1] = make_float4(ef[0], ef[1], ef[2], tau);
}

// One CTA per source leaf, one warp per chunk of the leaf's pool segment.
__global__ void k_frames_particles(const int32_t* __restrict__ leaf_ids, const int32_t* __restrict__ begin,
                                   const int32_t* __restrict__ end, const int32_t* __restrict__ pad_prefix,
                                   const double* __restrict__ x, const double* __restrict__ y,
                                   const double* __restrict__ z, float4* __restrict__ frame) {
  const int lf = blockIdx.x;
  const int c = leaf_ids[lf];
  const int64_t q0 = pad_prefix[lf] / kChunk, q1 = pad_prefix[lf + 1] / kChunk;
  const int lane = threadIdx.x & 31;
  for (int64_t q = q0 + (threadIdx.x >> 5); q < q1; q += blockDim.x >> 5) {
    const int64_t b = begin[c] + (q - q0) * kChunk;
    const int64_t e = min((int64_t)end[c], b + kChunk);
    // exact minima and maxima, on the order-preserving keys
    long long kn[3] = {kKeyPosInf, kKeyPosInf, kKeyPosInf}, kx[3] = {kKeyNegInf, kKeyNegInf, kKeyNegInf};
    for (int64_t i = b + lane; i < e; i += 32) {
      const long long v[3] = {okey(x[i]), okey(y[i]), okey(z[i])};
      for (int d = 0; d < 3; ++d) {
        kn[d] = min(kn[d], v[d]);
        kx[d] = max(kx[d], v[d]);
      }
    }
    for (int d = 0; d < 3; ++d)
      for (int off = 16; off; off >>= 1) {
        kn[d] = min(kn[d], __shfl_xor_sync(0xffffffffu, kn[d], off));
        kx[d] = max(kx[d], __shfl_xor_sync(0xffffffffu, kx[d], off));
      }
    if (lane == 0) {
      double c3[3], e3[3], mn[3], mx[3];
      for (int d = 0; d < 3; ++d) {
        mn[d] = okey_inv(kn[d]);
        mx[d] = okey_inv(kx[d]);
      }
      for (int d = 0; d < 3; ++d) {
        c3[d] = b < e ? 0.5 * (mn[d] + mx[d]) : 0.0;
        e3[d] = b < e ? 0.5 * (mx[d] - mn[d]) : 0.0;
      }
      store_chunk(frame, q, c3, e3, (int)(e > b ? e - b : 0), true);
    }
  }
}

__global__ void k_frames_proxies(int32_t nclusters, int64_t first_chunk, int32_t chunks_per_cluster,
                                 int32_t np, const double* __restrict__ center,
                                 const double* __restrict__ box, float4* __restrict__ frame) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nclusters * chunks_per_cluster) return;
  const int64_t c = t / chunks_per_cluster;
  const int k = (int)(t % chunks_per_cluster);
  double e3[3];
  for (int d = 0; d < 3; ++d) e3[d] = 0.5 * (box[c * 6 + 3 + d] - box[c * 6 + d]);
  store_chunk(frame, first_chunk + t, center + c * 3, e3, min(kChunk, np - k * kChunk), false);
}

// Frame residuals of the pool's particles, in the pool's pair-record layout
// (x0,x1, y0,y1, z0,z1, unused): read only by the careful path.
__global__ void k_pool_residuals(const int32_t* __restrict__ leaf_ids, const int32_t* __restrict__ begin,
                                 const int32_t* __restrict__ end, const int32_t* __restrict__ pad_prefix,
                                 const float4* __restrict__ frame, const double* __restrict__ x,
                                 const double* __restrict__ y, const double* __restrict__ z,
                                 float* __restrict__ res) {
  const int lf = blockIdx.x;
  const int c = leaf_ids[lf];
  const int64_t o = pad_prefix[lf];
  for (int32_t i = begin[c] + threadIdx.x; i < end[c]; i += blockDim.x) {
    const int64_t k = o + (i - begin[c]);
    const float4 f = frame[kChunkInfo * (k / kChunk)];
    const int64_t j = k % kChunk;
    float* r = res + ((k / kChunk) * (kChunk / 2) + j / 2) * 8 + (j & 1);
    const double v[3] = {x[i], y[i], z[i]};
    const float cf[3] = {f.x, f.y, f.z};
    for (int d = 0; d < 3; ++d) {
      float hi, lo;
      split_f64(v[d], hi, lo);
      r[2 * d] = frame_resid(hi, lo, cf[d]);
    }
  }
}

int build_chunk_frames(bldtt_plan* p, cudaStream_t s) {
  Counters& cnt = p->setup_counter;
  const Tree& T = p->st;
  const int64_t nchunks = p->pool_len / kChunk;
  BL_TRY(dalloc_n(&p->chunk_frame, (size_t)nchunks * kChunkInfo, s));
  const int64_t pchunks = p->pool_particles / kChunk;
  if (pchunks > 0) {
    k_frames_particles<<<T.nleaves, 128, 0, s>>>(T.leaf_ids, T.begin, T.end, p->pad_prefix, T.x, T.y,
                                                 T.z, p->chunk_frame);
    BL_LAUNCHED(cnt.launches);
  }
  for (int i = 0; i < p->deg.n; ++i) {
    if (!p->deg_used[i]) continue;
    const int32_t cpc = p->deg.np_pad[i] / kChunk;
    k_frames_proxies<<<nblk((int64_t)T.nclusters * cpc, 256), 256, 0, s>>>(
        T.nclusters, p->deg.proxy_base[i] / kChunk, cpc, p->deg.np[i], T.center, T.box,
        p->chunk_frame);
    BL_LAUNCHED(cnt.launches);
  }
  if (p->precision == BLDTT_FP32_BULK && pchunks > 0) {
    BL_TRY(dalloc_n(&p->pool_res, (size_t)p->pool_particles * 4, s));
    BL_CUDA(cudaMemsetAsync(p->pool_res, 0, (size_t)p->pool_particles * 4 * sizeof(float), s));
    k_pool_residuals<<<T.nleaves, 256, 0, s>>>(T.leaf_ids, T.begin, T.end, p->pad_prefix,
                                               p->chunk_frame, T.x, T.y, T.z, p->pool_res);
    BL_LAUNCHED(cnt.launches);
  }
  return BLDTT_OK;
}

// ---------------------------------------------------------------------------
// Downward pass
// ---------------------------------------------------------------------------

// Eq. (20) as three mode products with the transposed U_d, one CTA per
// (cluster, k1'): phi(t^c)[k1'][k2'][k3'] += sum_c U3[c][k3'] sum_b U2[b][k2']
// sum_a U1[a][k1'] phi(t^par)[a][b][c].
__global__ void __launch_bounds__(kXferThreads) k_down_parent(int32_t ls, const int32_t* __restrict__ parent,
                                                             const double* __restrict__ U, int n,
                                                             double* __restrict__ phit) {
  __shared__ double T1[kMaxP * kMaxP], T2[kMaxP * kMaxP];
  const int P = n + 1, P2 = P * P, np = P2 * P;
  const int c = ls + blockIdx.x, k1 = blockIdx.y;
  const double* Uc = U + (int64_t)c * 3 * P2;
  const double* A = phit + (int64_t)parent[c] * np;
  for (int o = threadIdx.x; o < P2; o += blockDim.x) {       // (b, c)
    double v = 0.0;
    for (int a = 0; a < P; ++a) v += Uc[a * P + k1] * A[a * P2 + o];
    T1[o] = v;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < P2; o += blockDim.x) {       // (k2', c)
    const int k2 = o / P, cc = o % P;
    double v = 0.0;
    for (int b = 0; b < P; ++b) v += Uc[P2 + b * P + k2] * T1[b * P + cc];
    T2[o] = v;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < P2; o += blockDim.x) {       // (k2', k3')
    const int k2 = o / P, k3 = o % P;
    double v = 0.0;
    for (int cc = 0; cc < P; ++cc) v += Uc[2 * P2 + cc * P + k3] * T2[k2 * P + cc];
    phit[(int64_t)c * np + k1 * P2 + o] += v;
  }
}

constexpr int kDownThreads = 128;

// Eq. (21) for every target leaf, then phi = (PP + PC part) + interpolated
// proxy potentials, scattered back to input order.
template <bool F32>
__global__ void __launch_bounds__(kDownThreads) k_down_leaf(
    const int32_t* __restrict__ leaf_ids, const int32_t* __restrict__ begin,
    const int32_t* __restrict__ end, const double* __restrict__ x, const double* __restrict__ y,
    const double* __restrict__ z, const int32_t* __restrict__ perm, const double* __restrict__ nodes,
    int n, const double* __restrict__ phit, const double* __restrict__ phi_near,
    double* __restrict__ phi_user) {
  using T = typename std::conditional<F32, float, double>::type;
  extern __shared__ double smem[];
  const int P = n + 1, np = P * P * P;
  const int stride = 3 * P + ((3 * P) % 2 == 0 ? 1 : 0);   // odd: conflict-free rows
  const int tstride = P | 1;
  double* snodes = smem;                                    // [3][P]
  double* sL = snodes + 3 * P;                              // [threads][stride]
  T* sphi = reinterpret_cast<T*>(sL + (size_t)kDownThreads * stride);   // [np]
  T* sLz = sphi + np;                                       // [threads][tstride] z factors in T
  float* shl = reinterpret_cast<float*>(sLz + (size_t)kDownThreads * tstride);   // [3][2][kMaxP]
  const int c = leaf_ids[blockIdx.x];
  for (int t = threadIdx.x; t < 3 * P; t += blockDim.x) {
    const double v = nodes[(int64_t)c * 3 * P + t];
    snodes[t] = v;
    float h, l;
    split_f64(v, h, l);
    shl[(t / P) * 2 * kMaxP + t % P] = h;
    shl[(t / P) * 2 * kMaxP + kMaxP + t % P] = l;
  }
  for (int o = threadIdx.x; o < np; o += blockDim.x) sphi[o] = (T)phit[(int64_t)c * np + o];
  __syncthreads();
  double* L = sL + (size_t)threadIdx.x * stride;
  float* Lf = reinterpret_cast<float*>(L);                  // FP32_BULK: the basis in float
  for (int32_t i = begin[c] + threadIdx.x; i < end[c]; i += blockDim.x) {
    T* Lz = sLz + (size_t)threadIdx.x * tstride;
    double acc = 0.0;
    if constexpr (F32) {
      basis_1d_f32(x[i], shl, n, Lf, 1);
      basis_1d_f32(y[i], shl + 2 * kMaxP, n, Lf + P, 1);
      basis_1d_f32(z[i], shl + 4 * kMaxP, n, Lz, 1);
      // s2 in float; the two outer sums compensated (exact products by FMA,
      // exact sums by TwoSum), so they add no rounding beyond s2's own.
      CompSum a1;
      for (int k1 = 0; k1 < P; ++k1) {
        CompSum a2;
        for (int k2 = 0; k2 < P; ++k2) {
          const T* row = sphi + (k1 * P + k2) * P;
          T s2 = (T)0;
          for (int k3 = 0; k3 < P; ++k3) s2 += Lz[k3] * row[k3];
          a2.add_prod(Lf[P + k2], (float)s2);
        }
        a1.add_prod(Lf[k1], a2.s);
        a1.add_prod(Lf[k1], a2.c);
      }
      acc = (double)a1.s + (double)a1.c;
    } else {
      basis_1d<double>(x[i], snodes, n, L, 1);
      basis_1d<double>(y[i], snodes + P, n, L + P, 1);
      basis_1d<double>(z[i], snodes + 2 * P, n, L + 2 * P, 1);
      for (int k3 = 0; k3 < P; ++k3) Lz[k3] = (T)L[2 * P + k3];
      for (int k1 = 0; k1 < P; ++k1) {
        double s1 = 0.0;
        for (int k2 = 0; k2 < P; ++k2) {
          const T* row = sphi + (k1 * P + k2) * P;
          T s2 = (T)0;
          for (int k3 = 0; k3 < P; ++k3) s2 += Lz[k3] * row[k3];
          s1 += L[P + k2] * (double)s2;
        }
        acc += L[k1] * s1;
      }
    }
    phi_user[perm[i]] = phi_near[i] + acc;
  }
}

// FP32_BULK form of k_down_leaf for a grid of P points fixed at compile time:
// the particle's three basis rows stay in registers and each (k1, k2) row of
// the proxy potentials is read as float4 broadcasts; the arithmetic and its
// order are those of k_down_leaf<true>.  A leaf's particles are shared by
// kDownF32Split CTAs (blockIdx.y), which balances the SMs at a few leaves each.
constexpr int kDownF32Threads = 256;
constexpr int kDownF32Split = 2;

template <int P>
__global__ void __launch_bounds__(kDownF32Threads, 3) k_down_leaf_f32(
    const int32_t* __restrict__ leaf_ids, const int32_t* __restrict__ begin,
    const int32_t* __restrict__ end, const double* __restrict__ x, const double* __restrict__ y,
    const double* __restrict__ z, const int32_t* __restrict__ perm, const double* __restrict__ nodes,
    const double* __restrict__ phit, const double* __restrict__ phi_near,
    double* __restrict__ phi_user) {
  constexpr int RS = (P + 3) / 4 * 4, NP = P * P * P;
  __shared__ __align__(16) float sphi[P * P][RS];
  __shared__ float shl[3][2 * kMaxP];
  const int c = leaf_ids[blockIdx.x];
  for (int t = threadIdx.x; t < 3 * P; t += blockDim.x) {
    float h, l;
    split_f64(nodes[(int64_t)c * 3 * P + t], h, l);
    shl[t / P][t % P] = h;
    shl[t / P][kMaxP + t % P] = l;
  }
  for (int o = threadIdx.x; o < P * P * RS; o += blockDim.x) {
    const int row = o / RS, k = o % RS;
    sphi[row][k] = k < P ? (float)phit[(int64_t)c * NP + row * P + k] : 0.f;
  }
  __syncthreads();
  for (int32_t i = begin[c] + blockIdx.y * blockDim.x + threadIdx.x; i < end[c];
       i += kDownF32Split * blockDim.x) {
    float L1[P], L2[P], L3[P];
    basis_f32_fixed<P>(x[i], shl[0], L1);
    basis_f32_fixed<P>(y[i], shl[1], L2);
    basis_f32_fixed<P>(z[i], shl[2], L3);
    CompSum a1;
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) {
      CompSum a2;
#pragma unroll
      for (int k2 = 0; k2 < P; ++k2) {
        float r[RS];
        const float4* row = reinterpret_cast<const float4*>(sphi[k1 * P + k2]);
#pragma unroll
        for (int v = 0; v < RS / 4; ++v) {
          const float4 t = row[v];
          r[4 * v] = t.x;
          r[4 * v + 1] = t.y;
          r[4 * v + 2] = t.z;
          r[4 * v + 3] = t.w;
        }
        float s2 = 0.f;
#pragma unroll
        for (int k3 = 0; k3 < P; ++k3) s2 = fmaf(L3[k3], r[k3], s2);
        a2.add_prod(L2[k2], s2);
      }
      a1.add_prod(L1[k1], a2.s);
      a1.add_prod(L1[k1], a2.c);
    }
    phi_user[perm[i]] = phi_near[i] + ((double)a1.s + (double)a1.c);
  }
}

int downward_pass(bldtt_plan* p, double* phi_user, cudaStream_t s) {
  Counters& cnt = p->compute_counter;
  const Tree& T = p->tt;
  // Proxy potentials of the lower degrees onto the highest degree's grid.
  for (int i = 0; i + 1 < p->deg.n; ++i) {
    if (!p->deg_used[i]) continue;   // no CP/CC entry wrote these proxy potentials
    const int Pi = p->deg.d[i] + 1, Pm = p->P;
    k_mode3<<<T.nclusters, kUpThreads, mode3_smem_bytes(Pi, Pm), s>>>(T.nclusters, p->xfer[i], 1, Pm,
                                                                      Pi, Pm, p->phit_d[i], p->phit, 1);
    BL_LAUNCHED(cnt.launches);
  }
  for (int lvl = 1; lvl < T.nlevels; ++lvl) {
    int32_t ls = T.level_start[lvl], nl = T.level_start[lvl + 1] - ls;
    k_down_parent<<<dim3(nl, p->P), kXferThreads, 0, s>>>(ls, T.parent, T.xfer_u, p->n, p->phit);
    BL_LAUNCHED(cnt.launches);
  }
  const int P = p->P, np = p->np;
  const int stride = 3 * P + ((3 * P) % 2 == 0 ? 1 : 0);
  const size_t tz = (size_t)kDownThreads * (P | 1);
  // Leaves written: all, or the leaf-order range of one shard.
  const int32_t leaf_lo = p->down_hi < 0 ? 0 : p->down_lo;
  const int32_t nleaves = (p->down_hi < 0 ? T.nleaves : p->down_hi) - leaf_lo;
  if (nleaves <= 0) return BLDTT_OK;
  const int32_t* leaf_ids = T.leaf_ids + leaf_lo;
  if (p->precision == BLDTT_FP32_BULK && p->down_engine == BLDTT_PASS_TENSOR && leaf_tc_supported(P))
    return down_leaf_tc(p, leaf_ids, nleaves, phi_user, s);
  if (p->precision == BLDTT_FP32_BULK && P >= kFixedPMin && P <= kFixedPMax) {
    switch (P) {
#define BL_DOWN_LEAF(PP)                                                                      \
  case PP:                                                                                    \
    k_down_leaf_f32<PP><<<dim3(nleaves, kDownF32Split), kDownF32Threads, 0, s>>>(leaf_ids, T.begin, T.end, T.x, \
                                                              T.y, T.z, T.perm, T.nodes,      \
                                                              p->phit, p->phi_near, phi_user); \
    break;
      BL_DOWN_LEAF(2) BL_DOWN_LEAF(3) BL_DOWN_LEAF(4) BL_DOWN_LEAF(5)
      BL_DOWN_LEAF(6) BL_DOWN_LEAF(7) BL_DOWN_LEAF(8) BL_DOWN_LEAF(9)
#undef BL_DOWN_LEAF
    }
  } else if (p->precision == BLDTT_FP32_BULK) {
    size_t bytes = sizeof(double) * (3 * P + (size_t)kDownThreads * stride) + sizeof(float) * (np + tz) +
                   sizeof(float) * 6 * kMaxP;
    k_down_leaf<true><<<nleaves, kDownThreads, bytes, s>>>(leaf_ids, T.begin, T.end, T.x, T.y,
                                                              T.z, T.perm, T.nodes, p->n, p->phit,
                                                              p->phi_near, phi_user);
  } else {
    size_t bytes = sizeof(double) * (3 * P + (size_t)kDownThreads * stride + np + tz) +
                   sizeof(float) * 6 * kMaxP;
    k_down_leaf<false><<<nleaves, kDownThreads, bytes, s>>>(leaf_ids, T.begin, T.end, T.x, T.y,
                                                               T.z, T.perm, T.nodes, p->n, p->phit,
                                                               p->phi_near, phi_user);
  }
  BL_LAUNCHED(cnt.launches);
  return BLDTT_OK;
}

// Opt the dynamic-shared-memory kernels in to large allocations (n up to 16).
int configure_pass_kernels() {
  int big = 200 * 1024;
  BL_CUDA(cudaFuncSetAttribute(k_down_leaf<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  BL_CUDA(cudaFuncSetAttribute(k_down_leaf<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  BL_CUDA(cudaFuncSetAttribute(k_mode3, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  return BLDTT_OK;
}

// ---------------------------------------------------------------------------
// Degree sets
// ---------------------------------------------------------------------------
__global__ void k_nodes_degree(int32_t C, int degree, const double* __restrict__ box,
                               double* __restrict__ nodes) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  const int P = degree + 1;
  const double* b = box + (int64_t)c * 6;
  for (int d = 0; d < 3; ++d) {   // the same expression as the tree's own proxy points
    const double lo = b[d], hi = b[3 + d];
    const double cc = __dmul_rn(__dadd_rn(lo, hi), 0.5);
    const double h = __dmul_rn(__dsub_rn(hi, lo), 0.5);
    for (int k = 0; k < P; ++k)
      nodes[((int64_t)c * 3 + d) * P + k] = __dadd_rn(cc, __dmul_rn(h, cheb_point(k, degree)));
  }
}

// Host: Chebyshev points of the 2nd kind on [-1, 1] and the barycentric basis
// with the coincident-point guard (Eqs. (3)-(5)).
static double host_cheb(int k, int n) {
  if (2 * k == n) return 0.0;
  if (2 * k < n) return std::cos(M_PI * (double)k / (double)n);
  return -std::cos(M_PI * (double)(n - k) / (double)n);
}
static void host_basis(double x, int n, double* out) {
  double sum = 0.0, r[kMaxP];
  int hit = -1;
  for (int k = 0; k <= n; ++k) {
    const double d = x - host_cheb(k, n);
    if (d == 0.0 && hit < 0) hit = k;
    double w = (k == 0 || k == n) ? 0.5 : 1.0;
    if (k & 1) w = -w;
    r[k] = d == 0.0 ? 0.0 : w / d;
    sum += r[k];
  }
  for (int k = 0; k <= n; ++k) out[k] = hit >= 0 ? (k == hit ? 1.0 : 0.0) : r[k] / sum;
}

static int transfer_matrices(Tree& T, int n, cudaStream_t s, Counters& cnt) {
  const int P = n + 1;
  const int64_t work = (int64_t)T.nclusters * 3 * P;
  BL_TRY(dalloc_n(&T.xfer_u, (size_t)work * P, s));
  k_transfer_matrices<<<nblk(work, 128), 128, 0, s>>>(T.nclusters, T.parent, T.nodes, n, T.xfer_u);
  BL_LAUNCHED(cnt.launches);
  return BLDTT_OK;
}

int setup_degrees(bldtt_plan* p, cudaStream_t s) {
  Counters& cnt = p->setup_counter;
  const int m = p->deg.n - 1, nmax = p->deg.d[m];
  BL_TRY(transfer_matrices(p->tt, nmax, s, cnt));
  if (p->shared_tree)
    p->st.xfer_u = p->tt.xfer_u;
  else
    BL_TRY(transfer_matrices(p->st, nmax, s, cnt));
  p->nodes_t[m] = p->tt.nodes;
  p->nodes_s[m] = p->st.nodes;
  for (int i = 0; i < m; ++i) {
    const int d = p->deg.d[i], P = d + 1;
    BL_TRY(dalloc_n(&p->nodes_t[i], (size_t)p->tt.nclusters * 3 * P, s));
    BL_TRY(dalloc_n(&p->nodes_s[i], (size_t)p->st.nclusters * 3 * P, s));
    k_nodes_degree<<<nblk(p->tt.nclusters, 128), 128, 0, s>>>(p->tt.nclusters, d, p->tt.box, p->nodes_t[i]);
    BL_LAUNCHED(cnt.launches);
    k_nodes_degree<<<nblk(p->st.nclusters, 128), 128, 0, s>>>(p->st.nclusters, d, p->st.box, p->nodes_s[i]);
    BL_LAUNCHED(cnt.launches);
    std::vector<double> A((size_t)P * (nmax + 1));
    std::vector<double> col(P);
    for (int kp = 0; kp <= nmax; ++kp) {   // A[k][k'] = L^(d)_k(s^(nmax)_k')
      host_basis(host_cheb(kp, nmax), d, col.data());
      for (int k = 0; k < P; ++k) A[(size_t)k * (nmax + 1) + kp] = col[k];
    }
    BL_TRY(dalloc_n(&p->xfer[i], A.size(), s));
    BL_CUDA(cudaMemcpyAsync(p->xfer[i], A.data(), A.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    BL_TRY(dalloc_n(&p->qhat_d[i], (size_t)p->st.nclusters * p->deg.np[i], s));
    BL_TRY(dalloc_n(&p->phit_d[i], (size_t)p->tt.nclusters * p->deg.np[i], s));
    BL_CUDA(cudaStreamSynchronize(s));   // the host matrix goes out of scope
  }
  return BLDTT_OK;
}

}  // namespace bldtt
