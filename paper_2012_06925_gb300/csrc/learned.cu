// Learned pair selector: a bfloat16 network that replaces the MAC of Alg. 2
// by a per-pair choice of interaction type and interpolation degree, its
// training kernels, and the per-pair error labels it is trained on.
//
// Features of a pair (t, s), R = |c_t - c_s| > 0, (r_t + r_s)/R < 1:
//   f = (plog2|C_t|/16, plog2|C_s|/16, r_t/R, r_s/R, (r_t + r_s)/R, kR/(1 + kR))
// in FP64 (plog2(m) = e + (f - 1) for m = f 2^e, 1 <= f < 2), rounded to
// float and then to bfloat16.  Network: three hidden ReLU layers of 64 and a
// linear output of 3 per degree, y[3 i + t] ~ log10 of the relative error of
// (PC, CP, CC)[t] at degree d[i] on the pair.  Every layer computes
// z_j = b_j + sum_k w_jk a_k in float, k in increasing order, with bf16
// weights and activations (their products are exact in float), then
// a_j = bf16(max(z_j, 0)); the same arithmetic on any device gives the same
// bits.  The cheapest option with y <= log10(budget) is taken (PP if it costs
// no more); none feasible means no approximation; features outside the
// training box fall back to the MAC.
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "internal.cuh"

namespace bldtt {

constexpr int kSelWarps = 8;   // pairs (or samples) per block, one warp each

__host__ __device__ inline int64_t sel_weight_count(int nout) {
  return (int64_t)kHidden * kFeatures + 2 * (int64_t)kHidden * kHidden + (int64_t)nout * kHidden;
}
__host__ __device__ inline int64_t sel_bias_count(int nout) { return 3 * (int64_t)kHidden + nout; }
// Offsets of W1..W4 and b1..b4 inside the packed master-parameter array.
struct ParamLayout {
  int64_t w[4], b[4], total;
  __host__ __device__ explicit ParamLayout(int nout) {
    const int64_t in[4] = {kFeatures, kHidden, kHidden, kHidden};
    const int64_t out[4] = {kHidden, kHidden, kHidden, nout};
    int64_t o = 0;
    for (int l = 0; l < 4; ++l) {
      w[l] = o;
      o += in[l] * out[l];
      b[l] = o;
      o += out[l];
    }
    total = o;
  }
};

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// ---- features ---------------------------------------------------------------
__device__ __forceinline__ double plog2(int64_t m) {
  int e;
  const double f = frexp((double)m, &e);   // m = f 2^e, 0.5 <= f < 1
  return __dadd_rn((double)(e - 1), __dsub_rn(__dmul_rn(2.0, f), 1.0));
}

struct PairTrees {
  const int32_t *tb, *te, *sb, *se;
  const double *tc, *sc, *tr, *sr;
};

// The FP64 features of pair (t, s); false if it cannot be approximated.
__device__ bool pair_features(const PairTrees& T, int t, int s, double kappa, double* f) {
  const double* ct = T.tc + (int64_t)t * 3;
  const double* cs = T.sc + (int64_t)s * 3;
  const double dx = __dsub_rn(ct[0], cs[0]), dy = __dsub_rn(ct[1], cs[1]), dz = __dsub_rn(ct[2], cs[2]);
  const double R = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
  if (!(R > 0.0)) return false;
  const double rt = T.tr[t], rs = T.sr[s];
  const double sep = __ddiv_rn(__dadd_rn(rt, rs), R);
  if (!(sep < 1.0)) return false;
  const double kr = __dmul_rn(kappa, R);
  f[0] = __ddiv_rn(plog2(T.te[t] - T.tb[t]), 16.0);
  f[1] = __ddiv_rn(plog2(T.se[s] - T.sb[s]), 16.0);
  f[2] = __ddiv_rn(rt, R);
  f[3] = __ddiv_rn(rs, R);
  f[4] = sep;
  f[5] = __ddiv_rn(kr, __dadd_rn(1.0, kr));
  return true;
}

// ---- network forward (one warp per sample) -----------------------------------
struct NetSmem {
  const __nv_bfloat16* w;   // W1 | W2 | W3 | W4, each stored transposed [in][out] in shared memory
  const float* b;           // b1 | b2 | b3 | b4
  int nout;
};

// z_j for neurons j = lane, lane + 32 (or lane < n for the output layer);
// Wt is the layer's weights transposed ([K][J]), so the lanes of a warp read
// consecutive entries; the sum over k runs in increasing order.
__device__ __forceinline__ float neuron(const __nv_bfloat16* Wt, const float* b, int j, int K, int J,
                                        const float* a) {
  float z = b[j];
  for (int k = 0; k < K; ++k) z = fmaf(__bfloat162float(Wt[(int64_t)k * J + j]), a[k], z);
  return z;
}

// x: 6 bf16-rounded inputs in shared memory; act: 2 x 64 floats of this warp.
// Writes y[lane] for lane < nout.  If keep != NULL the pre-activations and
// activations of each layer are stored there ([z1 a1 z2 a2 z3 a3] x 64).
__device__ float mlp_forward_warp(const NetSmem& net, const float* x, float* act, float* keep) {
  const int lane = threadIdx.x & 31;
  const __nv_bfloat16* W = net.w;
  const float* b = net.b;
  const int K[3] = {kFeatures, kHidden, kHidden};
  const float* in = x;
  float* bufs[2] = {act, act + kHidden};
  for (int l = 0; l < 3; ++l) {
    float* out = bufs[l & 1];
    float zz[2];
    for (int h = 0; h < 2; ++h) {
      const int j = lane + 32 * h;
      zz[h] = neuron(W, b, j, K[l], kHidden, in);
    }
    __syncwarp();
    for (int h = 0; h < 2; ++h) {
      const int j = lane + 32 * h;
      const float a = bf16r(zz[h] > 0.f ? zz[h] : 0.f);
      out[j] = a;
      if (keep) {
        keep[(2 * l) * kHidden + j] = zz[h];
        keep[(2 * l + 1) * kHidden + j] = a;
      }
    }
    __syncwarp();
    W += (int64_t)kHidden * K[l];
    b += kHidden;
    in = out;
  }
  return lane < net.nout ? neuron(W, b, lane, kHidden, net.nout, in) : 0.f;
}

// Load bf16 weights (row-major [out][in] in global memory, transposed to
// [in][out] in shared memory) and float biases.
__device__ void load_net(const __nv_bfloat16* gw, const float* gb, int nout, __nv_bfloat16* sw, float* sb) {
  const int K[4] = {kFeatures, kHidden, kHidden, kHidden};
  const int J[4] = {kHidden, kHidden, kHidden, nout};
  int64_t o = 0;
  for (int l = 0; l < 4; ++l) {
    const int64_t n = (int64_t)K[l] * J[l];
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      const int64_t j = i / K[l], k = i % K[l];
      sw[o + k * J[l] + j] = gw[o + i];
    }
    o += n;
  }
  const int64_t nb = sel_bias_count(nout);
  for (int64_t i = threadIdx.x; i < nb; i += blockDim.x) sb[i] = gb[i];
  __syncthreads();
}

__host__ __device__ inline size_t net_smem_bytes(int nout) {
  size_t w = (size_t)sel_weight_count(nout) * sizeof(__nv_bfloat16);
  w = (w + 15) / 16 * 16;
  return w + (size_t)sel_bias_count(nout) * sizeof(float) +
         (size_t)kSelWarps * (2 * kHidden + 8 + 32) * sizeof(float);
}

// ---- selection inside the traversal -----------------------------------------
struct SelParams {
  int nout, ndeg;
  int np[kMaxDegrees];
  float lo[kFeatures], hi[kFeatures];
  float log_eps;
  double kappa;
  int net;   // 0: no network (MAC fallback everywhere)
};

// Per-warp scratch of k_select: the MLP's activations, then the inputs and
// outputs of the warp's 32 pairs.
constexpr int kSelOutMax = 3 * kMaxDegrees;
constexpr int kSelWarpFloats = 2 * kHidden + 32 * 8 + 32 * kSelOutMax;

__host__ __device__ inline size_t select_smem_bytes(int nout) {
  size_t w = (size_t)sel_weight_count(nout) * sizeof(__nv_bfloat16);
  w = (w + 15) / 16 * 16;
  return w + (size_t)sel_bias_count(nout) * sizeof(float) +
         (size_t)kSelWarps * kSelWarpFloats * sizeof(float);
}

// A warp takes 32 pairs at a time: each lane computes its pair's features (the
// FP64 divisions and square root run on all lanes at once), the warp runs the
// network for every pair inside the box in turn, and each lane decides its own
// pair.  Same arithmetic as one pair per warp.
__global__ void k_select(const int2* __restrict__ pairs, int32_t F, PairTrees T, SelParams sp,
                         const __nv_bfloat16* __restrict__ gw, const float* __restrict__ gb,
                         int16_t* __restrict__ choice) {
  extern __shared__ __align__(16) unsigned char sraw[];
  __nv_bfloat16* sw = reinterpret_cast<__nv_bfloat16*>(sraw);
  size_t wbytes = ((size_t)sel_weight_count(sp.nout) * sizeof(__nv_bfloat16) + 15) / 16 * 16;
  float* sb = reinterpret_cast<float*>(sraw + wbytes);
  float* swarp = sb + sel_bias_count(sp.nout);
  if (sp.net) load_net(gw, gb, sp.nout, sw, sb);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* act = swarp + warp * kSelWarpFloats;
  float* xs = act + 2 * kHidden;      // [32][8]
  float* ys = xs + 32 * 8;            // [32][kSelOutMax]
  const NetSmem net{sw, sb, sp.nout};
  const int64_t stride = (int64_t)gridDim.x * kSelWarps * 32;
  for (int64_t base = ((int64_t)blockIdx.x * kSelWarps + warp) * 32; base < F; base += stride) {
    const int64_t i = base + lane;
    int state = 0;   // 0 no approximation, 1 fallback, 2 network
    int t = 0, s = 0;
    if (i < F) {
      t = pairs[i].x;
      s = pairs[i].y;
      double f[kFeatures];
      if (pair_features(T, t, s, sp.kappa, f)) {
        state = sp.net ? 2 : 1;
        for (int d = 0; d < kFeatures; ++d) {
          const float xd = bf16r(__double2float_rn(f[d]));
          xs[lane * 8 + d] = xd;
          if (xd < sp.lo[d] || xd > sp.hi[d]) state = 1;
        }
      }
    }
    __syncwarp();
    unsigned todo = __ballot_sync(0xffffffffu, state == 2);
    while (todo) {
      const int j = __ffs(todo) - 1;
      todo &= todo - 1;
      const float y = mlp_forward_warp(net, xs + j * 8, act, nullptr);
      if (lane < sp.nout) ys[j * kSelOutMax + lane] = y;
      __syncwarp();
    }
    if (i < F) {
      int16_t c = state == 0 ? kChoiceNoApprox : kChoiceFallback;
      if (state == 2) {
        const float* y = ys + lane * kSelOutMax;
        const int64_t ct = T.te[t] - T.tb[t], cs = T.se[s] - T.sb[s];
        int best = -1;
        int64_t best_cost = 0;
        for (int di = 0; di < sp.ndeg; ++di) {
          const int64_t np = sp.np[di];
          const int64_t cost[3] = {ct * np, np * cs, np * np};
          for (int ty = 0; ty < 3; ++ty)
            if (y[3 * di + ty] <= sp.log_eps && (best < 0 || cost[ty] < best_cost)) {
              best = 1 + 3 * di + ty;
              best_cost = cost[ty];
            }
        }
        c = best < 0 ? kChoiceNoApprox : (ct * cs <= best_cost ? (int16_t)0 : (int16_t)best);
      }
      choice[i] = c;
    }
    __syncwarp();
  }
}

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

static PairTrees pair_trees(const bldtt_plan* p) {
  return PairTrees{p->tt.begin, p->tt.end, p->st.begin, p->st.end,
                   p->tt.center, p->st.center, p->tt.radius, p->st.radius};
}

int select_pairs(bldtt_plan* p, const int2* pairs, int32_t F, int16_t* choice, cudaStream_t s) {
  SelParams sp{};
  sp.nout = p->sel_nout;
  sp.ndeg = p->deg.n;
  for (int i = 0; i < p->deg.n; ++i) sp.np[i] = p->deg.np[i];
  for (int d = 0; d < kFeatures; ++d) {
    sp.lo[d] = p->sel_lo[d];
    sp.hi[d] = p->sel_hi[d];
  }
  sp.log_eps = p->sel_log_eps;
  sp.kappa = p->kappa;
  sp.net = p->selector_net ? 1 : 0;
  const size_t sm = select_smem_bytes(p->sel_nout);
  BL_CUDA(cudaFuncSetAttribute(k_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  unsigned g = nblk(F, kSelWarps * 32);
  if (g > 4096) g = 4096;
  k_select<<<g, 32 * kSelWarps, sm, s>>>(pairs, F, pair_trees(p), sp,
                                          reinterpret_cast<const __nv_bfloat16*>(p->sel_w), p->sel_b,
                                          choice);
  BL_LAUNCHED(p->setup_counter.launches);
  return BLDTT_OK;
}

// ---- training ------------------------------------------------------------------
__global__ void k_to_bf16(const float* __restrict__ params, ParamLayout L, int nout,
                          __nv_bfloat16* __restrict__ w, float* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t in[4] = {kFeatures, kHidden, kHidden, kHidden};
  const int64_t out[4] = {kHidden, kHidden, kHidden, nout};
  int64_t wo = 0, bo = 0;
  for (int l = 0; l < 4; ++l) {
    const int64_t nw = in[l] * out[l];
    if (i < nw) w[wo + i] = __float2bfloat16_rn(params[L.w[l] + i]);
    if (i < out[l]) b[bo + i] = params[L.b[l] + i];
    wo += nw;
    bo += out[l];
  }
}

// Forward of a batch, keeping what the backward pass needs:
// keep[b] = [x(8) | z1 a1 z2 a2 z3 a3 (6 x 64)], y[b][nout].
constexpr int kKeep = 8 + 6 * kHidden;
__global__ void k_mlp_forward(const float* __restrict__ xin, int64_t B, const __nv_bfloat16* __restrict__ gw,
                              const float* __restrict__ gb, int nout, float* __restrict__ y,
                              float* __restrict__ keep) {
  extern __shared__ __align__(16) unsigned char sraw[];
  __nv_bfloat16* sw = reinterpret_cast<__nv_bfloat16*>(sraw);
  size_t wbytes = ((size_t)sel_weight_count(nout) * sizeof(__nv_bfloat16) + 15) / 16 * 16;
  float* sb = reinterpret_cast<float*>(sraw + wbytes);
  float* swarp = sb + sel_bias_count(nout);
  load_net(gw, gb, nout, sw, sb);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* act = swarp + warp * (2 * kHidden + 8 + 32);
  float* x = act + 2 * kHidden;
  const NetSmem net{sw, sb, nout};
  for (int64_t i = (int64_t)blockIdx.x * kSelWarps + warp; i < B; i += (int64_t)gridDim.x * kSelWarps) {
    if (lane < kFeatures) x[lane] = bf16r(xin[i * kFeatures + lane]);
    __syncwarp();
    float* kp = keep ? keep + i * kKeep : nullptr;
    if (kp && lane < kFeatures) kp[lane] = x[lane];
    const float v = mlp_forward_warp(net, x, act, kp ? kp + 8 : nullptr);
    if (lane < nout) y[i * nout + lane] = v;
    __syncwarp();
  }
}

// Deterministic block sums: out[0] = sum mask, out[1] = sum (mask (y - T))^2.
__global__ void k_loss_sums(const float* __restrict__ y, const float* __restrict__ T,
                            const float* __restrict__ mask, int64_t n, float* __restrict__ out) {
  __shared__ double s0[256], s1[256];
  double a = 0.0, b = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double d = (double)mask[i] * ((double)y[i] - (double)T[i]);
    a += mask[i];
    b += d * d;
  }
  s0[threadIdx.x] = a;
  s1[threadIdx.x] = b;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s0[threadIdx.x] += s0[threadIdx.x + w];
      s1[threadIdx.x] += s1[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double cnt = s0[0] > 1.0 ? s0[0] : 1.0;
    out[0] = (float)cnt;
    out[1] = (float)(s1[0] / cnt);
  }
}

// dL/dy = 2 mask (y - T) / cnt.
__global__ void k_out_grad(const float* __restrict__ y, const float* __restrict__ T,
                           const float* __restrict__ mask, int64_t n, const float* __restrict__ sums,
                           float* __restrict__ gy) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) gy[i] = 2.f * mask[i] * (y[i] - T[i]) / sums[0];
}

// dW[j][k] = sum_b g[b][j] a[b][k], db[j] = sum_b g[b][j] (sequential over b).
// a rows: a_of(b) = base + b * stride + off.
__global__ void k_weight_grad(const float* __restrict__ g, int gstride, int J, const float* __restrict__ a,
                              int64_t astride, int aoff, int K, int64_t B, float* __restrict__ dW,
                              float* __restrict__ db) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < (int64_t)J * K) {
    const int j = (int)(t / K), k = (int)(t % K);
    float acc = 0.f;
    for (int64_t b = 0; b < B; ++b) acc = fmaf(g[b * gstride + j], a[b * astride + aoff + k], acc);
    dW[t] = acc;
  } else if (t < (int64_t)J * K + J) {
    const int j = (int)(t - (int64_t)J * K);
    float acc = 0.f;
    for (int64_t b = 0; b < B; ++b) acc += g[b * gstride + j];
    db[j] = acc;
  }
}

// gz_prev[b][k] = (sum_j g[b][j] W[j][k]) [z_prev[b][k] > 0].
__global__ void k_back(const float* __restrict__ g, int J, const __nv_bfloat16* __restrict__ W, int K,
                       const float* __restrict__ keep, int zoff, int64_t B, float* __restrict__ gprev) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * K) return;
  const int64_t b = t / K;
  const int k = (int)(t % K);
  float acc = 0.f;
  for (int j = 0; j < J; ++j) acc = fmaf(g[b * J + j], __bfloat162float(W[(int64_t)j * K + k]), acc);
  gprev[t] = keep[b * kKeep + zoff + k] > 0.f ? acc : 0.f;
}

__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, int64_t n, float lr, float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float b1 = 0.9f, b2 = 0.999f;
  const float mi = b1 * m[i] + (1.f - b1) * g[i];
  const float vi = b2 * v[i] + (1.f - b2) * g[i] * g[i];
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

// ---- per-pair error labels ------------------------------------------------------
template <int KERN>
__device__ __forceinline__ double g64(double dx, double dy, double dz, double kappa) {
  const double r2 = dx * dx + dy * dy + dz * dz;
  if (!(r2 > 0.0)) return 0.0;
  if (KERN == BLDTT_REG_COULOMB) return rsqrt(r2 + kappa * kappa);
  const double ri = rsqrt(r2);
  if (KERN == BLDTT_COULOMB) return ri;
  if (KERN == BLDTT_OSCILLATORY) return ri * sin(kappa * (r2 * ri));
  if (KERN == BLDTT_YUKAWA) return ri * exp(-kappa * (r2 * ri));
  return 1.0 + dx - 2.0 * dy + 3.0 * dz + dx * dy - dy * dz + dx * dx * dz * dz - 0.5 * dy * dy;
}

__device__ __forceinline__ double bary_w(int k, int n) {
  const double w = (k == 0 || k == n) ? 0.5 : 1.0;
  return (k & 1) ? -w : w;
}
// L_k(x), k = 0..n, on the grid `nodes` with the coincident-point guard.
__device__ void basis(double x, const double* nodes, int n, double* out, int stride) {
  double sum = 0.0;
  int hit = -1;
  for (int k = 0; k <= n; ++k) {
    const double d = x - nodes[k];
    if (d == 0.0 && hit < 0) hit = k;
    const double r = d == 0.0 ? 0.0 : bary_w(k, n) / d;
    out[k * stride] = r;
    sum += r;
  }
  for (int k = 0; k <= n; ++k) out[k * stride] = hit >= 0 ? (k == hit ? 1.0 : 0.0) : out[k * stride] / sum;
}

constexpr int kErrThreads = 256;
constexpr int kErrChunk = 32;
constexpr int kErrMaxSources = 4096;   // larger source clusters: an evenly strided subset

struct ErrTrees {
  const int32_t *tb, *te, *sb, *se;
  const double *tbox, *sbox;
  const double *tx, *ty, *tz, *sx, *sy, *sz, *q;
};

// One block per (pair, degree): the relative l2 errors of PC, CP and CC at
// degree d against the exact pair sum (Eq. (6)), on up to S target samples
// spread evenly over C_t.  A source cluster of more than kErrMaxSources
// particles is represented by every stride-th particle (stride =
// ceil(|C_s| / kErrMaxSources)) in the exact sum and in all three
// approximations alike.  err[(pair * ndeg + di) * 3 + type].
template <int KERN>
__global__ void __launch_bounds__(kErrThreads) k_pair_errors(const int32_t* __restrict__ pairs, int64_t npairs,
                                                            ErrTrees T, DegreeSet deg, int S, double kappa,
                                                            double* __restrict__ err) {
  extern __shared__ double sm[];
  const int64_t blk = blockIdx.x;
  const int64_t pi = blk / deg.n;
  const int di = (int)(blk % deg.n);
  if (pi >= npairs) return;
  const int t = pairs[2 * pi], s = pairs[2 * pi + 1];
  const int d = deg.d[di], P = d + 1, np = P * P * P;
  const int32_t tb = T.tb[t], nt = T.te[t] - tb, sb = T.sb[s], ns_all = T.se[s] - sb;
  const int32_t sst = (ns_all + kErrMaxSources - 1) / kErrMaxSources;   // source stride
  const int32_t ns = (ns_all + sst - 1) / sst;                          // sources used
  const int m = nt < S ? nt : S;
  double* tn = sm;                     // [3][P] target nodes
  double* sn = tn + 3 * P;             // [3][P] source nodes
  double* qh = sn + 3 * P;             // [np] proxy charges of C_s
  double* ph = qh + np;                // [np] CP potentials at C_t's proxies
  double* pc2 = ph + np;               // [np] CC potentials at C_t's proxies
  double* Bj = pc2 + np;               // [3][P][kErrChunk] source basis of a chunk
  double* Bm = Bj + 3 * P * kErrChunk; // [3][P][S] target basis at the samples
  double* sv = Bm + 3 * P * S;         // [4][S]: exact, PC, CP, CC at the samples
  double* red = sv + 4 * S;            // [3][2] error sums
  for (int i = threadIdx.x; i < 3 * P; i += blockDim.x) {
    const int dd = i / P, k = i % P;
    const double* bt = T.tbox + (int64_t)t * 6;
    const double* bs = T.sbox + (int64_t)s * 6;
    double c = __dmul_rn(__dadd_rn(bt[dd], bt[3 + dd]), 0.5), h = __dmul_rn(__dsub_rn(bt[3 + dd], bt[dd]), 0.5);
    tn[i] = __dadd_rn(c, __dmul_rn(h, cheb_point(k, d)));
    c = __dmul_rn(__dadd_rn(bs[dd], bs[3 + dd]), 0.5);
    h = __dmul_rn(__dsub_rn(bs[3 + dd], bs[dd]), 0.5);
    sn[i] = __dadd_rn(c, __dmul_rn(h, cheb_point(k, d)));
  }
  for (int i = threadIdx.x; i < np; i += blockDim.x) qh[i] = 0.0;
  __syncthreads();
  // Eq. (9): proxy charges of C_s at degree d.
  for (int base = 0; base < ns; base += kErrChunk) {
    const int cnt = min(kErrChunk, ns - base);
    for (int task = threadIdx.x; task < 3 * kErrChunk; task += blockDim.x) {
      const int dd = task / kErrChunk, j = task % kErrChunk;
      const double* crd = dd == 0 ? T.sx : (dd == 1 ? T.sy : T.sz);
      if (j < cnt)
        basis(crd[sb + (int64_t)(base + j) * sst], sn + dd * P, d, Bj + (dd * P) * kErrChunk + j, kErrChunk);
      else
        for (int k = 0; k < P; ++k) Bj[(dd * P + k) * kErrChunk + j] = 0.0;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < np; o += blockDim.x) {
      const int k1 = o / (P * P), k2 = (o / P) % P, k3 = o % P;
      double a = 0.0;
      for (int j = 0; j < cnt; ++j)
        a += Bj[k1 * kErrChunk + j] * Bj[(P + k2) * kErrChunk + j] * Bj[(2 * P + k3) * kErrChunk + j] *
             T.q[sb + (int64_t)(base + j) * sst];
      qh[o] += a;
    }
    __syncthreads();
  }
  // Target samples and their basis; the exact and PC sums at the samples.
  for (int task = threadIdx.x; task < 3 * m; task += blockDim.x) {
    const int dd = task / m, i = task % m;
    const int64_t pos = tb + (int64_t)i * nt / m;
    const double* crd = dd == 0 ? T.tx : (dd == 1 ? T.ty : T.tz);
    basis(crd[pos], tn + dd * P, d, Bm + (dd * P) * S + i, S);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = warp; i < m; i += nw) {
    const int64_t pos = tb + (int64_t)i * nt / m;
    const double x = T.tx[pos], y = T.ty[pos], z = T.tz[pos];
    double ex = 0.0, pc = 0.0;
    for (int j = lane; j < ns; j += 32) {
      const int64_t y0 = sb + (int64_t)j * sst;
      ex += g64<KERN>(x - T.sx[y0], y - T.sy[y0], z - T.sz[y0], kappa) * T.q[y0];
    }
    for (int o = lane; o < np; o += 32) {
      const int k1 = o / (P * P), k2 = (o / P) % P, k3 = o % P;
      pc += g64<KERN>(x - sn[k1], y - sn[P + k2], z - sn[2 * P + k3], kappa) * qh[o];
    }
    for (int off = 16; off; off >>= 1) {
      ex += __shfl_xor_sync(0xffffffffu, ex, off);
      pc += __shfl_xor_sync(0xffffffffu, pc, off);
    }
    if (lane == 0) {
      sv[i] = ex;
      sv[S + i] = pc;
    }
  }
  // CP (Eq. (12)) and CC (Eq. (15)) at C_t's proxies.
  for (int o = threadIdx.x; o < np; o += blockDim.x) {
    const int k1 = o / (P * P), k2 = (o / P) % P, k3 = o % P;
    const double x = tn[k1], y = tn[P + k2], z = tn[2 * P + k3];
    double cp = 0.0, cc = 0.0;
    for (int j = 0; j < ns; ++j) {
      const int64_t y0 = sb + (int64_t)j * sst;
      cp += g64<KERN>(x - T.sx[y0], y - T.sy[y0], z - T.sz[y0], kappa) * T.q[y0];
    }
    for (int r = 0; r < np; ++r) {
      const int r1 = r / (P * P), r2 = (r / P) % P, r3 = r % P;
      cc += g64<KERN>(x - sn[r1], y - sn[P + r2], z - sn[2 * P + r3], kappa) * qh[r];
    }
    ph[o] = cp;
    pc2[o] = cc;
  }
  __syncthreads();
  // Interpolate to the samples (Eq. (21)).
  for (int i = warp; i < m; i += nw) {
    double a = 0.0, b = 0.0;
    for (int o = lane; o < np; o += 32) {
      const int k1 = o / (P * P), k2 = (o / P) % P, k3 = o % P;
      const double L = Bm[k1 * S + i] * Bm[(P + k2) * S + i] * Bm[(2 * P + k3) * S + i];
      a += L * ph[o];
      b += L * pc2[o];
    }
    for (int off = 16; off; off >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, off);
      b += __shfl_xor_sync(0xffffffffu, b, off);
    }
    if (lane == 0) {
      sv[2 * S + i] = a;
      sv[3 * S + i] = b;
    }
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double num = 0.0, den = 0.0;
    for (int i = 0; i < m; ++i) {
      const double e = sv[i], dlt = sv[(1 + threadIdx.x) * S + i] - e;
      num += dlt * dlt;
      den += e * e;
    }
    red[threadIdx.x] = den > 0.0 ? sqrt(num / den) : (num > 0.0 ? INFINITY : 0.0);
  }
  __syncthreads();
  if (threadIdx.x < 3) err[(pi * deg.n + di) * 3 + threadIdx.x] = red[threadIdx.x];
}

static size_t err_smem_bytes(int P, int S) {
  const int np = P * P * P;
  return sizeof(double) * (size_t)(6 * P + 3 * np + 3 * P * kErrChunk + 3 * P * S + 4 * S + 8);
}

__global__ void k_pair_features(const int32_t* __restrict__ pairs, int64_t n, PairTrees T, double kappa,
                                double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double f[kFeatures];
  const bool ok = pair_features(T, pairs[2 * i], pairs[2 * i + 1], kappa, f);
  for (int d = 0; d < kFeatures; ++d) out[i * kFeatures + d] = ok ? f[d] : NAN;
}

}  // namespace bldtt

using namespace bldtt;

extern "C" {

int64_t bldtt_selector_param_count(int num_degrees) {
  if (num_degrees < 1 || num_degrees > kMaxDegrees) return -1;
  return ParamLayout(3 * num_degrees).total;
}

int bldtt_mlp_forward(const float* params, int num_out, const float* x, int64_t batch, float* y,
                      void* cuda_stream) {
  if (!params || !x || !y || batch < 1 || num_out < 1 || num_out > 3 * kMaxDegrees) {
    set_error("mlp_forward: bad arguments");
    return BLDTT_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const ParamLayout L(num_out);
  __nv_bfloat16* w = nullptr;
  float* b = nullptr;
  BL_TRY(dalloc_n(&w, (size_t)sel_weight_count(num_out), s));
  BL_TRY(dalloc_n(&b, (size_t)sel_bias_count(num_out), s));
  k_to_bf16<<<nblk(kHidden * kHidden, 256), 256, 0, s>>>(params, L, num_out, w, b);
  int64_t dummy = 0;
  BL_LAUNCHED(dummy);
  const size_t sm = net_smem_bytes(num_out);
  BL_CUDA(cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_mlp_forward<<<nblk(batch, kSelWarps) > 4096 ? 4096 : nblk(batch, kSelWarps), 32 * kSelWarps, sm, s>>>(
      x, batch, w, b, num_out, y, nullptr);
  BL_LAUNCHED(dummy);
  dfree(w, s);
  dfree(b, s);
  return BLDTT_OK;
}

int bldtt_mlp_gradients(const float* params, int num_out, const float* x, const float* target,
                        const float* mask, int64_t batch, float* grads, float* loss, void* cuda_stream) {
  if (!params || !x || !target || !mask || !grads || batch < 1 || num_out < 1 ||
      num_out > 3 * kMaxDegrees) {
    set_error("mlp_gradients: bad arguments");
    return BLDTT_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const ParamLayout L(num_out);
  __nv_bfloat16* w = nullptr;
  float *b = nullptr, *y = nullptr, *keep = nullptr, *g1 = nullptr, *g2 = nullptr, *sums = nullptr;
  BL_TRY(dalloc_n(&w, (size_t)sel_weight_count(num_out), s));
  BL_TRY(dalloc_n(&b, (size_t)sel_bias_count(num_out), s));
  BL_TRY(dalloc_n(&y, (size_t)batch * num_out, s));
  BL_TRY(dalloc_n(&keep, (size_t)batch * kKeep, s));
  BL_TRY(dalloc_n(&g1, (size_t)batch * kHidden, s));
  BL_TRY(dalloc_n(&g2, (size_t)batch * kHidden, s));
  BL_TRY(dalloc_n(&sums, 2, s));
  int64_t dummy = 0;
  k_to_bf16<<<nblk(kHidden * kHidden, 256), 256, 0, s>>>(params, L, num_out, w, b);
  BL_LAUNCHED(dummy);
  const size_t sm = net_smem_bytes(num_out);
  BL_CUDA(cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_mlp_forward<<<nblk(batch, kSelWarps) > 4096 ? 4096 : nblk(batch, kSelWarps), 32 * kSelWarps, sm, s>>>(
      x, batch, w, b, num_out, y, keep);
  BL_LAUNCHED(dummy);
  const int64_t ny = batch * num_out;
  k_loss_sums<<<1, 256, 0, s>>>(y, target, mask, ny, sums);
  BL_LAUNCHED(dummy);
  // g1 <- dL/dy (batch x num_out, fits: num_out <= 24 < 64)
  k_out_grad<<<nblk(ny, 256), 256, 0, s>>>(y, target, mask, ny, sums, g1);
  BL_LAUNCHED(dummy);
  // layer 4 (output): a3 at keep offset 8 + 5*64
  const int aoff[4] = {0, 8 + 1 * kHidden, 8 + 3 * kHidden, 8 + 5 * kHidden};   // a0 = x, a1, a2, a3
  const int zoff[3] = {8 + 0 * kHidden, 8 + 2 * kHidden, 8 + 4 * kHidden};      // z1, z2, z3
  const int K[4] = {kFeatures, kHidden, kHidden, kHidden};
  const int J[4] = {kHidden, kHidden, kHidden, num_out};
  const __nv_bfloat16* Wl[4];
  {
    int64_t o = 0;
    for (int l = 0; l < 4; ++l) {
      Wl[l] = w + o;
      o += (int64_t)K[l] * J[l];
    }
  }
  float* g = g1;
  float* gn = g2;
  for (int l = 3; l >= 0; --l) {
    const int64_t nt = (int64_t)J[l] * K[l] + J[l];
    k_weight_grad<<<nblk(nt, 128), 128, 0, s>>>(g, J[l], J[l], keep, kKeep, aoff[l], K[l], batch,
                                                 grads + L.w[l], grads + L.b[l]);
    BL_LAUNCHED(dummy);
    if (l > 0) {
      k_back<<<nblk(batch * K[l], 256), 256, 0, s>>>(g, J[l], Wl[l], K[l], keep, zoff[l - 1], batch, gn);
      BL_LAUNCHED(dummy);
      float* tmp = g;
      g = gn;
      gn = tmp;
    }
  }
  if (loss) BL_CUDA(cudaMemcpyAsync(loss, sums + 1, sizeof(float), cudaMemcpyDeviceToDevice, s));
  dfree(w, s); dfree(b, s); dfree(y, s); dfree(keep, s); dfree(g1, s); dfree(g2, s); dfree(sums, s);
  return BLDTT_OK;
}

int bldtt_mlp_adam(float* params, float* m, float* v, const float* grads, int64_t count, int step,
                   float lr, void* cuda_stream) {
  if (!params || !m || !v || !grads || count < 1 || step < 1) {
    set_error("mlp_adam: bad arguments");
    return BLDTT_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const float c1 = 1.f - powf(0.9f, (float)step), c2 = 1.f - powf(0.999f, (float)step);
  k_adam<<<nblk(count, 256), 256, 0, s>>>(params, m, v, grads, count, lr, c1, c2);
  int64_t dummy = 0;
  BL_LAUNCHED(dummy);
  return BLDTT_OK;
}

int bldtt_pair_features(bldtt_plan* p, int64_t npairs, const int32_t* pairs, double* features,
                        void* cuda_stream) {
  if (!p || !pairs || !features || npairs < 1) {
    set_error("pair_features: bad arguments");
    return BLDTT_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  k_pair_features<<<nblk(npairs, 128), 128, 0, s>>>(pairs, npairs, pair_trees(p), p->kappa, features);
  int64_t dummy = 0;
  BL_LAUNCHED(dummy);
  return BLDTT_OK;
}

int bldtt_pair_errors(bldtt_plan* p, int64_t npairs, const int32_t* pairs, int samples, int num_degrees,
                      const int* degrees, double* err, void* cuda_stream) {
  if (!p || !pairs || !err || !degrees || npairs < 1 || samples < 1 || samples > 256 ||
      num_degrees < 1 || num_degrees > kMaxDegrees) {
    set_error("pair_errors: bad arguments");
    return BLDTT_EINVAL;
  }
  DegreeSet deg;
  deg.n = num_degrees;
  int pmax = 1;
  for (int i = 0; i < num_degrees; ++i) {
    if (degrees[i] < 1 || degrees[i] > kMaxDegree) {
      set_error("pair_errors: degree %d outside [1, %d]", degrees[i], kMaxDegree);
      return BLDTT_EINVAL;
    }
    deg.d[i] = degrees[i];
    deg.np[i] = (degrees[i] + 1) * (degrees[i] + 1) * (degrees[i] + 1);
    if (degrees[i] + 1 > pmax) pmax = degrees[i] + 1;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  ErrTrees T{p->tt.begin, p->tt.end, p->st.begin, p->st.end, p->tt.box, p->st.box,
             p->tt.x, p->tt.y, p->tt.z, p->st.x, p->st.y, p->st.z, p->q_tree};
  const size_t sm = err_smem_bytes(pmax, samples);
  if (sm > 200 * 1024) {
    set_error("pair_errors: degree and sample count need %zu bytes of shared memory", sm);
    return BLDTT_EINVAL;
  }
  const int64_t blocks = npairs * num_degrees;
  int64_t dummy = 0;
#define BL_ERR_LAUNCH(K)                                                                              \
  do {                                                                                               \
    BL_CUDA(cudaFuncSetAttribute(k_pair_errors<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)); \
    k_pair_errors<K><<<(unsigned)blocks, kErrThreads, sm, s>>>(pairs, npairs, T, deg, samples, p->kappa, err); \
    BL_LAUNCHED(dummy);                                                                              \
  } while (0)
  switch (p->kernel) {
    case BLDTT_COULOMB: BL_ERR_LAUNCH(BLDTT_COULOMB); break;
    case BLDTT_YUKAWA: BL_ERR_LAUNCH(BLDTT_YUKAWA); break;
    case BLDTT_OSCILLATORY: BL_ERR_LAUNCH(BLDTT_OSCILLATORY); break;
    case BLDTT_REG_COULOMB: BL_ERR_LAUNCH(BLDTT_REG_COULOMB); break;
    default: BL_ERR_LAUNCH(BLDTT_TEST_POLY); break;
  }
#undef BL_ERR_LAUNCH
  return BLDTT_OK;
}

}  // extern "C"
