// C ABI of the library (declared, with argument conventions, in include/bldtt.h).
#include <cmath>
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "internal.cuh"

namespace bldtt {
const char* last_error();
int configure_pass_kernels();
int configure_tc_kernels();
}  // namespace bldtt

using namespace bldtt;

namespace {

bool finite(double v) { return std::isfinite(v); }

int validate(int64_t M, int64_t N, int kernel, double kappa, int n, double theta, int N0, int M0,
             int precision) {
  if (M < 1 || N < 1 || M >= INT32_MAX || N >= INT32_MAX) {
    set_error("M=%lld and N=%lld must lie in [1, 2^31-1)", (long long)M, (long long)N);
    return BLDTT_EINVAL;
  }
  if (kernel != BLDTT_COULOMB && kernel != BLDTT_YUKAWA && kernel != BLDTT_OSCILLATORY &&
      kernel != BLDTT_REG_COULOMB && kernel != BLDTT_TEST_POLY) {
    set_error("unknown kernel %d", kernel);
    return BLDTT_EINVAL;
  }
  if ((kernel == BLDTT_YUKAWA || kernel == BLDTT_OSCILLATORY || kernel == BLDTT_REG_COULOMB) &&
      !(finite(kappa) && kappa >= 0.0)) {
    set_error("kernel parameter kappa must be finite and >= 0 (got %g)", kappa);
    return BLDTT_EINVAL;
  }
  if (n < 1 || n > kMaxDegree) {
    set_error("interpolation degree n=%d outside [1, %d]", n, kMaxDegree);
    return BLDTT_EINVAL;
  }
  if (!(finite(theta) && theta >= 0.0)) {
    set_error("MAC parameter theta must be finite and >= 0 (got %g)", theta);
    return BLDTT_EINVAL;
  }
  if (N0 < 1 || M0 < 1) {
    set_error("leaf sizes N0=%d, M0=%d must be >= 1", N0, M0);
    return BLDTT_EINVAL;
  }
  if (precision != BLDTT_FP64 && precision != BLDTT_FP32_BULK) {
    set_error("unknown precision %d", precision);
    return BLDTT_EINVAL;
  }
  return BLDTT_OK;
}

float elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
    cudaGetLastError();
    return -1.f;
  }
  return ms;
}

constexpr int kMaxDevices = 64;
std::mutex g_res_mu;
cudaMemPool_t g_pools[kMaxDevices] = {};
size_t g_pool_keep[kMaxDevices] = {};   // an eighth of the device's memory
std::vector<void*> g_pinned_free;

static size_t pool_keep(cudaMemPool_t pool) {
  std::lock_guard<std::mutex> lock(g_res_mu);
  for (int d = 0; d < kMaxDevices; ++d)
    if (g_pools[d] == pool) return g_pool_keep[d];
  return 0;
}


static void release_pool(bldtt_plan* p) {
  if (p->mempool) cudaMemPoolTrimTo(p->mempool, pool_keep(p->mempool));
  if (p->h_pinned) {
    std::lock_guard<std::mutex> lock(g_res_mu);
    g_pinned_free.push_back(p->h_pinned);
  }
  p->mempool = nullptr;
  p->h_pinned = nullptr;
}

void release(bldtt_plan* p) {
  if (!p) return;
  cudaStream_t s = p->stream;
  free_tree(p->tt, s);
  if (!p->shared_tree) free_tree(p->st, s);
  dfree_ptr(p->q_tree, s);
  dfree_ptr(p->list_ptr, s);
  dfree_ptr(p->list_src, s);
  dfree_ptr(p->list_tgt, s);
  dfree_ptr(p->pad_prefix, s);
  dfree(p->pool, s);
  p->pool = nullptr;
  dfree_ptr(p->items, s);
  dfree_ptr(p->item_counter, s);
  dfree_ptr(p->chunk_frame, s);
  dfree_ptr(p->pool_res, s);
  dfree_ptr(p->item_box, s);
  dfree_ptr(p->eval_part, s);
  dfree_ptr(p->eval_prox, s);
  dfree_ptr(p->sh_items, s);
  dfree_ptr(p->sh_item_box, s);
  dfree_ptr(p->qhat, s);
  dfree_ptr(p->phit, s);
  dfree_ptr(p->phi_near, s);
  dfree_ptr(p->dev_err, s);
  dfree_ptr(p->prob_kernel, s);
  dfree_ptr(p->prob_kappa, s);
  dfree_ptr(p->prob_prm, s);
  for (int i = 0; i + 1 < p->deg.n; ++i) {   // the highest degree aliases the tree/plan arrays
    dfree_ptr(p->nodes_t[i], s);
    dfree_ptr(p->nodes_s[i], s);
    dfree_ptr(p->qhat_d[i], s);
    dfree_ptr(p->phit_d[i], s);
    dfree_ptr(p->xfer[i], s);
  }
  dfree(p->sel_w, s);
  p->sel_w = nullptr;
  dfree_ptr(p->sel_b, s);
  if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
  cudaStreamSynchronize(s);
  release_pool(p);
  for (auto& e : p->ev)
    if (e) cudaEventDestroy(e);
  cudaGetLastError();
  delete p;
}

// FP32 form of each kernel's parameter, as the interaction kernel uses it.
float fp32_parameter(int kernel, double kappa) {
  if (kernel == BLDTT_YUKAWA) return (float)(-kappa * 1.4426950408889634);   // -kappa log2(e)
  if (kernel == BLDTT_REG_COULOMB) return (float)(kappa * kappa);
  return (float)kappa;
}

// Target and source trees of unequal sets are independent.  With the
// cooperative build each tree is one launch and the two run one after the
// other on the call's stream.  Level by level, the source tree is built on a
// second stream by a helper thread while this thread builds the target tree
// (each such build synchronises with the host once per level, so one thread
// would serialise the two); the stream of the call then waits for both.
static int build_two_trees(bldtt_plan* p, const double* targets, const double* sources,
                           const double* charges, cudaStream_t s) {
  if (tree_build_cooperative()) {
    BL_TRY(build_tree_checked(p->tt, targets, (int32_t)p->M, p->t_off, p->M0, p->n, nullptr, 0, s,
                              p->setup_counter));
    BL_TRY(morton_order_leaves(p->tt, p->M0, s, p->setup_counter));
    BL_TRY(build_tree_checked(p->st, sources, (int32_t)p->N, p->s_off, p->N0, p->n, charges, p->N, s,
                              p->setup_counter));
    return morton_order_leaves(p->st, p->N0, s, p->setup_counter);
  }
  cudaStream_t s2 = nullptr;
  cudaEvent_t go = nullptr, done = nullptr;
  BL_CUDA(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
  BL_CUDA(cudaEventCreateWithFlags(&go, cudaEventDisableTiming));
  BL_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
  BL_CUDA(cudaEventRecord(go, s));   // the inputs, as of this call
  BL_CUDA(cudaStreamWaitEvent(s2, go, 0));
  Counters c2;
  int rc2 = BLDTT_OK;
  std::string err2;
  std::thread worker([&] {
    PlanScope scope(p->mempool, static_cast<char*>(p->h_pinned) + kPinnedSlot);
    if (cudaSetDevice(p->device) != cudaSuccess) {
      rc2 = BLDTT_ECUDA;
      err2 = "cudaSetDevice failed in the source-tree thread";
      return;
    }
    rc2 = build_tree_checked(p->st, sources, (int32_t)p->N, p->s_off, p->N0, p->n, charges, p->N, s2, c2);
    if (rc2 == BLDTT_OK) rc2 = morton_order_leaves(p->st, p->N0, s2, c2);
    if (rc2 != BLDTT_OK) err2 = last_error();
  });
  int rc1 = build_tree_checked(p->tt, targets, (int32_t)p->M, p->t_off, p->M0, p->n, nullptr, 0, s,
                               p->setup_counter);
  if (rc1 == BLDTT_OK) rc1 = morton_order_leaves(p->tt, p->M0, s, p->setup_counter);
  worker.join();
  p->setup_counter.launches += c2.launches;
  const cudaError_t e1 = cudaEventRecord(done, s2);
  const cudaError_t e2 = cudaStreamWaitEvent(s, done, 0);
  cudaEventDestroy(go);
  cudaEventDestroy(done);
  cudaStreamDestroy(s2);   // released once its work has completed
  if (rc1 != BLDTT_OK) return rc1;
  if (rc2 != BLDTT_OK) {
    set_error("%s", err2.c_str());
    return rc2;
  }
  BL_CUDA(e1);
  BL_CUDA(e2);
  return BLDTT_OK;
}

int setup_impl(bldtt_plan* p, const double* targets, const double* sources, const double* charges) {
  cudaStream_t s = p->stream;
  BL_CUDA(cudaGetDevice(&p->device));
  BL_TRY(configure_pass_kernels());
  BL_TRY(configure_tc_kernels());
  for (auto& e : p->ev) BL_CUDA(cudaEventCreate(&e));
  {
    const int P = p->nprob;
    std::vector<float>& prm = p->prob_prm_h;   // the plan keeps the staged host vectors
    prm.resize(P);
    for (int i = 0; i < P; ++i) prm[i] = fp32_parameter(p->prob_kernel_h[i], p->prob_kappa_h[i]);
    BL_TRY(dalloc_n(&p->prob_kernel, P, s));
    BL_TRY(dalloc_n(&p->prob_kappa, P, s));
    BL_TRY(dalloc_n(&p->prob_prm, P, s));
    BL_CUDA(cudaMemcpyAsync(p->prob_kernel, p->prob_kernel_h.data(), P * sizeof(int),
                            cudaMemcpyHostToDevice, s));
    BL_CUDA(cudaMemcpyAsync(p->prob_kappa, p->prob_kappa_h.data(), P * sizeof(double),
                            cudaMemcpyHostToDevice, s));
    BL_CUDA(cudaMemcpyAsync(p->prob_prm, prm.data(), P * sizeof(float), cudaMemcpyHostToDevice, s));
  }
  BL_TRY(dalloc_n(&p->dev_err, 1, s));
  BL_CUDA(cudaMemsetAsync(p->dev_err, 0, sizeof(int), s));
  BL_CUDA(cudaEventRecord(p->ev[0], s));
  // Non-finite input is rejected by the tree build before any cluster splits
  // (a box of infinite extent would be split without end).
  // Targets that are the sources, with the same leaf size and problem
  // offsets, give two identical trees (the build is deterministic): build one
  // and let the source tree alias it.
  p->shared_tree = targets == sources && p->M == p->N && p->M0 == p->N0 && p->t_off == p->s_off;
  if (p->shared_tree) {
    BL_TRY(build_tree_checked(p->tt, targets, (int32_t)p->M, p->t_off, p->M0, p->n, charges, p->N, s,
                              p->setup_counter));
    BL_TRY(morton_order_leaves(p->tt, p->M0, s, p->setup_counter));
    p->st = p->tt;
  } else {
    BL_TRY(build_two_trees(p, targets, sources, charges, s));
  }
  BL_TRY(dalloc_n(&p->q_tree, p->N, s));
  BL_TRY(permute_charges(p, charges, s));
  BL_CUDA(cudaEventRecord(p->ev[1], s));
  // Default engine of the downward leaf contraction: the tensor cores when the
  // target leaves hold 512 particles or more on average (four 128-particle MMA
  // tiles per leaf), else SIMT.  Measured on a GB300: 0.15 against 0.18 ms at
  // 1E6 (leaves of ~1950), 1.04 against 1.11 ms on the unequal-set workload,
  // but 2.76 against 1.80 ms on the batched workload (leaves of ~250).
  p->down_engine = (p->tt.nleaves > 0 && p->M >= 512 * (int64_t)p->tt.nleaves) ? BLDTT_PASS_TENSOR
                                                                              : BLDTT_PASS_SIMT;
  BL_TRY(setup_degrees(p, s));
  BL_TRY(build_lists(p, s));
  BL_TRY(build_work_items(p, s));
  const size_t esz = p->precision == BLDTT_FP32_BULK ? sizeof(float4) : sizeof(double4);
  BL_TRY(dalloc(&p->pool, (size_t)p->pool_len * esz, s));
  BL_TRY(dalloc_n(&p->qhat, (size_t)p->st.nclusters * p->np, s));
  BL_TRY(dalloc_n(&p->phit, (size_t)p->tt.nclusters * p->np, s));
  p->qhat_d[p->deg.n - 1] = p->qhat;
  p->phit_d[p->deg.n - 1] = p->phit;
  BL_TRY(dalloc_n(&p->phi_near, (size_t)p->M, s));
  BL_TRY(dalloc_n(&p->item_counter, p->segments.size() > 0 ? p->segments.size() : 1, s));
  BL_TRY(build_chunk_frames(p, s));
  // Default layout: warps of empty rows skip their work when that saves at
  // least 2 % of the evaluations (many items smaller than a tile).
  const bool skip = p->skip_saved_evaluations > 0.02 * p->executed_noskip;
  p->executed_evaluations = skip ? p->executed_skip : p->executed_noskip;
  p->interact_layout = skip ? kLayoutSkip : 0;
  if (const char* lay = std::getenv("BLDTT_INTERACT_LAYOUT")) {
    int l = std::atoi(lay);
    p->interact_layout = (l >= 0 && l < kMaxLayouts) ? l : 0;
  }
  for (auto& seg : p->segments) {      // the requested layout where it is instantiated
    int cand[kMaxLayouts];
    const int nc = layouts_available(seg.kernel, cand);
    seg.layout = 0;
    for (int i = 0; i < nc; ++i)
      if (cand[i] == p->interact_layout) seg.layout = p->interact_layout;
  }
  BL_TRY(interaction_grids(p));
  BL_CUDA(cudaEventRecord(p->ev[2], s));
  BL_CUDA(cudaStreamSynchronize(s));
  // hand back what the set-up's temporaries held beyond the pool's keep; the plan's arrays stay
  BL_CUDA(cudaMemPoolTrimTo(p->mempool, pool_keep(p->mempool)));
  p->ms_tree = elapsed(p->ev[0], p->ev[1]);
  p->ms_lists = elapsed(p->ev[1], p->ev[2]);
  return BLDTT_OK;
}

int sync_plan(bldtt_plan* p) {
  BL_CUDA(cudaStreamSynchronize(p->stream));
  return BLDTT_OK;
}

int device_error(bldtt_plan* p) {
  int h = 0;
  BL_CUDA(cudaMemcpy(&h, p->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h == kDevErrTimeout) {
    set_error("a bounded wait in the interaction kernel timed out");
    return BLDTT_ETIMEOUT;
  }
  if (h != kDevErrNone) {
    set_error("device error flag %d", h);
    return BLDTT_EINTERNAL;
  }
  return BLDTT_OK;
}

}  // namespace

extern "C" {

const char* bldtt_status_string(int status) {
  switch (status) {
    case BLDTT_OK: return "BLDTT_OK";
    case BLDTT_EINVAL: return "BLDTT_EINVAL";
    case BLDTT_ENOMEM: return "BLDTT_ENOMEM";
    case BLDTT_ECUDA: return "BLDTT_ECUDA";
    case BLDTT_ETIMEOUT: return "BLDTT_ETIMEOUT";
    case BLDTT_EINTERNAL: return "BLDTT_EINTERNAL";
    default: return "BLDTT_UNKNOWN_STATUS";
  }
}

const char* bldtt_last_error(void) { return bldtt::last_error(); }

// Selector weights: float master weights (W1 b1 W2 b2 W3 b3 W4 b4, rows =
// outputs) -> bf16 weights (round to nearest even) and float biases.
static uint16_t host_bf16(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u = (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
  return (uint16_t)u;
}
static int upload_selector(bldtt_plan* p, const float* weights) {
  const int nout = p->sel_nout;
  const int in[4] = {kFeatures, kHidden, kHidden, kHidden};
  const int out[4] = {kHidden, kHidden, kHidden, nout};
  std::vector<uint16_t> w;
  std::vector<float> b;
  size_t o = 0;
  for (int l = 0; l < 4; ++l) {
    for (int i = 0; i < in[l] * out[l]; ++i) {
      if (!std::isfinite(weights[o + i])) {
        set_error("selector weight %zu is not finite", o + i);
        return BLDTT_EINVAL;
      }
      w.push_back(host_bf16(weights[o + i]));
    }
    o += (size_t)in[l] * out[l];
    for (int i = 0; i < out[l]; ++i) b.push_back(weights[o + i]);
    o += out[l];
  }
  cudaStream_t s = p->stream;
  uint16_t* dw = nullptr;
  BL_TRY(dalloc_n(&dw, w.size(), s));
  p->sel_w = dw;
  BL_TRY(dalloc_n(&p->sel_b, b.size(), s));
  BL_CUDA(cudaMemcpyAsync(p->sel_w, w.data(), w.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, s));
  BL_CUDA(cudaMemcpyAsync(p->sel_b, b.data(), b.size() * sizeof(float), cudaMemcpyHostToDevice, s));
  BL_CUDA(cudaStreamSynchronize(s));
  return BLDTT_OK;
}

// Device memory comes from one memory pool per device, shared by every plan
// of the process: memory freed by a plan stays reserved (release threshold at
// the maximum) for the next set-up, whose allocations then need no new
// mapping (at 1E8 particles, mapping the set-up's memory afresh took ~10 ms);
// set-ups and destroys trim the pool back to an eighth of the device's memory
// (or what live plans hold, if more).  The set-up's small device-to-host reads
// go through two pinned host slots per plan, recycled from a process-wide free
// list.
// The current device's shared pool (created on first use).
static int shared_pool(cudaMemPool_t* out) {
  int dev = 0;
  BL_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal %d beyond the supported %d", dev, kMaxDevices);
    return BLDTT_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_res_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    BL_CUDA(cudaMemPoolCreate(&pool, &props));
    uint64_t keep = UINT64_MAX;
    BL_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    size_t free_b = 0, total_b = 0;
    BL_CUDA(cudaMemGetInfo(&free_b, &total_b));
    g_pool_keep[dev] = total_b / 8;
    g_pools[dev] = pool;
  }
  *out = g_pools[dev];
  return BLDTT_OK;
}

static int create_pool(bldtt_plan* p) {
  BL_TRY(shared_pool(&p->mempool));
  std::lock_guard<std::mutex> lock(g_res_mu);
  if (!g_pinned_free.empty()) {
    p->h_pinned = g_pinned_free.back();
    g_pinned_free.pop_back();
  } else {
    BL_CUDA(cudaMallocHost(&p->h_pinned, 2 * kPinnedSlot));
  }
  return BLDTT_OK;
}

// Common set-up of a batch of nprob problems (nprob = 1 for bldtt_setup).
// t_off / s_off: host offsets (nprob + 1) of each problem's targets / sources.
static int setup_common(bldtt_plan** plan, const double* targets, const int64_t* t_off,
                        const double* sources, const int64_t* s_off, const double* charges,
                        int nprob, const int* kernels, const double* kappas, int n, double theta,
                        int N0, int M0, int precision, int variant, const bldtt_selector_t* sel,
                        void* cuda_stream) {
  if (!plan) {
    set_error("plan out-pointer is NULL");
    return BLDTT_EINVAL;
  }
  *plan = nullptr;
  if (!targets || !sources || !charges) {
    set_error("targets, sources and charges must be non-NULL device pointers");
    return BLDTT_EINVAL;
  }
  if (nprob < 1 || !t_off || !s_off || !kernels || !kappas) {
    set_error("a batch needs at least one problem, offsets, kernels and kappas");
    return BLDTT_EINVAL;
  }
  if (t_off[0] != 0 || s_off[0] != 0) {
    set_error("problem offsets must start at 0");
    return BLDTT_EINVAL;
  }
  for (int i = 0; i < nprob; ++i) {
    if (t_off[i + 1] <= t_off[i] || s_off[i + 1] <= s_off[i]) {
      set_error("problem %d has no targets or no sources (offsets must increase)", i);
      return BLDTT_EINVAL;
    }
    BL_TRY(validate(t_off[i + 1] - t_off[i], s_off[i + 1] - s_off[i], kernels[i], kappas[i], n,
                    theta, N0, M0, precision));
  }
  const int64_t M = t_off[nprob], N = s_off[nprob];
  BL_TRY(validate(M, N, kernels[0], kappas[0], n, theta, N0, M0, precision));
  if (sel) {
    if (sel->num_degrees < 1 || sel->num_degrees > kMaxDegrees) {
      set_error("selector: %d degrees (1..%d allowed)", sel->num_degrees, kMaxDegrees);
      return BLDTT_EINVAL;
    }
    for (int i = 0; i < sel->num_degrees; ++i)
      if (sel->degrees[i] < 1 || sel->degrees[i] > kMaxDegree ||
          (i > 0 && sel->degrees[i] <= sel->degrees[i - 1])) {
        set_error("selector: degrees must increase strictly within [1, %d]", kMaxDegree);
        return BLDTT_EINVAL;
      }
    if (sel->degrees[sel->num_degrees - 1] != n) {
      set_error("selector: the highest degree (%d) must equal params n (%d)",
                sel->degrees[sel->num_degrees - 1], n);
      return BLDTT_EINVAL;
    }
    for (int d = 0; d < 6; ++d)
      if (!(sel->feature_lo[d] <= sel->feature_hi[d])) {
        set_error("selector: feature box %d is empty or not finite", d);
        return BLDTT_EINVAL;
      }
    if (!std::isfinite(sel->log10_budget)) {
      set_error("selector: log10_budget is not finite");
      return BLDTT_EINVAL;
    }
  }
  if (variant != BLDTT_VARIANT_FULL && variant != BLDTT_VARIANT_CC_PP_ONLY) {
    set_error("unknown traversal variant %d", variant);
    return BLDTT_EINVAL;
  }
  bldtt_plan* p = new (std::nothrow) bldtt_plan;
  if (!p) {
    set_error("host allocation of the plan failed");
    return BLDTT_ENOMEM;
  }
  p->M = M;
  p->N = N;
  p->nprob = nprob;
  p->t_off.assign(t_off, t_off + nprob + 1);
  p->s_off.assign(s_off, s_off + nprob + 1);
  for (int i = 0; i < nprob; ++i) {
    const int k = kernels[i];
    const bool has_kappa = k == BLDTT_YUKAWA || k == BLDTT_OSCILLATORY || k == BLDTT_REG_COULOMB;
    p->prob_kernel_h.push_back(k);
    p->prob_kappa_h.push_back(has_kappa ? kappas[i] : 0.0);
  }
  p->kernels_present = p->prob_kernel_h;
  std::sort(p->kernels_present.begin(), p->kernels_present.end());
  p->kernels_present.erase(std::unique(p->kernels_present.begin(), p->kernels_present.end()),
                           p->kernels_present.end());
  {
    const auto& kp = p->kernels_present;
    const bool both = std::count(kp.begin(), kp.end(), (int)BLDTT_COULOMB) &&
                      std::count(kp.begin(), kp.end(), (int)BLDTT_YUKAWA);
    p->segment_kernels.clear();
    if (both) p->segment_kernels.push_back(kKernCoulombYukawa);
    for (int k : kp)
      if (!both || (k != BLDTT_COULOMB && k != BLDTT_YUKAWA)) p->segment_kernels.push_back(k);
  }
  p->kernel = kernels[0];
  p->kappa = p->prob_kappa_h[0];
  p->variant = variant;
  p->n = n;
  p->P = n + 1;
  p->np = p->P * p->P * p->P;
  p->theta = theta;
  p->N0 = N0;
  p->M0 = M0;
  p->precision = precision;
  p->stream = static_cast<cudaStream_t>(cuda_stream);
  p->deg.n = sel ? sel->num_degrees : 1;
  for (int i = 0; i < p->deg.n; ++i) {
    const int d = sel ? sel->degrees[i] : n;
    p->deg.d[i] = d;
    p->deg.np[i] = (d + 1) * (d + 1) * (d + 1);
    p->deg.np_pad[i] = (p->deg.np[i] + kChunk - 1) / kChunk * kChunk;
  }
  p->nclass = 1 + 3 * p->deg.n;
  int st = create_pool(p);
  PlanScope scope(p->mempool, p->h_pinned);
  if (st == BLDTT_OK && sel) {
    p->learned = true;
    p->selector_net = sel->weights != nullptr;
    p->sel_nout = 3 * p->deg.n;
    for (int d = 0; d < 6; ++d) {
      p->sel_lo[d] = sel->feature_lo[d];
      p->sel_hi[d] = sel->feature_hi[d];
    }
    p->sel_log_eps = sel->log10_budget;
    if (p->selector_net) st = upload_selector(p, sel->weights);
  }
  if (st == BLDTT_OK) st = setup_impl(p, targets, sources, charges);
  if (st != BLDTT_OK) {
    release(p);
    return st;
  }
  *plan = p;
  return BLDTT_OK;
}

int bldtt_setup(bldtt_plan** plan, const double* targets, int64_t M, const double* sources,
                int64_t N, const double* charges, int kernel, double kappa, int n, double theta,
                int N0, int M0, int precision, void* cuda_stream) {
  const int64_t t_off[2] = {0, M}, s_off[2] = {0, N};
  if (M < 1 || N < 1) {
    if (plan) *plan = nullptr;
    BL_TRY(validate(M, N, kernel, kappa, n, theta, N0, M0, precision));
  }
  return setup_common(plan, targets, t_off, sources, s_off, charges, 1, &kernel, &kappa, n, theta,
                      N0, M0, precision, BLDTT_VARIANT_FULL, nullptr, cuda_stream);
}

int bldtt_setup_ex(bldtt_plan** plan, const double* targets, int64_t M, const double* sources,
                   int64_t N, const double* charges, const bldtt_params_t* prm,
                   void* cuda_stream) {
  if (!prm) {
    if (plan) *plan = nullptr;
    set_error("params pointer is NULL");
    return BLDTT_EINVAL;
  }
  const int64_t t_off[2] = {0, M}, s_off[2] = {0, N};
  if (M < 1 || N < 1) {
    if (plan) *plan = nullptr;
    BL_TRY(validate(M, N, prm->kernel, prm->kappa, prm->n, prm->theta, prm->N0, prm->M0,
                    prm->precision));
  }
  return setup_common(plan, targets, t_off, sources, s_off, charges, 1, &prm->kernel, &prm->kappa,
                      prm->n, prm->theta, prm->N0, prm->M0, prm->precision, prm->variant, nullptr,
                      cuda_stream);
}

int bldtt_setup_batch(bldtt_plan** plan, int nprob, const double* targets, const int64_t* target_offsets,
                      const double* sources, const int64_t* source_offsets, const double* charges,
                      const int* kernels, const double* kappas, const bldtt_params_t* prm,
                      void* cuda_stream) {
  if (!prm) {
    if (plan) *plan = nullptr;
    set_error("params pointer is NULL");
    return BLDTT_EINVAL;
  }
  return setup_common(plan, targets, target_offsets, sources, source_offsets, charges, nprob,
                      kernels, kappas, prm->n, prm->theta, prm->N0, prm->M0, prm->precision,
                      prm->variant, nullptr, cuda_stream);
}

int bldtt_setup_learned(bldtt_plan** plan, const double* targets, int64_t M, const double* sources,
                        int64_t N, const double* charges, const bldtt_params_t* prm,
                        const bldtt_selector_t* sel, void* cuda_stream) {
  if (!prm || !sel) {
    if (plan) *plan = nullptr;
    set_error("params and selector pointers must be non-NULL");
    return BLDTT_EINVAL;
  }
  const int64_t t_off[2] = {0, M}, s_off[2] = {0, N};
  if (M < 1 || N < 1) {
    if (plan) *plan = nullptr;
    BL_TRY(validate(M, N, prm->kernel, prm->kappa, prm->n, prm->theta, prm->N0, prm->M0,
                    prm->precision));
  }
  return setup_common(plan, targets, t_off, sources, s_off, charges, 1, &prm->kernel, &prm->kappa,
                      prm->n, prm->theta, prm->N0, prm->M0, prm->precision, prm->variant, sel,
                      cuda_stream);
}

int bldtt_list_classes(bldtt_plan* p, int* num_classes, int* degrees, int* num_degrees) {
  if (!p) {
    set_error("plan is NULL");
    return BLDTT_EINVAL;
  }
  if (num_classes) *num_classes = p->nclass;
  if (num_degrees) *num_degrees = p->deg.n;
  if (degrees)
    for (int i = 0; i < p->deg.n; ++i) degrees[i] = p->deg.d[i];
  return BLDTT_OK;
}

int bldtt_set_charges(bldtt_plan* p, const double* charges, void* cuda_stream) {
  if (!p || !charges) {
    set_error("plan and charges must be non-NULL");
    return BLDTT_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  p->stream = s;
  int* bad = nullptr;
  BL_TRY(dalloc_n(&bad, 1, s));
  BL_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
  BL_TRY(permute_charges(p, charges, s));
  BL_TRY(check_finite(p->q_tree, p->N, bad, s, p->setup_counter));
  int h_bad = 0;
  BL_CUDA(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  BL_CUDA(cudaStreamSynchronize(s));
  dfree(bad, s);
  if (h_bad) {
    set_error("a charge is not finite");
    return BLDTT_EINVAL;
  }
  return BLDTT_OK;
}

int bldtt_compute(bldtt_plan* p, double* phi, void* cuda_stream) {
  if (!p || !phi) {
    set_error("plan and phi must be non-NULL");
    return BLDTT_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  p->stream = s;
  p->compute_counter.launches = 0;
  p->computed_evals = p->interactions[0] + p->interactions[1] + p->interactions[2] + p->interactions[3];
  return compute_body(p, phi, s);
}

int bldtt_compute_graph(bldtt_plan* p, double* phi, void* cuda_stream) {
  if (!p || !phi) {
    set_error("plan and phi must be non-NULL");
    return BLDTT_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread) {
    set_error("bldtt_compute_graph needs a created (non-default) stream to capture on");
    return BLDTT_EINVAL;
  }
  p->stream = s;
  p->computed_evals = p->interactions[0] + p->interactions[1] + p->interactions[2] + p->interactions[3];
  if (!p->graph_exec || p->graph_phi != phi) {
    if (p->graph_exec) {
      cudaGraphExecDestroy(p->graph_exec);
      p->graph_exec = nullptr;
    }
    BL_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    p->compute_counter.launches = 0;
    int st = compute_body(p, phi, s);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (st != BLDTT_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) {
      set_error("stream capture of the compute phase failed: %s", cudaGetErrorString(e));
      return BLDTT_ECUDA;
    }
    e = cudaGraphInstantiate(&p->graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      p->graph_exec = nullptr;
      set_error("graph instantiation failed: %s", cudaGetErrorString(e));
      return BLDTT_ECUDA;
    }
    p->graph_phi = phi;
  }
  BL_CUDA(cudaGraphLaunch(p->graph_exec, s));
  return BLDTT_OK;
}

int bldtt_autotune(bldtt_plan* p, double* phi, void* cuda_stream, int* chosen) {
  if (!p || !phi) {
    set_error("plan and phi must be non-NULL");
    return BLDTT_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  p->stream = s;
  // One full compute stages the pool; then every segment's launch is timed
  // alone for each layout (a launch only overwrites its own items' outputs).
  p->compute_counter.launches = 0;
  p->computed_evals = p->interactions[0] + p->interactions[1] + p->interactions[2] + p->interactions[3];
  BL_TRY(compute_body(p, phi, s));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  BL_CUDA(cudaEventCreate(&e0));
  BL_CUDA(cudaEventCreate(&e1));
  int rc = BLDTT_OK;
  p->tune_table.clear();
  p->tuned = false;
  for (size_t g = 0; g < p->segments.size() && rc == BLDTT_OK; ++g) {
    auto& seg = p->segments[g];
    int cand[kMaxLayouts];
    const int ncand = layouts_available(seg.kernel, cand);
    float best = -1.f;
    int best_layout = seg.layout;
    for (int i = 0; i < ncand && rc == BLDTT_OK; ++i) {
      seg.layout = cand[i];
      if ((rc = interaction_grids(p)) != BLDTT_OK) break;
      float t = 0.f;
      for (int rep = 0; rep < 3 && rc == BLDTT_OK; ++rep) {   // first run warms up
        if (cudaEventRecord(e0, s) != cudaSuccess || (rc = run_segment(p, (int)g, s)) != BLDTT_OK ||
            cudaEventRecord(e1, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
          if (rc == BLDTT_OK) rc = BLDTT_ECUDA;
          break;
        }
        if ((rc = device_error(p)) != BLDTT_OK) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep == 1 || (rep > 1 && ms < t)) t = ms;
      }
      if (rc == BLDTT_OK) p->tune_table.push_back({(int)g, seg.kernel, cand[i], t});
      if (rc == BLDTT_OK && (best < 0.f || t < best)) {
        best = t;
        best_layout = cand[i];
      }
    }
    seg.layout = best_layout;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  BL_TRY(rc);
  BL_TRY(interaction_grids(p));
  if (p->graph_exec) {                    // a captured graph used the old layouts
    cudaGraphExecDestroy(p->graph_exec);
    p->graph_exec = nullptr;
  }
  if (chosen) *chosen = p->segments.empty() ? 0 : p->segments[0].layout;
  p->tuned = true;
  return BLDTT_OK;
}

int bldtt_set_pass_engine(bldtt_plan* p, int upward, int downward) {
  auto valid = [](int e) { return e == BLDTT_PASS_SIMT || e == BLDTT_PASS_TENSOR; };
  if (!p || !valid(upward) || !valid(downward)) {
    set_error("set_pass_engine: plan must be non-NULL and each engine BLDTT_PASS_SIMT or "
              "BLDTT_PASS_TENSOR");
    return BLDTT_EINVAL;
  }
  p->up_engine = upward;
  p->down_engine = downward;
  if (p->graph_exec) {                    // a captured graph used the other kernels
    cudaGraphExecDestroy(p->graph_exec);
    p->graph_exec = nullptr;
  }
  return BLDTT_OK;
}

int bldtt_pass_engine_used(const bldtt_plan* p, int which) {
  if (!p || (which != 0 && which != 1)) return -1;
  const int e = which == 0 ? p->up_engine : p->down_engine;
  return (p->precision == BLDTT_FP32_BULK && e == BLDTT_PASS_TENSOR && leaf_tc_supported(p->P))
             ? BLDTT_PASS_TENSOR
             : BLDTT_PASS_SIMT;
}

int bldtt_autotune_table(const bldtt_plan* p, int capacity, int* rows, int* launch, int* kernel,
                         int* layout, float* ms) {
  if (!p || !rows || capacity < 0 || (capacity > 0 && (!launch || !kernel || !layout || !ms))) {
    set_error("autotune_table: plan, rows and (for capacity > 0) the four arrays must be non-NULL");
    return BLDTT_EINVAL;
  }
  if (!p->tuned) {
    set_error("autotune_table: the plan has not been autotuned");
    return BLDTT_EINVAL;
  }
  *rows = (int)p->tune_table.size();
  for (int i = 0; i < *rows && i < capacity; ++i) {
    launch[i] = p->tune_table[i].launch;
    kernel[i] = p->tune_table[i].kernel;
    layout[i] = p->tune_table[i].layout;
    ms[i] = p->tune_table[i].ms;
  }
  return BLDTT_OK;
}

}  // extern "C"

namespace bldtt {
int compute_body(bldtt_plan* p, double* phi, cudaStream_t s) {
  BL_CUDA(cudaEventRecord(p->ev[0], s));
  for (int i = 0; i < p->deg.n; ++i)
    BL_CUDA(cudaMemsetAsync(p->phit_d[i], 0, (size_t)p->tt.nclusters * p->deg.np[i] * sizeof(double), s));
  BL_CUDA(cudaMemsetAsync(p->phi_near, 0, (size_t)p->M * sizeof(double), s));
  BL_TRY(upward_pass(p, s));
  BL_TRY(build_pool(p, s));
  BL_CUDA(cudaEventRecord(p->ev[1], s));
  BL_TRY(run_interactions(p, s));
  BL_CUDA(cudaEventRecord(p->ev[2], s));
  BL_TRY(downward_pass(p, phi, s));
  BL_CUDA(cudaEventRecord(p->ev[3], s));
  p->have_compute_events = true;
  return BLDTT_OK;
}
}  // namespace bldtt

extern "C" {

int bldtt_check_error(bldtt_plan* p) {
  if (!p) return BLDTT_EINVAL;
  BL_TRY(sync_plan(p));
  return device_error(p);
}

int bldtt_stats(bldtt_plan* p, bldtt_stats_t* out) {
  if (!p || !out) {
    set_error("plan and out must be non-NULL");
    return BLDTT_EINVAL;
  }
  BL_TRY(sync_plan(p));
  std::memset(out, 0, sizeof(*out));
  out->num_targets = p->M;
  out->num_sources = p->N;
  out->num_target_clusters = p->tt.nclusters;
  out->num_source_clusters = p->st.nclusters;
  out->num_target_leaves = p->tt.nleaves;
  out->num_source_leaves = p->st.nleaves;
  out->target_levels = p->tt.nlevels;
  out->source_levels = p->st.nlevels;
  for (int k = 0; k < 4; ++k) {
    out->list_entries[k] = p->list_count[k];
    out->interactions[k] = p->interactions[k];
  }
  out->executed_evaluations = p->executed_evaluations;
  out->work_items = p->nitems;
  out->interact_grid = p->segments.empty() ? 0 : p->segments[0].grid;
  out->interact_threads = p->segments.empty() ? 0 : p->segments[0].threads;
  out->ms_tree = p->ms_tree;
  out->ms_lists = p->ms_lists;
  if (p->have_compute_events) {
    out->ms_upward = elapsed(p->ev[0], p->ev[1]);
    out->ms_interact = elapsed(p->ev[1], p->ev[2]);
    out->ms_downward = elapsed(p->ev[2], p->ev[3]);
    out->ms_compute = elapsed(p->ev[0], p->ev[3]);
  }
  out->launches_setup = p->setup_counter.launches;
  out->launches_compute = p->compute_counter.launches;
  out->computed_evaluations = p->computed_evals;
  return device_error(p);
}

void bldtt_destroy(bldtt_plan* p) { release(p); }

int bldtt_tree_size(bldtt_plan* p, int which, int32_t* num_clusters, int32_t* num_levels) {
  if (!p || (which != 0 && which != 1)) return BLDTT_EINVAL;
  const Tree& T = which == 0 ? p->tt : p->st;
  if (num_clusters) *num_clusters = T.nclusters;
  if (num_levels) *num_levels = T.nlevels;
  return BLDTT_OK;
}

int bldtt_export_tree(bldtt_plan* p, int which, int32_t* perm, int32_t* begin, int32_t* end,
                      double* lo, double* hi, int32_t* parent, int32_t* level) {
  if (!p || (which != 0 && which != 1)) {
    set_error("bad plan or tree selector");
    return BLDTT_EINVAL;
  }
  BL_TRY(sync_plan(p));
  const Tree& T = which == 0 ? p->tt : p->st;
  const size_t C = (size_t)T.nclusters;
  if (perm) BL_CUDA(cudaMemcpy(perm, T.perm, (size_t)T.n * 4, cudaMemcpyDeviceToHost));
  if (begin) BL_CUDA(cudaMemcpy(begin, T.begin, C * 4, cudaMemcpyDeviceToHost));
  if (end) BL_CUDA(cudaMemcpy(end, T.end, C * 4, cudaMemcpyDeviceToHost));
  if (parent) BL_CUDA(cudaMemcpy(parent, T.parent, C * 4, cudaMemcpyDeviceToHost));
  if (level) BL_CUDA(cudaMemcpy(level, T.level, C * 4, cudaMemcpyDeviceToHost));
  if (lo || hi) {
    std::vector<double> box(C * 6);
    BL_CUDA(cudaMemcpy(box.data(), T.box, C * 6 * sizeof(double), cudaMemcpyDeviceToHost));
    for (size_t c = 0; c < C; ++c)
      for (int d = 0; d < 3; ++d) {
        if (lo) lo[d * C + c] = box[c * 6 + d];
        if (hi) hi[d * C + c] = box[c * 6 + 3 + d];
      }
  }
  return BLDTT_OK;
}

int bldtt_export_lists(bldtt_plan* p, int type, int32_t* target, int32_t* source, int64_t* count) {
  if (!p || type < 0 || type >= p->nclass || !count) {
    set_error("bad plan, list class or count pointer");
    return BLDTT_EINVAL;
  }
  int64_t need = p->class_count[type];
  if (*count < need) {
    *count = need;
    set_error("list capacity %lld below the %lld entries", (long long)*count, (long long)need);
    return BLDTT_EINVAL;
  }
  *count = need;
  if (need == 0) return BLDTT_OK;
  BL_TRY(sync_plan(p));
  int32_t first = 0;
  BL_CUDA(cudaMemcpy(&first, p->list_ptr + (int64_t)type * p->tt.nclusters, sizeof(int32_t),
                     cudaMemcpyDeviceToHost));
  if (target)
    BL_CUDA(cudaMemcpy(target, p->list_tgt + first, need * sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (source)
    BL_CUDA(cudaMemcpy(source, p->list_src + first, need * sizeof(int32_t), cudaMemcpyDeviceToHost));
  return BLDTT_OK;
}

int bldtt_export_proxy_charges(bldtt_plan* p, double* qhat) {
  if (!p || !qhat) return BLDTT_EINVAL;
  BL_TRY(sync_plan(p));
  BL_CUDA(cudaMemcpy(qhat, p->qhat, (size_t)p->st.nclusters * p->np * sizeof(double),
                     cudaMemcpyDeviceToHost));
  return BLDTT_OK;
}

int bldtt_export_proxy_potentials(bldtt_plan* p, double* phit) {
  if (!p || !phit) return BLDTT_EINVAL;
  BL_TRY(sync_plan(p));
  BL_CUDA(cudaMemcpy(phit, p->phit, (size_t)p->tt.nclusters * p->np * sizeof(double),
                     cudaMemcpyDeviceToHost));
  return BLDTT_OK;
}

int bldtt_direct_sum(const double* targets, int64_t M, const double* sources, int64_t N,
                     const double* charges, int kernel, double kappa, double* phi,
                     void* cuda_stream) {
  if (!targets || !sources || !charges || !phi || M < 0 || N < 0) {
    set_error("direct sum: NULL pointer or negative size");
    return BLDTT_EINVAL;
  }
  if (kernel != BLDTT_COULOMB && kernel != BLDTT_YUKAWA && kernel != BLDTT_OSCILLATORY &&
      kernel != BLDTT_REG_COULOMB && kernel != BLDTT_TEST_POLY) {
    set_error("unknown kernel %d", kernel);
    return BLDTT_EINVAL;
  }
  if (M == 0) return BLDTT_OK;
  return direct_sum(targets, M, sources, N, charges, kernel, kappa, phi,
                    static_cast<cudaStream_t>(cuda_stream));
}

int bldtt_solve_host(const double* targets, int64_t M, const double* sources, int64_t N,
                     const double* charges, int kernel, double kappa, int n, double theta, int N0,
                     int M0, int precision, double* phi, bldtt_stats_t* stats) {
  if (!targets || !sources || !charges || !phi) {
    set_error("solve_host: NULL host pointer");
    return BLDTT_EINVAL;
  }
  BL_TRY(validate(M, N, kernel, kappa, n, theta, N0, M0, precision));
  cudaMemPool_t pool = nullptr;   // the input and output buffers come from the shared pool too
  BL_TRY(shared_pool(&pool));
  PlanScope scope(pool, nullptr);
  cudaStream_t s = nullptr;
  BL_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  const bool same = targets == sources && M == N;
  double *dt = nullptr, *ds = nullptr, *dq = nullptr, *dphi = nullptr;
  bldtt_plan* plan = nullptr;
  int st = BLDTT_OK;
  do {
    if ((st = dalloc_n(&dt, (size_t)3 * M, s)) != BLDTT_OK) break;
    if (!same && (st = dalloc_n(&ds, (size_t)3 * N, s)) != BLDTT_OK) break;
    if ((st = dalloc_n(&dq, (size_t)N, s)) != BLDTT_OK) break;
    if ((st = dalloc_n(&dphi, (size_t)M, s)) != BLDTT_OK) break;
    if (same) ds = dt;
    if (cudaMemcpyAsync(dt, targets, 3 * M * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        (!same && cudaMemcpyAsync(ds, sources, 3 * N * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess) ||
        cudaMemcpyAsync(dq, charges, N * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess) {
      set_error("solve_host: host-to-device copy failed");
      st = BLDTT_ECUDA;
      break;
    }
    if ((st = bldtt_setup(&plan, dt, M, ds, N, dq, kernel, kappa, n, theta, N0, M0, precision, s)) != BLDTT_OK) break;
    if ((st = bldtt_compute(plan, dphi, s)) != BLDTT_OK) break;
    if (cudaMemcpyAsync(phi, dphi, M * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) {
      set_error("solve_host: device-to-host copy failed");
      st = BLDTT_ECUDA;
      break;
    }
    if (stats) st = bldtt_stats(plan, stats);
    else st = bldtt_check_error(plan);
  } while (0);
  bldtt_destroy(plan);
  dfree(dt, s);
  if (!same) dfree(ds, s);
  dfree(dq, s);
  dfree(dphi, s);
  cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  cudaGetLastError();
  return st;
}

}  // extern "C"
