/*
 * bldtt.h - C ABI of the GB300 BLDTT library (libbldtt.so).
 *
 * The library computes the compute phase of the barycentric Lagrange dual
 * tree traversal (BLDTT) of Wilson, Vaughn & Krasny: the potentials
 *
 *     phi(x_i) = sum_j G(x_i, y_j) q_j,   i = 1..M          (Eq. (1))
 *
 * of M target particles due to N charged source particles, approximated with
 * particle-particle (PP), particle-cluster (PC), cluster-particle (CP) and
 * cluster-cluster (CC) interactions between the clusters of a target tree and
 * a source tree (Algorithm 1).  Every step runs in CUDA kernels on the device
 * that is current when bldtt_setup is called; there is no CPU fallback.
 *
 * Conventions shared by all entry points
 *  - Particle coordinates are float64 structure-of-arrays: a buffer of 3*M
 *    doubles holding x[0..M), then y[0..M), then z[0..M).
 *  - "device" pointers are CUDA device (or managed) memory of the current
 *    device; "host" pointers are ordinary host memory.
 *  - cuda_stream is a cudaStream_t passed as void*; NULL means the legacy
 *    default stream.  All work of a call is ordered on that stream.
 *  - Every int-returning function returns a bldtt_status; nothing throws and
 *    nothing aborts.  After an error the plan can still be destroyed.
 *  - Readings of the paper the library applies where the paper is silent:
 *    leaf iff |C| <= M0 (or all box extents are zero); up to 1, 2 or 3
 *    split dimensions for M0<|C|<=2M0, 2M0<|C|<=4M0, larger; a dimension is
 *    split only if L_d*L_d*2 >= L_max*L_max; split at the midpoint of the
 *    shrunk box, upper half iff coord >= midpoint; children ordered by
 *    (x,y,z) bits; cluster radius = half the box diagonal; MAC evaluated as
 *    r_t + r_s < theta*R; proxy points c + h*cos(pi k/n) per dimension;
 *    a pair at distance 0 contributes nothing.
 */
#ifndef BLDTT_H
#define BLDTT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
enum bldtt_status {
    BLDTT_OK = 0,
    BLDTT_EINVAL = 1,     /* invalid argument (size, degree, theta, kernel, NaN input ...) */
    BLDTT_ENOMEM = 2,     /* a device allocation failed */
    BLDTT_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed */
    BLDTT_ETIMEOUT = 4,   /* a bounded wait inside a kernel gave up (error flag set) */
    BLDTT_EINTERNAL = 5   /* an internal consistency check failed */
};

/* Interaction kernels G(x, y), with r = |x - y| (Sec. 4.6). */
enum bldtt_kernel {
    BLDTT_COULOMB = 0,    /* G = 1/r */
    BLDTT_YUKAWA = 1,     /* G = exp(-kappa r)/r, kappa >= 0 */
    BLDTT_OSCILLATORY = 2,   /* G = sin(kappa r)/r, kappa >= 0 (Sec. 4.6 uses kappa = pi) */
    BLDTT_REG_COULOMB = 3,   /* G = 1/sqrt(r^2 + kappa^2), kappa >= 0 (Sec. 4.6: 0.005);
                                a pair at r = 0 still contributes nothing */
    BLDTT_TEST_POLY = 99  /* test kernel of degree 2 in each coordinate, d = x - y:
                             G = 1 + d1 - 2 d2 + 3 d3 + d1 d2 - d2 d3 + d1^2 d3^2 - d2^2/2.
                             Interpolation of degree n >= 2 reproduces it exactly. */
};

/* Arithmetic of the kernel evaluations. */
enum bldtt_precision {
    BLDTT_FP64 = 0,       /* plain FP64 everywhere */
    BLDTT_FP32_BULK = 1   /* kernel evaluations and Lagrange contractions in FP32, in
                             coordinate frames local to each source cluster, summed in
                             FP64 every 256 sources; barycentric weights, the
                             coincident-point guard, proxy points, proxy charges,
                             proxy potentials and the final phi stay FP64 */
};

/* Traversal variants.  BLDTT_VARIANT_CC_PP_ONLY is the ablation of Sec. 4.3:
 * a well-separated pair interacts by CC when both clusters hold more than n_p
 * particles and by PP otherwise (no PC or CP). */
enum bldtt_variant { BLDTT_VARIANT_FULL = 0, BLDTT_VARIANT_CC_PP_ONLY = 1 };

/* Engines of the FP32_BULK leaf contractions (Eq. (9) of the upward pass and
 * Eq. (21) of the downward pass): SIMT FP32 arithmetic, or the tensor cores
 * (tcgen05 MMA on TF32 operands split in two parts, accumulators in tensor
 * memory), see bldtt_set_pass_engine. */
enum bldtt_pass_engine { BLDTT_PASS_SIMT = 0, BLDTT_PASS_TENSOR = 1 };

/* Interaction types (Sec. 2.4), used to index the list arrays below. */
enum bldtt_interaction { BLDTT_PP = 0, BLDTT_PC = 1, BLDTT_CP = 2, BLDTT_CC = 3 };

typedef struct bldtt_plan bldtt_plan;   /* opaque; owned by the library */

typedef struct bldtt_stats {
    int64_t num_targets, num_sources;
    int32_t num_target_clusters, num_source_clusters;
    int32_t num_target_leaves, num_source_leaves;
    int32_t target_levels, source_levels;
    int64_t list_entries[4];            /* entries per type PP, PC, CP, CC */
    double interactions[4];             /* kernel evaluations per type, as defined by
                                           Eqs. (6), (8), (12), (15): |C_t||C_s|,
                                           |C_t| n_p, n_p |C_s|, n_p^2 per entry */
    double executed_evaluations;        /* evaluations the interaction kernel performs
                                           in its default layout: every 32-target row group
                                           holding a real target meets every real source
                                           (the idle rows of such a group included) */
    int64_t work_items;                 /* target tiles drained by the interaction kernel */
    int32_t interact_grid;              /* CTAs of the persistent interaction kernel */
    int32_t interact_threads;           /* threads per CTA of that kernel */
    float ms_tree, ms_lists;            /* last bldtt_setup: trees; traversal + work lists */
    float ms_upward, ms_interact, ms_downward, ms_compute;   /* last bldtt_compute */
    int64_t launches_setup, launches_compute;                /* kernels launched */
    double computed_evaluations;        /* evaluations (as interactions[]) of the work
                                           items the last compute ran: all of them after
                                           bldtt_compute, one shard's after
                                           bldtt_compute_shard */
} bldtt_stats_t;

/*
 * bldtt_setup - build both trees (Sec. 2.3), run the dual tree traversal
 * (Algorithm 2) and lay out the work of the compute phase.
 *
 *  plan      out: receives a new plan; *plan is NULL on error.
 *  targets   device, 3*M float64, SoA (x block, y block, z block).
 *  M         number of targets, 1 <= M < 2^31.
 *  sources   device, 3*N float64, SoA.
 *  N         number of sources, 1 <= N < 2^31.
 *  charges   device, N float64 (input order of the sources).
 *  kernel    enum bldtt_kernel.
 *  kappa     parameter of BLDTT_YUKAWA, BLDTT_OSCILLATORY and BLDTT_REG_COULOMB:
 *            finite and >= 0 (else EINVAL); ignored by the other kernels.
 *  n         interpolation degree, 1 <= n <= 16; proxies per cluster n_p=(n+1)^3.
 *  theta     MAC parameter, theta >= 0 (theta = 0 gives only PP, i.e. the direct sum).
 *  N0, M0    maximum particles per source / target leaf, >= 1.
 *  precision enum bldtt_precision.
 *
 * The caller keeps ownership of targets/sources/charges; they are copied into
 * tree order before the call returns (the call synchronises the stream), so
 * they may be freed afterwards.  The plan owns all device memory it
 * allocates (stream-ordered allocations on cuda_stream, from one memory pool
 * per device that the library shares between its plans and trims to an
 * eighth of the device's memory when a set-up ends or a plan is destroyed).
 * Each tree is built, and the fixed-rule traversal run, by one cooperative
 * launch; with the environment variable BLDTT_LEVEL_BY_LEVEL=1 (or on a
 * device without cooperative launches) both run level by level from the
 * host instead, with identical results.  BLDTT_TREE_CAPACITY and
 * BLDTT_TRAVERSAL_CAPACITY override the initial cluster and traversal buffer
 * capacities (testing: a small start makes the launches regrow and resume;
 * the results do not change).
 * Errors: EINVAL for out-of-range sizes or parameters, a non-finite
 * coordinate or charge, an unknown kernel or precision; ENOMEM; ECUDA;
 * ETIMEOUT if a grid barrier of a cooperative launch waited 5 s in vain.
 */
int bldtt_setup(bldtt_plan** plan,
                const double* targets, int64_t M,
                const double* sources, int64_t N,
                const double* charges,
                int kernel, double kappa, int n, double theta, int N0, int M0,
                int precision, void* cuda_stream);

/* Parameters of bldtt_setup_ex: the method parameters of bldtt_setup plus
 * the traversal variant (enum bldtt_variant). */
typedef struct bldtt_params {
    int kernel;
    double kappa;
    int n;
    double theta;
    int N0, M0;
    int precision;
    int variant;
} bldtt_params_t;

/*
 * bldtt_setup_ex - bldtt_setup with the parameters in a struct, adding the
 * traversal variant.  Same arguments, ownership and errors as bldtt_setup;
 * EINVAL also for an unknown variant or a NULL params pointer.
 */
int bldtt_setup_ex(bldtt_plan** plan,
                   const double* targets, int64_t M,
                   const double* sources, int64_t N,
                   const double* charges,
                   const bldtt_params_t* params, void* cuda_stream);

/*
 * bldtt_setup_batch - set up nprob independent problems as one plan, so that
 * a single bldtt_compute (or one replay of bldtt_compute_graph) runs all of
 * them: the trees of all problems are built level by level together (a
 * forest with one root per problem), the traversal starts from every
 * problem's pair of roots, and the interaction work of all problems is
 * drained by one persistent launch per kernel type present in the batch
 * (work items are grouped by the kernel of their problem).  Problem i owns targets [target_offsets[i],
 * target_offsets[i+1]) and sources [source_offsets[i], source_offsets[i+1])
 * of the concatenated SoA arrays (targets 3*M, sources 3*N, charges N, with
 * M = target_offsets[nprob], N = source_offsets[nprob]); it interacts only
 * with itself, with kernel kernels[i] and parameter kappas[i].  phi of
 * bldtt_compute is the concatenation of the problems' potentials.
 *
 *  nprob                     >= 1 problems.
 *  target_/source_offsets    host, nprob + 1 int64, starting at 0, strictly
 *                            increasing (every problem has >= 1 target and
 *                            >= 1 source).
 *  kernels, kappas           host, nprob entries (enum bldtt_kernel, parameter).
 *  params                    n, theta, N0, M0, precision, variant shared by all
 *                            problems (its kernel and kappa are ignored).
 * Ownership, synchronisation and errors as bldtt_setup.
 */
int bldtt_setup_batch(bldtt_plan** plan, int nprob,
                      const double* targets, const int64_t* target_offsets,
                      const double* sources, const int64_t* source_offsets,
                      const double* charges, const int* kernels, const double* kappas,
                      const bldtt_params_t* params, void* cuda_stream);

/*
 * Learned pair selector (no counterpart in the paper: the paper fixes one
 * degree n and the MAC r_t + r_s < theta R of Alg. 2).  A network of three
 * hidden ReLU layers of 64 reads six features of a pair (C_t, C_s) with
 * R = |c_t - c_s| > 0 and (r_t + r_s)/R < 1:
 *   plog2(|C_t|)/16, plog2(|C_s|)/16, r_t/R, r_s/R, (r_t + r_s)/R, kappa R/(1 + kappa R)
 * (plog2(m) = e + (f - 1) for m = f 2^e, 1 <= f < 2; radii are half box
 * diagonals) and predicts, for each degree degrees[i], the log10 of the
 * relative l2 error of PC, CP and CC (Eqs. (8), (12), (15)) on the pair:
 * output 3 i + t, t = 0 PC, 1 CP, 2 CC.  The traversal takes the cheapest
 * option predicted at or below log10_budget (cost PC |C_t| n_p(d), CP
 * n_p(d) |C_s|, CC n_p(d)^2), or PP when |C_t||C_s| costs no more; with no
 * feasible option it descends as Alg. 2 does for a pair that fails the MAC.
 * Pairs whose features fall outside [feature_lo, feature_hi] are decided by
 * the MAC of Alg. 2 (params theta) at the highest degree.
 *
 * Arithmetic (identical on every device): features in FP64, rounded to
 * float and to bfloat16 (round to nearest even); bf16 weights; each neuron
 * z_j = b_j + sum_k w_jk a_k summed in float in increasing k (bf16 products
 * are exact in float); a_j = bf16(max(z_j, 0)); float biases.
 *
 * weights: host float32 master weights, rows = outputs, packed
 *   W1[64][6] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[3m][64] b4[3m]
 *   (m = num_degrees; bldtt_selector_param_count gives the length), or NULL:
 *   then every pair is decided by the MAC at the highest degree.
 */
typedef struct bldtt_selector {
    int num_degrees;                /* 1..8 */
    int degrees[8];                 /* strictly increasing, 1..16; the highest = params n */
    const float* weights;           /* host, see above, or NULL */
    float feature_lo[6], feature_hi[6];
    float log10_budget;             /* per-pair budget, log10 of the relative error */
} bldtt_selector_t;

/* Number of float32 master weights of a selector with num_degrees degrees
 * (-1 if num_degrees is outside 1..8). */
int64_t bldtt_selector_param_count(int num_degrees);

/*
 * bldtt_setup_learned - bldtt_setup_ex with the learned selector in place of
 * the MAC.  The plan carries proxies of every degree of sel (the proxy
 * charges of a lower degree d come from those of the highest n by the exact
 * transfer A(x)A(x)A, A[k][k'] = L^(d)_k(s^(n)_k'); proxy potentials of
 * degree d go back to the degree-n grid by its transpose before Eq. (20)).
 * Interaction lists are then classes: 0 = PP, 1 + 3 i + t = (PC, CP, CC)[t]
 * at degree degrees[i] (bldtt_list_classes, bldtt_export_lists).  Arguments,
 * ownership and errors as bldtt_setup_ex; EINVAL also for a bad selector
 * (degree count or order, highest degree != params n, empty feature box,
 * non-finite budget or weight).  The selector is copied; the caller keeps it.
 */
int bldtt_setup_learned(bldtt_plan** plan, const double* targets, int64_t M,
                        const double* sources, int64_t N, const double* charges,
                        const bldtt_params_t* params, const bldtt_selector_t* sel,
                        void* cuda_stream);

/* Interaction-list classes of a plan: *num_classes = 1 + 3 * num_degrees,
 * degrees (capacity 8, may be NULL) receives the plan's degrees. */
int bldtt_list_classes(bldtt_plan* plan, int* num_classes, int* degrees, int* num_degrees);

/*
 * Training of the selector network (device buffers throughout, asynchronous
 * on cuda_stream).  params: the packed float32 master weights; x: [batch][6]
 * float32 features (rounded to bf16 inside, as in the selector); y, target,
 * mask: [batch][num_out]; num_out = 3 * num_degrees <= 24.
 *  bldtt_mlp_forward:   y = network(x) with the selector's arithmetic.
 *  bldtt_mlp_gradients: loss = sum mask (y - target)^2 / max(1, sum mask)
 *                       (written to *loss, device, if non-NULL) and its
 *                       gradient for every master weight (grads, same
 *                       layout as params), ReLU' = [z > 0], the bf16
 *                       rounding of weights and activations passed through;
 *                       sums over the batch in float in increasing order.
 *  bldtt_mlp_adam:      one Adam step (beta 0.9, 0.999, eps 1e-8; step >= 1
 *                       counts from 1) on count weights with moments m, v.
 * Errors: EINVAL (NULL pointers, sizes), ENOMEM, ECUDA.
 */
int bldtt_mlp_forward(const float* params, int num_out, const float* x, int64_t batch, float* y,
                      void* cuda_stream);
int bldtt_mlp_gradients(const float* params, int num_out, const float* x, const float* target,
                        const float* mask, int64_t batch, float* grads, float* loss,
                        void* cuda_stream);
int bldtt_mlp_adam(float* params, float* m, float* v, const float* grads, int64_t count, int step,
                   float lr, void* cuda_stream);

/*
 * Training data from a plan's trees (cluster ids as bldtt_export_tree
 * numbers them; pairs: device int32 [npairs][2] = (target cluster, source
 * cluster)).
 *  bldtt_pair_features: the selector's six FP64 features per pair into
 *    features (device [npairs][6]); NaN for pairs that cannot be approximated.
 *  bldtt_pair_errors: in FP64, the relative l2 error of PC, CP and CC at each
 *    degree against the exact pair sum of Eq. (6) (the plan's kernel and
 *    charges), on min(samples, |C_t|) targets spread evenly over C_t (a
 *    source cluster of more than 4096 particles is represented, in the exact
 *    sum and the approximations alike, by every ceil(|C_s|/4096)-th one):
 *    err (device [npairs][num_degrees][3]).  samples <= 256, degrees in
 *    1..16 (host array of num_degrees <= 8).
 * Errors: EINVAL, ECUDA.
 */
int bldtt_pair_features(bldtt_plan* plan, int64_t npairs, const int32_t* pairs, double* features,
                        void* cuda_stream);
int bldtt_pair_errors(bldtt_plan* plan, int64_t npairs, const int32_t* pairs, int samples,
                      int num_degrees, const int* degrees, double* err, void* cuda_stream);

/*
 * bldtt_set_charges - replace the source charges of a plan (device, N
 * float64, input order).  Trees and interaction lists depend only on the
 * positions and parameters and are reused.  Errors: EINVAL (NULL arguments,
 * non-finite charge), ECUDA.
 */
int bldtt_set_charges(bldtt_plan* plan, const double* charges, void* cuda_stream);

/*
 * bldtt_compute - upward pass (Sec. 2.5), PP/PC/CP/CC interactions over the
 * lists (Sec. 2.4), downward pass (Sec. 2.7); writes phi.
 *
 *  phi  device, M float64, input order of the targets; overwritten.
 *
 * Asynchronous on cuda_stream (no host synchronisation; phase timings are
 * read later by bldtt_stats).  Errors: EINVAL, ECUDA, ETIMEOUT (reported by
 * the next call that synchronises, e.g. bldtt_stats or bldtt_check_error).
 */
int bldtt_compute(bldtt_plan* plan, double* phi, void* cuda_stream);

/*
 * bldtt_compute_shard - the compute phase for one shard of the target leaves,
 * for one process per GPU (no counterpart in the paper, whose distributed
 * runs partition both particle sets and exchange locally essential trees,
 * Sec. 3.2; here the sources stay whole on every GPU).  Every rank sets up the
 * same plan (set-up is deterministic), and rank `shard` of `nshards` calls
 * this instead of bldtt_compute: it runs the whole upward pass, the PP/PC
 * work items of its leaves, the CP/CC work items of every target cluster above
 * or at its leaves (shared ancestors are computed by every rank that needs
 * them, with the same result), and the downward pass, and writes phi only at
 * its own targets; every other entry of phi is left untouched.  The leaves, in
 * tree order, are split into nshards contiguous ranges of equal cost
 * (bldtt_partition_leaves; a leaf costs its particle items' kernel
 * evaluations plus, for every cluster on its path to the root, that cluster's
 * proxy-item evaluations divided among the leaves under it).  The union of
 * the shards' outputs equals bldtt_compute's phi bit for bit, so ranks that
 * zero-fill phi, compute their shard and sum phi over ranks (or gather their
 * entries) get the one-GPU result.
 *
 *  shard, nshards  0 <= shard < nshards; nshards = 1 is bldtt_compute.
 *  phi             device, M float64, input order; only the shard's targets
 *                  are written.
 *
 * The first call for a given nshards synchronises the stream once (costs to
 * the host); the shard's work list is kept in the plan until another shard is
 * computed.  Otherwise asynchronous on cuda_stream.  Errors: EINVAL, ENOMEM,
 * ECUDA, ETIMEOUT (reported by the next synchronising call).
 */
int bldtt_compute_shard(bldtt_plan* plan, int shard, int nshards, double* phi, void* cuda_stream);

/*
 * bldtt_partition_leaves - host-only: split nleaves leaves, in order, with
 * costs leaf_cost (host, >= 0, finite) into nshards contiguous ranges of
 * nearly equal total cost.  leaf_begin (host, nshards + 1 int32) receives the
 * first leaf of each range and nleaves last; the k-th boundary is the leaf
 * boundary nearest to k/nshards of the total cost (never before the previous
 * one), so ranges may be empty when there are fewer leaves than shards; if
 * every cost is zero the ranges hold equal numbers of leaves.
 * Deterministic; no device work.  Errors: EINVAL.
 */
int bldtt_partition_leaves(const double* leaf_cost, int32_t nleaves, int32_t nshards,
                           int32_t* leaf_begin);

/*
 * bldtt_compute_graph - bldtt_compute through a CUDA graph.  The first call
 * (and any call with a different phi pointer) captures the whole compute
 * phase on cuda_stream into a graph and instantiates it; every call then
 * launches that graph (one launch for all the compute-phase kernels).  The
 * stream must be a created stream (not NULL or a default stream).  The plan
 * keeps the graph until it is destroyed, re-captured or re-tuned.
 * Errors: EINVAL, ECUDA.
 */
int bldtt_compute_graph(bldtt_plan* plan, double* phi, void* cuda_stream);

/*
 * bldtt_autotune - pick the fastest launch shape of the interaction kernel
 * for each persistent launch of the plan: runs bldtt_compute once (phi,
 * device M float64, receives its potentials), then times each launch three
 * times per layout instantiated for its kernel with CUDA events and keeps the
 * fastest in the plan.  A layout fixes the CTA's tile of 256 targets (consumer
 * warps x targets per thread: 4 x 2 or 2 x 4), the CTAs per SM the registers
 * are sized for (6 or 5), the depth of the shared-memory ring of source
 * chunks (3 or 4 stages) and whether warps whose rows hold no real target
 * skip their work: layouts 0 = 4x2, 6 CTAs, 3 stages; 1 = 2x4, 6 CTAs, 3
 * stages; 2 = 4x2, 5 CTAs, 4 stages; 3-5 = the same with skipping (Coulomb
 * and the shared Coulomb/Yukawa launch; other kernels: layouts 0 and 3).
 * Results do not depend on the layout (bit for bit).  *chosen (may be NULL)
 * receives the layout picked for the plan's first launch; the searched table
 * is kept for bldtt_autotune_table.  Synchronous.  Errors: EINVAL, ECUDA,
 * ETIMEOUT.
 */
int bldtt_autotune(bldtt_plan* plan, double* phi, void* cuda_stream, int* chosen);

/*
 * bldtt_set_pass_engine - the engines of the plan's FP32_BULK leaf
 * contractions for the following computes: `upward` for Eq. (9) (leaf proxy
 * charges, Sec. 2.5), `downward` for Eq. (21) (leaf proxy potentials to the
 * particles, Sec. 2.7), each BLDTT_PASS_SIMT or BLDTT_PASS_TENSOR.  The
 * tensor engine runs each as one dense product on the tensor cores: upward,
 * the P^2 x m Khatri-Rao matrix of (L_k2 q)(L_k3) times the m x P matrix of
 * L_k1 per leaf of m particles, in chunks of 32 particles folded by TwoSum;
 * downward, the 128 x P matrix of L_k1 of 128 particles times the P x P^2
 * proxy potentials, then the k2, k3 sums per particle in FP32 (the k2 sum
 * compensated).  Operands are TF32 pairs a_h + a_l (four products per term,
 * the pair holding each operand to about 2^-22, FP32 accumulation).  Grids of 2..11 points
 * (P^2 <= 121); other grids, and FP64 plans, keep the SIMT kernels.  A new
 * plan starts with the upward pass on SIMT and the downward pass on the tensor
 * cores when its target leaves hold 512 particles or more on average (else
 * SIMT): the faster engine of each as measured on a GB300 (uniform points at
 * 1E6 and 1E7 with leaves of 2000, and the batched workload's leaves of 500).
 * A captured graph of the plan is dropped.  Errors: EINVAL.
 */
int bldtt_set_pass_engine(bldtt_plan* plan, int upward, int downward);

/* The engine the plan's upward (which = 0) or downward (which = 1) leaf
 * contraction runs on: BLDTT_PASS_TENSOR only when chosen and applicable,
 * else BLDTT_PASS_SIMT; -1 for a NULL plan or another `which`. */
int bldtt_pass_engine_used(const bldtt_plan* plan, int which);

/*
 * bldtt_autotune_table - the table the last bldtt_autotune searched: for each
 * of its *rows entries (at most capacity are written; *rows receives the
 * total), the launch index, the kernel id of that launch (1000: Coulomb and
 * Yukawa items in one launch), the layout and its best time in ms.  Host
 * arrays.  Errors: EINVAL (no autotune yet, or NULL arguments).
 */
int bldtt_autotune_table(const bldtt_plan* plan, int capacity, int* rows, int* launch, int* kernel,
                         int* layout, float* ms);

/*
 * bldtt_wait_probe - failure detection without a fault: one CTA waits, with
 * the interaction kernel's bounded-wait pattern (mbarrier try_wait until the
 * %globaltimer passes the limit, then the error flag is raised and the kernel
 * returns), on an mbarrier that nothing ever arrives on.  limit_ns in
 * [1000, 1e9].  Returns BLDTT_ETIMEOUT when the wait gave up as designed (the
 * expected outcome) and leaves the context usable; EINTERNAL if the wait
 * completed (it cannot), EINVAL for a limit out of range, ENOMEM, ECUDA.
 * Synchronous on cuda_stream.  No counterpart in the paper.
 */
int bldtt_wait_probe(int64_t limit_ns, void* cuda_stream);

/* Synchronise the plan's last stream and report a device-side error flag
 * (ETIMEOUT from a bounded wait, EINTERNAL from a bounds check). */
int bldtt_check_error(bldtt_plan* plan);

/* Fill *out with the counts above and the phase times of the last setup and
 * compute (synchronises the plan's stream).  Errors: EINVAL, ECUDA. */
int bldtt_stats(bldtt_plan* plan, bldtt_stats_t* out);

/* Release the plan and all its device memory.  NULL is ignored. */
void bldtt_destroy(bldtt_plan* plan);

/* Static, NUL-terminated name of a status code. */
const char* bldtt_status_string(int status);

/* Text of the last error raised by the calling host thread ("" if none). */
const char* bldtt_last_error(void);

/* ---- Introspection (host copies; each synchronises the plan's stream) ---- */

/*
 * bldtt_tree_size - number of clusters and levels of the target (which = 0)
 * or source (which = 1) tree.
 */
int bldtt_tree_size(bldtt_plan* plan, int which, int32_t* num_clusters, int32_t* num_levels);

/*
 * bldtt_export_tree - copy one tree to host buffers.  Clusters are numbered
 * level by level (parents before children).  perm[p] (num particles) is the
 * input index of the particle at tree position p; cluster c holds tree
 * positions [begin[c], end[c]); lo/hi are 3*C float64 SoA (x block, y block,
 * z block) of the shrunk box; parent[c] is -1 for the root; level[c] is the
 * depth.  Any pointer may be NULL to skip that array.
 */
int bldtt_export_tree(bldtt_plan* plan, int which, int32_t* perm, int32_t* begin, int32_t* end,
                      double* lo, double* hi, int32_t* parent, int32_t* level);

/*
 * bldtt_export_lists - copy the entries of one interaction-list class as
 * (target cluster, source cluster) pairs, sorted by target cluster.  For a
 * plan of one degree the classes are the types (enum bldtt_interaction);
 * see bldtt_setup_learned for plans of several degrees.  count is in/out: capacity on entry, entries on return
 * (EINVAL, with the needed count, if the capacity is too small).
 */
int bldtt_export_lists(bldtt_plan* plan, int type, int32_t* target, int32_t* source,
                       int64_t* count);

/* Copy the proxy charges q-hat (Eq. (9)) of every source cluster after the
 * last compute: num_source_clusters * n_p float64, cluster-major, proxy index
 * k = (k1*(n+1) + k2)*(n+1) + k3. */
int bldtt_export_proxy_charges(bldtt_plan* plan, double* qhat);

/* Copy the proxy potentials phi(t) of every target cluster after the
 * downward pass of the last compute (CP + CC of the cluster plus everything
 * interpolated down from its ancestors, Eq. (20)); same layout as q-hat. */
int bldtt_export_proxy_potentials(bldtt_plan* plan, double* phit);

/* ---- Helpers ---- */

/*
 * bldtt_direct_sum - FP64 direct summation, Eq. (1), on the device: for
 * every target i, phi[i] = sum_j G(x_i, y_j) q_j with pairs at distance 0
 * skipped.  Pointers are device memory in the layouts above.  Used to measure
 * the error of the fast method on sampled targets.  Asynchronous on
 * cuda_stream.  Errors: EINVAL, ECUDA.
 */
int bldtt_direct_sum(const double* targets, int64_t M, const double* sources, int64_t N,
                     const double* charges, int kernel, double kappa, double* phi,
                     void* cuda_stream);

/*
 * bldtt_solve_host - one-shot solve from host memory: copies the inputs to
 * the device, runs bldtt_setup and bldtt_compute, copies phi back and frees
 * everything.  targets (3*M), sources (3*N), charges (N) and phi (M) are
 * host float64 buffers; stats may be NULL.  Synchronous.
 */
int bldtt_solve_host(const double* targets, int64_t M, const double* sources, int64_t N,
                     const double* charges, int kernel, double kappa, int n, double theta,
                     int N0, int M0, int precision, double* phi, bldtt_stats_t* stats);

/* ---- Allocation-free entry point ---- */

/*
 * bldtt_bounding_box_noalloc - minimal bounding box of a particle set (the
 * box of a tree's root cluster), computed without allocating device memory.
 * The paper has no counterpart: it exists for callers that cannot call
 * cudaMalloc (a framework that owns all device memory, a real-time loop in
 * which allocation is forbidden).  bldtt_setup computes the same box with
 * scratch from the stream-ordered allocator; this variant keeps its scratch
 * in a fixed 56 KB __device__ array that every GPU loading the library holds
 * until the process exits.
 *
 *  points     device, 3*n float64, SoA (x block, y block, z block).
 *  n          1 <= n < 2^31 (larger sizes are rejected with EINVAL).
 *  box        device, 6 float64 written: lo x, lo y, lo z, hi x, hi y, hi z.
 *  nonfinite  device int or NULL; set to 1 if any coordinate is NaN or
 *             infinite (those values are left out of the box; a dimension
 *             with no finite value gets lo = +inf, hi = -inf), else 0.
 *
 * Minima and maxima are taken on the same order-preserving integer keys as
 * bldtt_setup, so the box equals the setup's root box bit for bit (-0.0 and
 * +0.0 compare equal and come back as +0.0).
 *
 * The first call on a device (with that device current) looks up the
 * array's device address with cudaGetSymbolAddress; make that first call
 * before any stream capture (a first call during capture returns EINVAL).
 * Later calls outside capture look the address up again, so a context
 * re-created by cudaDeviceReset gets the array's new address.  All calls
 * share the array and every call rewrites the slots it reads, but calls that
 * overlap on the GPU race on it: serialise them (one stream, or events).
 * Asynchronous on cuda_stream.  Errors: EINVAL, ECUDA.
 */
int bldtt_bounding_box_noalloc(const double* points, int64_t n, double* box, int* nonfinite,
                               void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* BLDTT_H */
