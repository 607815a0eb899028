/*
 * hgp.h -- C ABI of the GB300 library for incidence-constrained multilevel
 * hypergraph partitioning ("Incidence Constraints in Hypergraph Partitioning
 * on GPU", arXiv 2604.14411).
 *
 * Problem (Sec. II-A): a directed hypergraph G(N, E, omega); every hyperedge
 * e is a set of pins whose FIRST pin is its source src(e) and whose other
 * pins are its destinations dst(e).  in(n) = {e : n in dst(e)}.  A
 * partition rho must satisfy, for every part p,
 *     sum of node weights in p            <= Omega
 *     |union of in(n) over n in p|        <= Delta
 * and the method minimises the connectivity of Eq. (1),
 *     Conn = sum_e omega(e) * (number of distinct parts among e's pins - 1).
 *
 * Method (Sec. II-B, III, IV): coarsening levels (Eq. (2) neighbour scores,
 * bound-checked candidate per node, matching on the pairing pseudo-forest,
 * contraction) until ceil(W / Omega) nodes remain or no pair can merge; the
 * coarsest clusters are the initial parts; then per level, from coarsest to
 * finest, one or more refinement passes (Eq. (3) moves, sorted sequence,
 * in-sequence gains, best valid prefix) followed by projection.
 *
 * All computation runs in CUDA kernels on the current device, in stream
 * order on the stream given to hgp_create.  Ids and CSR offsets are int32;
 * the total pin count must be < 2^31.
 *
 * Thread safety: a handle is used by one host thread at a time.  Different
 * handles are independent.
 * Errors: every entry point returns an hgp_status; nothing is thrown across
 * the ABI.  hgp_last_error() gives a message for the last failure on a
 * handle.
 */
#ifndef HGP_H
#define HGP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HGP_OK = 0,
    HGP_ERR_INVALID_ARG = 1,   /* bad CSR, weights or bounds (see hgp_create) */
    HGP_ERR_INFEASIBLE = 2,    /* a single node already exceeds Omega or Delta */
    HGP_ERR_OOM = 3,           /* device allocation failed */
    HGP_ERR_CUDA = 4,          /* a CUDA call failed (message has the detail) */
    HGP_ERR_DEVICE_LIMIT = 5,  /* a bounded device loop ran out of its budget */
    HGP_ERR_STATE = 6,         /* call not valid in the handle's current state */
    HGP_ERR_SCRATCH_LIMIT = 7  /* input too large for hgp_score_noalloc's fixed scratch */
} hgp_status;

/* hgp_create flags */
#define HGP_INPUT_DEVICE 1u    /* offsets/pins/weights are device pointers */
#define HGP_DELTA_INCIDENT 4u  /* hgp_create: Delta bounds the distinct hyperedges incident to a part
                                  (in(n) = I(n)) instead of the inbound ones; the paper notes the
                                  generalisation in Sec. II-A */
#define HGP_DELTA_OUTBOUND 8u  /* hgp_create: Delta bounds the distinct hyperedges whose source lies
                                  in the part (in(n) = {e : src(e) = n}), the other direction of the
                                  same generalisation; not together with HGP_DELTA_INCIDENT */

/* hgp_result.out_flags */
#define HGP_OUTPUT_DEVICE 1u   /* part_ids/part_weight/part_inbound are device pointers */

/* hgp_options.debug bits */
#define HGP_DEBUG_KEEP_LEVELS 1u   /* keep per-level arrays for hgp_get_level_array */
#define HGP_DEBUG_TIMING 2u        /* time every phase with CUDA events (hgp_get_stats) */
#define HGP_DEBUG_FORCE_GLOBAL 4u  /* test knob: use the global-memory tables of the large-level
                                      paths for scoring and proposals at every level */
#define HGP_DEBUG_NO_BITMAP 8u     /* test knob: test in(n) membership by binary search instead
                                      of the shared-memory bitmap */
#define HGP_DEBUG_FORCE_CLUSTER 16u /* test knob: score every level with the 8-CTA cluster
                                       kernel (distributed shared-memory histogram) */
#define HGP_DEBUG_SMALL_TABLE 32u  /* test knob, with HGP_DEBUG_FORCE_GLOBAL: give the scoring
                                      kernel's per-CTA hash tables 64 slots, so a node with more
                                      distinct neighbours exhausts its bounded probe loop and the
                                      call returns HGP_ERR_DEVICE_LIMIT */
#define HGP_DEBUG_FORCE_WINDOW 128u /* test knob: score every level by per-node buckets with
                                       histogram pieces of max(64, |N_l| / 4) ids -- one CTA takes
                                       a node's neighbour-id window piece by piece, from the top
                                       ids down (the path of levels too large for one CTA) */
#define HGP_DEBUG_FORCE_HASH_BUCKET 256u /* test knob: as HGP_DEBUG_FORCE_WINDOW with single
                                       pieces, and a 1,024-slot hash table in shared memory for the
                                       nodes with at most 640 pin visits whose window takes more
                                       than one piece; the rest go to the 8-CTA cluster, so all
                                       three buckets take nodes */
#define HGP_DEBUG_REBUILD_INC 64u  /* test knob: keep no coarse level's I(n) until refinement;
                                      rebuild each from the level's pins when refinement reaches
                                      it (the path levels beyond the memory budget take) */

typedef struct hgp_graph hgp_graph;

/*
 * Device memory source of a handle (optional).  Every device buffer the
 * library uses for a handle -- the level-0 structure held by the handle, each
 * coarsening level kept until refinement reaches it, and the temporaries of a
 * call -- comes from alloc() in chunks (64 MiB or larger for levels and
 * temporaries, exact sizes for the handle's own arrays) and goes back through
 * free() with the same size.
 *   alloc(ctx, bytes, stream)      returns `bytes` of device memory on the
 *                                  current device, 256-byte aligned, usable in
 *                                  stream order on `stream`; NULL on failure
 *                                  (the call then returns HGP_ERR_OOM after
 *                                  returning every chunk it already holds)
 *   free(ctx, ptr, bytes, stream)  the library has enqueued every use of ptr
 *                                  on `stream` before this call; the memory
 *                                  may be reused by work ordered after it on
 *                                  that stream
 *   ctx                            passed back unchanged
 * `stream` is the handle's stream, or the per-instance stream that
 * hgp_partition_batch creates (destroyed, after a synchronise, when the call
 * returns).  The callbacks may be called from hgp_partition_batch's worker
 * threads concurrently.  The struct is copied by hgp_create; ctx and the
 * functions must stay valid until hgp_destroy.  A NULL allocator means
 * cudaMallocAsync / cudaFreeAsync on the same streams.  (A host program that
 * already owns a caching allocator, such as PyTorch's, passes it here so that
 * the library draws from the same pool.)
 */
typedef struct {
    void *(*alloc)(void *ctx, size_t bytes, void *stream);
    void (*free)(void *ctx, void *ptr, size_t bytes, void *stream);
    void *ctx;
} hgp_allocator;

/*
 * Build a hypergraph handle (the level-0 incidence structure of Sec. II-C:
 * pins of every hyperedge, and per node the sorted sets I(n) = in(n) u out(n)
 * and in(n)).
 *   num_nodes     |N| >= 1
 *   num_edges     |E| >= 0
 *   offsets       [num_edges + 1] int32, offsets[0] = 0, strictly increasing
 *                 (no empty hyperedge), offsets[E] = total pins < 2^31
 *   pins          [offsets[E]] int32 node ids in [0, num_nodes); first pin of
 *                 each edge is its source; no repeated pin within an edge
 *   node_weights  [num_nodes] int32 >= 1, or NULL for unit weights;
 *                 their sum must be < 2^31
 *   edge_weights  [num_edges] int32 >= 1, or NULL for unit weights (omega);
 *                 their sum must be < 2^31
 *   flags         HGP_INPUT_DEVICE: the four arrays are device memory
 *                 readable on `stream` (otherwise host memory);
 *                 HGP_DELTA_INCIDENT: Delta counts incident, not inbound, hyperedges;
 *                 HGP_DELTA_OUTBOUND: Delta counts outbound hyperedges (sourced in the
 *                 part); hgp_result.part_inbound then holds that count
 *   alloc         device memory source for everything the handle and its calls
 *                 use (see hgp_allocator), or NULL for cudaMallocAsync
 *   stream        cudaStream_t to run on (NULL = default stream)
 *   out           receives the handle
 * Ownership: inputs are copied; the caller may free them once the call has
 * returned (device inputs: once `stream` has reached this point).
 * Errors: HGP_ERR_INVALID_ARG for any violated rule above (checked on the
 * device), HGP_ERR_OOM, HGP_ERR_CUDA.  On error *out is NULL.
 */
int hgp_create(int32_t num_nodes, int32_t num_edges,
               const int32_t *offsets, const int32_t *pins,
               const int32_t *node_weights, const int32_t *edge_weights,
               uint32_t flags, const hgp_allocator *alloc, void *stream,
               hgp_graph **out);

/*
 * Learned candidate order (an extension; the paper has no counterpart).
 * A two-layer network scores each pair (n, m) from 8 features, symmetric in
 * n and m, each passed through lg1p(x) = k + (1 + x - 2^k) / 2^k for
 * 2^k <= 1 + x < 2^(k+1) (log2(1 + x) with a linear mantissa):
 *   x0 hist(n,m) (Eq. (2))          x1 |in(n) u in(m)|
 *   x2, x3 min, max of |I(n)|, |I(m)|   x4, x5 min, max of |in(n)|, |in(m)|
 *   x6, x7 min, max of w(n), w(m)
 *   h_j = relu(b1_j + sum_i W1_ji x_i) (j < 64),  s = b2 + sum_j W2_j h_j,
 *   key = floor(s * 2^key_bits) clamped to [-2^30, 2^30].
 * Weights are bfloat16 bit patterns widened exactly to float32; each sum is
 * a chain of fused multiply-adds in index order (h_j over i, then s over j,
 * folding in each h_j as it is computed), which makes the keys
 * reproducible bit for bit.  pair(n) is the valid m (the same Omega and
 * Delta checks as Sec. III-B.2) with the largest (key, hist, id); matching
 * compares (key, hist) then id.  A model whose weights are all zero gives
 * the plain order exactly.
 */
#define HGP_MLP_IN 8
#define HGP_MLP_HIDDEN 64
#define HGP_MLP_PARAMS 641         /* W1 (64 x 8), b1 (64), W2 (64), b2 */
typedef struct {
    uint16_t w1[HGP_MLP_HIDDEN * HGP_MLP_IN];   /* W1[j][i] at 8 j + i */
    uint16_t b1[HGP_MLP_HIDDEN];
    uint16_t w2[HGP_MLP_HIDDEN];
    uint16_t b2;
    int16_t key_bits;          /* 0..20 */
    int32_t reserved[3];       /* must be zero */
} hgp_model;

typedef struct {
    int32_t refine_passes;     /* refinement passes per level (default 1; 0 = none) */
    uint32_t debug;            /* HGP_DEBUG_* bits */
    int32_t max_levels;        /* > 0: stop coarsening after this many matchings, the clusters
                                  of the last one becoming the parts (as when the node target
                                  is reached); 0 = the paper's stop rule only */
    int32_t matching;          /* 0: the paper's two walks over the pairing pseudo-forest
                                  (Sec. III-B.3); 1: the exact maximum-weight matching of the
                                  same pseudo-forest (edge {n, pair(n)} weighs score(n)), by a
                                  tree DP -- the alternative the paper names as future work
                                  (Sec. III-A, VI).  Ties: a node matches its best child only
                                  for a positive gain; equal gains go to the larger id.  Plain
                                  order only (model must be NULL) */
    int32_t learned_eval;      /* with a model: 0 evaluates the network as the float32 FMA
                                  chains described above (keys reproducible bit for bit);
                                  1 evaluates its hidden layer on tensor cores (TF32 inputs,
                                  float32 accumulation, 32 candidates per warp-level MMA batch):
                                  scores agree with float32 to about 1e-3, not bit for bit */
    int32_t reserved[1];       /* must be zero */
    const hgp_model *model;    /* NULL: the paper's Eq. (2) order; else the learned order
                                  (host memory, read during the call) */
} hgp_options;

typedef struct {
    /* caller-provided outputs */
    int32_t *part_ids;         /* [num_nodes]: compacted part of every node (required) */
    int64_t *part_weight;      /* [num_nodes] or NULL: node weight of part p at [p] */
    int32_t *part_inbound;     /* [num_nodes] or NULL: |union in(n)| of part p at [p] */
    uint32_t out_flags;        /* HGP_OUTPUT_DEVICE: the three arrays are device memory */
    /* filled by hgp_partition */
    int64_t cost;              /* Eq. (1) connectivity of the result */
    int32_t num_parts;         /* parts are numbered 0..num_parts-1 */
    int32_t num_levels;        /* coarsening levels built (including level 0) */
} hgp_result;

/*
 * Partition the handle's hypergraph under node bound `omega` (>= 1) and
 * inbound-hyperedge bound `delta` (>= 0).  Parts are the non-empty clusters
 * of the final partition, renumbered 0..num_parts-1 in the order of their
 * internal ids.  The result is a pure function of (graph and its creation
 * flags, omega, delta, refine_passes, max_levels, matching, model, learned_eval).
 * Returns HGP_ERR_INFEASIBLE when some node alone has weight > omega or
 * |in(n)| > delta (then no partition exists), HGP_ERR_INVALID_ARG for bad
 * bounds/options/null part_ids.  Host outputs are complete on return; device
 * outputs are complete when `stream` reaches the end of the call.
 */
int hgp_partition(hgp_graph *g, int64_t omega, int64_t delta,
                  const hgp_options *opt, hgp_result *res);

/*
 * Partition `count` handles at once (the batched workload of many uneven
 * hypergraphs).  Instance i uses bounds omegas[i], deltas[i] and writes
 * res[i] exactly as hgp_partition(gs[i], omegas[i], deltas[i], opt, &res[i])
 * would (same options for all).  Worker threads (up to 16) run instances
 * concurrently, each on a CUDA stream of its own created for the call, so
 * the per-level kernels and host round trips of different instances overlap
 * on the device.  Handles must be distinct; their own streams are waited on
 * first.  status (optional, [count]) receives every instance's status; the
 * return value is the first non-OK status in index order, or HGP_OK.
 * Device outputs (HGP_OUTPUT_DEVICE) are complete when the call returns.
 */
int hgp_partition_batch(hgp_graph *const *gs, int32_t count, const int64_t *omegas,
                        const int64_t *deltas, const hgp_options *opt, hgp_result *res,
                        int32_t *status);

#define HGP_MAX_STAT_LEVELS 4096
typedef struct {
    int32_t num_levels;        /* levels of the last hgp_partition */
    int32_t num_parts;
    int64_t cost;
    double ms_create;          /* hgp_create wall time (host clock) */
    double ms_partition;       /* last hgp_partition wall time (host clock) */
    /* HGP_DEBUG_TIMING only (CUDA-event times, summed over levels): */
    double ms_coarsen;         /* first scoring kernel .. last contraction */
    double ms_refine;          /* refinement and projection */
    double ms_score;           /* scoring kernel (Eq. (2) + deferred checks) */
    double ms_match;           /* matching + gamma */
    double ms_contract;        /* contraction */
    int64_t score_launches;
    int64_t score_bytes;       /* algorithmic bytes of all scoring launches */
    int64_t contract_bytes;    /* HGP_DEBUG_TIMING: algorithmic bytes of all contractions
                                  (4 B per pin read, gathered and written; 4 B per I and in
                                  entry read and written; 12 B per hyperedge and node) */
    int64_t pins_total;        /* sum over built levels of the pin count */
    int64_t kernel_launches;   /* kernels launched by the last hgp_partition */
    int64_t moves_applied;     /* refinement moves applied, all levels */
    int64_t create_launches;   /* kernels launched by hgp_create */
    double ms_propose;         /* HGP_DEBUG_TIMING: Eq. (3) proposal kernel, summed */
    int64_t propose_launches;
    int64_t propose_bytes;     /* algorithmic bytes of all proposal launches */
    int64_t learned_evals;     /* HGP_DEBUG_TIMING, learned order: network evaluations (each
                                  8 lg1p features + 576 FMA + 64 ReLU) over all levels */
    double ms_contract_kernels; /* HGP_DEBUG_TIMING: device time of the contraction kernels
                                   (count and write phases, without the host read between) */
} hgp_stats;

/* Statistics of the handle's last hgp_partition (and hgp_create). */
int hgp_get_stats(const hgp_graph *g, hgp_stats *st);

/* Per-level arrays kept by HGP_DEBUG_KEEP_LEVELS (copied to host). */
enum {
    HGP_LEVEL_PAIR = 0,        /* [V_l] candidate of each node, -1 = none */
    HGP_LEVEL_SCORE = 1,       /* [V_l] hist(n, pair(n)), 0 when none */
    HGP_LEVEL_MATCH = 2,       /* [V_l] matched partner (self = single) */
    HGP_LEVEL_GAMMA = 3,       /* [V_l] coarse node of each node */
    HGP_LEVEL_RHO_IN = 4,      /* [V_l] partition entering refinement */
    HGP_LEVEL_RHO_OUT = 5,     /* [V_l] partition after refinement */
    HGP_LEVEL_WEIGHT = 6,      /* [V_l] node weights */
    HGP_LEVEL_REFINE = 7,      /* [3] proposed moves, applied prefix, gain (as int64) */
    HGP_LEVEL_KEY = 8,         /* [V_l] learned order only: key(n, pair(n)), 0 when none */
    HGP_LEVEL_GAIN_SEQ = 9     /* [M] in-sequence gain of each sorted move (last pass) */
};
/* Length of array `which` of level l (-1 if absent). */
int64_t hgp_get_level_len(const hgp_graph *g, int32_t level, int32_t which);
/* Copies array `which` of level l into host buffer out (int64 elements). */
int hgp_get_level_array(const hgp_graph *g, int32_t level, int32_t which, int64_t *out);

/*
 * The constraint-only comparison of the paper's evaluation (Sec. V): nodes in
 * id order are appended to the current part while w(part) + w(n) <= omega and
 * |in(part) u in(n)| <= delta, otherwise they open the next part.  res as
 * for hgp_partition (num_levels = 0); parts are numbered in opening order.
 * Same errors as hgp_partition.  A quality floor to compare costs with.
 */
int hgp_fill_baseline(hgp_graph *g, int64_t omega, int64_t delta, hgp_result *res);

/*
 * Training pairs for the learned order, labelled by a partition of the
 * handle's input (typically the plain method's result).  Slot
 * s = n * per_node + k (k < per_node) draws u0, u1 = outputs 2s and 2s + 1 of
 * SplitMix64 started at `seed`, takes e = the (u0 mod |I(n)|)-th hyperedge of
 * I(n) (ascending ids) and m = the (u1 mod |pins(e)|)-th pin of e in the
 * input's pin order, and stores the 8 features of (n, m) (as above) in
 * x[8 s .. 8 s + 8), the label [part_ids[n] == part_ids[m]] in y[s] and m in
 * partner[s]; when m = n or I(n) is empty the slot holds zeros, y = -1 and
 * partner = -1.  All arrays are device memory: part_ids [num_nodes], x
 * [num_nodes * per_node * 8] float, y [num_nodes * per_node] float,
 * partner [num_nodes * per_node] int32 or NULL.  Runs on the handle's
 * stream; the outputs are complete when it reaches the end of the call.
 */
int hgp_learn_samples(hgp_graph *g, const int32_t *part_ids, uint64_t seed, int32_t per_node,
                      float *x, float *y, int32_t *partner);

typedef struct {
    int32_t steps;             /* Adam steps */
    int32_t batch;             /* samples per step: step k uses samples k*batch .. k*batch +
                                  batch - 1, modulo count (labels < 0 are skipped) */
    float lr, beta1, beta2, eps;   /* Adam (Kingma and Ba, 2015) */
    int32_t first_step;        /* Adam step number t of the first step (>= 1) */
    int32_t reserved[3];       /* must be zero */
} hgp_train_options;

/*
 * Minibatch training of the learned order's network on the logistic loss
 * log(1 + e^s) - y s.  The forward pass uses the parameters rounded to
 * bfloat16 (nearest even) with float32 arithmetic; the gradient (ReLU
 * derivative 1 where the pre-activation is > 0) updates the float32 master
 * copy.  x [count * 8] and y [count] are device memory; params
 * [HGP_MLP_PARAMS] (W1 at 8 j + i, b1 at 512 + j, W2 at 576 + j, b2 at 640)
 * and adam [2 * HGP_MLP_PARAMS] (first then second moments) are host memory,
 * read and updated; loss (host, [steps] or NULL) receives each step's mean
 * batch loss before its update.  Deterministic: partial sums are added in a
 * fixed order.  Synchronous on `stream`.
 */
int hgp_train_mlp(const float *x, const float *y, int64_t count, const hgp_train_options *opt,
                  float *params, float *adam, float *loss, void *stream);

/* Model from float32 master parameters (round to nearest even bfloat16). */
int hgp_model_from_params(const float *params, int32_t key_bits, hgp_model *out);

const char *hgp_error_string(int status);
const char *hgp_last_error(const hgp_graph *g);

/* Frees the handle and all device memory it owns (after syncing its stream). */
void hgp_destroy(hgp_graph *g);

/*
 * hgp_score_noalloc -- candidate scoring of one level without any device
 * allocation.  (The paper has no counterpart: this exists for callers that
 * cannot allocate device memory while they run -- code inside another
 * framework's memory pool or allocator callback, runtimes that reserved all
 * device memory up front, or steps that must not incur the implicit
 * synchronisation of cudaMalloc/cudaFree.)
 *
 * Computes, for every node n, the same pair(n) and score(n) that
 * hgp_partition computes at its first level (HGP_LEVEL_PAIR / HGP_LEVEL_SCORE
 * of level 0): the first neighbour m in (hist desc, id desc) order with
 * w(n) + w(m) <= omega and |in(n) u in(m)| <= delta, -1 and 0 if none.
 * All pointers are device memory, readable/writable on `stream`:
 *   offsets[E+1], pins[P]          pins of every hyperedge
 *   inc_offsets[N+1], inc[P]       I(n), the hyperedges containing n
 *   in_offsets[N+1], in_edges[Q]   in(n), ascending edge ids
 *   node_weights[N], edge_weights[E] (both required, >= 1)
 *   pair[N], score[N]              outputs
 * Inputs are not validated beyond null pointers and sizes; they must satisfy
 * the rules of hgp_create.
 * Scratch: one library-owned 16 MiB device array per GPU (allocated when the
 * library is loaded, held until the process exits).  The in() bitmaps need
 * N * 4 * ceil(E / 128) * 16 bytes whenever 2 * max |in(n)| > delta; larger
 * inputs, or N too large for the shared-memory histogram (about 54,000
 * nodes), return HGP_ERR_SCRATCH_LIMIT without launching anything.  The call
 * clears the part of the array it uses, so the previous call's contents do not
 * matter; but every call on a device shares the array, so calls whose work
 * overlaps on the GPU (e.g. on two streams) race -- serialise them.
 * The first call on each device looks up the array's device address with
 * cudaGetSymbolAddress (with that device current); make that first call
 * before any stream capture.  The call synchronises `stream` once (to read
 * the largest |in(n)|).  Returns HGP_OK, HGP_ERR_INVALID_ARG,
 * HGP_ERR_SCRATCH_LIMIT or HGP_ERR_CUDA.
 */
int hgp_score_noalloc(int32_t num_nodes, int32_t num_edges,
                      const int32_t *offsets, const int32_t *pins,
                      const int32_t *inc_offsets, const int32_t *inc,
                      const int32_t *in_offsets, const int32_t *in_edges,
                      const int32_t *node_weights, const int32_t *edge_weights,
                      int64_t omega, int64_t delta,
                      int32_t *pair, int32_t *score, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* HGP_H */
