// C ABI of the library (include/hgp.h): handle lifetime, the level loop of
// Sec. II-B (coarsen until ceil(W / Omega) nodes or no merge, then refine
// from the coarsest level down while projecting), and result delivery.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <thread>
#include <string>
#include <vector>

#include "hgp_internal.cuh"

namespace hgp {
cudaError_t run_score(Arena &ar, Arena &roll, Level &L, const Level *prev, const int32_t *ew,
                      int64_t omega, int64_t delta, int32_t *pair, int32_t *score, int32_t *status,
                      unsigned long long *bytes, uint32_t debug, int64_t bm_budget, cudaStream_t s);
int64_t bitmap_budget();
cudaError_t run_score_learned(Arena &ar, const Level &L, const int32_t *ew, int64_t omega,
                              int64_t delta, const hgp_model *model, int32_t *pair,
                              int32_t *score, int32_t *key, int32_t *status,
                              unsigned long long *bytes, unsigned long long *evals,
                              uint32_t debug, int32_t tensor_cores, cudaStream_t s);
bool model_valid(const hgp_model *m);
cudaError_t run_learn_samples(const Level &L0, const int32_t *ew, const int32_t *part_ids,
                              uint64_t seed, int32_t per_node, float *x, float *y,
                              int32_t *partner, cudaStream_t s);
cudaError_t run_fill_baseline(Arena &ar, const Level &L0, int64_t omega, int64_t delta,
                              int32_t *part, int32_t *d_nparts, cudaStream_t s);
cudaError_t run_match(Arena &ar, int32_t V, const int32_t *pair, const int32_t *score,
                      const int32_t *key, int32_t *match, int32_t *gamma, int32_t *d_V2,
                      int32_t *status, cudaStream_t s, bool exact);
cudaError_t run_contract(Arena &keep, Arena &inc_ar, Arena &roll, Arena &tmp, const Level &L,
                         int32_t V2, Level &H, const int32_t *pair, const int32_t *score,
                         int32_t *status, cudaStream_t s, PropTiming *kt);
cudaError_t run_rebuild_incidence(Arena &ar, const Level &L, int32_t **ioff, int32_t **inc,
                                  cudaStream_t s);
int run_build_level0(Arena &keep, Arena &tmp, int32_t N, int32_t E, Level &L, const int32_t *ew,
                     int32_t delta_mode, int64_t *wsum_e, cudaError_t *cerr, std::string *why,
                     cudaStream_t s);
cudaError_t run_refine_pass(Arena &tmp, const Level &L, const int32_t *ew, int64_t wsum,
                            int32_t *rho, int32_t K, int64_t omega, int64_t delta,
                            long long *d_stats, unsigned long long *d_applied, uint32_t debug,
                            PropTiming *pt, const PropReuse &ru, std::vector<int32_t> *gseq_out,
                            cudaStream_t s);
void run_project(int32_t V, const int32_t *gamma, const int32_t *rho_c, int32_t *rho_f,
                 cudaStream_t s);
cudaError_t run_finalize(Arena &tmp, const Level &L, const int32_t *ew, const int32_t *rho,
                         int32_t K, int32_t *part_ids, int64_t *pw, int32_t *pin,
                         unsigned long long *d_cost, int32_t *d_nparts, cudaStream_t s);

__global__ void k_node_maxima(int32_t N, const int32_t *w, const int32_t *noff, int32_t E,
                              const int32_t *poff, int32_t *out) {
    int32_t mw = 0, mi = 0, me = 0;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N;
         n += (int64_t)gridDim.x * blockDim.x) {
        mw = max(mw, w[n]);
        mi = max(mi, noff[n + 1] - noff[n]);
    }
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
         e += (int64_t)gridDim.x * blockDim.x)
        me = max(me, poff[e + 1] - poff[e]);
    atomicMax(&out[0], mw);
    atomicMax(&out[1], mi);
    atomicMax(&out[2], me);
}

__global__ void k_fill_one(int32_t *p, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = 1;
}
}  // namespace hgp

using namespace hgp;

struct hgp_graph {
    cudaStream_t stream = nullptr;
    hgp_allocator allocator{};
    bool has_allocator = false;
    Arena keep;
    Level L0;
    int32_t *ew = nullptr;
    int32_t N = 0, E = 0;
    int64_t W = 0;
    int64_t wsum_e = 0;          // total edge weight (bounds every gain)
    int32_t max_w = 0, max_in = 0;
    std::string err;
    hgp_stats stats{};
    std::vector<std::vector<int64_t>> dbg[10];
    const hgp_allocator *user_allocator() const { return has_allocator ? &allocator : nullptr; }
};

static int fail(hgp_graph *g, int code, const std::string &msg) {
    if (g) g->err = msg;
    return code;
}

static int cuda_fail(hgp_graph *g, cudaError_t e, const char *where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    cudaGetLastError();   // clear a sticky launch error state where possible
    if (e == cudaErrorMemoryAllocation) return fail(g, HGP_ERR_OOM, m);
    return fail(g, HGP_ERR_CUDA, m);
}

#define CK(expr, where)                                   \
    do {                                                  \
        cudaError_t _e = (expr);                          \
        if (_e != cudaSuccess) return cuda_fail(g, _e, where); \
    } while (0)

static double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

static thread_local std::string t_create_err;

extern "C" int hgp_create(int32_t num_nodes, int32_t num_edges, const int32_t *offsets,
                          const int32_t *pins, const int32_t *node_weights,
                          const int32_t *edge_weights, uint32_t flags,
                          const hgp_allocator *alloc, void *stream, hgp_graph **out) {
    if (!out) return HGP_ERR_INVALID_ARG;
    *out = nullptr;
    if (num_nodes < 1 || num_edges < 0 || !offsets || (num_edges > 0 && !pins))
        return HGP_ERR_INVALID_ARG;
    if (alloc && (!alloc->alloc || !alloc->free)) return HGP_ERR_INVALID_ARG;
    if ((flags & ~(HGP_INPUT_DEVICE | HGP_DELTA_INCIDENT | HGP_DELTA_OUTBOUND)) != 0)
        return HGP_ERR_INVALID_ARG;
    if ((flags & HGP_DELTA_INCIDENT) && (flags & HGP_DELTA_OUTBOUND)) return HGP_ERR_INVALID_ARG;
    double t0 = now_ms();
    int64_t launches0 = g_launches;
    hgp_graph *g = new (std::nothrow) hgp_graph();
    if (!g) return HGP_ERR_OOM;
    g->stream = (cudaStream_t)stream;
    if (alloc) {
        g->allocator = *alloc;
        g->has_allocator = true;
    }
    g->keep.stream = g->stream;
    g->keep.user = g->user_allocator();
    g->N = num_nodes;
    g->E = num_edges;
    cudaStream_t s = g->stream;
    bool dev = (flags & HGP_INPUT_DEVICE) != 0;
    cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    Level &L = g->L0;
    L.V = num_nodes;
    L.E = num_edges;
    Arena tmp;
    tmp.stream = s;
    tmp.user = g->user_allocator();
    auto bail = [&](int code) {
        cudaStreamSynchronize(s);
        tmp.release_all();
        g->keep.release_all();
        cudaStreamSynchronize(s);
        t_create_err = g->err;
        delete g;
        return code;
    };
#define CKC(expr, where)                                             \
    do {                                                             \
        cudaError_t _e = (expr);                                     \
        if (_e != cudaSuccess) return bail(cuda_fail(g, _e, where)); \
    } while (0)
    CKC(dalloc(g->keep, &L.poff, (size_t)num_edges + 1), "alloc offsets");
    CKC(cudaMemcpyAsync(L.poff, offsets, sizeof(int32_t) * ((size_t)num_edges + 1), kind, s),
        "copy offsets");
    int32_t P = 0;
    if (dev) {
        CKC(cudaMemcpyAsync(&P, L.poff + num_edges, sizeof(int32_t), cudaMemcpyDeviceToHost, s),
            "read pin count");
        CKC(cudaStreamSynchronize(s), "sync");
    } else {
        P = offsets[num_edges];
    }
    if (P < 0 || (num_edges > 0 && P < num_edges)) {
        g->err = "offsets[num_edges] must be the pin count (>= one pin per edge)";
        return bail(HGP_ERR_INVALID_ARG);
    }
    CKC(dalloc(g->keep, &L.pins, P), "alloc pins");
    if (P > 0)
        CKC(cudaMemcpyAsync(L.pins, pins, sizeof(int32_t) * (size_t)P, kind, s), "copy pins");
    CKC(dalloc(g->keep, &L.w, num_nodes), "alloc node weights");
    CKC(dalloc(g->keep, &g->ew, num_edges), "alloc edge weights");
    if (node_weights)
        CKC(cudaMemcpyAsync(L.w, node_weights, sizeof(int32_t) * (size_t)num_nodes, kind, s),
            "copy node weights");
    else
        fill_i32(L.w, 1, num_nodes, s);
    if (num_edges > 0) {
        if (edge_weights)
            CKC(cudaMemcpyAsync(g->ew, edge_weights, sizeof(int32_t) * (size_t)num_edges, kind, s),
                "copy edge weights");
        else
            fill_i32(g->ew, 1, num_edges, s);
    }
    cudaError_t ce = cudaSuccess;
    std::string why;
    const int32_t delta_mode = (flags & HGP_DELTA_INCIDENT) ? 1 : (flags & HGP_DELTA_OUTBOUND) ? 2 : 0;
    int rc = run_build_level0(g->keep, tmp, num_nodes, num_edges, L, g->ew, delta_mode, &g->wsum_e,
                              &ce, &why, s);
    if (rc != 0) {
        tmp.release_all();
        if (rc < 0) return bail(cuda_fail(g, ce, "build level 0"));
        g->err = why;
        return bail(HGP_ERR_INVALID_ARG);
    }
    // node maxima and total weight for the singleton check and the stop rule
    int32_t *mx = nullptr;
    CKC(dalloc(tmp, &mx, 3), "alloc");
    CKC(cudaMemsetAsync(mx, 0, sizeof(int32_t) * 3, s), "memset");
    k_node_maxima<<<num_sms() * 4, 256, 0, s>>>(num_nodes, L.w, L.noff, num_edges, L.poff, mx);
    count_launch();
    int32_t hmx[3];
    CKC(cudaMemcpyAsync(hmx, mx, sizeof(hmx), cudaMemcpyDeviceToHost, s), "read maxima");
    std::vector<int32_t> hw;
    if (node_weights) {
        hw.resize(num_nodes);
        CKC(cudaMemcpyAsync(hw.data(), L.w, sizeof(int32_t) * (size_t)num_nodes,
                            cudaMemcpyDeviceToHost, s), "read weights");
    }
    CKC(cudaStreamSynchronize(s), "sync");
    tmp.release_all();
    g->max_w = hmx[0];
    g->max_in = hmx[1];
    L.max_in = hmx[1];
    L.max_edge = hmx[2];
    int64_t W = 0;
    if (node_weights) for (int32_t x : hw) W += x;
    else W = num_nodes;
    g->W = W;
    CKC(cudaStreamSynchronize(s), "sync");
#undef CKC
    g->stats.ms_create = now_ms() - t0;
    g->stats.create_launches = g_launches - launches0;
    *out = g;
    return HGP_OK;
}

namespace {
struct Timer {
    bool on = false;
    cudaStream_t s = nullptr;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[4];   // score, match, contract, refine
    void start(int k, cudaEvent_t *a) {
        if (!on) return;
        cudaEventCreate(a);
        cudaEventRecord(*a, s);
        (void)k;
    }
    void stop(int k, cudaEvent_t a) {
        if (!on) return;
        cudaEvent_t b;
        cudaEventCreate(&b);
        cudaEventRecord(b, s);
        ev[k].push_back({a, b});
    }
    double total(int k) {
        double t = 0;
        for (auto &p : ev[k]) {
            float ms = 0;
            cudaEventSynchronize(p.second);
            cudaEventElapsedTime(&ms, p.first, p.second);
            t += ms;
        }
        return t;
    }
    ~Timer() {
        for (auto &v : ev)
            for (auto &p : v) { cudaEventDestroy(p.first); cudaEventDestroy(p.second); }
    }
};

void keep_array(hgp_graph *g, int which, int level, const int32_t *d, int64_t n, cudaStream_t s) {
    auto &vv = g->dbg[which];
    if ((int)vv.size() <= level) vv.resize(level + 1);
    std::vector<int32_t> h(n > 0 ? n : 0);
    if (n > 0) {
        cudaMemcpyAsync(h.data(), d, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
    }
    vv[level].assign(h.begin(), h.end());
}
}  // namespace

// hgp_partition on an explicit stream (the batch entry point runs several
// handles concurrently, each on a stream of its own).
static int partition_on(hgp_graph *g, int64_t omega, int64_t delta, const hgp_options *opt,
                        hgp_result *res, cudaStream_t s) {
    if (!g || !res) return HGP_ERR_INVALID_ARG;
    if (omega < 1 || delta < 0) return fail(g, HGP_ERR_INVALID_ARG, "omega must be >= 1 and delta >= 0");
    if (!res->part_ids) return fail(g, HGP_ERR_INVALID_ARG, "part_ids is required");
    int32_t passes = 1;
    uint32_t debug = 0;
    int32_t max_levels = 0, matching = 0, learned_eval = 0;
    const hgp_model *model = nullptr;
    if (opt) {
        if (opt->refine_passes < 0) return fail(g, HGP_ERR_INVALID_ARG, "refine_passes must be >= 0");
        if (opt->reserved[0]) return fail(g, HGP_ERR_INVALID_ARG, "reserved options must be zero");
        if (opt->learned_eval < 0 || opt->learned_eval > 1 || (opt->learned_eval && !opt->model))
            return fail(g, HGP_ERR_INVALID_ARG, "learned_eval must be 0, or 1 with a model");
        learned_eval = opt->learned_eval;
        if (opt->matching < 0 || opt->matching > 1 || (opt->matching == 1 && opt->model))
            return fail(g, HGP_ERR_INVALID_ARG,
                        "matching must be 0 (two walks) or 1 (exact, plain order only)");
        matching = opt->matching;
        if (opt->model && !model_valid(opt->model))
            return fail(g, HGP_ERR_INVALID_ARG, "model: key_bits must be in 0..20 and reserved zero");
        if (opt->max_levels < 0) return fail(g, HGP_ERR_INVALID_ARG, "max_levels must be >= 0");
        max_levels = opt->max_levels;
        if (opt->debug & ~(uint32_t)(HGP_DEBUG_KEEP_LEVELS | HGP_DEBUG_TIMING | HGP_DEBUG_FORCE_GLOBAL |
                                     HGP_DEBUG_NO_BITMAP | HGP_DEBUG_FORCE_CLUSTER |
                                     HGP_DEBUG_SMALL_TABLE | HGP_DEBUG_REBUILD_INC |
                                     HGP_DEBUG_FORCE_WINDOW | HGP_DEBUG_FORCE_HASH_BUCKET))
            return fail(g, HGP_ERR_INVALID_ARG, "unknown debug bits");
        passes = opt->refine_passes;
        debug = opt->debug;
        model = opt->model;
    }
    if (g->max_w > omega || g->max_in > delta)
        return fail(g, HGP_ERR_INFEASIBLE, "a single node exceeds omega or delta; no partition exists");
    double t0 = now_ms();
    int64_t launches0 = g_launches;
    // Storage of the hierarchy:
    //   lv       what refinement reads at every level (weights, pins, sources,
    //            gamma, match) and I(n) while it fits the budget below
    //   roll[2]  in(n) and the carried scoring state (and I(n) past the
    //            budget): level l's live in roll[l & 1] and die when level
    //            l + 2 is built, so only two levels of them exist at a time
    //   rb       I(n) rebuilt from the pins when refinement reaches a level
    //            whose copy was not kept
    Arena lv, tmp, roll[2], rb;
    for (Arena *a : {&lv, &tmp, &roll[0], &roll[1], &rb}) {
        a->stream = s;
        a->user = g->user_allocator();
        a->min_chunk = (size_t)64 << 20;
    }
    size_t inc_budget = 0, inc_kept = 0;
    const int64_t bm_budget = model ? 0 : bitmap_budget();     // in() bitmaps per level
    if (!(debug & HGP_DEBUG_REBUILD_INC)) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) inc_budget = fr / 10 * 4;   // 40 % of free
    }
    Timer tm;
    tm.on = (debug & HGP_DEBUG_TIMING) != 0;
    tm.s = s;
    PropTiming ctime;                  // contraction kernels (timing runs)
    PropTiming ptime;                  // proposal kernels (timing runs)
    auto drop_events = [&]() {
        for (PropTiming *t : {&ptime, &ctime}) {
            for (auto &pr : t->ev) {
                if (pr.first) cudaEventDestroy(pr.first);
                if (pr.second) cudaEventDestroy(pr.second);
            }
            t->ev.clear();
        }
    };
    if (debug & HGP_DEBUG_KEEP_LEVELS)
        for (auto &v : g->dbg) v.clear();
    auto cleanup = [&]() {
        cudaStreamSynchronize(s);
        for (Arena *a : {&tmp, &lv, &roll[0], &roll[1], &rb}) a->release_all();
        cudaStreamSynchronize(s);
        drop_events();
    };
#define CKP(expr, where)                                        \
    do {                                                        \
        cudaError_t _e = (expr);                                \
        if (_e != cudaSuccess) { int _r = cuda_fail(g, _e, where); cleanup(); return _r; } \
    } while (0)

    int32_t *d_status = nullptr, *d_V2 = nullptr;
    unsigned long long *d_bytes = nullptr;
    CKP(dalloc(lv, &d_status, 1), "alloc");
    CKP(dalloc(lv, &d_V2, 1), "alloc");
    CKP(dalloc(lv, &d_bytes, 2), "alloc");          // [0] scoring bytes, [1] network evaluations
    CKP(cudaMemsetAsync(d_status, 0, sizeof(int32_t), s), "memset");
    CKP(cudaMemsetAsync(d_bytes, 0, 2 * sizeof(unsigned long long), s), "memset");

    int64_t target = g->W / omega + (g->W % omega != 0);
    std::vector<Level> levels;
    levels.push_back(g->L0);
    levels[0].gamma = nullptr;
    levels[0].match = nullptr;
    int32_t K = 0;
    bool top_gamma = false;
    int64_t pins_total = g->L0.P;
    cudaEvent_t ev_a;
    double c0 = now_ms();
    if ((int64_t)g->L0.V <= target) {
        K = g->L0.V;
    } else {
        for (;;) {
            Level &L = levels.back();
            int l = (int)levels.size() - 1;
            int32_t *pair, *score, *key = nullptr;
            CKP(dalloc(tmp, &pair, L.V), "alloc pair");
            CKP(dalloc(tmp, &score, L.V), "alloc score");
            if (model) CKP(dalloc(tmp, &key, L.V), "alloc key");
            CKP(dalloc(lv, &L.match, L.V), "alloc match");
            CKP(dalloc(lv, &L.gamma, L.V), "alloc gamma");
            tm.start(0, &ev_a);
            if (model)
                CKP(run_score_learned(tmp, L, g->ew, omega, delta, model, pair, score, key, d_status,
                                      tm.on ? d_bytes : nullptr, tm.on ? d_bytes + 1 : nullptr,
                                      debug, learned_eval, s), "score");
            else
                CKP(run_score(tmp, roll[l & 1], L, l > 0 ? &levels[l - 1] : nullptr, g->ew, omega,
                              delta, pair, score, d_status, tm.on ? d_bytes : nullptr, debug,
                              bm_budget, s), "score");
            tm.stop(0, ev_a);
            tm.start(1, &ev_a);
            CKP(run_match(tmp, L.V, pair, score, key, L.match, L.gamma, d_V2, d_status, s,
                          matching == 1), "match");
            tm.stop(1, ev_a);
            int32_t h[2];
            CKP(cudaMemcpyAsync(&h[0], d_V2, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "read V2");
            CKP(cudaMemcpyAsync(&h[1], d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "read status");
            CKP(cudaStreamSynchronize(s), "sync");
            if (h[1] != 0) {
                cleanup();
                return fail(g, h[1] == kDevLimit ? HGP_ERR_DEVICE_LIMIT : HGP_ERR_CUDA,
                            "device status " + std::to_string(h[1]) + " during coarsening");
            }
            if (debug & HGP_DEBUG_KEEP_LEVELS) {
                keep_array(g, HGP_LEVEL_PAIR, l, pair, L.V, s);
                keep_array(g, HGP_LEVEL_SCORE, l, score, L.V, s);
                if (key) keep_array(g, HGP_LEVEL_KEY, l, key, L.V, s);
                keep_array(g, HGP_LEVEL_MATCH, l, L.match, L.V, s);
                keep_array(g, HGP_LEVEL_WEIGHT, l, L.w, L.V, s);
            }
            int32_t V2 = h[0];
            if (V2 == L.V) {            // no cluster can be unified
                K = L.V;
                break;
            }
            if (debug & HGP_DEBUG_KEEP_LEVELS) keep_array(g, HGP_LEVEL_GAMMA, l, L.gamma, L.V, s);
            if ((int64_t)V2 <= target ||              // coarsest clusters become the parts
                (max_levels > 0 && (int)levels.size() >= max_levels)) {
                K = V2;
                top_gamma = true;
                break;
            }
            Level H;
            // level l + 1's in(n) and scoring state reuse the storage of
            // level l - 1's, which nothing reads any more
            Arena &ra = roll[(l + 1) & 1];
            ra.reset();
            if (l >= 1) {
                Level &O = levels[l - 1];
                O.noff = O.inn = nullptr;
                O.dead = O.merged = nullptr;
                O.thr = nullptr;
                O.old_id = nullptr;
                O.bm = nullptr;
                if (O.inc_rolling) O.ioff = O.inc = nullptr;
            }
            const size_t inc_bytes = 4 * ((size_t)L.P + (size_t)L.V + 1) + 512;   // H.P <= L.P
            const bool keep_inc = inc_kept + inc_bytes <= inc_budget;
            if (keep_inc) inc_kept += inc_bytes;
            tm.start(2, &ev_a);
            CKP(run_contract(lv, keep_inc ? lv : ra, ra, tmp, L, V2, H, pair, score, d_status, s,
                             tm.on ? &ctime : nullptr), "contract");
            tm.stop(2, ev_a);
            H.inc_rolling = !keep_inc;
            levels.push_back(H);
            pins_total += H.P;
            tmp.reset();               // stream order keeps the reuse safe
        }
    }
    double c1 = now_ms();
    int L = (int)levels.size() - 1;
    if (debug & HGP_DEBUG_KEEP_LEVELS) keep_array(g, HGP_LEVEL_WEIGHT, L, levels[L].w, levels[L].V, s);
    // initial partition of the coarsest level
    int32_t *rho = nullptr;
    CKP(dalloc(lv, &rho, levels[L].V), "alloc rho");
    if (top_gamma)
        CKP(cudaMemcpyAsync(rho, levels[L].gamma, sizeof(int32_t) * (size_t)levels[L].V,
                            cudaMemcpyDeviceToDevice, s), "copy gamma");
    else
        iota_i32(rho, levels[L].V, s);
    long long *d_rstat = nullptr;
    unsigned long long *d_applied = nullptr;
    CKP(dalloc(lv, &ptime.bytes, 1), "alloc");
    CKP(cudaMemsetAsync(ptime.bytes, 0, sizeof(unsigned long long), s), "memset");
    CKP(dalloc(lv, &d_rstat, 3 * levels.size()), "alloc");
    CKP(dalloc(lv, &d_applied, 1), "alloc");
    CKP(cudaMemsetAsync(d_rstat, 0, sizeof(long long) * 3 * levels.size(), s), "memset");
    CKP(cudaMemsetAsync(d_applied, 0, sizeof(unsigned long long), s), "memset");
    tm.start(3, &ev_a);
    // proposal buffers, alternating between levels so the coarser level's stay readable
    int32_t *pbuf[2][2];
    int32_t *d_flag = nullptr;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) CKP(dalloc(lv, &pbuf[i][j], g->L0.V), "alloc");
    CKP(dalloc(lv, &d_flag, 1), "alloc");
    CKP(cudaMemsetAsync(d_flag, 0, sizeof(int32_t), s), "memset");
    for (int l = L; l >= 0; --l) {
        Level &Lv = levels[l];
        if (!Lv.inc) {                // I(n) was not kept: rebuild it from the pins
            rb.reset();
            CKP(run_rebuild_incidence(rb, Lv, &Lv.ioff, &Lv.inc, s), "rebuild incidence");
        }
        if (debug & HGP_DEBUG_KEEP_LEVELS) keep_array(g, HGP_LEVEL_RHO_IN, l, rho, Lv.V, s);
        for (int p = 0; p < passes; ++p) {
            PropReuse ru;
            int cur = l & 1;
            ru.out_gain = pbuf[cur][0];
            ru.out_pd = pbuf[cur][1];
            ru.applied_flag = d_flag;
            if (p == 0 && l < L && passes > 0) {      // the coarser level's last pass is available
                ru.prev_gain = pbuf[cur ^ 1][0];
                ru.prev_pd = pbuf[cur ^ 1][1];
                ru.gamma = Lv.gamma;
                ru.match = Lv.match;
            }
            std::vector<int32_t> gs;
            const bool keep_gs = (debug & HGP_DEBUG_KEEP_LEVELS) && p == passes - 1;
            CKP(run_refine_pass(tmp, Lv, g->ew, g->wsum_e, rho, K, omega, delta, d_rstat + 3 * l,
                                d_applied, debug, tm.on ? &ptime : nullptr, ru,
                                keep_gs ? &gs : nullptr, s), "refine");
            if (keep_gs) {
                auto &vv = g->dbg[HGP_LEVEL_GAIN_SEQ];
                if ((int)vv.size() <= l) vv.resize(l + 1);
                vv[l].assign(gs.begin(), gs.end());
            }
            tmp.reset();
        }
        if (debug & HGP_DEBUG_KEEP_LEVELS) {
            keep_array(g, HGP_LEVEL_RHO_OUT, l, rho, Lv.V, s);
            long long st3[3];
            CKP(cudaMemcpyAsync(st3, d_rstat + 3 * l, sizeof(st3), cudaMemcpyDeviceToHost, s), "stats");
            CKP(cudaStreamSynchronize(s), "sync");
            auto &vv = g->dbg[HGP_LEVEL_REFINE];
            if ((int)vv.size() <= l) vv.resize(l + 1);
            vv[l] = {st3[0], st3[1], st3[2]};
        }
        if (l > 0) {
            int32_t *rf = nullptr;
            CKP(dalloc(lv, &rf, levels[l - 1].V), "alloc rho");
            run_project(levels[l - 1].V, levels[l - 1].gamma, rho, rf, s);
            rho = rf;
        }
    }
    tm.stop(3, ev_a);
    // result
    bool outdev = (res->out_flags & HGP_OUTPUT_DEVICE) != 0;
    int32_t N = g->N;
    int32_t *d_ids = outdev ? res->part_ids : nullptr;
    int64_t *d_pw = outdev ? res->part_weight : nullptr;
    int32_t *d_pin = outdev ? res->part_inbound : nullptr;
    if (!outdev) {
        CKP(dalloc(tmp, &d_ids, N), "alloc out");
        if (res->part_weight) CKP(dalloc(tmp, &d_pw, N), "alloc out");
        if (res->part_inbound) CKP(dalloc(tmp, &d_pin, N), "alloc out");
    }
    unsigned long long *d_cost = nullptr;
    int32_t *d_np = nullptr;
    CKP(dalloc(tmp, &d_cost, 1), "alloc");
    CKP(dalloc(tmp, &d_np, 1), "alloc");
    CKP(run_finalize(tmp, g->L0, g->ew, rho, K, d_ids, d_pw, d_pin, d_cost, d_np, s), "finalize");
    unsigned long long cost = 0, applied = 0;
    int32_t np = 0;
    CKP(cudaMemcpyAsync(&applied, d_applied, sizeof(applied), cudaMemcpyDeviceToHost, s), "read stats");
    CKP(cudaMemcpyAsync(&cost, d_cost, sizeof(cost), cudaMemcpyDeviceToHost, s), "read cost");
    CKP(cudaMemcpyAsync(&np, d_np, sizeof(np), cudaMemcpyDeviceToHost, s), "read parts");
    if (!outdev) {
        CKP(cudaMemcpyAsync(res->part_ids, d_ids, sizeof(int32_t) * (size_t)N,
                            cudaMemcpyDeviceToHost, s), "copy part ids");
        CKP(cudaStreamSynchronize(s), "sync");
        if (res->part_weight)
            CKP(cudaMemcpyAsync(res->part_weight, d_pw, sizeof(int64_t) * (size_t)np,
                                cudaMemcpyDeviceToHost, s), "copy part weights");
        if (res->part_inbound)
            CKP(cudaMemcpyAsync(res->part_inbound, d_pin, sizeof(int32_t) * (size_t)np,
                                cudaMemcpyDeviceToHost, s), "copy part inbound");
    }
    CKP(cudaStreamSynchronize(s), "sync");
    res->cost = (int64_t)cost;
    res->num_parts = np;
    res->num_levels = (int32_t)levels.size();
    hgp_stats &st = g->stats;
    double ms_create = st.ms_create;
    int64_t create_launches = st.create_launches;
    std::memset(&st, 0, sizeof(st));
    st.ms_create = ms_create;
    st.create_launches = create_launches;
    st.num_levels = res->num_levels;
    st.num_parts = np;
    st.cost = res->cost;
    st.pins_total = pins_total;
    st.moves_applied = (int64_t)applied;
    if (tm.on) {
        st.ms_score = tm.total(0);
        st.ms_match = tm.total(1);
        st.ms_contract = tm.total(2);
        st.ms_refine = tm.total(3);
        st.ms_coarsen = st.ms_score + st.ms_match + st.ms_contract;
        st.score_launches = (int64_t)tm.ev[0].size();
        unsigned long long b = 0;
        cudaMemcpy(&b, d_bytes, sizeof(b), cudaMemcpyDeviceToHost);
        st.score_bytes = (int64_t)b;
        unsigned long long ev = 0;
        cudaMemcpy(&ev, d_bytes + 1, sizeof(ev), cudaMemcpyDeviceToHost);
        st.learned_evals = (int64_t)ev;
        double tp = 0;
        for (auto &pr : ptime.ev) {
            float ms = 0;
            cudaEventSynchronize(pr.second);
            cudaEventElapsedTime(&ms, pr.first, pr.second);
            tp += ms;
        }
        st.ms_propose = tp;
        st.propose_launches = (int64_t)ptime.ev.size();
        unsigned long long pb = 0;
        cudaMemcpy(&pb, ptime.bytes, sizeof(pb), cudaMemcpyDeviceToHost);
        st.propose_bytes = (int64_t)pb;
        double tc = 0;
        for (auto &pr : ctime.ev) {
            float ms = 0;
            cudaEventSynchronize(pr.second);
            cudaEventElapsedTime(&ms, pr.first, pr.second);
            tc += ms;
        }
        st.ms_contract_kernels = tc;
        st.contract_bytes = (int64_t)ctime.host_bytes;
    }
    (void)c0; (void)c1;
    st.kernel_launches = g_launches - launches0;
    cleanup();
    st.ms_partition = now_ms() - t0;
    return HGP_OK;
#undef CKP
}

extern "C" int hgp_partition(hgp_graph *g, int64_t omega, int64_t delta, const hgp_options *opt,
                             hgp_result *res) {
    if (!g) return HGP_ERR_INVALID_ARG;
    return partition_on(g, omega, delta, opt, res, g->stream);
}

// The paper's constraint-only comparison: parts filled in node-id order.
extern "C" int hgp_fill_baseline(hgp_graph *g, int64_t omega, int64_t delta, hgp_result *res) {
    if (!g || !res) return HGP_ERR_INVALID_ARG;
    if (omega < 1 || delta < 0) return fail(g, HGP_ERR_INVALID_ARG, "omega must be >= 1 and delta >= 0");
    if (!res->part_ids) return fail(g, HGP_ERR_INVALID_ARG, "part_ids is required");
    if (g->max_w > omega || g->max_in > delta)
        return fail(g, HGP_ERR_INFEASIBLE, "a single node exceeds omega or delta; no partition exists");
    cudaStream_t s = g->stream;
    Arena tmp;
    tmp.stream = s;
    tmp.user = g->user_allocator();
    auto done = [&](cudaError_t e, const char *where) {
        cudaStreamSynchronize(s);
        tmp.release_all();
        cudaStreamSynchronize(s);
        return e ? cuda_fail(g, e, where) : HGP_OK;
    };
    const bool outdev = (res->out_flags & HGP_OUTPUT_DEVICE) != 0;
    const int32_t N = g->N;
    int32_t *rho = nullptr, *d_np = nullptr, *d_ids = outdev ? res->part_ids : nullptr;
    int64_t *d_pw = outdev ? res->part_weight : nullptr;
    int32_t *d_pin = outdev ? res->part_inbound : nullptr;
    unsigned long long *d_cost = nullptr;
    cudaError_t e = dalloc(tmp, &rho, N);
    if (!e) e = dalloc(tmp, &d_np, 2);
    if (!e) e = dalloc(tmp, &d_cost, 1);
    if (!e && !outdev) e = dalloc(tmp, &d_ids, N);
    if (!e && !outdev && res->part_weight) e = dalloc(tmp, &d_pw, N);
    if (!e && !outdev && res->part_inbound) e = dalloc(tmp, &d_pin, N);
    if (!e) e = run_fill_baseline(tmp, g->L0, omega, delta, rho, d_np, s);
    int32_t K = 0;
    if (!e) e = cudaMemcpyAsync(&K, d_np, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (!e) e = run_finalize(tmp, g->L0, g->ew, rho, K > 0 ? K : 1, d_ids, d_pw, d_pin, d_cost, d_np + 1, s);
    unsigned long long cost = 0;
    int32_t np = 0;
    if (!e) e = cudaMemcpyAsync(&cost, d_cost, sizeof(cost), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(&np, d_np + 1, sizeof(np), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (!e && !outdev) {
        e = cudaMemcpyAsync(res->part_ids, d_ids, sizeof(int32_t) * (size_t)N, cudaMemcpyDeviceToHost, s);
        if (!e && res->part_weight)
            e = cudaMemcpyAsync(res->part_weight, d_pw, sizeof(int64_t) * (size_t)np, cudaMemcpyDeviceToHost, s);
        if (!e && res->part_inbound)
            e = cudaMemcpyAsync(res->part_inbound, d_pin, sizeof(int32_t) * (size_t)np, cudaMemcpyDeviceToHost, s);
    }
    res->cost = (int64_t)cost;
    res->num_parts = np;
    res->num_levels = 0;
    return done(e, "fill baseline");
}

// Many handles at once: worker threads take instances from a shared counter
// and run each on a stream of their own, so the small per-level kernels and
// host round trips of different instances overlap on the GPU.  Every
// instance's result is exactly its hgp_partition result.
extern "C" int hgp_partition_batch(hgp_graph *const *gs, int32_t count, const int64_t *omegas,
                                   const int64_t *deltas, const hgp_options *opt,
                                   hgp_result *res, int32_t *status) {
    if (count < 0 || (count > 0 && (!gs || !omegas || !deltas || !res))) return HGP_ERR_INVALID_ARG;
    for (int32_t i = 0; i < count; ++i)
        if (!gs[i]) return HGP_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HGP_ERR_CUDA;
    // Instances are taken in index order.  (Largest-first ordering was tried:
    // it starts the biggest instances together, and their per-level storage
    // exhausted device memory on the 64-instance workload.)
    int workers = count < 16 ? count : 16;
    std::atomic<int32_t> next(0);
    std::vector<int> rc(count > 0 ? count : 1, HGP_OK);
    auto work = [&]() {
        cudaSetDevice(dev);
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) s = nullptr;
        for (;;) {
            int32_t i = next.fetch_add(1);
            if (i >= count) break;
            if (!s) { rc[i] = HGP_ERR_CUDA; continue; }
            cudaStreamSynchronize(gs[i]->stream);      // the handle's own work is done
            rc[i] = partition_on(gs[i], omegas[i], deltas[i], opt, &res[i], s);
        }
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    };
    std::vector<std::thread> pool;
    for (int w = 1; w < workers; ++w) pool.emplace_back(work);
    if (workers > 0) work();
    for (auto &t : pool) t.join();
    int first = HGP_OK;
    for (int32_t i = 0; i < count; ++i) {
        if (status) status[i] = rc[i];
        if (first == HGP_OK && rc[i] != HGP_OK) first = rc[i];
    }
    return first;
}

extern "C" int hgp_get_stats(const hgp_graph *g, hgp_stats *st) {
    if (!g || !st) return HGP_ERR_INVALID_ARG;
    *st = g->stats;
    return HGP_OK;
}

extern "C" int64_t hgp_get_level_len(const hgp_graph *g, int32_t level, int32_t which) {
    if (!g || which < 0 || which > HGP_LEVEL_GAIN_SEQ || level < 0) return -1;
    const auto &vv = g->dbg[which];
    if (level >= (int)vv.size() || (vv[level].empty() && which != HGP_LEVEL_REFINE)) return -1;
    return (int64_t)vv[level].size();
}

extern "C" int hgp_get_level_array(const hgp_graph *g, int32_t level, int32_t which, int64_t *out) {
    int64_t n = hgp_get_level_len(g, level, which);
    if (n < 0 || !out) return HGP_ERR_INVALID_ARG;
    const auto &v = g->dbg[which][level];
    for (int64_t i = 0; i < n; ++i) out[i] = v[i];
    return HGP_OK;
}

extern "C" int hgp_learn_samples(hgp_graph *g, const int32_t *part_ids, uint64_t seed,
                                 int32_t per_node, float *x, float *y, int32_t *partner) {
    if (!g) return HGP_ERR_INVALID_ARG;
    if (!part_ids || !x || !y || per_node < 1)
        return fail(g, HGP_ERR_INVALID_ARG, "part_ids, x, y are required and per_node must be >= 1");
    if ((int64_t)g->N * per_node > ((int64_t)1 << 40))
        return fail(g, HGP_ERR_INVALID_ARG, "num_nodes * per_node too large");
    cudaError_t e = run_learn_samples(g->L0, g->ew, part_ids, seed, per_node, x, y, partner, g->stream);
    if (e) return cuda_fail(g, e, "learn_samples");
    return HGP_OK;
}

extern "C" const char *hgp_error_string(int status) {
    switch (status) {
    case HGP_OK: return "ok";
    case HGP_ERR_INVALID_ARG: return "invalid argument";
    case HGP_ERR_INFEASIBLE: return "infeasible: a single node exceeds omega or delta";
    case HGP_ERR_OOM: return "out of device memory";
    case HGP_ERR_CUDA: return "CUDA error";
    case HGP_ERR_DEVICE_LIMIT: return "device loop budget exhausted";
    case HGP_ERR_STATE: return "invalid handle state";
    case HGP_ERR_SCRATCH_LIMIT: return "input exceeds the fixed scratch of hgp_score_noalloc";
    default: return "unknown status";
    }
}

extern "C" const char *hgp_last_error(const hgp_graph *g) {
    if (!g) return t_create_err.c_str();
    return g->err.c_str();
}

extern "C" void hgp_destroy(hgp_graph *g) {
    if (!g) return;
    cudaStreamSynchronize(g->stream);
    g->keep.release_all();
    cudaStreamSynchronize(g->stream);
    delete g;
}
