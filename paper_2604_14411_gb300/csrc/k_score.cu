// Host side of candidate scoring: mode selection (dense shared-memory
// histogram or global hash tables; in() bitmaps or sorted-list checks) and
// launch.  The kernels are in k_score.cuh.
#include "k_score.cuh"

namespace hgp {

bool launch_score_cluster(const ScoreArgs &a, int max_smem, cudaStream_t s, cudaError_t *err);

// bytes of in() bitmaps per level: a tenth of the device memory free when
// the partition started, at most 16 GiB (a popcount over two rows is far
// cheaper than searching sorted in() lists once unions grow to thousands of
// hyperedges); measured once per partition by the caller
int64_t bitmap_budget() {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return 1ll << 30;
    int64_t b = (int64_t)(fr / 10);
    return b < (16ll << 30) ? b : (16ll << 30);
}
constexpr int32_t kBitmapMaxWords = 8192;       // 32 KB row in shared memory
// Largest number of wcap-id pieces one scoring CTA takes for a node's window
// (each piece re-reads the node's pins; wider windows go to the 8-CTA cluster).
constexpr int32_t kMaxWindows = 8;

// ---- per-node work buckets for levels too large for one CTA's histogram ----
// A node whose neighbour ids all lie in a window of at most wcap ids (as in
// layered graphs, where neighbours are spatially close) is scored by one CTA
// with a dense histogram over that window; the others by the 8-CTA cluster
// (or the hash tables).  The window is the span of the pin ids of I(n).

// smallest and largest pin id of every hyperedge (warp per hyperedge)
static __global__ void k_edge_span(int32_t E, const int32_t *poff, const int32_t *pins,
                                   int32_t *emin, int32_t *emax) {
    int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = gw; e < E; e += nw) {
        int32_t lo = 0x7fffffff, hi = -1;
        for (int32_t j = poff[e] + lane_id(); j < poff[e + 1]; j += 32) {
            const int32_t m = pins[j];
            lo = min(lo, m);
            hi = max(hi, m);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane_id() == 0) { emin[e] = lo; emax[e] = hi; }
    }
}

// window of every node and its bucket: 0 = one CTA over the window, in
// pieces of wcap ids taken one after another (nodes known to have no
// candidate go there too, they are answered at once); 1 = one CTA with a
// shared hash table, when the window takes more than one piece, the node's pin
// visits (an upper bound on its distinct neighbours) stay below hmax_visits
// and its weight sum over I(n) (an upper bound on every hist(n, m)) below
// wlimit; 0 again when at most max_windows pieces cover the window; 2 = the rest
static __global__ void k_node_window(int32_t V, const int32_t *ioff, const int32_t *inc,
                                     const int32_t *poff, const int32_t *ew,
                                     const int32_t *emin, const int32_t *emax, const uint8_t *dead,
                                     int32_t wcap, int32_t max_windows, int64_t hmax_visits,
                                     int64_t wlimit,
                                     int32_t *wlo, int32_t *whi, int32_t *b0, int32_t *b1,
                                     int32_t *b2) {
    int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t n = gw; n < V; n += nw) {
        int32_t lo = 0x7fffffff, hi = -1;
        long long visits = 0, wsum = 0;
        for (int32_t k = ioff[n] + lane_id(); k < ioff[n + 1]; k += 32) {
            const int32_t e = inc[k];
            lo = min(lo, emin[e]);
            hi = max(hi, emax[e]);
            visits += poff[e + 1] - poff[e];
            wsum += ew[e];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
            visits += __shfl_xor_sync(0xffffffffu, visits, o);
            wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
        }
        if (lane_id() == 0) {
            if (hi < lo) { lo = 0; hi = -1; }            // no hyperedge: an empty window
            wlo[n] = lo;
            whi[n] = hi;
            const int64_t span = (int64_t)hi - lo + 1;
            const int one = (dead && dead[n]) || span <= wcap;
            const int h = !one && visits <= hmax_visits && wsum < wlimit;
            const int f = one || (!h && span <= (int64_t)wcap * max_windows);
            b0[n] = f;
            b1[n] = h;
            b2[n] = 1 - f - h;
        }
    }
}

static __global__ void k_bucket_lists(int32_t V, const int32_t *b0, const int32_t *b1,
                                      const int32_t *r0, const int32_t *r1, const int32_t *r2,
                                      int32_t *l0, int32_t *l1, int32_t *l2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (b0[i]) l0[r0[i]] = (int32_t)i;
        else if (b1[i]) l1[r1[i]] = (int32_t)i;
        else l2[r2[i]] = (int32_t)i;
    }
}

// Rows of the coarse level's in() bitmaps from the finer level's: coarse node
// c is the finer node a = old_id[c] or the pair {a, match[a]}, and in(c) is
// the union of its members' in(), so row(c) = row(a) | row(match[a]) (warp
// per row, 16-byte words).
static __global__ void k_bitmap_merge(int32_t V, int32_t words, const int32_t *old_id,
                                      const int32_t *match_prev, const uint32_t *bm_prev,
                                      uint32_t *bm) {
    int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t q = words >> 2;
    for (int64_t c = gw; c < V; c += nw) {
        const int32_t a = old_id[c], b = match_prev[a];
        const uint4 *ra = reinterpret_cast<const uint4 *>(bm_prev + (int64_t)a * words);
        const uint4 *rb = reinterpret_cast<const uint4 *>(bm_prev + (int64_t)b * words);
        uint4 *rc = reinterpret_cast<uint4 *>(bm + c * words);
        for (int32_t i = lane_id(); i < q; i += 32) {
            uint4 x = ra[i];
            if (b != a) {
                const uint4 y = rb[i];
                x.x |= y.x; x.y |= y.y; x.z |= y.z; x.w |= y.w;
            }
            rc[i] = x;
        }
    }
}

// roll: arena of this level's in() lists (the bitmaps are kept there, see
// Level::bm); prev: the finer level (null at level 0), whose bitmaps, match
// and this level's old_id let the rows be merged instead of rebuilt.
cudaError_t run_score(Arena &ar, Arena &roll, Level &L, const Level *prev, const int32_t *ew,
                      int64_t omega, int64_t delta, int32_t *pair, int32_t *score, int32_t *status,
                      unsigned long long *bytes, uint32_t debug, int64_t bm_budget, cudaStream_t s) {
    if (L.V <= 0) return cudaSuccess;
    int dev = 0;
    cudaGetDevice(&dev);
    int max_smem = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    ScoreArgs a{};
    a.V = L.V; a.E = L.E;
    a.w = L.w; a.poff = L.poff; a.pins = L.pins; a.ioff = L.ioff; a.inc = L.inc;
    a.noff = L.noff; a.inn = L.inn; a.ew = ew;
    a.omega = omega; a.delta = delta;
    a.pair = pair; a.score = score; a.status = status; a.bytes = bytes;
    a.dead = L.dead; a.merged = L.merged; a.thr = L.thr; a.old_id = L.old_id;
    a.vec_pins = 1;      // level pins live in arena chunks: 256-byte aligned, sizes rounded to 256
    cudaError_t e = dalloc(ar, &a.next, 1);
    if (!e) e = cudaMemsetAsync(a.next, 0, sizeof(int32_t), s);
    if (e) return e;
    // bitmaps only when some pair may need a union count
    int32_t words = ((L.E + 31) / 32 + 3) & ~3;
    bool need_union = 2 * (int64_t)L.max_in > delta;
    if (need_union && !(debug & HGP_DEBUG_NO_BITMAP) && words <= kBitmapMaxWords &&
        (int64_t)L.V * words * 4 <= bm_budget) {
        uint32_t *bm = nullptr;
        e = dalloc(roll, &bm, (size_t)L.V * words);
        if (e) return e;
        int blocks = div_up((int64_t)L.V * 32, 256);
        if (blocks > num_sms() * 16) blocks = num_sms() * 16;
        if (prev && prev->bm && prev->bm_words == words && L.old_id && prev->match) {
            k_bitmap_merge<<<blocks, 256, 0, s>>>(L.V, words, L.old_id, prev->match, prev->bm, bm);
        } else {
            e = cudaMemsetAsync(bm, 0, sizeof(uint32_t) * (size_t)L.V * words, s);
            if (e) return e;
            k_in_bitmap<<<blocks, 256, 0, s>>>(L.V, L.noff, L.inn, words, bm);
        }
        count_launch();
        a.bm = bm;
        a.bm_words = words;
        L.bm = bm;
        L.bm_words = words;
    }
    size_t row_bytes = sizeof(uint32_t) * (size_t)a.bm_words;
    size_t dense_smem = row_bytes + sizeof(int32_t) * (size_t)L.V;
    const uint32_t buckets = HGP_DEBUG_FORCE_WINDOW | HGP_DEBUG_FORCE_HASH_BUCKET;
    bool dense = dense_smem + 2048 <= (size_t)max_smem &&
                 !(debug & (HGP_DEBUG_FORCE_GLOBAL | HGP_DEBUG_FORCE_CLUSTER | buckets));
    int sms = num_sms();
    int64_t wcap = ((int64_t)max_smem - 2048 - (int64_t)row_bytes) / 4;
    if (debug & buckets) {                  // test knob: small windows, so every bucket is used
        int64_t small = L.V / 4 > 64 ? L.V / 4 : 64;
        if (small < wcap) wcap = small;
    }
    if (!dense && wcap >= 64 && !(debug & (HGP_DEBUG_FORCE_GLOBAL | HGP_DEBUG_FORCE_CLUSTER))) {
        int32_t *emin, *emax, *wlo, *whi, *bk[3], *rk[3], *lst[3], *cnt;
        e = dalloc(ar, &emin, L.E);
        if (!e) e = dalloc(ar, &emax, L.E);
        if (!e) e = dalloc(ar, &wlo, L.V);
        if (!e) e = dalloc(ar, &whi, L.V);
        for (int k = 0; k < 3 && !e; ++k) {
            e = dalloc(ar, &bk[k], L.V);
            if (!e) e = dalloc(ar, &rk[k], L.V);
            if (!e) e = dalloc(ar, &lst[k], L.V);
        }
        if (!e) e = dalloc(ar, &cnt, 3);
        if (e) return e;
        // shared hash bucket: packed 32-bit slots after row(n); the id field
        // holds id + 1 (0 = empty), the rest of the word the count
        const int kbits = 32 - __builtin_clz((unsigned)L.V);
        const int vbits = 32 - kbits;
        int64_t scap = ((int64_t)max_smem - 2048 - (int64_t)row_bytes) / 4;
        scap &= ~(int64_t)31;
        int64_t hvisits = scap * 5 / 8;                   // load factor at most 5/8
        int64_t wlimit = vbits >= 4 ? (1ll << vbits) : 0;
        if (debug & HGP_DEBUG_FORCE_HASH_BUCKET) {      // test knob: a small table
            scap = scap < 1024 ? scap : 1024;
            hvisits = scap * 5 / 8;
        }
        if (scap < 1024 || wlimit == 0 || (debug & HGP_DEBUG_FORCE_WINDOW)) hvisits = -1;
        int wb = div_up((int64_t)(L.E > L.V ? L.E : L.V) * 32, 256);
        if (wb > sms * 16) wb = sms * 16;
        if (wb < 1) wb = 1;
        if (L.E > 0) {
            k_edge_span<<<wb, 256, 0, s>>>(L.E, L.poff, L.pins, emin, emax);
            count_launch();
        }
        // windows per node: up to kMaxWindows pieces of wcap ids (single pieces
        // under the hash-bucket test knob, so that the cluster takes the rest)
        const int32_t maxw = (debug & HGP_DEBUG_FORCE_HASH_BUCKET) ? 1 : kMaxWindows;
        k_node_window<<<wb, 256, 0, s>>>(L.V, L.ioff, L.inc, L.poff, ew, emin, emax, L.dead,
                                         (int32_t)wcap, maxw, hvisits, wlimit, wlo, whi, bk[0],
                                         bk[1], bk[2]);
        count_launch();
        for (int k = 0; k < 3 && !e; ++k) e = exclusive_scan_i32(ar, bk[k], rk[k], L.V, cnt + k, s);
        if (e) return e;
        k_bucket_lists<<<div_up(L.V, 256) < sms * 8 ? div_up(L.V, 256) : sms * 8, 256, 0, s>>>(
            L.V, bk[0], bk[1], rk[0], rk[1], rk[2], lst[0], lst[1], lst[2]);
        count_launch();
        // bucket 0: one CTA per node over its window, piece by piece
        ScoreArgs w = a;
        w.nodes = lst[0];
        w.count = cnt;
        w.wlo = wlo;
        w.whi = whi;
        w.wcap = (int32_t)wcap;
        size_t wsmem = row_bytes + sizeof(int32_t) * (size_t)wcap;
        e = allow_dynamic_smem(k_score<true>);
        if (e) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_score<true>, kScoreThreads, wsmem);
        if (e) return e;
        if (per_sm < 1) per_sm = 1;
        int blocks = sms * per_sm;
        if (blocks > L.V) blocks = L.V;
        k_score<true><<<blocks, kScoreThreads, wsmem, s>>>(w);
        count_launch();
        e = cudaGetLastError();
        if (e) return e;
        // bucket 1: one CTA per node with a shared hash table
        if (hvisits > 0) {
            ScoreArgs h = a;
            h.nodes = lst[1];
            h.count = cnt + 1;
            h.scap = (int32_t)scap;
            h.vbits = vbits;
            e = dalloc(ar, &h.next, 1);
            if (!e) e = cudaMemsetAsync(h.next, 0, sizeof(int32_t), s);
            if (e) return e;
            size_t hsmem = row_bytes + sizeof(uint32_t) * (size_t)scap;
            auto hk = k_score<false, kScoreThreads, true>;
            e = allow_dynamic_smem(hk);
            if (e) return e;
            blocks = sms;
            if (blocks > L.V) blocks = L.V;
            hk<<<blocks, kScoreThreads, hsmem, s>>>(h);
            count_launch();
            e = cudaGetLastError();
            if (e) return e;
        }
        // bucket 2: the rest, on the cluster (or the hash tables below)
        a.nodes = lst[2];
        a.count = cnt + 2;
        e = dalloc(ar, &a.next, 1);
        if (!e) e = cudaMemsetAsync(a.next, 0, sizeof(int32_t), s);
        if (e) return e;
    }
    if (dense) {
        // (two 512-thread CTAs per SM were measured: slower on the 16k SNN,
        // 164 -> 197 ms of scoring per step)
        auto kern = k_score<true, kScoreThreads>;
        const int nt = kScoreThreads;
        e = allow_dynamic_smem(kern);
        if (e) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, dense_smem);
        if (e) return e;
        if (per_sm < 1) per_sm = 1;
        int blocks = sms * per_sm;
        if (blocks > L.V) blocks = L.V;
        kern<<<blocks, nt, dense_smem, s>>>(a);
        count_launch();
        return cudaGetLastError();
    }
    // levels too large for one CTA: the histogram spread over an 8-CTA cluster
    if (!(debug & HGP_DEBUG_FORCE_GLOBAL)) {
        if (launch_score_cluster(a, max_smem, s, &e)) return e ? e : cudaGetLastError();
    }
    // hash mode: per-CTA global tables sized for the heaviest node
    unsigned long long *d_work = nullptr;
    e = dalloc(ar, &d_work, 1);
    if (e) return e;
    cudaMemsetAsync(d_work, 0, sizeof(unsigned long long), s);
    k_max_work<<<sms * 8, 256, 0, s>>>(L.V, L.ioff, L.inc, L.poff, d_work);
    count_launch();
    unsigned long long h_work = 0;
    e = cudaMemcpyAsync(&h_work, d_work, sizeof(h_work), cudaMemcpyDeviceToHost, s);
    if (e) return e;
    e = cudaStreamSynchronize(s);
    if (e) return e;
    unsigned long long distinct = h_work < (unsigned long long)L.V ? h_work : (unsigned long long)L.V;
    unsigned long long gcap = 64;
    while (gcap < 2 * distinct && !(debug & HGP_DEBUG_SMALL_TABLE)) gcap <<= 1;
    if (gcap > (1ull << 30)) return cudaErrorMemoryAllocation;
    a.gcap = (int32_t)gcap;
    e = allow_dynamic_smem(k_score<false>);
    if (e) return e;
    int blocks = sms * 2;
    if (blocks > L.V) blocks = L.V;
    e = dalloc(ar, &a.gkeys, (size_t)blocks * gcap);
    if (!e) e = dalloc(ar, &a.gvals, (size_t)blocks * gcap);
    if (e) return e;
    k_score<false><<<blocks, kScoreThreads, row_bytes, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

}  // namespace hgp
