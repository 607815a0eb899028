// Host side of candidate scoring: mode selection (dense shared-memory
// histogram or global hash tables; in() bitmaps or sorted-list checks) and
// launch.  The kernels are in k_score.cuh.
#include "k_score.cuh"

namespace hgp {

bool launch_score_cluster(const ScoreArgs &a, int max_smem, cudaStream_t s, cudaError_t *err);

constexpr int64_t kBitmapBudget = 1ll << 30;   // bytes of in() bitmaps per level
constexpr int32_t kBitmapMaxWords = 8192;       // 32 KB row in shared memory

cudaError_t run_score(Arena &ar, const Level &L, const int32_t *ew, int64_t omega, int64_t delta,
                      int32_t *pair, int32_t *score, int32_t *status,
                      unsigned long long *bytes, uint32_t debug, cudaStream_t s) {
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
        (int64_t)L.V * words * 4 <= kBitmapBudget) {
        uint32_t *bm = nullptr;
        e = dalloc(ar, &bm, (size_t)L.V * words);
        if (e) return e;
        e = cudaMemsetAsync(bm, 0, sizeof(uint32_t) * (size_t)L.V * words, s);
        if (e) return e;
        int blocks = div_up((int64_t)L.V * 32, 256);
        if (blocks > num_sms() * 16) blocks = num_sms() * 16;
        k_in_bitmap<<<blocks, 256, 0, s>>>(L.V, L.noff, L.inn, words, bm);
        count_launch();
        a.bm = bm;
        a.bm_words = words;
    }
    size_t row_bytes = sizeof(uint32_t) * (size_t)a.bm_words;
    size_t dense_smem = row_bytes + sizeof(int32_t) * (size_t)L.V;
    bool dense = dense_smem + 2048 <= (size_t)max_smem &&
                 !(debug & (HGP_DEBUG_FORCE_GLOBAL | HGP_DEBUG_FORCE_CLUSTER));
    int sms = num_sms();
    if (dense) {
        e = allow_dynamic_smem(k_score<true>);
        if (e) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_score<true>, kScoreThreads,
                                                          dense_smem);
        if (e) return e;
        if (per_sm < 1) per_sm = 1;
        int blocks = sms * per_sm;
        if (blocks > L.V) blocks = L.V;
        k_score<true><<<blocks, kScoreThreads, dense_smem, s>>>(a);
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
