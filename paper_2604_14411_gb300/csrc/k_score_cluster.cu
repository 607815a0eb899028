// Candidate scoring for levels whose node count does not fit one CTA's shared
// memory: a thread-block cluster of 8 CTAs (8 SMs) holds the Eq. (2)
// histogram of one node in distributed shared memory, each CTA owning a
// contiguous slice of node ids.  All 8 CTAs walk the node's hyperedges and add
// omega(e) into the owning CTA's slice with remote shared-memory atomics; the
// extraction by decreasing hist value then reduces across the cluster (each
// CTA checks the tie-group candidates of its own slice).  Same answer as the
// single-CTA kernel, for up to 8 x ~48k node ids on chip.
#include <cooperative_groups.h>

#include "k_score.cuh"

namespace cg = cooperative_groups;

namespace hgp {

constexpr int kClusterCtas = 8;

__global__ void __cluster_dims__(kClusterCtas, 1, 1) __launch_bounds__(kScoreThreads)
k_score_cluster(ScoreArgs a, int32_t slice) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *row_n = reinterpret_cast<uint32_t *>(smem);
    int32_t *hist = reinterpret_cast<int32_t *>(smem + sizeof(uint32_t) * (size_t)a.bm_words);
    __shared__ int32_t red[2 * kScoreWarps];
    __shared__ int32_t s_node, s_xchg[2], s_bcast[2];
    __shared__ unsigned long long red64[kScoreWarps], s_xkey, s_bkey;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int32_t id0 = rank * slice;
    const int32_t len = max(0, min(slice, a.V - id0));
    unsigned long long bytes = 0;

    const int32_t count = a.nodes ? *a.count : a.V;
    for (int32_t i = threadIdx.x; i < len; i += kScoreThreads) hist[i] = 0;
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) {
            int32_t t = atomicAdd(a.next, 1);
            s_node = t < count ? (a.nodes ? a.nodes[t] : t) : a.V;
        }
        cl.sync();                                   // slices cleared, node published
        const int32_t n = *cl.map_shared_rank(&s_node, 0);
        if (n >= a.V) {
            cl.sync();       // no CTA leaves while a peer may still read its shared memory
            break;
        }
        if (a.dead && a.dead[n]) {
            if (rank == 0 && threadIdx.x == 0) { a.pair[n] = -1; a.score[n] = 0; }
            cl.sync();                               // everyone has read s_node
            continue;
        }
        const unsigned long long thr = a.thr ? a.thr[n] : 0ull;
        if (a.bm_words) {
            const uint4 *src = reinterpret_cast<const uint4 *>(a.bm + (int64_t)n * a.bm_words);
            uint4 *dst = reinterpret_cast<uint4 *>(row_n);
            for (int32_t i = threadIdx.x; i < (a.bm_words >> 2); i += kScoreThreads) dst[i] = src[i];
        }
        // ---- Eq. (2): hyperedges of I(n) interleaved over the cluster's warps ----
        {
            const int32_t i0 = a.ioff[n], deg = a.ioff[n + 1] - i0;
            const int32_t gw = rank * kScoreWarps + warp_id(), nw = kClusterCtas * kScoreWarps;
            const int32_t mine = (deg - gw + nw - 1) / nw;
            warp_accumulate(a, n, i0, gw, nw, mine,
                            [&](int32_t m, int32_t wt) {
                                const int32_t owner = m / slice;
                                atomicAdd(cl.map_shared_rank(hist, owner) + (m - owner * slice), wt);
                            }, bytes);
        }
        cl.sync();                                   // histogram complete, row(n) staged
        // ---- extraction by decreasing hist value, reduced over the cluster ----
        // As in k_score: ineligible neighbours are cleared from the slice once;
        // each round checks one band of values and finds the next lower value in
        // the same scan, and one exchange over the cluster settles both.
        int32_t hloc = 0;
        for (int32_t i = threadIdx.x; i < len; i += kScoreThreads) {
            const int32_t h = hist[i];
            if (h <= 0) continue;
            if (!eligible(a, id0 + i, h, thr)) hist[i] = 0;
            else hloc = max(hloc, h);
        }
        hloc = block_max_i32(hloc, red);
        if (threadIdx.x == 0) { s_xchg[0] = -1; s_xchg[1] = hloc; }
        cl.sync();
        if (threadIdx.x == 0) {
            int32_t v = 0;
            for (int r = 0; r < kClusterCtas; ++r) v = max(v, cl.map_shared_rank(s_xchg, r)[1]);
            s_bcast[1] = v;
        }
        cl.sync();                                   // all reads of s_xchg done
        int32_t hmax = s_bcast[1];
        const int64_t in_n = a.noff[n + 1] - a.noff[n];
        int32_t result = -1, rscore = 0;
        const int32_t per_warp = (((len + kScoreWarps - 1) / kScoreWarps) + 31) & ~31;
        const int32_t lo = warp_id() * per_warp, hi = min(len, lo + per_warp);
        // bands of values [bot, top] as in k_score: the largest valid (hist, id)
        // in the band wins, the band doubles after a round without one
        int32_t top = hmax, width = 1;
        while (top > 0) {
            const int32_t bot = max(1, top - width + 1);
            unsigned long long best = 0ull;
            int32_t nxt = 0;
            for (int32_t base = lo + ((hi - lo - 1) & ~31); base >= lo; base -= 32) {
                const int32_t i = base + lane_id();
                const int32_t h = i < hi ? hist[i] : 0;
                if (h < bot) nxt = max(nxt, h);
                const unsigned long long key = cand_key(h, id0 + i);
                unsigned ball = __ballot_sync(0xffffffffu, h >= bot && h <= top && key > best);
                while (ball) {
                    const int src = 31 - __clz(ball);
                    ball &= ~(1u << src);
                    const unsigned long long ck = __shfl_sync(0xffffffffu, key, src);
                    if (ck > best && warp_check(a, n, (int32_t)(ck & 0xffffffffu), row_n, in_n, bytes))
                        best = ck;
                }
                if ((int32_t)(best >> 32) == top) break;   // nothing in the band beats it
            }
            block_max_key(best, nxt, red64, red);
            if (threadIdx.x == 0) { s_xkey = best; s_xchg[1] = nxt; }
            cl.sync();
            if (threadIdx.x == 0) {
                unsigned long long b = 0ull;
                int32_t x = 0;
                for (int r = 0; r < kClusterCtas; ++r) {
                    const unsigned long long k = *cl.map_shared_rank(&s_xkey, r);
                    b = k > b ? k : b;
                    x = max(x, cl.map_shared_rank(s_xchg, r)[1]);
                }
                s_bkey = b;
                s_bcast[1] = x;
            }
            cl.sync();
            if (s_bkey) { result = (int32_t)(s_bkey & 0xffffffffu); rscore = (int32_t)(s_bkey >> 32); break; }
            top = s_bcast[1];
            width <<= 1;
        }
        if (rank == 0 && threadIdx.x == 0) {
            a.pair[n] = result;
            a.score[n] = result >= 0 ? rscore : 0;
            bytes += 16ull;
        }
        for (int32_t i = threadIdx.x; i < len; i += kScoreThreads) hist[i] = 0;
        // the cl.sync() at the top of the loop orders these clears before the next adds
    }
    if (a.bytes) {
        bytes = warp_sum(bytes);
        if (lane_id() == 0 && bytes) atomicAdd(a.bytes, bytes);
    }
}

// Launches the cluster kernel if a slice fits on chip; returns false (and
// launches nothing) otherwise.
bool launch_score_cluster(const ScoreArgs &a, int max_smem, cudaStream_t s, cudaError_t *err) {
    *err = cudaSuccess;
    int32_t slice = (a.V + kClusterCtas - 1) / kClusterCtas;
    size_t smem = sizeof(uint32_t) * (size_t)a.bm_words + sizeof(int32_t) * (size_t)slice;
    if (smem + 4096 > (size_t)max_smem) return false;
    cudaError_t e = allow_dynamic_smem(k_score_cluster);
    if (e) { *err = e; return true; }
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kScoreThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = kClusterCtas;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    cfg.gridDim = dim3(kClusterCtas);
    e = cudaOccupancyMaxActiveClusters(&clusters, k_score_cluster, &cfg);
    if (e || clusters < 1) clusters = 1;
    int want = (a.V + 0) > clusters ? clusters : a.V;
    cfg.gridDim = dim3(kClusterCtas * want);
    cfg.attrs = nullptr;       // the cluster shape comes from __cluster_dims__
    cfg.numAttrs = 0;
    e = cudaLaunchKernelEx(&cfg, k_score_cluster, a, slice);
    count_launch();
    *err = e;
    return true;
}

}  // namespace hgp
