// Candidate scoring (Sec. III-A, Eq. (2)) fused with the deferred validity
// checks of Sec. III-B.2.
//
// One CTA per node n (persistent grid, nodes strided over CTAs).
//   1. hist(n, m) = sum of omega(e) over e in I(n), m in e, m != n.
//      Each warp takes hyperedges of I(n); its lanes read the pins of one
//      hyperedge with coalesced int32 loads and add omega(e) into the
//      histogram:
//        dense mode  -- a |N_l|-entry int32 array in shared memory,
//                       indexed by node id (one smem atomic per pin visit);
//        hash mode   -- a per-CTA open-addressing table in global memory
//                       (levels whose node count does not fit on chip).
//   2. Candidates are extracted by decreasing hist value.  For the current
//      top value h, every neighbour with hist = h is checked in parallel
//      (one warp per candidate); the valid one of largest id wins.  If none
//      is valid the next lower value is taken.  This visits candidates in
//      the paper's (hist desc, id desc) order and returns the first valid
//      one, checking a whole tie group at once.
//   3. Check of a pair (n, m): w(n) + w(m) <= Omega, and
//      |in(n) u in(m)| <= Delta.  When |in(n)| + |in(m)| <= Delta the pair is
//      valid without counting.  Otherwise the union is counted either
//        bitmap mode -- as popcount(row(n) | row(m)) over per-node bitmaps of
//                       in() with one bit per hyperedge (row(n) staged in
//                       shared memory, row(m) read with 16-byte loads), or
//        list mode   -- as |in(n)| + |in(m) \ in(n)| with a binary search in
//                       the sorted in(n), stopping as soon as Delta is
//                       exceeded (levels whose bitmaps would not fit).
#pragma once
#include "hgp_internal.cuh"

namespace hgp {

constexpr int kScoreThreads = 1024;
constexpr int kScoreWarps = kScoreThreads / 32;

struct ScoreArgs {
    int32_t V, E;
    const int32_t *w, *poff, *pins, *ioff, *inc, *noff, *inn, *ew;
    int64_t omega, delta;
    int32_t *pair, *score;
    int32_t *status;
    int32_t *gkeys, *gvals;          // hash mode: per-CTA tables of gcap entries
    int32_t gcap;
    int32_t wcap;                    // dense mode: table entries (0 = V, one window)
    // shared hash mode: scap packed slots ((id + 1) << vbits | hist) in shared
    // memory; every node scored this way has fewer pin visits than 5/8 scap and
    // a weight sum over I(n) below 2^vbits, so neither probing nor a count can overflow
    int32_t scap, vbits;
    unsigned long long *bytes;
    const uint32_t *bm;              // bitmap mode: [V][bm_words] rows of in()
    int32_t bm_words;                // multiple of 4 (16-byte rows); 0 = list mode
    const uint8_t *dead, *merged;    // carried level state (null at level 0)
    const unsigned long long *thr;
    const int32_t *old_id;
    int32_t *next;                   // work counter: nodes are taken dynamically
    int32_t vec_pins;                // pins readable as 16-byte vectors: 16-byte aligned, and
                                     // the allocation extends to a multiple of 16 bytes
    // per-node work lists (null: every node 0..V-1): nodes[0 .. *count)
    const int32_t *nodes, *count;
    // dense mode, windowed: node n's neighbours all lie in [wlo[n], whi[n]] and
    // its histogram holds only that window (null: the whole id range)
    const int32_t *wlo, *whi;
};

// m is worth checking for n: alive, and either newly merged or ranked below
// n's previous candidate (the ones above it were already invalid).
__device__ __forceinline__ bool eligible(const ScoreArgs &a, int32_t m, int32_t h,
                                         unsigned long long thr) {
    if (a.dead && a.dead[m]) return false;
    if (thr == 0ull || a.merged[m]) return true;
    unsigned long long key = ((unsigned long long)(uint32_t)h << 32) | (uint32_t)a.old_id[m];
    return key < thr;
}

__device__ __forceinline__ uint32_t hash_u32(uint32_t x) {
    x ^= x >> 16; x *= 0x7feb352dU; x ^= x >> 15; x *= 0x846ca68bU; x ^= x >> 16;
    return x;
}

template <int NW = kScoreWarps>
__device__ __forceinline__ int32_t block_max_i32(int32_t v, int32_t *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane_id() == 0) red[warp_id()] = v;
    __syncthreads();
    int32_t r = red[0];
#pragma unroll
    for (int i = 1; i < NW; ++i) r = max(r, red[i]);
    return r;
}

// Eq. (2) accumulation over the hyperedges of I(n) that one warp owns
// (entries i0 + first + stride * r of inc, r < count): add(m, omega(e)) for
// every pin m != n of each.  Each lane first fetches one hyperedge's
// (omega, pin range); then four hyperedges at a time, every lane loads its
// 16-byte slice of each before any of its adds, so a warp keeps up to 2 KB
// of pin loads in flight instead of one 128-byte load per hyperedge (the
// loop is otherwise bound by load latency).  Slices are aligned to 4 pins
// and masked to the hyperedge's range; warp shuffles then give each add
// instruction 32 consecutive pins.  With vec_pins = 0 pins are read one per
// lane.
constexpr int kAccEdges = 4;

template <typename Add>
__device__ __forceinline__ void warp_accumulate(const ScoreArgs &a, int32_t n, int32_t i0,
                                                int32_t first, int32_t stride, int32_t count,
                                                Add &&add, unsigned long long &bytes) {
    const int lane = lane_id();
    for (int32_t r0 = 0; r0 < count; r0 += 32) {
        int32_t we = 0, p0 = 0, p1 = 0;
        if (r0 + lane < count) {
            const int32_t e = a.inc[i0 + first + stride * (r0 + lane)];
            we = a.ew[e];
            p0 = a.poff[e];
            p1 = a.poff[e + 1];
        }
        const int32_t cnt = min(32, count - r0);     // lanes >= cnt hold empty ranges
        if (!a.vec_pins) {
            for (int32_t t = 0; t < cnt; ++t) {
                const int32_t wt = __shfl_sync(0xffffffffu, we, t);
                const int32_t b0 = __shfl_sync(0xffffffffu, p0, t);
                const int32_t b1 = __shfl_sync(0xffffffffu, p1, t);
                for (int32_t j = b0 + lane; j < b1; j += 32) {
                    const int32_t m = a.pins[j];
                    if (m != n) add(m, wt);
                }
                if (lane == 0) bytes += 16ull + 4ull * (unsigned long long)(b1 - b0);
            }
            continue;
        }
        const int4 *pv = reinterpret_cast<const int4 *>(a.pins);
        for (int32_t t = 0; t < cnt; t += kAccEdges) {
            int32_t wt[kAccEdges], q0[kAccEdges], b0[kAccEdges], b1[kAccEdges];
            int32_t span = 0;
#pragma unroll
            for (int u = 0; u < kAccEdges; ++u) {
                const int src = (t + u) & 31;            // t + u < 32; past cnt: empty range
                wt[u] = __shfl_sync(0xffffffffu, we, src);
                b0[u] = __shfl_sync(0xffffffffu, p0, src);
                b1[u] = __shfl_sync(0xffffffffu, p1, src);
                if (t + u >= cnt) b0[u] = b1[u] = 0;
                q0[u] = b0[u] >> 2;
                span = max(span, ((b1[u] + 3) >> 2) - q0[u]);
                if (lane == 0) bytes += t + u < cnt ? 16ull + 4ull * (unsigned long long)(b1[u] - b0[u]) : 0ull;
            }
            for (int32_t kb = 0; kb < span; kb += 32) {
                // lane l loads pins 4 (q0 + kb + l) .. + 3 of every hyperedge ...
                int4 v[kAccEdges];
#pragma unroll
                for (int u = 0; u < kAccEdges; ++u)
                    v[u] = 4 * (q0[u] + kb + lane) < b1[u] ? pv[q0[u] + kb + lane] : make_int4(-1, -1, -1, -1);
                // ... and the warp's 128 pins are handed out so that step c gives
                // lane l pin 32 c + l: each add instruction then covers 32
                // consecutive pins, as a scalar walk would (consecutive ids --
                // sorted targets -- then fall in distinct banks, and in one
                // remote CTA's slice on the cluster)
#pragma unroll
                for (int u = 0; u < kAccEdges; ++u) {
                    const int32_t j0 = 4 * (q0[u] + kb);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int from = 8 * c + (lane >> 2);
                        const int32_t x = __shfl_sync(0xffffffffu, v[u].x, from);
                        const int32_t y = __shfl_sync(0xffffffffu, v[u].y, from);
                        const int32_t z = __shfl_sync(0xffffffffu, v[u].z, from);
                        const int32_t w = __shfl_sync(0xffffffffu, v[u].w, from);
                        const int sel = lane & 3;
                        const int32_t m = sel == 0 ? x : sel == 1 ? y : sel == 2 ? z : w;
                        const int32_t j = j0 + 32 * c + lane;
                        if (j >= b0[u] && j < b1[u] && m != n) add(m, wt[u]);
                    }
                }
            }
        }
    }
}

// CTA-wide maxima of two values at once over NW warps (red: 2 * NW entries).
template <int NW = kScoreWarps>
__device__ __forceinline__ void block_max2_i32(int32_t &x, int32_t &y, int32_t *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x = max(x, __shfl_xor_sync(0xffffffffu, x, o));
        y = max(y, __shfl_xor_sync(0xffffffffu, y, o));
    }
    __syncthreads();
    if (lane_id() == 0) { red[warp_id()] = x; red[NW + warp_id()] = y; }
    __syncthreads();
    x = red[0];
    y = red[NW];
#pragma unroll
    for (int i = 1; i < NW; ++i) { x = max(x, red[i]); y = max(y, red[NW + i]); }
}

// CTA-wide maxima of a 64-bit key and a 32-bit value over NW warps.
template <int NW = kScoreWarps>
__device__ __forceinline__ void block_max_key(unsigned long long &k, int32_t &x,
                                              unsigned long long *red64, int32_t *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, k, o);
        k = k2 > k ? k2 : k;
        x = max(x, __shfl_xor_sync(0xffffffffu, x, o));
    }
    __syncthreads();
    if (lane_id() == 0) { red64[warp_id()] = k; red[warp_id()] = x; }
    __syncthreads();
    k = red64[0];
    x = red[0];
#pragma unroll
    for (int i = 1; i < NW; ++i) { k = red64[i] > k ? red64[i] : k; x = max(x, red[i]); }
}

// Candidate key in the extraction order: (hist, id), larger first.
__device__ __forceinline__ unsigned long long cand_key(int32_t h, int32_t id) {
    return ((unsigned long long)(uint32_t)h << 32) | (uint32_t)id;
}

// Warp-cooperative validity test of pair (n, m); all lanes return the same.
static __device__ bool warp_check(const ScoreArgs &a, int32_t n, int32_t m, const uint32_t *row_n,
                           int64_t in_n, unsigned long long &bytes) {
    if ((int64_t)a.w[n] + a.w[m] > a.omega) return false;
    int32_t m0 = a.noff[m], m1 = a.noff[m + 1];
    int64_t in_m = m1 - m0;
    if (in_n + in_m <= a.delta) return true;
    if (a.bm_words && in_m <= (int64_t)a.bm_words) {
        // in(m) is shorter than a bitmap row: walk its list and probe row(n)
        // in shared memory; |in(n) u in(m)| = |in(n)| + |in(m) \ in(n)|
        const int64_t room = a.delta - in_n;
        int64_t extra = 0;
        int32_t seen = 0;
        for (int32_t base = m0; base < m1; base += 128) {
            int32_t miss = 0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int32_t j = base + u * 32 + lane_id();
                if (j < m1) {
                    const int32_t e = a.inn[j];
                    miss += ((row_n[e >> 5] >> (e & 31)) & 1u) ? 0 : 1;
                }
            }
            extra += warp_sum(miss);
            seen += min(128, m1 - base);
            if (extra > room) break;
        }
        if (lane_id() == 0) bytes += 4ull * (unsigned long long)seen;
        return extra <= room;
    }
    if (a.bm_words) {
        const uint4 *rm = reinterpret_cast<const uint4 *>(a.bm + (int64_t)m * a.bm_words);
        const uint4 *rn = reinterpret_cast<const uint4 *>(row_n);
        int32_t q = a.bm_words >> 2;
        int32_t u = 0;
        for (int32_t i = lane_id(); i < q; i += 32) {
            uint4 x = rm[i], y = rn[i];
            u += __popc(x.x | y.x) + __popc(x.y | y.y) + __popc(x.z | y.z) + __popc(x.w | y.w);
        }
        u = warp_sum(u);
        if (lane_id() == 0) bytes += 4ull * (unsigned long long)a.bm_words;
        return u <= a.delta;
    }
    int32_t n0 = a.noff[n], n1 = a.noff[n + 1];
    int64_t room = a.delta - in_n;          // edges of in(m) allowed outside in(n)
    int64_t extra = 0;
    int32_t seen = 0;
    for (int32_t base = m0; base < m1; base += 128) {
        int32_t miss = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int32_t j = base + u * 32 + lane_id();
            if (j < m1) miss += contains_sorted(a.inn, n0, n1, a.inn[j]) ? 0 : 1;
        }
        extra += warp_sum(miss);
        seen += min(128, m1 - base);
        if (extra > room) break;
    }
    if (lane_id() == 0) bytes += 4ull * (unsigned long long)seen;
    return extra <= room;
}

// NT threads per CTA: 1024 (one CTA per SM), or 512 with two CTAs per SM when
// two histograms fit (shorter barriers, one CTA's extraction overlapping the
// other's gather).
template <bool DENSE, int NT = kScoreThreads, bool SHASH = false>
__global__ void __launch_bounds__(NT, kScoreThreads / NT)
k_score(ScoreArgs a) {
    constexpr int NW = NT / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    // layout: [row of in(n): bm_words][dense hist V]
    uint32_t *row_n = reinterpret_cast<uint32_t *>(smem);
    int32_t *hist = reinterpret_cast<int32_t *>(smem + sizeof(uint32_t) * (size_t)a.bm_words);
    __shared__ int32_t red[2 * NW];
    __shared__ unsigned long long red64[NW];

    int32_t *gkeys = (DENSE || SHASH) ? nullptr : a.gkeys + (int64_t)blockIdx.x * a.gcap;
    int32_t *gvals = (DENSE || SHASH) ? nullptr : a.gvals + (int64_t)blockIdx.x * a.gcap;
    uint32_t *stab = reinterpret_cast<uint32_t *>(hist);       // shared hash slots
    const uint32_t vmask = SHASH ? ((1u << a.vbits) - 1u) : 0u;
    const uint32_t mask = (uint32_t)a.gcap - 1u;
    unsigned long long bytes = 0;

    __shared__ int32_t s_n;
    const int32_t count = a.nodes ? *a.count : a.V;
    for (;;) {
        if (threadIdx.x == 0) s_n = atomicAdd(a.next, 1);
        __syncthreads();
        const int32_t t = s_n;
        if (t >= count) break;
        const int32_t n = a.nodes ? a.nodes[t] : t;
        if (a.dead && a.dead[n]) {              // no valid candidate can exist
            if (threadIdx.x == 0) { a.pair[n] = -1; a.score[n] = 0; }
            __syncthreads();
            continue;
        }
        const unsigned long long thr = a.thr ? a.thr[n] : 0ull;
        if (a.bm_words) {
            const uint4 *src = reinterpret_cast<const uint4 *>(a.bm + (int64_t)n * a.bm_words);
            uint4 *dst = reinterpret_cast<uint4 *>(row_n);
            for (int32_t i = threadIdx.x; i < (a.bm_words >> 2); i += NT) dst[i] = src[i];
        }
        const int64_t in_n = a.noff[n + 1] - a.noff[n];
        // Dense table: the node's neighbour ids lo_n .. hi_n (its window, or
        // all ids) in windows of at most wcap ids, taken from the top down;
        // the hash modes have one table.  The answer is the largest valid
        // (hist, id) over all windows.
        const int32_t lo_n = (DENSE && a.wlo) ? a.wlo[n] : 0;
        const int32_t hi_n = DENSE ? (a.wlo ? a.whi[n] : a.V - 1) : 0;
        const int32_t wcap = a.wcap > 0 ? a.wcap : a.V;
        unsigned long long best_all = 0ull;
        for (int32_t wtop = hi_n;; wtop -= wcap) {
            const int32_t base = DENSE ? max(lo_n, wtop - wcap + 1) : 0;
            const int32_t cap = DENSE ? max(0, wtop - base + 1) : (SHASH ? a.scap : a.gcap);
            // ---- clear ----
            for (int32_t i = threadIdx.x; i < cap; i += NT) {
                if (DENSE) hist[i] = 0;
                else if (SHASH) stab[i] = 0u;
                else { gkeys[i] = -1; gvals[i] = 0; }
            }
            __syncthreads();
            // ---- Eq. (2) accumulation: warp w takes hyperedges i0 + w, i0 + w + W, ... ----
            {
                const int32_t i0 = a.ioff[n], deg = a.ioff[n + 1] - i0;
                const int32_t mine = (deg - warp_id() + NW - 1) / NW;
                if (DENSE) {
                    warp_accumulate(a, n, i0, warp_id(), NW, mine,
                                    [&](int32_t m, int32_t wt) {
                                        if ((uint32_t)(m - base) < (uint32_t)cap) atomicAdd(&hist[m - base], wt);
                                    }, bytes);
                } else if (SHASH) {
                    // linear probing from a multiplicative hash; a slot's id never
                    // changes once set, so a plain read that sees it is conclusive
                    warp_accumulate(a, n, i0, warp_id(), NW, mine,
                                    [&](int32_t m, int32_t wt) {
                                        const uint32_t tag = (uint32_t)(m + 1) << a.vbits;
                                        uint32_t slot = (uint32_t)(((unsigned long long)hash_u32((uint32_t)m) *
                                                                    (uint32_t)cap) >> 32);
                                        for (int32_t probes = 0;;) {
                                            uint32_t cur = *reinterpret_cast<volatile uint32_t *>(&stab[slot]);
                                            if (cur == 0u) {
                                                cur = atomicCAS(&stab[slot], 0u, tag | (uint32_t)wt);
                                                if (cur == 0u) break;
                                            }
                                            if ((cur & ~vmask) == tag) { atomicAdd(&stab[slot], (uint32_t)wt); break; }
                                            slot = slot + 1u == (uint32_t)cap ? 0u : slot + 1u;
                                            if (++probes >= cap) { set_status(a.status, kDevLimit); break; }
                                        }
                                    }, bytes);
                } else {
                    warp_accumulate(a, n, i0, warp_id(), NW, mine,
                                    [&](int32_t m, int32_t wt) {
                                        uint32_t slot = hash_u32((uint32_t)m) & mask;
                                        for (int32_t probes = 0;;) {
                                            int32_t kk = atomicCAS(&gkeys[slot], -1, m);
                                            if (kk == -1 || kk == m) { atomicAdd(&gvals[slot], wt); break; }
                                            slot = (slot + 1) & mask;
                                            if (++probes >= a.gcap) { set_status(a.status, kDevLimit); break; }
                                        }
                                    }, bytes);
                }
            }
            __syncthreads();
            // ---- extraction by decreasing hist value ----
            // Which neighbours may be the candidate does not change during the
            // extraction (eligible() depends on m and hist(n, m) only), so the
            // others are cleared from the table once; every round then scans the
            // table in shared memory alone, checking the tie group of value hmax
            // and finding the next lower value in the same pass.
            int32_t hmax = 0;
            for (int32_t i = threadIdx.x; i < cap; i += NT) {
                const int32_t h = DENSE ? hist[i]
                                  : SHASH ? (int32_t)(stab[i] & vmask) : (gkeys[i] >= 0 ? gvals[i] : 0);
                if (h <= 0) continue;
                const int32_t m = DENSE ? base + i : SHASH ? (int32_t)(stab[i] >> a.vbits) - 1 : gkeys[i];
                if (!eligible(a, m, h, thr)) {
                    if (DENSE) hist[i] = 0;
                    else if (SHASH) stab[i] &= ~vmask;        // the id stays, the count drops to 0
                    else gvals[i] = 0;
                } else {
                    hmax = max(hmax, h);
                }
            }
            hmax = block_max_i32<NW>(hmax, red);
            const int32_t per_warp = (((cap + NW - 1) / NW) + 31) & ~31;
            const int32_t lo = warp_id() * per_warp, hi = min(cap, lo + per_warp);
            // Rounds over bands of values [bot, top]: every candidate in the band
            // that beats the best so far is checked and the largest valid (hist,
            // id) wins -- the first valid one in the (hist desc, id desc) order,
            // since every value above the band has been checked already.  The
            // first band is the top value alone; after each round without a valid
            // candidate the band doubles (a node facing saturated clusters fails
            // many groups in a row).  nxt = the largest value below the band,
            // complete whenever no warp ended its scan early (only a find at the
            // band's top ends it).  best_all carries the best of the windows above,
            // whose ids are all larger: only a larger hist can beat it here.
            int32_t top = hmax, width = 1;
            while (top > (int32_t)(best_all >> 32)) {
                const int32_t bot = max(1, top - width + 1);
                unsigned long long best = best_all;       // this warp's best valid key
                int32_t nxt = 0;
                if (DENSE) {
                    // ids are table indices: scan downwards, so within one value the
                    // first valid candidate is the warp's best
                    for (int32_t b0 = lo + ((hi - lo - 1) & ~31); b0 >= lo; b0 -= 32) {
                        const int32_t i = b0 + lane_id();
                        const int32_t h = i < hi ? hist[i] : 0;
                        if (h < bot) nxt = max(nxt, h);
                        const unsigned long long key = cand_key(h, base + i);
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
                } else {
                    for (int32_t b0 = lo; b0 < hi; b0 += 32) {
                        const int32_t i = b0 + lane_id();
                        int32_t h = 0;
                        unsigned long long key = 0ull;
                        if (SHASH) {
                            const uint32_t u = i < hi ? stab[i] : 0u;
                            h = (int32_t)(u & vmask);
                            key = cand_key(h, (int32_t)(u >> a.vbits) - 1);
                            if (h < bot) nxt = max(nxt, h);
                        } else if (i < hi && gkeys[i] >= 0) {
                            h = gvals[i];
                            key = cand_key(h, gkeys[i]);
                            if (h < bot) nxt = max(nxt, h);
                        }
                        unsigned ball = __ballot_sync(0xffffffffu, h >= bot && h <= top && key > best);
                        while (ball) {
                            const int src = __ffs(ball) - 1;
                            ball &= ball - 1;
                            const unsigned long long ck = __shfl_sync(0xffffffffu, key, src);
                            if (ck > best && warp_check(a, n, (int32_t)(ck & 0xffffffffu), row_n, in_n, bytes))
                                best = ck;
                        }
                    }
                }
                block_max_key<NW>(best, nxt, red64, red);
                best_all = best;
                if ((int32_t)(best_all >> 32) >= bot) break;   // nothing below the band beats it
                top = nxt;
                width <<= 1;
            }
            if (!DENSE || base <= lo_n) break;
            __syncthreads();      // every read of this window done before the next one's clear
        }
        const int32_t result = best_all ? (int32_t)(best_all & 0xffffffffu) : -1;
        const int32_t rscore = (int32_t)(best_all >> 32);
        if (threadIdx.x == 0) {
            a.pair[n] = result;
            a.score[n] = result >= 0 ? rscore : 0;
            bytes += 8ull + 8ull;   // I(n) offsets, pair/score writes
        }
        __syncthreads();
    }
    if (a.bytes) {
        bytes = warp_sum(bytes);
        if (lane_id() == 0 && bytes) atomicAdd(a.bytes, bytes);
    }
}

// Largest per-node pin-visit count sum_{e in I(n)} |e| (bounds the distinct
// neighbours and sizes the hash tables).
static __global__ void k_max_work(int32_t V, const int32_t *ioff, const int32_t *inc, const int32_t *poff,
                           unsigned long long *out) {
    int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t n = gw; n < V; n += nw) {
        unsigned long long s = 0;
        for (int32_t k = ioff[n] + lane_id(); k < ioff[n + 1]; k += 32) {
            int32_t e = inc[k];
            s += (unsigned long long)(poff[e + 1] - poff[e]);
        }
        s = warp_sum(s);
        if (lane_id() == 0) atomicMax(out, s);
    }
}

// Rows of in(): bit e of row n is set iff e in in(n).
static __global__ void k_in_bitmap(int32_t V, const int32_t *noff, const int32_t *inn, int32_t words,
                            uint32_t *bm) {
    int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t n = gw; n < V; n += nw) {
        uint32_t *row = bm + n * words;
        for (int32_t j = noff[n] + lane_id(); j < noff[n + 1]; j += 32) {
            int32_t e = inn[j];
            atomicOr(&row[e >> 5], 1u << (e & 31));
        }
    }
}

}  // namespace hgp
