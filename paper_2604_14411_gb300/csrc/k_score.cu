// Candidate scoring (Sec. III-A, Eq. (2)) fused with the deferred validity
// checks of Sec. III-B.2.
//
// One CTA per node n (persistent grid, nodes strided over CTAs).
//   1. hist(n, m) = sum of omega(e) over e in I(n), m in e, m != n.
//      Each warp takes hyperedges of I(n); its lanes read the pins of one
//      hyperedge with coalesced int32 loads and add omega(e) into the
//      histogram:
//        dense mode  -- a |N_l|-entry int32 array in shared memory,
//                       indexed by node id (no hashing, one smem atomic
//                       per pin visit);
//        hash mode   -- a per-CTA open-addressing table in global memory
//                       (levels whose node count does not fit on chip).
//   2. Candidates are taken in the order (hist desc, id desc).  The first is
//      found by a CTA-wide argmax and checked; if it fails, the remaining
//      neighbours are compacted into shared memory, bitonic-sorted, and
//      checked 1 per warp in parallel batches; the first valid one in order
//      wins (the same answer as extracting one at a time).
//   3. Check of a pair (n, m): w(n) + w(m) <= Omega, and
//      |in(n)| + |in(m) \ in(n)| <= Delta, where membership in in(n) is a
//      bit test in a shared-memory bitmap over E (or a binary search in the
//      sorted in(n) when E is too large for the bitmap).  When
//      |in(n)| + |in(m)| <= Delta the pair is valid without any test.
#include "hgp_internal.cuh"

namespace hgp {

constexpr int kScoreThreads = 512;
constexpr int kScoreWarps = kScoreThreads / 32;
constexpr int kListCap = 2048;             // sorted candidate list (u64 keys)
constexpr int kBitmapMaxEdges = 1 << 18;   // bitmap of in(n) up to 256K edges (32 KB)

struct ScoreArgs {
    int32_t V, E;
    const int32_t *w, *poff, *pins, *ioff, *inc, *noff, *inn, *ew;
    int64_t omega, delta;
    int32_t *pair, *score;
    int32_t *status;
    int32_t *gkeys, *gvals;   // hash mode: per-CTA tables of gcap entries
    int32_t gcap;
    unsigned long long *bytes;
    int32_t use_bitmap;
    int32_t bm_words;
};

__device__ __forceinline__ uint32_t hash_u32(uint32_t x) {
    x ^= x >> 16; x *= 0x7feb352dU; x ^= x >> 15; x *= 0x846ca68bU; x ^= x >> 16;
    return x;
}

template <typename T>
__device__ T block_max_u64(T v, T *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T y = __shfl_xor_sync(0xffffffffu, v, o);
        v = y > v ? y : v;
    }
    __syncthreads();
    if (lane_id() == 0) red[warp_id()] = v;
    __syncthreads();
    T r = 0;
    for (int i = 0; i < kScoreWarps; ++i) r = red[i] > r ? red[i] : r;
    return r;
}

__device__ int32_t block_sum_i32(int32_t v, int32_t *red) {
    v = warp_sum(v);
    __syncthreads();
    if (lane_id() == 0) red[warp_id()] = v;
    __syncthreads();
    int32_t r = 0;
    for (int i = 0; i < kScoreWarps; ++i) r += red[i];
    return r;
}

// Warp-cooperative validity test of pair (n, m); all lanes return the same.
__device__ bool warp_check(const ScoreArgs &a, int32_t n, int32_t m, const uint32_t *bm,
                           unsigned long long &bytes) {
    if ((int64_t)a.w[n] + a.w[m] > a.omega) return false;
    int32_t n0 = a.noff[n], n1 = a.noff[n + 1];
    int32_t m0 = a.noff[m], m1 = a.noff[m + 1];
    int64_t in_n = n1 - n0, in_m = m1 - m0;
    if (in_n + in_m <= a.delta) return true;
    int64_t room = a.delta - in_n;          // edges of in(m) allowed outside in(n)
    int64_t extra = 0;
    for (int32_t base = m0; base < m1; base += 32) {
        int32_t j = base + lane_id();
        int32_t miss = 0;
        if (j < m1) {
            int32_t e = a.inn[j];
            bool member = bm ? ((bm[e >> 5] >> (e & 31)) & 1u) : contains_sorted(a.inn, n0, n1, e);
            miss = member ? 0 : 1;
        }
        extra += __popc(__ballot_sync(0xffffffffu, miss));
        if (extra > room) break;
    }
    if (lane_id() == 0) bytes += 4ull * (unsigned long long)(m1 - m0);
    return extra <= room;
}

template <bool DENSE>
__global__ void __launch_bounds__(kScoreThreads)
k_score(ScoreArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    // layout: [bitmap words][u64 list kListCap][dense hist V]
    uint32_t *bm = reinterpret_cast<uint32_t *>(smem);
    unsigned long long *list =
        reinterpret_cast<unsigned long long *>(smem + sizeof(uint32_t) * (size_t)a.bm_words);
    int32_t *hist = reinterpret_cast<int32_t *>(list + kListCap);
    __shared__ unsigned long long red64[kScoreWarps];
    __shared__ int32_t red32[kScoreWarps];
    __shared__ int32_t s_cnt, s_found, s_bm_ready;
    __shared__ int32_t s_wvalid[kScoreWarps];

    int32_t *gkeys = DENSE ? nullptr : a.gkeys + (int64_t)blockIdx.x * a.gcap;
    int32_t *gvals = DENSE ? nullptr : a.gvals + (int64_t)blockIdx.x * a.gcap;
    const int32_t cap = DENSE ? a.V : a.gcap;
    const uint32_t mask = (uint32_t)a.gcap - 1u;
    unsigned long long bytes = 0;

    for (int32_t n = blockIdx.x; n < a.V; n += gridDim.x) {
        // ---- clear ----
        for (int32_t i = threadIdx.x; i < cap; i += kScoreThreads) {
            if (DENSE) hist[i] = 0;
            else { gkeys[i] = -1; gvals[i] = 0; }
        }
        if (threadIdx.x == 0) s_bm_ready = 0;
        __syncthreads();
        // ---- Eq. (2) accumulation ----
        int32_t i0 = a.ioff[n], i1 = a.ioff[n + 1];
        for (int32_t k = i0 + warp_id(); k < i1; k += kScoreWarps) {
            int32_t e = a.inc[k];
            int32_t we = a.ew[e];
            int32_t p0 = a.poff[e], p1 = a.poff[e + 1];
            for (int32_t j = p0 + lane_id(); j < p1; j += 32) {
                int32_t m = a.pins[j];
                if (m == n) continue;
                if (DENSE) {
                    atomicAdd(&hist[m], we);
                } else {
                    uint32_t slot = hash_u32((uint32_t)m) & mask;
                    int32_t probes = 0;
                    for (;;) {
                        int32_t k0 = atomicCAS(&gkeys[slot], -1, m);
                        if (k0 == -1 || k0 == m) { atomicAdd(&gvals[slot], we); break; }
                        slot = (slot + 1) & mask;
                        if (++probes >= a.gcap) { set_status(a.status, kDevLimit); break; }
                    }
                }
            }
            if (lane_id() == 0)
                bytes += 16ull + 4ull * (unsigned long long)(p1 - p0);  // inc, omega, 2 offsets, pins
        }
        __syncthreads();
        // ---- first candidate: CTA-wide argmax of (hist, id) ----
        unsigned long long mx = 0;
        for (int32_t i = threadIdx.x; i < cap; i += kScoreThreads) {
            int32_t h, m;
            if (DENSE) { h = hist[i]; m = i; }
            else { m = gkeys[i]; h = m >= 0 ? gvals[i] : 0; }
            if (h > 0) {
                unsigned long long key = ((unsigned long long)(uint32_t)h << 32) | (uint32_t)m;
                mx = key > mx ? key : mx;
            }
        }
        unsigned long long best = block_max_u64(mx, red64);
        int32_t result = -1, rscore = 0;
        if (best != 0) {
            int32_t m = (int32_t)(best & 0xffffffffu);
            // the bitmap is needed only if some check must count the union
            int64_t in_n = a.noff[n + 1] - a.noff[n];
            int64_t in_m = a.noff[m + 1] - a.noff[m];
            bool need_bm = a.use_bitmap && (in_n + in_m > a.delta);
            if (need_bm) {
                for (int32_t i = threadIdx.x; i < a.bm_words; i += kScoreThreads) bm[i] = 0u;
                __syncthreads();
                for (int32_t j = a.noff[n] + threadIdx.x; j < a.noff[n + 1]; j += kScoreThreads) {
                    int32_t e = a.inn[j];
                    atomicOr(&bm[e >> 5], 1u << (e & 31));
                }
                if (threadIdx.x == 0) s_bm_ready = 1;
                __syncthreads();
            }
            if (warp_id() == 0) {
                bool ok = warp_check(a, n, m, a.use_bitmap ? bm : nullptr, bytes);
                if (lane_id() == 0) s_found = ok ? 1 : 0;
            }
            __syncthreads();
            if (s_found) {
                result = m;
                rscore = (int32_t)(best >> 32);
            } else {
                // ---- remaining candidates, in order ----
                if (a.use_bitmap && !s_bm_ready) {
                    for (int32_t i = threadIdx.x; i < a.bm_words; i += kScoreThreads) bm[i] = 0u;
                    __syncthreads();
                    for (int32_t j = a.noff[n] + threadIdx.x; j < a.noff[n + 1]; j += kScoreThreads) {
                        int32_t e = a.inn[j];
                        atomicOr(&bm[e >> 5], 1u << (e & 31));
                    }
                    __syncthreads();
                }
                int32_t cnt_local = 0;
                for (int32_t i = threadIdx.x; i < cap; i += kScoreThreads) {
                    int32_t h, mm;
                    if (DENSE) { h = hist[i]; mm = i; }
                    else { mm = gkeys[i]; h = mm >= 0 ? gvals[i] : 0; }
                    if (h > 0) {
                        unsigned long long key = ((unsigned long long)(uint32_t)h << 32) | (uint32_t)mm;
                        cnt_local += key < best ? 1 : 0;
                    }
                }
                int32_t cnt = block_sum_i32(cnt_local, red32);
                if (cnt <= kListCap) {
                    // compact, pad, bitonic sort (descending), check in batches
                    if (threadIdx.x == 0) s_cnt = 0;
                    __syncthreads();
                    for (int32_t i = threadIdx.x; i < cap; i += kScoreThreads) {
                        int32_t h, mm;
                        if (DENSE) { h = hist[i]; mm = i; }
                        else { mm = gkeys[i]; h = mm >= 0 ? gvals[i] : 0; }
                        if (h > 0) {
                            unsigned long long key = ((unsigned long long)(uint32_t)h << 32) | (uint32_t)mm;
                            if (key < best) list[atomicAdd(&s_cnt, 1)] = key;
                        }
                    }
                    __syncthreads();
                    int32_t len = 1;
                    while (len < cnt) len <<= 1;
                    for (int32_t i = cnt + threadIdx.x; i < len; i += kScoreThreads) list[i] = 0ull;
                    __syncthreads();
                    for (int32_t k = 2; k <= len; k <<= 1) {
                        for (int32_t jj = k >> 1; jj > 0; jj >>= 1) {
                            for (int32_t i = threadIdx.x; i < len; i += kScoreThreads) {
                                int32_t ixj = i ^ jj;
                                if (ixj > i) {
                                    unsigned long long x = list[i], y = list[ixj];
                                    bool desc = (i & k) == 0;
                                    if (desc ? (x < y) : (x > y)) { list[i] = y; list[ixj] = x; }
                                }
                            }
                            __syncthreads();
                        }
                    }
                    for (int32_t b = 0; b < cnt; b += kScoreWarps) {
                        int32_t idx = b + warp_id();
                        bool ok = false;
                        if (idx < cnt) {
                            int32_t mm = (int32_t)(list[idx] & 0xffffffffu);
                            ok = warp_check(a, n, mm, a.use_bitmap ? bm : nullptr, bytes);
                        }
                        if (lane_id() == 0) s_wvalid[warp_id()] = ok ? 1 : 0;
                        __syncthreads();
                        int32_t first = -1;
                        for (int q = 0; q < kScoreWarps; ++q)
                            if (s_wvalid[q]) { first = q; break; }
                        __syncthreads();
                        if (first >= 0) {
                            unsigned long long key = list[b + first];
                            result = (int32_t)(key & 0xffffffffu);
                            rscore = (int32_t)(key >> 32);
                            break;
                        }
                    }
                } else {
                    // many candidates: one extraction per round (same order)
                    unsigned long long thr = best;
                    for (int32_t round = 0; round < cnt; ++round) {
                        unsigned long long lm = 0;
                        for (int32_t i = threadIdx.x; i < cap; i += kScoreThreads) {
                            int32_t h, mm;
                            if (DENSE) { h = hist[i]; mm = i; }
                            else { mm = gkeys[i]; h = mm >= 0 ? gvals[i] : 0; }
                            if (h > 0) {
                                unsigned long long key = ((unsigned long long)(uint32_t)h << 32) | (uint32_t)mm;
                                if (key < thr && key > lm) lm = key;
                            }
                        }
                        unsigned long long nb = block_max_u64(lm, red64);
                        if (nb == 0) break;
                        if (warp_id() == 0) {
                            bool ok = warp_check(a, n, (int32_t)(nb & 0xffffffffu),
                                                 a.use_bitmap ? bm : nullptr, bytes);
                            if (lane_id() == 0) s_found = ok ? 1 : 0;
                        }
                        __syncthreads();
                        if (s_found) {
                            result = (int32_t)(nb & 0xffffffffu);
                            rscore = (int32_t)(nb >> 32);
                            break;
                        }
                        thr = nb;
                    }
                }
            }
        }
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
__global__ void k_max_work(int32_t V, const int32_t *ioff, const int32_t *inc, const int32_t *poff,
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

struct ScoreLaunch {
    bool dense;
    size_t smem;
    int blocks;
};

static size_t score_smem(bool dense, int32_t V, int32_t bm_words) {
    return sizeof(uint32_t) * (size_t)bm_words + sizeof(unsigned long long) * kListCap +
           (dense ? sizeof(int32_t) * (size_t)V : 0);
}

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
    a.use_bitmap = (L.E <= kBitmapMaxEdges && !(debug & HGP_DEBUG_NO_BITMAP)) ? 1 : 0;
    a.bm_words = a.use_bitmap ? (((L.E + 31) / 32 + 3) & ~3) : 0;   // keeps the u64 list 16-byte aligned
    // static smem of the kernel is small (< 1 KB); keep 2 KB of headroom
    size_t dense_smem = score_smem(true, L.V, a.bm_words);
    bool dense = dense_smem + 2048 <= (size_t)max_smem && !(debug & HGP_DEBUG_FORCE_GLOBAL);
    size_t smem = dense ? dense_smem : score_smem(false, L.V, a.bm_words);
    int sms = num_sms();
    int blocks = 0;
    cudaError_t e;
    if (dense) {
        e = cudaFuncSetAttribute(k_score<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e) return e;
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_score<true>, kScoreThreads, smem);
        if (per_sm < 1) per_sm = 1;
        blocks = sms * per_sm;
        if (blocks > L.V) blocks = L.V;
        k_score<true><<<blocks, kScoreThreads, smem, s>>>(a);
        count_launch();
        return cudaGetLastError();
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
    while (gcap < 2 * distinct) gcap <<= 1;
    if (gcap > (1ull << 30)) return cudaErrorMemoryAllocation;
    a.gcap = (int32_t)gcap;
    e = cudaFuncSetAttribute(k_score<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    blocks = sms * 2;
    if (blocks > L.V) blocks = L.V;
    e = dalloc(ar, &a.gkeys, (size_t)blocks * gcap);
    if (!e) e = dalloc(ar, &a.gvals, (size_t)blocks * gcap);
    if (e) return e;
    k_score<false><<<blocks, kScoreThreads, smem, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

}  // namespace hgp
