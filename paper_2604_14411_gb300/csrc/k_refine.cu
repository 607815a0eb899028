// Constrained refinement (Sec. IV).
//
// pins(p, e) is kept sparse: for every hyperedge a list of (part, count,
// count of destination pins) runs, sorted by part, in the hyperedge's own
// CSR segment.  It is built by two stable radix sorts of the (edge, part)
// pairs (by part, then by edge) and a warp per edge that compacts the runs.
// pins_in(p, e) = pins(p, e) minus the source pin when the source is not
// also a destination; inb(p) = #{e : pins_in(p, e) > 0} (Sec. IV-B.1).
//
// Proposals (Eq. (3)): a CTA per node accumulates, in a shared-memory table
// over parts, pres(n, p) = sum of omega(e) over e in I(n) with pins(p,e) > 0;
// then loss(n, p) = W_I(n) - pres(n, p) and gain = saving(n) - loss(n, p).
// Parts sharing no hyperedge with n have gain <= 0, so only the parts in the
// runs of n's hyperedges are candidates; parts with size(p) + w(n) > Omega
// are excluded; the best gain wins, ties to the smaller part id; a move is
// proposed iff its gain is > 0.
//
// Sequence: stable radix sort by gain (descending), node id ascending.
// In-sequence gain of move k: a CTA walks I(n_k) and the pins of each
// hyperedge, counts how the moves before k changed pins(ps, e), pins(pd, e)
// and their destination-only variants, and applies the exact change of
// Eq. (1); the same walk yields how many inbound hyperedges ps loses and pd
// gains.  Validity of every prefix then follows from per-part events
// (part, k, d_size, d_inbound): stable sort by part, per-part prefix sums,
// transitions valid <-> invalid, and a prefix sum over k of the transition
// deltas gives the number of violated parts after each move (Sec. IV-B.4).
// The applied prefix is the valid one of largest summed gain (the longest
// among equals), applied only if that gain is > 0.
#include "hgp_internal.cuh"

namespace hgp {

constexpr int kPropThreads = 1024;
constexpr int kPartsDenseMax = 12288;   // pres + touched list: 96 KB of smem

static int grid1d(int64_t n) {
    int b = div_up(n, 256);
    int cap = num_sms() * 8;
    return b < 1 ? 1 : (b > cap ? cap : b);
}

static int grid_warps(int64_t items) {
    int b = div_up(items * 32, 256);
    int cap = num_sms() * 16;
    return b < 1 ? 1 : (b > cap ? cap : b);
}

// ---------------------------------------------------------------- runs
__global__ void k_part_sizes(int32_t V, const int32_t *rho, const int32_t *w, int32_t *size) {
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&size[rho[n]], w[n]);
}

__global__ void k_pin_parts(int64_t P, const int32_t *pins, const int32_t *rho,
                            const int32_t *row_of, uint32_t *kp, int32_t *ve) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < P;
         j += (int64_t)gridDim.x * blockDim.x) {
        kp[j] = (uint32_t)rho[pins[j]];
        ve[j] = row_of[j];
    }
}

// Parts of each edge's pins after sorting; with a combined key the part is
// key - e * K, otherwise the sorted parts are given directly.
struct PartsView {
    const int32_t *parts;      // two-sort path
    const uint32_t *ekp;       // combined-key path
    int32_t K;
    __device__ __forceinline__ int32_t at(int64_t e, int32_t j) const {
        return parts ? parts[j] : (int32_t)(ekp[j] - (uint32_t)e * (uint32_t)K);
    }
};

__global__ void k_pin_ekp(int64_t P, const int32_t *pins, const int32_t *rho, const int32_t *row_of,
                          int32_t K, uint32_t *key) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < P;
         j += (int64_t)gridDim.x * blockDim.x)
        key[j] = (uint32_t)row_of[j] * (uint32_t)K + (uint32_t)rho[pins[j]];
}

__global__ void k_runs(int32_t E, const int32_t *poff, PartsView pv,
                       const int32_t *src, const uint8_t *sdst, const int32_t *rho,
                       int32_t *rpart, int32_t *rcnt, int32_t *rcin, int32_t *rpos,
                       int32_t *nrun, int32_t *inb, int32_t K, int32_t use_smem) {
    extern __shared__ int32_t inb_s[];       // per-CTA inbound counts (use_smem)
    if (use_smem) {
        for (int32_t i = threadIdx.x; i < K; i += blockDim.x) inb_s[i] = 0;
        __syncthreads();
    }
    int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned lt = (1u << lane_id()) - 1u;
    for (int64_t e = gw; e < E; e += nw) {
        int32_t p0 = poff[e], p1 = poff[e + 1];
        int32_t r = 0;
        for (int32_t base = p0; base < p1; base += 32) {
            int32_t j = base + lane_id();
            bool st = false;
            int32_t p = 0;
            if (j < p1) {
                p = pv.at(e, j);
                st = (j == p0) || pv.at(e, j - 1) != p;
            }
            unsigned ball = __ballot_sync(0xffffffffu, st);
            if (st) {
                int32_t q = p0 + r + __popc(ball & lt);
                rpart[q] = p;
                rpos[q] = j;
            }
            r += __popc(ball);
        }
        __syncwarp();
        int32_t srcpart = rho[src[e]];
        const uint8_t role = sdst[e];
        for (int32_t q = lane_id(); q < r; q += 32) {
            int32_t end = (q + 1 < r) ? rpos[p0 + q + 1] : p1;
            int32_t c = end - rpos[p0 + q];
            int32_t p = rpart[p0 + q];
            // pins of the run that have e in their in(): the source's node by
            // bit 0 of the role, every other node by bit 1
            const int32_t has_src = p == srcpart ? 1 : 0;
            int32_t ci = ((role & 2) ? c - has_src : 0) + ((role & 1) ? has_src : 0);
            rcnt[p0 + q] = c;
            rcin[p0 + q] = ci;
            if (inb && ci > 0) atomicAdd(use_smem ? &inb_s[p] : &inb[p], 1);
        }
        if (lane_id() == 0) nrun[e] = r;
    }
    if (use_smem) {
        __syncthreads();
        for (int32_t i = threadIdx.x; i < K; i += blockDim.x)
            if (inb_s[i]) atomicAdd(&inb[i], inb_s[i]);
    }
}

// The same runs for levels whose hyperedges have at most kRunsEdgeMax pins,
// without the global sort: a warp loads the parts of its hyperedge's pins
// into shared memory, sorts them (bitonic, padded to a power of two), and
// cuts the sorted parts into runs -- the ascending (part, count) sequence the
// stable sort by (edge, part) gives.
constexpr int kRunsEdgeMax = 256;
constexpr int kRunsWarps = 8;

__global__ void __launch_bounds__(kRunsWarps * 32)
k_runs_small(int32_t E, const int32_t *poff, const int32_t *pins, const int32_t *src,
             const uint8_t *sdst, const int32_t *rho, int32_t *rpart, int32_t *rcnt,
             int32_t *rcin, int32_t *rpos, int32_t *nrun, int32_t *inb, int32_t K,
             int32_t use_smem) {
    extern __shared__ int32_t inb_s[];       // per-CTA inbound counts (use_smem)
    __shared__ int32_t buf[kRunsWarps][kRunsEdgeMax];
    if (use_smem) {
        for (int32_t i = threadIdx.x; i < K; i += blockDim.x) inb_s[i] = 0;
        __syncthreads();
    }
    const int w = warp_id(), lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    int32_t *b = buf[w];
    int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = gw; e < E; e += nw) {
        const int32_t p0 = poff[e], p1 = poff[e + 1], len = p1 - p0;
        int32_t sz = 32;
        while (sz < len) sz <<= 1;
        for (int32_t i = lane; i < sz; i += 32) b[i] = i < len ? rho[pins[p0 + i]] : 0x7fffffff;
        __syncwarp();
        for (int32_t k = 2; k <= sz; k <<= 1)
            for (int32_t j = k >> 1; j > 0; j >>= 1) {
                for (int32_t i = lane; i < sz; i += 32) {
                    const int32_t x = i ^ j;
                    if (x > i) {
                        const int32_t u = b[i], v = b[x];
                        if ((u > v) == ((i & k) == 0)) { b[i] = v; b[x] = u; }
                    }
                }
                __syncwarp();
            }
        int32_t r = 0;
        for (int32_t base = 0; base < len; base += 32) {
            const int32_t i = base + lane;
            const bool st = i < len && (i == 0 || b[i - 1] != b[i]);
            const unsigned ball = __ballot_sync(0xffffffffu, st);
            if (st) {
                const int32_t q = p0 + r + __popc(ball & lt);
                rpart[q] = b[i];
                rpos[q] = i;
            }
            r += __popc(ball);
        }
        __syncwarp();
        const int32_t srcpart = rho[src[e]];
        const uint8_t role = sdst[e];
        for (int32_t q = lane; q < r; q += 32) {
            const int32_t end = (q + 1 < r) ? rpos[p0 + q + 1] : len;
            const int32_t c = end - rpos[p0 + q];
            const int32_t p = rpart[p0 + q];
            const int32_t has_src = p == srcpart ? 1 : 0;
            const int32_t ci = ((role & 2) ? c - has_src : 0) + ((role & 1) ? has_src : 0);
            rcnt[p0 + q] = c;
            rcin[p0 + q] = ci;
            if (inb && ci > 0) atomicAdd(use_smem ? &inb_s[p] : &inb[p], 1);
        }
        if (lane == 0) nrun[e] = r;
        __syncwarp();                        // b is reused by the warp's next hyperedge
    }
    if (use_smem) {
        __syncthreads();
        for (int32_t i = threadIdx.x; i < K; i += blockDim.x)
            if (inb_s[i]) atomicAdd(&inb[i], inb_s[i]);
    }
}

struct Runs {
    int32_t *rpart, *rcnt, *rcin, *nrun;
};

static cudaError_t build_runs(Arena &tmp, const Level &L, const int32_t *rho, int32_t K,
                              Runs &R, int32_t *inb, cudaStream_t s) {
    int64_t P = L.P;
    int32_t *row_of, *rpos;
    cudaError_t e = dalloc(tmp, &row_of, P);
    if (!e) e = dalloc(tmp, &rpos, P);
    if (!e) e = dalloc(tmp, &R.rpart, P);
    if (!e) e = dalloc(tmp, &R.rcnt, P);
    if (!e) e = dalloc(tmp, &R.rcin, P);
    if (!e) e = dalloc(tmp, &R.nrun, L.E);
    if (e) return e;
    if (L.max_edge <= kRunsEdgeMax) {
        if (L.E > 0) {
            const int32_t use_smem = (inb && K <= 16384) ? 1 : 0;
            const size_t smem = use_smem ? sizeof(int32_t) * (size_t)K : 0;
            int blocks = div_up((int64_t)L.E * 32, kRunsWarps * 32);
            if (blocks > num_sms() * 8) blocks = num_sms() * 8;
            if (use_smem && blocks > num_sms() * 4) blocks = num_sms() * 4;   // fewer flushes
            if (use_smem) {
                cudaError_t ea = allow_dynamic_smem(k_runs_small);
                if (ea) return ea;
            }
            k_runs_small<<<blocks, kRunsWarps * 32, smem, s>>>(L.E, L.poff, L.pins, L.src, L.sdst,
                                                               rho, R.rpart, R.rcnt, R.rcin, rpos,
                                                               R.nrun, inb, K, use_smem);
            count_launch();
        }
        return cudaGetLastError();
    }
    expand_rows(L.poff, L.E, row_of, s);
    PartsView pv{nullptr, nullptr, K};
    if ((int64_t)L.E * K <= (int64_t)UINT32_MAX) {
        // one stable sort of (edge * K + part): each edge's segment sorted by part
        uint32_t *k1, *k2;
        e = dalloc(tmp, &k1, P);
        if (!e) e = dalloc(tmp, &k2, P);
        if (e) return e;
        if (P > 0) {
            k_pin_ekp<<<grid1d(P), 256, 0, s>>>(P, L.pins, rho, row_of, K, k1);
            count_launch();
        }
        e = radix_sort_pairs(tmp, k1, nullptr, k2, nullptr, P,
                             bits_for((int64_t)L.E * K > 0 ? (int64_t)L.E * K - 1 : 0), s);
        if (e) return e;
        pv.ekp = k2;
    } else {
        // stable by part, then stable by edge
        int32_t *ve, *ve2, *ps2;
        uint32_t *kp, *kp2, *ke2;
        e = dalloc(tmp, &kp, P);
        if (!e) e = dalloc(tmp, &ve, P);
        if (!e) e = dalloc(tmp, &kp2, P);
        if (!e) e = dalloc(tmp, &ve2, P);
        if (!e) e = dalloc(tmp, &ke2, P);
        if (!e) e = dalloc(tmp, &ps2, P);
        if (e) return e;
        if (P > 0) {
            k_pin_parts<<<grid1d(P), 256, 0, s>>>(P, L.pins, rho, row_of, kp, ve);
            count_launch();
        }
        e = radix_sort_pairs(tmp, kp, ve, kp2, ve2, P, bits_for(K > 0 ? K - 1 : 0), s);
        if (!e) e = radix_sort_pairs(tmp, reinterpret_cast<uint32_t *>(ve2),
                                     reinterpret_cast<int32_t *>(kp2), ke2, ps2, P,
                                     bits_for(L.E > 0 ? L.E - 1 : 0), s);
        if (e) return e;
        pv.parts = ps2;
    }
    if (L.E > 0) {
        int32_t use_smem = (inb && K <= 16384) ? 1 : 0;
        size_t smem = use_smem ? sizeof(int32_t) * (size_t)K : 0;
        int blocks = grid_warps(L.E);
        if (use_smem && blocks > num_sms() * 4) blocks = num_sms() * 4;   // fewer flushes
        if (use_smem) {
            cudaError_t ea = allow_dynamic_smem(k_runs);
            if (ea) return ea;
        }
        k_runs<<<blocks, 256, smem, s>>>(L.E, L.poff, pv, L.src, L.sdst, rho, R.rpart, R.rcnt,
                                         R.rcin, rpos, R.nrun, inb, K, use_smem);
        count_launch();
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- proposals
struct PropArgs {
    int32_t V, K;
    const int32_t *w, *ioff, *inc, *poff, *ew, *rho, *size;
    const int32_t *rpart, *rcnt, *nrun;
    int64_t omega;
    int32_t *gain, *pd;
    int32_t *gpres;     // per-CTA global tables when K is large
    int32_t *next;      // work counter: nodes are taken dynamically
    unsigned long long *bytes;   // algorithmic bytes (timing runs only)
    // Reuse of the previous (one level coarser) pass's proposals: when that pass
    // applied no move, a node that was not split by the last matching keeps
    // exactly its coarse node's proposal (part presence on its hyperedges, part
    // sizes and its own savings are unchanged by splitting a pair inside one part).
    const int32_t *prev_gain, *prev_pd;   // proposals of the coarser level (null = none)
    const int32_t *gamma, *match;         // this level's map to the coarser level
    const int32_t *prev_applied;          // device flag: the coarser pass applied moves
    const int32_t *list;                  // nodes left to compute (the others were reused)
    int32_t *count;
};

// Reused proposals are copied here, one thread per node; every other node is
// appended to the work list of k_propose, so reuse costs the CTAs nothing.
__global__ void k_prop_worklist(PropArgs a) {
    const bool reuse = a.prev_gain && *a.prev_applied == 0;
    unsigned long long nbytes = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.V;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t n = (int32_t)i;
        if (reuse && a.match[n] == n) {
            int32_t c = a.gamma[n];
            a.gain[n] = a.prev_gain[c];
            a.pd[n] = a.prev_pd[c];
            nbytes += 24ull;
        } else {
            const_cast<int32_t *>(a.list)[atomicAdd(a.count, 1)] = n;
        }
    }
    if (a.bytes) {
        nbytes = warp_sum(nbytes);
        if (lane_id() == 0 && nbytes) atomicAdd(a.bytes, nbytes);
    }
}

template <bool DENSE, int NT>
__global__ void __launch_bounds__(NT) k_propose(PropArgs a) {
    constexpr int NW = NT / 32;
    extern __shared__ __align__(16) int32_t smem_p[];
    __shared__ unsigned long long red64[NW];
    __shared__ long long red_s[NW], red_w[NW];
    __shared__ int32_t s_nt;
    // pres(n, p) per part, and the list of parts touched for this node
    int32_t *pres = DENSE ? smem_p : a.gpres + (int64_t)blockIdx.x * 2 * a.K;
    int32_t *touched = pres + a.K;
    // the next node is fetched while the current one is worked on (double buffer)
    __shared__ int32_t s_nb[2];
    unsigned long long nbytes = 0;
    for (int32_t i = threadIdx.x; i < a.K; i += NT) pres[i] = 0;
    const int32_t work = *a.count;
    if (threadIdx.x == 0) {
        s_nt = 0;
        const int32_t t = atomicAdd(a.next, 1);
        s_nb[0] = t < work ? a.list[t] : a.V;
    }
    __syncthreads();
    for (int cur = 0;; cur ^= 1) {
        const int32_t n = s_nb[cur];
        if (n >= a.V) break;
        int32_t t_next = 0;
        if (threadIdx.x == 0) t_next = atomicAdd(a.next, 1);
        int32_t ps = a.rho[n];
        int32_t i0 = a.ioff[n], i1 = a.ioff[n + 1];
        long long sav = 0, wI = 0;
        // each lane fetches one hyperedge's (omega, run range); the warp walks them
        int32_t mine = (i1 - i0 - warp_id() + NW - 1) / NW;
        for (int32_t c0 = 0; c0 < mine; c0 += 32) {
            int32_t k = i0 + warp_id() + NW * (c0 + lane_id());
            int32_t we = 0, r0 = 0, r1 = 0;
            if (c0 + lane_id() < mine) {
                int32_t e = a.inc[k];
                we = a.ew[e];
                r0 = a.poff[e];
                r1 = r0 + a.nrun[e];
                wI += we;
            }
            int32_t cnt = min(32, mine - c0);
            if (a.bytes && c0 + lane_id() < mine) nbytes += 16ull + 4ull * (unsigned long long)(r1 - r0);
            for (int32_t t = 0; t < cnt; ++t) {
                int32_t wt = __shfl_sync(0xffffffffu, we, t);
                int32_t b0 = __shfl_sync(0xffffffffu, r0, t);
                int32_t b1 = __shfl_sync(0xffffffffu, r1, t);
                for (int32_t q = b0 + lane_id(); q < b1; q += 32) {
                    int32_t p = a.rpart[q];
                    if (p == ps) {
                        if (a.rcnt[q] == 1) sav += wt;
                    } else if (atomicAdd(&pres[p], wt) == 0) {
                        touched[atomicAdd(&s_nt, 1)] = p;
                    }
                }
            }
        }
        sav = warp_sum(sav);
        wI = warp_sum(wI);
        if (lane_id() == 0) { red_s[warp_id()] = sav; red_w[warp_id()] = wI; }
        __syncthreads();
        // best admissible part: max pres, ties to the smaller id
        int32_t nt = s_nt;
        int32_t wn = a.w[n];
        unsigned long long best = 0;
        for (int32_t t = threadIdx.x; t < nt; t += NT) {
            int32_t p = touched[t];
            if ((int64_t)a.size[p] + wn <= a.omega) {
                unsigned long long key = ((unsigned long long)(uint32_t)pres[p] << 32) |
                                         (uint32_t)(0x7fffffff - p);
                best = key > best ? key : best;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long y = __shfl_xor_sync(0xffffffffu, best, o);
            best = y > best ? y : best;
        }
        if (lane_id() == 0) red64[warp_id()] = best;
        __syncthreads();
        for (int32_t t = threadIdx.x; t < nt; t += NT) pres[touched[t]] = 0;
        if (threadIdx.x == 0) {
            unsigned long long b = 0;
            long long S = 0, W = 0;
            for (int q = 0; q < NW; ++q) {
                b = red64[q] > b ? red64[q] : b;
                S += red_s[q];
                W += red_w[q];
            }
            int32_t g = 0, pd = -1;
            if (b != 0) {
                long long presb = (long long)(b >> 32);
                long long gain = S - (W - presb);
                if (gain > 0) { g = (int32_t)gain; pd = 0x7fffffff - (int32_t)(b & 0xffffffffu); }
            }
            a.gain[n] = g;
            a.pd[n] = pd;
            s_nt = 0;
            s_nb[cur ^ 1] = t_next < work ? a.list[t_next] : a.V;
            nbytes += 8ull + 12ull;   // gain/pd writes; rho, w, I(n) offsets
        }
        __syncthreads();
    }
    if (a.bytes) {
        nbytes = warp_sum(nbytes);
        if (lane_id() == 0 && nbytes) atomicAdd(a.bytes, nbytes);
    }
}

// ---------------------------------------------------------------- sequence
__global__ void k_move_keys(int32_t V, const int32_t *gain, const int32_t *rank, uint32_t *key,
                            int32_t *node, int64_t wsum) {
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x) {
        int32_t g = gain[n];
        if (g > 0) {
            int32_t r = rank[n];
            key[r] = (uint32_t)(wsum - g);     // ascending key = descending gain (1 <= g <= wsum)
            node[r] = (int32_t)n;
        }
    }
}

__global__ void k_move_info(int32_t Mcap, const int32_t *dM, const int32_t *mv_n, const int32_t *rho,
                            const int32_t *pd, int32_t *mv_ps, int32_t *mv_pd, int32_t *idx_of) {
    const int32_t M = min(*dM, Mcap);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < M;
         k += (int64_t)gridDim.x * blockDim.x) {
        int32_t n = mv_n[k];
        mv_ps[k] = rho[n];
        mv_pd[k] = pd[n];
        idx_of[n] = (int32_t)k;
    }
}

__device__ __forceinline__ void run_lookup(const int32_t *rpart, const int32_t *rcnt,
                                           const int32_t *rcin, int32_t r0, int32_t r1, int32_t p,
                                           int32_t &c, int32_t &ci) {
    int32_t q = lower_bound_i32(rpart, r0, r1, p);
    if (q < r1 && rpart[q] == p) { c = rcnt[q]; ci = rcin[q]; }
    else { c = 0; ci = 0; }
}

// In-sequence gains from per-(edge, part) events.  Move k emits, for every
// e in I(n_k), a "leave" event on (e, ps_k) and an "enter" event on
// (e, pd_k), both tagged with k and with whether n_k is a destination of e.
// Stably sorted by (e, part) the events of one pair are in move order, so a
// segmented prefix sum gives pins(p, e) and pins_in(p, e) just before each
// move; the exact Eq. (1) change of the move and its inbound-set changes
// follow from those counts (== 1 when leaving, == 0 when entering).
__global__ void k_move_deg(int32_t M, const int32_t *mv_n, const int32_t *ioff, int32_t *deg) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < M;
         k += (int64_t)gridDim.x * blockDim.x) {
        int32_t n = mv_n[k];
        deg[k] = 2 * (ioff[n + 1] - ioff[n]);
    }
}

__global__ void k_seq_events(int32_t M, const int32_t *mv_n, const int32_t *mv_ps,
                             const int32_t *mv_pd, const int32_t *ioff, const int32_t *inc,
                             const int32_t *src, const uint8_t *sdst, const int32_t *evoff,
                             uint32_t *ev_p, int32_t *ev_e, int32_t *ev_k, uint8_t *ev_dst,
                             int32_t *ev_id) {
    int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = gw; k < M; k += nw) {
        int32_t n = mv_n[k], ps = mv_ps[k], pd = mv_pd[k];
        int32_t base = evoff[k], i0 = ioff[n], d = ioff[n + 1] - i0;
        for (int32_t t = lane_id(); t < d; t += 32) {
            int32_t e = inc[i0 + t];
            uint8_t isdst = counts_in(n, src[e], sdst[e]) ? 1 : 0;
            int32_t j = base + 2 * t;
            ev_p[j] = (uint32_t)ps;  ev_e[j] = e; ev_k[j] = (int32_t)k; ev_dst[j] = isdst; ev_id[j] = j;
            ev_p[j + 1] = (uint32_t)pd; ev_e[j + 1] = e; ev_k[j + 1] = (int32_t)k; ev_dst[j + 1] = isdst;
            ev_id[j + 1] = j + 1;
        }
    }
}

// Edge-centric in-sequence gains (hyperedges of at most kSeqEdgeMax pins): a
// warp per hyperedge gathers its moving pins and sorts them by move index;
// for every mover it adds up how the movers before it changed pins(ps, e),
// pins(pd, e) and their destination-only variants, and adds the move's
// Eq. (1) change on e and its inbound-set changes to the move's totals.
constexpr int kSeqEdgeMax = 256;
constexpr int kSeqWarps = 8;

__global__ void __launch_bounds__(kSeqWarps * 32)
k_seq_edge(int32_t E, const int32_t *poff, const int32_t *pins, const int32_t *idx_of,
           const int32_t *mv_ps, const int32_t *mv_pd, const int32_t *src, const uint8_t *sdst,
           const int32_t *nrun, const int32_t *rpart, const int32_t *rcnt, const int32_t *rcin,
           const int32_t *ew, int32_t *gseq, int32_t *lose_in, int32_t *gain_in) {
    // per warp: the movers of one hyperedge, first as sort keys (move index,
    // node) in the lower half, then expanded in move order to {ps, pd, weight,
    // move index}; the weight 1 + 2^16 * [destination] adds a mover to both
    // the plain and the destination-only count, kept in the low and high half
    // of one register (both are pin counts of e, so at most kSeqEdgeMax).
    // srp: the part ids of the hyperedge's runs, searched for the pre-move counts.
    __shared__ int4 smv[kSeqWarps][kSeqEdgeMax];
    __shared__ int32_t srp[kSeqWarps][kSeqEdgeMax];
    const int w = warp_id();
    unsigned long long *skey = reinterpret_cast<unsigned long long *>(smv[w]);
    const unsigned lt = (1u << lane_id()) - 1u;
    int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = gw; e < E; e += nw) {
        const int32_t p0 = poff[e], p1 = poff[e + 1];
        int32_t cnt = 0;
        for (int32_t base = p0; base < p1; base += 32) {
            const int32_t j = base + lane_id();
            const int32_t m = j < p1 ? pins[j] : -1;
            const int32_t k = m >= 0 ? idx_of[m] : -1;
            const unsigned ball = __ballot_sync(0xffffffffu, k >= 0);
            if (k >= 0) skey[cnt + __popc(ball & lt)] = ((unsigned long long)k << 32) | (uint32_t)m;
            cnt += __popc(ball);
        }
        if (cnt == 0) continue;                      // warp-uniform
        const int32_t nr = nrun[e];
        for (int32_t i = lane_id(); i < nr; i += 32) srp[w][i] = rpart[p0 + i];
        // bitonic sort of the keys, padded to a power of two: move order
        int32_t P = 1;
        while (P < cnt) P <<= 1;
        for (int32_t i = cnt + lane_id(); i < P; i += 32) skey[i] = ~0ull;
        __syncwarp();
        for (int32_t k2 = 2; k2 <= P; k2 <<= 1)
            for (int32_t j = k2 >> 1; j > 0; j >>= 1) {
                for (int32_t t = lane_id(); t < (P >> 1); t += 32) {
                    const int32_t a = ((t & ~(j - 1)) << 1) | (t & (j - 1)), b = a + j;
                    const unsigned long long x = skey[a], y = skey[b];
                    if ((x > y) == ((a & k2) == 0)) { skey[a] = y; skey[b] = x; }
                }
                __syncwarp();
            }
        // expand in place through registers (an entry outgrows its key)
        const int32_t se = src[e];
        const uint8_t role = sdst[e];
        unsigned long long mine[kSeqEdgeMax / 32];
#pragma unroll
        for (int c = 0; c < kSeqEdgeMax / 32; ++c) {
            const int32_t i = c * 32 + lane_id();
            mine[c] = i < cnt ? skey[i] : 0ull;
        }
        __syncwarp();
#pragma unroll
        for (int c = 0; c < kSeqEdgeMax / 32; ++c) {
            const int32_t i = c * 32 + lane_id();
            if (i < cnt) {
                const int32_t k = (int32_t)(mine[c] >> 32), m = (int32_t)(uint32_t)mine[c];
                smv[w][i] = make_int4(mv_ps[k], mv_pd[k], counts_in(m, se, role) ? 0x10001 : 1, k);
            }
        }
        __syncwarp();
        // mover i sees the movers before it in move order; chunks of 32 are
        // dealt out in alternating directions so every lane scans about as
        // many predecessors as the others
        const int32_t we = ew[e];
        for (int32_t c = 0; c * 32 < cnt; ++c) {
            const int32_t i = c * 32 + ((c & 1) ? 31 - lane_id() : lane_id());
            if (i >= cnt) continue;
            const int4 me = smv[w][i];
            // pre-move counts: ps is always a run of e (the mover is a pin of e)
            const int32_t qs = lower_bound_i32(srp[w], 0, nr, me.x);
            const int32_t qd = lower_bound_i32(srp[w], 0, nr, me.y);
            int32_t as = rcnt[p0 + qs] | (rcin[p0 + qs] << 16), ad = 0;
            if (qd < nr && srp[w][qd] == me.y) ad = rcnt[p0 + qd] | (rcin[p0 + qd] << 16);
            for (int32_t t = 0; t < i; ++t) {
                const int4 v = smv[w][t];
                if (v.y == me.x) as += v.z;
                if (v.x == me.x) as -= v.z;
                if (v.y == me.y) ad += v.z;
                if (v.x == me.y) ad -= v.z;
            }
            const int32_t cs = as & 0xffff, csi = as >> 16, cd = ad & 0xffff, cdi = ad >> 16;
            const bool dst = me.z != 1;
            // integer sums: the order of the atomic adds does not matter
            const int32_t g = we * ((cs == 1 ? 1 : 0) - (cd == 0 ? 1 : 0));
            if (g) atomicAdd(gseq + me.w, g);
            if (dst && csi == 1) atomicAdd(lose_in + me.w, 1);
            if (dst && cdi == 0) atomicAdd(gain_in + me.w, 1);
        }
        __syncwarp();
    }
}

__global__ void k_event_ekp(int64_t n, const int32_t *ev_e, const uint32_t *ev_p, int32_t K,
                            uint32_t *key) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        key[i] = (uint32_t)ev_e[i] * (uint32_t)K + ev_p[i];
}

__global__ void k_key_edge(int64_t n, const uint32_t *key, int32_t K, uint32_t *edge) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        edge[i] = key[i] / (uint32_t)K;
}

__global__ void k_gather_u32(int64_t n, const int32_t *src, const int32_t *idx, uint32_t *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (uint32_t)src[idx[i]];
}

// after the sorts: part of each event, the +-1 deltas (events at even ids
// leave, at odd ids enter) and the first-of-(e, p)-group flags
__global__ void k_seq_prep(int64_t nev, const uint32_t *eS, const int32_t *jS, const uint32_t *ev_p,
                           const uint8_t *ev_dst, int32_t *pS, int32_t *d_all, int32_t *d_in,
                           int32_t *head) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nev;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t j = jS[i];
        int32_t d = (j & 1) ? 1 : -1;
        int32_t p = (int32_t)ev_p[j];
        pS[i] = p;
        d_all[i] = d;
        d_in[i] = ev_dst[j] ? d : 0;
        head[i] = (i == 0 || eS[i - 1] != eS[i] || (int32_t)ev_p[jS[i - 1]] != p) ? 1 : 0;
    }
}

// position of the first event of every group (gidx = exclusive count of heads)
__global__ void k_group_starts(int64_t nev, const int32_t *head, const int32_t *gidx, int32_t *gstart) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nev;
         i += (int64_t)gridDim.x * blockDim.x)
        if (head[i]) gstart[gidx[i]] = (int32_t)i;
}

__global__ void k_seq_apply(int64_t nev, const uint32_t *eS, const int32_t *pS, const int32_t *jS,
                            const int32_t *head, const int32_t *gidx, const int32_t *gstart,
                            const int32_t *pre_all, const int32_t *pre_in, const int32_t *ev_k,
                            const uint8_t *ev_dst, const int32_t *poff, const int32_t *nrun,
                            const int32_t *rpart, const int32_t *rcnt, const int32_t *rcin,
                            const int32_t *ew, int32_t *c_gain, uint8_t *c_in) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nev;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t e = eS[i];
        int32_t p = pS[i];
        // first event of the same (e, p) group
        int64_t lo = gstart[gidx[i] + head[i] - 1];
        int32_t r0 = poff[e], r1 = r0 + nrun[e];
        int32_t q = lower_bound_i32(rpart, r0, r1, p);
        int32_t c0 = 0, c0in = 0;
        if (q < r1 && rpart[q] == p) { c0 = rcnt[q]; c0in = rcin[q]; }
        int32_t c = c0 + pre_all[i] - pre_all[lo];
        int32_t ci = c0in + pre_in[i] - pre_in[lo];
        int32_t j = jS[i];
        bool dst = ev_dst[j] != 0;
        // contribution of event j (stored at its own id; ids of move k are
        // contiguous, so a per-move reduction needs no atomics)
        if ((j & 1) == 0) {                                  // leaves ps
            c_gain[j] = (c == 1) ? ew[e] : 0;
            c_in[j] = (dst && ci == 1) ? 1 : 0;              // ps loses an inbound edge
        } else {                                             // enters pd
            c_gain[j] = (c == 0) ? -ew[e] : 0;
            c_in[j] = (dst && ci == 0) ? 1 : 0;              // pd gains an inbound edge
        }
    }
}

// one warp per move: gain = sum of its events' contributions; lose / gain_in =
// counts of its leave / enter events that change an inbound set
__global__ void k_move_reduce(int32_t M, const int32_t *evoff, const int32_t *c_gain,
                              const uint8_t *c_in, int32_t *gseq, int32_t *lose_in,
                              int32_t *gain_in) {
    int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = gw; k < M; k += nw) {
        int32_t g = 0, lo = 0, gi = 0;
        for (int32_t j = evoff[k] + lane_id(); j < evoff[k + 1]; j += 32) {
            g += c_gain[j];
            if (j & 1) gi += c_in[j]; else lo += c_in[j];
        }
        g = warp_sum(g);
        lo = warp_sum(lo);
        gi = warp_sum(gi);
        if (lane_id() == 0) { gseq[k] = g; lose_in[k] = lo; gain_in[k] = gi; }
    }
}

// events: 2 per move, (ps, k, -w, -lose) then (pd, k, +w, +gain_in)
__global__ void k_events(int32_t Mcap, const int32_t *dM, const int32_t *mv_n, const int32_t *mv_ps,
                         const int32_t *mv_pd, const int32_t *w, uint32_t pad, uint32_t *ekey,
                         int32_t *eid) {
    const int32_t M = *dM;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < Mcap;
         k += (int64_t)gridDim.x * blockDim.x) {
        ekey[2 * k] = k < M ? (uint32_t)mv_ps[k] : pad;        // padding sorts last
        ekey[2 * k + 1] = k < M ? (uint32_t)mv_pd[k] : pad;
        eid[2 * k] = (int32_t)(2 * k);
        eid[2 * k + 1] = (int32_t)(2 * k + 1);
    }
}

__global__ void k_event_deltas(int64_t nev, const int32_t *dM, const int32_t *eid_sorted,
                               const int32_t *mv_n, const int32_t *w, const int32_t *lose_in,
                               const int32_t *gain_in, int64_t *dsz, int64_t *dinb) {
    const int32_t M = *dM;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nev;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t id = eid_sorted[i];
        int32_t k = id >> 1;
        if (k >= M) { dsz[i] = 0; dinb[i] = 0; continue; }
        bool leave = (id & 1) == 0;
        int32_t wn = w[mv_n[k]];
        dsz[i] = leave ? -wn : wn;
        dinb[i] = leave ? -lose_in[k] : gain_in[k];
    }
}

__global__ void k_transitions(int64_t nev, const uint32_t *ekey_sorted, const int32_t *eid_sorted,
                              const int64_t *csz, const int64_t *cinb, const int32_t *size0,
                              const int32_t *inb0, int64_t omega, int64_t delta, uint32_t pad,
                              int32_t *vdelta) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nev;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t p = ekey_sorted[i];
        if (p == pad) continue;                        // padding events
        // first event of this part
        int64_t lo = 0, hi = i;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (ekey_sorted[mid] < p) lo = mid + 1; else hi = mid;
        }
        int64_t start = lo;
        int64_t bsz = start > 0 ? csz[start - 1] : 0;
        int64_t binb = start > 0 ? cinb[start - 1] : 0;
        int64_t s_after = size0[p] + (csz[i] - bsz);
        int64_t n_after = inb0[p] + (cinb[i] - binb);
        bool v_after = s_after <= omega && n_after <= delta;
        bool v_before;
        if (i == start) {
            v_before = (int64_t)size0[p] <= omega && (int64_t)inb0[p] <= delta;
        } else {
            int64_t sb = size0[p] + (csz[i - 1] - bsz);
            int64_t nb = inb0[p] + (cinb[i - 1] - binb);
            v_before = sb <= omega && nb <= delta;
        }
        int32_t k = eid_sorted[i] >> 1;
        if (v_before && !v_after) atomicAdd(&vdelta[k], 1);
        if (!v_before && v_after) atomicAdd(&vdelta[k], -1);
    }
}

__global__ void k_gseq_i64(int32_t M, const int32_t *gseq, const int32_t *vdelta, int64_t *g64,
                           int64_t *v64) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < M;
         k += (int64_t)gridDim.x * blockDim.x) {
        g64[k] = gseq[k];
        v64[k] = vdelta[k];
    }
}

// single CTA: k* = argmax over valid prefixes of (G, length); apply iff G > 0.
// stats[0..2] = (M, k*, gain); *applied accumulates k* over passes.
__global__ void k_select(int32_t Mcap, const int32_t *dM, const int64_t *G, const int64_t *viol,
                         int32_t *kstar, long long *stats, unsigned long long *applied,
                         int32_t *applied_flag) {
    const int32_t M = min(*dM, Mcap);
    __shared__ long long bg[1024];
    __shared__ int32_t bk[1024];
    long long g = 0;
    int32_t kk = 0;
    for (int32_t k = threadIdx.x; k < M; k += blockDim.x) {
        if (viol[k] != 0) continue;
        long long gk = G[k];
        if (kk == 0 || gk > g || (gk == g && k + 1 > kk)) { g = gk; kk = k + 1; }
    }
    bg[threadIdx.x] = g;
    bk[threadIdx.x] = kk;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            long long g2 = bg[threadIdx.x + o];
            int32_t k2 = bk[threadIdx.x + o];
            if (k2 != 0 && (bk[threadIdx.x] == 0 || g2 > bg[threadIdx.x] ||
                            (g2 == bg[threadIdx.x] && k2 > bk[threadIdx.x]))) {
                bg[threadIdx.x] = g2;
                bk[threadIdx.x] = k2;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        bool apply = bk[0] != 0 && bg[0] > 0;
        *kstar = apply ? bk[0] : 0;
        if (stats) { stats[0] = M; stats[1] = apply ? bk[0] : 0; stats[2] = apply ? bg[0] : 0; }
        if (applied && apply) atomicAdd(applied, (unsigned long long)bk[0]);
        if (applied_flag) *applied_flag = apply ? 1 : 0;
    }
}

__global__ void k_apply(int32_t Mcap, const int32_t *kstar, const int32_t *mv_n, const int32_t *mv_pd,
                        int32_t *rho) {
    const int32_t M = Mcap;
    int32_t ks = *kstar;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < ks && k < M;
         k += (int64_t)gridDim.x * blockDim.x)
        rho[mv_n[k]] = mv_pd[k];
}

__global__ void k_project(int32_t V, const int32_t *gamma, const int32_t *rho_coarse,
                          int32_t *rho_fine) {
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x)
        rho_fine[n] = rho_coarse[gamma[n]];
}

void run_project(int32_t V, const int32_t *gamma, const int32_t *rho_c, int32_t *rho_f,
                 cudaStream_t s) {
    if (V <= 0) return;
    k_project<<<grid1d(V), 256, 0, s>>>(V, gamma, rho_c, rho_f);
    count_launch();
}

__global__ void k_gain_flag(int32_t V, const int32_t *gain, int32_t *flag) {
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x)
        flag[n] = gain[n] > 0 ? 1 : 0;
}

// One refinement pass on level L; rho is updated in place on the device.
// d_stats (device, 3 x int64) receives (M, k*, gain); *d_applied adds k*.
cudaError_t run_refine_pass(Arena &tmp, const Level &L, const int32_t *ew, int64_t wsum,
                            int32_t *rho, int32_t K, int64_t omega, int64_t delta,
                            long long *d_stats, unsigned long long *d_applied, uint32_t debug,
                            PropTiming *pt, const PropReuse &ru, std::vector<int32_t> *gseq_out,
                            cudaStream_t s) {
    int32_t V = L.V;
    int32_t *size, *inb;
    cudaError_t e = dalloc(tmp, &size, K);
    if (!e) e = dalloc(tmp, &inb, K);
    if (e) return e;
    cudaMemsetAsync(size, 0, sizeof(int32_t) * (size_t)K, s);
    cudaMemsetAsync(inb, 0, sizeof(int32_t) * (size_t)K, s);
    k_part_sizes<<<grid1d(V), 256, 0, s>>>(V, rho, L.w, size);
    count_launch();
    Runs R{};
    e = build_runs(tmp, L, rho, K, R, inb, s);
    if (e) return e;
    // proposals
    int32_t *pg = ru.out_gain, *ppd = ru.out_pd;     // kept for the next finer level
    PropArgs pa{};
    pa.V = V; pa.K = K; pa.w = L.w; pa.ioff = L.ioff; pa.inc = L.inc; pa.poff = L.poff;
    pa.ew = ew; pa.rho = rho; pa.size = size; pa.rpart = R.rpart; pa.rcnt = R.rcnt;
    pa.nrun = R.nrun; pa.omega = omega; pa.gain = pg; pa.pd = ppd;
    pa.prev_gain = ru.prev_gain; pa.prev_pd = ru.prev_pd;
    pa.gamma = ru.gamma; pa.match = ru.match; pa.prev_applied = ru.applied_flag;
    int32_t *wl = nullptr, *wcount = nullptr;
    e = dalloc(tmp, &pa.next, 2);
    if (!e) e = dalloc(tmp, &wl, V);
    if (!e) e = cudaMemsetAsync(pa.next, 0, 2 * sizeof(int32_t), s);
    if (e) return e;
    wcount = pa.next + 1;
    pa.list = wl;
    pa.count = wcount;
    pa.bytes = pt ? pt->bytes : nullptr;
    if (pt) {
        cudaEvent_t ev;
        cudaEventCreate(&ev);
        cudaEventRecord(ev, s);
        pt->ev.push_back({ev, nullptr});
    }
    k_prop_worklist<<<grid1d(V), 256, 0, s>>>(pa);
    count_launch();
    int sms = num_sms();
    if (K <= kPartsDenseMax && !(debug & HGP_DEBUG_FORCE_GLOBAL)) {
        size_t smem = 2 * sizeof(int32_t) * (size_t)K;
        e = allow_dynamic_smem(k_propose<true, kPropThreads>);
        if (e) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_propose<true, kPropThreads>,
                                                          kPropThreads, smem);
        if (e) return e;
        if (per_sm < 1) per_sm = 1;
        int blocks = sms * per_sm;
        if (blocks > V) blocks = V;
        k_propose<true, kPropThreads><<<blocks, kPropThreads, smem, s>>>(pa);
    } else {
        int blocks = sms * 4;
        if (blocks > V) blocks = V;
        e = dalloc(tmp, &pa.gpres, (size_t)blocks * 2 * K);
        if (e) return e;
        k_propose<false, kPropThreads><<<blocks, kPropThreads, 0, s>>>(pa);
    }
    count_launch();
    if (pt) {
        cudaEventCreate(&pt->ev.back().second);
        cudaEventRecord(pt->ev.back().second, s);
    }
    // compact proposals in node order.  Levels whose hyperedges are small keep
    // the move count M on the device (arrays sized by V, padding sorted last);
    // the event path needs M on the host to size its events.
    int32_t *flag, *rank, *dM;
    e = dalloc(tmp, &flag, V);
    if (!e) e = dalloc(tmp, &rank, V);
    if (!e) e = dalloc(tmp, &dM, 1);
    if (e) return e;
    k_gain_flag<<<grid1d(V), 256, 0, s>>>(V, pg, flag);
    count_launch();
    e = exclusive_scan_i32(tmp, flag, rank, V, dM, s);
    if (e) return e;
    const bool edge_path = L.max_edge <= kSeqEdgeMax;
    int32_t M = V;                       // capacity: exact M on the event path
    if (!edge_path) {
        e = cudaMemcpyAsync(&M, dM, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaStreamSynchronize(s);
        if (e) return e;
        if (M == 0) {
            e = cudaMemsetAsync(d_stats, 0, 3 * sizeof(long long), s);
            if (!e) e = cudaMemsetAsync(ru.applied_flag, 0, sizeof(int32_t), s);
            return e;
        }
    }
    uint32_t *mkey, *mkey2;
    int32_t *mnode, *mv_n, *mv_ps, *mv_pd, *idx_of, *gseq, *lose, *gin;
    e = dalloc(tmp, &mkey, M);
    if (!e) e = dalloc(tmp, &mkey2, M);
    if (!e) e = dalloc(tmp, &mnode, M);
    if (!e) e = dalloc(tmp, &mv_n, M);
    if (!e) e = dalloc(tmp, &mv_ps, M);
    if (!e) e = dalloc(tmp, &mv_pd, M);
    if (!e) e = dalloc(tmp, &idx_of, V);
    if (!e) e = dalloc(tmp, &gseq, 3 * (size_t)M);     // gseq, lose, gin: one block
    if (e) return e;
    lose = gseq + M;
    gin = gseq + 2 * (size_t)M;
    const int mbits = bits_for(wsum);
    if (edge_path) {            // unused slots: maximal key, sorted after every move
        fill_i32(reinterpret_cast<int32_t *>(mkey), (int32_t)((1u << mbits) - 1u), M, s);
        fill_i32(mnode, -1, M, s);
    }
    k_move_keys<<<grid1d(V), 256, 0, s>>>(V, pg, rank, mkey, mnode, wsum);
    count_launch();
    e = radix_sort_pairs(tmp, mkey, mnode, mkey2, mv_n, M, mbits, s);
    if (e) return e;
    fill_i32(idx_of, -1, V, s);
    k_move_info<<<grid1d(M), 256, 0, s>>>(M, dM, mv_n, rho, ppd, mv_ps, mv_pd, idx_of);
    count_launch();
    // in-sequence gains: edge-centric when every hyperedge is small, otherwise
    // from per-(edge, part) events
    if (L.max_edge <= kSeqEdgeMax) {
        e = cudaMemsetAsync(gseq, 0, sizeof(int32_t) * 3 * (size_t)M, s);   // gseq, lose, gin
        if (e) return e;
        int blocks = div_up((int64_t)L.E * 32, kSeqWarps * 32);
        if (blocks > num_sms() * 8) blocks = num_sms() * 8;
        if (blocks < 1) blocks = 1;
        k_seq_edge<<<blocks, kSeqWarps * 32, 0, s>>>(L.E, L.poff, L.pins, idx_of, mv_ps, mv_pd,
                                                     L.src, L.sdst, R.nrun, R.rpart, R.rcnt, R.rcin,
                                                     ew, gseq, lose, gin);
        count_launch();
    } else
    {
        int32_t *deg, *evoff, *dNev;
        e = dalloc(tmp, &deg, M);
        if (!e) e = dalloc(tmp, &evoff, (size_t)M + 1);
        if (e) return e;
        k_move_deg<<<grid1d(M), 256, 0, s>>>(M, mv_n, L.ioff, deg);
        count_launch();
        e = counts_to_offsets(tmp, deg, evoff, M, s);
        if (e) return e;
        dNev = evoff + M;
        int32_t hnev = 0;
        e = cudaMemcpyAsync(&hnev, dNev, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaStreamSynchronize(s);
        if (e) return e;
        int64_t nq = hnev;
        uint32_t *ev_p, *p1, *e1, *eS;
        int32_t *ev_e, *ev_k, *ev_id, *j1, *jS, *pS, *d_all, *d_in, *pre_all, *pre_in;
        uint8_t *ev_dst;
        e = dalloc(tmp, &ev_p, nq);
        if (!e) e = dalloc(tmp, &ev_e, nq);
        if (!e) e = dalloc(tmp, &ev_k, nq);
        if (!e) e = dalloc(tmp, &ev_dst, nq);
        if (!e) e = dalloc(tmp, &ev_id, nq);
        if (!e) e = dalloc(tmp, &p1, nq);
        if (!e) e = dalloc(tmp, &j1, nq);
        if (!e) e = dalloc(tmp, &e1, nq);
        if (!e) e = dalloc(tmp, &eS, nq);
        if (!e) e = dalloc(tmp, &jS, nq);
        if (!e) e = dalloc(tmp, &pS, nq);
        if (!e) e = dalloc(tmp, &d_all, nq);
        if (!e) e = dalloc(tmp, &d_in, nq);
        if (!e) e = dalloc(tmp, &pre_all, nq);
        if (!e) e = dalloc(tmp, &pre_in, nq);
        if (e) return e;
        k_seq_events<<<grid_warps(M), 256, 0, s>>>(M, mv_n, mv_ps, mv_pd, L.ioff, L.inc, L.src,
                                                   L.sdst, evoff, ev_p, ev_e, ev_k, ev_dst, ev_id);
        count_launch();
        // grouped by (e, p), move order inside each group
        if ((int64_t)L.E * K <= (int64_t)UINT32_MAX) {
            k_event_ekp<<<grid1d(nq), 256, 0, s>>>(nq, ev_e, ev_p, K, p1);
            count_launch();
            e = radix_sort_pairs(tmp, p1, ev_id, e1, jS, nq,
                                 bits_for((int64_t)L.E * K > 0 ? (int64_t)L.E * K - 1 : 0), s);
            if (e) return e;
            k_key_edge<<<grid1d(nq), 256, 0, s>>>(nq, e1, K, eS);
            count_launch();
        } else {    // stable by part, then stable by edge
            e = radix_sort_pairs(tmp, ev_p, ev_id, p1, j1, nq, bits_for(K > 0 ? K - 1 : 0), s);
            if (e) return e;
            k_gather_u32<<<grid1d(nq), 256, 0, s>>>(nq, ev_e, j1, e1);
            count_launch();
            e = radix_sort_pairs(tmp, e1, j1, eS, jS, nq, bits_for(L.E > 0 ? L.E - 1 : 0), s);
            if (e) return e;
        }
        int32_t *head, *gidx, *gstart;
        e = dalloc(tmp, &head, nq);
        if (!e) e = dalloc(tmp, &gidx, nq);
        if (!e) e = dalloc(tmp, &gstart, nq);
        if (e) return e;
        k_seq_prep<<<grid1d(nq), 256, 0, s>>>(nq, eS, jS, ev_p, ev_dst, pS, d_all, d_in, head);
        count_launch();
        e = exclusive_scan_i32(tmp, d_all, pre_all, nq, nullptr, s);
        if (!e) e = exclusive_scan_i32(tmp, d_in, pre_in, nq, nullptr, s);
        if (!e) e = exclusive_scan_i32(tmp, head, gidx, nq, nullptr, s);
        if (e) return e;
        k_group_starts<<<grid1d(nq), 256, 0, s>>>(nq, head, gidx, gstart);
        count_launch();
        int32_t *c_gain;
        uint8_t *c_in;
        e = dalloc(tmp, &c_gain, nq);
        if (!e) e = dalloc(tmp, &c_in, nq);
        if (e) return e;
        k_seq_apply<<<grid1d(nq), 256, 0, s>>>(nq, eS, pS, jS, head, gidx, gstart, pre_all, pre_in,
                                               ev_k, ev_dst, L.poff, R.nrun, R.rpart, R.rcnt, R.rcin,
                                               ew, c_gain, c_in);
        count_launch();
        k_move_reduce<<<grid_warps(M), 256, 0, s>>>(M, evoff, c_gain, c_in, gseq, lose, gin);
        count_launch();
    }
    // prefix validity from per-part events
    int64_t nev = 2 * (int64_t)M;
    uint32_t *ekey, *ekey2;
    int32_t *eid, *eid2, *vdelta;
    int64_t *dsz, *dinb, *csz, *cinb, *g64, *v64, *G, *viol;
    e = dalloc(tmp, &ekey, nev);
    if (!e) e = dalloc(tmp, &ekey2, nev);
    if (!e) e = dalloc(tmp, &eid, nev);
    if (!e) e = dalloc(tmp, &eid2, nev);
    if (!e) e = dalloc(tmp, &dsz, nev);
    if (!e) e = dalloc(tmp, &dinb, nev);
    if (!e) e = dalloc(tmp, &csz, nev);
    if (!e) e = dalloc(tmp, &cinb, nev);
    if (!e) e = dalloc(tmp, &vdelta, M);
    if (!e) e = dalloc(tmp, &g64, M);
    if (!e) e = dalloc(tmp, &v64, M);
    if (!e) e = dalloc(tmp, &G, M);
    if (!e) e = dalloc(tmp, &viol, M);
    if (e) return e;
    const int pbits = bits_for(K);
    const uint32_t pad = (1u << pbits) - 1u;          // > every part id
    k_events<<<grid1d(M), 256, 0, s>>>(M, dM, mv_n, mv_ps, mv_pd, L.w, pad, ekey, eid);
    count_launch();
    e = radix_sort_pairs(tmp, ekey, eid, ekey2, eid2, nev, pbits, s);
    if (e) return e;
    k_event_deltas<<<grid1d(nev), 256, 0, s>>>(nev, dM, eid2, mv_n, L.w, lose, gin, dsz, dinb);
    count_launch();
    e = inclusive_scan_i64(tmp, dsz, csz, nev, s);
    if (!e) e = inclusive_scan_i64(tmp, dinb, cinb, nev, s);
    if (e) return e;
    cudaMemsetAsync(vdelta, 0, sizeof(int32_t) * (size_t)M, s);
    k_transitions<<<grid1d(nev), 256, 0, s>>>(nev, ekey2, eid2, csz, cinb, size, inb, omega, delta,
                                              pad, vdelta);
    count_launch();
    k_gseq_i64<<<grid1d(M), 256, 0, s>>>(M, gseq, vdelta, g64, v64);
    count_launch();
    e = inclusive_scan_i64(tmp, g64, G, M, s);
    if (!e) e = inclusive_scan_i64(tmp, v64, viol, M, s);
    if (e) return e;
    int32_t *dk;
    e = dalloc(tmp, &dk, 1);
    if (e) return e;
    k_select<<<1, 1024, 0, s>>>(M, dM, G, viol, dk, d_stats, d_applied, ru.applied_flag);
    count_launch();
    k_apply<<<grid1d(M), 256, 0, s>>>(M, dk, mv_n, mv_pd, rho);
    count_launch();
    if (gseq_out) {            // debug trace: the in-sequence gains of the sorted moves
        int32_t hm = 0;
        e = cudaMemcpyAsync(&hm, dM, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaStreamSynchronize(s);
        if (e) return e;
        if (hm > M) hm = M;
        gseq_out->assign(hm > 0 ? hm : 0, 0);
        if (hm > 0)
            e = cudaMemcpyAsync(gseq_out->data(), gseq, sizeof(int32_t) * (size_t)hm,
                                cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaStreamSynchronize(s);
        if (e) return e;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- output
__global__ void k_nonempty(int32_t K, const int32_t *size, int32_t *flag) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < K;
         p += (int64_t)gridDim.x * blockDim.x)
        flag[p] = size[p] > 0 ? 1 : 0;
}

__global__ void k_relabel(int32_t V, const int32_t *rho, const int32_t *newid, int32_t *part_ids) {
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x)
        part_ids[n] = newid[rho[n]];
}

__global__ void k_part_out(int32_t K, const int32_t *size, const int32_t *inb, const int32_t *newid,
                           int64_t *pw, int32_t *pin) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < K;
         p += (int64_t)gridDim.x * blockDim.x) {
        if (size[p] > 0) {
            int32_t q = newid[p];
            if (pw) pw[q] = size[p];
            if (pin) pin[q] = inb[p];
        }
    }
}

// Eq. (1): cost = sum_e omega(e) * (number of runs of e - 1)
__global__ void k_cost(int32_t E, const int32_t *nrun, const int32_t *ew, unsigned long long *cost) {
    unsigned long long c = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
         e += (int64_t)gridDim.x * blockDim.x)
        c += (unsigned long long)ew[e] * (unsigned long long)(nrun[e] - 1);
    c = warp_sum(c);
    if (lane_id() == 0 && c) atomicAdd(cost, c);
}

// Final output on level 0 for partition rho (part ids < K): compacted ids,
// per-part weight and distinct inbound count, connectivity and part count.
cudaError_t run_finalize(Arena &tmp, const Level &L, const int32_t *ew, const int32_t *rho,
                         int32_t K, int32_t *part_ids, int64_t *pw, int32_t *pin,
                         unsigned long long *d_cost, int32_t *d_nparts, cudaStream_t s) {
    int32_t *size, *inb, *flag, *newid;
    cudaError_t e = dalloc(tmp, &size, K);
    if (!e) e = dalloc(tmp, &inb, K);
    if (!e) e = dalloc(tmp, &flag, K);
    if (!e) e = dalloc(tmp, &newid, K);
    if (e) return e;
    cudaMemsetAsync(size, 0, sizeof(int32_t) * (size_t)K, s);
    cudaMemsetAsync(inb, 0, sizeof(int32_t) * (size_t)K, s);
    cudaMemsetAsync(d_cost, 0, sizeof(unsigned long long), s);
    k_part_sizes<<<grid1d(L.V), 256, 0, s>>>(L.V, rho, L.w, size);
    count_launch();
    Runs R{};
    e = build_runs(tmp, L, rho, K, R, inb, s);
    if (e) return e;
    k_nonempty<<<grid1d(K), 256, 0, s>>>(K, size, flag);
    count_launch();
    e = exclusive_scan_i32(tmp, flag, newid, K, d_nparts, s);
    if (e) return e;
    k_relabel<<<grid1d(L.V), 256, 0, s>>>(L.V, rho, newid, part_ids);
    count_launch();
    k_part_out<<<grid1d(K), 256, 0, s>>>(K, size, inb, newid, pw, pin);
    count_launch();
    if (L.E > 0) {
        k_cost<<<grid1d(L.E), 256, 0, s>>>(L.E, R.nrun, ew, d_cost);
        count_launch();
    }
    return cudaGetLastError();
}

}  // namespace hgp
