// Matching on the pairing pseudo-forest (Sec. III-A, III-B.3) and the gamma
// map of the coarse level (Sec. III-B.4).
//
// best(m): the child n (pair(n) = m) with the largest (score(n), n) -- one
//   64-bit atomicMax per node, independent of launch order (the paper's
//   upward placement of scores).
// lock(n): two-cycle roots lock; otherwise n locks to pair(n) iff n is its
//   candidate's best child and pair(n) did not lock to its own candidate.
//   Each thread follows the chain of "best child" links from its node to the
//   first node that settles the value (a root, or a node that is not its
//   candidate's best child) and takes the parity of the distance.  This is
//   the downward walk of the paper written as a closed form, so every thread
//   reaches the same decision regardless of scheduling.
// match(n) = pair(n) if lock(n); else best(n) if n has a child; else n.
// gamma(n) = rank of min(n, match(n)) among all such representatives.
#include "hgp_internal.cuh"

namespace hgp {

__global__ void k_best(int32_t V, const int32_t *pair, const int32_t *score,
                       unsigned long long *best) {
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x) {
        int32_t m = pair[n];
        if (m >= 0)
            atomicMax(&best[m], ((unsigned long long)(uint32_t)score[n] << 32) | (uint32_t)n);
    }
}

__global__ void k_lock_match(int32_t V, const int32_t *pair, const unsigned long long *best,
                             int32_t *match, int32_t *rep_flag, int32_t *status) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t n = (int32_t)i;
        // lock(n) by walking the best-child chain
        int32_t x = n, k = 0, t = 0;
        for (;;) {
            int32_t px = pair[x];
            if (px < 0) { t = 0; break; }
            if (pair[px] == x) { t = 1; break; }
            if ((int32_t)(best[px] & 0xffffffffu) != x) { t = 0; break; }
            x = px;
            if (++k > V) { set_status(status, kDevInternal); t = 0; break; }
        }
        int32_t lock = t ^ (k & 1);
        int32_t m;
        if (lock) m = pair[n];
        else if (best[n] != 0ull) m = (int32_t)(best[n] & 0xffffffffu);
        else m = n;
        match[n] = m;
        rep_flag[n] = m >= n ? 1 : 0;
    }
}

__global__ void k_gamma(int32_t V, const int32_t *match, const int32_t *rank, int32_t *gamma) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t n = (int32_t)i, m = match[n];
        gamma[n] = rank[m < n ? m : n];
    }
}

static int grid1d(int64_t n) {
    int b = div_up(n, 256);
    int cap = num_sms() * 8;
    return b < 1 ? 1 : (b > cap ? cap : b);
}

__global__ void k_best_key(int32_t V, const int32_t *pair, const int32_t *score,
                           const int32_t *key, unsigned long long *bkey);
__global__ void k_best_id(int32_t V, const int32_t *pair, const int32_t *score, const int32_t *key,
                          const unsigned long long *bkey, unsigned long long *best);

// ---------------- exact maximum-weight matching (tree DP) ----------------
// The alternative to the two walks that the paper leaves as future work:
// the largest total score over all matchings of the pairing pseudo-forest
// (edges {n, pair(n)} of weight score(n)).  A root two-cycle {a, b} is one
// edge; b = max(a, b) becomes a child of a.  For every node v:
//   up(v) = sum over children c of best(c)                 (int64)
//   g(v)  = max over children c of score(c) - max(0, g(c)), c*(v) its child
//           (ties: larger id), packed as ((g + 2^31) << 32 | c) so that one
//           64-bit atomicMax keeps both; 0 = no child
//   best(v) = up(v) + max(0, g(v))
// Bottom-up without barriers: every leaf starts a thread that folds its
// values into its parent with atomics and a fence, then counts the parent's
// pending children down; the thread that brings the count to zero owns the
// parent and continues from it (each node is finished exactly once).
// Top-down, in closed form as for the lock: v is taken by its parent iff the
// parent chose it (g > 0) and the parent is free; following these links up
// to the first node that is free, the parity of the distance decides.

__device__ __forceinline__ int32_t dp_parent(const int32_t *pair, int32_t n) {
    const int32_t m = pair[n];
    if (m < 0) return -1;
    if (pair[m] == n) return n < m ? -1 : m;          // root two-cycle: the smaller is the root
    return m;
}

__global__ void k_dp_children(int32_t V, const int32_t *pair, int32_t *pending) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = dp_parent(pair, (int32_t)i);
        if (p >= 0) atomicAdd(&pending[p], 1);
    }
}

// nchild: the child counts (read-only, decides who starts); pending: a copy
// that the children count down
__global__ void k_dp_up(int32_t V, const int32_t *pair, const int32_t *score, const int32_t *nchild,
                        int32_t *pending, unsigned long long *up, unsigned long long *best,
                        int32_t *status) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t v = (int32_t)i;
        if (nchild[v] != 0) continue;                  // not a leaf: a child's thread finishes it
        for (int32_t steps = 0;; ++steps) {
            if (steps > V) { set_status(status, kDevInternal); break; }
            const int32_t p = dp_parent(pair, v);
            if (p < 0) break;
            // v is complete: its children have all been folded into up/best[v]
            const unsigned long long bv = atomicAdd(&best[v], 0ull);
            const long long gv = bv ? (long long)(bv >> 32) - 2147483648ll : 0;
            const long long gc = gv > 0 ? gv : 0;
            const long long upv = (long long)atomicAdd(&up[v], 0ull);
            atomicAdd(&up[p], (unsigned long long)(upv + gc));
            const long long gain = (long long)score[v] - gc;
            atomicMax(&best[p], ((unsigned long long)(gain + 2147483648ll) << 32) | (uint32_t)v);
            __threadfence();
            if (atomicSub(&pending[p], 1) != 1) break;  // a sibling is still running
            __threadfence();
            v = p;
        }
    }
}

__device__ __forceinline__ int32_t dp_choice(const unsigned long long *best, int32_t v) {
    const unsigned long long b = best[v];
    if (!b) return -1;
    return (long long)(b >> 32) - 2147483648ll > 0 ? (int32_t)(b & 0xffffffffu) : -1;
}

__global__ void k_dp_down(int32_t V, const int32_t *pair, const unsigned long long *best,
                          int32_t *match, int32_t *rep_flag, int32_t *status) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t n = (int32_t)i;
        int32_t x = n, k = 0;
        for (;;) {
            const int32_t p = dp_parent(pair, x);
            if (p < 0 || dp_choice(best, p) != x) break;
            x = p;
            if (++k > V) { set_status(status, kDevInternal); k = 0; break; }
        }
        int32_t m;
        if (k & 1) m = dp_parent(pair, n);              // taken by its parent
        else {
            const int32_t c = dp_choice(best, n);
            m = c >= 0 ? c : n;
        }
        match[n] = m;
        rep_flag[n] = m >= n ? 1 : 0;
    }
}

// pair/score (and the learned order's keys, or null) -> match, gamma;
// *d_V2 receives the coarse node count.  exact: the tree-DP matching above
// (plain order only) instead of the two walks.
cudaError_t run_match(Arena &ar, int32_t V, const int32_t *pair, const int32_t *score,
                      const int32_t *key, int32_t *match, int32_t *gamma, int32_t *d_V2,
                      int32_t *status, cudaStream_t s, bool exact) {
    if (exact) {
        unsigned long long *up = nullptr, *best = nullptr;
        int32_t *nchild = nullptr, *pending = nullptr, *flag = nullptr, *rank = nullptr;
        cudaError_t e = dalloc(ar, &up, V);
        if (!e) e = dalloc(ar, &best, V);
        if (!e) e = dalloc(ar, &nchild, V);
        if (!e) e = dalloc(ar, &pending, V);
        if (!e) e = dalloc(ar, &flag, V);
        if (!e) e = dalloc(ar, &rank, V);
        if (!e) e = cudaMemsetAsync(up, 0, sizeof(unsigned long long) * (size_t)V, s);
        if (!e) e = cudaMemsetAsync(best, 0, sizeof(unsigned long long) * (size_t)V, s);
        if (!e) e = cudaMemsetAsync(nchild, 0, sizeof(int32_t) * (size_t)V, s);
        if (e) return e;
        k_dp_children<<<grid1d(V), 256, 0, s>>>(V, pair, nchild);
        e = cudaMemcpyAsync(pending, nchild, sizeof(int32_t) * (size_t)V, cudaMemcpyDeviceToDevice, s);
        if (e) return e;
        k_dp_up<<<grid1d(V), 256, 0, s>>>(V, pair, score, nchild, pending, up, best, status);
        k_dp_down<<<grid1d(V), 256, 0, s>>>(V, pair, best, match, flag, status);
        count_launch();
        count_launch();
        count_launch();
        e = exclusive_scan_i32(ar, flag, rank, V, d_V2, s);
        if (e) return e;
        k_gamma<<<grid1d(V), 256, 0, s>>>(V, match, rank, gamma);
        count_launch();
        return cudaGetLastError();
    }
    unsigned long long *best = nullptr;
    int32_t *flag = nullptr, *rank = nullptr;
    cudaError_t e = dalloc(ar, &best, V);
    if (!e) e = dalloc(ar, &flag, V);
    if (!e) e = dalloc(ar, &rank, V);
    if (e) return e;
    e = cudaMemsetAsync(best, 0, sizeof(unsigned long long) * (size_t)V, s);
    if (e) return e;
    if (key) {
        unsigned long long *bkey = nullptr;
        e = dalloc(ar, &bkey, V);
        if (!e) e = cudaMemsetAsync(bkey, 0, sizeof(unsigned long long) * (size_t)V, s);
        if (e) return e;
        k_best_key<<<grid1d(V), 256, 0, s>>>(V, pair, score, key, bkey);
        k_best_id<<<grid1d(V), 256, 0, s>>>(V, pair, score, key, bkey, best);
        count_launch();
        count_launch();
    } else {
        k_best<<<grid1d(V), 256, 0, s>>>(V, pair, score, best);
        count_launch();
    }
    k_lock_match<<<grid1d(V), 256, 0, s>>>(V, pair, best, match, flag, status);
    count_launch();
    e = exclusive_scan_i32(ar, flag, rank, V, d_V2, s);
    if (e) return e;
    k_gamma<<<grid1d(V), 256, 0, s>>>(V, match, rank, gamma);
    count_launch();
    return cudaGetLastError();
}

}  // namespace hgp
