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

// pair/score (and the learned order's keys, or null) -> match, gamma;
// *d_V2 receives the coarse node count.
cudaError_t run_match(Arena &ar, int32_t V, const int32_t *pair, const int32_t *score,
                      const int32_t *key, int32_t *match, int32_t *gamma, int32_t *d_V2,
                      int32_t *status, cudaStream_t s) {
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
