// Constraint-only baseline of the paper's evaluation (Sec. V): nodes are
// taken in id order and appended to the current part while w(part) + w(n) <=
// Omega and |in(part) u in(n)| <= Delta; otherwise n opens the next part.
// The decision for a node depends on all earlier ones, so one CTA walks the
// nodes in order; its threads split in(n) to count the hyperedges not yet in
// the current part's union, which is kept as a per-hyperedge stamp (the id of
// the last part that took it) in global memory, so starting a part costs
// nothing.
#include "hgp_internal.cuh"

namespace hgp {

constexpr int kFillThreads = 256;

__global__ void __launch_bounds__(kFillThreads)
k_fill_baseline(int32_t V, const int32_t *w, const int32_t *noff, const int32_t *inn,
                int64_t omega, int64_t delta, int32_t *stamp, int32_t *part, int32_t *nparts) {
    __shared__ int32_t red[kFillThreads / 32];
    int32_t p = -1;
    int64_t pw = 0, pu = 0;
    for (int32_t n = 0; n < V; ++n) {
        const int32_t j0 = noff[n], j1 = noff[n + 1];
        int32_t fresh = 0;
        if (p >= 0)
            for (int32_t j = j0 + threadIdx.x; j < j1; j += kFillThreads) fresh += stamp[inn[j]] != p;
        fresh = warp_sum(fresh);
        if (lane_id() == 0) red[warp_id()] = fresh;
        __syncthreads();
        int32_t f = 0;
        for (int i = 0; i < kFillThreads / 32; ++i) f += red[i];
        const int64_t wn = w[n];
        if (p < 0 || pw + wn > omega || pu + f > delta) {     // same decision in every thread
            p++;
            pw = 0;
            pu = 0;
            f = j1 - j0;
        }
        pw += wn;
        pu += f;
        for (int32_t j = j0 + threadIdx.x; j < j1; j += kFillThreads) stamp[inn[j]] = p;
        if (threadIdx.x == 0) part[n] = p;
        __syncthreads();          // stamps and red visible before the next node
    }
    if (threadIdx.x == 0) *nparts = p + 1;
}

cudaError_t run_fill_baseline(Arena &ar, const Level &L0, int64_t omega, int64_t delta,
                              int32_t *part, int32_t *d_nparts, cudaStream_t s) {
    int32_t *stamp = nullptr;
    cudaError_t e = dalloc(ar, &stamp, L0.E);
    if (!e) e = cudaMemsetAsync(stamp, 0xff, sizeof(int32_t) * (size_t)(L0.E > 0 ? L0.E : 1), s);
    if (e) return e;
    k_fill_baseline<<<1, kFillThreads, 0, s>>>(L0.V, L0.w, L0.noff, L0.inn, omega, delta, stamp, part,
                                               d_nparts);
    count_launch();
    return cudaGetLastError();
}

}  // namespace hgp
