// Coarse hypergraph construction (Sec. III-B.4).
//
// Every coarse node c is one node or one matched pair {a, b} (a < b), so the
// set unions of the paper are unions of at most two sorted lists:
//   I'(c)  = I(a) u I(b)       in'(c) = in(a) u in(b)
// Unmatched nodes keep their lists (counted and copied by whole CTAs).  A CTA
// per matched pair merges the two sorted lists with duplicates removed, both
// staged in shared memory: each element finds its output slot from a binary
// search in the other list and a CTA-wide ballot prefix of the duplicates
// before it, so the result is sorted without any sort.  The lengths are
// counted first, prefix-summed into the new offsets, then written.
// pins'(e) = gamma(pins(e)) as a set: a pin is dropped only when it is the
// larger member b of a pair whose smaller member a is also a pin of e (tested
// by a binary search of e in the sorted I(a)); the rest are mapped through
// gamma and compacted in place order with a warp ballot.  All |E| hyperedges
// are kept.
#include "hgp_internal.cuh"

namespace hgp {

__global__ void k_coarse_nodes(int32_t V, const int32_t *match, const int32_t *gamma,
                               const int32_t *w, int32_t *rep_of, int32_t *w2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t n = (int32_t)i, m = match[n];
        if (m >= n) {
            int32_t c = gamma[n];
            rep_of[c] = n;
            w2[c] = w[n] + (m != n ? w[m] : 0);
        }
    }
}

// |A u B| (count) or the merged sorted list (write), CTA-cooperative: each
// element's output slot is its index plus its rank in the other list minus
// the duplicates before it (a CTA-wide ballot prefix).
template <bool WRITE>
__device__ int32_t block_union(const int32_t *A, int32_t na, const int32_t *B, int32_t nb,
                               int32_t *out, int32_t *s_w) {
    const int nw = blockDim.x >> 5;
    unsigned lt = (1u << lane_id()) - 1u;
    int32_t dupA = 0;
    for (int32_t base = 0; base < na; base += blockDim.x) {
        int32_t i = base + threadIdx.x;
        bool valid = i < na;
        int32_t x = valid ? A[i] : 0;
        int32_t lb = valid ? lower_bound_i32(B, 0, nb, x) : 0;
        bool inB = valid && lb < nb && B[lb] == x;
        unsigned ball = __ballot_sync(0xffffffffu, inB);
        if (lane_id() == 0) s_w[warp_id()] = __popc(ball);
        __syncthreads();
        int32_t pre = 0, tot = 0;
        for (int q = 0; q < nw; ++q) { pre += q < warp_id() ? s_w[q] : 0; tot += s_w[q]; }
        if (WRITE && valid) out[i + lb - (dupA + pre + __popc(ball & lt))] = x;
        dupA += tot;
        __syncthreads();
    }
    if (!WRITE) return na + nb - dupA;
    int32_t dupB = 0;
    for (int32_t base = 0; base < nb; base += blockDim.x) {
        int32_t j = base + threadIdx.x;
        bool valid = j < nb;
        int32_t y = valid ? B[j] : 0;
        int32_t lb = valid ? lower_bound_i32(A, 0, na, y) : 0;
        bool inA = valid && lb < na && A[lb] == y;
        unsigned ball = __ballot_sync(0xffffffffu, inA);
        if (lane_id() == 0) s_w[warp_id()] = __popc(ball);
        __syncthreads();
        int32_t pre = 0, tot = 0;
        for (int q = 0; q < nw; ++q) { pre += q < warp_id() ? s_w[q] : 0; tot += s_w[q]; }
        if (valid && !inA) out[lb + j - (dupB + pre + __popc(ball & lt))] = y;
        dupB += tot;
        __syncthreads();
    }
    return na + nb - dupA;
}

// Count pass for unmatched nodes (their lists are kept); matched pairs are
// queued for k_union_merged.
__global__ void k_union_count(int32_t V2, const int32_t *rep_of, const int32_t *match,
                              const int32_t *ioff, const int32_t *noff, int32_t *cntI,
                              int32_t *cntN, int32_t *max_in, int32_t *mlist, int32_t *mcount) {
    int32_t mi = 0;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < V2;
         c += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = rep_of[c];
        if (match[a] == a) {
            cntI[c] = ioff[a + 1] - ioff[a];
            cntN[c] = noff[a + 1] - noff[a];
            mi = max(mi, cntN[c]);
        } else {
            mlist[atomicAdd(mcount, 1)] = (int32_t)c;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mi = max(mi, __shfl_xor_sync(0xffffffffu, mi, o));
    if (lane_id() == 0 && mi) atomicMax(max_in, mi);
}

// Matched pairs: a CTA per pair, both lists staged in shared memory when
// they fit (binary searches then stay on chip).
template <bool WRITE>
__global__ void k_union_merged(const int32_t *mlist, const int32_t *mcount, const int32_t *rep_of,
                               const int32_t *match, const int32_t *ioff, const int32_t *inc,
                               const int32_t *noff, const int32_t *inn, int32_t *cntI,
                               int32_t *cntN, int32_t *max_in, const int32_t *ioff2, int32_t *inc2,
                               const int32_t *noff2, int32_t *inn2, int32_t cap) {
    extern __shared__ int32_t stage[];
    __shared__ int32_t s_w[32];
    int32_t nm = *mcount;
    for (int32_t t = blockIdx.x; t < nm; t += gridDim.x) {
        int32_t c = mlist[t], a = rep_of[c], b = match[a];
        int32_t res[2];
        for (int which = 0; which < 2; ++which) {
            const int32_t *off = which ? noff : ioff;
            const int32_t *dat = which ? inn : inc;
            const int32_t *A = dat + off[a], *B = dat + off[b];
            int32_t na = off[a + 1] - off[a], nb = off[b + 1] - off[b];
            if (na + nb <= cap) {
                for (int32_t i = threadIdx.x; i < na; i += blockDim.x) stage[i] = A[i];
                for (int32_t i = threadIdx.x; i < nb; i += blockDim.x) stage[na + i] = B[i];
                __syncthreads();
                A = stage;
                B = stage + na;
            }
            int32_t *out = nullptr;
            if (WRITE) out = which ? inn2 + noff2[c] : inc2 + ioff2[c];
            res[which] = block_union<WRITE>(A, na, B, nb, out, s_w);
            __syncthreads();
        }
        if (!WRITE && threadIdx.x == 0) {
            cntI[c] = res[0];
            cntN[c] = res[1];
            atomicMax(max_in, res[1]);
        }
    }
}

// Write pass for unmatched nodes: the whole CTA copies the kept lists.
__global__ void k_union_copy(int32_t V2, const int32_t *rep_of, const int32_t *match,
                             const int32_t *ioff, const int32_t *inc, const int32_t *noff,
                             const int32_t *inn, const int32_t *ioff2, int32_t *inc2,
                             const int32_t *noff2, int32_t *inn2) {
    for (int32_t c = blockIdx.x; c < V2; c += gridDim.x) {
        int32_t a = rep_of[c];
        if (match[a] != a) continue;
        int32_t i0 = ioff[a], n0 = noff[a];
        int32_t ni = ioff[a + 1] - i0, nn = noff[a + 1] - n0;
        int32_t *oi = inc2 + ioff2[c], *on = inn2 + noff2[c];
        for (int32_t t = threadIdx.x; t < ni; t += blockDim.x) oi[t] = inc[i0 + t];
        for (int32_t t = threadIdx.x; t < nn; t += blockDim.x) on[t] = inn[n0 + t];
    }
}

__device__ __forceinline__ bool keep_pin(int32_t m, int32_t e, const int32_t *match,
                                         const int32_t *ioff, const int32_t *inc) {
    int32_t a = match[m];
    if (a >= m) return true;                              // m represents its pair
    return !contains_sorted(inc, ioff[a], ioff[a + 1], e);  // drop if partner a is in e
}

template <bool WRITE>
__global__ void k_coarse_pins(int32_t E, const int32_t *poff, const int32_t *pins,
                              const int32_t *match, const int32_t *gamma, const int32_t *ioff,
                              const int32_t *inc, int32_t *cnt, const int32_t *poff2,
                              int32_t *pins2, int32_t *max_edge) {
    int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned lt = (1u << lane_id()) - 1u;
    for (int64_t e = gw; e < E; e += nw) {
        int32_t p0 = poff[e], p1 = poff[e + 1];
        int32_t outpos = WRITE ? poff2[e] : 0;
        int32_t kept = 0;
        for (int32_t base = p0; base < p1; base += 32) {
            int32_t j = base + lane_id();
            bool k = false;
            int32_t m = 0;
            if (j < p1) {
                m = pins[j];
                k = keep_pin(m, (int32_t)e, match, ioff, inc);
            }
            unsigned ball = __ballot_sync(0xffffffffu, k);
            if (WRITE && k) pins2[outpos + kept + __popc(ball & lt)] = gamma[m];
            kept += __popc(ball);
        }
        if (!WRITE && lane_id() == 0) { cnt[e] = kept; atomicMax(max_edge, kept); }
    }
}

// State carried into the next level's scoring (see Level::dead/merged/thr).
__global__ void k_carry(int32_t V, const int32_t *pair, const int32_t *score, const int32_t *match,
                        const int32_t *gamma, const uint8_t *dead, uint8_t *dead2, uint8_t *merged2,
                        unsigned long long *thr2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t n = (int32_t)i, m = match[n], c = gamma[n];
        if (m != n) {
            if (m > n) { merged2[c] = 1; dead2[c] = 0; thr2[c] = 0ull; }
        } else {
            merged2[c] = 0;
            bool d = pair[n] < 0 || (dead && dead[n]);
            dead2[c] = d ? 1 : 0;
            thr2[c] = d ? 0ull : (((unsigned long long)(uint32_t)score[n] << 32) | (uint32_t)pair[n]);
        }
    }
}

__global__ void k_coarse_src(int32_t E, const int32_t *src, const uint8_t *sdst,
                             const int32_t *gamma, const int32_t *noff2, const int32_t *inn2,
                             int32_t *src2, uint8_t *sdst2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < E;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t e = (int32_t)i;
        int32_t s = gamma[src[e]];
        src2[e] = s;
        // bit 1 is fixed by the Delta mode; bit 0 turns on once the source's
        // coarse node has e in its in() (a merged destination, inbound mode)
        const uint8_t r = sdst[e];
        sdst2[e] = (uint8_t)((r & 2) | (((r & 1) || contains_sorted(inn2, noff2[s], noff2[s + 1], e)) ? 1 : 0));
    }
}

static int grid_warps(int64_t items) {
    int b = div_up(items * 32, 256);
    int cap = num_sms() * 16;
    return b < 1 ? 1 : (b > cap ? cap : b);
}

static int grid1d(int64_t n) {
    int b = div_up(n, 256);
    int cap = num_sms() * 8;
    return b < 1 ? 1 : (b > cap ? cap : b);
}

// Builds level `H` (V2 nodes) from level `L` and its match/gamma.  Device
// allocations of H go to `keep` (what refinement reads: weights, pins,
// sources), `inc_ar` (I(n)) and `roll` (in(n) and the state carried into the
// next scoring, dead once H itself is contracted); temporaries to `tmp`.
// With `kt` set, CUDA events bracket the two kernel phases (count, write) so
// that their device time excludes the host read of the new sizes between
// them, and kt->host_bytes gains the contraction's algorithmic bytes: per
// level 4 B per pin read, gamma-gathered and written (pins), 4 B per entry
// read and written (I, in), and 12 B per hyperedge and per node (offsets).
cudaError_t run_contract(Arena &keep, Arena &inc_ar, Arena &roll, Arena &tmp, const Level &L,
                         int32_t V2, Level &H, const int32_t *pair, const int32_t *score,
                         int32_t *status, cudaStream_t s, PropTiming *kt) {
    cudaError_t e;
    auto ev_begin = [&]() {
        if (!kt) return;
        cudaEvent_t a;
        cudaEventCreate(&a);
        cudaEventRecord(a, s);
        kt->ev.push_back({a, nullptr});
    };
    auto ev_end = [&]() {
        if (!kt) return;
        cudaEventCreate(&kt->ev.back().second);
        cudaEventRecord(kt->ev.back().second, s);
    };
    H.V = V2;
    H.E = L.E;
    int32_t *rep_of = nullptr, *cntI = nullptr, *cntN = nullptr, *cntP = nullptr, *dmax = nullptr;
    int32_t *mlist = nullptr;
    e = dalloc(tmp, &rep_of, V2);
    if (!e) e = dalloc(tmp, &mlist, V2);
    if (!e) e = dalloc(tmp, &dmax, 3);    // [0] largest |in'|, [1] pairs queued, [2] largest |e'|
    if (!e) e = cudaMemsetAsync(dmax, 0, 3 * sizeof(int32_t), s);
    if (!e) e = dalloc(tmp, &cntI, V2);
    if (!e) e = dalloc(tmp, &cntN, V2);
    if (!e) e = dalloc(tmp, &cntP, L.E);
    if (!e) e = dalloc(keep, &H.w, V2);
    if (!e) e = dalloc(inc_ar, &H.ioff, (size_t)V2 + 1);
    if (!e) e = dalloc(roll, &H.noff, (size_t)V2 + 1);
    if (!e) e = dalloc(keep, &H.poff, (size_t)L.E + 1);
    if (!e) e = dalloc(keep, &H.src, L.E);
    if (!e) e = dalloc(keep, &H.sdst, L.E);
    if (!e) e = dalloc(roll, &H.dead, V2);
    if (!e) e = dalloc(roll, &H.merged, V2);
    if (!e) e = dalloc(roll, &H.thr, V2);
    if (!e) e = dalloc(roll, &H.old_id, V2);
    if (e) return e;
    ev_begin();
    k_coarse_nodes<<<grid1d(L.V), 256, 0, s>>>(L.V, L.match, L.gamma, L.w, rep_of, H.w);
    count_launch();
    k_carry<<<grid1d(L.V), 256, 0, s>>>(L.V, pair, score, L.match, L.gamma, L.dead, H.dead,
                                        H.merged, H.thr);
    count_launch();
    e = cudaMemcpyAsync(H.old_id, rep_of, sizeof(int32_t) * (size_t)V2, cudaMemcpyDeviceToDevice, s);
    if (e) return e;
    const int32_t cap = 12288;                  // staged list elements (48 KB)
    const size_t ssm = sizeof(int32_t) * (size_t)cap;
    int mblocks = num_sms() * 2;
    k_union_count<<<grid1d(V2), 256, 0, s>>>(V2, rep_of, L.match, L.ioff, L.noff, cntI, cntN, dmax,
                                             mlist, dmax + 1);
    count_launch();
    e = allow_dynamic_smem(k_union_merged<false>);
    if (!e) e = allow_dynamic_smem(k_union_merged<true>);
    if (e) return e;
    k_union_merged<false><<<mblocks, 256, ssm, s>>>(mlist, dmax + 1, rep_of, L.match, L.ioff, L.inc,
                                                    L.noff, L.inn, cntI, cntN, dmax, nullptr, nullptr,
                                                    nullptr, nullptr, cap);
    count_launch();
    k_coarse_pins<false><<<grid_warps(L.E), 256, 0, s>>>(L.E, L.poff, L.pins, L.match, L.gamma,
                                                         L.ioff, L.inc, cntP, nullptr, nullptr,
                                                         dmax + 2);
    count_launch();
    e = counts_to_offsets(tmp, cntI, H.ioff, V2, s);
    if (!e) e = counts_to_offsets(tmp, cntN, H.noff, V2, s);
    if (!e) e = counts_to_offsets(tmp, cntP, H.poff, L.E, s);
    if (e) return e;
    ev_end();
    int32_t tot[5];
    e = cudaMemcpyAsync(&tot[3], dmax, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(&tot[4], dmax + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(&tot[0], H.ioff + V2, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(&tot[1], H.noff + V2, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(&tot[2], H.poff + L.E, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return e;
    if (tot[0] != tot[2]) return cudaErrorInvalidValue;   // I' must be the transpose of pins'
    H.P = tot[0];
    H.Q = tot[1];
    H.max_in = tot[3];
    H.max_edge = tot[4];
    e = dalloc(inc_ar, &H.inc, H.P);
    if (!e) e = dalloc(roll, &H.inn, H.Q);
    if (!e) e = dalloc(keep, &H.pins, H.P);
    if (e) return e;
    ev_begin();
    {
        int blocks = V2 < num_sms() * 16 ? V2 : num_sms() * 16;
        k_union_copy<<<blocks, 256, 0, s>>>(V2, rep_of, L.match, L.ioff, L.inc, L.noff, L.inn,
                                            H.ioff, H.inc, H.noff, H.inn);
        count_launch();
        k_union_merged<true><<<mblocks, 256, ssm, s>>>(mlist, dmax + 1, rep_of, L.match, L.ioff,
                                                       L.inc, L.noff, L.inn, nullptr, nullptr,
                                                       nullptr, H.ioff, H.inc, H.noff, H.inn, cap);
    }
    count_launch();
    k_coarse_pins<true><<<grid_warps(L.E), 256, 0, s>>>(L.E, L.poff, L.pins, L.match, L.gamma,
                                                        L.ioff, L.inc, nullptr, H.poff, H.pins,
                                                        nullptr);
    count_launch();
    k_coarse_src<<<grid1d(L.E), 256, 0, s>>>(L.E, L.src, L.sdst, L.gamma, H.noff, H.inn, H.src,
                                             H.sdst);
    count_launch();
    ev_end();
    if (kt)
        kt->host_bytes += 4ull * (unsigned long long)(3 * L.P + H.P) +      // pins
                          4ull * (unsigned long long)(L.P + H.P) +          // I
                          4ull * (unsigned long long)(L.Q + H.Q) +          // in
                          12ull * (unsigned long long)((int64_t)L.E + L.V);  // offsets
    (void)status;
    return cudaGetLastError();
}

}  // namespace hgp
