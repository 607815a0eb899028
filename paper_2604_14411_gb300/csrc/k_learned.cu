// Learned candidate order: a two-layer network ranks the candidates of a node
// before Eq. (2)'s hist (an extension of Sec. III-A; the paper has none).
//
//   x     = 8 features of the pair (n, m), symmetric in n and m:
//           lg1p of hist(n,m), |in(n) u in(m)|, min/max |I|, min/max |in|,
//           min/max w, where lg1p(x) = k + (1 + x - 2^k) / 2^k for
//           2^k <= 1 + x < 2^(k+1) (log2(1 + x) with a linear mantissa)
//   h_j   = relu(b1_j + sum_i W1_ji x_i), s = b2 + sum_j W2_j h_j
//   key   = floor(s * 2^key_bits), clamped to [-2^30, 2^30]
//   pair(n) = the valid m with the largest (key, hist, id)
// Weights are bfloat16, widened exactly to float; every sum is a chain of
// fused multiply-adds in index order (h_j over i, then s over j with each
// h_j folded in as soon as it is computed).  That order is part of the
// definition, so the keys are bit-identical to any other implementation
// that follows it.  The weights travel in the kernel's parameter space, so
// every FMA takes its weight from the constant bank.
//
// Scoring kernel: one 1024-thread CTA per node.  Pass 1 accumulates, per
// neighbour m, hist(n, m) and inter(n, m) = |in(n) n in(m)| (a hyperedge e
// of I(n) is in in(x) for every pin x except its source, unless the source's
// node also holds a destination of e); |in(n) u in(m)| = |in(n)| + |in(m)| -
// inter(n, m), so the Delta check needs no per-pair set union.  Pass 2
// evaluates the network for every valid neighbour and reduces (key, hist,
// id) over the CTA.  Histograms: two dense shared-memory arrays when the
// level fits on chip, otherwise per-CTA open-addressing tables in global
// memory.
//
// Levels too large for one CTA but with weighted degrees and inbound counts
// below 2^16 use a thread-block cluster of 8 CTAs instead: each holds a slice
// of node ids with hist and inter packed into one 32-bit word (hist << 16 |
// inter) in its shared memory, the cluster's warps add into the owners'
// slices with remote shared-memory atomics, each CTA evaluates the network
// on its own slice, and the cluster reduces (key, hist, id).  Other levels
// fall back to per-CTA hash tables in global memory.
//
// Training kernels: features and co-location labels of sampled pairs, and
// minibatch Adam steps on the logistic loss with the forward pass in
// bfloat16 weights and float32 arithmetic; per-warp partial gradients are
// summed in a fixed order, so training is deterministic.
#include <cooperative_groups.h>
#include <cstring>

#include "hgp_internal.cuh"

namespace hgp {

constexpr int kMlpIn = HGP_MLP_IN;
constexpr int kMlpHid = HGP_MLP_HIDDEN;
constexpr int kMlpParams = HGP_MLP_PARAMS;
constexpr int kLearnThreads = 1024;
constexpr int kLearnWarps = kLearnThreads / 32;
constexpr int32_t kKeyBias = 1 << 30;

struct MlpParams {
    float w1[kMlpHid * kMlpIn];
    float b1[kMlpHid];
    float w2[kMlpHid];
    float b2;
    int32_t key_bits;
};

struct LearnedArgs {
    int32_t V, E;
    const int32_t *w, *poff, *pins, *ioff, *inc, *noff, *ew, *src;
    const uint8_t *sdst, *dead;
    int64_t omega, delta;
    int32_t *pair, *score, *key;
    int32_t *next, *status;
    int32_t *gkeys, *gvals, *ginter, *gused;
    int32_t gcap;
    unsigned long long *bytes, *evals;
    int32_t tc;                  // 1: evaluate the network on tensor cores (mlp_eval_tc)
    const float *tcw;            // tc: W1 (512), b1 (64), W2 (64), b2 as float32, device memory
};

__device__ __forceinline__ float pow2_exact(int k) {       // 2^k, -126 <= k <= 127
    return __int_as_float((127 + k) << 23);
}

__device__ __forceinline__ float lg1p_dev(int64_t x) {
    unsigned long long y = (unsigned long long)x + 1ull;
    int k = 63 - __clzll((long long)y);
    float frac = __fmul_rn(__ull2float_rn(y - (1ull << k)), pow2_exact(-k));
    return __fadd_rn((float)k, frac);
}

__device__ __forceinline__ float mlp_eval(const MlpParams &M, const float *x) {
    float s = M.b2;
#pragma unroll
    for (int j = 0; j < kMlpHid; ++j) {
        float h = M.b1[j];
#pragma unroll
        for (int i = 0; i < kMlpIn; ++i) h = __fmaf_rn(M.w1[j * kMlpIn + i], x[i], h);
        h = h > 0.0f ? h : 0.0f;
        s = __fmaf_rn(M.w2[j], h, s);
    }
    return s;
}

// ---- tensor-core evaluation (hgp_options.learned_eval = 1) ----
// The warp's 32 queued candidates are two 16 x 8 tiles of features; the
// hidden layer is those tiles times W1^T (8 x 64, eight 8-column tiles) by
// mma.sync m16n8k8 with TF32 inputs and FP32 accumulation (16 MMAs per 32
// candidates instead of 32 x 512 FMAs).  Bias, ReLU and the output layer are
// applied to the accumulator fragments and summed over the four lanes that
// hold a row.  The bfloat16 weights are exact in TF32; the features are
// rounded to TF32 (10-bit mantissa), so scores differ from the FMA chains in
// the last bits -- this mode is checked against a float32 reference within
// a tolerance, not bit for bit.
__device__ __forceinline__ uint32_t to_tf32(float f) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(f));
    return r;
}

__device__ __forceinline__ void mma_tf32_m16n8k8(float &d0, float &d1, float &d2, float &d3,
                                                 uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                                 uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 "
                 "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
                 : "+f"(d0), "+f"(d1), "+f"(d2), "+f"(d3)
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float pick4(float v0, float v1, float v2, float v3, int i) {
    return i == 0 ? v0 : i == 1 ? v1 : i == 2 ? v2 : v3;
}

// Score of lane r's candidate (row r); x = this lane's 8 features, sw = the
// network staged in shared memory (W1 at 8 j + i, b1 at 512 + j, W2 at
// 576 + j, b2 at 640).  All 32 lanes must call it.
__device__ __forceinline__ float mlp_eval_tc(const float *x, const float *sw) {
    const int lane = lane_id(), g = lane >> 2, tq = lane & 3;
    // A fragments (row-major 16 x 8): a0 = (g, tq), a1 = (g + 8, tq),
    // a2 = (g, tq + 4), a3 = (g + 8, tq + 4), rows taken from the lanes
    // that hold them
    uint32_t A[2][4];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        float ra[kMlpIn], rb[kMlpIn];
#pragma unroll
        for (int k = 0; k < kMlpIn; ++k) {
            ra[k] = __shfl_sync(0xffffffffu, x[k], 16 * t + g);
            rb[k] = __shfl_sync(0xffffffffu, x[k], 16 * t + g + 8);
        }
        A[t][0] = to_tf32(pick4(ra[0], ra[1], ra[2], ra[3], tq));
        A[t][1] = to_tf32(pick4(rb[0], rb[1], rb[2], rb[3], tq));
        A[t][2] = to_tf32(pick4(ra[4], ra[5], ra[6], ra[7], tq));
        A[t][3] = to_tf32(pick4(rb[4], rb[5], rb[6], rb[7], tq));
    }
    float p[2][2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};        // [tile][row g or g + 8]
#pragma unroll
    for (int nt = 0; nt < kMlpHid / 8; ++nt) {
        // B fragment (column-major 8 x 8 of W1^T): b0 = (k = tq, n = g), b1 = (tq + 4, g)
        const int j = nt * 8 + g;
        const uint32_t b0 = __float_as_uint(sw[j * kMlpIn + tq]);
        const uint32_t b1 = __float_as_uint(sw[j * kMlpIn + tq + 4]);
        // accumulators: columns 2 tq, 2 tq + 1 of rows g (d0, d1) and g + 8 (d2, d3)
        const int c0 = nt * 8 + 2 * tq, c1 = c0 + 1;
        const float bb0 = sw[512 + c0], bb1 = sw[512 + c1];
        const float ww0 = sw[576 + c0], ww1 = sw[576 + c1];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            float d0 = 0.0f, d1 = 0.0f, d2 = 0.0f, d3 = 0.0f;
            mma_tf32_m16n8k8(d0, d1, d2, d3, A[t][0], A[t][1], A[t][2], A[t][3], b0, b1);
            p[t][0] = fmaf(ww0, fmaxf(d0 + bb0, 0.0f), p[t][0]);
            p[t][0] = fmaf(ww1, fmaxf(d1 + bb1, 0.0f), p[t][0]);
            p[t][1] = fmaf(ww0, fmaxf(d2 + bb0, 0.0f), p[t][1]);
            p[t][1] = fmaf(ww1, fmaxf(d3 + bb1, 0.0f), p[t][1]);
        }
    }
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            p[t][h] += __shfl_xor_sync(0xffffffffu, p[t][h], 1);
            p[t][h] += __shfl_xor_sync(0xffffffffu, p[t][h], 2);
        }
    // row r = 16 t + 8 h + g' is complete in lanes 4 g' .. 4 g' + 3
    const int src = 4 * (lane & 7);
    const float v00 = __shfl_sync(0xffffffffu, p[0][0], src);
    const float v01 = __shfl_sync(0xffffffffu, p[0][1], src);
    const float v10 = __shfl_sync(0xffffffffu, p[1][0], src);
    const float v11 = __shfl_sync(0xffffffffu, p[1][1], src);
    const int t = lane >> 4, h = (lane >> 3) & 1;
    return sw[640] + (t == 0 ? (h == 0 ? v00 : v01) : (h == 0 ? v10 : v11));
}

__device__ __forceinline__ int32_t key_of(float s, int32_t key_bits) {
    float q = floorf(__fmul_rn(s, pow2_exact(key_bits)));
    if (!(q > -1073741824.0f)) return -kKeyBias;
    if (q > 1073741824.0f) return kKeyBias;
    return (int32_t)q;
}

__device__ __forceinline__ unsigned long long composite(int32_t key, int32_t hist) {
    return ((unsigned long long)(uint32_t)(key + kKeyBias) << 32) | (uint32_t)hist;
}

__device__ __forceinline__ void features(const LearnedArgs &a, int32_t n, int32_t m, int32_t hist,
                                         int64_t uni, int64_t in_n, int64_t in_m, float *x) {
    int64_t dn = a.ioff[n + 1] - a.ioff[n], dm = a.ioff[m + 1] - a.ioff[m];
    int64_t wn = a.w[n], wm = a.w[m];
    x[0] = lg1p_dev(hist);
    x[1] = lg1p_dev(uni);
    x[2] = lg1p_dev(min(dn, dm));
    x[3] = lg1p_dev(max(dn, dm));
    x[4] = lg1p_dev(min(in_n, in_m));
    x[5] = lg1p_dev(max(in_n, in_m));
    x[6] = lg1p_dev(min(wn, wm));
    x[7] = lg1p_dev(max(wn, wm));
}

// (comp, id) lexicographic maximum over the CTA; every thread gets it.
__device__ void block_argmax(unsigned long long &comp, int32_t &id, unsigned long long *s_c,
                             int32_t *s_i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long c2 = __shfl_xor_sync(0xffffffffu, comp, o);
        int32_t i2 = __shfl_xor_sync(0xffffffffu, id, o);
        if (c2 > comp || (c2 == comp && i2 > id)) { comp = c2; id = i2; }
    }
    __syncthreads();
    if (lane_id() == 0) { s_c[warp_id()] = comp; s_i[warp_id()] = id; }
    __syncthreads();
    comp = s_c[0];
    id = s_i[0];
    for (int w = 1; w < kLearnWarps; ++w)
        if (s_c[w] > comp || (s_c[w] == comp && s_i[w] > id)) { comp = s_c[w]; id = s_i[w]; }
}

__device__ __forceinline__ uint32_t hash_node(uint32_t x) {
    x ^= x >> 16; x *= 0x7feb352dU; x ^= x >> 15; x *= 0x846ca68bU; x ^= x >> 16;
    return x;
}

// Candidates of one node: each warp tests 32 ids at a time and queues the
// valid ones in shared memory; whenever 32 are queued the warp evaluates the
// network on all of them at once.  So the network runs on full warps even
// where few ids are neighbours, with no CTA-wide barrier.  load(i, m, h, it)
// reads entry i; the running best (comp, id) is kept per thread.
struct LearnQueue {
    int32_t m[kLearnWarps][64], h[kLearnWarps][64], it[kLearnWarps][64];
};

template <typename Load>
__device__ __forceinline__ void eval_candidates(const LearnedArgs &a, const MlpParams &M, int32_t n,
                                                int32_t cap, Load load, LearnQueue &Q,
                                                unsigned long long &best_c, int32_t &best_m,
                                                unsigned long long &bytes,
                                                unsigned long long &evals, const float *sw) {
    const int w = warp_id(), lane = lane_id();
    int32_t *qm = Q.m[w], *qh = Q.h[w], *qi = Q.it[w];
    const int64_t in_n = a.noff[n + 1] - a.noff[n];
    const int64_t wn = a.w[n];
    auto evaluate = [&](int32_t slot) {
        const int32_t m = qm[slot], h = qh[slot], it = qi[slot];
        const int64_t in_m = a.noff[m + 1] - a.noff[m];
        const int64_t uni = in_n + in_m - it;
        float x[kMlpIn];
        features(a, n, m, h, uni, in_n, in_m, x);
        const int32_t k = key_of(mlp_eval(M, x), M.key_bits);
        const unsigned long long c = composite(k, h);
        if (best_m < 0 || c > best_c || (c == best_c && m > best_m)) { best_c = c; best_m = m; }
        bytes += 20ull;
        evals += 1ull;
    };
    // tensor cores: the first `valid` queue slots at once (all lanes call it)
    auto evaluate_tc = [&](int32_t valid) {
        const bool ok = lane < valid;
        float x[kMlpIn];
        int32_t m = 0, h = 0;
        if (ok) {
            m = qm[lane];
            h = qh[lane];
            const int64_t in_m = a.noff[m + 1] - a.noff[m];
            features(a, n, m, h, in_n + in_m - qi[lane], in_n, in_m, x);
        } else {
#pragma unroll
            for (int k = 0; k < kMlpIn; ++k) x[k] = 0.0f;
        }
        const float sc = mlp_eval_tc(x, sw);
        if (ok) {
            const unsigned long long c = composite(key_of(sc, M.key_bits), h);
            if (best_m < 0 || c > best_c || (c == best_c && m > best_m)) { best_c = c; best_m = m; }
            bytes += 20ull;
            evals += 1ull;
        }
    };
    int32_t qn = 0;                                      // warp-uniform queue length (< 32 here)
    for (int32_t base = w * 32; base < cap; base += kLearnThreads) {
        const int32_t i = base + lane;
        int32_t m = 0, h = 0, it = 0;
        bool ok = false;
        if (i < cap) {
            load(i, m, h, it);
            ok = h != 0 && !(a.dead && a.dead[m]) && wn + a.w[m] <= a.omega &&
                 in_n + (a.noff[m + 1] - a.noff[m]) - it <= a.delta;
        }
        const unsigned ball = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            const int32_t pos = qn + __popc(ball & ((1u << lane) - 1u));
            qm[pos] = m;
            qh[pos] = h;
            qi[pos] = it;
        }
        qn += __popc(ball);
        __syncwarp();
        if (qn >= 32) {
            if (a.tc) evaluate_tc(32);
            else evaluate(lane);
            __syncwarp();
            if (lane < qn - 32) {
                qm[lane] = qm[32 + lane];
                qh[lane] = qh[32 + lane];
                qi[lane] = qi[32 + lane];
            }
            __syncwarp();
            qn -= 32;
        }
    }
    if (a.tc) {
        if (qn > 0) evaluate_tc(qn);
    } else if (lane < qn) {
        evaluate(lane);
    }
    __syncwarp();                                        // the queue is reused by the next node
}

template <bool DENSE>
__global__ void __launch_bounds__(kLearnThreads)
k_score_learned(LearnedArgs a, MlpParams M) {
    extern __shared__ __align__(16) unsigned char smem[];
    int32_t *hist = reinterpret_cast<int32_t *>(smem);
    int32_t *inter = hist + (DENSE ? a.V : 0);
    __shared__ unsigned long long s_c[kLearnWarps];
    __shared__ int32_t s_i[kLearnWarps];
    __shared__ int32_t s_n, s_used;
    __shared__ LearnQueue s_queue;
    __shared__ float s_w[kMlpParams];         // the network, for tensor-core evaluation
    if (a.tc)
        for (int i = threadIdx.x; i < kMlpParams; i += kLearnThreads) s_w[i] = a.tcw[i];
    // hash mode: the table is cleared once here, then only the slots a node
    // used (listed in gu) are visited and reset
    int32_t *gk = DENSE ? nullptr : a.gkeys + (int64_t)blockIdx.x * a.gcap;
    int32_t *gv = DENSE ? nullptr : a.gvals + (int64_t)blockIdx.x * a.gcap;
    int32_t *gi = DENSE ? nullptr : a.ginter + (int64_t)blockIdx.x * a.gcap;
    int32_t *gu = DENSE ? nullptr : a.gused + (int64_t)blockIdx.x * a.gcap;
    const uint32_t mask = (uint32_t)a.gcap - 1u;
    unsigned long long bytes = 0, evals = 0;
    if (!DENSE) {
        for (int32_t i = threadIdx.x; i < a.gcap; i += kLearnThreads) { gk[i] = -1; gv[i] = 0; gi[i] = 0; }
        if (threadIdx.x == 0) s_used = 0;
    }

    for (;;) {
        if (threadIdx.x == 0) s_n = atomicAdd(a.next, 1);
        __syncthreads();
        const int32_t n = s_n;
        if (n >= a.V) break;
        if (a.dead && a.dead[n]) {              // no valid candidate can exist
            if (threadIdx.x == 0) { a.pair[n] = -1; a.score[n] = 0; a.key[n] = 0; }
            __syncthreads();
            continue;
        }
        if (DENSE)
            for (int32_t i = threadIdx.x; i < a.V; i += kLearnThreads) { hist[i] = 0; inter[i] = 0; }
        __syncthreads();
        // ---- pass 1: hist(n, .) and inter(n, .) ----
        const int32_t i0 = a.ioff[n], i1 = a.ioff[n + 1];
        const int32_t mine = (i1 - i0 - warp_id() + kLearnWarps - 1) / kLearnWarps;
        for (int32_t r0 = 0; r0 < mine; r0 += 32) {
            int32_t we = 0, p0 = 0, p1 = 0, se = -1, sd = 0;
            if (r0 + lane_id() < mine) {
                int32_t e = a.inc[i0 + warp_id() + kLearnWarps * (r0 + lane_id())];
                we = a.ew[e];
                p0 = a.poff[e];
                p1 = a.poff[e + 1];
                se = a.src[e];
                sd = a.sdst[e];
            }
            const int32_t cnt = min(32, mine - r0);
            for (int32_t t = 0; t < cnt; ++t) {
                const int32_t wt = __shfl_sync(0xffffffffu, we, t);
                const int32_t b0 = __shfl_sync(0xffffffffu, p0, t);
                const int32_t b1 = __shfl_sync(0xffffffffu, p1, t);
                const int32_t s_e = __shfl_sync(0xffffffffu, se, t);
                const int32_t sd_e = __shfl_sync(0xffffffffu, sd, t);
                const bool n_in = counts_in(n, s_e, (uint8_t)sd_e);     // e in in(n)
                for (int32_t j = b0 + lane_id(); j < b1; j += 32) {
                    const int32_t m = a.pins[j];
                    if (m == n) continue;
                    const int32_t both = (n_in && counts_in(m, s_e, (uint8_t)sd_e)) ? 1 : 0;
                    if (DENSE) {
                        atomicAdd(&hist[m], wt);
                        if (both) atomicAdd(&inter[m], 1);
                    } else {
                        uint32_t slot = hash_node((uint32_t)m) & mask;
                        for (int32_t probes = 0;; ++probes) {
                            int32_t kk = atomicCAS(&gk[slot], -1, m);
                            if (kk == -1) gu[atomicAdd(&s_used, 1)] = (int32_t)slot;
                            if (kk == -1 || kk == m) {
                                atomicAdd(&gv[slot], wt);
                                if (both) atomicAdd(&gi[slot], 1);
                                break;
                            }
                            slot = (slot + 1) & mask;
                            if (probes + 1 >= a.gcap) { set_status(a.status, kDevLimit); break; }
                        }
                    }
                }
                if (lane_id() == 0) bytes += 24ull + 4ull * (unsigned long long)(b1 - b0);
            }
        }
        __syncthreads();
        // ---- pass 2: the network on every valid neighbour ----
        unsigned long long best_c = 0ull;
        int32_t best_m = -1;
        const int32_t cap = DENSE ? a.V : s_used;
        eval_candidates(a, M, n, cap,
                        [&](int32_t i, int32_t &m, int32_t &h, int32_t &it) {
                            if (DENSE) { m = i; h = hist[i]; it = inter[i]; }
                            else { int32_t sl = gu[i]; m = gk[sl]; h = gv[sl]; it = gi[sl]; }
                        },
                        s_queue, best_c, best_m, bytes, evals, s_w);
        block_argmax(best_c, best_m, s_c, s_i);
        if (threadIdx.x == 0) {
            a.pair[n] = best_m;
            a.score[n] = best_m >= 0 ? (int32_t)(best_c & 0xffffffffull) : 0;
            a.key[n] = best_m >= 0 ? (int32_t)(best_c >> 32) - kKeyBias : 0;
            bytes += 24ull;
        }
        if (!DENSE) {
            for (int32_t i = threadIdx.x; i < cap; i += kLearnThreads) {
                int32_t sl = gu[i];
                gk[sl] = -1; gv[sl] = 0; gi[sl] = 0;
            }
            __syncthreads();
            if (threadIdx.x == 0) s_used = 0;
        }
        __syncthreads();
    }
    if (a.bytes) {
        bytes = warp_sum(bytes);
        evals = warp_sum(evals);
        if (lane_id() == 0 && bytes) atomicAdd(a.bytes, bytes);
        if (lane_id() == 0 && evals && a.evals) atomicAdd(a.evals, evals);
    }
}

namespace cg = cooperative_groups;
constexpr int kLearnCluster = 8;

__global__ void __cluster_dims__(kLearnCluster, 1, 1) __launch_bounds__(kLearnThreads)
k_score_learned_cluster(LearnedArgs a, MlpParams M, int32_t slice) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *cnt = reinterpret_cast<uint32_t *>(smem);      // [slice]: hist << 16 | inter
    __shared__ unsigned long long s_c[kLearnWarps];
    __shared__ int32_t s_i[kLearnWarps];
    __shared__ int32_t s_node;
    __shared__ LearnQueue s_queue;
    __shared__ unsigned long long s_xc;
    __shared__ int32_t s_xi;
    __shared__ float s_w[kMlpParams];         // the network, for tensor-core evaluation
    if (a.tc)
        for (int i = threadIdx.x; i < kMlpParams; i += kLearnThreads) s_w[i] = a.tcw[i];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int32_t id0 = rank * slice;
    const int32_t len = max(0, min(slice, a.V - id0));
    unsigned long long bytes = 0, evals = 0;
    for (int32_t i = threadIdx.x; i < len; i += kLearnThreads) cnt[i] = 0u;
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) {
            int32_t t = atomicAdd(a.next, 1);
            s_node = t < a.V ? t : a.V;
        }
        cl.sync();                                   // slices cleared, node published
        const int32_t n = *cl.map_shared_rank(&s_node, 0);
        if (n >= a.V) {
            cl.sync();       // no CTA leaves while a peer may still read its shared memory
            break;
        }
        if (a.dead && a.dead[n]) {
            if (rank == 0 && threadIdx.x == 0) { a.pair[n] = -1; a.score[n] = 0; a.key[n] = 0; }
            cl.sync();                               // everyone has read s_node
            continue;
        }
        // ---- pass 1: packed hist / inter over the cluster's warps ----
        const int32_t i0 = a.ioff[n], i1 = a.ioff[n + 1];
        const int32_t gw = rank * kLearnWarps + warp_id(), nw = kLearnCluster * kLearnWarps;
        const int32_t mine = (i1 - i0 - gw + nw - 1) / nw;
        for (int32_t r0 = 0; r0 < mine; r0 += 32) {
            int32_t we = 0, p0 = 0, p1 = 0, se = -1, sd = 0;
            if (r0 + lane_id() < mine) {
                int32_t e = a.inc[i0 + gw + nw * (r0 + lane_id())];
                we = a.ew[e];
                p0 = a.poff[e];
                p1 = a.poff[e + 1];
                se = a.src[e];
                sd = a.sdst[e];
            }
            const int32_t c = min(32, mine - r0);
            for (int32_t t = 0; t < c; ++t) {
                const uint32_t wt = (uint32_t)__shfl_sync(0xffffffffu, we, t);
                const int32_t b0 = __shfl_sync(0xffffffffu, p0, t);
                const int32_t b1 = __shfl_sync(0xffffffffu, p1, t);
                const int32_t s_e = __shfl_sync(0xffffffffu, se, t);
                const int32_t sd_e = __shfl_sync(0xffffffffu, sd, t);
                const bool n_in = counts_in(n, s_e, (uint8_t)sd_e);
                for (int32_t j = b0 + lane_id(); j < b1; j += 32) {
                    const int32_t m = a.pins[j];
                    if (m == n) continue;
                    const uint32_t both = (n_in && counts_in(m, s_e, (uint8_t)sd_e)) ? 1u : 0u;
                    const int32_t owner = m / slice;
                    atomicAdd(cl.map_shared_rank(cnt, owner) + (m - owner * slice), (wt << 16) | both);
                }
                if (lane_id() == 0) bytes += 24ull + 4ull * (unsigned long long)(b1 - b0);
            }
        }
        cl.sync();                                   // every slice complete
        // ---- pass 2: the network on this CTA's slice ----
        unsigned long long best_c = 0ull;
        int32_t best_m = -1;
        eval_candidates(a, M, n, len,
                        [&](int32_t i, int32_t &m, int32_t &h, int32_t &it) {
                            const uint32_t v = cnt[i];
                            m = id0 + i;
                            h = (int32_t)(v >> 16);
                            it = (int32_t)(v & 0xffffu);
                        },
                        s_queue, best_c, best_m, bytes, evals, s_w);
        block_argmax(best_c, best_m, s_c, s_i);
        if (threadIdx.x == 0) { s_xc = best_c; s_xi = best_m; }
        for (int32_t i = threadIdx.x; i < len; i += kLearnThreads) cnt[i] = 0u;
        cl.sync();                                   // every CTA's best published
        if (rank == 0 && threadIdx.x == 0) {
            unsigned long long bc = 0ull;
            int32_t bm = -1;
            for (int r = 0; r < kLearnCluster; ++r) {
                unsigned long long c2 = *cl.map_shared_rank(&s_xc, r);
                int32_t m2 = *cl.map_shared_rank(&s_xi, r);
                if (m2 >= 0 && (bm < 0 || c2 > bc || (c2 == bc && m2 > bm))) { bc = c2; bm = m2; }
            }
            a.pair[n] = bm;
            a.score[n] = bm >= 0 ? (int32_t)(bc & 0xffffffffull) : 0;
            a.key[n] = bm >= 0 ? (int32_t)(bc >> 32) - kKeyBias : 0;
            bytes += 24ull;
        }
        cl.sync();                                   // rank 0 has read every s_xc / s_xi
    }
    if (a.bytes) {
        bytes = warp_sum(bytes);
        evals = warp_sum(evals);
        if (lane_id() == 0 && bytes) atomicAdd(a.bytes, bytes);
        if (lane_id() == 0 && evals && a.evals) atomicAdd(a.evals, evals);
    }
}

// out[0] = largest sum of |e| over I(n) (pin visits of a node); out[1] =
// largest sum of omega(e) over I(n) (bounds every hist(n, .)).
static __global__ void k_max_visits(int32_t V, const int32_t *ioff, const int32_t *inc,
                                    const int32_t *poff, const int32_t *ew,
                                    unsigned long long *out) {
    int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t n = gw; n < V; n += nw) {
        unsigned long long s = 0, w = 0;
        for (int32_t k = ioff[n] + lane_id(); k < ioff[n + 1]; k += 32) {
            int32_t e = inc[k];
            s += (unsigned long long)(poff[e + 1] - poff[e]);
            w += (unsigned long long)ew[e];
        }
        s = warp_sum(s);
        w = warp_sum(w);
        if (lane_id() == 0) { atomicMax(&out[0], s); atomicMax(&out[1], w); }
    }
}

// Host copy of a model's weights, widened from bfloat16 (exact).
static float bf16_bits_to_float(uint16_t b) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, sizeof(f));
    return f;
}

bool model_valid(const hgp_model *m) {
    if (m->key_bits < 0 || m->key_bits > 20) return false;
    for (int i = 0; i < 3; ++i)
        if (m->reserved[i]) return false;
    return true;
}

static MlpParams widen(const hgp_model *m) {
    MlpParams P;
    for (int q = 0; q < kMlpHid * kMlpIn; ++q) P.w1[q] = bf16_bits_to_float(m->w1[q]);
    for (int j = 0; j < kMlpHid; ++j) {
        P.b1[j] = bf16_bits_to_float(m->b1[j]);
        P.w2[j] = bf16_bits_to_float(m->w2[j]);
    }
    P.b2 = bf16_bits_to_float(m->b2);
    P.key_bits = m->key_bits;
    return P;
}

cudaError_t run_score_learned(Arena &ar, const Level &L, const int32_t *ew, int64_t omega,
                              int64_t delta, const hgp_model *model, int32_t *pair,
                              int32_t *score, int32_t *key, int32_t *status,
                              unsigned long long *bytes, unsigned long long *evals,
                              uint32_t debug, int32_t tensor_cores, cudaStream_t s) {
    if (L.V <= 0) return cudaSuccess;
    int dev = 0;
    cudaGetDevice(&dev);
    int max_smem = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    LearnedArgs a{};
    a.V = L.V; a.E = L.E;
    a.w = L.w; a.poff = L.poff; a.pins = L.pins; a.ioff = L.ioff; a.inc = L.inc;
    a.noff = L.noff; a.ew = ew; a.src = L.src; a.sdst = L.sdst; a.dead = L.dead;
    a.omega = omega; a.delta = delta;
    a.pair = pair; a.score = score; a.key = key; a.status = status; a.bytes = bytes;
    a.evals = evals;
    const MlpParams M = widen(model);
    cudaError_t e = dalloc(ar, &a.next, 1);
    if (!e) e = cudaMemsetAsync(a.next, 0, sizeof(int32_t), s);
    if (e) return e;
    if (tensor_cores) {           // W1, b1, W2, b2 are the first 641 floats of MlpParams
        float *w = nullptr;
        e = dalloc(ar, &w, kMlpParams);
        if (!e) e = cudaMemcpyAsync(w, &M, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, s);
        if (e) return e;
        a.tc = 1;
        a.tcw = w;
    }
    const int sms = num_sms();
    const size_t dense_smem = 2 * sizeof(int32_t) * (size_t)L.V;
    if (dense_smem + sizeof(LearnQueue) + 4096 <= (size_t)max_smem &&
        !(debug & (HGP_DEBUG_FORCE_GLOBAL | HGP_DEBUG_FORCE_CLUSTER))) {
        e = allow_dynamic_smem(k_score_learned<true>);
        if (e) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_score_learned<true>,
                                                          kLearnThreads, dense_smem);
        if (e) return e;
        if (per_sm < 1) per_sm = 1;
        int blocks = sms * per_sm;
        if (blocks > L.V) blocks = L.V;
        k_score_learned<true><<<blocks, kLearnThreads, dense_smem, s>>>(a, M);
        count_launch();
        return cudaGetLastError();
    }
    unsigned long long *d_work = nullptr;
    e = dalloc(ar, &d_work, 2);
    if (!e) e = cudaMemsetAsync(d_work, 0, 2 * sizeof(unsigned long long), s);
    if (e) return e;
    k_max_visits<<<sms * 8, 256, 0, s>>>(L.V, L.ioff, L.inc, L.poff, ew, d_work);
    count_launch();
    unsigned long long h_max[2] = {0, 0};
    e = cudaMemcpyAsync(h_max, d_work, sizeof(h_max), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return e;
    const unsigned long long h_work = h_max[0];
    // packed 16-bit counters fit: every hist(n, .) <= sum of omega over I(n),
    // every inter(n, .) <= |in(n)|
    const int32_t slice = (L.V + kLearnCluster - 1) / kLearnCluster;
    const size_t cl_smem = sizeof(uint32_t) * (size_t)slice;
    if (!(debug & HGP_DEBUG_FORCE_GLOBAL) && h_max[1] < 65536ull && L.max_in < 65536 &&
        cl_smem + sizeof(LearnQueue) + 4096 <= (size_t)max_smem) {
        e = allow_dynamic_smem(k_score_learned_cluster);
        if (e) return e;
        cudaLaunchConfig_t cfg = {};
        cfg.blockDim = dim3(kLearnThreads);
        cfg.dynamicSmemBytes = cl_smem;
        cfg.stream = s;
        cudaLaunchAttribute attr;
        attr.id = cudaLaunchAttributeClusterDimension;
        attr.val.clusterDim.x = kLearnCluster;
        attr.val.clusterDim.y = 1;
        attr.val.clusterDim.z = 1;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        cfg.gridDim = dim3(kLearnCluster);
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, k_score_learned_cluster, &cfg) != cudaSuccess ||
            clusters < 1)
            clusters = 1;
        (void)cudaGetLastError();
        if (clusters > L.V) clusters = L.V;
        cfg.gridDim = dim3(kLearnCluster * clusters);
        cfg.attrs = nullptr;       // the cluster shape comes from __cluster_dims__
        cfg.numAttrs = 0;
        e = cudaLaunchKernelEx(&cfg, k_score_learned_cluster, a, M, slice);
        count_launch();
        return e ? e : cudaGetLastError();
    }
    unsigned long long distinct = h_work < (unsigned long long)L.V ? h_work : (unsigned long long)L.V;
    unsigned long long gcap = 64;
    while (gcap < 2 * distinct) gcap <<= 1;
    if (gcap > (1ull << 30)) return cudaErrorMemoryAllocation;
    a.gcap = (int32_t)gcap;
    int blocks = sms * 2;
    if (blocks > L.V) blocks = L.V;
    e = dalloc(ar, &a.gkeys, (size_t)blocks * gcap);
    if (!e) e = dalloc(ar, &a.gvals, (size_t)blocks * gcap);
    if (!e) e = dalloc(ar, &a.ginter, (size_t)blocks * gcap);
    if (!e) e = dalloc(ar, &a.gused, (size_t)blocks * gcap);
    if (e) return e;
    k_score_learned<false><<<blocks, kLearnThreads, 0, s>>>(a, M);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------- matching
// best(m) over the children of m by (key, hist, id): the largest composite
// (key, hist) first, then the largest id among the children holding it.
__global__ void k_best_key(int32_t V, const int32_t *pair, const int32_t *score,
                           const int32_t *key, unsigned long long *bkey) {
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x) {
        int32_t m = pair[n];
        if (m >= 0) atomicMax(&bkey[m], composite(key[n], score[n]));
    }
}

__global__ void k_best_id(int32_t V, const int32_t *pair, const int32_t *score, const int32_t *key,
                          const unsigned long long *bkey, unsigned long long *best) {
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x) {
        int32_t m = pair[n];
        if (m >= 0 && composite(key[n], score[n]) == bkey[m])
            atomicMax(&best[m], (1ull << 32) | (uint32_t)n);
    }
}

// ---------------------------------------------------------------- training data
// The i-th output of SplitMix64 started at `seed` (Steele, Lea and Flood,
// 2014): golden-ratio increment, then two xor-shift-multiply rounds and a
// final xor-shift.
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed,
                                                            unsigned long long i) {
    unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// |A n B| of two ascending lists, and the summed weight of the common items.
__device__ __forceinline__ void intersect(const int32_t *A, int32_t a0, int32_t a1, const int32_t *B,
                                          int32_t b0, int32_t b1, const int32_t *wt, int64_t *cnt,
                                          int64_t *wsum) {
    int64_t c = 0, s = 0;
    while (a0 < a1 && b0 < b1) {
        int32_t x = A[a0], y = B[b0];
        if (x < y) ++a0;
        else if (x > y) ++b0;
        else { ++c; if (wt) s += wt[x]; ++a0; ++b0; }
    }
    *cnt = c;
    *wsum = s;
}

// Slot s = n * per_node + k: e = I(n)[u0 mod |I(n)|], m = pins(e)[u1 mod |e|]
// (input pin order), u0/u1 = outputs 2s and 2s + 1 of SplitMix64(seed).
__global__ void k_learn_samples(int32_t N, int32_t per_node, unsigned long long seed,
                                const int32_t *part, const int32_t *w, const int32_t *poff,
                                const int32_t *pins, const int32_t *ioff, const int32_t *inc,
                                const int32_t *noff, const int32_t *inn, const int32_t *ew,
                                float *x, float *y, int32_t *partner) {
    const int64_t S = (int64_t)N * per_node;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < S;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int32_t n = (int32_t)(s / per_node);
        const int32_t deg = ioff[n + 1] - ioff[n];
        int32_t m = n;
        if (deg > 0) {
            unsigned long long u0 = splitmix64_at(seed, 2ull * (unsigned long long)s);
            unsigned long long u1 = splitmix64_at(seed, 2ull * (unsigned long long)s + 1ull);
            int32_t e = inc[ioff[n] + (int32_t)(u0 % (unsigned long long)deg)];
            int32_t sz = poff[e + 1] - poff[e];
            m = pins[poff[e] + (int32_t)(u1 % (unsigned long long)sz)];
        }
        float *xs = x + s * kMlpIn;
        if (m == n) {
            for (int i = 0; i < kMlpIn; ++i) xs[i] = 0.0f;
            y[s] = -1.0f;
            if (partner) partner[s] = -1;
            continue;
        }
        int64_t shared = 0, hist = 0, inter = 0, dummy = 0;
        intersect(inc, ioff[n], ioff[n + 1], inc, ioff[m], ioff[m + 1], ew, &shared, &hist);
        intersect(inn, noff[n], noff[n + 1], inn, noff[m], noff[m + 1], nullptr, &inter, &dummy);
        const int64_t in_n = noff[n + 1] - noff[n], in_m = noff[m + 1] - noff[m];
        const int64_t dn = deg, dm = ioff[m + 1] - ioff[m];
        const int64_t wn = w[n], wm = w[m];
        xs[0] = lg1p_dev(hist);
        xs[1] = lg1p_dev(in_n + in_m - inter);
        xs[2] = lg1p_dev(min(dn, dm));
        xs[3] = lg1p_dev(max(dn, dm));
        xs[4] = lg1p_dev(min(in_n, in_m));
        xs[5] = lg1p_dev(max(in_n, in_m));
        xs[6] = lg1p_dev(min(wn, wm));
        xs[7] = lg1p_dev(max(wn, wm));
        y[s] = part[n] == part[m] ? 1.0f : 0.0f;
        if (partner) partner[s] = m;
    }
}

cudaError_t run_learn_samples(const Level &L0, const int32_t *ew, const int32_t *part_ids,
                              uint64_t seed, int32_t per_node, float *x, float *y,
                              int32_t *partner, cudaStream_t s) {
    int64_t S = (int64_t)L0.V * per_node;
    int blocks = div_up(S, 256);
    if (blocks > num_sms() * 16) blocks = num_sms() * 16;
    if (blocks < 1) blocks = 1;
    k_learn_samples<<<blocks, 256, 0, s>>>(L0.V, per_node, seed, part_ids, L0.w, L0.poff, L0.pins,
                                           L0.ioff, L0.inc, L0.noff, L0.inn, ew, x, y, partner);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------- training
constexpr int kTrainThreads = 256;
constexpr int kTrainWarps = kTrainThreads / 32;
constexpr int kTrainRow = kMlpParams + 2;          // gradients, loss sum, valid count

// round-to-nearest-even to bfloat16, back to float
__device__ __forceinline__ float round_bf16(float f) {
    uint32_t u = __float_as_uint(f);
    u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
    return __uint_as_float(u);
}

// Gradient of the mean logistic loss over samples start .. start + B - 1
// (indices taken modulo count; samples with label < 0 skipped).  Layout of
// the parameters: W1[j][i] at 8 j + i, b1 at 512 + j, W2 at 576 + j, b2 at 640.
// Each block writes its sums to partial[blockIdx.x][0 .. kTrainRow).
__global__ void __launch_bounds__(kTrainThreads)
k_train_grad(const float *x, const float *y, int64_t count, int64_t start, int32_t B,
             const float *params, float *partial) {
    __shared__ float W[kMlpParams];
    __shared__ float acc[kTrainWarps][kTrainRow];
    for (int q = threadIdx.x; q < kMlpParams; q += kTrainThreads) W[q] = round_bf16(params[q]);
    for (int q = lane_id(); q < kTrainRow; q += 32) acc[warp_id()][q] = 0.0f;
    __syncthreads();
    const int32_t per_round = gridDim.x * kTrainThreads;
    for (int32_t base = blockIdx.x * kTrainThreads; base < B; base += per_round) {
        // warp-uniform loop: every lane takes part in the reductions
        const int32_t t = base + threadIdx.x;
        bool ok = t < B;
        float xs[kMlpIn];
        float yy = 0.0f;
        if (ok) {
            int64_t idx = (start + t) % count;
            yy = y[idx];
            ok = yy >= 0.0f;
#pragma unroll
            for (int i = 0; i < kMlpIn; ++i) xs[i] = x[idx * kMlpIn + i];
        }
        if (!ok) {
#pragma unroll
            for (int i = 0; i < kMlpIn; ++i) xs[i] = 0.0f;
        }
        float a[kMlpHid];
        float s = W[640];
#pragma unroll
        for (int j = 0; j < kMlpHid; ++j) {
            float h = W[512 + j];
#pragma unroll
            for (int i = 0; i < kMlpIn; ++i) h = fmaf(W[j * kMlpIn + i], xs[i], h);
            a[j] = h;
            s = fmaf(W[576 + j], h > 0.0f ? h : 0.0f, s);
        }
        const float ds = ok ? 1.0f / (1.0f + expf(-s)) - yy : 0.0f;
        const float loss = ok ? fmaxf(s, 0.0f) - s * yy + log1pf(expf(-fabsf(s))) : 0.0f;
        float r = warp_sum(loss);
        float c = warp_sum(ok ? 1.0f : 0.0f);
        float g2 = warp_sum(ds);
        if (lane_id() == 0) {
            acc[warp_id()][kMlpParams] += r;
            acc[warp_id()][kMlpParams + 1] += c;
            acc[warp_id()][640] += g2;
        }
#pragma unroll
        for (int j = 0; j < kMlpHid; ++j) {
            const float h = a[j] > 0.0f ? a[j] : 0.0f;
            const float da = a[j] > 0.0f ? ds * W[576 + j] : 0.0f;
            float gw2 = warp_sum(ds * h);
            float gb1 = warp_sum(da);
            float gw1[kMlpIn];
#pragma unroll
            for (int i = 0; i < kMlpIn; ++i) gw1[i] = warp_sum(da * xs[i]);
            if (lane_id() == 0) {
                acc[warp_id()][576 + j] += gw2;
                acc[warp_id()][512 + j] += gb1;
#pragma unroll
                for (int i = 0; i < kMlpIn; ++i) acc[warp_id()][j * kMlpIn + i] += gw1[i];
            }
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kTrainRow; q += kTrainThreads) {
        float v = 0.0f;
        for (int w = 0; w < kTrainWarps; ++w) v += acc[w][q];
        partial[(int64_t)blockIdx.x * kTrainRow + q] = v;
    }
}

// Sums the blocks' partials in block order and applies one Adam step
// (Kingma and Ba, 2015) to the float32 master parameters.
__global__ void k_train_adam(const float *partial, int32_t blocks, float *params, float *m,
                             float *v, int32_t t, float lr, float beta1, float beta2, float eps,
                             float *loss_out) {
    __shared__ float s_cnt;
    if (threadIdx.x == 0) {
        float c = 0.0f, l = 0.0f;
        for (int b = 0; b < blocks; ++b) {
            c += partial[(int64_t)b * kTrainRow + kMlpParams + 1];
            l += partial[(int64_t)b * kTrainRow + kMlpParams];
        }
        s_cnt = c;
        if (loss_out) *loss_out = c > 0.0f ? l / c : 0.0f;
    }
    __syncthreads();
    const float cnt = s_cnt;
    for (int q = threadIdx.x; q < kMlpParams; q += blockDim.x) {
        float g = 0.0f;
        for (int b = 0; b < blocks; ++b) g += partial[(int64_t)b * kTrainRow + q];
        g = cnt > 0.0f ? g / cnt : 0.0f;
        float mq = beta1 * m[q] + (1.0f - beta1) * g;
        float vq = beta2 * v[q] + (1.0f - beta2) * g * g;
        m[q] = mq;
        v[q] = vq;
        float mh = mq / (1.0f - powf(beta1, (float)t));
        float vh = vq / (1.0f - powf(beta2, (float)t));
        params[q] -= lr * mh / (sqrtf(vh) + eps);
    }
}

}  // namespace hgp

using namespace hgp;

extern "C" int hgp_train_mlp(const float *x, const float *y, int64_t count,
                             const hgp_train_options *opt, float *params, float *adam, float *loss,
                             void *stream) {
    if (!x || !y || !opt || !params || !adam || count < 1) return HGP_ERR_INVALID_ARG;
    if (opt->steps < 0 || opt->batch < 1 || opt->first_step < 1 || !(opt->lr > 0.0f) ||
        !(opt->beta1 >= 0.0f && opt->beta1 < 1.0f) || !(opt->beta2 >= 0.0f && opt->beta2 < 1.0f) ||
        !(opt->eps > 0.0f))
        return HGP_ERR_INVALID_ARG;
    for (int i = 0; i < 3; ++i)
        if (opt->reserved[i]) return HGP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int blocks = div_up(opt->batch, kTrainThreads);
    if (blocks > 128) blocks = 128;
    float *d_p = nullptr, *d_partial = nullptr, *d_loss = nullptr;
    size_t np = (size_t)kMlpParams;
    size_t loss_n = opt->steps > 0 ? (size_t)opt->steps : 1;
    cudaError_t e = cudaMallocAsync(&d_p, sizeof(float) * 3 * np, s);
    if (!e) e = cudaMallocAsync(&d_partial, sizeof(float) * (size_t)blocks * kTrainRow, s);
    if (!e) e = cudaMallocAsync(&d_loss, sizeof(float) * loss_n, s);
    if (!e) e = cudaMemcpyAsync(d_p, params, sizeof(float) * np, cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(d_p + np, adam, sizeof(float) * 2 * np, cudaMemcpyHostToDevice, s);
    for (int32_t k = 0; !e && k < opt->steps; ++k) {
        int64_t start = ((int64_t)k * opt->batch) % count;
        k_train_grad<<<blocks, kTrainThreads, 0, s>>>(x, y, count, start, opt->batch, d_p, d_partial);
        k_train_adam<<<1, 704, 0, s>>>(d_partial, blocks, d_p, d_p + np, d_p + 2 * np,
                                       opt->first_step + k, opt->lr, opt->beta1, opt->beta2, opt->eps,
                                       d_loss + k);
        count_launch();
        count_launch();
        e = cudaGetLastError();
    }
    if (!e) e = cudaMemcpyAsync(params, d_p, sizeof(float) * np, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(adam, d_p + np, sizeof(float) * 2 * np, cudaMemcpyDeviceToHost, s);
    if (!e && loss && opt->steps > 0)
        e = cudaMemcpyAsync(loss, d_loss, sizeof(float) * (size_t)opt->steps, cudaMemcpyDeviceToHost, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (d_p) cudaFreeAsync(d_p, s);
    if (d_partial) cudaFreeAsync(d_partial, s);
    if (d_loss) cudaFreeAsync(d_loss, s);
    cudaStreamSynchronize(s);
    return (e || e2) ? HGP_ERR_CUDA : HGP_OK;
}

extern "C" int hgp_model_from_params(const float *params, int32_t key_bits, hgp_model *out) {
    if (!params || !out || key_bits < 0 || key_bits > 20) return HGP_ERR_INVALID_ARG;
    auto to_bf16 = [](float f) -> uint16_t {
        uint32_t u;
        memcpy(&u, &f, sizeof(u));
        return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
    };
    memset(out, 0, sizeof(*out));
    for (int q = 0; q < kMlpHid * kMlpIn; ++q) out->w1[q] = to_bf16(params[q]);
    for (int j = 0; j < kMlpHid; ++j) {
        out->b1[j] = to_bf16(params[512 + j]);
        out->w2[j] = to_bf16(params[576 + j]);
    }
    out->b2 = to_bf16(params[640]);
    out->key_bits = (int16_t)key_bits;
    return HGP_OK;
}
