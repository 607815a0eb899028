// Level-0 incidence structure (Sec. II-A, II-C): validation of the input CSR,
// then I(n) and in(n) as sorted compressed-sparse sets.
//
// I(n) is the transpose of the pins: the (node, edge) pairs are stably
// radix-sorted by node, and since they are produced in edge order each
// node's list comes out in ascending edge order.  in(n) is the same
// transpose restricted to destination pins (every pin but the first of its
// edge).  A repeated pin inside an edge shows up as two equal adjacent
// entries of a node's I(n) list.
#include "hgp_internal.cuh"

namespace hgp {

struct ValidateOut {
    int32_t bad;                 // first failing rule (0 = none)
    int32_t pad;
    unsigned long long wsum, esum;
};

__global__ void k_validate_edges(int32_t E, const int32_t *off, const int32_t *ew,
                                 ValidateOut *out) {
    unsigned long long es = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < E;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (off[i + 1] <= off[i]) atomicCAS(&out->bad, 0, 1);     // empty or decreasing
        int32_t w = ew[i];
        if (w < 1) atomicCAS(&out->bad, 0, 4);
        es += (unsigned long long)(w > 0 ? w : 0);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && off[0] != 0) atomicCAS(&out->bad, 0, 1);
    es = warp_sum(es);
    if (lane_id() == 0 && es) atomicAdd(&out->esum, es);
}

__global__ void k_validate_nodes(int32_t N, int64_t P, const int32_t *pins, const int32_t *w,
                                 ValidateOut *out) {
    unsigned long long ws = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t v = pins[i];
        if (v < 0 || v >= N) atomicCAS(&out->bad, 0, 2);
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t x = w[i];
        if (x < 1) atomicCAS(&out->bad, 0, 5);
        ws += (unsigned long long)(x > 0 ? x : 0);
    }
    ws = warp_sum(ws);
    if (lane_id() == 0 && ws) atomicAdd(&out->wsum, ws);
}

// pairs (node, edge) of all pins and (with dst_pairs) of destination pins
__global__ void k_incidence_pairs(int32_t E, const int32_t *off, const int32_t *pins,
                                  const int32_t *row_of, uint32_t *kI, int32_t *vI, uint32_t *kN,
                                  int32_t *vN, int32_t *src, int32_t *degI, int32_t *degN,
                                  int32_t dst_pairs) {
    int64_t P = off[E];
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < P;
         j += (int64_t)gridDim.x * blockDim.x) {
        int32_t e = row_of[j], n = pins[j];
        kI[j] = (uint32_t)n;
        vI[j] = e;
        atomicAdd(&degI[n], 1);
        if (j == off[e]) {
            src[e] = n;
        } else if (dst_pairs) {
            int64_t q = j - e - 1;     // each edge drops exactly its first pin
            kN[q] = (uint32_t)n;
            vN[q] = e;
            atomicAdd(&degN[n], 1);
        }
    }
}

// outbound Delta: in(n) = {e : src(e) = n}, one (source, edge) pair per edge
__global__ void k_source_pairs(int32_t E, const int32_t *src, uint32_t *kN, int32_t *vN,
                               int32_t *degN) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
         e += (int64_t)gridDim.x * blockDim.x) {
        kN[e] = (uint32_t)src[e];
        vN[e] = (int32_t)e;
        atomicAdd(&degN[src[e]], 1);
    }
}

__global__ void k_check_dups(int32_t N, const int32_t *ioff, const int32_t *inc,
                             ValidateOut *out) {
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N;
         n += (int64_t)gridDim.x * blockDim.x) {
        for (int32_t k = ioff[n] + 1; k < ioff[n + 1]; ++k)
            if (inc[k] == inc[k - 1]) { atomicCAS(&out->bad, 0, 3); break; }
    }
}

static int grid1d(int64_t n) {
    int b = div_up(n, 256);
    int cap = num_sms() * 8;
    return b < 1 ? 1 : (b > cap ? cap : b);
}

// Validates (offsets, pins, w, ew) already on the device and builds level 0.
// delta_mode chooses the hyperedge sets that Delta counts, in(n): 0 inbound
// (n a destination of e: the paper's), 1 incident (in(n) = I(n)), 2 outbound
// (n the source of e); the role bytes sdst follow it (see Level).
// Returns 0 on success, or the failing rule code (> 0), or -1 on CUDA error
// (then *cerr holds it).
int run_build_level0(Arena &keep, Arena &tmp, int32_t N, int32_t E, Level &L, const int32_t *ew,
                     int32_t delta_mode, int64_t *wsum_e, cudaError_t *cerr, std::string *why,
                     cudaStream_t s) {
    *cerr = cudaSuccess;
    ValidateOut *dv = nullptr;
    cudaError_t e = dalloc(tmp, &dv, 1);
    if (e) { *cerr = e; return -1; }
    cudaMemsetAsync(dv, 0, sizeof(ValidateOut), s);
    if (E > 0) {
        k_validate_edges<<<grid1d(E), 256, 0, s>>>(E, L.poff, ew, dv);
        count_launch();
    }
    int32_t h_P = 0;
    e = cudaMemcpyAsync(&h_P, L.poff + E, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    ValidateOut hv{};
    if (!e) e = cudaMemcpyAsync(&hv, dv, sizeof(hv), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) { *cerr = e; return -1; }
    if (hv.bad) {
        *why = "offsets must start at 0 and increase strictly (no empty hyperedge); edge weights >= 1";
        return hv.bad;
    }
    if (hv.esum > 0x7fffffffull) { *why = "sum of edge weights must be < 2^31"; return 6; }
    *wsum_e = (int64_t)hv.esum;
    int64_t P = h_P;
    L.P = P;
    k_validate_nodes<<<grid1d(P > N ? P : N), 256, 0, s>>>(N, P, L.pins, L.w, dv);
    count_launch();
    e = cudaMemcpyAsync(&hv, dv, sizeof(hv), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) { *cerr = e; return -1; }
    if (hv.bad) { *why = "pins must lie in [0, num_nodes) and node weights must be >= 1"; return hv.bad; }
    if (hv.wsum > 0x7fffffffull) { *why = "sum of node weights must be < 2^31"; return 6; }

    int64_t Q = delta_mode == 0 ? P - E : delta_mode == 2 ? E : 0;
    L.Q = Q;
    int32_t *row_of = nullptr, *vI = nullptr, *vN = nullptr, *degI = nullptr, *degN = nullptr;
    uint32_t *kI = nullptr, *kN = nullptr, *kIs = nullptr, *kNs = nullptr;
    e = dalloc(tmp, &row_of, P);
    if (!e) e = dalloc(tmp, &kI, P);
    if (!e) e = dalloc(tmp, &vI, P);
    if (!e) e = dalloc(tmp, &kN, Q);
    if (!e) e = dalloc(tmp, &vN, Q);
    if (!e) e = dalloc(tmp, &kIs, P);
    if (!e) e = dalloc(tmp, &kNs, Q);
    if (!e) e = dalloc(tmp, &degI, N);
    if (!e) e = dalloc(tmp, &degN, N);
    if (!e) e = dalloc(keep, &L.inc, P);
    if (!e) e = dalloc(keep, &L.ioff, (size_t)N + 1);
    if (!e && delta_mode != 1) e = dalloc(keep, &L.inn, Q);
    if (!e && delta_mode != 1) e = dalloc(keep, &L.noff, (size_t)N + 1);
    if (!e) e = dalloc(keep, &L.src, E);
    if (!e) e = dalloc(keep, &L.sdst, E);
    if (e) { *cerr = e; return -1; }
    cudaMemsetAsync(degI, 0, sizeof(int32_t) * (size_t)N, s);
    cudaMemsetAsync(degN, 0, sizeof(int32_t) * (size_t)N, s);
    // role bytes at level 0: inbound 2 (no node is both the source and a
    // destination of one edge), incident 3, outbound 1
    const int role = delta_mode == 0 ? 2 : delta_mode == 1 ? 3 : 1;
    cudaMemsetAsync(L.sdst, role, (size_t)(E > 0 ? E : 1), s);
    expand_rows(L.poff, E, row_of, s);
    if (P > 0) {
        k_incidence_pairs<<<grid1d(P), 256, 0, s>>>(E, L.poff, L.pins, row_of, kI, vI, kN, vN,
                                                    L.src, degI, degN, delta_mode == 0 ? 1 : 0);
        count_launch();
    }
    if (delta_mode == 2 && E > 0) {
        k_source_pairs<<<grid1d(E), 256, 0, s>>>(E, L.src, kN, vN, degN);
        count_launch();
    }
    int bits = bits_for(N > 0 ? N - 1 : 0);
    e = radix_sort_pairs(tmp, kI, vI, kIs, L.inc, P, bits, s);
    if (!e) e = counts_to_offsets(tmp, degI, L.ioff, N, s);
    if (delta_mode == 1) {                 // in(n) = I(n)
        L.noff = L.ioff;
        L.inn = L.inc;
        L.Q = P;
    } else {
        if (!e) e = radix_sort_pairs(tmp, kN, vN, kNs, L.inn, Q, bits, s);
        if (!e) e = counts_to_offsets(tmp, degN, L.noff, N, s);
    }
    if (e) { *cerr = e; return -1; }
    k_check_dups<<<grid1d(N), 256, 0, s>>>(N, L.ioff, L.inc, dv);
    count_launch();
    e = cudaMemcpyAsync(&hv, dv, sizeof(hv), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) { *cerr = e; return -1; }
    if (hv.bad) { *why = "a pin is repeated within a hyperedge"; return hv.bad; }
    return 0;
}

__global__ void k_pin_node_pairs(int64_t P, const int32_t *pins, int32_t *deg, uint32_t *key) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < P;
         j += (int64_t)gridDim.x * blockDim.x) {
        int32_t n = pins[j];
        key[j] = (uint32_t)n;
        atomicAdd(&deg[n], 1);
    }
}

// I(n) of a level from its pins (the transpose, as at level 0): pins are
// listed in edge order, so a stable sort by node leaves each node's
// hyperedges ascending -- the same sorted sets contraction forms as unions.
cudaError_t run_rebuild_incidence(Arena &ar, const Level &L, int32_t **ioff, int32_t **inc,
                                  cudaStream_t s) {
    int32_t *row_of = nullptr, *deg = nullptr;
    uint32_t *key = nullptr, *key_s = nullptr;
    cudaError_t e = dalloc(ar, ioff, (size_t)L.V + 1);
    if (!e) e = dalloc(ar, inc, L.P);
    if (!e) e = dalloc(ar, &row_of, L.P);
    if (!e) e = dalloc(ar, &deg, L.V);
    if (!e) e = dalloc(ar, &key, L.P);
    if (!e) e = dalloc(ar, &key_s, L.P);
    if (!e) e = cudaMemsetAsync(deg, 0, sizeof(int32_t) * (size_t)L.V, s);
    if (e) return e;
    expand_rows(L.poff, L.E, row_of, s);
    if (L.P > 0) {
        k_pin_node_pairs<<<grid1d(L.P), 256, 0, s>>>(L.P, L.pins, deg, key);
        count_launch();
    }
    e = radix_sort_pairs(ar, key, row_of, key_s, *inc, L.P, bits_for(L.V > 0 ? L.V - 1 : 0), s);
    if (!e) e = counts_to_offsets(ar, deg, *ioff, L.V, s);
    return e;
}

}  // namespace hgp
