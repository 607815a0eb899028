// hgp_score_noalloc: candidate scoring of one hypergraph level without any
// device allocation.
//
// Some callers cannot allocate device memory while they run: code executing
// inside another framework's memory pool or allocator callback, a runtime
// that has reserved all device memory up front, or a step that must not
// synchronise the device the way cudaMalloc/cudaFree can.  This entry point
// runs the same scoring kernel as hgp_partition's first level, but its only
// scratch -- the per-node bitmaps of in() used for union counts, and a small
// header word for the largest |in(n)| -- lives in one file-scope device array
// of fixed size, so nothing is allocated per call.
//
// The array's host-side name is only a stand-in for the device object, so the
// device address is looked up with cudaGetSymbolAddress once per device (with
// that device current) on the first call made on it, and that address is the
// one passed to the kernels.
#include "k_score.cuh"

namespace hgp {

// 16 MiB, held by every GPU that loads the library until the process exits.
constexpr size_t kNoAllocScratchBytes = 16u << 20;
constexpr size_t kNoAllocHeaderBytes = 256;          // [0] = largest |in(n)|
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocScratchBytes / 4];

constexpr int kMaxDevices = 64;
static void *s_scratch_ptr[kMaxDevices];             // per-device address, set once

static __global__ void k_noalloc_max_in(int32_t V, const int32_t *noff, int32_t *out) {
    int32_t mi = 0;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x)
        mi = max(mi, noff[n + 1] - noff[n]);
    mi = max(mi, __shfl_xor_sync(0xffffffffu, mi, 16));
    mi = max(mi, __shfl_xor_sync(0xffffffffu, mi, 8));
    mi = max(mi, __shfl_xor_sync(0xffffffffu, mi, 4));
    mi = max(mi, __shfl_xor_sync(0xffffffffu, mi, 2));
    mi = max(mi, __shfl_xor_sync(0xffffffffu, mi, 1));
    if (lane_id() == 0) atomicMax(out, mi);
}

}  // namespace hgp

using namespace hgp;

extern "C" int hgp_score_noalloc(int32_t num_nodes, int32_t num_edges, const int32_t *offsets,
                                 const int32_t *pins, const int32_t *inc_offsets,
                                 const int32_t *inc, const int32_t *in_offsets,
                                 const int32_t *in_edges, const int32_t *node_weights,
                                 const int32_t *edge_weights, int64_t omega, int64_t delta,
                                 int32_t *pair, int32_t *score, void *stream) {
    if (num_nodes < 1 || num_edges < 0 || omega < 1 || delta < 0) return HGP_ERR_INVALID_ARG;
    if (!offsets || !inc_offsets || !in_offsets || !node_weights || !pair || !score)
        return HGP_ERR_INVALID_ARG;
    if (num_edges > 0 && (!pins || !inc || !in_edges || !edge_weights)) return HGP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HGP_ERR_CUDA;
    if (!s_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return HGP_ERR_CUDA;
        s_scratch_ptr[dev] = p;
    }
    unsigned char *scratch = static_cast<unsigned char *>(s_scratch_ptr[dev]);
    int32_t *d_max_in = reinterpret_cast<int32_t *>(scratch);
    uint32_t *bm_area = reinterpret_cast<uint32_t *>(scratch + kNoAllocHeaderBytes);

    int max_smem = 0;
    if (cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return HGP_ERR_CUDA;
    int32_t words = ((num_edges + 31) / 32 + 3) & ~3;
    ScoreArgs a{};
    a.V = num_nodes; a.E = num_edges;
    a.w = node_weights; a.poff = offsets; a.pins = pins; a.ioff = inc_offsets; a.inc = inc;
    a.noff = in_offsets; a.inn = in_edges; a.ew = edge_weights;
    a.omega = omega; a.delta = delta;
    a.pair = pair; a.score = score;
    a.status = d_max_in + 1;          // the kernel's status word (limits are never hit here)
    a.next = d_max_in + 2;            // the kernel's node counter
    a.vec_pins = 0;                   // the caller's pins: no alignment or padding is promised
    // largest |in(n)|: union counts (and bitmaps) are needed only if 2 * max > Delta
    if (cudaMemsetAsync(d_max_in, 0, 3 * sizeof(int32_t), s) != cudaSuccess) return HGP_ERR_CUDA;
    k_noalloc_max_in<<<num_sms() * 4, 256, 0, s>>>(num_nodes, in_offsets, d_max_in);
    int32_t max_in = 0;
    if (cudaMemcpyAsync(&max_in, d_max_in, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return HGP_ERR_CUDA;
    if (2 * (int64_t)max_in > delta) {
        size_t need = sizeof(uint32_t) * (size_t)num_nodes * (size_t)words;
        if (words > 8192 || need > kNoAllocScratchBytes - kNoAllocHeaderBytes)
            return HGP_ERR_SCRATCH_LIMIT;
        // the array keeps the previous call's bits: clear this call's rows
        if (cudaMemsetAsync(bm_area, 0, need, s) != cudaSuccess) return HGP_ERR_CUDA;
        int blocks = div_up((int64_t)num_nodes * 32, 256);
        if (blocks > num_sms() * 16) blocks = num_sms() * 16;
        k_in_bitmap<<<blocks, 256, 0, s>>>(num_nodes, in_offsets, in_edges, words, bm_area);
        a.bm = bm_area;
        a.bm_words = words;
    }
    // dense shared-memory histogram only (no global tables)
    size_t smem = sizeof(uint32_t) * (size_t)a.bm_words + sizeof(int32_t) * (size_t)num_nodes;
    if (smem + 2048 > (size_t)max_smem) return HGP_ERR_SCRATCH_LIMIT;
    if (allow_dynamic_smem(k_score<true>) != cudaSuccess)
        return HGP_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_score<true>, kScoreThreads, smem) !=
        cudaSuccess)
        return HGP_ERR_CUDA;
    if (per_sm < 1) per_sm = 1;
    int blocks = num_sms() * per_sm;
    if (blocks > num_nodes) blocks = num_nodes;
    k_score<true><<<blocks, kScoreThreads, smem, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? HGP_OK : HGP_ERR_CUDA;
}
