// Internal declarations of the GB300 partitioning library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/hgp.h"

namespace hgp {

constexpr int kWarp = 32;

// Device-side status word (first failure wins; host reads it at sync points).
enum DevStatus : int32_t {
    kDevOk = 0,
    kDevLimit = 1,        // a bounded loop ran out of budget
    kDevBadInput = 2,     // input validation failed
    kDevInternal = 3      // a consistency check failed
};

// One level of the hierarchy, all arrays in device memory (int32 CSR).
//   pins(e)  : poff[E+1], pins[P]  node set of each hyperedge (any order)
//   I(n)     : ioff[V+1], inc[P]   incident hyperedges, ascending
//   in(n)    : noff[V+1], inn[Q]   inbound hyperedges, ascending
//   src[e]   : the level's node holding the source of e
//   sdst[e]  : role byte of e for the Delta count (see counts_in): bit 0 --
//              the node holding the source has e in its in(); bit 1 -- every
//              other node of e does.  Inbound Delta (the paper's): 2, plus 1
//              once the source's node also holds a destination; incident: 3;
//              outbound: 1
struct Level {
    int32_t V = 0, E = 0;
    int64_t P = 0, Q = 0;
    int32_t max_in = 0;         // largest |in(n)| of the level
    int32_t max_edge = 0;       // largest |pins(e)| of the level
    int32_t *w = nullptr;
    int32_t *poff = nullptr, *pins = nullptr;
    int32_t *ioff = nullptr, *inc = nullptr;
    int32_t *noff = nullptr, *inn = nullptr;
    int32_t *src = nullptr;
    uint8_t *sdst = nullptr;
    int32_t *gamma = nullptr;   // [V] map to level+1 (when this level was contracted)
    int32_t *match = nullptr;   // [V]
    // carried from the previous level's scoring (null at level 0):
    //   dead[n]   n had no valid candidate one level down; validity only shrinks
    //             under merging, so n has none now and is no one's candidate
    //   merged[n] n is a pair formed by the last matching
    //   thr[n]    (score << 32 | id) of n's previous candidate, in previous-level
    //             ids, for unmerged n (0 otherwise): every unmerged neighbour
    //             ranked above it was already found invalid
    //   old_id[n] previous-level id of n's smaller member
    uint8_t *dead = nullptr, *merged = nullptr;
    unsigned long long *thr = nullptr;
    int32_t *old_id = nullptr;
    // I(n) lives with in(n) in storage that the next-but-one contraction
    // reuses; refinement then rebuilds it from the pins
    bool inc_rolling = false;
    // in() bitmaps of this level's scoring (null when it used none): row n is
    // bm[n * bm_words ..], bit e set iff e in in(n); kept with in(n), so the
    // next level can build its rows as ORs of the matched pairs' rows
    uint32_t *bm = nullptr;
    int32_t bm_words = 0;
};

// ---------------- stream-ordered device memory ----------------
// Bump allocator over device chunks obtained on `stream` from the handle's
// hgp_allocator (cudaMallocAsync / cudaFreeAsync when it has none).  reset()
// makes every allocation dead and reuses the chunks from the start; this is
// safe because all work runs in order on the one stream.  With min_chunk = 0
// every allocation gets an exact chunk of its own.
struct Arena {
    struct Chunk { char *base; size_t size; };
    cudaStream_t stream = nullptr;
    const hgp_allocator *user = nullptr;   // null: cudaMallocAsync / cudaFreeAsync
    size_t min_chunk = 0;
    std::vector<Chunk> chunks;
    size_t cur = 0, off = 0;
    cudaError_t alloc(void **p, size_t bytes);
    void reset() { cur = 0; off = 0; }
    void release_all();
};

template <typename T>
inline cudaError_t dalloc(Arena &a, T **p, size_t count) {
    return a.alloc(reinterpret_cast<void **>(p), sizeof(T) * (count ? count : 1));
}

// Event pairs around every proposal launch (or contraction phase) of a
// partition (timing runs), with the algorithmic bytes they move.
struct PropTiming {
    unsigned long long *bytes = nullptr;   // device counter
    unsigned long long host_bytes = 0;     // counted on the host
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
};

// Proposal buffers carried from one refinement pass to the next finer level.
struct PropReuse {
    int32_t *out_gain = nullptr, *out_pd = nullptr;          // this pass's proposals [V]
    const int32_t *prev_gain = nullptr, *prev_pd = nullptr;  // coarser level's, or null
    const int32_t *gamma = nullptr, *match = nullptr;        // this level's gamma / match
    int32_t *applied_flag = nullptr;   // device: in = coarser pass applied moves; out = this pass
};

// ---------------- launch bookkeeping ----------------
extern thread_local int64_t g_launches;
inline void count_launch() { ++g_launches; }

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Raises a kernel's dynamic shared-memory limit to the device maximum, once
// per (device, kernel) under a lock.  The limit is process-wide state, so
// setting it per launch from several host threads (hgp_partition_batch)
// could lower it between another thread's set and launch.
cudaError_t allow_dynamic_smem_ptr(const void *kernel);
template <typename K>
inline cudaError_t allow_dynamic_smem(K kernel) {
    return allow_dynamic_smem_ptr(reinterpret_cast<const void *>(kernel));
}
int num_sms();

// ---------------- primitives (k_prims.cu) ----------------
// Exclusive scan of n int32 values (in may alias out); if total != null the
// sum of all values is written to *total (device pointer).
cudaError_t exclusive_scan_i32(Arena &a, const int32_t *in, int32_t *out, int64_t n,
                               int32_t *total, cudaStream_t s);
cudaError_t inclusive_scan_i64(Arena &a, const int64_t *in, int64_t *out, int64_t n,
                               cudaStream_t s);
// Stable LSD radix sort of (key, value) pairs by the low `bits` bits of the
// key.  Sorted data ends in keys_out/vals_out (may be null vals).
cudaError_t radix_sort_pairs(Arena &a, const uint32_t *keys_in, const int32_t *vals_in,
                             uint32_t *keys_out, int32_t *vals_out, int64_t n, int bits,
                             cudaStream_t s);
// Row id of every CSR entry: row_of[j] = r for off[r] <= j < off[r+1].
void expand_rows(const int32_t *off, int32_t rows, int32_t *row_of, cudaStream_t s);
// off[r] = exclusive prefix of counts (rows+1 entries); total in off[rows].
cudaError_t counts_to_offsets(Arena &a, const int32_t *counts, int32_t *off, int32_t rows,
                              cudaStream_t s);
void fill_i32(int32_t *p, int32_t v, int64_t n, cudaStream_t s);
void iota_i32(int32_t *p, int64_t n, cudaStream_t s);

inline int bits_for(int64_t maxval) {   // bits to hold values in [0, maxval]
    int b = 0;
    while (b < 32 && ((int64_t)1 << b) <= maxval) ++b;
    return b < 1 ? 1 : b;
}

// ---------------- device helpers ----------------
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }

// Whether level node m has hyperedge e in its in() (the set Delta counts),
// from e's source node and role byte.
__device__ __forceinline__ bool counts_in(int32_t m, int32_t src_e, uint8_t role) {
    return (m == src_e) ? (role & 1) != 0 : (role & 2) != 0;
}

__device__ __forceinline__ void set_status(int32_t *status, int32_t code) {
    atomicCAS(status, 0, code);
}

// lower_bound over ascending a[lo, hi)
__device__ __forceinline__ int32_t lower_bound_i32(const int32_t *a, int32_t lo, int32_t hi,
                                                   int32_t x) {
    while (lo < hi) {
        int32_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ bool contains_sorted(const int32_t *a, int32_t lo, int32_t hi,
                                                int32_t x) {
    int32_t p = lower_bound_i32(a, lo, hi, x);
    return p < hi && a[p] == x;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace hgp
