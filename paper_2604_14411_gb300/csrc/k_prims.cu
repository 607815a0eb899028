// Device-wide primitives: scans, stable LSD radix sort, CSR helpers.
// These are the prefix-sum and sort building blocks of the level-0 incidence
// build (Sec. II-C) and of refinement (Sec. IV-B): all integer, all stable,
// so every result is deterministic.
#include <mutex>
#include <set>
#include <utility>

#include "hgp_internal.cuh"

namespace hgp {

cudaError_t allow_dynamic_smem_ptr(const void *kernel) {
    static std::mutex mu;
    static std::set<std::pair<int, const void *>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return e;
    std::lock_guard<std::mutex> lk(mu);
    if (done.count({dev, kernel})) return cudaSuccess;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kernel);
    if (e) return e;
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e) return e;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes);
    if (!e) done.insert({dev, kernel});
    return e;
}

thread_local int64_t g_launches = 0;

int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

cudaError_t Arena::alloc(void **p, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    // chunks from `empty` on hold nothing allocated since the last reset
    size_t empty = off == 0 ? cur : cur + 1;
    while (cur < chunks.size()) {
        if (off + bytes <= chunks[cur].size) {
            *p = chunks[cur].base + off;
            off += bytes;
            return cudaSuccess;
        }
        ++cur;
        off = 0;
    }
    // None of them fits.  Return them instead of keeping them: every earlier
    // use of them was enqueued on the stream before this point.  (Keeping them
    // let an arena grow without bound when allocation sizes creep upwards from
    // cycle to cycle, as they do when refinement walks from coarse to fine
    // levels.)  Pooled chunks get 1/8 slack for the same reason.
    for (size_t i = empty; i < chunks.size(); ++i) {
        if (user) user->free(user->ctx, chunks[i].base, chunks[i].size, stream);
        else cudaFreeAsync(chunks[i].base, stream);
    }
    if (empty < chunks.size()) chunks.resize(empty);
    size_t sz = min_chunk ? bytes + (bytes >> 3) : bytes;
    if (sz < min_chunk) sz = min_chunk;
    sz = (sz + 255) & ~(size_t)255;
    void *b = nullptr;
    if (user) {
        b = user->alloc(user->ctx, sz, stream);
        if (!b) return cudaErrorMemoryAllocation;
    } else {
        cudaError_t e = cudaMallocAsync(&b, sz, stream);
        if (e != cudaSuccess) return e;
    }
    chunks.push_back({static_cast<char *>(b), sz});
    cur = chunks.size() - 1;
    off = bytes;
    *p = b;
    return cudaSuccess;
}

void Arena::release_all() {
    for (auto &c : chunks) {
        if (user) user->free(user->ctx, c.base, c.size, stream);
        else cudaFreeAsync(c.base, stream);
    }
    chunks.clear();
    cur = off = 0;
}

// ---------------------------------------------------------------- scans
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ T block_exclusive_scan(T v, T *warp_tot, T *block_total) {
    int lane = lane_id(), w = warp_id();
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        T t = lane < (kScanThreads / 32) ? warp_tot[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = t;   // inclusive warp totals
    }
    __syncthreads();
    T before = (w > 0 ? warp_tot[w - 1] : T(0)) + x - v;
    if (block_total) *block_total = warp_tot[kScanThreads / 32 - 1];
    return before;
}

template <typename T>
__global__ void k_tile_sums(const T *in, int64_t n, T *sums) {
    __shared__ T wt[kScanThreads / 32];
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    T s = 0;
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        int64_t j = base + i;
        if (j < n) s += in[j];
    }
    s = warp_sum(s);
    if (lane_id() == 0) wt[warp_id()] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        T t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) t += wt[w];
        sums[blockIdx.x] = t;
    }
}

template <typename T, bool Inclusive>
__global__ void k_tile_scan(const T *in, T *out, int64_t n, const T *tile_offsets, T *total,
                            const T *tile_sums) {
    __shared__ T tile[kScanTile];
    __shared__ T wt[kScanThreads / 32];
    __shared__ T btot;
    __shared__ T s_off;
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    if (tile_sums) {               // offset of this tile = sum of the earlier tiles' sums
        T acc = 0;
        for (int t = threadIdx.x; t < (int)blockIdx.x; t += kScanThreads) acc += tile_sums[t];
        acc = warp_sum(acc);
        if (lane_id() == 0) wt[warp_id()] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            T o = 0;
            for (int w = 0; w < kScanThreads / 32; ++w) o += wt[w];
            s_off = o;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        int64_t j = base + i;
        tile[i] = j < n ? in[j] : T(0);
    }
    __syncthreads();
    T loc[kScanItems];
    T s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        loc[k] = tile[threadIdx.x * kScanItems + k];
        s += loc[k];
    }
    T pre = block_exclusive_scan<T>(s, wt, &btot);
    T off = tile_sums ? s_off : (tile_offsets ? tile_offsets[blockIdx.x] : T(0));
    T run = off + pre;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (Inclusive) { run += loc[k]; tile[threadIdx.x * kScanItems + k] = run; }
        else { tile[threadIdx.x * kScanItems + k] = run; run += loc[k]; }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        int64_t j = base + i;
        if (j < n) out[j] = tile[i];
    }
    if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total = off + btot;
}

template <typename T, bool Inclusive>
static cudaError_t scan_impl(Arena &a, const T *in, T *out, int64_t n, T *total, cudaStream_t s) {
    if (n <= 0) {
        if (total) return cudaMemsetAsync(total, 0, sizeof(T), s);
        return cudaSuccess;
    }
    int64_t tiles = (n + kScanTile - 1) / kScanTile;
    T *offs = nullptr, *sums = nullptr;
    if (tiles > 1) {
        cudaError_t e = dalloc(a, &sums, tiles);
        if (e) return e;
        k_tile_sums<T><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sums);
        count_launch();
        if (tiles > 4096) {        // many tiles: scan the tile sums recursively
            e = dalloc(a, &offs, tiles);
            if (e) return e;
            e = scan_impl<T, false>(a, sums, offs, tiles, (T *)nullptr, s);
            if (e) return e;
            sums = nullptr;
        }
    }
    k_tile_scan<T, Inclusive><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, n, offs, total, sums);
    count_launch();
    return cudaGetLastError();
}

cudaError_t exclusive_scan_i32(Arena &a, const int32_t *in, int32_t *out, int64_t n,
                               int32_t *total, cudaStream_t s) {
    return scan_impl<int32_t, false>(a, in, out, n, total, s);
}

cudaError_t inclusive_scan_i64(Arena &a, const int64_t *in, int64_t *out, int64_t n,
                               cudaStream_t s) {
    return scan_impl<int64_t, true>(a, in, out, n, (int64_t *)nullptr, s);
}

// ---------------------------------------------------------------- radix sort
// Stable LSD radix sort, 8-bit digits.  A tile of 2048 keys is ranked in 8
// rounds of 256 (one key per thread, in input order); within a round the
// rank among equal digits comes from __match_any_sync inside the warp plus
// per-warp digit counts of the lower warps, so equal keys keep input order.
constexpr int kSortThreads = 256;
constexpr int kSortRounds = 8;
constexpr int kSortTile = kSortThreads * kSortRounds;

__global__ void k_radix_hist(const uint32_t *keys, int64_t n, int shift, int32_t *counts,
                             int ntiles) {
    __shared__ int32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortRounds; ++r) {
        int64_t j = base + r * kSortThreads + threadIdx.x;
        if (j < n) atomicAdd(&h[(keys[j] >> shift) & 255u], 1);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_radix_scatter(const uint32_t *keys, const int32_t *vals, uint32_t *ko,
                                int32_t *vo, int64_t n, int shift, const int32_t *offsets,
                                int ntiles) {
    __shared__ int32_t base_cnt[256];
    __shared__ int32_t gofs[256];
    __shared__ int32_t wcnt[kSortThreads / 32][256];
    int tid = threadIdx.x, lane = lane_id(), w = warp_id();
    base_cnt[tid] = 0;
    gofs[tid] = offsets[(int64_t)tid * ntiles + blockIdx.x];
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < kSortRounds; ++r) {
#pragma unroll
        for (int q = 0; q < kSortThreads / 32; ++q) wcnt[q][tid] = 0;
        __syncthreads();
        int64_t j = base + r * kSortThreads + tid;
        bool valid = j < n;
        uint32_t key = valid ? keys[j] : 0u;
        int d = valid ? (int)((key >> shift) & 255u) : 256;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & lt);
        if (valid && rank == 0) wcnt[w][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            int pre = base_cnt[d];
            for (int q = 0; q < w; ++q) pre += wcnt[q][d];
            int64_t pos = (int64_t)gofs[d] + pre + rank;
            ko[pos] = key;
            if (vals) vo[pos] = vals[j];
        }
        __syncthreads();
        int add = 0;
#pragma unroll
        for (int q = 0; q < kSortThreads / 32; ++q) add += wcnt[q][tid];
        base_cnt[tid] += add;
        __syncthreads();
    }
}

cudaError_t radix_sort_pairs(Arena &a, const uint32_t *keys_in, const int32_t *vals_in,
                             uint32_t *keys_out, int32_t *vals_out, int64_t n, int bits,
                             cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int passes = (bits + 7) / 8;
    if (passes < 1) passes = 1;
    int ntiles = (int)((n + kSortTile - 1) / kSortTile);
    int32_t *counts = nullptr, *offs = nullptr;
    uint32_t *kt = nullptr;
    int32_t *vt = nullptr;
    cudaError_t e = dalloc(a, &counts, (size_t)256 * ntiles);
    if (!e) e = dalloc(a, &offs, (size_t)256 * ntiles);
    if (!e && passes > 1) e = dalloc(a, &kt, n);
    if (!e && passes > 1 && vals_out) e = dalloc(a, &vt, n);
    if (e) return e;
    // ping-pong so that the last pass lands in keys_out/vals_out
    const uint32_t *ksrc = keys_in;
    const int32_t *vsrc = vals_in;
    for (int p = 0; p < passes; ++p) {
        bool to_out = ((passes - 1 - p) % 2) == 0;
        uint32_t *kd = to_out ? keys_out : kt;
        int32_t *vd = to_out ? vals_out : vt;
        k_radix_hist<<<ntiles, kSortThreads, 0, s>>>(ksrc, n, 8 * p, counts, ntiles);
        count_launch();
        e = exclusive_scan_i32(a, counts, offs, (int64_t)256 * ntiles, nullptr, s);
        if (e) return e;
        k_radix_scatter<<<ntiles, kSortThreads, 0, s>>>(ksrc, vals_out ? vsrc : nullptr, kd, vd,
                                                        n, 8 * p, offs, ntiles);
        count_launch();
        ksrc = kd;
        vsrc = vd;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- CSR helpers
__global__ void k_expand_rows(const int32_t *off, int32_t rows, int32_t *row_of) {
    int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = gw; r < rows; r += nw)
        for (int32_t j = off[r] + lane_id(); j < off[r + 1]; j += 32) row_of[j] = (int32_t)r;
}

void expand_rows(const int32_t *off, int32_t rows, int32_t *row_of, cudaStream_t s) {
    if (rows <= 0) return;
    int blocks = div_up((int64_t)rows * 32, 256);
    int cap = num_sms() * 16;
    if (blocks > cap) blocks = cap;
    k_expand_rows<<<blocks, 256, 0, s>>>(off, rows, row_of);
    count_launch();
}

__global__ void k_fill(int32_t *p, int32_t v, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void k_iota(int32_t *p, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (int32_t)i;
}

static int grid_for(int64_t n) {
    int b = div_up(n, 256);
    int cap = num_sms() * 8;
    return b < 1 ? 1 : (b > cap ? cap : b);
}

void fill_i32(int32_t *p, int32_t v, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    k_fill<<<grid_for(n), 256, 0, s>>>(p, v, n);
    count_launch();
}

void iota_i32(int32_t *p, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    k_iota<<<grid_for(n), 256, 0, s>>>(p, n);
    count_launch();
}

cudaError_t counts_to_offsets(Arena &a, const int32_t *counts, int32_t *off, int32_t rows,
                              cudaStream_t s) {
    // off has rows+1 entries; off[rows] receives the total.
    return exclusive_scan_i32(a, counts, off, rows, off + rows, s);
}

}  // namespace hgp
