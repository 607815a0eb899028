/*
 * Seeded synthetic hypergraph generators.
 *
 * These build the inputs that both the CPU oracle and the CUDA path are fed.
 * They hold none of the partitioning method's arithmetic: they only draw
 * random pins.  Shapes follow the spiking-neural-network workloads of the
 * paper's Table I (one hyperedge per neuron: the neuron itself as source,
 * followed by its synaptic targets).
 *
 * Random numbers: splitmix64 seeds one xoshiro256** state per hyperedge
 * (the state depends only on (seed, edge id)), so every edge can be
 * regenerated on its own and the output does not depend on call order.
 * Distinct targets are drawn with Floyd's sampling; the targets of an edge
 * are emitted in ascending id order after the source.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static uint64_t splitmix64(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s[4]; } xoshiro;

static uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t xo_next(xoshiro *r) {
    uint64_t *s = r->s;
    const uint64_t result = rotl64(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}

static void xo_seed(xoshiro *r, uint64_t seed, uint64_t stream) {
    uint64_t x = seed * 0xD1B54A32D192ED03ull ^ (stream + 0x8CB92BA72F3D8DD7ull);
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&x);
}

/* Uniform integer in [0, n) by Lemire's multiply-shift with rejection. */
static uint32_t xo_below(xoshiro *r, uint32_t n) {
    uint64_t m = (uint64_t)(uint32_t)(xo_next(r) >> 32) * n;
    uint32_t l = (uint32_t)m;
    if (l < n) {
        uint32_t t = (uint32_t)(-n) % n;
        while (l < t) {
            m = (uint64_t)(uint32_t)(xo_next(r) >> 32) * n;
            l = (uint32_t)m;
        }
    }
    return (uint32_t)(m >> 32);
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Floyd's algorithm: k distinct values of [0, n) into out[0..k), using
 * stamp[] (size n, initialised to a value != tag) as the membership set. */
static void floyd(xoshiro *r, uint32_t n, uint32_t k, int32_t *out,
                  int64_t *stamp, int64_t tag) {
    uint32_t c = 0;
    for (uint32_t j = n - k; j < n; ++j) {
        uint32_t t = xo_below(r, j + 1);
        if (stamp[t] == tag) t = j;
        stamp[t] = tag;
        out[c++] = (int32_t)t;
    }
}

/* ---------------- random SNN: one edge per node ---------------- */

static uint32_t rand_size(xoshiro *r, int32_t kmin, int32_t kmax) {
    if (kmax <= kmin) return (uint32_t)kmin;
    return (uint32_t)kmin + xo_below(r, (uint32_t)(kmax - kmin + 1));
}

/* Pass 1: offsets[num_nodes+1] of the random SNN hypergraph whose edge e has
 * source e and a size drawn uniformly from [kmin, kmax] (clamped to N). */
int synth_random_offsets(int32_t num_nodes, int32_t kmin, int32_t kmax,
                         uint64_t seed, int64_t *offsets) {
    if (num_nodes < 1 || kmin < 1 || kmax < kmin) return 1;
    offsets[0] = 0;
    for (int32_t e = 0; e < num_nodes; ++e) {
        xoshiro r;
        xo_seed(&r, seed, (uint64_t)e);
        uint32_t k = rand_size(&r, kmin, kmax);
        if (k > (uint32_t)num_nodes) k = (uint32_t)num_nodes;
        offsets[e + 1] = offsets[e] + k;
    }
    return 0;
}

/* Pass 2: fill pins.  Edge e = [e, sorted distinct targets from N \ {e}]. */
int synth_random_fill(int32_t num_nodes, int32_t kmin, int32_t kmax,
                      uint64_t seed, const int64_t *offsets, int32_t *pins) {
    int64_t *stamp = (int64_t *)malloc(sizeof(int64_t) * (size_t)num_nodes);
    if (!stamp) return 2;
    for (int32_t i = 0; i < num_nodes; ++i) stamp[i] = -1;
    for (int32_t e = 0; e < num_nodes; ++e) {
        xoshiro r;
        xo_seed(&r, seed, (uint64_t)e);
        uint32_t k = rand_size(&r, kmin, kmax);
        if (k > (uint32_t)num_nodes) k = (uint32_t)num_nodes;
        int32_t *p = pins + offsets[e];
        p[0] = e;
        if (k > 1) {
            floyd(&r, (uint32_t)num_nodes - 1, k - 1, p + 1, stamp, e);
            for (uint32_t j = 1; j < k; ++j)
                if (p[j] >= e) p[j] += 1; /* skip the source itself */
            qsort(p + 1, k - 1, sizeof(int32_t), cmp_i32);
        }
    }
    free(stamp);
    return 0;
}

/* ---------------- layered convolution-style SNN ----------------
 * layers x (side x side spatial x ch channels).  Node id =
 * layer*side*side*ch + (y*side + x)*ch + c.  A node of layer l < layers-1
 * draws C ~ U{cmin..cmax} distinct channels of layer l+1 and connects to
 * those channels at every position of the 3x3 window around (y, x) that lies
 * inside the grid.  Nodes of the last layer have the single-pin edge {src}. */

static uint32_t conv_edge_size(int32_t side, int32_t ch, int32_t cmin,
                               int32_t cmax, xoshiro *r, int32_t y, int32_t x,
                               int last) {
    if (last) return 1;
    uint32_t c = rand_size(r, cmin, cmax);
    if (c > (uint32_t)ch) c = (uint32_t)ch;
    int ny = 0, nx = 0;
    for (int d = -1; d <= 1; ++d) {
        if (y + d >= 0 && y + d < side) ny++;
        if (x + d >= 0 && x + d < side) nx++;
    }
    return 1 + (uint32_t)(ny * nx) * c;
}

int synth_conv_offsets(int32_t layers, int32_t side, int32_t ch, int32_t cmin,
                       int32_t cmax, uint64_t seed, int64_t *offsets) {
    if (layers < 1 || side < 1 || ch < 1 || cmin < 1 || cmax < cmin) return 1;
    int64_t per = (int64_t)side * side * ch;
    int64_t n = per * layers;
    offsets[0] = 0;
    for (int64_t id = 0; id < n; ++id) {
        int32_t l = (int32_t)(id / per);
        int64_t rem = id % per;
        int32_t pos = (int32_t)(rem / ch);
        xoshiro r;
        xo_seed(&r, seed, (uint64_t)id);
        offsets[id + 1] = offsets[id] + conv_edge_size(side, ch, cmin, cmax, &r,
                                                       pos / side, pos % side,
                                                       l == layers - 1);
    }
    return 0;
}

int synth_conv_fill(int32_t layers, int32_t side, int32_t ch, int32_t cmin,
                    int32_t cmax, uint64_t seed, const int64_t *offsets,
                    int32_t *pins) {
    int64_t per = (int64_t)side * side * ch;
    int64_t n = per * layers;
    int64_t *stamp = (int64_t *)malloc(sizeof(int64_t) * (size_t)ch);
    int32_t *chans = (int32_t *)malloc(sizeof(int32_t) * (size_t)ch);
    if (!stamp || !chans) { free(stamp); free(chans); return 2; }
    for (int32_t i = 0; i < ch; ++i) stamp[i] = -1;
    for (int64_t id = 0; id < n; ++id) {
        int32_t l = (int32_t)(id / per);
        int64_t rem = id % per;
        int32_t pos = (int32_t)(rem / ch);
        int32_t y = pos / side, x = pos % side;
        int32_t *p = pins + offsets[id];
        p[0] = (int32_t)id;
        if (l == layers - 1) continue;
        xoshiro r;
        xo_seed(&r, seed, (uint64_t)id);
        uint32_t c = rand_size(&r, cmin, cmax);
        if (c > (uint32_t)ch) c = (uint32_t)ch;
        floyd(&r, (uint32_t)ch, c, chans, stamp, id);
        qsort(chans, c, sizeof(int32_t), cmp_i32);
        int64_t base = (int64_t)(l + 1) * per;
        int64_t k = 1;
        /* window positions in ascending (y, x) order, channels ascending:
         * node ids come out sorted. */
        for (int dy = -1; dy <= 1; ++dy) {
            int yy = y + dy;
            if (yy < 0 || yy >= side) continue;
            for (int dx = -1; dx <= 1; ++dx) {
                int xx = x + dx;
                if (xx < 0 || xx >= side) continue;
                for (uint32_t j = 0; j < c; ++j)
                    p[k++] = (int32_t)(base + (int64_t)(yy * side + xx) * ch + chans[j]);
            }
        }
    }
    free(stamp);
    free(chans);
    return 0;
}

/* One uniform double in [0, 1) from (seed, index); used for instance sizes. */
double synth_uniform01(uint64_t seed, uint64_t index) {
    xoshiro r;
    xo_seed(&r, seed, index);
    return (double)(xo_next(&r) >> 11) * (1.0 / 9007199254740992.0);
}
