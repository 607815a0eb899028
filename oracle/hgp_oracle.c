/*
 * CPU oracle for incidence-constrained multilevel hypergraph partitioning
 * ("Incidence Constraints in Hypergraph Partitioning on GPU", arXiv 2604.14411).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded
 * restatement of the method, written to be checked against the paper by eye.
 * It shares no code with the CUDA library.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the product path
 * never calls it.
 *
 * The method is a heuristic, so the oracle follows the paper's steps in the
 * paper's order:
 *   Sec. II-A       problem model: in(n), I(n), Omega, Delta, Eq. (1)
 *   Sec. II-B       level loop and stop rule (ceil(|N| / Omega) nodes)
 *   Sec. III-A, Eq. (2)   neighbour histogram, repeated argmax extraction,
 *                         deferred size / inbound-union checks, pair, score
 *   Sec. III-A, III-B.3   matching over the pairing pseudo-forest
 *                         (upward placement of scores, downward locking)
 *   Sec. III-B.4    coarse hypergraph: gamma map and set unions
 *   Sec. IV-A, Eq. (3)    in-isolation moves, sort by gain, in-sequence
 *                         gain, validity along the sequence, best prefix
 *
 * Readings taken where the paper is silent or ambiguous are marked
 * "Reading:" at the place they apply.
 *
 * Integers throughout: node/edge ids int32, weights int32 on input, sums
 * int64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_OK = 0, ORC_INVALID = 1, ORC_INFEASIBLE = 2, ORC_OOM = 3, ORC_INTERNAL = 4 };

/* ------------------------------------------------------------------ */
/* One level of the hierarchy: G_l(N_l, E, omega).                     */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t V, E;
    int64_t *w;      /* [V]   node weight = summed weight of member nodes  */
    int64_t *poff;   /* [E+1] pins(e): node set of hyperedge e, ascending   */
    int32_t *pins;
    int64_t *ioff;   /* [V+1] I(n) = in(n) u out(n), ascending edge ids     */
    int32_t *inc;
    int64_t *noff;   /* [V+1] in(n): edges having n as a destination        */
    int32_t *in;
} olevel;

static void olevel_free(olevel *g) {
    free(g->w); free(g->poff); free(g->pins);
    free(g->ioff); free(g->inc); free(g->noff); free(g->in);
    memset(g, 0, sizeof(*g));
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Sort and deduplicate v[0..n); returns the new length. */
static int64_t sort_unique(int32_t *v, int64_t n) {
    if (n <= 1) return n;
    qsort(v, (size_t)n, sizeof(int32_t), cmp_i32);
    int64_t k = 1;
    for (int64_t i = 1; i < n; ++i)
        if (v[i] != v[k - 1]) v[k++] = v[i];
    return k;
}

/* Transpose of a set family given as CSR over `rows` rows with entries in
 * [0, cols): out row c lists, ascending, the rows r whose set contains c. */
static int transpose(int32_t rows, int32_t cols, const int64_t *off,
                     const int32_t *data, int64_t **out_off, int32_t **out_data) {
    int64_t *o = (int64_t *)calloc((size_t)cols + 1, sizeof(int64_t));
    int32_t *d = (int32_t *)malloc(sizeof(int32_t) * (size_t)(off[rows] > 0 ? off[rows] : 1));
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * ((size_t)cols + 1));
    if (!o || !d || !cur) { free(o); free(d); free(cur); return ORC_OOM; }
    for (int64_t j = 0; j < off[rows]; ++j) o[data[j] + 1]++;
    for (int32_t c = 0; c < cols; ++c) o[c + 1] += o[c];
    memcpy(cur, o, sizeof(int64_t) * (size_t)cols);
    for (int32_t r = 0; r < rows; ++r)          /* rows in ascending order, */
        for (int64_t j = off[r]; j < off[r + 1]; ++j)   /* so each output */
            d[cur[data[j]]++] = r;                         /* row is sorted */
    free(cur);
    *out_off = o;
    *out_data = d;
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Input validation and level 0 (Sec. II-A, II-C).                     */
/* ------------------------------------------------------------------ */
/*
 * Reading: the first pin of every hyperedge is its source src(e); the other
 * pins are its destinations dst(e) (one source per neuron in the SNN
 * workloads).  in(n) = {e : n in dst(e)}, I(n) = {e : n in e}.
 * Reading: hyperedges must be non-empty and without repeated pins; edge
 * weights must be >= 1 (the objective is a sum of positive cut weights) and
 * their total must fit int32; node weights must be >= 1 with an int32 total.
 */
static int build_level0(int32_t N, int32_t E, const int32_t *offsets,
                        const int32_t *pins, const int32_t *nw, const int32_t *ew,
                        int32_t mode, olevel *g, int32_t **src_out) {
    if (N < 1 || E < 0 || !offsets || (E > 0 && !pins)) return ORC_INVALID;
    if (offsets[0] != 0) return ORC_INVALID;
    for (int32_t e = 0; e < E; ++e)
        if (offsets[e + 1] <= offsets[e]) return ORC_INVALID;   /* empty edge */
    int64_t P = offsets[E];
    for (int64_t j = 0; j < P; ++j)
        if (pins[j] < 0 || pins[j] >= N) return ORC_INVALID;
    int64_t tw = 0, te = 0;
    if (nw) for (int32_t n = 0; n < N; ++n) { if (nw[n] < 1) return ORC_INVALID; tw += nw[n]; }
    if (ew) for (int32_t e = 0; e < E; ++e) { if (ew[e] < 1) return ORC_INVALID; te += ew[e]; }
    if (!nw) tw = N;
    if (!ew) te = E;
    if (tw > INT32_MAX || te > INT32_MAX) return ORC_INVALID;

    memset(g, 0, sizeof(*g));
    g->V = N; g->E = E;
    g->w = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    g->poff = (int64_t *)malloc(sizeof(int64_t) * ((size_t)E + 1));
    g->pins = (int32_t *)malloc(sizeof(int32_t) * (size_t)(P > 0 ? P : 1));
    int32_t *src = (int32_t *)malloc(sizeof(int32_t) * (size_t)(E > 0 ? E : 1));
    if (!g->w || !g->poff || !g->pins || !src) { free(src); olevel_free(g); return ORC_OOM; }
    for (int32_t n = 0; n < N; ++n) g->w[n] = nw ? nw[n] : 1;
    for (int32_t e = 0; e <= E; ++e) g->poff[e] = offsets[e];
    memcpy(g->pins, pins, sizeof(int32_t) * (size_t)P);
    for (int32_t e = 0; e < E; ++e) {
        src[e] = pins[offsets[e]];
        int64_t len = g->poff[e + 1] - g->poff[e];
        if (sort_unique(g->pins + g->poff[e], len) != len) {   /* repeated pin */
            free(src); olevel_free(g); return ORC_INVALID;
        }
    }
    int rc = transpose(E, N, g->poff, g->pins, &g->ioff, &g->inc);
    if (rc) { free(src); olevel_free(g); return rc; }
    /* in(n): the same transpose restricted to destination pins (mode 0).
     * The paper calls the other directions a trivial generalisation: mode 1
     * counts every incident hyperedge, in(n) = I(n); mode 2 the outbound
     * ones, in(n) = {e : src(e) = n}. */
    int64_t *dcount = (int64_t *)calloc((size_t)E + 1, sizeof(int64_t));
    int32_t *dst = (int32_t *)malloc(sizeof(int32_t) * (size_t)(P > 0 ? P : 1));
    if (!dcount || !dst) { free(dcount); free(dst); free(src); olevel_free(g); return ORC_OOM; }
    int64_t k = 0;
    for (int32_t e = 0; e < E; ++e) {
        dcount[e] = k;
        for (int64_t j = g->poff[e]; j < g->poff[e + 1]; ++j)
            if (mode == 1 || (mode == 0) == (g->pins[j] != src[e])) dst[k++] = g->pins[j];
    }
    dcount[E] = k;
    rc = transpose(E, N, dcount, dst, &g->noff, &g->in);
    free(dcount); free(dst);
    if (rc) { free(src); olevel_free(g); return rc; }
    *src_out = src;
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Candidate selection: Eq. (2) and the deferred checks (Sec. III-A).  */
/* ------------------------------------------------------------------ */
/*
 * hist(n, m) = sum of omega(e) over e in I(n) with m in e.
 * Reading: m = n is excluded (a node is not its own candidate).
 * pair(n) is found by repeatedly extracting the argmax of hist(n, .) --
 * larger hist first, and among equal hist the larger id (the max_id of the
 * pair definition) -- until an extracted m passes both checks:
 *   w(n) + w(m) <= Omega            (cluster size)
 *   |in(n) u in(m)| <= Delta         (distinct inbound hyperedges)
 * score(n) = hist(n, pair(n)).  pair(n) = -1 when no neighbour is valid.
 * Every neighbour has hist >= 1 because omega >= 1, so hist > 0 doubles as
 * the "is a neighbour" mark.
 * The union is counted as in Sec. III-B.2: |in(n)| plus the edges of in(m)
 * not present in in(n) (in(n) is marked in `stamp`).  When
 * |in(n)| + |in(m)| <= Delta the union cannot exceed Delta and the count is
 * skipped.
 * Extraction order: the first argmax is taken by a linear scan (usually it
 * is valid); if it fails, the remaining neighbours are sorted once into the
 * same order and taken one by one.
 */
typedef struct { int64_t h; int32_t m; } ocand;

static int cmp_cand(const void *a, const void *b) {
    const ocand *x = (const ocand *)a, *y = (const ocand *)b;
    if (x->h != y->h) return x->h > y->h ? -1 : 1;
    return (x->m < y->m) - (x->m > y->m);
}

static int pair_valid(const olevel *g, int32_t n, int32_t m, int64_t omega, int64_t delta,
                      const int32_t *stamp) {
    if (g->w[n] + g->w[m] > omega) return 0;
    int64_t in_n = g->noff[n + 1] - g->noff[n];
    int64_t in_m = g->noff[m + 1] - g->noff[m];
    if (in_n + in_m <= delta) return 1;
    int64_t extra = 0;
    for (int64_t j = g->noff[m]; j < g->noff[m + 1]; ++j) extra += stamp[g->in[j]] != n;
    return in_n + extra <= delta;
}

/* Candidate of one node n (the steps above), with caller scratch. */
static void score_node(const olevel *g, const int32_t *ew, int64_t omega, int64_t delta,
                       int32_t n, int32_t *pair, int32_t *score, int64_t *hist_scratch,
                       int32_t *touched, int32_t *stamp, ocand *cand) {
    int32_t nt = 0;
    for (int64_t i = g->ioff[n]; i < g->ioff[n + 1]; ++i) {
        int32_t e = g->inc[i];
        int64_t we = ew ? ew[e] : 1;
        for (int64_t j = g->poff[e]; j < g->poff[e + 1]; ++j) {
            int32_t m = g->pins[j];
            if (m == n) continue;
            if (hist_scratch[m] == 0) touched[nt++] = m;
            hist_scratch[m] += we;
        }
    }
    for (int64_t j = g->noff[n]; j < g->noff[n + 1]; ++j) stamp[g->in[j]] = n;
    *pair = -1;
    *score = 0;
    int32_t best = -1;
    for (int32_t t = 0; t < nt; ++t) {
        int32_t m = touched[t];
        if (best < 0 || hist_scratch[m] > hist_scratch[best] ||
            (hist_scratch[m] == hist_scratch[best] && m > best))
            best = m;
    }
    if (best >= 0 && pair_valid(g, n, best, omega, delta, stamp)) {
        *pair = best;
        *score = (int32_t)hist_scratch[best];
    } else if (best >= 0) {
        int32_t nc = 0;
        for (int32_t t = 0; t < nt; ++t)
            if (touched[t] != best) { cand[nc].h = hist_scratch[touched[t]]; cand[nc].m = touched[t]; nc++; }
        qsort(cand, (size_t)nc, sizeof(ocand), cmp_cand);
        for (int32_t c = 0; c < nc; ++c) {
            if (pair_valid(g, n, cand[c].m, omega, delta, stamp)) {
                *pair = cand[c].m;
                *score = (int32_t)cand[c].h;
                break;
            }
        }
    }
    for (int32_t t = 0; t < nt; ++t) hist_scratch[touched[t]] = 0;
}

/* nodes = NULL: every node of the level; otherwise only nodes[0..count). */
static int score_level(const olevel *g, const int32_t *ew, int64_t omega,
                       int64_t delta, int32_t *pair, int32_t *score,
                       int64_t *hist_scratch, int32_t *touched,
                       const int32_t *nodes, int32_t count) {
    int32_t *stamp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->E > 0 ? g->E : 1));
    ocand *cand = (ocand *)malloc(sizeof(ocand) * (size_t)g->V);
    if (!stamp || !cand) { free(stamp); free(cand); return ORC_OOM; }
    for (int32_t e = 0; e < g->E; ++e) stamp[e] = -1;
    int32_t total = nodes ? count : g->V;
    for (int32_t t = 0; t < total; ++t) {
        int32_t n = nodes ? nodes[t] : t;
        score_node(g, ew, omega, delta, n, pair + t, score + t, hist_scratch, touched, stamp, cand);
    }
    free(stamp); free(cand);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Learned merge proposal (an extension; the paper has none).          */
/* ------------------------------------------------------------------ */
/*
 * A two-layer network reorders the candidates of Eq. (2):
 *   x      = 8 features of the pair (n, m), symmetric in n and m (below)
 *   h_j    = max(0, b1_j + sum_i W1_ji x_i)            j = 0..63
 *   s      = b2 + sum_j W2_j h_j
 *   key    = floor(s * 2^key_bits), clamped to [-2^30, 2^30]
 * Weights are bfloat16 bit patterns, widened exactly to float.  Every sum is
 * evaluated in float32 as a chain of fused multiply-adds in index order
 * (h_j over i = 0..7, then s over j = 0..63, each h_j folded in as soon as it
 * is known); this order is part of the definition, so any implementation
 * that follows it gets bit-identical keys.
 * pair(n) = the valid m (same two checks as Sec. III-B.2) with the largest
 * (key, hist, id); score(n) = hist(n, pair(n)).  With every weight zero all
 * keys are equal and the order is the plain (hist, id) order.
 * Because (key, hist) is symmetric in n and m, every cycle of the pairing
 * graph is a two-cycle by the same argument as for hist alone, and matching
 * runs on the composite (key, hist) score.
 *
 * Features, each through lg1p (log2(1 + x) with a linear mantissa):
 *   x0 hist(n,m)          x1 |in(n) u in(m)|
 *   x2 min(|I(n)|,|I(m)|) x3 max(|I(n)|,|I(m)|)
 *   x4 min(|in(n)|,|in(m)|) x5 max(|in(n)|,|in(m)|)
 *   x6 min(w(n),w(m))     x7 max(w(n),w(m))
 */
#define OMLP_IN 8
#define OMLP_HID 64
#define OMLP_PARAMS (OMLP_HID * OMLP_IN + OMLP_HID + OMLP_HID + 1)

typedef struct {
    float w1[OMLP_HID][OMLP_IN], b1[OMLP_HID], w2[OMLP_HID], b2;
    int32_t key_bits;
} omodel;

static float bf16_to_f32(uint16_t b) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, sizeof(f));
    return f;
}

/* 2^k as a float, exact for -126 <= k <= 127. */
static float pow2f_exact(int k) {
    uint32_t u = (uint32_t)(127 + k) << 23;
    float f;
    memcpy(&f, &u, sizeof(f));
    return f;
}

/* log2(1 + x) for integer x >= 0, with the mantissa taken linearly: if
 * 2^k <= 1 + x < 2^(k+1) the value is k + (1 + x - 2^k) / 2^k.  Exact at
 * every power of two and at most 0.0861 below log2(1 + x) elsewhere.  The
 * integer remainder is rounded to float once (round to nearest even); the
 * division by 2^k is exact. */
static float lg1p(int64_t x) {
    uint64_t y = (uint64_t)x + 1u;
    int k = 0;
    while (k < 63 && (y >> (k + 1)) != 0) ++k;
    float frac = (float)(y - ((uint64_t)1 << k)) * pow2f_exact(-k);
    return (float)k + frac;
}

static float mlp_score(const omodel *M, const float *x) {
    float s = M->b2;
    for (int j = 0; j < OMLP_HID; ++j) {
        float h = M->b1[j];
        for (int i = 0; i < OMLP_IN; ++i) h = fmaf(M->w1[j][i], x[i], h);
        h = h > 0.0f ? h : 0.0f;
        s = fmaf(M->w2[j], h, s);
    }
    return s;
}

static int32_t score_key(float s, int32_t key_bits) {
    float q = floorf(s * pow2f_exact(key_bits));
    if (!(q > -1073741824.0f)) return -1073741824;     /* also NaN */
    if (q > 1073741824.0f) return 1073741824;
    return (int32_t)q;
}

static int model_from_bits(const uint16_t *w1, const uint16_t *b1, const uint16_t *w2, uint16_t b2,
                           int32_t key_bits, omodel *M) {
    if (key_bits < 0 || key_bits > 20) return ORC_INVALID;
    for (int j = 0; j < OMLP_HID; ++j) {
        for (int i = 0; i < OMLP_IN; ++i) M->w1[j][i] = bf16_to_f32(w1[j * OMLP_IN + i]);
        M->b1[j] = bf16_to_f32(b1[j]);
        M->w2[j] = bf16_to_f32(w2[j]);
    }
    M->b2 = bf16_to_f32(b2);
    M->key_bits = key_bits;
    return ORC_OK;
}

/* |in(n) u in(m)| with in(n) marked in `stamp`. */
static int64_t union_size(const olevel *g, int32_t n, int32_t m, const int32_t *stamp) {
    int64_t u = g->noff[n + 1] - g->noff[n];
    for (int64_t j = g->noff[m]; j < g->noff[m + 1]; ++j) u += stamp[g->in[j]] != n;
    return u;
}

static void pair_features(const olevel *g, int32_t n, int32_t m, int64_t hist, int64_t uni, float *x) {
    int64_t dn = g->ioff[n + 1] - g->ioff[n], dm = g->ioff[m + 1] - g->ioff[m];
    int64_t in_n = g->noff[n + 1] - g->noff[n], in_m = g->noff[m + 1] - g->noff[m];
    int64_t wn = g->w[n], wm = g->w[m];
    x[0] = lg1p(hist);
    x[1] = lg1p(uni);
    x[2] = lg1p(dn < dm ? dn : dm);
    x[3] = lg1p(dn < dm ? dm : dn);
    x[4] = lg1p(in_n < in_m ? in_n : in_m);
    x[5] = lg1p(in_n < in_m ? in_m : in_n);
    x[6] = lg1p(wn < wm ? wn : wm);
    x[7] = lg1p(wn < wm ? wm : wn);
}

static void score_node_learned(const olevel *g, const int32_t *ew, int64_t omega, int64_t delta,
                               const omodel *M, int32_t n, int32_t *pair, int32_t *score,
                               int32_t *key, int64_t *hist_scratch, int32_t *touched,
                               int32_t *stamp) {
    int32_t nt = 0;
    for (int64_t i = g->ioff[n]; i < g->ioff[n + 1]; ++i) {
        int32_t e = g->inc[i];
        int64_t we = ew ? ew[e] : 1;
        for (int64_t j = g->poff[e]; j < g->poff[e + 1]; ++j) {
            int32_t m = g->pins[j];
            if (m == n) continue;
            if (hist_scratch[m] == 0) touched[nt++] = m;
            hist_scratch[m] += we;
        }
    }
    for (int64_t j = g->noff[n]; j < g->noff[n + 1]; ++j) stamp[g->in[j]] = n;
    int32_t best = -1, bk = 0;
    int64_t bh = 0;
    for (int32_t t = 0; t < nt; ++t) {
        int32_t m = touched[t];
        if (g->w[n] + g->w[m] > omega) continue;
        int64_t uni = union_size(g, n, m, stamp);
        if (uni > delta) continue;
        float x[OMLP_IN];
        pair_features(g, n, m, hist_scratch[m], uni, x);
        int32_t k = score_key(mlp_score(M, x), M->key_bits);
        int64_t h = hist_scratch[m];
        if (best < 0 || k > bk || (k == bk && (h > bh || (h == bh && m > best)))) {
            best = m; bk = k; bh = h;
        }
    }
    *pair = best;
    *score = best >= 0 ? (int32_t)bh : 0;
    *key = best >= 0 ? bk : 0;
    for (int32_t t = 0; t < nt; ++t) hist_scratch[touched[t]] = 0;
}

static int score_level_learned(const olevel *g, const int32_t *ew, int64_t omega, int64_t delta,
                               const omodel *M, int32_t *pair, int32_t *score, int32_t *key,
                               int64_t *hist_scratch, int32_t *touched) {
    int32_t *stamp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->E > 0 ? g->E : 1));
    if (!stamp) return ORC_OOM;
    for (int32_t e = 0; e < g->E; ++e) stamp[e] = -1;
    for (int32_t n = 0; n < g->V; ++n)
        score_node_learned(g, ew, omega, delta, M, n, pair + n, score + n, key + n, hist_scratch,
                           touched, stamp);
    free(stamp);
    return ORC_OK;
}

/* Composite matching score of the learned order: (key, hist) as one int64. */
static int64_t learned_composite(int32_t key, int32_t hist) {
    return ((int64_t)key + 1073741824) * ((int64_t)1 << 32) + (int64_t)hist;
}

/* ------------------------------------------------------------------ */
/* Matching over the pairing pseudo-forest (Sec. III-A, III-B.3).      */
/* ------------------------------------------------------------------ */
static int beats(const int64_t *score, int32_t a, int32_t b) {
    /* (score(a), a) > (score(b), b): ties on score broken by the larger id.
     * Scores are int64 so that the learned order's composite (key, hist)
     * compares the same way. */
    return score[a] > score[b] || (score[a] == score[b] && a > b);
}

/*
 * Formulation 1: the paper's two walks.
 * Upward: every node n with a candidate places (score(n), n) on
 * match(pair(n)); a placement wins when match(pair(n)) is still pair(n) or
 * when it beats the one already there.  Two-cycles are the roots and are
 * matched.  Downward, from the roots towards the leaves (any order in which
 * a node's path to its root has been settled first -- here: increasing
 * depth), n locks match(n) = pair(n) iff it still sees match(pair(n)) = n.
 * Returns ORC_INTERNAL if the pairing graph has a cycle longer than two,
 * which the paper shows cannot happen.
 */
static int match_walks(int32_t V, const int32_t *pair, const int64_t *score, int32_t *match) {
    int32_t *depth = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
    int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
    int64_t *bucket = (int64_t *)calloc((size_t)V + 2, sizeof(int64_t));
    if (!depth || !order || !stack || !bucket) { free(depth); free(order); free(stack); free(bucket); return ORC_OOM; }
    for (int32_t n = 0; n < V; ++n) match[n] = n;
    for (int32_t n = 0; n < V; ++n) {
        if (pair[n] < 0) continue;
        int32_t m = pair[n], c = match[m];
        if (c == m || beats(score, n, c)) match[m] = n;
    }
    /* two-cycles form a match by default (with scores from Eq. (2) the
     * partner always wins the placement above anyway) */
    for (int32_t n = 0; n < V; ++n)
        if (pair[n] >= 0 && pair[pair[n]] == n) match[n] = pair[n];
    /* depth along pair to the root two-cycle; -1 = no candidate, -2 = unknown */
    for (int32_t n = 0; n < V; ++n) {
        if (pair[n] < 0) depth[n] = -1;
        else if (pair[pair[n]] == n) depth[n] = 0;
        else depth[n] = -2;
    }
    for (int32_t n = 0; n < V; ++n) {
        if (depth[n] != -2) continue;
        int32_t sp = 0, x = n;
        while (depth[x] == -2) {
            if (sp >= V) { free(depth); free(order); free(stack); free(bucket); return ORC_INTERNAL; }
            stack[sp++] = x;
            x = pair[x];
        }
        if (depth[x] == -1) { free(depth); free(order); free(stack); free(bucket); return ORC_INTERNAL; }
        while (sp > 0) { int32_t y = stack[--sp]; depth[y] = depth[pair[y]] + 1; }
    }
    /* counting sort of nodes with a candidate by depth */
    for (int32_t n = 0; n < V; ++n) if (depth[n] >= 0) bucket[depth[n] + 1]++;
    for (int32_t d = 0; d <= V; ++d) bucket[d + 1] += bucket[d];
    for (int32_t n = 0; n < V; ++n) if (depth[n] >= 0) order[bucket[depth[n]]++] = n;
    int64_t cnt = bucket[V];
    for (int64_t i = 0; i < cnt; ++i) {
        int32_t n = order[i];
        if (depth[n] == 0) continue;                /* roots matched already */
        if (match[pair[n]] == n) match[n] = pair[n];
    }
    free(depth); free(order); free(stack); free(bucket);
    return ORC_OK;
}

/*
 * Exact maximum-weight matching of the pairing pseudo-forest, the exact
 * alternative to the two walks that the paper leaves as future work.
 * Edges are {n, pair(n)} with weight score(n).  Every cycle is a root
 * two-cycle {a, b} (Sec. III-A) whose two directed edges are one edge of
 * weight score(a) = score(b); making b = max(a, b) a child of a = min(a, b)
 * turns each component into a tree rooted at a.  Nodes with no candidate are
 * roots without children.  With w(c) the weight of the edge from child c to
 * its parent, children before parents:
 *   up(v)   = sum over children c of best(c)   (v not matched below itself)
 *   g(v)    = max over children c of w(c) - max(0, g(c)) (no term for a leaf):
 *             what matching v to a child adds to up(v); c*(v) = the child
 *             with the largest (that value, id)
 *   best(v) = up(v) + max(0, g(v))
 * and parents before children: a root is free; a free node v with g(v) > 0
 * is matched to c*(v), which is then taken; all other nodes are left to
 * their own subtree.  (A zero gain leaves v free.)  The matched weight is
 * the sum of best over the roots, the maximum over all matchings.
 */
static int match_dp(int32_t V, const int32_t *pair, const int64_t *score, int32_t *match) {
    int32_t *par = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
    int32_t *depth = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
    int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
    int32_t *cstar = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
    int64_t *up = (int64_t *)calloc((size_t)V, sizeof(int64_t));
    int64_t *g = (int64_t *)malloc(sizeof(int64_t) * (size_t)V);
    int64_t *bucket = (int64_t *)calloc((size_t)V + 2, sizeof(int64_t));
    signed char *taken = (signed char *)calloc((size_t)V, 1);
    int rc = ORC_OK;
    if (!par || !depth || !order || !stack || !cstar || !up || !g || !bucket || !taken) {
        rc = ORC_OOM;
        goto done;
    }
    for (int32_t n = 0; n < V; ++n) {
        int32_t m = pair[n];
        if (m < 0) par[n] = -1;
        else if (pair[m] == n) par[n] = n < m ? -1 : m;     /* root two-cycle */
        else par[n] = m;
        cstar[n] = -1;
        g[n] = 0;
        depth[n] = par[n] < 0 ? 0 : -1;
        match[n] = n;
    }
    for (int32_t n = 0; n < V; ++n) {               /* depth below the root */
        int32_t sp = 0, x = n;
        while (depth[x] < 0) {
            if (sp >= V) { rc = ORC_INTERNAL; goto done; }
            stack[sp++] = x;
            x = par[x];
        }
        while (sp > 0) { int32_t y = stack[--sp]; depth[y] = depth[par[y]] + 1; }
    }
    for (int32_t n = 0; n < V; ++n) bucket[depth[n] + 1]++;
    for (int32_t d = 0; d <= V; ++d) bucket[d + 1] += bucket[d];
    for (int32_t n = 0; n < V; ++n) order[bucket[depth[n]]++] = n;
    /* children before parents */
    for (int32_t i = V - 1; i >= 0; --i) {
        int32_t c = order[i], p = par[c];
        if (p < 0) continue;
        int64_t gc = cstar[c] >= 0 && g[c] > 0 ? g[c] : 0;
        up[p] += up[c] + gc;                         /* best(c) */
        int64_t gain = score[c] - gc;
        if (cstar[p] < 0 || gain > g[p] || (gain == g[p] && c > cstar[p])) {
            g[p] = gain;
            cstar[p] = c;
        }
    }
    /* parents before children */
    for (int32_t i = 0; i < V; ++i) {
        int32_t v = order[i];
        if (taken[v] || cstar[v] < 0 || g[v] <= 0) continue;
        match[v] = cstar[v];
        match[cstar[v]] = v;
        taken[cstar[v]] = 1;
    }
done:
    free(par); free(depth); free(order); free(stack); free(cstar); free(up); free(g);
    free(bucket); free(taken);
    return rc;
}

/*
 * Formulation 2 (independent restatement used as a cross-check):
 * best(m) = the child of m with the largest (score, id);
 * lock(n) = true for the two nodes of a root two-cycle, otherwise
 * lock(n) = [best(pair(n)) = n] and not lock(pair(n)).
 * match(n) = pair(n) if lock(n); else best(n) if n has a child; else n.
 */
static int match_locks(int32_t V, const int32_t *pair, const int64_t *score, int32_t *match) {
    int32_t *best = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
    signed char *lock = (signed char *)malloc((size_t)V);
    int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
    if (!best || !lock || !stack) { free(best); free(lock); free(stack); return ORC_OOM; }
    for (int32_t n = 0; n < V; ++n) { best[n] = -1; lock[n] = -1; }
    for (int32_t n = 0; n < V; ++n) {
        if (pair[n] < 0) continue;
        int32_t m = pair[n];
        if (best[m] < 0 || beats(score, n, best[m])) best[m] = n;
    }
    for (int32_t n = 0; n < V; ++n) {
        if (pair[n] < 0) lock[n] = 0;
        else if (pair[pair[n]] == n) lock[n] = 1;
        else if (best[pair[n]] != n) lock[n] = 0;
    }
    for (int32_t n = 0; n < V; ++n) {
        int32_t sp = 0, x = n;
        while (lock[x] < 0) {
            if (sp >= V) { free(best); free(lock); free(stack); return ORC_INTERNAL; }
            stack[sp++] = x;
            x = pair[x];
        }
        while (sp > 0) { int32_t y = stack[--sp]; lock[y] = (signed char)!lock[pair[y]]; }
    }
    for (int32_t n = 0; n < V; ++n)
        match[n] = lock[n] ? pair[n] : (best[n] >= 0 ? best[n] : n);
    free(best); free(lock); free(stack);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Coarse hypergraph (Sec. III-B.4).                                   */
/* ------------------------------------------------------------------ */
/*
 * Reading: the coarse node of a pair {n, match(n)} is numbered by the rank
 * of its smaller member among all such representatives (ascending).
 * Returns |N'|.
 */
static int32_t gamma_from_match(int32_t V, const int32_t *match, int32_t *gamma) {
    int32_t cnt = 0;
    for (int32_t n = 0; n < V; ++n)
        if (match[n] >= n) gamma[n] = cnt++;      /* n is its pair's smaller id */
    for (int32_t n = 0; n < V; ++n)
        if (match[n] < n) gamma[n] = gamma[match[n]];
    return cnt;
}

/*
 * G' = (N', E, omega): w'(n') = sum of member weights; pins'(e) = gamma(pins(e))
 * as a set; in'(n') = union of the members' in(); I' follows from pins'.
 * Reading: all |E| hyperedges are kept, also those that collapse to a single
 * pin (they still count towards Delta) and duplicates of each other.
 */
static int contract(const olevel *g, const int32_t *gamma, int32_t V2, olevel *h) {
    memset(h, 0, sizeof(*h));
    h->V = V2; h->E = g->E;
    int64_t P = g->poff[g->E];
    h->w = (int64_t *)calloc((size_t)V2, sizeof(int64_t));
    h->poff = (int64_t *)malloc(sizeof(int64_t) * ((size_t)g->E + 1));
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(P > 0 ? P : 1));
    if (!h->w || !h->poff || !tmp) { free(tmp); olevel_free(h); return ORC_OOM; }
    for (int32_t n = 0; n < g->V; ++n) h->w[gamma[n]] += g->w[n];
    int64_t k = 0;
    h->poff[0] = 0;
    for (int32_t e = 0; e < g->E; ++e) {
        int64_t s = k;
        for (int64_t j = g->poff[e]; j < g->poff[e + 1]; ++j) tmp[k++] = gamma[g->pins[j]];
        k = s + sort_unique(tmp + s, k - s);
        h->poff[e + 1] = k;
    }
    h->pins = (int32_t *)malloc(sizeof(int32_t) * (size_t)(k > 0 ? k : 1));
    if (!h->pins) { free(tmp); olevel_free(h); return ORC_OOM; }
    memcpy(h->pins, tmp, sizeof(int32_t) * (size_t)k);
    free(tmp);
    int rc = transpose(h->E, V2, h->poff, h->pins, &h->ioff, &h->inc);
    if (rc) { olevel_free(h); return rc; }
    /* in'(n'): concatenate the members' in() lists, then sort-unique. */
    int64_t *cap = (int64_t *)calloc((size_t)V2 + 1, sizeof(int64_t));
    int64_t Q = g->noff[g->V];
    int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(Q > 0 ? Q : 1));
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * ((size_t)V2 + 1));
    h->noff = (int64_t *)malloc(sizeof(int64_t) * ((size_t)V2 + 1));
    if (!cap || !buf || !cur || !h->noff) { free(cap); free(buf); free(cur); olevel_free(h); return ORC_OOM; }
    for (int32_t n = 0; n < g->V; ++n) cap[gamma[n] + 1] += g->noff[n + 1] - g->noff[n];
    for (int32_t c = 0; c < V2; ++c) cap[c + 1] += cap[c];
    memcpy(cur, cap, sizeof(int64_t) * (size_t)V2);
    for (int32_t n = 0; n < g->V; ++n)
        for (int64_t j = g->noff[n]; j < g->noff[n + 1]; ++j) buf[cur[gamma[n]]++] = g->in[j];
    int64_t q = 0;
    h->noff[0] = 0;
    for (int32_t c = 0; c < V2; ++c) {
        int64_t len = sort_unique(buf + cap[c], cap[c + 1] - cap[c]);
        memmove(buf + q, buf + cap[c], sizeof(int32_t) * (size_t)len);
        q += len;
        h->noff[c + 1] = q;
    }
    h->in = buf;
    free(cap); free(cur);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Refinement (Sec. IV).                                               */
/* ------------------------------------------------------------------ */
typedef struct { int32_t n, ps, pd, gain; } omove;

/* pins(p, e) and pins_in(p, e) of one hyperedge, kept as a small list. */
typedef struct { int32_t p, cnt, cnt_in; } pcount;

typedef struct {
    int64_t *off;   /* [E+1] capacity |pins(e)| per edge */
    int32_t *len;   /* [E]   live entries                 */
    pcount *a;
} edge_parts;

static pcount *ep_find(const edge_parts *ep, int32_t e, int32_t p) {
    pcount *s = ep->a + ep->off[e];
    for (int32_t i = 0; i < ep->len[e]; ++i) if (s[i].p == p) return s + i;
    return NULL;
}

/* adds (d, d_in) to the counts of part p on edge e; drops empty entries */
static void ep_add(edge_parts *ep, int32_t e, int32_t p, int32_t d, int32_t d_in) {
    pcount *c = ep_find(ep, e, p);
    if (!c) {
        c = ep->a + ep->off[e] + ep->len[e]++;
        c->p = p; c->cnt = 0; c->cnt_in = 0;
    }
    c->cnt += d;
    c->cnt_in += d_in;
    if (c->cnt == 0) {
        pcount *last = ep->a + ep->off[e] + (--ep->len[e]);
        *c = *last;
    }
}

typedef struct {
    int32_t M;            /* proposed moves */
    int32_t kstar;        /* chosen prefix length (0 = none applied) */
    int64_t gain;         /* connectivity drop of the applied prefix */
    omove *moves;         /* [M] sorted sequence */
    int32_t *gain_seq;    /* [M] in-sequence gains */
    int32_t *viol;        /* [M] violations after moves 0..k applied */
} rtrace;

static int cmp_move(const void *a, const void *b) {
    const omove *x = (const omove *)a, *y = (const omove *)b;
    if (x->gain != y->gain) return x->gain > y->gain ? -1 : 1;   /* gain desc */
    return (x->n > y->n) - (x->n < y->n);                         /* id asc */
}

/*
 * One refinement pass on level g with partition rho (part ids in [0, K)).
 *  - size(p) = sum of w; pins(p, e) = pins of e in p; pins_in(p, e) = pins of
 *    e in p having e inbound; inb(p) = #{e : pins_in(p, e) > 0} (Sec. IV-B.1).
 *  - Eq. (3): saving(n) = sum omega(e), e in I(n), pins(rho(n), e) = 1;
 *    loss(n, p) = sum omega(e), e in I(n), pins(p, e) = 0; gain = saving - loss.
 *    Reading: a part p is excluded when size(p) + w(n) > Omega (at unit
 *    weights: when it already holds Omega nodes).  The best p != rho(n) is
 *    proposed iff its gain is > 0; ties go to the smallest p.  A part sharing
 *    no hyperedge with n has loss = sum omega over I(n) >= saving, so gain <= 0:
 *    only parts adjacent to n can be proposed, and only those are scanned.
 *  - Moves sorted by gain, descending; Reading: equal gains by node id.
 *  - In-sequence gain of move k = the exact change of Eq. (1) when it is
 *    applied after moves 0..k-1 (the four printed cases are the non-zero
 *    terms of that change).  Validity after each move: every part has
 *    size <= Omega and inb <= Delta.
 *  - Reading: among prefixes 1..M whose state is valid, take the one of
 *    maximum summed gain, the longest on ties; apply it iff that sum is > 0.
 */
static int refine_pass(const olevel *g, const int32_t *ew, int32_t *rho, int32_t K,
                       int64_t omega, int64_t delta, rtrace *tr) {
    int32_t V = g->V, E = g->E;
    int rc = ORC_OOM;
    int64_t *size = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    int64_t *inb = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    int64_t *pres = (int64_t *)calloc((size_t)K, sizeof(int64_t));
    char *seen = (char *)calloc((size_t)K, 1);
    int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)K);
    omove *moves = (omove *)malloc(sizeof(omove) * (size_t)V);
    int32_t *gseq = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
    int32_t *viol = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
    int64_t *doff = NULL; int32_t *dst = NULL;
    edge_parts ep = {0};
    ep.off = (int64_t *)malloc(sizeof(int64_t) * ((size_t)E + 1));
    ep.len = (int32_t *)calloc((size_t)E + 1, sizeof(int32_t));
    ep.a = (pcount *)malloc(sizeof(pcount) * (size_t)(g->poff[E] > 0 ? g->poff[E] : 1));
    if (!size || !inb || !pres || !seen || !touched || !moves || !gseq || !viol ||
        !ep.off || !ep.len || !ep.a) goto done;
    /* dst_l(e) = {n : e in in(n)} */
    if (transpose(V, E, g->noff, g->in, &doff, &dst)) goto done;

    for (int32_t n = 0; n < V; ++n) size[rho[n]] += g->w[n];
    for (int32_t e = 0; e <= E; ++e) ep.off[e] = g->poff[e];
    for (int32_t e = 0; e < E; ++e) {
        for (int64_t j = g->poff[e]; j < g->poff[e + 1]; ++j) ep_add(&ep, e, rho[g->pins[j]], 1, 0);
        for (int64_t j = doff[e]; j < doff[e + 1]; ++j) ep_add(&ep, e, rho[dst[j]], 0, 1);
        for (int32_t i = 0; i < ep.len[e]; ++i)
            if (ep.a[ep.off[e] + i].cnt_in > 0) inb[ep.a[ep.off[e] + i].p]++;
    }

    /* in-isolation proposals, Eq. (3) */
    int32_t M = 0;
    for (int32_t n = 0; n < V; ++n) {
        int32_t ps = rho[n];
        int64_t saving = 0, wI = 0;
        int32_t nt = 0;
        for (int64_t i = g->ioff[n]; i < g->ioff[n + 1]; ++i) {
            int32_t e = g->inc[i];
            int64_t we = ew ? ew[e] : 1;
            wI += we;
            pcount *s = ep.a + ep.off[e];
            for (int32_t t = 0; t < ep.len[e]; ++t) {
                int32_t p = s[t].p;
                if (p == ps) { if (s[t].cnt == 1) saving += we; continue; }
                if (!seen[p]) { seen[p] = 1; touched[nt++] = p; }
                pres[p] += we;                 /* loss(n, p) = wI - pres(p) */
            }
        }
        int32_t bestp = -1;
        int64_t bestg = 0;
        for (int32_t t = 0; t < nt; ++t) {
            int32_t p = touched[t];
            if (size[p] + g->w[n] <= omega) {
                int64_t gain = saving - (wI - pres[p]);
                if (bestp < 0 || gain > bestg || (gain == bestg && p < bestp)) { bestp = p; bestg = gain; }
            }
        }
        for (int32_t t = 0; t < nt; ++t) { seen[touched[t]] = 0; pres[touched[t]] = 0; }
        if (bestp >= 0 && bestg > 0) {
            moves[M].n = n; moves[M].ps = ps; moves[M].pd = bestp; moves[M].gain = (int32_t)bestg;
            M++;
        }
    }
    qsort(moves, (size_t)M, sizeof(omove), cmp_move);

    /* apply the sequence to a copy of the state, one move at a time */
    int64_t nviol = 0;     /* the starting partition is valid, checked below */
    for (int32_t p = 0; p < K; ++p) if (size[p] > omega || inb[p] > delta) nviol++;
    if (nviol != 0) { rc = ORC_INTERNAL; goto done; }
    for (int32_t k = 0; k < M; ++k) {
        int32_t n = moves[k].n, ps = moves[k].ps, pd = moves[k].pd;
        int64_t old_bad = (size[ps] > omega || inb[ps] > delta) + (size[pd] > omega || inb[pd] > delta);
        int64_t gk = 0;
        int64_t j = g->noff[n];               /* in(n) is a sorted subset of I(n) */
        for (int64_t i = g->ioff[n]; i < g->ioff[n + 1]; ++i) {
            int32_t e = g->inc[i];
            int64_t we = ew ? ew[e] : 1;
            int32_t isin = (j < g->noff[n + 1] && g->in[j] == e);
            if (isin) j++;
            pcount *c = ep_find(&ep, e, ps);  /* n is a pin of e, so c exists */
            pcount *d = ep_find(&ep, e, pd);
            if (c->cnt == 1) gk += we;                 /* e leaves ps: one cut less */
            if (!d || d->cnt == 0) gk -= we;           /* e reaches pd: one cut more */
            if (isin && c->cnt_in == 1) inb[ps]--;     /* ps loses inbound e */
            if (isin && (!d || d->cnt_in == 0)) inb[pd]++;  /* pd gains inbound e */
            ep_add(&ep, e, ps, -1, -isin);
            ep_add(&ep, e, pd, +1, +isin);
        }
        size[ps] -= g->w[n];
        size[pd] += g->w[n];
        int64_t new_bad = (size[ps] > omega || inb[ps] > delta) + (size[pd] > omega || inb[pd] > delta);
        nviol += new_bad - old_bad;
        gseq[k] = (int32_t)gk;
        viol[k] = (int32_t)nviol;
        rho[n] = pd;                 /* provisional; undone below if not chosen */
    }
    /* best valid prefix */
    int32_t kstar = 0;
    int64_t G = 0, bestG = 0;
    int have = 0;
    for (int32_t k = 1; k <= M; ++k) {
        G += gseq[k - 1];
        if (viol[k - 1] != 0) continue;
        if (!have || G >= bestG) { bestG = G; kstar = k; have = 1; }
    }
    if (!have || bestG <= 0) kstar = 0;
    for (int32_t k = M - 1; k >= kstar; --k) rho[moves[k].n] = moves[k].ps;   /* undo the rest */
    if (tr) {
        tr->M = M; tr->kstar = kstar; tr->gain = kstar > 0 ? bestG : 0;
        tr->moves = moves; tr->gain_seq = gseq; tr->viol = viol;
        moves = NULL; gseq = NULL; viol = NULL;
    }
    rc = ORC_OK;
done:
    free(size); free(inb); free(pres); free(seen); free(touched);
    free(moves); free(gseq); free(viol); free(doff); free(dst);
    free(ep.off); free(ep.len); free(ep.a);
    return rc;
}

/* ------------------------------------------------------------------ */
/* The whole method (Sec. II-B): coarsen, then refine while projecting. */
/* ------------------------------------------------------------------ */
typedef struct {
    /* per level; every level removes at least one node, so |N| + 1 slots
     * always suffice */
    int32_t cap;
    olevel *G;                    /* G[0] = input hypergraph */
    int32_t **pair, **score, **match, **gamma, **rho_in, **rho_out;
    int32_t **key;                /* learned order only: key(n, pair(n)) */
    rtrace *rt;                   /* trace of the last pass at each level */
    int32_t nlev;                 /* levels built (L + 1) */
    int32_t top_is_gamma;         /* coarsest level ended by the node target */
    int32_t K;                    /* part-id range during refinement */
    int32_t *src;                 /* src(e) of the input */
    int32_t *ew;                  /* edge weights or NULL (unit) */
    int32_t *in_off, *in_pins;    /* the input CSR as given (pin order kept) */
    const omodel *model;          /* learned order, or NULL for Eq. (2) */
    int32_t *part_ids;            /* [N] final, compacted */
    int64_t *part_weight;         /* [num_parts] */
    int32_t *part_inbound;        /* [num_parts] */
    int32_t num_parts;
    int64_t cost;
    int32_t done;
} orun;

static void orun_clear(orun *r) {
    for (int l = 0; l < r->cap; ++l) {
        if (l > 0) olevel_free(&r->G[l]);
        free(r->pair[l]); free(r->score[l]); free(r->match[l]); free(r->gamma[l]);
        free(r->rho_in[l]); free(r->rho_out[l]); free(r->key[l]);
        free(r->rt[l].moves); free(r->rt[l].gain_seq); free(r->rt[l].viol);
        r->pair[l] = r->score[l] = r->match[l] = r->gamma[l] = r->key[l] = NULL;
        r->rho_in[l] = r->rho_out[l] = NULL;
        memset(&r->rt[l], 0, sizeof(rtrace));
    }
    free(r->part_ids); free(r->part_weight); free(r->part_inbound);
    r->part_ids = NULL; r->part_weight = NULL; r->part_inbound = NULL;
    r->nlev = 1; r->done = 0; r->num_parts = 0; r->cost = 0;   /* level 0 always exists */
}

static int orun_create_mode(int32_t N, int32_t E, const int32_t *offsets, const int32_t *pins,
                            const int32_t *node_w, const int32_t *edge_w, int32_t incident,
                            orun **out);

int orun_create(int32_t N, int32_t E, const int32_t *offsets, const int32_t *pins,
                const int32_t *node_w, const int32_t *edge_w, orun **out) {
    return orun_create_mode(N, E, offsets, pins, node_w, edge_w, 0, out);
}

/* Delta counting every incident hyperedge instead of the inbound ones. */
int orun_create_incident(int32_t N, int32_t E, const int32_t *offsets, const int32_t *pins,
                         const int32_t *node_w, const int32_t *edge_w, orun **out) {
    return orun_create_mode(N, E, offsets, pins, node_w, edge_w, 1, out);
}

/* Delta counting the hyperedges whose source lies in the part. */
int orun_create_outbound(int32_t N, int32_t E, const int32_t *offsets, const int32_t *pins,
                         const int32_t *node_w, const int32_t *edge_w, orun **out) {
    return orun_create_mode(N, E, offsets, pins, node_w, edge_w, 2, out);
}

static int orun_create_mode(int32_t N, int32_t E, const int32_t *offsets, const int32_t *pins,
                            const int32_t *node_w, const int32_t *edge_w, int32_t incident,
                            orun **out) {
    orun *r = (orun *)calloc(1, sizeof(orun));
    if (!r) return ORC_OOM;
    if (N < 1) { free(r); return ORC_INVALID; }
    r->cap = N + 1;
    r->G = (olevel *)calloc((size_t)r->cap, sizeof(olevel));
    r->pair = (int32_t **)calloc((size_t)r->cap, sizeof(int32_t *));
    r->score = (int32_t **)calloc((size_t)r->cap, sizeof(int32_t *));
    r->match = (int32_t **)calloc((size_t)r->cap, sizeof(int32_t *));
    r->gamma = (int32_t **)calloc((size_t)r->cap, sizeof(int32_t *));
    r->rho_in = (int32_t **)calloc((size_t)r->cap, sizeof(int32_t *));
    r->rho_out = (int32_t **)calloc((size_t)r->cap, sizeof(int32_t *));
    r->key = (int32_t **)calloc((size_t)r->cap, sizeof(int32_t *));
    r->rt = (rtrace *)calloc((size_t)r->cap, sizeof(rtrace));
    int rc = ORC_OOM;
    if (r->G && r->pair && r->score && r->match && r->gamma && r->rho_in && r->rho_out && r->key && r->rt)
        rc = build_level0(N, E, offsets, pins, node_w, edge_w, incident, &r->G[0], &r->src);
    if (!rc) {
        r->in_off = (int32_t *)malloc(sizeof(int32_t) * ((size_t)E + 1));
        r->in_pins = (int32_t *)malloc(sizeof(int32_t) * (size_t)(offsets[E] > 0 ? offsets[E] : 1));
        if (!r->in_off || !r->in_pins) {
            rc = ORC_OOM;
            olevel_free(&r->G[0]);
            free(r->src);
        } else {
            memcpy(r->in_off, offsets, sizeof(int32_t) * ((size_t)E + 1));
            memcpy(r->in_pins, pins, sizeof(int32_t) * (size_t)offsets[E]);
        }
    }
    if (rc) {
        free(r->in_off); free(r->in_pins);
        free(r->G); free(r->pair); free(r->score); free(r->match); free(r->gamma);
        free(r->rho_in); free(r->rho_out); free(r->key); free(r->rt); free(r);
        return rc;
    }
    r->nlev = 1;
    if (edge_w) {
        r->ew = (int32_t *)malloc(sizeof(int32_t) * (size_t)(E > 0 ? E : 1));
        if (!r->ew) { olevel_free(&r->G[0]); free(r->src); free(r); return ORC_OOM; }
        memcpy(r->ew, edge_w, sizeof(int32_t) * (size_t)E);
    }
    *out = r;
    return ORC_OK;
}

void orun_destroy(orun *r) {
    if (!r) return;
    orun_clear(r);
    olevel_free(&r->G[0]);
    free(r->src); free(r->ew); free(r->in_off); free(r->in_pins);
    free(r->G); free(r->pair); free(r->score); free(r->match); free(r->gamma);
    free(r->rho_in); free(r->rho_out); free(r->key); free(r->rt);
    free(r);
}

/* Eq. (1): sum over e of omega(e) * (number of distinct parts in e - 1). */
static int64_t connectivity(const olevel *g, const int32_t *ew, const int32_t *rho, int32_t K) {
    int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * (size_t)(K > 0 ? K : 1));
    if (!mark) return -1;
    for (int32_t p = 0; p < K; ++p) mark[p] = -1;
    int64_t c = 0;
    for (int32_t e = 0; e < g->E; ++e) {
        int64_t lam = 0;
        for (int64_t j = g->poff[e]; j < g->poff[e + 1]; ++j) {
            int32_t p = rho[g->pins[j]];
            if (mark[p] != e) { mark[p] = e; lam++; }
        }
        c += (int64_t)(ew ? ew[e] : 1) * (lam - 1);
    }
    free(mark);
    return c;
}

/* max_levels > 0 stops coarsening after that many matchings, the clusters
 * of the last one becoming the parts exactly as when the node target is
 * reached; 0 applies the paper's stop rule alone.  (Not part of the method:
 * a bounded prefix of it, for timing samples and large-input checks.) */
static int partition_impl(orun *r, int64_t omega, int64_t delta, int32_t refine_passes,
                          int32_t max_levels, int32_t matching) {
    if (omega < 1 || delta < 0 || refine_passes < 0) return ORC_INVALID;
    orun_clear(r);
    olevel *G0 = &r->G[0];
    /* Singletons must already satisfy both bounds, or no partition exists. */
    int64_t W = 0;
    for (int32_t n = 0; n < G0->V; ++n) {
        if (G0->w[n] > omega || G0->noff[n + 1] - G0->noff[n] > delta) return ORC_INFEASIBLE;
        W += G0->w[n];
    }
    /* Sec. II-B: stop at ceil(|N| / Omega) nodes.  Reading: |N| is the total
     * node weight (equal to |N| at unit weights). */
    int64_t target = W / omega + (W % omega != 0);
    int rc = ORC_OK;
    int32_t l = 0;
    int32_t *rho = NULL;
    r->nlev = 1;
    r->top_is_gamma = 0;
    if (G0->V <= target) {
        r->K = G0->V;
    } else {
        for (;;) {
            olevel *g = &r->G[l];
            int32_t V = g->V;
            r->pair[l] = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
            r->score[l] = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
            r->match[l] = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
            int64_t *hist = (int64_t *)calloc((size_t)V, sizeof(int64_t));
            int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
            if (!r->pair[l] || !r->score[l] || !r->match[l] || !hist || !touched) {
                free(hist); free(touched); rc = ORC_OOM; goto fail;
            }
            int64_t *mscore = (int64_t *)malloc(sizeof(int64_t) * (size_t)V);
            if (r->model) r->key[l] = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
            if (!mscore || (r->model && !r->key[l])) {
                free(hist); free(touched); free(mscore); rc = ORC_OOM; goto fail;
            }
            if (r->model)
                rc = score_level_learned(g, r->ew, omega, delta, r->model, r->pair[l], r->score[l],
                                         r->key[l], hist, touched);
            else
                rc = score_level(g, r->ew, omega, delta, r->pair[l], r->score[l], hist, touched, NULL, 0);
            free(hist); free(touched);
            if (rc) { free(mscore); goto fail; }
            for (int32_t n = 0; n < V; ++n)
                mscore[n] = r->model ? learned_composite(r->key[l][n], r->score[l][n]) : r->score[l][n];
            /* matching 1: the exact maximum-weight matching (plain order only) */
            rc = matching == 1 ? match_dp(V, r->pair[l], mscore, r->match[l])
                               : match_walks(V, r->pair[l], mscore, r->match[l]);
            free(mscore);
            if (rc) goto fail;
            int32_t matched = 0;
            for (int32_t n = 0; n < V; ++n) matched += r->match[l][n] != n;
            if (matched == 0) {                 /* no cluster can be unified */
                r->K = V;
                break;
            }
            r->gamma[l] = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
            if (!r->gamma[l]) { rc = ORC_OOM; goto fail; }
            int32_t V2 = gamma_from_match(V, r->match[l], r->gamma[l]);
            /* Sec. III-B.4: once the target is reached the clusters become
             * the partitions without building another level. */
            if (V2 <= target || (max_levels > 0 && l + 1 >= max_levels)) {
                r->K = V2;
                r->top_is_gamma = 1;
                break;
            }
            if (l + 1 >= r->cap) { rc = ORC_INTERNAL; goto fail; }
            rc = contract(g, r->gamma[l], V2, &r->G[l + 1]);
            if (rc) goto fail;
            l++;
            r->nlev = l + 1;
        }
    }
    /* initial partition of the coarsest level */
    {
        int32_t V = r->G[l].V;
        rho = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
        if (!rho) { rc = ORC_OOM; goto fail; }
        for (int32_t n = 0; n < V; ++n) rho[n] = r->top_is_gamma ? r->gamma[l][n] : n;
    }
    /* refine every level from the coarsest to the input, projecting down */
    for (int32_t lv = l; lv >= 0; --lv) {
        int32_t V = r->G[lv].V;
        r->rho_in[lv] = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
        r->rho_out[lv] = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
        if (!r->rho_in[lv] || !r->rho_out[lv]) { rc = ORC_OOM; goto fail; }
        memcpy(r->rho_in[lv], rho, sizeof(int32_t) * (size_t)V);
        for (int32_t p = 0; p < refine_passes; ++p) {
            free(r->rt[lv].moves); free(r->rt[lv].gain_seq); free(r->rt[lv].viol);
            memset(&r->rt[lv], 0, sizeof(rtrace));
            rc = refine_pass(&r->G[lv], r->ew, rho, r->K, omega, delta, &r->rt[lv]);
            if (rc) goto fail;
        }
        memcpy(r->rho_out[lv], rho, sizeof(int32_t) * (size_t)V);
        if (lv > 0) {            /* rho_{l-1}(n) = rho_l(gamma_{l-1}(n)) */
            int32_t Vf = r->G[lv - 1].V;
            int32_t *fine = (int32_t *)malloc(sizeof(int32_t) * (size_t)Vf);
            if (!fine) { rc = ORC_OOM; goto fail; }
            for (int32_t n = 0; n < Vf; ++n) fine[n] = rho[r->gamma[lv - 1][n]];
            free(rho);
            rho = fine;
        }
    }
    /* output: keep the non-empty parts, numbered in their old order */
    {
        int32_t K = r->K, N = G0->V;
        int64_t *wsum = (int64_t *)calloc((size_t)K, sizeof(int64_t));
        int32_t *newid = (int32_t *)malloc(sizeof(int32_t) * (size_t)K);
        r->part_ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
        if (!wsum || !newid || !r->part_ids) { free(wsum); free(newid); rc = ORC_OOM; goto fail; }
        for (int32_t n = 0; n < N; ++n) wsum[rho[n]] += G0->w[n];
        int32_t np = 0;
        for (int32_t p = 0; p < K; ++p) newid[p] = wsum[p] > 0 ? np++ : -1;
        for (int32_t n = 0; n < N; ++n) r->part_ids[n] = newid[rho[n]];
        r->num_parts = np;
        r->part_weight = (int64_t *)calloc((size_t)(np > 0 ? np : 1), sizeof(int64_t));
        r->part_inbound = (int32_t *)calloc((size_t)(np > 0 ? np : 1), sizeof(int32_t));
        int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * (size_t)(G0->E > 0 ? G0->E : 1));
        if (!r->part_weight || !r->part_inbound || !mark) { free(wsum); free(newid); free(mark); rc = ORC_OOM; goto fail; }
        for (int32_t p = 0; p < K; ++p) if (newid[p] >= 0) r->part_weight[newid[p]] = wsum[p];
        /* part_inbound(p) = |union of in(n) over n in p| (Sec. II-A) */
        int32_t *members_off = (int32_t *)calloc((size_t)np + 1, sizeof(int32_t));
        int32_t *members = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
        if (!members_off || !members) { free(wsum); free(newid); free(mark); free(members_off); free(members); rc = ORC_OOM; goto fail; }
        for (int32_t n = 0; n < N; ++n) members_off[r->part_ids[n] + 1]++;
        for (int32_t p = 0; p < np; ++p) members_off[p + 1] += members_off[p];
        {
            int32_t *cur = (int32_t *)malloc(sizeof(int32_t) * (size_t)(np > 0 ? np : 1));
            if (!cur) { free(wsum); free(newid); free(mark); free(members_off); free(members); rc = ORC_OOM; goto fail; }
            memcpy(cur, members_off, sizeof(int32_t) * (size_t)np);
            for (int32_t n = 0; n < N; ++n) members[cur[r->part_ids[n]]++] = n;
            free(cur);
        }
        for (int32_t e = 0; e < G0->E; ++e) mark[e] = -1;
        for (int32_t p = 0; p < np; ++p) {
            int32_t cnt = 0;
            for (int32_t i = members_off[p]; i < members_off[p + 1]; ++i) {
                int32_t n = members[i];
                for (int64_t j = G0->noff[n]; j < G0->noff[n + 1]; ++j)
                    if (mark[G0->in[j]] != p) { mark[G0->in[j]] = p; cnt++; }
            }
            r->part_inbound[p] = cnt;
        }
        free(members_off); free(members); free(mark);
        r->cost = connectivity(G0, r->ew, r->part_ids, np > 0 ? np : 1);
        free(wsum); free(newid);
    }
    free(rho);
    r->done = 1;
    return ORC_OK;
fail:
    free(rho);
    orun_clear(r);
    return rc;
}

/* The method as printed (Eq. (2) order). */
int orun_partition(orun *r, int64_t omega, int64_t delta, int32_t refine_passes) {
    r->model = NULL;
    return partition_impl(r, omega, delta, refine_passes, 0, 0);
}

/* The same, coarsening cut after max_levels matchings (see partition_impl). */
int orun_partition_cut(orun *r, int64_t omega, int64_t delta, int32_t refine_passes,
                       int32_t max_levels) {
    if (max_levels < 0) return ORC_INVALID;
    r->model = NULL;
    return partition_impl(r, omega, delta, refine_passes, max_levels, 0);
}

/* With a choice of matching: 0 the two walks (Sec. III-B.3), 1 the exact
 * maximum-weight matching of the pairing pseudo-forest (match_dp). */
int orun_partition_ex(orun *r, int64_t omega, int64_t delta, int32_t refine_passes,
                      int32_t max_levels, int32_t matching) {
    if (max_levels < 0 || matching < 0 || matching > 1) return ORC_INVALID;
    r->model = NULL;
    return partition_impl(r, omega, delta, refine_passes, max_levels, matching);
}

/* The same with the learned candidate order (model as bfloat16 bits). */
int orun_partition_learned(orun *r, int64_t omega, int64_t delta, int32_t refine_passes,
                           const uint16_t *w1, const uint16_t *b1, const uint16_t *w2, uint16_t b2,
                           int32_t key_bits) {
    omodel M;
    int rc = model_from_bits(w1, b1, w2, b2, key_bits, &M);
    if (rc) return rc;
    r->model = &M;
    rc = partition_impl(r, omega, delta, refine_passes, 0, 0);
    r->model = NULL;
    return rc;
}

/* ------------------------------------------------------------------ */
/* Accessors (read-only views for the test suite).                     */
/* ------------------------------------------------------------------ */
enum {
    ORC_A_PAIR = 0, ORC_A_SCORE = 1, ORC_A_MATCH = 2, ORC_A_GAMMA = 3,
    ORC_A_RHO_IN = 4, ORC_A_RHO_OUT = 5, ORC_A_W = 6, ORC_A_KEY = 19,
    ORC_A_PINS_OFF = 7, ORC_A_PINS = 8, ORC_A_INC_OFF = 9, ORC_A_INC = 10,
    ORC_A_IN_OFF = 11, ORC_A_IN = 12,
    ORC_A_MOVE_N = 13, ORC_A_MOVE_PS = 14, ORC_A_MOVE_PD = 15, ORC_A_MOVE_GAIN = 16,
    ORC_A_GAIN_SEQ = 17, ORC_A_VIOL = 18
};

int32_t orun_num_levels(const orun *r) { return r->nlev; }
int32_t orun_top_is_gamma(const orun *r) { return r->top_is_gamma; }
int32_t orun_K(const orun *r) { return r->K; }
int64_t orun_cost(const orun *r) { return r->cost; }
int32_t orun_num_parts(const orun *r) { return r->num_parts; }
int32_t orun_level_V(const orun *r, int32_t l) { return (l >= 0 && l < r->nlev) ? r->G[l].V : -1; }
int64_t orun_level_P(const orun *r, int32_t l) { return (l >= 0 && l < r->nlev) ? r->G[l].poff[r->G[l].E] : -1; }
int64_t orun_level_in_total(const orun *r, int32_t l) { return (l >= 0 && l < r->nlev) ? r->G[l].noff[r->G[l].V] : -1; }
int32_t orun_refine_M(const orun *r, int32_t l) { return r->rt[l].M; }
int32_t orun_refine_kstar(const orun *r, int32_t l) { return r->rt[l].kstar; }
int64_t orun_refine_gain(const orun *r, int32_t l) { return r->rt[l].gain; }

/* Length of array `which` at level l, or -1 if it does not exist. */
int64_t orun_array_len(const orun *r, int32_t l, int32_t which) {
    if (l < 0 || l >= r->nlev) return -1;
    const olevel *g = &r->G[l];
    switch (which) {
    case ORC_A_PAIR: return r->pair[l] ? g->V : -1;
    case ORC_A_SCORE: return r->score[l] ? g->V : -1;
    case ORC_A_MATCH: return r->match[l] ? g->V : -1;
    case ORC_A_GAMMA: return r->gamma[l] ? g->V : -1;
    case ORC_A_RHO_IN: return r->rho_in[l] ? g->V : -1;
    case ORC_A_RHO_OUT: return r->rho_out[l] ? g->V : -1;
    case ORC_A_KEY: return r->key[l] ? g->V : -1;
    case ORC_A_W: return g->V;
    case ORC_A_PINS_OFF: return (int64_t)g->E + 1;
    case ORC_A_PINS: return g->poff[g->E];
    case ORC_A_INC_OFF: return (int64_t)g->V + 1;
    case ORC_A_INC: return g->ioff[g->V];
    case ORC_A_IN_OFF: return (int64_t)g->V + 1;
    case ORC_A_IN: return g->noff[g->V];
    case ORC_A_MOVE_N: case ORC_A_MOVE_PS: case ORC_A_MOVE_PD: case ORC_A_MOVE_GAIN:
    case ORC_A_GAIN_SEQ: case ORC_A_VIOL: return r->rt[l].M;
    default: return -1;
    }
}

/* Copies array `which` of level l into out (int64 elements). */
int orun_array(const orun *r, int32_t l, int32_t which, int64_t *out) {
    int64_t len = orun_array_len(r, l, which);
    if (len < 0) return ORC_INVALID;
    const olevel *g = &r->G[l];
    for (int64_t i = 0; i < len; ++i) {
        int64_t v = 0;
        switch (which) {
        case ORC_A_PAIR: v = r->pair[l][i]; break;
        case ORC_A_SCORE: v = r->score[l][i]; break;
        case ORC_A_MATCH: v = r->match[l][i]; break;
        case ORC_A_GAMMA: v = r->gamma[l][i]; break;
        case ORC_A_RHO_IN: v = r->rho_in[l][i]; break;
        case ORC_A_RHO_OUT: v = r->rho_out[l][i]; break;
        case ORC_A_KEY: v = r->key[l][i]; break;
        case ORC_A_W: v = g->w[i]; break;
        case ORC_A_PINS_OFF: v = g->poff[i]; break;
        case ORC_A_PINS: v = g->pins[i]; break;
        case ORC_A_INC_OFF: v = g->ioff[i]; break;
        case ORC_A_INC: v = g->inc[i]; break;
        case ORC_A_IN_OFF: v = g->noff[i]; break;
        case ORC_A_IN: v = g->in[i]; break;
        case ORC_A_MOVE_N: v = r->rt[l].moves[i].n; break;
        case ORC_A_MOVE_PS: v = r->rt[l].moves[i].ps; break;
        case ORC_A_MOVE_PD: v = r->rt[l].moves[i].pd; break;
        case ORC_A_MOVE_GAIN: v = r->rt[l].moves[i].gain; break;
        case ORC_A_GAIN_SEQ: v = r->rt[l].gain_seq[i]; break;
        case ORC_A_VIOL: v = r->rt[l].viol[i]; break;
        }
        out[i] = v;
    }
    return ORC_OK;
}

int orun_part_ids(const orun *r, int32_t *out) {
    if (!r->done) return ORC_INVALID;
    memcpy(out, r->part_ids, sizeof(int32_t) * (size_t)r->G[0].V);
    return ORC_OK;
}

int orun_part_stats(const orun *r, int64_t *weight, int32_t *inbound) {
    if (!r->done) return ORC_INVALID;
    if (weight) memcpy(weight, r->part_weight, sizeof(int64_t) * (size_t)r->num_parts);
    if (inbound) memcpy(inbound, r->part_inbound, sizeof(int32_t) * (size_t)r->num_parts);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Single steps on caller-given data (for the pinning tests).          */
/* ------------------------------------------------------------------ */

/* hist(n, .) of level l as a dense row (Eq. (2)); out[m] for every m. */
int orun_hist_row(const orun *r, int32_t l, int32_t n, int64_t *out) {
    if (l < 0 || l >= r->nlev) return ORC_INVALID;
    const olevel *g = &r->G[l];
    if (n < 0 || n >= g->V) return ORC_INVALID;
    memset(out, 0, sizeof(int64_t) * (size_t)g->V);
    for (int64_t i = g->ioff[n]; i < g->ioff[n + 1]; ++i) {
        int32_t e = g->inc[i];
        for (int64_t j = g->poff[e]; j < g->poff[e + 1]; ++j)
            if (g->pins[j] != n) out[g->pins[j]] += r->ew ? r->ew[e] : 1;
    }
    return ORC_OK;
}

/* Candidate selection on level 0 of the input alone. */
int orun_score0(const orun *r, int64_t omega, int64_t delta, int32_t *pair, int32_t *score) {
    const olevel *g = &r->G[0];
    int64_t *hist = (int64_t *)calloc((size_t)g->V, sizeof(int64_t));
    int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)g->V);
    if (!hist || !touched) { free(hist); free(touched); return ORC_OOM; }
    int rc = score_level(g, r->ew, omega, delta, pair, score, hist, touched, NULL, 0);
    free(hist); free(touched);
    return rc;
}

/* Candidate selection on level 0 for the listed nodes only (pair[t], score[t]
 * belong to nodes[t]). */
int orun_score0_nodes(const orun *r, int64_t omega, int64_t delta, const int32_t *nodes,
                      int32_t count, int32_t *pair, int32_t *score) {
    const olevel *g = &r->G[0];
    for (int32_t t = 0; t < count; ++t) if (nodes[t] < 0 || nodes[t] >= g->V) return ORC_INVALID;
    int64_t *hist = (int64_t *)calloc((size_t)g->V, sizeof(int64_t));
    int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)g->V);
    if (!hist || !touched) { free(hist); free(touched); return ORC_OOM; }
    int rc = score_level(g, r->ew, omega, delta, pair, score, hist, touched, nodes, count);
    free(hist); free(touched);
    return rc;
}

/* Matching of an arbitrary pairing graph; method 0 = the two walks,
 * method 1 = the lock recursion. */
int oracle_match64(int32_t V, const int32_t *pair, const int64_t *score, int32_t method, int32_t *match);

int oracle_match(int32_t V, const int32_t *pair, const int32_t *score, int32_t method, int32_t *match) {
    int64_t *s64 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(V > 0 ? V : 1));
    if (!s64) return ORC_OOM;
    for (int32_t n = 0; n < V; ++n) s64[n] = score[n];
    int rc = oracle_match64(V, pair, s64, method, match);
    free(s64);
    return rc;
}

/* Same with int64 scores (the learned order's composite keys).
 * method 0: the two walks; 1: the lock restatement; 2: exact DP. */
int oracle_match64(int32_t V, const int32_t *pair, const int64_t *score, int32_t method, int32_t *match) {
    if (method == 2) return match_dp(V, pair, score, match);
    return method == 0 ? match_walks(V, pair, score, match) : match_locks(V, pair, score, match);
}

int32_t oracle_gamma(int32_t V, const int32_t *match, int32_t *gamma) {
    return gamma_from_match(V, match, gamma);
}

/* One refinement pass on level 0 of the input with a caller partition
 * rho (part ids in [0, K)); rho is updated in place.  The trace arrays
 * (each of length >= N) receive the sorted moves, in-sequence gains and
 * violation counts; *M and *kstar their count and the applied prefix. */
int orun_refine0(const orun *r, int32_t *rho, int32_t K, int64_t omega, int64_t delta,
                 int32_t *M, int32_t *kstar, int64_t *gain,
                 int32_t *mv_n, int32_t *mv_ps, int32_t *mv_pd, int32_t *mv_gain,
                 int32_t *gain_seq, int32_t *viol) {
    for (int32_t n = 0; n < r->G[0].V; ++n) if (rho[n] < 0 || rho[n] >= K) return ORC_INVALID;
    rtrace t = {0};
    int rc = refine_pass(&r->G[0], r->ew, rho, K, omega, delta, &t);
    if (rc) return rc;
    *M = t.M; *kstar = t.kstar; *gain = t.gain;
    for (int32_t i = 0; i < t.M; ++i) {
        mv_n[i] = t.moves[i].n; mv_ps[i] = t.moves[i].ps; mv_pd[i] = t.moves[i].pd;
        mv_gain[i] = t.moves[i].gain; gain_seq[i] = t.gain_seq[i]; viol[i] = t.viol[i];
    }
    free(t.moves); free(t.gain_seq); free(t.viol);
    return ORC_OK;
}

/* Contraction of level 0 by a caller matching: fills the coarse level as
 * level 1 of the run (replacing any previous hierarchy). */
int orun_contract0(orun *r, const int32_t *match) {
    orun_clear(r);
    int32_t V = r->G[0].V;
    r->match[0] = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
    r->gamma[0] = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
    if (!r->match[0] || !r->gamma[0]) return ORC_OOM;
    memcpy(r->match[0], match, sizeof(int32_t) * (size_t)V);
    for (int32_t n = 0; n < V; ++n)
        if (match[n] < 0 || match[n] >= V || match[match[n]] != n) return ORC_INVALID;
    int32_t V2 = gamma_from_match(V, match, r->gamma[0]);
    int rc = contract(&r->G[0], r->gamma[0], V2, &r->G[1]);
    if (rc) return rc;
    r->nlev = 2;
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Learned order: single steps and training (for the pinning tests).   */
/* ------------------------------------------------------------------ */
float oracle_lg1p(int64_t x) { return lg1p(x); }

/* Network score and key of one feature vector. */
int oracle_mlp(const uint16_t *w1, const uint16_t *b1, const uint16_t *w2, uint16_t b2,
               int32_t key_bits, const float *x, float *score, int32_t *key) {
    omodel M;
    int rc = model_from_bits(w1, b1, w2, b2, key_bits, &M);
    if (rc) return rc;
    *score = mlp_score(&M, x);
    *key = score_key(*score, key_bits);
    return ORC_OK;
}

/* Features of the level-0 pair (n, m), m != n: hist as the weight of
 * I(n) n I(m) (a merge of the two sorted lists), the union by marking. */
static void features0(const orun *r, int32_t n, int32_t m, int32_t *stamp, float *x) {
    const olevel *g = &r->G[0];
    int64_t h = 0, a = g->ioff[n], b = g->ioff[m];
    while (a < g->ioff[n + 1] && b < g->ioff[m + 1]) {
        if (g->inc[a] < g->inc[b]) ++a;
        else if (g->inc[a] > g->inc[b]) ++b;
        else { h += r->ew ? r->ew[g->inc[a]] : 1; ++a; ++b; }
    }
    for (int64_t j = g->noff[n]; j < g->noff[n + 1]; ++j) stamp[g->in[j]] = n;
    int64_t uni = union_size(g, n, m, stamp);
    for (int64_t j = g->noff[n]; j < g->noff[n + 1]; ++j) stamp[g->in[j]] = -1;
    pair_features(g, n, m, h, uni, x);
}

int orun_features0(const orun *r, int32_t n, int32_t m, float *x) {
    const olevel *g = &r->G[0];
    if (n < 0 || m < 0 || n >= g->V || m >= g->V || n == m) return ORC_INVALID;
    int32_t *stamp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->E > 0 ? g->E : 1));
    if (!stamp) return ORC_OOM;
    for (int32_t e = 0; e < g->E; ++e) stamp[e] = -1;
    features0(r, n, m, stamp, x);
    free(stamp);
    return ORC_OK;
}

/* The i-th output (i >= 0) of the SplitMix64 generator started at `seed`
 * (Steele, Lea and Flood, 2014): the state advances by the golden-ratio
 * increment before each output, which is then mixed by two xor-shift-
 * multiply rounds and a final xor-shift. */
static uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/*
 * Training pairs for the learned order, labelled by a partition of the
 * input (part_ids): slot s = n * per_node + k (k < per_node) draws
 *   u0 = splitmix64_at(seed, 2 s), u1 = splitmix64_at(seed, 2 s + 1),
 *   e  = the (u0 mod |I(n)|)-th hyperedge of I(n) (ascending ids),
 *   m  = the (u1 mod |pins(e)|)-th pin of e in the input's pin order,
 * so neighbours are drawn in proportion to the hyperedges they share with n.
 * The slot holds the features of (n, m), label 1 if both are in the same
 * part, else 0; label -1 (no sample) when m = n or I(n) is empty.
 */
int orun_learn_samples(const orun *r, const int32_t *part_ids, uint64_t seed, int32_t per_node,
                       float *x, float *y, int32_t *partner) {
    const olevel *g = &r->G[0];
    if (per_node < 1) return ORC_INVALID;
    int32_t *stamp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->E > 0 ? g->E : 1));
    if (!stamp) return ORC_OOM;
    for (int32_t e = 0; e < g->E; ++e) stamp[e] = -1;
    for (int32_t n = 0; n < g->V; ++n) {
        for (int32_t k = 0; k < per_node; ++k) {
            int64_t s = (int64_t)n * per_node + k;
            float *xs = x + s * OMLP_IN;
            int64_t deg = g->ioff[n + 1] - g->ioff[n];
            int32_t m = n;
            if (deg > 0) {
                uint64_t u0 = splitmix64_at(seed, 2u * (uint64_t)s);
                uint64_t u1 = splitmix64_at(seed, 2u * (uint64_t)s + 1u);
                int32_t e = g->inc[g->ioff[n] + (int64_t)(u0 % (uint64_t)deg)];
                int64_t sz = r->in_off[e + 1] - r->in_off[e];
                m = r->in_pins[r->in_off[e] + (int64_t)(u1 % (uint64_t)sz)];
            }
            if (m == n) {
                for (int i = 0; i < OMLP_IN; ++i) xs[i] = 0.0f;
                y[s] = -1.0f;
                if (partner) partner[s] = -1;
                continue;
            }
            features0(r, n, m, stamp, xs);
            y[s] = part_ids[n] == part_ids[m] ? 1.0f : 0.0f;
            if (partner) partner[s] = m;
        }
    }
    free(stamp);
    return ORC_OK;
}

/* float -> bfloat16 -> float with round-to-nearest-even on the dropped 16 bits. */
static double round_bf16(float f) {
    uint32_t u;
    memcpy(&u, &f, sizeof(u));
    u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
    float r;
    memcpy(&r, &u, sizeof(r));
    return (double)r;
}

/*
 * One training step of the learned order's network, in double precision:
 * parameters p (float32 master copy; layout W1[j][i] at 8 j + i, then b1,
 * W2, b2 -- 641 values) are rounded to bfloat16 for the forward pass; the
 * loss is the mean over samples with label >= 0 of the logistic loss
 * log(1 + e^s) - y s; its gradient is taken by backpropagation (ReLU
 * derivative 1 where the pre-activation is > 0) and applied to the master
 * copy with Adam (Kingma and Ba, 2015) at step t >= 1:
 *   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
 *   p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
 */
int oracle_train_step(const float *p, const float *x, const float *y, int64_t count, double lr,
                      double beta1, double beta2, double eps, int32_t t, const double *m_in,
                      const double *v_in, double *grad, double *loss, double *p_out,
                      double *m_out, double *v_out) {
    if (count < 0 || t < 1) return ORC_INVALID;
    double W1[OMLP_HID][OMLP_IN], B1[OMLP_HID], W2[OMLP_HID], B2;
    for (int j = 0; j < OMLP_HID; ++j) {
        for (int i = 0; i < OMLP_IN; ++i) W1[j][i] = round_bf16(p[j * OMLP_IN + i]);
        B1[j] = round_bf16(p[512 + j]);
        W2[j] = round_bf16(p[576 + j]);
    }
    B2 = round_bf16(p[640]);
    for (int q = 0; q < OMLP_PARAMS; ++q) grad[q] = 0.0;
    double total = 0.0;
    int64_t valid = 0;
    for (int64_t s = 0; s < count; ++s) {
        if (y[s] < 0.0f) continue;
        const float *xs = x + s * OMLP_IN;
        double a[OMLP_HID], h[OMLP_HID], out = B2;
        for (int j = 0; j < OMLP_HID; ++j) {
            a[j] = B1[j];
            for (int i = 0; i < OMLP_IN; ++i) a[j] += W1[j][i] * (double)xs[i];
            h[j] = a[j] > 0.0 ? a[j] : 0.0;
            out += W2[j] * h[j];
        }
        double yy = (double)y[s];
        total += (out > 0.0 ? out : 0.0) - out * yy + log1p(exp(-fabs(out)));
        double ds = 1.0 / (1.0 + exp(-out)) - yy;
        for (int j = 0; j < OMLP_HID; ++j) {
            grad[576 + j] += ds * h[j];
            double da = a[j] > 0.0 ? ds * W2[j] : 0.0;
            for (int i = 0; i < OMLP_IN; ++i) grad[j * OMLP_IN + i] += da * (double)xs[i];
            grad[512 + j] += da;
        }
        grad[640] += ds;
        valid++;
    }
    if (valid > 0) {
        for (int q = 0; q < OMLP_PARAMS; ++q) grad[q] /= (double)valid;
        total /= (double)valid;
    }
    *loss = total;
    double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
    for (int q = 0; q < OMLP_PARAMS; ++q) {
        m_out[q] = beta1 * m_in[q] + (1.0 - beta1) * grad[q];
        v_out[q] = beta2 * v_in[q] + (1.0 - beta2) * grad[q] * grad[q];
        p_out[q] = (double)p[q] - lr * (m_out[q] / c1) / (sqrt(v_out[q] / c2) + eps);
    }
    return ORC_OK;
}

uint64_t oracle_splitmix64_at(uint64_t seed, uint64_t i) { return splitmix64_at(seed, i); }

/* Learned-order candidate of the listed level-0 nodes only (pair[t], score[t],
 * key[t] belong to nodes[t]). */
int orun_score0_learned_nodes(const orun *r, int64_t omega, int64_t delta, const uint16_t *w1,
                              const uint16_t *b1, const uint16_t *w2, uint16_t b2, int32_t key_bits,
                              const int32_t *nodes, int32_t count, int32_t *pair, int32_t *score,
                              int32_t *key) {
    const olevel *g = &r->G[0];
    omodel M;
    int rc = model_from_bits(w1, b1, w2, b2, key_bits, &M);
    if (rc) return rc;
    for (int32_t t = 0; t < count; ++t) if (nodes[t] < 0 || nodes[t] >= g->V) return ORC_INVALID;
    int64_t *hist = (int64_t *)calloc((size_t)g->V, sizeof(int64_t));
    int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)g->V);
    int32_t *stamp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->E > 0 ? g->E : 1));
    if (!hist || !touched || !stamp) { free(hist); free(touched); free(stamp); return ORC_OOM; }
    for (int32_t e = 0; e < g->E; ++e) stamp[e] = -1;
    for (int32_t t = 0; t < count; ++t)
        score_node_learned(g, r->ew, omega, delta, &M, nodes[t], pair + t, score + t, key + t, hist,
                           touched, stamp);
    free(hist); free(touched); free(stamp);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Constraint-only baseline (the paper's one-pass comparison, Sec. V). */
/* ------------------------------------------------------------------ */
/*
 * Nodes are taken in id order and appended to the current part while both
 * bounds hold: w(part) + w(n) <= Omega and |in(part) u in(n)| <= Delta;
 * otherwise n opens the next part.  Reading: this is the paper's baseline
 * that fills partitions one at a time in node order, with no regard to
 * connectivity.  Parts are numbered in opening order.
 * Returns the number of parts (or a negative ORC_ code).
 */
int32_t orun_fill_baseline(const orun *r, int64_t omega, int64_t delta, int32_t *part_ids) {
    const olevel *g = &r->G[0];
    if (omega < 1 || delta < 0) return -ORC_INVALID;
    int32_t *stamp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->E > 0 ? g->E : 1));
    if (!stamp) return -ORC_OOM;
    for (int32_t e = 0; e < g->E; ++e) stamp[e] = -1;
    int32_t p = -1;
    int64_t w = 0, u = 0;
    for (int32_t n = 0; n < g->V; ++n) {
        if (g->w[n] > omega || g->noff[n + 1] - g->noff[n] > delta) { free(stamp); return -ORC_INFEASIBLE; }
        int64_t fresh = 0;
        if (p >= 0)
            for (int64_t j = g->noff[n]; j < g->noff[n + 1]; ++j) fresh += stamp[g->in[j]] != p;
        if (p < 0 || w + g->w[n] > omega || u + fresh > delta) {
            p++;
            w = 0;
            u = 0;
            fresh = g->noff[n + 1] - g->noff[n];
        }
        for (int64_t j = g->noff[n]; j < g->noff[n + 1]; ++j) stamp[g->in[j]] = p;
        w += g->w[n];
        u += fresh;
        part_ids[n] = p;
    }
    free(stamp);
    return p + 1;
}
