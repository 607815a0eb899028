/*
 * Exhaustive optimum of the constrained partitioning problem (Sec. II-A) on
 * hypergraphs of at most 16 nodes and 64 hyperedges, for pinning the oracle.
 * Test infrastructure only; it shares nothing with the oracle or the library
 * and follows the problem definition alone:
 *   every part p must have  sum of w(n) over p <= omega  and
 *                           |union of in(n) over p| <= delta,
 *   cost = sum_e omega(e) * (distinct parts among the pins of e - 1)  (Eq. 1).
 * Every set partition of the nodes is visited once, as a restricted-growth
 * string (node i joins one of the parts opened by nodes 0..i-1, or opens the
 * next one).  A branch stops as soon as a part breaks a bound: adding nodes
 * to a part never lowers its weight or its inbound count, so no completion
 * of that branch is feasible.  Cost is kept incrementally per hyperedge as a
 * bit set of the parts holding its pins.
 */
#include <stdint.h>
#include <string.h>

#define BR_MAX_N 16
#define BR_MAX_E 64

typedef struct {
    int n, e;
    int64_t omega, delta;
    int32_t w[BR_MAX_N];
    uint64_t in_mask[BR_MAX_N];      /* bit e: e in in(n) */
    int32_t ew[BR_MAX_E];
    int32_t nedges_of[BR_MAX_N];
    int32_t edges_of[BR_MAX_N][BR_MAX_E];
    /* state */
    int64_t part_w[BR_MAX_N];
    uint64_t part_in[BR_MAX_N];
    uint32_t edge_parts[BR_MAX_E];
    int64_t cost;
    int64_t best;
    int64_t feasible;
} br_state;

static int popcount64(uint64_t x) {
    int c = 0;
    while (x) { x &= x - 1; ++c; }
    return c;
}

static void visit(br_state *s, int i, int parts) {
    if (i == s->n) {
        s->feasible++;
        if (s->best < 0 || s->cost < s->best) s->best = s->cost;
        return;
    }
    for (int v = 0; v <= parts && v < BR_MAX_N; ++v) {
        int64_t w_old = s->part_w[v];
        uint64_t in_old = s->part_in[v];
        int64_t nw = w_old + s->w[i];
        uint64_t nin = in_old | s->in_mask[i];
        if (nw > s->omega || popcount64(nin) > s->delta) continue;
        uint32_t saved[BR_MAX_E];
        int64_t cost_old = s->cost;
        for (int k = 0; k < s->nedges_of[i]; ++k) {
            int e = s->edges_of[i][k];
            saved[k] = s->edge_parts[e];
            if (!(s->edge_parts[e] & (1u << v))) {
                if (s->edge_parts[e]) s->cost += s->ew[e];
                s->edge_parts[e] |= 1u << v;
            }
        }
        s->part_w[v] = nw;
        s->part_in[v] = nin;
        visit(s, i + 1, v == parts ? parts + 1 : parts);
        s->part_w[v] = w_old;
        s->part_in[v] = in_old;
        for (int k = 0; k < s->nedges_of[i]; ++k) s->edge_parts[s->edges_of[i][k]] = saved[k];
        s->cost = cost_old;
    }
}

/*
 * offsets[E+1], pins[P]: CSR, first pin of each edge is its source.
 * node_weights / edge_weights may be NULL (unit).  mode chooses what the
 * second bound counts: 0 the hyperedges with a destination in the part
 * (inbound), 1 every hyperedge with a pin in it (incident), 2 the
 * hyperedges whose source is in it (outbound).
 * Writes the optimum cost to *best (-1 when no partition is feasible) and the
 * number of feasible partitions to *count.  Returns 0, or -1 on sizes beyond
 * 16 nodes / 64 edges.
 */
int brute_optimum(int32_t n, int32_t e, const int32_t *offsets, const int32_t *pins,
                  const int32_t *node_weights, const int32_t *edge_weights, int64_t omega,
                  int64_t delta, int32_t mode, int64_t *best, int64_t *count) {
    if (n < 1 || n > BR_MAX_N || e < 0 || e > BR_MAX_E) return -1;
    static br_state s;
    memset(&s, 0, sizeof(s));
    s.n = n;
    s.e = e;
    s.omega = omega;
    s.delta = delta;
    for (int i = 0; i < n; ++i) s.w[i] = node_weights ? node_weights[i] : 1;
    for (int k = 0; k < e; ++k) {
        s.ew[k] = edge_weights ? edge_weights[k] : 1;
        for (int j = offsets[k]; j < offsets[k + 1]; ++j) {
            int m = pins[j];
            if (m < 0 || m >= n) return -1;
            const int is_src = j == offsets[k];
            if (mode == 1 || (mode == 0 && !is_src) || (mode == 2 && is_src))
                s.in_mask[m] |= (uint64_t)1 << k;
            s.edges_of[m][s.nedges_of[m]++] = k;
        }
    }
    s.best = -1;
    visit(&s, 0, 0);
    *best = s.best;
    *count = s.feasible;
    return 0;
}
