"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the
hand-worked fixtures in tests/golden (derived from Sec. II-IV by hand),
incidence-matrix products, exhaustive enumeration, closed forms and the
invariants the paper proves (Sec. III-A).  CPU only.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth
from brute import (brute_opt, brute_opt_c, conn, edges_of, feasible, in_sets, incidence,
                   part_stats)
from conftest import read_golden


def tiny_random(n, m, kmax, seed):
    """m hyperedges over n nodes with random sources and sizes 1..kmax."""
    rng = np.random.default_rng(seed)
    off, pins = [0], []
    for _ in range(m):
        k = int(rng.integers(1, kmax + 1))
        ed = rng.choice(n, size=min(k, n), replace=False).tolist()
        pins += ed
        off.append(len(pins))
    return np.array(off, np.int32), np.array(pins, np.int32)


# ---------------------------------------------------------------- golden
def test_golden_six_node_case_a_and_b():
    g = read_golden("six_node_example.txt")
    off, pins, N = g["offsets"], g["pins"], g["num_nodes"][0]
    r = oracle.Run(N, off, pins)
    for n in (0, 2, 3, 5):
        assert r.hist_row(0, n).tolist() == g[f"hist_row_{n}"]
    for case in ("A", "B"):
        om, de = g[f"{case}.omega"][0], g[f"{case}.delta"][0]
        pair, score = r.score0(om, de)
        assert pair.tolist() == g[f"{case}.pair0"]
        assert score.tolist() == g[f"{case}.score0"]
        for method in (0, 1):
            assert oracle.match(pair, score, method).tolist() == g[f"{case}.match0"]
        res = r.partition(om, de)
        assert r.array(0, oracle.A_GAMMA).tolist() == g[f"{case}.gamma0"]
        assert [r.level_V(l) for l in range(r.num_levels)] == g[f"{case}.level_V"]
        assert res.part_ids.tolist() == g[f"{case}.part_ids"]
        assert res.cost == g[f"{case}.cost"][0]
        assert res.num_parts == g[f"{case}.num_parts"][0]
        assert res.part_weight.tolist() == g[f"{case}.part_weight"]
        assert res.part_inbound.tolist() == g[f"{case}.part_inbound"]
        if case == "A":
            w, poff, p, _, _, noff, inn = r.level_csr(1)
            assert w.tolist() == g["A.level1_w"]
            assert poff.tolist() == g["A.level1_pins_off"]
            assert p.tolist() == g["A.level1_pins"]
            assert noff.tolist() == g["A.level1_in_off"]
            assert inn.tolist() == g["A.level1_in"]
        else:
            assert r.array(0, oracle.A_MOVE_N).tolist() == g["B.level0_moves_n"]
            assert r.array(0, oracle.A_MOVE_PS).tolist() == g["B.level0_moves_ps"]
            assert r.array(0, oracle.A_MOVE_PD).tolist() == g["B.level0_moves_pd"]
            assert r.array(0, oracle.A_MOVE_GAIN).tolist() == g["B.level0_moves_gain"]
            assert r.array(0, oracle.A_GAIN_SEQ).tolist() == g["B.level0_gain_seq"]
            assert r.array(0, oracle.A_VIOL).tolist() == g["B.level0_viol"]
            assert r.refine_stats(0)[1] == g["B.level0_kstar"][0]


def test_golden_refine_pass():
    g = read_golden("refine_example.txt")
    r = oracle.Run(g["num_nodes"][0], g["offsets"], g["pins"])
    rho, t = r.refine0(g["rho_in"], g["K"][0], g["omega"][0], g["delta"][0])
    assert t["n"].tolist() == g["moves_n"]
    assert t["ps"].tolist() == g["moves_ps"]
    assert t["pd"].tolist() == g["moves_pd"]
    assert t["gain_iso"].tolist() == g["moves_gain"]
    assert t["gain_seq"].tolist() == g["gain_seq"]
    assert t["viol"].tolist() == g["viol"]
    assert t["kstar"] == g["kstar"][0] and t["gain"] == g["gain"][0]
    assert rho.tolist() == g["rho_out"]


# ---------------------------------------------------------------- Eq. (2)
@pytest.mark.parametrize("seed", range(4))
def test_hist_equals_incidence_product(seed):
    off, pins = tiny_random(40, 60, 9, seed)
    ew = np.random.default_rng(seed + 9).integers(1, 5, size=len(off) - 1).astype(np.int32)
    r = oracle.Run(40, off, pins, edge_weights=ew)
    B = incidence(40, off, pins)
    H = B.T @ np.diag(ew.astype(np.int64)) @ B          # H[n,m] = sum_e w(e)[n in e][m in e]
    np.fill_diagonal(H, 0)
    assert np.array_equal(H, H.T)                        # symmetry used in Sec. III-A
    for n in range(40):
        assert np.array_equal(r.hist_row(0, n), H[n])


@pytest.mark.parametrize("seed", range(4))
def test_pair_is_first_valid_in_hist_order(seed):
    N = 48
    off, pins = tiny_random(N, 70, 8, seed)
    nw = np.random.default_rng(seed).integers(1, 4, size=N).astype(np.int32)
    r = oracle.Run(N, off, pins, node_weights=nw)
    B = incidence(N, off, pins)
    H = B.T @ B
    np.fill_diagonal(H, 0)
    ins = in_sets(N, off, pins)
    om, de = 5, 9
    pair, score = r.score0(om, de)
    for n in range(N):
        valid = [m for m in range(N) if m != n and H[n, m] > 0 and nw[n] + nw[m] <= om
                 and len(ins[n] | ins[m]) <= de]
        if not valid:
            assert pair[n] == -1
            continue
        best = max(valid, key=lambda m: (H[n, m], m))
        assert pair[n] == best and score[n] == H[n, best]
    # Sec. III-A: pair(m) = n  =>  score(n) >= score(m); every cycle has length two.
    for m in range(N):
        if pair[m] >= 0:
            assert score[pair[m]] >= score[m]
            x, seen = m, set()
            while x not in seen:
                seen.add(x)
                x = pair[x]
            assert pair[pair[x]] == x


def test_score_of_sampled_nodes_matches_full_scoring():
    g = synth.random_snn(600, 12, 2)
    r = oracle.Run.from_graph(g)
    pair, score = r.score0(10, 60)
    nodes = np.array([5, 0, 599, 77, 300, 77], np.int32)
    p2, s2 = r.score0_nodes(10, 60, nodes)
    assert np.array_equal(p2, pair[nodes]) and np.array_equal(s2, score[nodes])


# ---------------------------------------------------------------- matching
def _check_matching(pair, score, match):
    V = len(pair)
    for n in range(V):
        m = match[n]
        assert match[m] == n                              # involution
        if m != n:
            assert pair[n] == m or pair[m] == n           # only pairing edges
        if pair[n] >= 0 and pair[pair[n]] == n:
            assert m == pair[n]                           # two-cycles are matched
        if pair[n] >= 0 and m == n:
            assert match[pair[n]] != pair[n]              # a free node's candidate is taken


@pytest.mark.parametrize("seed", range(6))
def test_matching_formulations_agree_on_scored_graphs(seed):
    N = 300
    g = synth.random_snn(N, 6, seed)
    r = oracle.Run.from_graph(g)
    for om, de in [(4, 40), (8, 12), (2, 1000)]:
        pair, score = r.score0(om, de)
        a = oracle.match(pair, score, 0)
        b = oracle.match(pair, score, 1)
        assert np.array_equal(a, b)
        _check_matching(pair, score, a)


def _random_forest(V, rng):
    """Random pairing graph with the structure Sec. III-A proves for scored
    graphs: a child c of x never beats x's own choice, i.e.
    (score(c), c) < (score(x), pair(x)); roots are two-cycles."""
    pair = -np.ones(V, np.int32)
    score = np.zeros(V, np.int32)
    order = rng.permutation(V)
    roots = max(1, V // 10)
    for i in range(0, 2 * roots, 2):
        a, b = order[i], order[i + 1]
        pair[a], pair[b] = b, a
        score[a] = score[b] = rng.integers(5, 9)
    for n in order[2 * roots:]:
        if rng.random() < 0.1:
            continue
        placed = [x for x in order if pair[x] >= 0]
        par = placed[rng.integers(len(placed))]
        s = int(rng.integers(0, score[par] + 1))
        if s == score[par] and n > pair[par]:
            if s == 0:
                continue
            s -= 1
        pair[n] = par
        score[n] = s
    return pair, score


def _forest_edges(pair, score):
    """Undirected edges {n, pair(n)} with weight score(n); a root two-cycle
    is one edge."""
    edges = {}
    for n, m in enumerate(pair.tolist()):
        if m >= 0:
            edges[(min(n, m), max(n, m))] = int(score[n])
    return edges


def _brute_max_matching(V, edges):
    """Largest total weight over all sets of vertex-disjoint edges."""
    items = list(edges.items())
    best = 0

    def rec(i, used, tot):
        nonlocal best
        if i == len(items):
            best = max(best, tot)
            return
        rec(i + 1, used, tot)
        (a, b), w = items[i]
        if not (used >> a) & 1 and not (used >> b) & 1:
            rec(i + 1, used | (1 << a) | (1 << b), tot + w)

    rec(0, 0, 0)
    return best


def _matched_weight(match, edges):
    tot = 0
    for n, m in enumerate(match.tolist()):
        assert match[m] == n                       # an involution
        if m > n:
            assert (n, m) in edges                 # along an edge of the pseudo-forest
            tot += edges[(n, m)]
    return tot


def _random_pseudo_forest(V, rng):
    """Trees hanging off root two-cycles (or lone nodes), arbitrary weights:
    the shape of a pairing graph without the score order of Sec. III-A."""
    pair = -np.ones(V, np.int32)
    score = np.zeros(V, np.int32)
    order = rng.permutation(V)
    k = 0
    while k + 1 < V and rng.random() < 0.7 or k == 0:
        a, b = order[k], order[k + 1]
        pair[a], pair[b] = b, a
        score[a] = score[b] = rng.integers(1, 10)
        k += 2
    for n in order[k:]:
        if rng.random() < 0.15:
            continue
        placed = [x for x in order if pair[x] >= 0]
        pair[n] = placed[rng.integers(len(placed))]
        score[n] = rng.integers(1, 10)
    return pair, score


@pytest.mark.parametrize("seed", range(40))
def test_dp_matching_is_a_maximum_weight_matching(seed):
    """The exact matching (oracle method 2) against brute force over every
    set of disjoint edges, on pseudo-forests of 10 to 14 nodes."""
    rng = np.random.default_rng(1000 + seed)
    V = 10 + seed % 5
    pair, score = (_random_forest if seed % 2 else _random_pseudo_forest)(V, rng)
    edges = _forest_edges(pair, score)
    m = oracle.match(pair, score, 2)
    assert _matched_weight(m, edges) == _brute_max_matching(V, edges)


@pytest.mark.parametrize("seed", range(6))
def test_dp_matching_never_below_the_two_walks(seed):
    """On real scored levels (Eq. (2) candidates of random SNNs) and on
    larger random forests: at least the two walks' matched weight."""
    rng = np.random.default_rng(2000 + seed)
    if seed < 3:
        g = synth.random_snn(400 + 200 * seed, 12, 80 + seed)
        with oracle.Run.from_graph(g) as r:
            pair, score = r.score0(24, 120)
    else:
        pair, score = _random_forest(300, rng)
    edges = _forest_edges(pair, score)
    w_dp = _matched_weight(oracle.match(pair, score, 2), edges)
    w_walks = _matched_weight(oracle.match(pair, score, 0), edges)
    assert w_dp >= w_walks


@pytest.mark.parametrize("seed", range(6))
def test_whole_method_with_dp_matching(seed):
    """matching = 1 (exact matching at every level): feasible results with
    recounted cost, never below the exhaustive optimum on <= 12 nodes; the
    first level's matching is the DP of the first level's candidates."""
    rng = np.random.default_rng(400 + seed)
    N = 10 + seed % 3
    off, pins = tiny_random(N, int(rng.integers(6, 13)), 5, 400 + seed)
    ins = in_sets(N, off, pins)
    omega, delta = int(rng.integers(2, 6)), max(len(x) for x in ins) + int(rng.integers(0, 3))
    opt, _ = brute_opt_c(N, off, pins, omega, delta)
    with oracle.Run(N, off, pins) as r:
        res = r.partition(omega, delta, matching=1)
        p0, s0 = r.array(0, oracle.A_PAIR), r.array(0, oracle.A_SCORE)
        assert np.array_equal(r.array(0, oracle.A_MATCH), oracle.match(p0, s0, 2))
    _check_result(off, pins, N, res, omega, delta)
    assert res.cost >= opt
    g = synth.random_snn(700, 12, 90 + seed)
    with oracle.Run.from_graph(g) as r:
        res = r.partition(24, 120, matching=1)
    _check_result(g.offsets, g.pins, g.num_nodes, res, 24, 120)


@pytest.mark.parametrize("seed", range(20))
def test_matching_formulations_agree_on_random_forests(seed):
    rng = np.random.default_rng(seed)
    pair, score = _random_forest(60, rng)
    a = oracle.match(pair, score, 0)
    assert np.array_equal(a, oracle.match(pair, score, 1))
    _check_matching(pair, score, a)


def test_matching_chain_alternates():
    # a path 0 -> 1 -> 2 -> 3 <-> 4 with every node its parent's favourite:
    # (3,4) root, 2 blocked, 1 matches 2, 0 single.
    pair = np.array([1, 2, 3, 4, 3], np.int32)
    score = np.array([1, 2, 3, 4, 4], np.int32)
    m = oracle.match(pair, score, 0)
    assert m.tolist() == [0, 2, 1, 4, 3]


def test_gamma_ranks_representatives():
    g, v2 = oracle.gamma(np.array([0, 3, 2, 1, 5, 4], np.int32))
    assert g.tolist() == [0, 1, 2, 1, 3, 3] and v2 == 4


# ---------------------------------------------------------------- contraction
@pytest.mark.parametrize("seed", range(4))
def test_contraction_conserves(seed):
    N = 200
    g = synth.random_snn(N, 7, seed)
    nw = np.random.default_rng(seed).integers(1, 3, size=N).astype(np.int32)
    r = oracle.Run(N, g.offsets, g.pins, node_weights=nw)
    pair, score = r.score0(6, 60)
    match = oracle.match(pair, score, 0)
    r.contract0(match)
    gam, V2 = oracle.gamma(match)
    w1, poff, p1, ioff, inc, noff, inn = r.level_csr(1)
    assert len(w1) == V2 and w1.sum() == nw.sum()
    for c in range(V2):
        assert w1[c] == nw[gam == c].sum()
    assert len(poff) == g.num_edges + 1
    ins = in_sets(N, g.offsets, g.pins)
    for e, ed in enumerate(edges_of(g.offsets, g.pins)):
        assert p1[poff[e]:poff[e + 1]].tolist() == sorted({int(gam[n]) for n in ed})
    for c in range(V2):
        want = set().union(*[ins[n] for n in np.nonzero(gam == c)[0]])
        assert inn[noff[c]:noff[c + 1]].tolist() == sorted(want)
        assert inc[ioff[c]:ioff[c + 1]].tolist() == [e for e in range(g.num_edges)
                                                     if c in set(p1[poff[e]:poff[e + 1]].tolist())]
    # Eq. (1) is invariant under projection: Conn_1(rho) = Conn_0(rho o gamma)
    rng = np.random.default_rng(seed)
    for _ in range(3):
        rho1 = rng.integers(0, 7, size=V2)
        assert conn(poff, p1, rho1) == conn(g.offsets, g.pins, rho1[gam])


# ---------------------------------------------------------------- refinement
def _brute_proposals(N, off, pins, rho, K, omega, nw=None):
    """Eq. (3) by its meaning: gain = Conn drop when n alone moves to p."""
    base = conn(off, pins, rho)
    size = np.zeros(K, np.int64)
    for n in range(N):
        size[rho[n]] += 1 if nw is None else nw[n]
    props = []
    for n in range(N):
        best = None
        for p in range(K):
            if p == rho[n] or size[p] + (1 if nw is None else nw[n]) > omega:
                continue
            r2 = rho.copy()
            r2[n] = p
            gain = base - conn(off, pins, r2)
            if best is None or gain > best[1]:
                best = (p, gain)
        if best and best[1] > 0:
            props.append((n, int(rho[n]), best[0], best[1]))
    props.sort(key=lambda t: (-t[3], t[0]))
    return props


@pytest.mark.parametrize("seed", range(8))
def test_refine_pass_against_recomputation(seed):
    N, K = 30, 6
    off, pins = tiny_random(N, 45, 6, seed)
    rng = np.random.default_rng(seed)
    rho0 = rng.integers(0, K, size=N).astype(np.int32)
    stats = part_stats(N, off, pins, rho0)
    omega = max(w for w, _ in stats.values()) + 2
    delta = max(d for _, d in stats.values()) + int(rng.integers(0, 3))
    r = oracle.Run(N, off, pins)
    rho, t = r.refine0(rho0, K, omega, delta)
    props = _brute_proposals(N, off, pins, rho0, K, omega)
    assert [(int(a), int(b), int(c), int(d)) for a, b, c, d in
            zip(t["n"], t["ps"], t["pd"], t["gain_iso"])] == props
    # in-sequence gains = exact Conn differences; violations = recount
    cur = rho0.copy()
    G, best = 0, (0, 0)
    for k in range(t["M"]):
        before = conn(off, pins, cur)
        cur[t["n"][k]] = t["pd"][k]
        assert t["gain_seq"][k] == before - conn(off, pins, cur)
        bad = sum(1 for w, d in part_stats(N, off, pins, cur).values() if w > omega or d > delta)
        assert t["viol"][k] == bad
        G += t["gain_seq"][k]
        if bad == 0 and G >= best[0]:
            best = (G, k + 1)
    kstar = best[1] if best[0] > 0 else 0
    assert t["kstar"] == kstar
    want = rho0.copy()
    for k in range(kstar):
        want[t["n"][k]] = t["pd"][k]
    assert np.array_equal(rho, want)
    assert conn(off, pins, rho0) - conn(off, pins, rho) == t["gain"]
    assert feasible(N, off, pins, rho, omega, delta)


# ---------------------------------------------------------------- whole method
def _check_result(g_off, g_pins, N, res, omega, delta, nw=None, ew=None):
    assert conn(g_off, g_pins, res.part_ids, ew) == res.cost
    st = part_stats(N, g_off, g_pins, res.part_ids, nw)
    assert sorted(st) == list(range(res.num_parts))
    assert [st[p][0] for p in range(res.num_parts)] == res.part_weight.tolist()
    assert [st[p][1] for p in range(res.num_parts)] == res.part_inbound.tolist()
    assert all(w <= omega and d <= delta for w, d in st.values())
    # compaction keeps old order: first occurrences of part ids are increasing? (ids dense)
    assert set(res.part_ids.tolist()) == set(range(res.num_parts))


@pytest.mark.parametrize("seed", range(12))
def test_whole_method_vs_exhaustive(seed):
    rng = np.random.default_rng(seed)
    N = int(rng.integers(5, 10))
    off, pins = tiny_random(N, int(rng.integers(3, 9)), 5, seed)
    omega = int(rng.integers(1, 5))
    ins = in_sets(N, off, pins)
    delta = int(rng.integers(0, 5))
    r = oracle.Run(N, off, pins)
    single_ok = all(len(s) <= delta for s in ins) and omega >= 1
    opt, nfeas = brute_opt(N, off, pins, omega, delta)
    assert (nfeas > 0) == single_ok                       # singletons decide feasibility
    if not single_ok:
        with pytest.raises(oracle.OracleError) as ei:
            r.partition(omega, delta)
        assert ei.value.code == oracle.INFEASIBLE
        return
    res = r.partition(omega, delta)
    _check_result(off, pins, N, res, omega, delta)
    assert res.cost >= opt


@pytest.mark.parametrize("seed", range(8))
def test_c_enumerator_agrees_with_python_enumerator(seed):
    """The C enumerator (with branch cuts) against the plain Python
    enumeration over every set partition, weighted and unweighted, both
    bound kinds."""
    rng = np.random.default_rng(900 + seed)
    N = int(rng.integers(4, 8))
    off, pins = tiny_random(N, int(rng.integers(2, 8)), 4, 900 + seed)
    nw = rng.integers(1, 3, size=N).astype(np.int32) if seed % 2 else None
    ew = rng.integers(1, 4, size=len(off) - 1).astype(np.int32) if seed % 2 else None
    omega, delta = int(rng.integers(1, 6)), int(rng.integers(0, 5))
    assert brute_opt_c(N, off, pins, omega, delta, nw, ew) == brute_opt(N, off, pins, omega, delta, nw, ew)
    # incident count: in(n) replaced by every hyperedge holding n
    best, nfeas = None, 0
    inc = [set(e for e, ed in enumerate(edges_of(off, pins)) if n in ed) for n in range(N)]
    import brute
    for rho in brute.set_partitions(N):
        st = {}
        for n in range(N):
            w, d = st.get(rho[n], (0, set()))
            st[rho[n]] = (w + (1 if nw is None else int(nw[n])), d | inc[n])
        if all(w <= omega and len(d) <= delta for w, d in st.values()):
            nfeas += 1
            c = conn(off, pins, rho, ew)
            best = c if best is None or c < best else best
    assert brute_opt_c(N, off, pins, omega, delta, nw, ew, incident=True) == (best, nfeas)
    # outbound count: every hyperedge sourced in the part
    best, nfeas = None, 0
    outs = [set(e for e, ed in enumerate(edges_of(off, pins)) if ed[0] == n) for n in range(N)]
    for rho in brute.set_partitions(N):
        st = {}
        for n in range(N):
            w, d = st.get(rho[n], (0, set()))
            st[rho[n]] = (w + (1 if nw is None else int(nw[n])), d | outs[n])
        if all(w <= omega and len(d) <= delta for w, d in st.values()):
            nfeas += 1
            c = conn(off, pins, rho, ew)
            best = c if best is None or c < best else best
    assert brute_opt_c(N, off, pins, omega, delta, nw, ew, outbound=True) == (best, nfeas)


@pytest.mark.parametrize("seed", range(12))
def test_whole_method_vs_exhaustive_up_to_12_nodes(seed):
    """10 to 12 nodes (Bell(12) = 4,213,597 set partitions): the oracle's
    result is feasible, its recounted cost is never below the optimum, and a
    partition exists exactly when every node alone fits both bounds."""
    rng = np.random.default_rng(300 + seed)
    N = 10 + seed % 3
    off, pins = tiny_random(N, int(rng.integers(6, 13)), 5, 300 + seed)
    nw = rng.integers(1, 3, size=N).astype(np.int32) if seed % 4 == 3 else None
    ew = rng.integers(1, 4, size=len(off) - 1).astype(np.int32) if seed % 4 == 3 else None
    ins = in_sets(N, off, pins)
    omega = int(rng.integers(2, 6))
    top = max(len(s) for s in ins)
    delta = top + int(rng.integers(0, 4)) if seed % 6 != 5 else top - 1
    single_ok = all(len(s) <= delta for s in ins) and (nw is None or int(nw.max()) <= omega)
    opt, nfeas = brute_opt_c(N, off, pins, omega, delta, nw, ew)
    assert (nfeas > 0) == single_ok
    r = oracle.Run(N, off, pins, nw, ew)
    if not single_ok:
        with pytest.raises(oracle.OracleError) as ei:
            r.partition(omega, delta)
        assert ei.value.code == oracle.INFEASIBLE
        return
    res = r.partition(omega, delta)
    _check_result(off, pins, N, res, omega, delta, nw, ew)
    assert res.cost >= opt


@pytest.mark.parametrize("seed", range(4))
def test_incident_mode_vs_exhaustive_up_to_12_nodes(seed):
    rng = np.random.default_rng(700 + seed)
    N = 11 + seed % 2
    off, pins = tiny_random(N, int(rng.integers(6, 11)), 4, 700 + seed)
    g = synth.Hypergraph(N, off, pins)
    omega = 4
    delta = max(len([e for e, ed in enumerate(edges_of(off, pins)) if n in ed]) for n in range(N)) + 1
    opt, nfeas = brute_opt_c(N, off, pins, omega, delta, incident=True)
    assert nfeas > 0
    with oracle.Run.from_graph(g, incident=True) as r:
        res = r.partition(omega, delta)
    st = _incident_stats(g, res.part_ids)
    assert all(w <= omega and d <= delta for w, d in st.values())
    assert conn(off, pins, res.part_ids) == res.cost >= opt


@pytest.mark.parametrize("seed", range(3))
def test_cut_prefix_of_the_method(seed):
    """max_levels bounds coarsening only: a cut at or beyond the natural level
    count changes nothing; a cut after k matchings starts refinement from the
    clusters of the k-th matching (gamma composed down the levels), and the
    result is feasible with its cost recounted from sets."""
    g = synth.random_snn(500 + 200 * seed, 12, 60 + seed)
    omega, delta = 24, 120
    with oracle.Run.from_graph(g) as r:
        full = r.partition(omega, delta)
        L = r.num_levels
        gam = [r.array(l, oracle.A_GAMMA) for l in range(L - 1)]
        same = r.partition(omega, delta, 1, L + 3)
        assert np.array_equal(same.part_ids, full.part_ids) and same.cost == full.cost
        for k in (1, 2, min(4, L)):
            res = r.partition(omega, delta, 1, k)
            assert r.num_levels == k and r.top_is_gamma
            top = r.array(k - 1, oracle.A_RHO_IN)
            assert np.array_equal(top, r.array(k - 1, oracle.A_GAMMA))
            # the levels below the cut are the uncut run's, and each one's
            # refinement starts from the coarser result projected by gamma
            for l in range(k - 1):
                assert np.array_equal(r.array(l, oracle.A_GAMMA), gam[l])
                assert np.array_equal(r.array(l, oracle.A_RHO_IN),
                                      r.array(l + 1, oracle.A_RHO_OUT)[gam[l]])
            _check_result(g.offsets, g.pins, g.num_nodes, res, omega, delta)


def _outbound_stats(g, rho):
    """{part: (weight, |{e : src(e) in part}|)} recounted with sets."""
    st = {}
    for n in range(g.num_nodes):
        p = int(rho[n])
        w, s = st.get(p, (0, set()))
        st[p] = (w + (1 if g.node_weights is None else int(g.node_weights[n])), s)
    for e, ed in enumerate(edges_of(g.offsets, g.pins)):
        st[int(rho[ed[0]])][1].add(e)
    return {p: (w, len(s)) for p, (w, s) in st.items()}


@pytest.mark.parametrize("seed", range(3))
def test_outbound_mode_recounts(seed):
    """Delta over the hyperedges sourced in a part: the result is feasible
    under that count and the reported per-part counts equal a set recount."""
    g = synth.random_snn(400 + 100 * seed, 10, 70 + seed, size_max=20)
    if seed == 2:
        rng = np.random.default_rng(3)
        g.node_weights = rng.integers(1, 3, size=g.num_nodes).astype(np.int32)
    omega, delta = 24, 9
    with oracle.Run.from_graph(g, outbound=True) as r:
        res = r.partition(omega, delta)
    st = _outbound_stats(g, res.part_ids)
    assert sorted(st) == list(range(res.num_parts))
    assert [st[p][1] for p in range(res.num_parts)] == res.part_inbound.tolist()
    assert all(w <= omega and d <= delta for w, d in st.values())
    assert conn(g.offsets, g.pins, res.part_ids) == res.cost
    # one hyperedge sourced per neuron: a part's outbound count is its node count
    if g.node_weights is None:
        assert res.part_inbound.tolist() == np.bincount(res.part_ids).tolist()


def test_outbound_mode_equals_inbound_when_delta_never_binds():
    g = synth.random_snn(500, 12, 8)
    a = oracle.partition(g, 20, 10 ** 6)
    with oracle.Run.from_graph(g, outbound=True) as r:
        b = r.partition(20, 10 ** 6)
    assert np.array_equal(a.part_ids, b.part_ids) and a.cost == b.cost


@pytest.mark.parametrize("seed", range(6))
def test_outbound_mode_vs_exhaustive_up_to_12_nodes(seed):
    rng = np.random.default_rng(800 + seed)
    N = 10 + seed % 3
    off, pins = tiny_random(N, int(rng.integers(6, 13)), 4, 800 + seed)
    g = synth.Hypergraph(N, off, pins)
    omega = int(rng.integers(3, 6))
    top = max(sum(1 for e in range(len(off) - 1) if pins[off[e]] == n) for n in range(N))
    delta = top + int(rng.integers(0, 3))
    opt, nfeas = brute_opt_c(N, off, pins, omega, delta, outbound=True)
    assert nfeas > 0
    with oracle.Run.from_graph(g, outbound=True) as r:
        res = r.partition(omega, delta)
    st = _outbound_stats(g, res.part_ids)
    assert all(w <= omega and d <= delta for w, d in st.values())
    assert conn(off, pins, res.part_ids) == res.cost >= opt
    # a node sourcing more than Delta hyperedges makes the input infeasible
    if top >= 1:
        with oracle.Run.from_graph(g, outbound=True) as r:
            with pytest.raises(oracle.OracleError) as ei:
                r.partition(omega, top - 1)
            assert ei.value.code == oracle.INFEASIBLE
        assert brute_opt_c(N, off, pins, omega, top - 1, outbound=True) == (None, 0)


def test_omega_one_closed_form():
    g = synth.random_snn(300, 9, 3)
    res = oracle.partition(g, 1, 10_000)
    assert res.num_parts == 300
    assert res.cost == sum(len(e) - 1 for e in edges_of(g.offsets, g.pins))
    assert sorted(res.part_ids.tolist()) == list(range(300))


def test_unbounded_connected_closed_form():
    g = synth.random_snn(500, 12, 4)
    res = oracle.partition(g, 500, g.num_edges)
    assert res.num_parts == 1 and res.cost == 0


def test_disjoint_components_closed_form():
    # 6 components of 8 nodes, each one hyperedge per node inside the component
    offs, pins = [0], []
    rng = np.random.default_rng(0)
    for c in range(6):
        base = 8 * c
        for i in range(8):
            tg = rng.choice([j for j in range(8) if j != i], size=3, replace=False)
            pins += [base + i] + sorted((base + tg).tolist())
            offs.append(len(pins))
    off, p = np.array(offs, np.int32), np.array(pins, np.int32)
    r = oracle.Run(48, off, p)
    res = r.partition(8, 1000)
    assert res.num_parts == 6 and res.cost == 0
    for c in range(6):
        assert len(set(res.part_ids[8 * c:8 * c + 8].tolist())) == 1


def test_c1_result_feasible_and_recounted():
    g = synth.snn_2k()
    with oracle.Run.from_graph(g) as r:
        res = r.partition(128, 512)
        _check_result(g.offsets, g.pins, g.num_nodes, res, 128, 512)
        # refinement never raises Eq. (1) and every level's partition is valid
        for l in range(r.num_levels):
            w, poff, p, _, _, noff, inn = r.level_csr(l)
            ri, ro = r.array(l, oracle.A_RHO_IN), r.array(l, oracle.A_RHO_OUT)
            assert conn(poff, p, ro) <= conn(poff, p, ri)
            assert conn(poff, p, ri) - conn(poff, p, ro) == r.refine_stats(l)[2]
        res2 = r.partition(128, 512)
        assert np.array_equal(res.part_ids, res2.part_ids) and res.cost == res2.cost


def test_weighted_result_feasible():
    g = synth.random_snn(400, 10, 5)
    rng = np.random.default_rng(1)
    nw = rng.integers(1, 4, size=400).astype(np.int32)
    ew = rng.integers(1, 6, size=g.num_edges).astype(np.int32)
    r = oracle.Run(400, g.offsets, g.pins, nw, ew)
    res = r.partition(20, 60)
    _check_result(g.offsets, g.pins, 400, res, 20, 60, nw, ew)


@pytest.mark.parametrize("bad", ["empty_edge", "dup_pin", "range", "zero_w", "zero_ew"])
def test_invalid_inputs_rejected(bad):
    off = np.array([0, 3, 5], np.int32)
    pins = np.array([0, 1, 2, 2, 3], np.int32)
    nw = ew = None
    N = 4
    if bad == "empty_edge":
        off = np.array([0, 3, 3, 5], np.int32)
    elif bad == "dup_pin":
        pins = np.array([0, 1, 0, 2, 3], np.int32)
    elif bad == "range":
        pins = np.array([0, 1, 4, 2, 3], np.int32)
    elif bad == "zero_w":
        nw = np.array([1, 0, 1, 1], np.int32)
    elif bad == "zero_ew":
        ew = np.array([1, 0], np.int32)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.Run(N, off, pins, nw, ew)
    assert ei.value.code == oracle.INVALID


def test_infeasible_singleton():
    off = np.array([0, 2, 4, 6], np.int32)
    pins = np.array([0, 3, 1, 3, 2, 3], np.int32)        # in(3) has 3 edges
    r = oracle.Run(4, off, pins)
    with pytest.raises(oracle.OracleError) as ei:
        r.partition(4, 2)
    assert ei.value.code == oracle.INFEASIBLE
    assert r.partition(4, 3).num_parts >= 1


# ---------------------------------------------------------------- fill baseline
@pytest.mark.parametrize("seed,omega,delta", [(0, 6, 30), (1, 10, 60), (2, 3, 200), (3, 50, 25)])
def test_fill_baseline_definition(seed, omega, delta):
    """Constraint-only baseline: parts are consecutive id ranges, each
    feasible, and each range's successor node would break a bound if added."""
    g = synth.random_snn(300, 8, seed, size_max=14)
    ins = in_sets(g.num_nodes, g.offsets, g.pins)
    if max(len(s) for s in ins) > delta:
        pytest.skip("a single node exceeds delta")
    with oracle.Run.from_graph(g) as r:
        ids, k = r.fill_baseline(omega, delta)
    assert ids[0] == 0 and np.all(np.diff(ids) >= 0) and np.all(np.diff(ids) <= 1)
    assert ids[-1] == k - 1
    st = part_stats(g.num_nodes, g.offsets, g.pins, ids)
    assert all(w <= omega and d <= delta for w, d in st.values())
    for p in range(k - 1):
        members = np.nonzero(ids == p)[0]
        nxt = members[-1] + 1
        u = set().union(*(ins[n] for n in members))
        assert len(members) + 1 > omega or len(u | ins[nxt]) > delta


def test_fill_baseline_weighted():
    """Node weights count towards Omega: every part respects it and each next
    part's first node would have broken a bound."""
    g = synth.random_snn(250, 8, 9, size_max=12)
    g.node_weights = np.random.default_rng(2).integers(1, 5, size=250).astype(np.int32)
    omega, delta = 12, 50
    ins = in_sets(g.num_nodes, g.offsets, g.pins)
    with oracle.Run.from_graph(g) as r:
        ids, k = r.fill_baseline(omega, delta)
    st = part_stats(g.num_nodes, g.offsets, g.pins, ids, g.node_weights)
    assert all(w <= omega and d <= delta for w, d in st.values())
    for p in range(k - 1):
        members = np.nonzero(ids == p)[0]
        nxt = members[-1] + 1
        u = set().union(*(ins[n] for n in members))
        assert int(g.node_weights[members].sum() + g.node_weights[nxt]) > omega or len(u | ins[nxt]) > delta


def test_fill_baseline_closed_forms():
    g = synth.random_snn(100, 5, 1)
    with oracle.Run.from_graph(g) as r:
        ids, k = r.fill_baseline(1, 10_000)          # every node alone
        assert k == 100 and ids.tolist() == list(range(100))
        ids, k = r.fill_baseline(100, 10_000)        # everything in one part
        assert k == 1 and not ids.any()
        ids, k = r.fill_baseline(7, 10_000)          # Omega alone decides: blocks of 7
        assert ids.tolist() == [n // 7 for n in range(100)]


# ---------------------------------------------------------------- incident Delta
def _incident_stats(g, rho):
    """{part: (node count, |union of I(n)|)} from Python sets."""
    eds = edges_of(g.offsets, g.pins)
    inc = [set() for _ in range(g.num_nodes)]
    for e, ed in enumerate(eds):
        for v in ed:
            inc[v].add(e)
    st = {}
    for n in range(g.num_nodes):
        w, s = st.get(int(rho[n]), (0, set()))
        st[int(rho[n])] = (w + 1, s | inc[n])
    return {p: (w, len(s)) for p, (w, s) in st.items()}


@pytest.mark.parametrize("seed", range(3))
def test_incident_mode_counts_every_incident_hyperedge(seed):
    g = synth.random_snn(400, 10, seed, size_max=16)
    omega, delta = 16, 60
    with oracle.Run.from_graph(g, incident=True) as r:
        res = r.partition(omega, delta)
    st = _incident_stats(g, res.part_ids)
    assert sorted(st) == list(range(res.num_parts))
    assert all(w <= omega and d <= delta for w, d in st.values())
    assert [st[p][1] for p in range(res.num_parts)] == res.part_inbound.tolist()
    assert conn(g.offsets, g.pins, res.part_ids) == res.cost


def test_incident_mode_equals_inbound_mode_when_delta_never_binds():
    g = synth.random_snn(500, 12, 4)
    a = oracle.partition(g, 20, 10 ** 6)
    with oracle.Run.from_graph(g, incident=True) as r:
        b = r.partition(20, 10 ** 6)
    assert np.array_equal(a.part_ids, b.part_ids) and a.cost == b.cost


@pytest.mark.parametrize("seed", range(6))
def test_incident_mode_exhaustive(seed):
    """Tiny graphs: feasible under the incident count, never below the optimum
    found by enumerating every set partition."""
    rng = np.random.default_rng(50 + seed)
    N = 7
    off, pins = [0], []
    for _ in range(5):
        k = int(rng.integers(2, 4))
        pins += rng.choice(N, size=k, replace=False).tolist()
        off.append(len(pins))
    g = synth.Hypergraph(N, np.array(off, np.int32), np.array(pins, np.int32))
    omega, delta = 3, 4
    # brute force over all set partitions with the incident-hyperedge count
    best = None
    for rho in __import__("brute").set_partitions(N):
        st = _incident_stats(g, np.array(rho))
        if all(w <= omega and d <= delta for w, d in st.values()):
            c = conn(g.offsets, g.pins, rho)
            best = c if best is None or c < best else best
    with oracle.Run.from_graph(g, incident=True) as r:
        if best is None:
            with pytest.raises(oracle.OracleError):
                r.partition(omega, delta)
            return
        try:
            res = r.partition(omega, delta)
        except oracle.OracleError:
            # only possible when a single node alone breaks the incident bound
            assert any(len([e for e, ed in enumerate(edges_of(g.offsets, g.pins)) if n in ed]) > delta
                       for n in range(N))
            return
    st = _incident_stats(g, res.part_ids)
    assert all(w <= omega and d <= delta for w, d in st.values())
    assert res.cost >= best
