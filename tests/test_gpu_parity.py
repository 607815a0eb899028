"""CUDA path vs the CPU oracle, through the C ABI.

Bit-exact on every integer output: per-level candidate, score, matching,
gamma, the partition entering and leaving each level's refinement, the
refinement counts, and the final part ids, cost, part weights and inbound
counts.
"""
import hashlib
import os

import numpy as np
import pytest

import oracle
import synth
from brute import conn, part_stats
from conftest import ROOT, read_golden

pytestmark = pytest.mark.gpu

hgp = pytest.importorskip("paper_2604_14411_gb300")
from paper_2604_14411_gb300 import hgp as H  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    hgp.load()


TRACE = [(H.HGP_LEVEL_PAIR, oracle.A_PAIR), (H.HGP_LEVEL_SCORE, oracle.A_SCORE),
         (H.HGP_LEVEL_MATCH, oracle.A_MATCH), (H.HGP_LEVEL_GAMMA, oracle.A_GAMMA),
         (H.HGP_LEVEL_RHO_IN, oracle.A_RHO_IN), (H.HGP_LEVEL_RHO_OUT, oracle.A_RHO_OUT)]


def compare(g, omega, delta, passes=1, debug=0, trace=True, incident=False, outbound=False,
            matching=0):
    with oracle.Run.from_graph(g, incident=incident, outbound=outbound) as r:
        want = r.partition(omega, delta, passes, matching=matching)
        with hgp.Graph.from_hypergraph(g, incident=incident, outbound=outbound) as G:
            got = G.partition(omega, delta, passes,
                              debug=(H.HGP_DEBUG_KEEP_LEVELS if trace else 0) | debug,
                              matching=matching)
            assert got.num_levels == r.num_levels
            if trace:
                for l in range(r.num_levels):
                    for hw, ow in TRACE:
                        a = G.level_array(l, hw)
                        b = r.array(l, ow)
                        assert (a is None) == (b is None), (l, hw)
                        if a is not None:
                            assert np.array_equal(a, b), f"level {l} array {hw} differs"
                    ref = G.level_array(l, H.HGP_LEVEL_REFINE)
                    assert tuple(ref.tolist()) == r.refine_stats(l), f"level {l} refinement"
                    a, b = G.level_array(l, H.HGP_LEVEL_GAIN_SEQ), r.array(l, oracle.A_GAIN_SEQ)
                    a = np.zeros(0, np.int64) if a is None else a
                    b = np.zeros(0, np.int64) if b is None else b
                    assert np.array_equal(a, b), f"level {l} in-sequence gains differ"
    assert np.array_equal(got.part_ids, want.part_ids)
    assert got.cost == want.cost
    assert got.num_parts == want.num_parts
    assert np.array_equal(got.part_weight, want.part_weight)
    assert np.array_equal(got.part_inbound, want.part_inbound)
    return got


def test_golden_six_node():
    gd = read_golden("six_node_example.txt")
    for case in ("A", "B"):
        with hgp.Graph(gd["num_nodes"][0], gd["offsets"], gd["pins"]) as G:
            res = G.partition(gd[f"{case}.omega"][0], gd[f"{case}.delta"][0],
                              debug=H.HGP_DEBUG_KEEP_LEVELS)
            assert G.level_array(0, H.HGP_LEVEL_PAIR).tolist() == gd[f"{case}.pair0"]
            assert G.level_array(0, H.HGP_LEVEL_SCORE).tolist() == gd[f"{case}.score0"]
            assert G.level_array(0, H.HGP_LEVEL_MATCH).tolist() == gd[f"{case}.match0"]
            assert G.level_array(0, H.HGP_LEVEL_GAMMA).tolist() == gd[f"{case}.gamma0"]
        assert res.part_ids.tolist() == gd[f"{case}.part_ids"]
        assert res.cost == gd[f"{case}.cost"][0]
        assert res.part_weight.tolist() == gd[f"{case}.part_weight"]
        assert res.part_inbound.tolist() == gd[f"{case}.part_inbound"]


@pytest.mark.parametrize("n,size,omega,delta,seed", [
    (64, 4, 4, 12, 0), (200, 6, 8, 20, 1), (300, 9, 6, 40, 2), (500, 12, 16, 60, 3),
    (777, 8, 10, 30, 4), (1000, 16, 32, 120, 5), (1200, 24, 40, 300, 6)])
def test_random_snn_bitexact(n, size, omega, delta, seed):
    compare(synth.random_snn(n, size, seed), omega, delta)


def test_snn_2k_bitexact():
    """2,048 neurons, edges of 32 pins, Omega 128, Delta 512."""
    compare(synth.snn_2k(0), 128, 512)


@pytest.mark.parametrize("seed", [0, 1])
def test_variable_size_edges(seed):
    compare(synth.random_snn(900, 8, seed, size_max=40), 24, 150)


def test_large_hyperedges_use_the_event_path():
    """Hyperedges above 256 pins route in-sequence gains through the sorted
    (edge, part) events instead of the per-hyperedge kernel."""
    compare(synth.random_snn(1500, 8, 12, size_max=300), 40, 2000)


def test_conv_style():
    compare(synth.conv_snn(4, 6, 8, 5, 8, 3), 48, 400)


def _weighted_graph():
    g = synth.random_snn(600, 10, 11)
    rng = np.random.default_rng(5)
    g.node_weights = rng.integers(1, 4, size=600).astype(np.int32)
    g.edge_weights = rng.integers(1, 7, size=g.num_edges).astype(np.int32)
    return g


def test_weighted():
    compare(_weighted_graph(), 30, 90)


@pytest.mark.parametrize("debug", [H.HGP_DEBUG_FORCE_GLOBAL, H.HGP_DEBUG_NO_BITMAP,
                                   H.HGP_DEBUG_FORCE_GLOBAL | H.HGP_DEBUG_NO_BITMAP,
                                   H.HGP_DEBUG_FORCE_CLUSTER,
                                   H.HGP_DEBUG_FORCE_CLUSTER | H.HGP_DEBUG_NO_BITMAP,
                                   H.HGP_DEBUG_REBUILD_INC, H.HGP_DEBUG_FORCE_WINDOW,
                                   H.HGP_DEBUG_FORCE_WINDOW | H.HGP_DEBUG_NO_BITMAP,
                                   H.HGP_DEBUG_FORCE_HASH_BUCKET,
                                   H.HGP_DEBUG_FORCE_HASH_BUCKET | H.HGP_DEBUG_NO_BITMAP])
def test_fallback_paths(debug):
    compare(synth.random_snn(700, 12, 8), 20, 80, debug=debug)


@pytest.mark.parametrize("make,omega,delta", [
    (lambda: synth.conv_snn(4, 6, 8, 5, 8, 3), 48, 400),
    (lambda: synth.conv_snn(6, 8, 8, 6, 12, 5), 64, 300),
    (lambda: synth.snn_2k(0), 128, 512)])
def test_window_buckets(make, omega, delta):
    """Per-node buckets (the path of levels too large for one CTA): one CTA
    takes a node's neighbour-id window in pieces of a quarter of the ids,
    from the top down, carrying the best valid candidate across pieces;
    layered graphs need one piece for most nodes, random ones up to four."""
    compare(make(), omega, delta, debug=H.HGP_DEBUG_FORCE_WINDOW)


@pytest.mark.parametrize("seed", [0, 1])
def test_window_pieces_weighted(seed):
    """Pieces with weighted hyperedges and nodes: ties and near-ties of hist
    across piece boundaries decide the pair by id."""
    g = synth.random_snn(800, 10, 30 + seed, size_max=30)
    rng = np.random.default_rng(seed)
    g.node_weights = rng.integers(1, 4, size=g.num_nodes).astype(np.int32)
    g.edge_weights = rng.integers(1, 4, size=g.num_edges).astype(np.int32)
    compare(g, 30, 120, debug=H.HGP_DEBUG_FORCE_WINDOW)


@pytest.mark.parametrize("make,omega,delta", [
    (lambda: synth.random_snn(1200, 16, 21), 24, 160),
    (lambda: synth.random_snn(900, 24, 4, size_max=40), 40, 300),
    (lambda: synth.conv_snn(6, 8, 8, 6, 12, 5), 64, 300),
    (lambda: synth.snn_2k(0), 128, 512)])
def test_hash_bucket(make, omega, delta):
    """The shared-memory hash bucket of large levels: nodes with few pin
    visits are scored by one CTA whose histogram is a hash table of packed
    (id, count) slots in shared memory, between the window bucket and the
    8-CTA cluster; the knob cuts the table to 1,024 slots so that all three
    buckets take nodes."""
    compare(make(), omega, delta, debug=H.HGP_DEBUG_FORCE_HASH_BUCKET)


@pytest.mark.parametrize("make,omega,delta,passes,incident", [
    (lambda: synth.snn_2k(0), 128, 512, 1, False),
    (lambda: synth.random_snn(1500, 8, 12, size_max=300), 40, 2000, 1, False),
    (lambda: synth.conv_snn(4, 6, 8, 5, 8, 3), 48, 400, 2, False),
    (_weighted_graph, 30, 90, 1, False),
    (lambda: synth.random_snn(600, 10, 3), 16, 60, 1, True)])
def test_rebuilt_incidence_levels(make, omega, delta, passes, incident):
    """Coarse levels whose I(n) is not kept (beyond the memory budget; forced
    here at every level) rebuild it from their pins for refinement: the
    whole trace stays bit-exact."""
    compare(make(), omega, delta, passes, debug=H.HGP_DEBUG_REBUILD_INC, incident=incident)


@pytest.mark.parametrize("make,omega,delta,cut", [
    (lambda: synth.random_snn(1200, 24, 6), 40, 300, 1),
    (lambda: synth.random_snn(1200, 24, 6), 40, 300, 3),
    (lambda: synth.snn_2k(0), 128, 512, 5),
    (lambda: synth.snn_16k(0), 1024, 4096, 1)])
def test_cut_partition_bitexact(make, omega, delta, cut):
    """Coarsening cut after `cut` matchings (hgp_options.max_levels; the
    oracle's bounded prefix of the method), the clusters of the last one
    becoming the parts: identical results.  The 16k case is the bench
    workload's CPU-baseline sample."""
    g = make()
    with oracle.Run.from_graph(g) as r:
        want = r.partition(omega, delta, 1, cut)
        assert r.num_levels == cut
    with hgp.Graph.from_hypergraph(g) as G:
        got = G.partition(omega, delta, max_levels=cut)
    assert got.num_levels == cut
    assert np.array_equal(got.part_ids, want.part_ids)
    assert got.cost == want.cost and got.num_parts == want.num_parts
    assert np.array_equal(got.part_weight, want.part_weight)
    assert np.array_equal(got.part_inbound, want.part_inbound)


def test_cluster_path_on_the_2k_snn():
    compare(synth.snn_2k(0), 128, 512, debug=H.HGP_DEBUG_FORCE_CLUSTER)


def test_multiple_passes():
    compare(synth.random_snn(800, 10, 9), 24, 100, passes=3)


def test_no_refinement():
    compare(synth.random_snn(800, 10, 9), 24, 100, passes=0)


def test_omega_one_and_unbounded():
    g = synth.random_snn(300, 9, 3)
    res = compare(g, 1, 10_000)
    assert res.num_parts == 300
    compare(synth.random_snn(400, 12, 4), 400, 400)


def test_no_edges_and_single_node():
    with hgp.Graph(5, np.array([0], np.int32), np.array([], np.int32)) as G:
        r = G.partition(2, 0)
    want = oracle.partition(synth.Hypergraph(5, np.array([0], np.int32), np.array([], np.int32)), 2, 0)
    assert np.array_equal(r.part_ids, want.part_ids) and r.cost == want.cost == 0
    with hgp.Graph(1, np.array([0, 1], np.int32), np.array([0], np.int32)) as G:
        r = G.partition(1, 0)
    assert r.part_ids.tolist() == [0] and r.cost == 0 and r.num_parts == 1


def test_infeasible_and_invalid():
    off = np.array([0, 2, 4, 6], np.int32)
    pins = np.array([0, 3, 1, 3, 2, 3], np.int32)
    with hgp.Graph(4, off, pins) as G:
        with pytest.raises(H.HgpError) as ei:
            G.partition(4, 2)
        assert ei.value.code == H.HGP_ERR_INFEASIBLE
        with pytest.raises(H.HgpError) as ei:
            G.partition(0, 2)
        assert ei.value.code == H.HGP_ERR_INVALID_ARG
    bad = [
        (np.array([0, 3, 3, 5], np.int32), np.array([0, 1, 2, 2, 3], np.int32), None, None),
        (np.array([0, 3, 5], np.int32), np.array([0, 1, 0, 2, 3], np.int32), None, None),
        (np.array([0, 3, 5], np.int32), np.array([0, 1, 4, 2, 3], np.int32), None, None),
        (np.array([0, 3, 5], np.int32), np.array([0, 1, 2, 2, 3], np.int32),
         np.array([1, 0, 1, 1], np.int32), None),
        (np.array([0, 3, 5], np.int32), np.array([0, 1, 2, 2, 3], np.int32), None,
         np.array([1, 0], np.int32)),
        (np.array([1, 3, 5], np.int32), np.array([0, 1, 2, 2, 3], np.int32), None, None),
    ]
    for off, pins, nw, ew in bad:
        with pytest.raises(H.HgpError) as ei:
            hgp.Graph(4, off, pins, nw, ew)
        assert ei.value.code == H.HGP_ERR_INVALID_ARG


def test_device_inputs_and_outputs():
    import torch
    g = synth.random_snn(1000, 12, 21)
    want = oracle.partition(g, 30, 100)
    dev = torch.device("cuda:0")
    t = lambda a: torch.from_numpy(np.asarray(a, np.int32)).to(dev)
    with hgp.Graph(g.num_nodes, t(g.offsets), t(g.pins)) as G:
        ids = torch.empty(g.num_nodes, dtype=torch.int32, device=dev)
        pw = torch.empty(g.num_nodes, dtype=torch.int64, device=dev)
        pin = torch.empty(g.num_nodes, dtype=torch.int32, device=dev)
        cost, npart, _ = G.partition_device(30, 100, ids, pw, pin)
        torch.cuda.synchronize()
    assert cost == want.cost and npart == want.num_parts
    assert np.array_equal(ids.cpu().numpy(), want.part_ids)
    assert np.array_equal(pw.cpu().numpy()[:npart], want.part_weight)
    assert np.array_equal(pin.cpu().numpy()[:npart], want.part_inbound)


def test_deterministic_and_reusable_handle():
    g = synth.random_snn(1500, 20, 2)
    with hgp.Graph.from_hypergraph(g) as G:
        a = G.partition(40, 200)
        b = G.partition(40, 200)
        c = G.partition(60, 260)
    assert np.array_equal(a.part_ids, b.part_ids) and a.cost == b.cost
    want = oracle.partition(g, 60, 260)
    assert np.array_equal(c.part_ids, want.part_ids) and c.cost == want.cost


def _digest(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


@pytest.mark.parametrize("name,make", [("snn4k", lambda: synth.random_snn(4096, 64, 0)),
                                       ("snn16k", lambda: synth.snn_16k(0))])
def test_stored_expected(name, make):
    """Workloads whose oracle run is too slow for the suite: compare with the
    values tests/golden/make_expected.py stored from the oracle."""
    path = os.path.join(ROOT, "tests", "golden", f"expected_{name}.txt")
    if not os.path.exists(path):
        pytest.skip(f"{path} not generated")
    exp = {}
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split(":", 1)
                exp[k.strip()] = v.strip()
    g = make()
    with hgp.Graph.from_hypergraph(g) as G:
        res = G.partition(int(exp["omega"]), int(exp["delta"]))
    assert res.cost == int(exp["cost"])
    assert res.num_parts == int(exp["num_parts"])
    assert res.num_levels == int(exp["num_levels"])
    assert _digest(res.part_ids.astype("<i4")) == exp["sha_part_ids"]
    stats = np.stack([res.part_weight.astype(np.int64), res.part_inbound.astype(np.int64)], axis=1)
    assert _digest(stats.astype("<i8")) == exp["sha_part_stats"]
    # properties that hold at any size, recounted independently
    assert conn(g.offsets, g.pins, res.part_ids) == res.cost
    st = part_stats(g.num_nodes, g.offsets, g.pins, res.part_ids)
    assert all(w <= int(exp["omega"]) and d <= int(exp["delta"]) for w, d in st.values())


@pytest.mark.parametrize("make,omega,delta", [
    (lambda: synth.random_snn(300, 9, 3), 10, 40),
    (lambda: synth.random_snn(2000, 16, 4, size_max=40), 64, 400),
    (_weighted_graph, 30, 90),
    (lambda: synth.conv_snn(4, 6, 8, 5, 8, 3), 48, 400),
    (lambda: synth.snn_16k(0), 1024, 4096)])
def test_fill_baseline_bitexact(make, omega, delta):
    """The constraint-only comparison (parts filled in node-id order), up to
    the bench workload at full size."""
    g = make()
    with oracle.Run.from_graph(g) as r:
        ids, k = r.fill_baseline(omega, delta)
    with hgp.Graph.from_hypergraph(g) as G:
        res = G.fill_baseline(omega, delta)
    assert np.array_equal(res.part_ids, ids) and res.num_parts == k
    assert res.cost == conn(g.offsets, g.pins, ids, g.edge_weights)
    st = part_stats(g.num_nodes, g.offsets, g.pins, ids, g.node_weights)
    assert [st[p][0] for p in range(k)] == res.part_weight.tolist()
    assert [st[p][1] for p in range(k)] == res.part_inbound.tolist()


@pytest.mark.parametrize("make,omega,delta", [
    (lambda: synth.random_snn(600, 10, 3), 16, 60),
    (lambda: synth.snn_2k(0), 128, 1024),
    (_weighted_graph, 30, 150),
    (lambda: synth.conv_snn(4, 6, 8, 5, 8, 3), 48, 600)])
def test_incident_mode_bitexact(make, omega, delta):
    """Delta counting every incident hyperedge (HGP_DELTA_INCIDENT)."""
    compare(make(), omega, delta, incident=True)


def test_incident_mode_learned_and_fill():
    g = synth.random_snn(900, 12, 5)
    model = synth.random_model(21, 0.5, 6)
    with oracle.Run.from_graph(g, incident=True) as r:
        want = r.partition_learned(20, 120, model)
        ids, k = r.fill_baseline(20, 120)
    with hgp.Graph.from_hypergraph(g, incident=True) as G:
        got = G.partition(20, 120, model=model)
        fill = G.fill_baseline(20, 120)
    assert np.array_equal(got.part_ids, want.part_ids) and got.cost == want.cost
    assert np.array_equal(got.part_inbound, want.part_inbound)
    assert np.array_equal(fill.part_ids, ids) and fill.num_parts == k


@pytest.mark.parametrize("make,omega,delta,passes", [
    (lambda: synth.random_snn(600, 10, 3), 16, 9, 1),
    (lambda: synth.snn_2k(0), 128, 40, 1),
    (_weighted_graph, 30, 12, 2),
    (lambda: synth.conv_snn(4, 6, 8, 5, 8, 3), 48, 30, 1),
    (lambda: synth.random_snn(1500, 8, 12, size_max=300), 40, 25, 1)])
def test_outbound_mode_bitexact(make, omega, delta, passes):
    """Delta counting the hyperedges sourced in a part (HGP_DELTA_OUTBOUND):
    level by level identical to the oracle, also on the event path of large
    hyperedges and with several passes."""
    compare(make(), omega, delta, passes, outbound=True)


def test_outbound_mode_learned_fill_and_rebuild():
    g = synth.random_snn(900, 12, 5)
    model = synth.random_model(22, 0.5, 6)
    with oracle.Run.from_graph(g, outbound=True) as r:
        want = r.partition_learned(20, 11, model)
        ids, k = r.fill_baseline(20, 11)
    with hgp.Graph.from_hypergraph(g, outbound=True) as G:
        got = G.partition(20, 11, model=model)
        fill = G.fill_baseline(20, 11)
    assert np.array_equal(got.part_ids, want.part_ids) and got.cost == want.cost
    assert np.array_equal(got.part_inbound, want.part_inbound)
    assert np.array_equal(fill.part_ids, ids) and fill.num_parts == k
    compare(g, 20, 11, debug=H.HGP_DEBUG_REBUILD_INC | H.HGP_DEBUG_FORCE_CLUSTER, outbound=True)
    with pytest.raises(H.HgpError) as ei:
        hgp.Graph.from_hypergraph(g, incident=True, outbound=True)
    assert ei.value.code == H.HGP_ERR_INVALID_ARG


@pytest.mark.parametrize("make,omega,delta,kw", [
    (lambda: synth.random_snn(300, 9, 3), 10, 40, {}),
    (lambda: synth.random_snn(1200, 24, 6), 40, 300, {}),
    (lambda: synth.snn_2k(0), 128, 512, {}),
    (_weighted_graph, 30, 90, {}),
    (lambda: synth.conv_snn(4, 6, 8, 5, 8, 3), 48, 400, {"debug": H.HGP_DEBUG_FORCE_CLUSTER}),
    (lambda: synth.random_snn(600, 10, 3), 16, 9, {"outbound": True}),
    (lambda: synth.random_snn(800, 10, 9), 24, 100, {"passes": 3})])
def test_exact_matching_bitexact(make, omega, delta, kw):
    """matching = 1: the exact maximum-weight matching of every level's
    pairing pseudo-forest (tree DP), identical level by level to the
    oracle's DP."""
    compare(make(), omega, delta, matching=1, **kw)


def test_exact_matching_on_the_16k_workload_and_its_weight():
    """The bench workload at full size: the GPU's DP matching equals the
    oracle's DP on the first level's candidates, and it never matches less
    score than the two walks."""
    g = synth.snn_16k(0)
    with hgp.Graph.from_hypergraph(g) as G:
        G.partition(1024, 4096, debug=H.HGP_DEBUG_KEEP_LEVELS, max_levels=1, matching=1)
        pair = G.level_array(0, H.HGP_LEVEL_PAIR).astype(np.int32)
        score = G.level_array(0, H.HGP_LEVEL_SCORE).astype(np.int32)
        got = G.level_array(0, H.HGP_LEVEL_MATCH).astype(np.int32)
    with oracle.Run.from_graph(g) as r:
        p0, s0 = r.score0(1024, 4096)
    assert np.array_equal(pair, p0) and np.array_equal(score, s0)
    assert np.array_equal(got, oracle.match(pair, score, 2))
    walks = oracle.match(pair, score, 0)
    w = lambda m: int(sum(score[n] for n in range(len(m)) if m[n] > n and pair[n] == m[n]) +
                      sum(score[m[n]] for n in range(len(m)) if m[n] > n and pair[n] != m[n]))
    assert w(got) >= w(walks)


def test_exact_matching_rejects_a_model():
    g = synth.random_snn(200, 8, 1)
    with hgp.Graph.from_hypergraph(g) as G:
        with pytest.raises(H.HgpError) as ei:
            G.partition(10, 60, matching=1, model=synth.random_model(1, 0.5, 6))
        assert ei.value.code == H.HGP_ERR_INVALID_ARG
