"""Learned candidate order on the GPU vs the CPU oracle, through the C ABI.

Scoring, matching and the whole level loop with a network-ranked candidate
order are bit-exact with the oracle (keys included) for seeded random
models; training pairs are bit-exact; a training step agrees with the
oracle's double-precision gradient and Adam update within float32 rounding.
Models fed to the oracle come from the seeded generator, never from a GPU
training run; a GPU-trained model is checked by recounted properties only.
"""
import numpy as np
import pytest

import oracle
import synth
from brute import conn, part_stats

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
         (H.HGP_LEVEL_KEY, oracle.A_KEY), (H.HGP_LEVEL_MATCH, oracle.A_MATCH),
         (H.HGP_LEVEL_GAMMA, oracle.A_GAMMA), (H.HGP_LEVEL_RHO_IN, oracle.A_RHO_IN),
         (H.HGP_LEVEL_RHO_OUT, oracle.A_RHO_OUT)]


def compare_learned(g, omega, delta, model, passes=1, debug=0):
    with oracle.Run.from_graph(g) as r:
        want = r.partition_learned(omega, delta, model, passes)
        with hgp.Graph.from_hypergraph(g) as G:
            got = G.partition(omega, delta, passes, debug=H.HGP_DEBUG_KEEP_LEVELS | debug, model=model)
            assert got.num_levels == r.num_levels
            for l in range(r.num_levels):
                for hw, ow in TRACE:
                    a, b = G.level_array(l, hw), r.array(l, ow)
                    assert (a is None) == (b is None), (l, hw)
                    if a is not None:
                        assert np.array_equal(a, b), f"level {l} array {hw} differs"
                assert tuple(G.level_array(l, H.HGP_LEVEL_REFINE).tolist()) == r.refine_stats(l)
                a, b = G.level_array(l, H.HGP_LEVEL_GAIN_SEQ), r.array(l, oracle.A_GAIN_SEQ)
                a = np.zeros(0, np.int64) if a is None else a
                b = np.zeros(0, np.int64) if b is None else b
                assert np.array_equal(a, b), f"level {l} in-sequence gains differ"
    assert np.array_equal(got.part_ids, want.part_ids)
    assert got.cost == want.cost and got.num_parts == want.num_parts
    assert np.array_equal(got.part_weight, want.part_weight)
    assert np.array_equal(got.part_inbound, want.part_inbound)
    return got


def _weighted():
    g = synth.random_snn(600, 10, 11)
    rng = np.random.default_rng(5)
    g.node_weights = rng.integers(1, 4, size=600).astype(np.int32)
    g.edge_weights = rng.integers(1, 7, size=g.num_edges).astype(np.int32)
    return g


@pytest.mark.parametrize("make,omega,delta,mseed,scale,kb", [
    (lambda: synth.random_snn(300, 9, 3), 10, 40, 0, 0.5, 6),
    (lambda: synth.random_snn(1000, 16, 5), 32, 120, 1, 0.3, 8),
    (lambda: synth.random_snn(900, 8, 1, size_max=40), 24, 150, 2, 1.0, 4),
    (_weighted, 30, 90, 3, 0.5, 6),
    (lambda: synth.conv_snn(4, 6, 8, 5, 8, 3), 48, 400, 4, 0.5, 6),
    (lambda: synth.snn_2k(0), 128, 512, 5, 0.4, 6)])
def test_learned_partition_bitexact(make, omega, delta, mseed, scale, kb):
    compare_learned(make(), omega, delta, synth.random_model(mseed, scale, kb))


def test_learned_hash_tables_and_no_refinement():
    g = synth.random_snn(700, 12, 8)
    compare_learned(g, 20, 80, synth.random_model(6, 0.5, 6), debug=H.HGP_DEBUG_FORCE_GLOBAL)
    compare_learned(g, 20, 80, synth.random_model(7, 0.5, 6), passes=0)


@pytest.mark.parametrize("make,omega,delta,mseed", [
    (lambda: synth.random_snn(700, 12, 8), 20, 80, 8),
    (lambda: synth.snn_2k(0), 128, 512, 9),
    (_weighted, 30, 90, 10)])
def test_learned_cluster_path(make, omega, delta, mseed):
    """The 8-CTA cluster scorer (packed 16-bit hist / inter in distributed
    shared memory), forced at every level."""
    compare_learned(make(), omega, delta, synth.random_model(mseed, 0.5, 6),
                    debug=H.HGP_DEBUG_FORCE_CLUSTER)


def test_zero_model_equals_the_plain_path():
    g = synth.random_snn(1200, 24, 6)
    with hgp.Graph.from_hypergraph(g) as G:
        a = G.partition(40, 300)
        b = G.partition(40, 300, model=synth.zero_model(8))
    assert np.array_equal(a.part_ids, b.part_ids) and a.cost == b.cost and a.num_levels == b.num_levels


def test_invalid_model_rejected():
    g = synth.random_snn(200, 8, 1)
    m = synth.random_model(0, 0.5, 21)
    with hgp.Graph.from_hypergraph(g) as G:
        with pytest.raises(H.HgpError) as ei:
            G.partition(10, 40, model=m)
    assert ei.value.code == H.HGP_ERR_INVALID_ARG


def test_learned_first_level_of_the_16k_workload_sampled():
    """Full size, the launch configuration of the bench: level-0 candidates and
    keys of 256 seeded nodes against the oracle, computed one node at a time."""
    g = synth.snn_16k(0)
    model = synth.random_model(11, 0.3, 6)
    with hgp.Graph.from_hypergraph(g) as G:
        G.partition(1024, 4096, 0, debug=H.HGP_DEBUG_KEEP_LEVELS, max_levels=1, model=model)
        pair, score, key = (G.level_array(0, w) for w in (H.HGP_LEVEL_PAIR, H.HGP_LEVEL_SCORE,
                                                           H.HGP_LEVEL_KEY))
        match = G.level_array(0, H.HGP_LEVEL_MATCH)
    nodes = np.random.default_rng(3).choice(g.num_nodes, size=256, replace=False).astype(np.int32)
    with oracle.Run.from_graph(g) as r:
        p, s, k = r.score0_learned_nodes(1024, 4096, model, nodes)
    assert np.array_equal(pair[nodes], p) and np.array_equal(score[nodes], s)
    assert np.array_equal(key[nodes], k)
    assert np.array_equal(match[match], np.arange(g.num_nodes))       # an involution
    comp = (key.astype(np.int64) + 2 ** 30) * 2 ** 32 + score
    assert np.array_equal(oracle.match64(pair, comp, 1), match)


# ------------------------------------------------------------- training
def _device(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.to("cuda") if dtype is None else t.to("cuda", dtype)


@pytest.mark.parametrize("weighted", [False, True])
def test_learn_samples_bitexact(weighted):
    g = synth.random_snn(2000, 16, 4, size_max=40)
    if weighted:
        rng = np.random.default_rng(1)
        g.node_weights = rng.integers(1, 5, size=2000).astype(np.int32)
        g.edge_weights = rng.integers(1, 9, size=g.num_edges).astype(np.int32)
    with oracle.Run.from_graph(g) as r:
        part = r.partition(64, 400).part_ids
        xo, yo, po = r.learn_samples(part, 77, 5)
    with hgp.Graph.from_hypergraph(g) as G:
        x, y, p = G.learn_samples(_device(part), 77, 5)
        import torch
        torch.cuda.synchronize()
    assert np.array_equal(x.cpu().numpy(), xo)
    assert np.array_equal(y.cpu().numpy(), yo)
    assert np.array_equal(p.cpu().numpy(), po)


def _samples():
    g = synth.random_snn(2000, 16, 9, size_max=48)
    with oracle.Run.from_graph(g) as r:
        part = r.partition(64, 400).part_ids
        return r.learn_samples(part, 5, 4)[:2]


def test_train_step_against_the_oracle():
    x, y = _samples()
    p0 = synth.initial_params(2)
    z = np.zeros(oracle.N_PARAMS)
    want = oracle.train_step(p0, x, y, 1e-2, 0.9, 0.999, 1e-8, 1, z, z)
    params = p0.copy()
    adam = np.zeros(2 * oracle.N_PARAMS, np.float32)
    loss = H.hgp_train_mlp(_device(x), _device(y), params, adam, 1, len(y), 1e-2)
    g_gpu = adam[:oracle.N_PARAMS].astype(np.float64) / (1 - 0.9)
    g_or = want["grad"]
    scale = np.abs(g_or).max()
    assert np.all(np.abs(g_gpu - g_or) <= 1e-4 * scale + 1e-3 * np.abs(g_or))
    assert abs(loss[0] - want["loss"]) <= 1e-5 * abs(want["loss"])
    # Adam's first step moves every parameter by lr * g / (|g| + eps): compare where |g| is not noise
    big = np.abs(g_or) > 1e-3 * scale
    dp_gpu = params.astype(np.float64) - p0
    dp_or = want["params"] - p0.astype(np.float64)
    assert np.all(np.abs(dp_gpu[big] - dp_or[big]) <= 1e-4 * 1e-2 + 1e-3 * np.abs(dp_or[big]))
    assert np.all(np.abs(dp_gpu) <= 1e-2 * 1.0001)


def test_training_is_deterministic_and_learns():
    x, y = _samples()
    runs = []
    for _ in range(2):
        params = synth.initial_params(4)
        adam = np.zeros(2 * oracle.N_PARAMS, np.float32)
        loss = H.hgp_train_mlp(_device(x), _device(y), params, adam, 300, 1024, 3e-3)
        runs.append((params, loss))
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    loss = runs[0][1]
    assert loss[-50:].mean() < 0.9 * loss[:10].mean()


def test_trained_model_partitions_are_feasible():
    graphs = [synth.random_snn(3000, 24, 100 + i, size_max=48) for i in range(2)]
    model, losses = H.train_model(graphs, 96, 600, seed=1, per_node=8, steps=300, batch=2048)
    g = synth.random_snn(3000, 24, 7, size_max=48)
    with hgp.Graph.from_hypergraph(g) as G:
        res = G.partition(96, 600, model=model)
        plain = G.partition(96, 600)
    assert conn(g.offsets, g.pins, res.part_ids) == res.cost
    st = part_stats(g.num_nodes, g.offsets, g.pins, res.part_ids)
    assert all(w <= 96 and d <= 600 for w, d in st.values())
    assert sorted(st) == list(range(res.num_parts))
    assert [st[p][1] for p in range(res.num_parts)] == res.part_inbound.tolist()
    assert plain.cost > 0 and res.cost > 0


def _tol(s):
    """Score tolerance of the tensor-core mode: 1e-2 relative, at least 1e-2
    absolute (a key step at key_bits = 6 is 1/64)."""
    return 1e-2 * max(1.0, abs(s))


@pytest.mark.parametrize("seed,scale", [(31, 0.5), (32, 1.0), (33, 0.25)])
def test_tensor_core_scores_within_tolerance(seed, scale):
    """learned_eval = 1: the network's hidden layer on tensor cores (TF32
    inputs, float32 accumulation).  With key_bits = 20 a key carries its
    score to 2^-20.  On every first-level node: a node with no valid
    neighbour has none either way (the checks are exact); otherwise the
    chosen neighbour is valid, its tensor-core score matches the float32
    oracle's score of the same pair within the tolerance, and that float32
    score is within the tolerance of the best the float32 order finds."""
    from brute import in_sets
    g = synth.random_snn(1200, 20, seed)
    omega, delta = 40, 240
    model = synth.random_model(seed, scale, 20)
    with hgp.Graph.from_hypergraph(g) as G:
        G.partition(omega, delta, 0, debug=H.HGP_DEBUG_KEEP_LEVELS, max_levels=1, model=model,
                    learned_eval=1)
        pair = G.level_array(0, H.HGP_LEVEL_PAIR)
        key = G.level_array(0, H.HGP_LEVEL_KEY)
    ins = in_sets(g.num_nodes, g.offsets, g.pins)
    checked = 0
    with oracle.Run.from_graph(g) as r:
        rp, _, rk = r.score0_learned_nodes(omega, delta, model, np.arange(g.num_nodes))
        for n in range(g.num_nodes):
            m = int(pair[n])
            if rp[n] < 0:
                assert m == -1
                continue
            assert m >= 0 and m != n
            assert 2 <= omega and len(ins[n] | ins[m]) <= delta
            s_ref, _ = oracle.mlp(model, r.features0(n, m))
            s_tc = key[n] / 2.0 ** 20
            assert abs(s_tc - s_ref) <= _tol(s_ref) + 2.0 ** -19, (n, m, s_tc, s_ref)
            s_best = rk[n] / 2.0 ** 20
            assert s_ref >= s_best - 2 * _tol(s_best) - 2.0 ** -19, (n, s_ref, s_best)
            checked += 1
    assert checked > g.num_nodes // 2


def test_tensor_core_partitions_are_feasible():
    """Whole partitions with the tensor-core evaluation, dense and cluster
    scorers: feasible, cost recounted, and close to the FMA-chain order's."""
    g = synth.random_snn(3000, 24, 7)
    omega, delta = 48, 300
    model = synth.random_model(5, 0.5, 6)
    for debug in (0, H.HGP_DEBUG_FORCE_CLUSTER):
        with hgp.Graph.from_hypergraph(g) as G:
            tc = G.partition(omega, delta, debug=debug, model=model, learned_eval=1)
            fma = G.partition(omega, delta, debug=debug, model=model)
        assert conn(g.offsets, g.pins, tc.part_ids) == tc.cost
        st = part_stats(g.num_nodes, g.offsets, g.pins, tc.part_ids)
        assert all(w <= omega and d <= delta for w, d in st.values())
        assert abs(tc.cost - fma.cost) <= 0.05 * fma.cost
    with hgp.Graph.from_hypergraph(g) as G:
        with pytest.raises(H.HgpError) as ei:
            G.partition(omega, delta, learned_eval=1)          # no model
        assert ei.value.code == H.HGP_ERR_INVALID_ARG
