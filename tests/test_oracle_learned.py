"""Pins of the oracle's learned candidate order (an extension of Sec. III-A:
a small network's key ranks the candidates before Eq. (2)'s hist) and of its
training step, against closed forms, numpy evaluations, brute force over
Python sets, published generator values and finite differences.  CPU only.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from brute import conn, edges_of, in_sets, part_stats

LG_MAX_ERR = 0.0861      # max of log2(1 + t) - t on [0, 1] (at t = 1/ln 2 - 1)


def bf16_values(bits):
    return (np.asarray(bits, dtype=np.uint32) << 16).view(np.float32).astype(np.float64)


def np_score(model, x):
    """Network score in float64 from the decoded bfloat16 weights."""
    w1, b1, w2 = bf16_values(model.w1), bf16_values(model.b1), bf16_values(model.w2)
    b2 = bf16_values(np.array([model.b2]))[0]
    h = np.maximum(w1 @ np.asarray(x, np.float64) + b1, 0.0)
    return float(b2 + w2 @ h), float(abs(b2) + np.abs(w2) @ (np.abs(w1) @ np.abs(x) + np.abs(b1)))


def tiny_graph(n, m, kmax, seed):
    rng = np.random.default_rng(seed)
    off, pins = [0], []
    for _ in range(m):
        k = int(rng.integers(2, kmax + 1))
        pins += rng.choice(n, size=min(k, n), replace=False).tolist()
        off.append(len(pins))
    return synth.Hypergraph(n, np.array(off, np.int32), np.array(pins, np.int32))


# ------------------------------------------------------------- lg1p
def test_lg1p_exact_at_powers_of_two():
    for k in range(32):
        assert oracle.lg1p(2 ** k - 1) == float(k)


def test_lg1p_linear_mantissa_and_error_bound():
    assert oracle.lg1p(2) == 1.5                      # 1 + (3 - 2) / 2
    assert oracle.lg1p(5) == 2.5                      # 2 + (6 - 4) / 4
    rng = np.random.default_rng(0)
    xs = np.concatenate([np.arange(0, 5000), rng.integers(0, 2 ** 31 - 1, size=5000)])
    prev = None
    for x in sorted(set(int(v) for v in xs)):
        v = oracle.lg1p(x)
        d = math.log2(1 + x) - v
        assert -1e-6 <= d <= LG_MAX_ERR + 1e-6, x
        if prev is not None and x < 2 ** 24:
            assert v > prev                              # strictly increasing
        prev = v


# ------------------------------------------------------------- network
@pytest.mark.parametrize("seed", range(6))
def test_mlp_matches_float64_evaluation(seed):
    model = synth.random_model(seed, scale=0.5, key_bits=6)
    rng = np.random.default_rng(100 + seed)
    for _ in range(50):
        x = rng.uniform(0, 20, size=8).astype(np.float32)
        s, k = oracle.mlp(model, x)
        ref, mag = np_score(model, x.astype(np.float64))
        assert abs(s - ref) <= 1e-5 * mag + 1e-6
        q = ref * 64.0
        if abs(q - round(q)) > 1e-3 * max(1.0, mag):
            assert k == math.floor(q)


def test_mlp_closed_forms():
    z = synth.zero_model(8)
    assert oracle.mlp(z, np.arange(8, dtype=np.float32)) == (0.0, 0)
    m = synth.zero_model(4)
    m.w1[0, 0] = 0x3F80          # 1.0
    m.w2[0] = 0x4000             # 2.0
    m.b2 = 0xBF80                # -1.0
    s, k = oracle.mlp(m, np.array([3.25, 9, 9, 9, 9, 9, 9, 9], np.float32))
    assert s == 2 * 3.25 - 1 and k == math.floor(5.5 * 16)
    s, k = oracle.mlp(m, np.array([-3.0] + [0.0] * 7, np.float32))      # ReLU cuts it
    assert s == -1.0 and k == -16
    m.b2 = 0x7F80                # +inf -> clamped key
    assert oracle.mlp(m, np.zeros(8, np.float32))[1] == 2 ** 30


# ------------------------------------------------------------- features and pairs
def brute_features(g, n, m, ins, ew=None):
    eds = edges_of(g.offsets, g.pins)
    inc = [set() for _ in range(g.num_nodes)]
    for e, ed in enumerate(eds):
        for v in ed:
            inc[v].add(e)
    w = np.ones(g.num_nodes, np.int64) if g.node_weights is None else g.node_weights
    hist = sum(1 if ew is None else int(ew[e]) for e in inc[n] & inc[m])
    vals = [hist, len(ins[n] | ins[m]), min(len(inc[n]), len(inc[m])), max(len(inc[n]), len(inc[m])),
            min(len(ins[n]), len(ins[m])), max(len(ins[n]), len(ins[m])),
            min(int(w[n]), int(w[m])), max(int(w[n]), int(w[m]))]
    return hist, np.array([oracle.lg1p(v) for v in vals], np.float32)


@pytest.mark.parametrize("seed", range(4))
def test_features_against_sets(seed):
    g = tiny_graph(14, 12, 6, seed)
    ins = in_sets(g.num_nodes, g.offsets, g.pins)
    with oracle.Run.from_graph(g) as r:
        for n in range(g.num_nodes):
            for m in range(g.num_nodes):
                if m != n:
                    assert np.array_equal(r.features0(n, m), brute_features(g, n, m, ins)[1])


@pytest.mark.parametrize("seed", range(8))
def test_learned_pair_against_brute_force(seed):
    """pair(n) = the valid neighbour with the largest (key, hist, id)."""
    g = tiny_graph(16, 14, 7, seed)
    if seed % 2:
        g.node_weights = np.random.default_rng(seed).integers(1, 4, size=16).astype(np.int32)
    model = synth.random_model(seed, scale=0.7, key_bits=3)
    omega, delta = 5, 9
    ins = in_sets(g.num_nodes, g.offsets, g.pins)
    w = np.ones(16, np.int64) if g.node_weights is None else g.node_weights
    with oracle.Run.from_graph(g) as r:
        if any(w[n] > omega or len(ins[n]) > delta for n in range(16)):
            pytest.skip("infeasible draw")
        r.partition_learned(omega, delta, model)
        pair, key, score = r.array(0, oracle.A_PAIR), r.array(0, oracle.A_KEY), r.array(0, oracle.A_SCORE)
        for n in range(16):
            best = None
            for m in range(16):
                if m == n:
                    continue
                hist, x = brute_features(g, n, m, ins)
                if hist == 0 or w[n] + w[m] > omega or len(ins[n] | ins[m]) > delta:
                    continue
                k = oracle.mlp(model, x)[1]
                cand = (k, hist, m)
                best = cand if best is None or cand > best else best
            if best is None:
                assert pair[n] == -1
            else:
                assert (key[n], score[n], pair[n]) == best, n


def _traces_equal(r1, r2, arrays):
    assert r1.num_levels == r2.num_levels
    for l in range(r1.num_levels):
        for a in arrays:
            x, y = r1.array(l, a), r2.array(l, a)
            assert (x is None) == (y is None)
            if x is not None:
                assert np.array_equal(x, y), (l, a)


@pytest.mark.parametrize("make,omega,delta", [
    (lambda: synth.random_snn(300, 9, 3), 10, 40),
    (lambda: synth.random_snn(500, 12, 4, size_max=30), 16, 90),
    (lambda: synth.conv_snn(3, 5, 6, 4, 6, 1), 24, 200)])
def test_zero_model_reduces_to_the_plain_order(make, omega, delta):
    g = make()
    with oracle.Run.from_graph(g) as a, oracle.Run.from_graph(g) as b:
        ra = a.partition(omega, delta)
        rb = b.partition_learned(omega, delta, synth.zero_model(8))
        _traces_equal(a, b, [oracle.A_PAIR, oracle.A_SCORE, oracle.A_MATCH, oracle.A_GAMMA,
                             oracle.A_RHO_OUT])
    assert np.array_equal(ra.part_ids, rb.part_ids) and ra.cost == rb.cost


def test_hist_monotone_model_reduces_to_the_plain_order():
    """score = lg1p(hist) is strictly increasing in hist, and 2^20 resolution
    keeps it so after flooring: the order is the plain one."""
    m = synth.zero_model(20)
    m.w1[0, 0] = 0x3F80
    m.w2[0] = 0x3F80
    g = synth.random_snn(400, 10, 7)
    with oracle.Run.from_graph(g) as a, oracle.Run.from_graph(g) as b:
        ra = a.partition(12, 60)
        rb = b.partition_learned(12, 60, m)
        _traces_equal(a, b, [oracle.A_PAIR, oracle.A_SCORE, oracle.A_MATCH])
    assert np.array_equal(ra.part_ids, rb.part_ids)


@pytest.mark.parametrize("seed", range(4))
def test_learned_partition_invariants(seed):
    g = synth.random_snn(600, 10, 20 + seed, size_max=24)
    model = synth.random_model(seed, scale=0.5, key_bits=6)
    omega, delta = 20, 120
    with oracle.Run.from_graph(g) as r:
        res = r.partition_learned(omega, delta, model)
        for l in range(r.num_levels):
            pair = r.array(l, oracle.A_PAIR)
            if pair is None:
                continue
            key, score = r.array(l, oracle.A_KEY), r.array(l, oracle.A_SCORE)
            # pairing cycles are two-cycles: follow pair from every node
            for n in range(len(pair)):
                seen, x = set(), n
                while x >= 0 and x not in seen:
                    seen.add(x)
                    x = pair[x]
                if x >= 0:
                    assert pair[pair[x]] == x
            comp = (key + 2 ** 30) * 2 ** 32 + score
            m0 = oracle.match64(pair, comp, 0)
            assert np.array_equal(m0, oracle.match64(pair, comp, 1))
            assert np.array_equal(m0, r.array(l, oracle.A_MATCH))
            assert np.array_equal(m0[m0], np.arange(len(m0)))
    assert conn(g.offsets, g.pins, res.part_ids) == res.cost
    st = part_stats(g.num_nodes, g.offsets, g.pins, res.part_ids)
    assert all(w <= omega and d <= delta for w, d in st.values())
    assert sorted(st) == list(range(res.num_parts))
    assert [st[p][0] for p in range(res.num_parts)] == res.part_weight.tolist()
    assert [st[p][1] for p in range(res.num_parts)] == res.part_inbound.tolist()


# ------------------------------------------------------------- training data
def test_splitmix64_published_values():
    # first outputs of SplitMix64 seeded with 0
    assert oracle.splitmix64_at(0, 0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64_at(0, 1) == 0x6E789E6AA1B965F4
    assert oracle.splitmix64_at(0, 2) == 0x06C45D188009454F


def test_learn_samples_properties():
    g = synth.random_snn(400, 12, 5, size_max=20)
    ins = in_sets(g.num_nodes, g.offsets, g.pins)
    eds = edges_of(g.offsets, g.pins)
    part = (np.arange(g.num_nodes) * 7919 % 13).astype(np.int32)
    with oracle.Run.from_graph(g) as r:
        x, y, partner = r.learn_samples(part, 1234, 4)
        for s in range(len(y)):
            n = s // 4
            if y[s] < 0:
                assert partner[s] == -1
                continue
            m = partner[s]
            assert m != n and any(n in ed and m in ed for ed in eds)
            assert y[s] == float(part[n] == part[m])
            assert np.array_equal(x[s], brute_features(g, n, m, ins)[1])
        # neighbours are drawn by shared hyperedges: the chosen edge is I(n)[u0 mod |I(n)|]
        s = 9
        n = s // 4
        inc = sorted(e for e, ed in enumerate(eds) if n in ed)
        e = inc[oracle.splitmix64_at(1234, 2 * s) % len(inc)]
        m = eds[e][oracle.splitmix64_at(1234, 2 * s + 1) % len(eds[e])]
        assert partner[s] == (m if m != n else -1)


# ------------------------------------------------------------- training step
def np_loss(p, x, y):
    W1, b1, W2, b2 = p[:512].reshape(64, 8), p[512:576], p[576:640], p[640]
    v = y >= 0
    s = np.maximum(x[v] @ W1.T + b1, 0.0) @ W2 + b2
    return float(np.mean(np.maximum(s, 0) - s * y[v] + np.log1p(np.exp(-np.abs(s)))))


def bf16_exact_params(seed):
    p = synth.initial_params(seed).astype(np.float32)
    p[512:576] = np.random.default_rng(seed).normal(size=64) * 0.1
    p[640] = 0.3
    return ((p.view(np.uint32) >> 16) << 16).view(np.float32)          # exactly bfloat16


def test_train_step_gradient_by_finite_differences():
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 8, size=(64, 8)).astype(np.float32)
    y = rng.integers(0, 2, size=64).astype(np.float32)
    y[::7] = -1.0
    p = bf16_exact_params(1)
    z = np.zeros(oracle.N_PARAMS)
    out = oracle.train_step(p, x, y, 1e-3, 0.9, 0.999, 1e-8, 1, z, z)
    p64 = p.astype(np.float64)
    assert abs(out["loss"] - np_loss(p64, x.astype(np.float64), y)) < 1e-12
    for q in list(range(0, 512, 37)) + list(range(512, 641, 9)) + [640]:
        d = np.zeros_like(p64)
        d[q] = 1e-6
        fd = (np_loss(p64 + d, x.astype(np.float64), y) - np_loss(p64 - d, x.astype(np.float64), y)) / 2e-6
        assert abs(fd - out["grad"][q]) <= 1e-6 + 1e-5 * abs(fd), q


def test_train_step_closed_forms():
    x = np.random.default_rng(0).uniform(0, 4, size=(10, 8)).astype(np.float32)
    y = np.array([1, 0, 1, 1, -1, 0, 1, 0, 0, 1], np.float32)
    z = np.zeros(oracle.N_PARAMS)
    out = oracle.train_step(np.zeros(oracle.N_PARAMS, np.float32), x, y, 0.01, 0.9, 0.999, 1e-8, 1, z, z)
    v = y >= 0
    assert abs(out["loss"] - math.log(2)) < 1e-15                      # s = 0 everywhere
    assert abs(out["grad"][640] - np.mean(0.5 - y[v].astype(np.float64))) < 1e-15
    assert np.all(out["grad"][:640] == 0.0)                            # hidden units are all 0
    g = out["grad"][640]
    # Adam's first step: m_hat = g, v_hat = g^2
    assert abs(out["params"][640] - (-0.01 * g / (abs(g) + 1e-8))) < 1e-15
    assert np.all(out["params"][:640] == 0.0)
