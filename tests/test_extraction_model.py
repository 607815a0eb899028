"""The order in which the GPU scorer visits candidates, restated in Python and
checked on the CPU against the oracle's Eq. (2) candidate (Sec. III-A).

The scorer does not walk candidates one by one in (hist desc, id desc) order.
It takes a node's neighbour ids in pieces of at most W ids from the top ids
down; within a piece it checks bands of hist values [bot, top] whose width
doubles after each band without a valid candidate, keeps the largest valid
(hist, id) key among the candidates that beat the best so far, stops a piece
as soon as the best's hist reaches the band's bottom, and carries the best
into the next piece, where only a larger hist can win (its ids are smaller).
The claim is that this always yields the first valid candidate of the
paper's order.  This test runs exactly that procedure on small graphs with
tight bounds (so that many candidates fail), for one piece, a few pieces and
many small ones, and compares every node's candidate and score with the
oracle's.  Validity is the paper's check restated on the level-0 sets:
w(n) + w(m) <= Omega and |in(n) u in(m)| <= Delta."""
import numpy as np
import pytest

import oracle
import synth


def _model_pair(n, hist, valid, V, W):
    best = 0                                       # key = hist << 32 | id; 0 = none yet
    wtop = V - 1
    while True:
        base = max(0, wtop - W + 1)
        piece = {i: int(hist[i]) for i in range(base, wtop + 1) if hist[i] > 0 and i != n}
        top, width = max(piece.values(), default=0), 1
        while top > (best >> 32):
            bot = max(1, top - width + 1)
            band = [(h << 32) | i for i, h in piece.items() if bot <= h <= top and ((h << 32) | i) > best]
            for key in band:                       # any order: the largest valid key is kept
                if key > best and valid(n, key & 0xffffffff):
                    best = key
            if (best >> 32) >= bot:
                break
            top = max((h for h in piece.values() if h < bot), default=0)
            width *= 2
        if base <= 0:
            break
        wtop -= W
    return (int(best & 0xffffffff), int(best >> 32)) if best else (-1, 0)


def _graph(kind, seed):
    if kind == "random":
        g = synth.random_snn(150, 6, seed, size_max=12)
    else:
        g = synth.conv_snn(3, 4, 4, 2, 4, seed)
    rng = np.random.default_rng(seed)
    g.node_weights = rng.integers(1, 4, size=g.num_nodes).astype(np.int32)
    g.edge_weights = rng.integers(1, 4, size=g.num_edges).astype(np.int32)
    return g


@pytest.mark.parametrize("kind,seed,omega,delta", [
    ("random", 1, 4, 14), ("random", 2, 5, 10), ("random", 3, 3, 18), ("conv", 4, 4, 40),
    ("conv", 5, 6, 25)])
@pytest.mark.parametrize("pieces", [1, 3, 17])
def test_piecewise_banded_extraction_equals_the_paper_order(kind, seed, omega, delta, pieces):
    g = _graph(kind, seed)
    V = g.num_nodes
    W = max(1, -(-V // pieces))
    with oracle.Run.from_graph(g) as r:
        want_pair, want_score = r.score0(omega, delta)
        w, _, _, _, _, in_off, inn = r.level_csr(0)
        ins = [set(inn[in_off[n]:in_off[n + 1]].tolist()) for n in range(V)]

        def valid(n, m):
            return int(w[n]) + int(w[m]) <= omega and len(ins[n] | ins[m]) <= delta

        failed = 0
        for n in range(V):
            hist = r.hist_row(0, n)
            got = _model_pair(n, hist, valid, V, W)
            assert got == (int(want_pair[n]), int(want_score[n])), (n, got)
            failed += int(want_pair[n] >= 0 and hist[want_pair[n]] < hist.max())
    assert failed > 0              # the bounds are tight enough that top candidates fail
