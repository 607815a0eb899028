"""hgp_score_noalloc: the scoring entry point for callers that cannot allocate
device memory while they run (code inside another framework's allocator or
memory pool, runtimes that reserved all device memory up front).  Its only
scratch is a fixed library-owned device array, so it must give exactly the
first-level candidates and scores of the CPU oracle's Eq. (2) scoring with
the Omega/Delta checks, call after call, and refuse inputs whose scratch
would not fit.

Kept in a file of its own that sorts last, so a failure here comes after
every other test has run.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

hgp = pytest.importorskip("paper_2604_14411_gb300")
from paper_2604_14411_gb300 import hgp as H  # noqa: E402


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


def incidence(g):
    """I(n) and in(n) as CSR (ascending edge ids), built on the host."""
    N, E = g.num_nodes, g.num_edges
    off = g.offsets.astype(np.int64)
    pins = g.pins.astype(np.int64)
    eid = np.repeat(np.arange(E), np.diff(off))
    order = np.lexsort((eid, pins))
    inc = eid[order]
    ioff = np.concatenate([[0], np.cumsum(np.bincount(pins, minlength=N))])
    first = np.zeros(len(pins), bool)
    first[off[:-1]] = True
    dn, de = pins[~first], eid[~first]
    order = np.lexsort((de, dn))
    inn = de[order]
    noff = np.concatenate([[0], np.cumsum(np.bincount(dn, minlength=N))])
    return ioff, inc, noff, inn


def score_noalloc(torch, g, omega, delta):
    dev = torch.device("cuda:0")
    ioff, inc, noff, inn = incidence(g)
    nw = g.node_weights if g.node_weights is not None else np.ones(g.num_nodes, np.int32)
    ew = g.edge_weights if g.edge_weights is not None else np.ones(g.num_edges, np.int32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).to(dev)
    args = [t(g.offsets), t(g.pins), t(ioff), t(inc), t(noff), t(inn), t(nw), t(ew)]
    pair = torch.full((g.num_nodes,), -7, dtype=torch.int32, device=dev)
    score = torch.full((g.num_nodes,), -7, dtype=torch.int32, device=dev)
    lib = H.load()
    stream = torch.cuda.current_stream()
    rc = lib.hgp_score_noalloc(g.num_nodes, g.num_edges, *[a.data_ptr() for a in args],
                               int(omega), int(delta), pair.data_ptr(), score.data_ptr(),
                               ctypes.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    return rc, pair.cpu().numpy(), score.cpu().numpy()


def reference(g, omega, delta):
    """pair(n) and score(n) of every input node, from the CPU oracle."""
    with oracle.Run.from_graph(g) as r:
        return r.score0(omega, delta)


def _max_in(g):
    _, _, noff, _ = incidence(g)
    return int(np.diff(noff).max())


def _cases():
    a = synth.random_snn(2000, 32, 3)
    w = synth.random_snn(1500, 20, 4)
    rng = np.random.default_rng(2)
    w.node_weights = rng.integers(1, 4, size=1500).astype(np.int32)
    w.edge_weights = rng.integers(1, 5, size=w.num_edges).astype(np.int32)
    return [
        ("union counts on in() bitmaps", a, 8, _max_in(a) + 5),
        ("no union needed", synth.snn_2k(0), 128, 512),
        ("weighted", w, 12, _max_in(w) + 3),
    ]


@pytest.mark.parametrize("case", range(3))
def test_noalloc_matches_oracle_first_level_twice(torch_cuda, case):
    name, g, omega, delta = _cases()[case]
    want_pair, want_score = reference(g, omega, delta)
    for _ in range(2):          # the shared scratch keeps the previous call's bits
        rc, pair, score = score_noalloc(torch_cuda, g, omega, delta)
        assert rc == H.HGP_OK, (name, H.hgp_error_string(rc))
        assert np.array_equal(pair, want_pair), name
        assert np.array_equal(score, want_score), name


def test_noalloc_rejects_inputs_beyond_its_scratch(torch_cuda):
    g = synth.random_snn(16384, 16, 0)      # 16,384 rows of 2 KiB bitmaps > 16 MiB
    rc, pair, _ = score_noalloc(torch_cuda, g, 4, _max_in(g) + 1)
    assert rc == H.HGP_ERR_SCRATCH_LIMIT
    assert (pair == -7).all()               # nothing was launched
