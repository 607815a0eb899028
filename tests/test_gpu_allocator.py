"""The device-memory hook of hgp_create (hgp_allocator) and failure handling
that needs no GPU fault.

* Partitions drawn from PyTorch's caching allocator (TorchAllocator) are
  bit-exact with the CPU oracle, single and batched (the batch calls the
  callbacks from its worker threads), and every chunk handed out is returned.
* Out-of-memory handling: the allocator reports failure (NULL) at the k-th
  request, for every k of a whole create + partition; each call must return
  HGP_ERR_OOM and give back every chunk it already held, and the next call
  must succeed.
* A bounded device loop that runs out (HGP_DEBUG_SMALL_TABLE shrinks the
  scoring kernel's hash tables to 64 slots) returns HGP_ERR_DEVICE_LIMIT; the
  loop gives up after 64 probes, so nothing hangs, and the context stays
  usable.
"""
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
    H.load()
    return torch


def _same(got, want):
    assert np.array_equal(got.part_ids, want.part_ids)
    assert got.cost == want.cost and got.num_parts == want.num_parts
    assert np.array_equal(got.part_weight, want.part_weight)
    assert np.array_equal(got.part_inbound, want.part_inbound)


CASES = [(synth.random_snn(700, 24, 11), 24, 140), (synth.snn_2k(0), 128, 512)]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_torch_allocator_partition_is_bitexact_and_returns_every_chunk(torch_cuda, case):
    g, omega, delta = CASES[case]
    alloc = H.TorchAllocator()
    with hgp.Graph.from_hypergraph(g, allocator=alloc) as G:
        got = G.partition(omega, delta)
        assert alloc.allocs > 0
        assert alloc.live, "the handle keeps its level-0 arrays"
    torch_cuda.cuda.synchronize()
    assert alloc.live == {} and alloc.allocs == alloc.frees
    _same(got, oracle.partition(g, omega, delta))


def test_torch_allocator_batch_from_worker_threads(torch_cuda):
    inst = [synth.random_snn(300 + 90 * i, 16 + 2 * i, 40 + i) for i in range(6)]
    alloc = H.TorchAllocator()
    graphs = [hgp.Graph.from_hypergraph(g, allocator=alloc) for g in inst]
    try:
        res = H.hgp_partition_batch(graphs, [32] * 6, [200] * 6)
    finally:
        for G in graphs:
            G.close()
    torch_cuda.cuda.synchronize()
    assert alloc.live == {} and alloc.allocs == alloc.frees
    for g, r in zip(inst, res):
        _same(r, oracle.partition(g, 32, 200))


def test_allocation_failure_at_every_request_returns_oom_without_leaks(torch_cuda):
    g, omega, delta = synth.random_snn(400, 20, 5), 24, 150
    want = oracle.partition(g, omega, delta)
    probe = H.TorchAllocator()
    with hgp.Graph.from_hypergraph(g, allocator=probe) as G:
        G.partition(omega, delta)
    total = probe.allocs                  # requests of one whole create + partition
    assert total >= 3
    alloc = H.TorchAllocator()
    failed_in = {"create": 0, "partition": 0}
    for k in range(1, total + 1):
        alloc.fail_at = k
        try:
            G = hgp.Graph.from_hypergraph(g, allocator=alloc)
        except H.HgpError as e:
            assert e.code == H.HGP_ERR_OOM, e
            failed_in["create"] += 1
        else:
            with G:
                with pytest.raises(H.HgpError) as ei:
                    G.partition(omega, delta)
                assert ei.value.code == H.HGP_ERR_OOM
                failed_in["partition"] += 1
                alloc.fail_at = 0
                _same(G.partition(omega, delta), want)     # the handle is still usable
        torch_cuda.cuda.synchronize()
        assert alloc.live == {}, f"chunks leaked after a failure at request {k}"
        assert alloc.allocs == alloc.frees
    assert failed_in["create"] > 0 and failed_in["partition"] > 0


def test_exhausted_probe_loop_reports_device_limit(torch_cuda):
    g, omega, delta = synth.random_snn(600, 24, 3), 32, 300     # > 64 distinct neighbours per node
    with hgp.Graph.from_hypergraph(g) as G:
        with pytest.raises(H.HgpError) as ei:
            G.partition(omega, delta, debug=H.HGP_DEBUG_FORCE_GLOBAL | H.HGP_DEBUG_SMALL_TABLE)
        assert ei.value.code == H.HGP_ERR_DEVICE_LIMIT
        # the context and the handle remain usable
        _same(G.partition(omega, delta), oracle.partition(g, omega, delta))
