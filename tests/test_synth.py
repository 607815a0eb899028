"""The seeded input generators shared by the oracle tests and the GPU tests
(`synth/`) produce the shapes the design states for the paper's workloads:
one hyperedge per neuron, its first pin the neuron itself, then distinct
targets in ascending order; layered graphs connect a neuron to the same
channels at every in-grid position of the 3x3 window of the next layer.
These are properties of the inputs only: nothing of the method is tested."""
import math

import numpy as np
import pytest

import synth


def _edges(g):
    off = g.offsets.astype(np.int64)
    return [g.pins[off[e]:off[e + 1]] for e in range(g.num_edges)]


@pytest.mark.parametrize("n,size,size_max,seed", [(500, 16, None, 3), (700, 8, 40, 11), (64, 64, None, 0)])
def test_random_snn_structure(n, size, size_max, seed):
    g = synth.random_snn(n, size, seed, size_max=size_max)
    assert g.num_nodes == n and g.num_edges == n
    assert g.offsets.dtype == np.int32 and g.pins.dtype == np.int32
    hi = size if size_max is None else size_max
    for e, pins in enumerate(_edges(g)):
        assert pins[0] == e                                     # the source first
        t = pins[1:]
        assert size <= len(pins) <= min(hi, n)
        assert np.all(np.diff(t) > 0)                           # distinct, ascending
        assert np.all((t >= 0) & (t < n)) and not np.any(t == e)


def test_random_snn_sizes_cover_the_range():
    g = synth.random_snn(4000, 8, 5, size_max=16)
    sizes = np.diff(g.offsets)
    assert sizes.min() == 8 and sizes.max() == 16
    assert set(np.unique(sizes)) == set(range(8, 17))


def test_generators_are_deterministic_and_seeded():
    a, b = synth.random_snn(300, 12, 7), synth.random_snn(300, 12, 7)
    assert np.array_equal(a.offsets, b.offsets) and np.array_equal(a.pins, b.pins)
    c = synth.random_snn(300, 12, 8)
    assert not np.array_equal(a.pins, c.pins)
    x, y = synth.conv_snn(3, 5, 6, 3, 6, 2), synth.conv_snn(3, 5, 6, 3, 6, 2)
    assert np.array_equal(x.pins, y.pins)
    assert synth.uniform01(3, 17) == synth.uniform01(3, 17)
    assert 0.0 <= synth.uniform01(3, 17) < 1.0


def test_named_workload_shapes():
    g = synth.snn_2k(0)
    assert (g.num_nodes, g.num_pins) == (2048, 65_536)
    assert set(np.diff(g.offsets)) == {32}
    g = synth.snn_16k(0)
    assert (g.num_nodes, g.num_pins) == (16_384, 2_097_152)
    assert set(np.diff(g.offsets)) == {128}


@pytest.mark.parametrize("layers,side,ch,cmin,cmax,seed", [(4, 6, 8, 5, 8, 3), (3, 4, 5, 1, 5, 9)])
def test_conv_snn_structure(layers, side, ch, cmin, cmax, seed):
    g = synth.conv_snn(layers, side, ch, cmin, cmax, seed)
    per = side * side * ch
    assert g.num_nodes == layers * per
    for e, pins in enumerate(_edges(g)):
        l, rem = divmod(e, per)
        pos, c = divmod(rem, ch)
        y, x = divmod(pos, side)
        assert pins[0] == e
        t = pins[1:]
        if l == layers - 1:
            assert len(t) == 0                                  # last layer: single-pin edge
            continue
        assert np.all(np.diff(t) > 0)
        assert np.all((t >= (l + 1) * per) & (t < (l + 2) * per))
        tpos, tc = np.divmod(t - (l + 1) * per, ch)
        ty, tx = np.divmod(tpos, side)
        assert np.all(np.abs(ty - y) <= 1) and np.all(np.abs(tx - x) <= 1)
        cells = {(int(a), int(b)) for a, b in zip(ty, tx)}
        want = {(y + dy, x + dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                if 0 <= y + dy < side and 0 <= x + dx < side}
        assert cells == want                                    # every in-grid window cell
        chans = {cell: sorted(int(k) for k, a, b in zip(tc, ty, tx) if (a, b) == cell) for cell in cells}
        first = next(iter(chans.values()))
        assert all(v == first for v in chans.values())          # the same channels everywhere
        assert cmin <= len(first) <= min(cmax, ch)


def test_batch_instances_shapes():
    inst = synth.batch_instances(8, 0)
    assert len(inst) == 8
    for i, g in enumerate(inst):
        u = synth.uniform01(0, 10_000 + i)
        n = int(math.floor(math.exp(math.log(2048) + u * (math.log(65536) - math.log(2048)))))
        if i % 2 == 0:
            assert g.num_nodes == n
            sizes = np.diff(g.offsets)
            assert sizes.min() >= 32 and sizes.max() <= 256
        else:
            ch = max(1, n // (8 * 256))
            assert g.num_nodes == 8 * 16 * 16 * ch            # layered: 8 layers of 16 x 16 x ch
        assert 2048 <= n < 65536


def test_training_graphs_recipe():
    gs = synth.training_graphs(3, 100, sizes=(2048, 4096))
    assert [g.num_nodes for g in gs] == [2048, 4096, 2048]
    for g in gs:
        sizes = np.diff(g.offsets)
        assert sizes.min() >= 128 and sizes.max() <= 256
    assert not np.array_equal(gs[0].pins, gs[2].pins)          # seeds 100 and 102
