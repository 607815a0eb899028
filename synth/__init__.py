"""Seeded synthetic hypergraphs shaped like the paper's SNN workloads (Table I).

This module only draws random pins; it contains none of the partitioning
method's arithmetic.  It is the one piece shared by the CPU oracle tests and
the CUDA path's tests and benchmark, so both always see identical inputs.

Every hypergraph is returned as int32 CSR: ``offsets[E+1]`` and ``pins[P]``,
with one hyperedge per neuron whose first pin is its source (the neuron) and
whose remaining pins are its distinct targets in ascending id order.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "_synth.so")
_lock = threading.Lock()
_lib = None


def build() -> str:
    """Compile the generator library in place (gcc, no GPU needed)."""
    if (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32, i64, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
            p64 = ctypes.POINTER(ctypes.c_int64)
            p32 = ctypes.POINTER(ctypes.c_int32)
            lib.synth_random_offsets.argtypes = [i32, i32, i32, u64, p64]
            lib.synth_random_fill.argtypes = [i32, i32, i32, u64, p64, p32]
            lib.synth_conv_offsets.argtypes = [i32, i32, i32, i32, i32, u64, p64]
            lib.synth_conv_fill.argtypes = [i32, i32, i32, i32, i32, u64, p64, p32]
            lib.synth_uniform01.argtypes = [u64, u64]
            lib.synth_uniform01.restype = ctypes.c_double
            _lib = lib
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


@dataclass
class Hypergraph:
    """int32 CSR hypergraph plus optional weights (None = unit)."""
    num_nodes: int
    offsets: np.ndarray          # int32 [E+1]
    pins: np.ndarray             # int32 [P]
    node_weights: np.ndarray | None = None   # int32 [N]
    edge_weights: np.ndarray | None = None   # int32 [E]
    name: str = ""

    @property
    def num_edges(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def num_pins(self) -> int:
        return int(self.offsets[-1])


def _finish(num_nodes, off64, pins, name):
    if off64[-1] >= 2**31:
        raise ValueError("hypergraph has 2^31 or more pins; int32 CSR cannot hold it")
    return Hypergraph(num_nodes, off64.astype(np.int32), pins, None, None, name)


def random_snn(num_nodes: int, size: int, seed: int, size_max: int | None = None) -> Hypergraph:
    """One hyperedge per node: [node, size-1 distinct uniform targets].

    With ``size_max`` the size of each edge is uniform in [size, size_max].
    """
    lib = _load()
    kmax = size if size_max is None else size_max
    off = np.empty(num_nodes + 1, dtype=np.int64)
    rc = lib.synth_random_offsets(num_nodes, size, kmax, seed, _ptr(off, ctypes.c_int64))
    if rc:
        raise ValueError("bad random_snn parameters")
    pins = np.empty(int(off[-1]), dtype=np.int32)
    rc = lib.synth_random_fill(num_nodes, size, kmax, seed, _ptr(off, ctypes.c_int64),
                               _ptr(pins, ctypes.c_int32))
    if rc:
        raise MemoryError("synth_random_fill")
    return _finish(num_nodes, off, pins, f"rand{num_nodes}x{size}" + (f"-{kmax}" if kmax != size else "") + f"s{seed}")


def conv_snn(layers: int, side: int, ch: int, cmin: int, cmax: int, seed: int) -> Hypergraph:
    """Layered convolution-style SNN: each neuron reaches a 3x3 window of the
    next layer on C ~ U{cmin..cmax} distinct channels (same channels at every
    window position); last-layer neurons have single-pin edges."""
    lib = _load()
    n = layers * side * side * ch
    off = np.empty(n + 1, dtype=np.int64)
    rc = lib.synth_conv_offsets(layers, side, ch, cmin, cmax, seed, _ptr(off, ctypes.c_int64))
    if rc:
        raise ValueError("bad conv_snn parameters")
    pins = np.empty(int(off[-1]), dtype=np.int32)
    rc = lib.synth_conv_fill(layers, side, ch, cmin, cmax, seed, _ptr(off, ctypes.c_int64),
                             _ptr(pins, ctypes.c_int32))
    if rc:
        raise MemoryError("synth_conv_fill")
    return _finish(n, off, pins, f"conv{layers}x{side}x{side}x{ch}c{cmin}-{cmax}s{seed}")


def uniform01(seed: int, index: int) -> float:
    return float(_load().synth_uniform01(seed, index))


def random_weights(n: int, lo: int, hi: int, seed: int, stream: int) -> np.ndarray:
    """n integer weights uniform in [lo, hi], from (seed, stream)."""
    u = np.array([uniform01(seed * 1_000_003 + stream, i) for i in range(n)])
    return (lo + np.floor(u * (hi - lo + 1))).astype(np.int32)


# ---------------- the workloads ----------------

def snn_2k(seed: int = 0) -> Hypergraph:
    """2,048 neurons, edges of size 32 (source + 31 targets), ~65k pins."""
    return random_snn(2048, 32, seed)


def snn_16k(seed: int = 0) -> Hypergraph:
    """16,384 neurons, edges of size 128 (source + 127 targets), ~2.1M pins
    (the paper's 16k-rand shape)."""
    return random_snn(16384, 128, seed)


def snn_256k(seed: int = 0) -> Hypergraph:
    """262,144 neurons, edges of size 256, ~67M pins (256k-rand shape)."""
    return random_snn(262144, 256, seed)


def conv_200k(seed: int = 0) -> Hypergraph:
    """8 layers of 16x16x100 neurons (204,800), 3x3 windows on 88..100
    channels, ~1.4e8 pins (alexnet-like shape)."""
    return conv_snn(8, 16, 100, 88, 100, seed)


def batch_instances(count: int = 64, seed: int = 0) -> list[Hypergraph]:
    """Uneven batch: sizes log-uniform in [2048, 65536]; even instances random
    with edge size uniform in 32..256, odd instances layered conv-style."""
    out = []
    for i in range(count):
        u = uniform01(seed, 10_000 + i)
        n = int(math.floor(math.exp(math.log(2048) + u * (math.log(65536) - math.log(2048)))))
        if i % 2 == 0:
            out.append(random_snn(n, 32, seed * 1000 + i, size_max=256))
        else:
            ch = max(1, n // (8 * 256))
            out.append(conv_snn(8, 16, ch, max(1, math.ceil(0.88 * ch)), ch, seed * 1000 + i))
    return out


# ---------------- models for the learned candidate order ----------------

@dataclass
class Model:
    """Weights of the learned order's network as bfloat16 bit patterns:
    hidden = relu(b1 + W1 x) (64 x 8), score = b2 + W2 . hidden; key_bits sets
    the key resolution (key = floor(score * 2^key_bits))."""
    w1: np.ndarray
    b1: np.ndarray
    w2: np.ndarray
    b2: int
    key_bits: int


def _bf16_bits_truncated(a: np.ndarray) -> np.ndarray:
    return (np.ascontiguousarray(a, dtype=np.float32).view(np.uint32) >> 16).astype(np.uint16)


def random_model(seed: int, scale: float = 1.0, key_bits: int = 8) -> Model:
    """Seeded random weights (normal, times `scale`, truncated to bfloat16)."""
    rng = np.random.default_rng(seed)
    w1 = _bf16_bits_truncated(rng.normal(size=(64, 8)) * scale)
    b1 = _bf16_bits_truncated(rng.normal(size=64) * scale)
    w2 = _bf16_bits_truncated(rng.normal(size=64) * scale)
    b2 = int(_bf16_bits_truncated(rng.normal(size=1) * scale)[0])
    return Model(w1, b1, w2, b2, key_bits)


def zero_model(key_bits: int = 8) -> Model:
    z = np.zeros(64, dtype=np.uint16)
    return Model(np.zeros((64, 8), dtype=np.uint16), z.copy(), z.copy(), 0, key_bits)


def initial_params(seed: int) -> np.ndarray:
    """Seeded float32 starting point of training (641 values: W1 uniform in
    +-1/sqrt(8), W2 uniform in +-1/8, biases 0)."""
    rng = np.random.default_rng(seed)
    p = np.zeros(641, dtype=np.float32)
    p[:512] = rng.uniform(-1, 1, size=512) / np.sqrt(8.0)
    p[576:640] = rng.uniform(-1, 1, size=64) / 8.0
    return p


def training_graphs(count: int = 4, first_seed: int = 100, sizes=(16384,)) -> list[Hypergraph]:
    """Random SNN training graphs: node counts cycling through `sizes`,
    hyperedge sizes uniform in 128..256, seeds first_seed, first_seed + 1, ..."""
    return [random_snn(sizes[i % len(sizes)], 128, first_seed + i, size_max=256)
            for i in range(count)]
