"""Independent brute-force helpers for pinning the oracle (and the CUDA path).

Everything here is computed from the problem definition of Sec. II-A by a
different route than the oracle takes: incidence matrices, Python sets and
exhaustive enumeration.  No code is shared with the oracle or the library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
import threading

import numpy as np


def edges_of(offsets, pins):
    off = np.asarray(offsets)
    p = np.asarray(pins)
    return [p[off[e]:off[e + 1]].tolist() for e in range(len(off) - 1)]


def in_sets(num_nodes, offsets, pins):
    """in(n) as Python sets; the first pin of an edge is its source."""
    ins = [set() for _ in range(num_nodes)]
    for e, ed in enumerate(edges_of(offsets, pins)):
        for n in ed[1:]:
            ins[n].add(e)
    return ins


def incidence(num_nodes, offsets, pins):
    """Dense E x N 0/1 pin matrix."""
    E = len(offsets) - 1
    B = np.zeros((E, num_nodes), dtype=np.int64)
    for e, ed in enumerate(edges_of(offsets, pins)):
        B[e, ed] = 1
    return B


def conn(offsets, pins, rho, ew=None):
    """Eq. (1) computed with Python sets."""
    c = 0
    for e, ed in enumerate(edges_of(offsets, pins)):
        c += (1 if ew is None else int(ew[e])) * (len({int(rho[n]) for n in ed}) - 1)
    return c


def part_stats(num_nodes, offsets, pins, rho, nw=None):
    """{part: (weight, |union of in(n)|)} recounted from scratch."""
    ins = in_sets(num_nodes, offsets, pins)
    st = {}
    for n in range(num_nodes):
        p = int(rho[n])
        w, s = st.get(p, (0, set()))
        st[p] = (w + (1 if nw is None else int(nw[n])), s | ins[n])
    return {p: (w, len(s)) for p, (w, s) in st.items()}


def feasible(num_nodes, offsets, pins, rho, omega, delta, nw=None):
    return all(w <= omega and d <= delta for w, d in part_stats(num_nodes, offsets, pins, rho, nw).values())


def set_partitions(n):
    """All set partitions of range(n) as restricted-growth strings."""
    a = [0] * n

    def rec(i, m):
        if i == n:
            yield list(a)
            return
        for v in range(m + 1):
            a[i] = v
            yield from rec(i + 1, m + 1 if v == m else m)

    if n == 0:
        yield []
        return
    a[0] = 0
    yield from rec(1, 1)


def brute_opt(num_nodes, offsets, pins, omega, delta, nw=None, ew=None):
    """(optimal Eq. (1) cost, number of feasible partitions) by enumeration."""
    best, nfeas = None, 0
    for rho in set_partitions(num_nodes):
        if not feasible(num_nodes, offsets, pins, rho, omega, delta, nw):
            continue
        nfeas += 1
        c = conn(offsets, pins, rho, ew)
        if best is None or c < best:
            best = c
    return best, nfeas


_C_SRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "brute_opt.c")
_c_lib = None
_c_lock = threading.Lock()


def _brute_c():
    """The C enumerator of brute_opt.c, compiled once per process into a
    temporary directory (gcc, no GPU)."""
    global _c_lib
    with _c_lock:
        if _c_lib is None:
            d = tempfile.mkdtemp(prefix="hgp_brute_")
            so = os.path.join(d, "brute_opt.so")
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _C_SRC, "-o", so])
            lib = ctypes.CDLL(so)
            vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
            lib.brute_optimum.argtypes = [i32, i32, vp, vp, vp, vp, i64, i64, i32,
                                          ctypes.POINTER(i64), ctypes.POINTER(i64)]
            lib.brute_optimum.restype = ctypes.c_int
            _c_lib = lib
    return _c_lib


def brute_opt_c(num_nodes, offsets, pins, omega, delta, nw=None, ew=None, incident=False,
                outbound=False):
    """brute_opt by the C enumerator (up to 16 nodes, 64 hyperedges): every set
    partition visited, branches cut as soon as a part breaks a bound.  The
    second bound counts inbound hyperedges, or every incident one
    (incident=True), or those sourced in the part (outbound=True).
    Returns (optimal cost or None, number of feasible partitions)."""
    arrs = [np.ascontiguousarray(a, dtype=np.int32) if a is not None else None
            for a in (offsets, pins, nw, ew)]
    best, count = ctypes.c_int64(), ctypes.c_int64()
    rc = _brute_c().brute_optimum(int(num_nodes), len(arrs[0]) - 1,
                                  *[a.ctypes.data if a is not None else None for a in arrs],
                                  int(omega), int(delta), 1 if incident else 2 if outbound else 0,
                                  ctypes.byref(best), ctypes.byref(count))
    if rc != 0:
        raise ValueError("brute_optimum: graph too large for the enumerator")
    return (None if best.value < 0 else int(best.value)), int(count.value)
