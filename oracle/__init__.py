"""ctypes view of the CPU oracle (``hgp_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the
benchmark's CPU-baseline leg load this module; the library's product path
never does.  It shares no code with the CUDA library.

The oracle is a plain single-threaded C restatement of the paper's method:
Eq. (2) candidate scoring with deferred size/inbound checks, matching over
the pairing pseudo-forest, contraction (Sec. III), and Eq. (3) refinement
with in-sequence gains and best valid prefix (Sec. IV).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hgp_oracle.c")
_LIB = os.path.join(_HERE, "_hgp_oracle.so")
_lock = threading.Lock()
_lib = None

OK, INVALID, INFEASIBLE, OOM, INTERNAL = 0, 1, 2, 3, 4

A_PAIR, A_SCORE, A_MATCH, A_GAMMA, A_RHO_IN, A_RHO_OUT, A_W = 0, 1, 2, 3, 4, 5, 6
A_PINS_OFF, A_PINS, A_INC_OFF, A_INC, A_IN_OFF, A_IN = 7, 8, 9, 10, 11, 12
A_MOVE_N, A_MOVE_PS, A_MOVE_PD, A_MOVE_GAIN, A_GAIN_SEQ, A_VIOL = 13, 14, 15, 16, 17, 18
A_KEY = 19
N_PARAMS = 641          # W1 (64 x 8), b1 (64), W2 (64), b2


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with code {code}")
        self.code = code


def build() -> str:
    """Compile the oracle with gcc (plain C11, -O2)."""
    if (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", _SRC,
                               "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
            lib.orun_create.argtypes = [i32, i32, vp, vp, vp, vp, ctypes.POINTER(vp)]
            lib.orun_create_incident.argtypes = [i32, i32, vp, vp, vp, vp, ctypes.POINTER(vp)]
            lib.orun_create_outbound.argtypes = [i32, i32, vp, vp, vp, vp, ctypes.POINTER(vp)]
            lib.orun_destroy.argtypes = [vp]
            lib.orun_partition.argtypes = [vp, i64, i64, i32]
            lib.orun_partition_cut.argtypes = [vp, i64, i64, i32, i32]
            lib.orun_partition_ex.argtypes = [vp, i64, i64, i32, i32, i32]
            for name, rt in [("orun_num_levels", i32), ("orun_top_is_gamma", i32), ("orun_K", i32),
                             ("orun_cost", i64), ("orun_num_parts", i32)]:
                getattr(lib, name).argtypes = [vp]
                getattr(lib, name).restype = rt
            for name, rt in [("orun_level_V", i32), ("orun_level_P", i64), ("orun_level_in_total", i64),
                             ("orun_refine_M", i32), ("orun_refine_kstar", i32), ("orun_refine_gain", i64)]:
                getattr(lib, name).argtypes = [vp, i32]
                getattr(lib, name).restype = rt
            lib.orun_array_len.argtypes = [vp, i32, i32]
            lib.orun_array_len.restype = i64
            lib.orun_array.argtypes = [vp, i32, i32, vp]
            lib.orun_part_ids.argtypes = [vp, vp]
            lib.orun_part_stats.argtypes = [vp, vp, vp]
            lib.orun_hist_row.argtypes = [vp, i32, i32, vp]
            lib.orun_score0.argtypes = [vp, i64, i64, vp, vp]
            lib.orun_score0_nodes.argtypes = [vp, i64, i64, vp, i32, vp, vp]
            lib.oracle_match.argtypes = [i32, vp, vp, i32, vp]
            lib.oracle_gamma.argtypes = [i32, vp, vp]
            lib.oracle_gamma.restype = i32
            lib.orun_refine0.argtypes = [vp, vp, i32, i64, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp]
            lib.orun_contract0.argtypes = [vp, vp]
            u16, u64, f64 = ctypes.c_uint16, ctypes.c_uint64, ctypes.c_double
            lib.oracle_match64.argtypes = [i32, vp, vp, i32, vp]
            lib.orun_partition_learned.argtypes = [vp, i64, i64, i32, vp, vp, vp, u16, i32]
            lib.oracle_lg1p.argtypes = [i64]
            lib.oracle_lg1p.restype = ctypes.c_float
            lib.oracle_mlp.argtypes = [vp, vp, vp, u16, i32, vp, vp, vp]
            lib.orun_features0.argtypes = [vp, i32, i32, vp]
            lib.orun_learn_samples.argtypes = [vp, vp, u64, i32, vp, vp, vp]
            lib.orun_score0_learned_nodes.argtypes = [vp, i64, i64, vp, vp, vp, u16, i32, vp, i32,
                                                      vp, vp, vp]
            lib.orun_fill_baseline.argtypes = [vp, i64, i64, vp]
            lib.orun_fill_baseline.restype = i32
            lib.oracle_splitmix64_at.argtypes = [u64, u64]
            lib.oracle_splitmix64_at.restype = u64
            lib.oracle_train_step.argtypes = [vp, vp, vp, i64, f64, f64, f64, f64, i32, vp, vp,
                                              vp, vp, vp, vp, vp]
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _i32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.int32)


@dataclass
class Result:
    part_ids: np.ndarray
    cost: int
    num_parts: int
    part_weight: np.ndarray
    part_inbound: np.ndarray


class Run:
    """One input hypergraph held by the oracle; ``partition`` runs the method
    and keeps every level's arrays for inspection."""

    def __init__(self, num_nodes, offsets, pins, node_weights=None, edge_weights=None,
                 incident=False, outbound=False):
        """incident=True: Delta counts every incident hyperedge (in(n) = I(n));
        outbound=True: the hyperedges sourced in the part (in(n) = {e : src(e) = n})."""
        lib = _load()
        self._keep = [_i32(offsets), _i32(pins), _i32(node_weights), _i32(edge_weights)]
        h = ctypes.c_void_p()
        if incident and outbound:
            raise ValueError("incident and outbound are exclusive")
        create = (lib.orun_create_incident if incident else
                  lib.orun_create_outbound if outbound else lib.orun_create)
        rc = create(int(num_nodes), int(len(offsets) - 1), *[_p(a) for a in self._keep],
                    ctypes.byref(h))
        if rc:
            raise OracleError(rc, "create")
        self._h = h
        self.num_nodes = int(num_nodes)

    @classmethod
    def from_graph(cls, g, incident=False, outbound=False):
        return cls(g.num_nodes, g.offsets, g.pins, g.node_weights, g.edge_weights, incident, outbound)

    def close(self):
        if getattr(self, "_h", None):
            _load().orun_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- whole method ----
    def partition(self, omega: int, delta: int, refine_passes: int = 1, max_levels: int = 0,
                  matching: int = 0) -> Result:
        """max_levels > 0: coarsening stops after that many matchings (the
        library's hgp_options.max_levels), a bounded prefix of the method.
        matching = 1: the exact maximum-weight matching of the pairing
        pseudo-forest instead of the paper's two walks."""
        lib = _load()
        if matching:
            rc = lib.orun_partition_ex(self._h, int(omega), int(delta), int(refine_passes),
                                       int(max_levels), int(matching))
        elif max_levels:
            rc = lib.orun_partition_cut(self._h, int(omega), int(delta), int(refine_passes),
                                        int(max_levels))
        else:
            rc = lib.orun_partition(self._h, int(omega), int(delta), int(refine_passes))
        if rc:
            raise OracleError(rc, "partition")
        np_ = lib.orun_num_parts(self._h)
        ids = np.empty(self.num_nodes, dtype=np.int32)
        lib.orun_part_ids(self._h, _p(ids))
        w = np.empty(max(np_, 1), dtype=np.int64)
        inb = np.empty(max(np_, 1), dtype=np.int32)
        lib.orun_part_stats(self._h, _p(w), _p(inb))
        return Result(ids, int(lib.orun_cost(self._h)), int(np_), w[:np_], inb[:np_])

    def partition_learned(self, omega: int, delta: int, model, refine_passes: int = 1) -> Result:
        """The method with the learned candidate order; `model` has bfloat16
        bit arrays w1 [64, 8], b1 [64], w2 [64], the scalar b2 and key_bits."""
        lib = _load()
        w1, b1, w2 = _model_arrays(model)
        rc = lib.orun_partition_learned(self._h, int(omega), int(delta), int(refine_passes),
                                        _p(w1), _p(b1), _p(w2), int(model.b2), int(model.key_bits))
        if rc:
            raise OracleError(rc, "partition_learned")
        np_ = lib.orun_num_parts(self._h)
        ids = np.empty(self.num_nodes, dtype=np.int32)
        lib.orun_part_ids(self._h, _p(ids))
        w = np.empty(max(np_, 1), dtype=np.int64)
        inb = np.empty(max(np_, 1), dtype=np.int32)
        lib.orun_part_stats(self._h, _p(w), _p(inb))
        return Result(ids, int(lib.orun_cost(self._h)), int(np_), w[:np_], inb[:np_])

    def score0_learned_nodes(self, omega, delta, model, nodes):
        """Learned-order (pair, score, key) of the listed level-0 nodes only."""
        w1, b1, w2 = _model_arrays(model)
        nodes = _i32(nodes)
        out = [np.empty(len(nodes), dtype=np.int32) for _ in range(3)]
        rc = _load().orun_score0_learned_nodes(self._h, int(omega), int(delta), _p(w1), _p(b1), _p(w2),
                                               int(model.b2), int(model.key_bits), _p(nodes), len(nodes),
                                               *[_p(o) for o in out])
        if rc:
            raise OracleError(rc, "score0_learned_nodes")
        return tuple(out)

    def fill_baseline(self, omega, delta):
        """The constraint-only baseline: (part ids, number of parts)."""
        ids = np.empty(self.num_nodes, dtype=np.int32)
        k = _load().orun_fill_baseline(self._h, int(omega), int(delta), _p(ids))
        if k < 0:
            raise OracleError(-k, "fill_baseline")
        return ids, int(k)

    def features0(self, n, m):
        x = np.empty(8, dtype=np.float32)
        rc = _load().orun_features0(self._h, int(n), int(m), _p(x))
        if rc:
            raise OracleError(rc, "features0")
        return x

    def learn_samples(self, part_ids, seed, per_node):
        """Training pairs labelled by part_ids: (x [N*per_node, 8], y, partner)."""
        S = self.num_nodes * int(per_node)
        x = np.empty((S, 8), dtype=np.float32)
        y = np.empty(S, dtype=np.float32)
        partner = np.empty(S, dtype=np.int32)
        rc = _load().orun_learn_samples(self._h, _p(_i32(part_ids)), ctypes.c_uint64(int(seed)),
                                        int(per_node), _p(x), _p(y), _p(partner))
        if rc:
            raise OracleError(rc, "learn_samples")
        return x, y, partner

    # ---- trace ----
    @property
    def num_levels(self) -> int:
        return int(_load().orun_num_levels(self._h))

    @property
    def top_is_gamma(self) -> bool:
        return bool(_load().orun_top_is_gamma(self._h))

    @property
    def K(self) -> int:
        return int(_load().orun_K(self._h))

    def level_V(self, l):
        return int(_load().orun_level_V(self._h, l))

    def level_P(self, l):
        return int(_load().orun_level_P(self._h, l))

    def refine_stats(self, l):
        lib = _load()
        return (int(lib.orun_refine_M(self._h, l)), int(lib.orun_refine_kstar(self._h, l)),
                int(lib.orun_refine_gain(self._h, l)))

    def array(self, l: int, which: int):
        lib = _load()
        n = lib.orun_array_len(self._h, l, which)
        if n < 0:
            return None
        out = np.empty(max(n, 1), dtype=np.int64)
        rc = lib.orun_array(self._h, l, which, _p(out))
        if rc:
            raise OracleError(rc, "array")
        return out[:n]

    def level_csr(self, l):
        """(w, pins_off, pins, inc_off, inc, in_off, in) of level l."""
        return tuple(self.array(l, a) for a in (A_W, A_PINS_OFF, A_PINS, A_INC_OFF, A_INC, A_IN_OFF, A_IN))

    # ---- single steps ----
    def hist_row(self, l, n):
        V = self.level_V(l)
        out = np.empty(V, dtype=np.int64)
        rc = _load().orun_hist_row(self._h, l, n, _p(out))
        if rc:
            raise OracleError(rc, "hist_row")
        return out

    def score0(self, omega, delta):
        pair = np.empty(self.num_nodes, dtype=np.int32)
        score = np.empty(self.num_nodes, dtype=np.int32)
        rc = _load().orun_score0(self._h, int(omega), int(delta), _p(pair), _p(score))
        if rc:
            raise OracleError(rc, "score0")
        return pair, score

    def score0_nodes(self, omega, delta, nodes):
        """Candidate and score of the listed level-0 nodes only."""
        nodes = _i32(nodes)
        pair = np.empty(len(nodes), dtype=np.int32)
        score = np.empty(len(nodes), dtype=np.int32)
        rc = _load().orun_score0_nodes(self._h, int(omega), int(delta), _p(nodes), len(nodes),
                                       _p(pair), _p(score))
        if rc:
            raise OracleError(rc, "score0_nodes")
        return pair, score

    def refine0(self, rho, K, omega, delta):
        """One refinement pass on the input level from partition rho.
        Returns (new_rho, dict with M, kstar, gain, moves, gain_seq, viol)."""
        N = self.num_nodes
        rho = np.array(rho, dtype=np.int32)
        bufs = [np.empty(N, dtype=np.int32) for _ in range(6)]
        M, ks, g = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        rc = _load().orun_refine0(self._h, _p(rho), int(K), int(omega), int(delta), ctypes.byref(M),
                                  ctypes.byref(ks), ctypes.byref(g), *[_p(b) for b in bufs])
        if rc:
            raise OracleError(rc, "refine0")
        m = M.value
        return rho, dict(M=m, kstar=ks.value, gain=g.value, n=bufs[0][:m], ps=bufs[1][:m],
                         pd=bufs[2][:m], gain_iso=bufs[3][:m], gain_seq=bufs[4][:m], viol=bufs[5][:m])

    def contract0(self, match):
        m = _i32(match)
        rc = _load().orun_contract0(self._h, _p(m))
        if rc:
            raise OracleError(rc, "contract0")


def match(pair, score, method: int = 0):
    """method 0: the two walks; 1: the lock restatement; 2: exact DP."""
    pair = _i32(pair)
    score = _i32(score)
    out = np.empty(len(pair), dtype=np.int32)
    rc = _load().oracle_match(len(pair), _p(pair), _p(score), int(method), _p(out))
    if rc:
        raise OracleError(rc, "match")
    return out


def gamma(match_arr):
    m = _i32(match_arr)
    out = np.empty(len(m), dtype=np.int32)
    v2 = _load().oracle_gamma(len(m), _p(m), _p(out))
    return out, int(v2)


def partition(g, omega, delta, refine_passes=1) -> Result:
    with Run.from_graph(g) as r:
        return r.partition(omega, delta, refine_passes)


def _model_arrays(model):
    w1 = np.ascontiguousarray(model.w1, dtype=np.uint16).reshape(64, 8)
    b1 = np.ascontiguousarray(model.b1, dtype=np.uint16).reshape(64)
    w2 = np.ascontiguousarray(model.w2, dtype=np.uint16).reshape(64)
    return w1, b1, w2


def match64(pair, score64, method: int = 0):
    pair = _i32(pair)
    s = np.ascontiguousarray(score64, dtype=np.int64)
    out = np.empty(len(pair), dtype=np.int32)
    rc = _load().oracle_match64(len(pair), _p(pair), _p(s), int(method), _p(out))
    if rc:
        raise OracleError(rc, "match64")
    return out


def lg1p(x: int) -> float:
    return float(_load().oracle_lg1p(int(x)))


def mlp(model, x):
    """(score, key) of one feature vector under `model`."""
    w1, b1, w2 = _model_arrays(model)
    xx = np.ascontiguousarray(x, dtype=np.float32)
    s = ctypes.c_float()
    k = ctypes.c_int32()
    rc = _load().oracle_mlp(_p(w1), _p(b1), _p(w2), int(model.b2), int(model.key_bits), _p(xx),
                            ctypes.byref(s), ctypes.byref(k))
    if rc:
        raise OracleError(rc, "mlp")
    return s.value, k.value


def train_step(params, x, y, lr, beta1, beta2, eps, t, m, v):
    """One Adam step in double precision; returns dict(grad, loss, params, m, v)."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    xx = np.ascontiguousarray(x, dtype=np.float32)
    yy = np.ascontiguousarray(y, dtype=np.float32)
    mm = np.ascontiguousarray(m, dtype=np.float64)
    vv = np.ascontiguousarray(v, dtype=np.float64)
    out = {k: np.empty(N_PARAMS) for k in ("grad", "params", "m", "v")}
    loss = ctypes.c_double()
    rc = _load().oracle_train_step(_p(p), _p(xx), _p(yy), len(yy), float(lr), float(beta1),
                                   float(beta2), float(eps), int(t), _p(mm), _p(vv),
                                   _p(out["grad"]), ctypes.byref(loss), _p(out["params"]),
                                   _p(out["m"]), _p(out["v"]))
    if rc:
        raise OracleError(rc, "train_step")
    out["loss"] = loss.value
    return out


def partition_learned(g, omega, delta, model, refine_passes=1) -> Result:
    with Run.from_graph(g) as r:
        return r.partition_learned(omega, delta, model, refine_passes)


def splitmix64_at(seed: int, i: int) -> int:
    return int(_load().oracle_splitmix64_at(ctypes.c_uint64(seed), ctypes.c_uint64(i)))
