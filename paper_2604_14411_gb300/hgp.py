"""ctypes binding of libhgp.so (include/hgp.h): argument marshalling only.

Every step of the partitioning runs in the library's CUDA kernels.  If the
library has not been built this module raises on import of the binding's
functions -- there is no fallback of any kind.

Host arrays are numpy int32/int64; device arrays are torch CUDA tensors
(passed with HGP_INPUT_DEVICE / HGP_OUTPUT_DEVICE).  PyTorch is used only for
device memory and streams.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhgp.so")

HGP_OK, HGP_ERR_INVALID_ARG, HGP_ERR_INFEASIBLE, HGP_ERR_OOM = 0, 1, 2, 3
HGP_ERR_CUDA, HGP_ERR_DEVICE_LIMIT, HGP_ERR_STATE, HGP_ERR_SCRATCH_LIMIT = 4, 5, 6, 7
HGP_INPUT_DEVICE = 1
HGP_DELTA_INCIDENT = 4
HGP_DELTA_OUTBOUND = 8
HGP_OUTPUT_DEVICE = 1
HGP_DEBUG_KEEP_LEVELS = 1
HGP_DEBUG_TIMING = 2
HGP_DEBUG_FORCE_GLOBAL = 4
HGP_DEBUG_NO_BITMAP = 8
HGP_DEBUG_FORCE_CLUSTER = 16
HGP_DEBUG_SMALL_TABLE = 32
HGP_DEBUG_REBUILD_INC = 64
HGP_DEBUG_FORCE_WINDOW = 128
HGP_DEBUG_FORCE_HASH_BUCKET = 256
(HGP_LEVEL_PAIR, HGP_LEVEL_SCORE, HGP_LEVEL_MATCH, HGP_LEVEL_GAMMA, HGP_LEVEL_RHO_IN,
 HGP_LEVEL_RHO_OUT, HGP_LEVEL_WEIGHT, HGP_LEVEL_REFINE, HGP_LEVEL_KEY,
 HGP_LEVEL_GAIN_SEQ) = range(10)
HGP_MLP_PARAMS = 641


class HgpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"hgp error {code}: {msg}")
        self.code = code


class hgp_model(ctypes.Structure):
    _fields_ = [("w1", ctypes.c_uint16 * 512), ("b1", ctypes.c_uint16 * 64),
                ("w2", ctypes.c_uint16 * 64), ("b2", ctypes.c_uint16), ("key_bits", ctypes.c_int16),
                ("reserved", ctypes.c_int32 * 3)]


class hgp_options(ctypes.Structure):
    _fields_ = [("refine_passes", ctypes.c_int32), ("debug", ctypes.c_uint32),
                ("max_levels", ctypes.c_int32), ("matching", ctypes.c_int32),
                ("learned_eval", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1),
                ("model", ctypes.POINTER(hgp_model))]


class hgp_train_options(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("first_step", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


@dataclass
class Model:
    """The learned order's network as bfloat16 bit patterns (see hgp_model)."""
    w1: np.ndarray      # uint16 [64, 8]
    b1: np.ndarray      # uint16 [64]
    w2: np.ndarray      # uint16 [64]
    b2: int
    key_bits: int


def _c_model(model):
    if model is None:
        return None
    m = hgp_model()
    ctypes.memmove(m.w1, np.ascontiguousarray(model.w1, dtype=np.uint16).reshape(512).ctypes.data, 1024)
    ctypes.memmove(m.b1, np.ascontiguousarray(model.b1, dtype=np.uint16).reshape(64).ctypes.data, 128)
    ctypes.memmove(m.w2, np.ascontiguousarray(model.w2, dtype=np.uint16).reshape(64).ctypes.data, 128)
    m.b2 = int(model.b2)
    m.key_bits = int(model.key_bits)
    return m


def _options(refine_passes, debug, max_levels, model, matching=0, learned_eval=0):
    opt = hgp_options(refine_passes, debug, max_levels, matching, learned_eval)
    cm = _c_model(model)
    if cm is not None:
        opt.model = ctypes.pointer(cm)
    return opt, cm


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class hgp_allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", ctypes.c_void_p)]


class TorchAllocator:
    """An hgp_allocator that draws the library's device memory from PyTorch's
    CUDA caching allocator (torch.cuda.caching_allocator_alloc / _delete), so
    that the library and the surrounding PyTorch program share one pool.

    Keeps host-side counts for inspection: ``allocs``, ``frees``, ``live``
    (pointer -> bytes of the chunks not yet returned), ``peak_bytes`` (the
    most held at once).  ``fail_at`` = k > 0
    makes the k-th allocation from now report failure (returns NULL) without
    allocating -- a host-side fault injection for out-of-memory handling.
    Pass the object as ``allocator=`` to Graph / hgp_create and keep it alive
    until the handle is destroyed (Graph keeps a reference)."""

    def __init__(self, device=None):
        import threading
        import torch
        self._torch = torch
        self.device = torch.cuda.current_device() if device is None else int(device)
        self.live = {}
        self.allocs = 0
        self.frees = 0
        self.fail_at = 0
        self.peak_bytes = 0
        self._live_bytes = 0
        self._mu = threading.Lock()

        def _alloc(ctx, nbytes, stream):
            try:
                with self._mu:
                    if self.fail_at > 0:
                        self.fail_at -= 1
                        if self.fail_at == 0:
                            return None
                ptr = self._torch.cuda.caching_allocator_alloc(int(nbytes), self.device, int(stream or 0))
                with self._mu:
                    self.live[int(ptr)] = int(nbytes)
                    self.allocs += 1
                    self._live_bytes += int(nbytes)
                    self.peak_bytes = max(self.peak_bytes, self._live_bytes)
                return int(ptr)
            except Exception:       # out of memory or any other failure: report NULL
                return None

        def _free(ctx, ptr, nbytes, stream):
            try:
                with self._mu:
                    self._live_bytes -= self.live.pop(int(ptr), 0)
                    self.frees += 1
                self._torch.cuda.caching_allocator_delete(int(ptr))
            except Exception:
                pass

        self._c = hgp_allocator(_ALLOC_FN(_alloc), _FREE_FN(_free), None)

    @property
    def live_bytes(self) -> int:
        with self._mu:
            return self._live_bytes


class hgp_result(ctypes.Structure):
    _fields_ = [("part_ids", ctypes.c_void_p), ("part_weight", ctypes.c_void_p),
                ("part_inbound", ctypes.c_void_p), ("out_flags", ctypes.c_uint32),
                ("cost", ctypes.c_int64), ("num_parts", ctypes.c_int32),
                ("num_levels", ctypes.c_int32)]


class hgp_stats(ctypes.Structure):
    _fields_ = [("num_levels", ctypes.c_int32), ("num_parts", ctypes.c_int32),
                ("cost", ctypes.c_int64), ("ms_create", ctypes.c_double),
                ("ms_partition", ctypes.c_double), ("ms_coarsen", ctypes.c_double),
                ("ms_refine", ctypes.c_double), ("ms_score", ctypes.c_double),
                ("ms_match", ctypes.c_double), ("ms_contract", ctypes.c_double),
                ("score_launches", ctypes.c_int64), ("score_bytes", ctypes.c_int64),
                ("contract_bytes", ctypes.c_int64), ("pins_total", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("moves_applied", ctypes.c_int64),
                ("create_launches", ctypes.c_int64), ("ms_propose", ctypes.c_double),
                ("propose_launches", ctypes.c_int64), ("propose_bytes", ctypes.c_int64),
                ("learned_evals", ctypes.c_int64), ("ms_contract_kernels", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# every symbol declared in include/hgp.h
EXPORTS = ("hgp_create", "hgp_partition", "hgp_get_stats", "hgp_get_level_len",
           "hgp_get_level_array", "hgp_error_string", "hgp_last_error", "hgp_destroy",
           "hgp_score_noalloc", "hgp_partition_batch", "hgp_learn_samples", "hgp_train_mlp",
           "hgp_model_from_params", "hgp_fill_baseline")

_lib = None


def load(path: str = LIB_PATH):
    """Loads libhgp.so; raises if it is missing (build it with
    paper_2604_14411_gb300._build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libhgp.so not built at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    lib.hgp_create.argtypes = [i32, i32, vp, vp, vp, vp, u32, ctypes.POINTER(hgp_allocator), vp,
                               ctypes.POINTER(vp)]
    lib.hgp_create.restype = ctypes.c_int
    lib.hgp_partition.argtypes = [vp, i64, i64, ctypes.POINTER(hgp_options), ctypes.POINTER(hgp_result)]
    lib.hgp_partition.restype = ctypes.c_int
    lib.hgp_get_stats.argtypes = [vp, ctypes.POINTER(hgp_stats)]
    lib.hgp_get_level_len.argtypes = [vp, i32, i32]
    lib.hgp_get_level_len.restype = i64
    lib.hgp_get_level_array.argtypes = [vp, i32, i32, vp]
    lib.hgp_error_string.argtypes = [ctypes.c_int]
    lib.hgp_error_string.restype = ctypes.c_char_p
    lib.hgp_last_error.argtypes = [vp]
    lib.hgp_last_error.restype = ctypes.c_char_p
    lib.hgp_destroy.argtypes = [vp]
    lib.hgp_destroy.restype = None
    lib.hgp_score_noalloc.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, i64, i64, vp, vp, vp]
    lib.hgp_partition_batch.argtypes = [vp, i32, vp, vp, ctypes.POINTER(hgp_options), vp, vp]
    lib.hgp_partition_batch.restype = ctypes.c_int
    lib.hgp_score_noalloc.restype = ctypes.c_int
    lib.hgp_learn_samples.argtypes = [vp, vp, ctypes.c_uint64, i32, vp, vp, vp]
    lib.hgp_learn_samples.restype = ctypes.c_int
    lib.hgp_train_mlp.argtypes = [vp, vp, i64, ctypes.POINTER(hgp_train_options), vp, vp, vp, vp]
    lib.hgp_train_mlp.restype = ctypes.c_int
    lib.hgp_model_from_params.argtypes = [vp, i32, ctypes.POINTER(hgp_model)]
    lib.hgp_model_from_params.restype = ctypes.c_int
    lib.hgp_fill_baseline.argtypes = [vp, i64, i64, ctypes.POINTER(hgp_result)]
    lib.hgp_fill_baseline.restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(a):
    """Address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _is_device(a) -> bool:
    return a is not None and not isinstance(a, np.ndarray) and getattr(a, "is_cuda", False)


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


def _check(rc, handle=None):
    if rc != HGP_OK:
        lib = load()
        msg = lib.hgp_last_error(handle).decode() or lib.hgp_error_string(rc).decode()
        raise HgpError(rc, msg)


def hgp_create(num_nodes, offsets, pins, node_weights=None, edge_weights=None, stream=None,
               incident=False, allocator=None, outbound=False):
    """hgp_create: returns an opaque handle.  Arrays are all host numpy int32 or
    all torch int32 CUDA tensors.  incident=True: Delta counts every incident
    hyperedge (HGP_DELTA_INCIDENT); outbound=True: the hyperedges sourced in
    the part (HGP_DELTA_OUTBOUND).  allocator: a TorchAllocator (or None for
    the library's cudaMallocAsync); it must outlive the handle."""
    lib = load()
    dev = _is_device(offsets)
    arrs = [offsets, pins, node_weights, edge_weights]
    if not dev:
        arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.int32) for a in arrs]
    else:
        for a in arrs:
            if a is not None and (not _is_device(a) or str(a.dtype) != "torch.int32" or not a.is_contiguous()):
                raise TypeError("device inputs must be contiguous torch.int32 CUDA tensors")
    h = ctypes.c_void_p()
    E = int(arrs[0].shape[0]) - 1
    flags = ((HGP_INPUT_DEVICE if dev else 0) | (HGP_DELTA_INCIDENT if incident else 0) |
             (HGP_DELTA_OUTBOUND if outbound else 0))
    c_alloc = ctypes.byref(allocator._c) if allocator is not None else None
    rc = lib.hgp_create(int(num_nodes), E, *[_ptr(a) for a in arrs],
                        flags, c_alloc, _stream_handle(stream), ctypes.byref(h))
    _check(rc, None)
    return h


def hgp_partition(handle, omega, delta, part_ids, part_weight=None, part_inbound=None,
                  refine_passes=1, debug=0, max_levels=0, model=None, matching=0, learned_eval=0):
    """hgp_partition into caller buffers (host numpy or device torch tensors).
    matching=1: the exact maximum-weight matching instead of the two walks.
    learned_eval=1 (with a model): the network's hidden layer on tensor cores.
    Returns (cost, num_parts, num_levels)."""
    lib = load()
    opt, _keep = _options(refine_passes, debug, max_levels, model, matching, learned_eval)
    res = hgp_result()
    res.part_ids = _ptr(part_ids)
    res.part_weight = _ptr(part_weight)
    res.part_inbound = _ptr(part_inbound)
    res.out_flags = HGP_OUTPUT_DEVICE if _is_device(part_ids) else 0
    rc = lib.hgp_partition(handle, int(omega), int(delta), ctypes.byref(opt), ctypes.byref(res))
    _check(rc, handle)
    return int(res.cost), int(res.num_parts), int(res.num_levels)


def hgp_get_stats(handle) -> dict:
    st = hgp_stats()
    _check(load().hgp_get_stats(handle, ctypes.byref(st)), handle)
    return st.as_dict()


def hgp_get_level_array(handle, level, which):
    lib = load()
    n = lib.hgp_get_level_len(handle, int(level), int(which))
    if n < 0:
        return None
    out = np.empty(max(n, 1), dtype=np.int64)
    _check(lib.hgp_get_level_array(handle, int(level), int(which), out.ctypes.data), handle)
    return out[:n]


def hgp_error_string(code) -> str:
    return load().hgp_error_string(int(code)).decode()


def hgp_last_error(handle) -> str:
    return load().hgp_last_error(handle).decode()


def hgp_destroy(handle):
    if handle:
        load().hgp_destroy(handle)


def hgp_partition_batch(graphs, omegas, deltas, refine_passes=1, debug=0, max_levels=0, model=None,
                        matching=0):
    """Partitions several Graph objects concurrently; returns a list of Result."""
    lib = load()
    n = len(graphs)
    handles = (ctypes.c_void_p * n)(*[g._h.value for g in graphs])
    om = np.ascontiguousarray(omegas, dtype=np.int64)
    de = np.ascontiguousarray(deltas, dtype=np.int64)
    res = (hgp_result * n)()
    bufs = []
    for i, g in enumerate(graphs):
        ids = np.empty(g.num_nodes, dtype=np.int32)
        pw = np.empty(g.num_nodes, dtype=np.int64)
        pin = np.empty(g.num_nodes, dtype=np.int32)
        bufs.append((ids, pw, pin))
        res[i].part_ids, res[i].part_weight, res[i].part_inbound = ids.ctypes.data, pw.ctypes.data, pin.ctypes.data
        res[i].out_flags = 0
    status = np.zeros(max(n, 1), dtype=np.int32)
    opt, _keep = _options(refine_passes, debug, max_levels, model, matching)
    rc = lib.hgp_partition_batch(handles, n, om.ctypes.data, de.ctypes.data, ctypes.byref(opt),
                                 ctypes.addressof(res), status.ctypes.data)
    if rc != HGP_OK:
        bad = int(np.nonzero(status[:n])[0][0])
        raise HgpError(rc, f"instance {bad}: " + lib.hgp_last_error(graphs[bad]._h).decode())
    out = []
    for i, (ids, pw, pin) in enumerate(bufs):
        k = res[i].num_parts
        out.append(Result(ids, int(res[i].cost), int(k), int(res[i].num_levels), pw[:k], pin[:k]))
    return out


def hgp_train_mlp(x, y, params, adam, steps, batch, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                  first_step=1, stream=None):
    """hgp_train_mlp on torch CUDA tensors x [count, 8], y [count]; params
    (641) and adam (2 x 641) float32 numpy arrays are updated in place.
    Returns the per-step mean batch losses."""
    opt = hgp_train_options(int(steps), int(batch), float(lr), float(beta1), float(beta2),
                            float(eps), int(first_step))
    if params.dtype != np.float32 or adam.dtype != np.float32 or not params.flags.c_contiguous \
            or not adam.flags.c_contiguous:
        raise TypeError("params and adam must be contiguous float32 numpy arrays")
    loss = np.zeros(max(int(steps), 1), dtype=np.float32)
    rc = load().hgp_train_mlp(_ptr(x), _ptr(y), int(y.shape[0]), ctypes.byref(opt), _ptr(params),
                              _ptr(adam), _ptr(loss), _stream_handle(stream))
    _check(rc, None)
    return loss[:int(steps)]


def hgp_model_from_params(params, key_bits) -> Model:
    p = np.ascontiguousarray(params, dtype=np.float32)
    m = hgp_model()
    _check(load().hgp_model_from_params(_ptr(p), int(key_bits), ctypes.byref(m)), None)
    return Model(np.frombuffer(bytes(m.w1), dtype=np.uint16).reshape(64, 8).copy(),
                 np.frombuffer(bytes(m.b1), dtype=np.uint16).copy(),
                 np.frombuffer(bytes(m.w2), dtype=np.uint16).copy(), int(m.b2), int(m.key_bits))


@dataclass
class Result:
    part_ids: np.ndarray
    cost: int
    num_parts: int
    num_levels: int
    part_weight: np.ndarray
    part_inbound: np.ndarray


class Graph:
    """Owning wrapper around an hgp_graph handle."""

    def __init__(self, num_nodes, offsets, pins, node_weights=None, edge_weights=None, stream=None,
                 incident=False, allocator=None, outbound=False):
        self.num_nodes = int(num_nodes)
        self._allocator = allocator          # must outlive the handle
        self._h = hgp_create(num_nodes, offsets, pins, node_weights, edge_weights, stream, incident,
                             allocator, outbound)

    @classmethod
    def from_hypergraph(cls, g, stream=None, incident=False, allocator=None, outbound=False):
        return cls(g.num_nodes, g.offsets, g.pins, g.node_weights, g.edge_weights, stream, incident,
                   allocator, outbound)

    def partition(self, omega, delta, refine_passes=1, debug=0, max_levels=0, model=None,
                  matching=0, learned_eval=0) -> Result:
        ids = np.empty(self.num_nodes, dtype=np.int32)
        pw = np.empty(self.num_nodes, dtype=np.int64)
        pin = np.empty(self.num_nodes, dtype=np.int32)
        cost, npart, nlev = hgp_partition(self._h, omega, delta, ids, pw, pin, refine_passes, debug,
                                          max_levels, model, matching, learned_eval)
        return Result(ids, cost, npart, nlev, pw[:npart], pin[:npart])

    def partition_device(self, omega, delta, part_ids, part_weight=None, part_inbound=None,
                         refine_passes=1, debug=0, model=None):
        return hgp_partition(self._h, omega, delta, part_ids, part_weight, part_inbound,
                             refine_passes, debug, 0, model)

    def fill_baseline(self, omega, delta) -> Result:
        """hgp_fill_baseline: parts filled in node-id order (constraint-only)."""
        ids = np.empty(self.num_nodes, dtype=np.int32)
        pw = np.empty(self.num_nodes, dtype=np.int64)
        pin = np.empty(self.num_nodes, dtype=np.int32)
        res = hgp_result()
        res.part_ids, res.part_weight, res.part_inbound = ids.ctypes.data, pw.ctypes.data, pin.ctypes.data
        res.out_flags = 0
        _check(load().hgp_fill_baseline(self._h, int(omega), int(delta), ctypes.byref(res)), self._h)
        k = int(res.num_parts)
        return Result(ids, int(res.cost), k, 0, pw[:k], pin[:k])

    def learn_samples(self, part_ids, seed, per_node, with_partner=True):
        """hgp_learn_samples into new torch CUDA tensors: (x [S, 8], y [S],
        partner [S] or None), S = num_nodes * per_node; part_ids is a torch
        int32 CUDA tensor."""
        import torch
        S = self.num_nodes * int(per_node)
        dev = part_ids.device
        x = torch.empty((S, 8), dtype=torch.float32, device=dev)
        y = torch.empty(S, dtype=torch.float32, device=dev)
        partner = torch.empty(S, dtype=torch.int32, device=dev) if with_partner else None
        rc = load().hgp_learn_samples(self._h, _ptr(part_ids), ctypes.c_uint64(int(seed)),
                                      int(per_node), _ptr(x), _ptr(y), _ptr(partner))
        _check(rc, self._h)
        return x, y, partner

    def stats(self) -> dict:
        return hgp_get_stats(self._h)

    def level_array(self, level, which):
        return hgp_get_level_array(self._h, level, which)

    def close(self):
        if getattr(self, "_h", None):
            hgp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def train_model(graphs, omega, delta, seed=0, per_node=16, steps=2000, batch=4096, lr=3e-3,
                key_bits=6, init_params=None, stream=None):
    """The learned order's training pipeline, every step a library call:
    partition each training graph with the plain order (hgp_partition, part
    ids kept on the device), draw labelled pairs from it (hgp_learn_samples),
    train on all of them (hgp_train_mlp) and round the result to a model
    (hgp_model_from_params).  Returns (model, per-step losses)."""
    import torch
    xs, ys = [], []
    for i, g in enumerate(graphs):
        with Graph.from_hypergraph(g, stream) as G:
            ids = torch.empty(g.num_nodes, dtype=torch.int32, device="cuda")
            G.partition_device(omega, delta, ids)
            x, y, _ = G.learn_samples(ids, seed * 1_000_003 + i, per_node, with_partner=False)
            xs.append(x)
            ys.append(y)
    x = torch.cat(xs)
    y = torch.cat(ys)
    # one fixed shuffle so that consecutive minibatches mix graphs and nodes
    gen = torch.Generator(device="cpu").manual_seed(int(seed))
    perm = torch.randperm(x.shape[0], generator=gen).to(x.device)
    x = x[perm].contiguous()
    y = y[perm].contiguous()
    if init_params is None:
        # seeded start: W1 uniform in +-1/sqrt(8), W2 uniform in +-1/8, biases 0
        # (an all-zero start never breaks the hidden units' symmetry)
        rng = np.random.default_rng(seed)
        params = np.zeros(HGP_MLP_PARAMS, np.float32)
        params[:512] = rng.uniform(-1, 1, size=512) / np.sqrt(8.0)
        params[576:640] = rng.uniform(-1, 1, size=64) / 8.0
    else:
        params = np.array(init_params, dtype=np.float32)
    adam = np.zeros(2 * HGP_MLP_PARAMS, np.float32)
    torch.cuda.synchronize()
    losses = hgp_train_mlp(x, y, params, adam, steps, batch, lr, stream=stream)
    return hgp_model_from_params(params, key_bits), losses
