"""CPU-side checks of the C ABI: the library builds, loads and exports every
symbol declared in include/hgp.h (no compute calls: there is no GPU here)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "hgp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hgp_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("hgp_create", "hgp_partition", "hgp_destroy", "hgp_get_stats",
              "hgp_error_string", "hgp_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2604_14411_gb300 import _build
    from paper_2604_14411_gb300 import hgp as H
    lib_path = _build.build()
    try:
        lib = ctypes.CDLL(lib_path)
    except OSError as e:          # no CUDA driver in this container
        pytest.skip(f"cannot dlopen without the CUDA driver: {e}")
    for n in _declared():
        assert hasattr(lib, n), n
    assert set(H.EXPORTS) == set(_declared())


def test_exports_via_nm():
    """Symbol table check that works without a CUDA driver."""
    import shutil
    import subprocess
    from paper_2604_14411_gb300 import _build
    lib_path = _build.build()
    nm = shutil.which("nm")
    if not nm:
        pytest.skip("nm not available")
    out = subprocess.run([nm, "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for n in _declared():
        assert n in syms, n


def test_error_strings_without_gpu():
    from paper_2604_14411_gb300 import _build
    try:
        lib = ctypes.CDLL(_build.build())
    except OSError as e:
        pytest.skip(f"cannot dlopen without the CUDA driver: {e}")
    lib.hgp_error_string.restype = ctypes.c_char_p
    assert lib.hgp_error_string(2).decode().startswith("infeasible")
    # invalid arguments are rejected on the host before any device work
    h = ctypes.c_void_p()
    assert lib.hgp_create(0, 0, None, None, None, None, 0, None, None, ctypes.byref(h)) == 1


def test_struct_layouts_match_the_header():
    """The binding's ctypes structs have the sizes the header implies."""
    from paper_2604_14411_gb300 import hgp as H
    assert ctypes.sizeof(H.hgp_model) == 2 * (512 + 64 + 64 + 1) + 2 + 12
    assert ctypes.sizeof(H.hgp_options) == 32
    assert H.hgp_options.model.offset == 24
    assert ctypes.sizeof(H.hgp_train_options) == 40
    assert ctypes.sizeof(H.hgp_allocator) == 24
    assert H.hgp_allocator.ctx.offset == 16


def test_create_rejects_an_incomplete_allocator_on_the_host():
    """An hgp_allocator without both callbacks is refused before any device
    work (so this runs without a GPU)."""
    from paper_2604_14411_gb300 import _build
    from paper_2604_14411_gb300 import hgp as H
    _build.build()
    try:
        lib = H.load()
    except OSError as e:
        pytest.skip(f"cannot dlopen without the CUDA driver: {e}")
    import numpy as np
    off = np.array([0, 2], np.int32)
    pins = np.array([0, 1], np.int32)
    half = H.hgp_allocator()            # both callbacks NULL
    h = ctypes.c_void_p()
    rc = lib.hgp_create(2, 1, off.ctypes.data, pins.ctypes.data, None, None, 0, ctypes.byref(half),
                        None, ctypes.byref(h))
    assert rc == H.HGP_ERR_INVALID_ARG and not h.value


def test_model_from_params_rounds_to_nearest_even():
    """hgp_model_from_params is host-only; its bfloat16 rounding against the
    exact value: the nearest bfloat16, ties to an even mantissa."""
    from paper_2604_14411_gb300 import _build
    from paper_2604_14411_gb300 import hgp as H
    _build.build()
    try:
        H.load()
    except OSError as e:
        pytest.skip(f"cannot dlopen without the CUDA driver: {e}")
    import numpy as np
    rng = np.random.default_rng(0)
    p = rng.normal(size=641).astype(np.float32)
    # exact ties: bit 15 set and nothing below it
    p[:4] = (np.array([0x3F808000, 0x3F818000, 0xBF808000, 0x40000000], np.uint32)).view(np.float32)
    m = H.hgp_model_from_params(p, 7)
    got = np.concatenate([m.w1.reshape(-1), m.b1, m.w2, [m.b2]]).astype(np.uint32)
    exact = p.astype(np.float64)
    lo = (p.view(np.uint32) >> 16).astype(np.uint32)
    for q in range(641):
        cands = [int(lo[q]), int(lo[q]) + 1]
        vals = [(np.uint32(c) << 16).view(np.float32).astype(np.float64) for c in cands]
        d = [abs(v - exact[q]) for v in vals]
        if d[0] != d[1]:
            assert got[q] == cands[int(d[1] < d[0])], q
        else:
            assert got[q] == cands[0] if cands[0] % 2 == 0 else cands[1], q
    assert m.key_bits == 7
    assert got[:4].tolist() == [0x3F80, 0x3F82, 0xBF80, 0x4000]
    with pytest.raises(H.HgpError):
        H.hgp_model_from_params(p, 21)


def test_binding_constants_match_the_header():
    """Every integer #define of include/hgp.h that the binding mirrors has the
    header's value, and every flag and debug bit is mirrored."""
    from paper_2604_14411_gb300 import hgp as H
    src = open(os.path.join(ROOT, "include", "hgp.h")).read()
    defs = {k: int(v, 0) for k, v in re.findall(r"#define\s+(HGP_[A-Z0-9_]+)\s+(0x[0-9a-fA-F]+|\d+)u?\b", src)}
    assert defs, "no #define constants found"
    mirrored = 0
    for name, value in defs.items():
        if hasattr(H, name):
            assert getattr(H, name) == value, name
            mirrored += 1
        else:
            assert not name.startswith(("HGP_DEBUG_", "HGP_DELTA_", "HGP_ERR_")), f"{name} not in the binding"
    assert mirrored >= 10
    bits = [v for k, v in defs.items() if k.startswith("HGP_DEBUG_")]
    assert all(b & (b - 1) == 0 for b in bits) and len(set(bits)) == len(bits)   # distinct single bits
