"""C-ABI checks that need no GPU: the library loads, exports every entry
point declared in include/bte.h, and validates inputs before touching CUDA."""
import ctypes
import os
import re

import numpy as np
import pytest

import bte_inputs as bi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2503_23657_gb300 import build, binding
    build.build()
    return binding.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "bte.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bte_[A-Za-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    from paper_2503_23657_gb300 import binding
    names = declared_functions()
    assert names, "no declarations found"
    for n in names:
        assert hasattr(lib, n), f"{n} not exported"
    assert sorted(binding.EXPORTS) == names


def test_version(lib):
    assert b"sm_103a" in lib.bte_version()


def _create(lib, p, **over):
    from paper_2503_23657_gb300 import binding as bd
    mask = np.ascontiguousarray(over.get("mask", p.mask), dtype=np.uint8)
    C = np.ascontiguousarray(over.get("C", p.C), dtype=np.float64)
    v = np.ascontiguousarray(p.v, dtype=np.float64)
    tau = np.ascontiguousarray(over.get("tau", p.tau), dtype=np.float64)
    ts = np.ascontiguousarray(p.tau_scale, dtype=np.float64)
    s = np.ascontiguousarray(p.s, dtype=np.float64).reshape(-1)
    w = np.ascontiguousarray(over.get("w", p.w), dtype=np.float64)
    g = bd.Grid()
    g.dim = over.get("dim", p.dim)
    for a in range(3):
        g.n[a] = over.get("n", p.n)[a]
        g.length[a] = p.length[a]
    bands = bd.Bands(p.B, C.ctypes.data, v.ctypes.data, tau.ctypes.data, ts.size, ts.ctypes.data)
    quad = bd.Quad(p.D, s.ctypes.data, w.ctypes.data)
    bcs = bd.BCs()
    types = over.get("bc_type", p.bc_type)
    for f in range(6):
        bcs.type[f] = int(types[f])
        bcs.T[f] = float(p.bc_T[f])
    out = ctypes.c_void_p()
    rc = lib.bte_create(ctypes.byref(g), mask.ctypes.data, ctypes.byref(bands), ctypes.byref(quad),
                        ctypes.byref(bcs), None, ctypes.byref(out))
    return rc, out.value, lib.bte_last_error(None).decode()


@pytest.mark.parametrize("case,over,frag", [
    ("weights", lambda p: dict(w=p.w * 1.01), "4 pi"),
    ("tau", lambda p: dict(tau=-p.tau), "tau"),
    ("capacity", lambda p: dict(C=0 * p.C), "C, v, tau"),
    ("mask_region", lambda p: dict(mask=np.full(p.n_cells, 3, np.uint8)), "regions"),
    ("empty_mask", lambda p: dict(mask=np.zeros(p.n_cells, np.uint8)), "no solid"),
    ("adiabatic", lambda p: dict(bc_type=[1] * 6), "isothermal"),
    ("dim", lambda p: dict(dim=4), "dim"),
    ("unused_axis", lambda p: dict(dim=1), "axes >= dim"),
])
def test_invalid_inputs_rejected_before_cuda(lib, case, over, frag):
    p = bi.tiny(2, n=(4, 3, 1), B=2)
    rc, h, msg = _create(lib, p, **over(p))
    assert rc == -1 and h is None
    assert frag in msg


def test_valid_input_reaches_the_device_step(lib):
    """With valid inputs validation passes; without a GPU the call then fails
    with ECUDA (and with a GPU it succeeds)."""
    p = bi.tiny(2, n=(4, 3, 1), B=2)
    rc, h, msg = _create(lib, p)
    assert rc in (0, -3)
    if rc == 0:
        lib.bte_destroy(ctypes.c_void_p(h))
