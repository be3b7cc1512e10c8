"""FP64 CPU oracle for the steady RTA phonon BTE (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library in ``paper_2503_23657_gb300``; both read their inputs from
``bte_inputs``, which holds no solver arithmetic.

Two independent parts:

* ``solve`` / ``adjoint`` wrap ``bte_oracle.c``: the paper's outer source
  iteration (Methods, solution procedure) with exact per-(band, direction)
  upwind sweeps -- with step faces, or with the second-order Green-Gauss
  faces of "Spatial discretization" as a deferred correction
  (``problem.order = 2``) -- and the transposed fixed-point iteration of the
  discrete adjoint (Forward and inverse modelling workflow), with the
  gradients w.r.t. tau_b, the wall temperatures, the source amplitude and
  the domain lengths.
* ``transient`` wraps the implicit-Euler time stepping of the transient BTE
  (the extension the paper's Conclusion announces).
* ``dense`` assembles the linear system (L - P W - R) e = s that the
  iteration converges to and solves it directly (tiny grids only).

Parity status: the iterative solver and the direct solve are pinned against
closed forms (ballistic limit, diffusive limit), invariants (scattering
conservation, global energy balance, mirror symmetry), each other, a
continuum integral-equation solution of the gray slab, and central finite
differences; see ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bte_oracle.c")
_LIB = os.path.join(_HERE, "_bte_oracle.so")


def compile_c(src: str, out: str) -> str:
    """gcc, plain -O2, no FP contraction, so x86 and Arm hosts round alike."""
    tmp = out + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
                           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the C oracle next to its source (idempotent)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        compile_c(_SRC, _LIB)
    return _LIB


def load_library(path: str):
    """Load a build of the oracle's C source (the default one when ``path``
    is the standard location)."""
    lib = ctypes.CDLL(path)
    lib.orc_solve.restype = ctypes.c_int
    lib.orc_adjoint.restype = ctypes.c_int
    lib.orc_transient.restype = ctypes.c_int
    return lib


class _Problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("h", ctypes.c_double * 3),
        ("mask", ctypes.c_void_p),
        ("B", ctypes.c_int),
        ("C", ctypes.c_void_p),
        ("v", ctypes.c_void_p),
        ("tau", ctypes.c_void_p),
        ("R", ctypes.c_int),
        ("tau_scale", ctypes.c_void_p),
        ("D", ctypes.c_int),
        ("s", ctypes.c_void_p),
        ("w", ctypes.c_void_p),
        ("bc_type", ctypes.c_void_p),
        ("bc_T", ctypes.c_void_p),
        ("phi", ctypes.c_void_p),
        ("Q_amp", ctypes.c_double),
        ("order", ctypes.c_int),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = load_library(build())
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _marshal(p, keep):
    """Build the C struct; ``keep`` holds the arrays alive."""
    arrs = dict(
        mask=np.ascontiguousarray(p.mask, dtype=np.uint8),
        C=np.ascontiguousarray(p.C, dtype=np.float64),
        v=np.ascontiguousarray(p.v, dtype=np.float64),
        tau=np.ascontiguousarray(p.tau, dtype=np.float64),
        tau_scale=np.ascontiguousarray(p.tau_scale, dtype=np.float64),
        s=np.ascontiguousarray(p.s, dtype=np.float64).reshape(-1),
        w=np.ascontiguousarray(p.w, dtype=np.float64),
        bc_type=np.ascontiguousarray(p.bc_type, dtype=np.int32),
        bc_T=np.ascontiguousarray(p.bc_T, dtype=np.float64),
        phi=None if p.phi is None else np.ascontiguousarray(p.phi, dtype=np.float64),
    )
    keep.append(arrs)
    st = _Problem()
    st.dim = p.dim
    for a in range(3):
        st.n[a] = int(p.n[a])
        st.h[a] = float(p.length[a]) / int(p.n[a])
    st.mask = _ptr(arrs["mask"])
    st.B = p.B
    st.C, st.v, st.tau = _ptr(arrs["C"]), _ptr(arrs["v"]), _ptr(arrs["tau"])
    st.R = int(arrs["tau_scale"].shape[0])
    st.tau_scale = _ptr(arrs["tau_scale"])
    st.D = p.D
    st.s, st.w = _ptr(arrs["s"]), _ptr(arrs["w"])
    st.bc_type, st.bc_T = _ptr(arrs["bc_type"]), _ptr(arrs["bc_T"])
    st.phi = _ptr(arrs["phi"])
    st.Q_amp = float(p.Q_amp)
    st.order = int(getattr(p, "order", 1))
    return st


def solve(p, max_iter: int = 100000, tol: float = None, T_init=None, lib=None):
    """Source iteration from T_init (default ``p.T_init``).  ``tol=None`` uses
    ``p.tol``; ``tol=0`` runs exactly ``max_iter`` iterations.

    Returns dict(T [N], e [N,B,D], q [N,3], iters, eps [iters]).
    ``lib`` selects another build of the same C source (used by the tests
    that plant mistakes in a copy of it)."""
    lib = lib or _load()
    keep = []
    st = _marshal(p, keep)
    N = p.n_cells
    T = np.empty(N)
    T[:] = p.T_init if T_init is None else T_init
    T[p.mask == 0] = 0.0
    e = np.empty((N, p.B, p.D))
    eps = np.zeros(max_iter)
    tol = p.tol if tol is None else tol
    it = lib.orc_solve(ctypes.byref(st), _ptr(T), _ptr(e), ctypes.c_int(max_iter),
                       ctypes.c_double(tol), _ptr(eps))
    if it == -2:
        raise ValueError("oracle: a specular face needs the mirror of every direction in the direction set")
    if it < 0:
        raise MemoryError("oracle: allocation failed")
    q = np.empty((N, 3))
    lib.orc_flux(ctypes.byref(st), _ptr(e), _ptr(q))
    return dict(T=T, e=e, q=q, iters=it, eps=eps[:it].copy())


def adjoint(p, e, T, g, max_iter: int = 100000, tol: float = 1e-13, want_mu: bool = False,
            lib=None):
    """Discrete adjoint of the converged state for dJ/dT = g.

    Returns dict(g_tau [B], g_Tw [6], g_Q, iters[, mu])."""
    lib = lib or _load()
    keep = []
    st = _marshal(p, keep)
    e = np.ascontiguousarray(e, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    g_tau = np.zeros(p.B)
    g_Tw = np.zeros(6)
    g_Q = ctypes.c_double(0.0)
    g_L = np.zeros(3)
    mu = np.empty_like(e) if want_mu else None
    it = lib.orc_adjoint(ctypes.byref(st), _ptr(e), _ptr(T), _ptr(g), ctypes.c_int(max_iter),
                         ctypes.c_double(tol), _ptr(g_tau), _ptr(g_Tw), ctypes.byref(g_Q),
                         _ptr(g_L), _ptr(mu))
    if it == -2:
        raise ValueError("oracle: a specular face needs the mirror of every direction in the direction set")
    if it == -3:
        raise ValueError("oracle: the adjoint is that of the first-order (step face) system")
    if it < 0:
        raise MemoryError("oracle: allocation failed")
    out = dict(g_tau=g_tau, g_Tw=g_Tw, g_Q=g_Q.value, g_L=g_L, iters=it)
    if want_mu:
        out["mu"] = mu
    return out


def transient(p, dt, n_steps, max_iter: int = 100000, tol: float = 1e-13, T_init=None, lib=None):
    """Implicit Euler time steps of the transient BTE from the equilibrium at
    T_init (default ``p.T_init``), each converged to eps_T < tol.

    Returns dict(T [N] final, e [N,B,D] final, T_hist [n_steps, N],
    iters [n_steps], total)."""
    lib = lib or _load()
    keep = []
    st = _marshal(p, keep)
    N = p.n_cells
    T = np.empty(N)
    T[:] = p.T_init if T_init is None else T_init
    T[p.mask == 0] = 0.0
    e = np.empty((N, p.B, p.D))
    T_hist = np.zeros((n_steps, N))
    iters = np.zeros(n_steps, dtype=np.int32)
    total = lib.orc_transient(ctypes.byref(st), _ptr(T), _ptr(e), ctypes.c_double(dt), ctypes.c_int(n_steps),
                              ctypes.c_int(max_iter), ctypes.c_double(tol), _ptr(T_hist), _ptr(iters))
    if total == -2:
        raise ValueError("oracle: a specular face needs the mirror of every direction in the direction set")
    if total < 0:
        raise MemoryError("oracle: allocation failed")
    return dict(T=T, e=e, T_hist=T_hist, iters=iters, total=total)


def flux(p, e, lib=None):
    lib = lib or _load()
    keep = []
    st = _marshal(p, keep)
    e = np.ascontiguousarray(e, dtype=np.float64)
    q = np.empty((p.n_cells, 3))
    lib.orc_flux(ctypes.byref(st), _ptr(e), _ptr(q))
    return q
