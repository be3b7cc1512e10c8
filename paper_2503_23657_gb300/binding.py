"""ctypes binding of libbte (include/bte.h).

Argument marshalling only: every step of the solve runs in libbte's CUDA
kernels.  There is no CPU fallback -- ``load()`` raises if the shared
library is missing or no CUDA device is visible.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbte.so")

BTE_OK = 0
BTE_EINVAL = -1
BTE_ENOMEM = -2
BTE_ECUDA = -3
BTE_ENOTCONVERGED = -4
BTE_ETIMEOUT = -5
BTE_ENUMERIC = -6
BTE_ESTATE = -7
BTE_ECORRUPT = -8
BTE_FP32 = 0
BTE_FP64 = 1

ERROR_NAMES = {
    BTE_EINVAL: "EINVAL", BTE_ENOMEM: "ENOMEM", BTE_ECUDA: "ECUDA",
    BTE_ENOTCONVERGED: "ENOTCONVERGED", BTE_ETIMEOUT: "ETIMEOUT",
    BTE_ENUMERIC: "ENUMERIC", BTE_ESTATE: "ESTATE", BTE_ECORRUPT: "ECORRUPT",
}

# every entry point declared in include/bte.h
EXPORTS = ["bte_create", "bte_solve", "bte_adjoint", "bte_destroy", "bte_last_error",
           "bte_version", "bte_default_opts", "bte_eps_history", "bte_profile_sweep",
           "bte_set_sweep_timing", "bte_eps_T_noalloc", "bte_batch_create", "bte_batch_solve",
           "bte_batch_destroy", "bte_batch_last_error", "bte_batch_set_sweep_timing", "bte_adjoint_ex",
           "bte_transient", "bte_debug_set_wait_limit", "bte_get_state", "bte_debug_overwrite_guard",
           "bte_face_count", "bte_shard_begin", "bte_shard_sweep", "bte_shard_apply"]


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("length", ctypes.c_double * 3)]


class Bands(ctypes.Structure):
    _fields_ = [("B", ctypes.c_int), ("C", ctypes.c_void_p), ("v", ctypes.c_void_p),
                ("tau", ctypes.c_void_p), ("R", ctypes.c_int), ("tau_scale", ctypes.c_void_p)]


class Quad(ctypes.Structure):
    _fields_ = [("D", ctypes.c_int), ("s", ctypes.c_void_p), ("w", ctypes.c_void_p)]


class BCs(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int * 6), ("T", ctypes.c_double * 6)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("T_init", ctypes.c_void_p), ("T_init_uniform", ctypes.c_double),
                ("Q_amp", ctypes.c_double), ("tau", ctypes.c_void_p), ("T_wall", ctypes.c_void_p),
                ("stream", ctypes.c_void_p), ("poll_every", ctypes.c_int),
                ("dirs_per_lane", ctypes.c_int), ("store_e_every_iter", ctypes.c_int),
                ("tile_kind", ctypes.c_int), ("dirs_per_cta", ctypes.c_int), ("source_staging", ctypes.c_int),
                ("warps_z", ctypes.c_int), ("lane_axis", ctypes.c_int), ("face_order", ctypes.c_int),
                ("Q_amp_each", ctypes.c_void_p), ("ein_init", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("eps_T", ctypes.c_double),
                ("T_max", ctypes.c_double), ("seconds", ctypes.c_double),
                ("updates_per_s", ctypes.c_double), ("dirs_per_lane", ctypes.c_int),
                ("kernel_launches", ctypes.c_longlong), ("tile_kind", ctypes.c_int),
                ("dirs_per_cta", ctypes.c_int), ("sweep_seconds", ctypes.c_double),
                ("sweep_launches", ctypes.c_longlong), ("source_staged", ctypes.c_int),
                ("warps_z", ctypes.c_int), ("lane_axis", ctypes.c_int), ("eps_q", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


class BatchStats(ctypes.Structure):
    _fields_ = [("instances", ctypes.c_int), ("converged", ctypes.c_int), ("max_iterations", ctypes.c_int),
                ("seconds", ctypes.c_double), ("updates", ctypes.c_double), ("updates_per_s", ctypes.c_double),
                ("kernel_launches", ctypes.c_longlong), ("classes", ctypes.c_int),
                ("sweep_seconds", ctypes.c_double), ("sweep_iterations", ctypes.c_longlong)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def load(path: str = LIB_PATH):
    """Load libbte.so (built in-tree by ``paper_2503_23657_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libbte.so not built ({path}); run paper_2503_23657_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.bte_create.argtypes = [ctypes.POINTER(Grid), vp, ctypes.POINTER(Bands), ctypes.POINTER(Quad),
                               ctypes.POINTER(BCs), vp, ctypes.POINTER(vp)]
    lib.bte_create.restype = ip
    lib.bte_solve.argtypes = [vp, ctypes.POINTER(SolveOpts), vp, vp, vp, ctypes.POINTER(Stats)]
    lib.bte_solve.restype = ip
    lib.bte_adjoint.argtypes = [vp, vp, dp, ip, vp, vp, vp, ctypes.POINTER(Stats)]
    lib.bte_adjoint.restype = ip
    lib.bte_destroy.argtypes = [vp]
    lib.bte_destroy.restype = None
    lib.bte_last_error.argtypes = [vp]
    lib.bte_last_error.restype = ctypes.c_char_p
    lib.bte_version.argtypes = []
    lib.bte_version.restype = ctypes.c_char_p
    lib.bte_default_opts.argtypes = [ctypes.POINTER(SolveOpts)]
    lib.bte_default_opts.restype = None
    lib.bte_eps_history.argtypes = [vp, vp, ip]
    lib.bte_eps_history.restype = ip
    lib.bte_profile_sweep.argtypes = [vp, ip, ctypes.POINTER(dp)]
    lib.bte_profile_sweep.restype = ip
    lib.bte_set_sweep_timing.argtypes = [vp, ip]
    lib.bte_set_sweep_timing.restype = ip
    lib.bte_batch_create.argtypes = [ip, ctypes.POINTER(vp), ctypes.POINTER(vp)]
    lib.bte_batch_create.restype = ip
    lib.bte_batch_solve.argtypes = [vp, ctypes.POINTER(SolveOpts), vp, vp, ctypes.POINTER(BatchStats)]
    lib.bte_batch_solve.restype = ip
    lib.bte_batch_destroy.argtypes = [vp]
    lib.bte_batch_destroy.restype = None
    lib.bte_batch_last_error.argtypes = [vp]
    lib.bte_batch_last_error.restype = ctypes.c_char_p
    lib.bte_batch_set_sweep_timing.argtypes = [vp, ip]
    lib.bte_batch_set_sweep_timing.restype = ip
    lib.bte_eps_T_noalloc.argtypes = [vp, vp, vp, ctypes.c_longlong, vp, vp]
    lib.bte_eps_T_noalloc.restype = ip
    lib.bte_adjoint_ex.argtypes = [vp, vp, dp, ip, vp, vp, vp, vp, ctypes.POINTER(Stats)]
    lib.bte_adjoint_ex.restype = ip
    lib.bte_transient.argtypes = [vp, ctypes.POINTER(SolveOpts), dp, ip, vp, vp, ctypes.POINTER(Stats)]
    lib.bte_transient.restype = ip
    lib.bte_debug_set_wait_limit.argtypes = [vp, ctypes.c_longlong]
    lib.bte_debug_set_wait_limit.restype = ip
    lib.bte_get_state.argtypes = [vp, vp, vp]
    lib.bte_get_state.restype = ip
    lib.bte_debug_overwrite_guard.argtypes = [vp]
    lib.bte_debug_overwrite_guard.restype = ip
    lib.bte_face_count.argtypes = [vp]
    lib.bte_face_count.restype = ip
    lib.bte_shard_begin.argtypes = [vp, ctypes.POINTER(SolveOpts)]
    lib.bte_shard_begin.restype = ip
    lib.bte_shard_sweep.argtypes = [vp, ip, ip, vp]
    lib.bte_shard_sweep.restype = ip
    lib.bte_shard_apply.argtypes = [vp, vp, vp, ctypes.POINTER(ctypes.c_double)]
    lib.bte_shard_apply.restype = ip
    _lib = lib
    return lib


class BTEError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def eps_T_noalloc(T_old, T_new, out, mask=None, stream=None):
    """bte_eps_T_noalloc: eps_T of two device temperature fields, written to
    the device buffer ``out`` (3 doubles), without any device allocation --
    for callers that cannot call cudaMalloc where they need the measure."""
    import torch

    n = int(T_new.numel())
    for name, t, dt, size in (("T_old", T_old, torch.float64, n), ("T_new", T_new, torch.float64, n),
                              ("out", out, torch.float64, 3), ("mask", mask, torch.uint8, n)):
        if t is None and name == "mask":
            continue
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"eps_T_noalloc: {name} must be a CUDA tensor")
        if t.dtype != dt or not t.is_contiguous():
            raise TypeError(f"eps_T_noalloc: {name} must be a contiguous {dt} tensor")
        if (t.numel() < size) if name == "out" else (t.numel() != size):
            raise ValueError(f"eps_T_noalloc: {name} has {t.numel()} elements, expected {size}")
    lib = load()
    rc = lib.bte_eps_T_noalloc(_addr(T_old), _addr(T_new), _addr(mask), n, _addr(out), stream)
    if rc != BTE_OK:
        raise BTEError(rc, lib.bte_last_error(None).decode())
    return rc


def _addr(x):
    """Address of a numpy array or a torch tensor (host or device)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError(f"unsupported buffer type {type(x)}")


class Plan:
    """A libbte plan for one problem (``bte_inputs.Problem`` layout)."""

    def __init__(self, problem):
        lib = load()
        p = problem
        self.problem = p
        self._keep = dict(
            mask=np.ascontiguousarray(p.mask, dtype=np.uint8),
            C=np.ascontiguousarray(p.C, dtype=np.float64),
            v=np.ascontiguousarray(p.v, dtype=np.float64),
            tau=np.ascontiguousarray(p.tau, dtype=np.float64),
            tau_scale=np.ascontiguousarray(p.tau_scale, dtype=np.float64),
            s=np.ascontiguousarray(p.s, dtype=np.float64).reshape(-1),
            w=np.ascontiguousarray(p.w, dtype=np.float64),
            phi=None if p.phi is None else np.ascontiguousarray(p.phi, dtype=np.float64),
        )
        k = self._keep
        g = Grid()
        g.dim = p.dim
        for a in range(3):
            g.n[a] = int(p.n[a])
            g.length[a] = float(p.length[a])
        bands = Bands(p.B, _addr(k["C"]), _addr(k["v"]), _addr(k["tau"]), int(k["tau_scale"].size),
                      _addr(k["tau_scale"]))
        quad = Quad(p.D, _addr(k["s"]), _addr(k["w"]))
        bcs = BCs()
        for f in range(6):
            bcs.type[f] = int(p.bc_type[f])
            bcs.T[f] = float(p.bc_T[f])
        out = ctypes.c_void_p()
        rc = lib.bte_create(ctypes.byref(g), _addr(k["mask"]), ctypes.byref(bands), ctypes.byref(quad),
                            ctypes.byref(bcs), _addr(k["phi"]), ctypes.byref(out))
        if rc != BTE_OK:
            raise BTEError(rc, lib.bte_last_error(None).decode())
        self._h = out.value
        self._lib = lib

    def close(self):
        if getattr(self, "_h", None):
            self._lib.bte_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def error(self) -> str:
        return self._lib.bte_last_error(self._h).decode()

    def _opts(self, precision, tol, max_iter, T_init, T_init_uniform, Q_amp, tau, T_wall, stream, poll_every,
              dirs_per_lane, store_e_every_iter, tile_kind, dirs_per_cta, source_staging, warps_z, lane_axis,
              face_order, keep, ein_init=None):
        p = self.problem
        o = SolveOpts()
        self._lib.bte_default_opts(ctypes.byref(o))
        o.precision = precision
        o.tol = tol
        o.max_iter = max_iter
        o.T_init = _addr(T_init)
        o.T_init_uniform = p.T_init if T_init_uniform is None else T_init_uniform
        o.Q_amp = p.Q_amp if Q_amp is None else Q_amp
        tau_a = None if tau is None else np.ascontiguousarray(tau, dtype=np.float64)
        tw_a = None if T_wall is None else np.ascontiguousarray(T_wall, dtype=np.float64)
        keep += [tau_a, tw_a]
        o.tau = _addr(tau_a)
        o.T_wall = _addr(tw_a)
        o.stream = stream
        o.poll_every = poll_every
        o.dirs_per_lane = dirs_per_lane
        o.store_e_every_iter = 1 if store_e_every_iter else 0
        o.tile_kind = tile_kind
        o.dirs_per_cta = dirs_per_cta
        o.source_staging = source_staging
        o.warps_z = warps_z
        o.lane_axis = lane_axis
        o.face_order = face_order
        o.ein_init = _addr(ein_init)
        return o

    def transient(self, dt, n_steps, T_out, T_hist=None, precision=BTE_FP64, tol=1e-10, max_iter=100000,
                  T_init=None, T_init_uniform=None, Q_amp=None, tau=None, T_wall=None, stream=None, poll_every=32,
                  tile_kind=0, dirs_per_lane=0, warps_z=0, lane_axis=0, check=True):
        """Run bte_transient: n_steps implicit-Euler steps of length dt.
        Returns (rc, stats dict)."""
        keep = []
        o = self._opts(precision, tol, max_iter, T_init, T_init_uniform, Q_amp, tau, T_wall, stream, poll_every,
                       dirs_per_lane, False, tile_kind, 0, 0, warps_z, lane_axis, 1, keep)
        st = Stats()
        rc = self._lib.bte_transient(self._h, ctypes.byref(o), float(dt), int(n_steps), _addr(T_out), _addr(T_hist),
                                     ctypes.byref(st))
        if check and rc != BTE_OK:
            raise BTEError(rc, self.error())
        return rc, st.as_dict()

    def solve(self, T_out, q_out=None, e_out=None, precision=BTE_FP32, tol=1e-6, max_iter=100000,
              T_init=None, T_init_uniform=None, Q_amp=None, tau=None, T_wall=None, stream=None,
              poll_every=32, dirs_per_lane=0, store_e_every_iter=False, tile_kind=0, dirs_per_cta=0,
              source_staging=0, warps_z=0, lane_axis=0, face_order=1, ein_init=None, check=True):
        """Run bte_solve.  Buffers are numpy arrays (host) or torch tensors
        (host or CUDA) of the documented sizes; T_init with ein_init (B x F)
        resumes a state from get_state().  Returns (rc, stats dict)."""
        p = self.problem
        keep = []
        o = self._opts(precision, tol, max_iter, T_init, T_init_uniform, Q_amp, tau, T_wall, stream, poll_every,
                       dirs_per_lane, store_e_every_iter, tile_kind, dirs_per_cta, source_staging, warps_z,
                       lane_axis, face_order, keep, ein_init)
        st = Stats()
        rc = self._lib.bte_solve(self._h, ctypes.byref(o), _addr(T_out), _addr(q_out), _addr(e_out),
                                 ctypes.byref(st))
        if check and rc not in (BTE_OK,):
            raise BTEError(rc, self.error())
        return rc, st.as_dict()

    def adjoint(self, dJ_dT, tol=1e-10, max_iter=100000, check=True, lengths=False):
        """Run bte_adjoint (bte_adjoint_ex with lengths=True); returns (rc,
        g_tau [B], g_Twall [6], g_Qamp, stats), and g_L [3] last when
        lengths=True."""
        p = self.problem
        g_tau = np.zeros(p.B)
        g_Tw = np.zeros(6)
        g_Q = np.zeros(1)
        g_L = np.zeros(3) if lengths else None
        st = Stats()
        rc = self._lib.bte_adjoint_ex(self._h, _addr(dJ_dT), tol, max_iter, _addr(g_tau), _addr(g_Tw),
                                      _addr(g_Q), _addr(g_L), ctypes.byref(st))
        if check and rc != BTE_OK:
            raise BTEError(rc, self.error())
        if lengths:
            return rc, g_tau, g_Tw, float(g_Q[0]), st.as_dict(), g_L
        return rc, g_tau, g_Tw, float(g_Q[0]), st.as_dict()

    def profile_sweep(self, reps=20):
        """Mean duration (ms) of one forward sweep launch (CUDA events)."""
        ms = ctypes.c_double()
        rc = self._lib.bte_profile_sweep(self._h, reps, ctypes.byref(ms))
        if rc != BTE_OK:
            raise BTEError(rc, self.error())
        return ms.value

    def set_sweep_timing(self, every=1):
        """bte_set_sweep_timing: bracket the sweep launch of every `every`-th
        iteration with CUDA events (0 = off); stats then carry sweep_seconds /
        sweep_launches."""
        rc = self._lib.bte_set_sweep_timing(self._h, int(every))
        if rc != BTE_OK:
            raise BTEError(rc, self.error())

    def shard_begin(self, precision=BTE_FP32, T_init=None, T_init_uniform=None, Q_amp=None, tau=None,
                    T_wall=None, stream=None, tile_kind=0, dirs_per_lane=0, dirs_per_cta=0, source_staging=0,
                    warps_z=0, lane_axis=0, ein_init=None):
        """bte_shard_begin: the initial state of a band-sharded solve."""
        keep = []
        o = self._opts(precision, 0.0, 1, T_init, T_init_uniform, Q_amp, tau, T_wall, stream, 32, dirs_per_lane,
                       False, tile_kind, dirs_per_cta, source_staging, warps_z, lane_axis, 1, keep, ein_init)
        rc = self._lib.bte_shard_begin(self._h, ctypes.byref(o))
        if rc != BTE_OK:
            raise BTEError(rc, self.error())

    def shard_sweep(self, b0, b1, W_out):
        """bte_shard_sweep: sweep bands [b0, b1); W_out [N] receives their
        band-weighted sums."""
        rc = self._lib.bte_shard_sweep(self._h, int(b0), int(b1), _addr(W_out))
        if rc != BTE_OK:
            raise BTEError(rc, self.error())

    def shard_apply(self, W, T_out=None):
        """bte_shard_apply: T^{n+1} from W (every band's sums); returns eps_T."""
        eps = ctypes.c_double()
        rc = self._lib.bte_shard_apply(self._h, _addr(W), _addr(T_out), ctypes.byref(eps))
        if rc != BTE_OK:
            raise BTEError(rc, self.error())
        return eps.value

    def n_faces(self):
        """bte_face_count: the number of boundary faces F."""
        return int(self._lib.bte_face_count(self._h))

    def get_state(self):
        """bte_get_state: (T [N], e_in [B, F]) of the last solve's final
        iterate, the checkpoint that solve(T_init=T, ein_init=e_in) resumes."""
        p = self.problem
        T = np.zeros(p.n_cells)
        F = self.n_faces()
        ein = np.zeros((p.B, max(F, 0)))
        rc = self._lib.bte_get_state(self._h, _addr(T), _addr(ein) if F > 0 else None)
        if rc != BTE_OK:
            raise BTEError(rc, self.error())
        return T, ein

    def debug_overwrite_guard(self):
        """bte_debug_overwrite_guard (test hook, BTE_DEBUG set): overwrite one
        guard byte so that the next solve reports BTE_ECORRUPT."""
        rc = self._lib.bte_debug_overwrite_guard(self._h)
        if rc != BTE_OK:
            raise BTEError(rc, self.error())

    def set_wait_limit(self, polls):
        """bte_debug_set_wait_limit (test hook): polls before a row-pipeline
        wait gives up (0: the default)."""
        rc = self._lib.bte_debug_set_wait_limit(self._h, int(polls))
        if rc != BTE_OK:
            raise BTEError(rc, self.error())

    def eps_history(self, n):
        out = np.zeros(n)
        m = self._lib.bte_eps_history(self._h, _addr(out), n)
        if m < 0:
            raise BTEError(m, "eps history")
        return out[:m]


class Batch:
    """A batch of 2D plans solved together (bte_batch_create / bte_batch_solve).
    The plans must outlive the batch."""

    def __init__(self, plans):
        lib = load()
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[pl._h for pl in self.plans])
        out = ctypes.c_void_p()
        rc = lib.bte_batch_create(len(self.plans), arr, ctypes.byref(out))
        if rc != BTE_OK:
            raise BTEError(rc, lib.bte_batch_last_error(None).decode())
        self._h = out.value
        self._lib = lib
        self.n_cells = [pl.problem.n_cells for pl in self.plans]
        self.offsets = np.concatenate([[0], np.cumsum(self.n_cells)]).astype(np.int64)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.bte_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def error(self) -> str:
        return self._lib.bte_batch_last_error(self._h).decode()

    def set_sweep_timing(self, on=True):
        rc = self._lib.bte_batch_set_sweep_timing(self._h, 1 if on else 0)
        if rc != BTE_OK:
            raise BTEError(rc, self.error())

    def solve(self, T_out, precision=BTE_FP32, tol=1e-6, max_iter=100000, T_init_uniform=300.0, Q_amp=None,
              tau=None, stream=None, poll_every=32, dirs_per_lane=0, dirs_per_cta=0, check=True):
        """Run bte_batch_solve.  T_out holds sum(n_cells) doubles (numpy or
        torch, host or CUDA), instances concatenated in plan order.  Q_amp:
        None = each instance's own problem's amplitude, a number = that one
        for all, a sequence = one per instance.  Returns (rc, [per-instance
        stats], batch stats)."""
        o = SolveOpts()
        self._lib.bte_default_opts(ctypes.byref(o))
        o.precision = precision
        o.tol = tol
        o.max_iter = max_iter
        o.T_init_uniform = T_init_uniform
        if Q_amp is None:
            Q_amp = [pl.problem.Q_amp for pl in self.plans]
        q_a = None
        if np.ndim(Q_amp) == 0:
            o.Q_amp = float(Q_amp)
        else:
            q_a = np.ascontiguousarray(Q_amp, dtype=np.float64)
            if q_a.shape != (len(self.plans),):
                raise ValueError("Q_amp: one amplitude per instance")
            o.Q_amp = 0.0
            o.Q_amp_each = _addr(q_a)
        tau_a = None if tau is None else np.ascontiguousarray(tau, dtype=np.float64)
        o.tau = _addr(tau_a)
        o.stream = stream
        o.poll_every = poll_every
        o.dirs_per_lane = dirs_per_lane
        o.dirs_per_cta = dirs_per_cta
        o.tile_kind = 0
        st = (Stats * len(self.plans))()
        bs = BatchStats()
        rc = self._lib.bte_batch_solve(self._h, ctypes.byref(o), _addr(T_out), ctypes.cast(st, ctypes.c_void_p),
                                       ctypes.byref(bs))
        if check and rc != BTE_OK:
            raise BTEError(rc, self.error())
        return rc, [s.as_dict() for s in st], bs.as_dict()
