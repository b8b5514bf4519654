"""Python binding of the GB300 EREM library (``liberem.so``, C ABI in include/erem.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels and host C++ code.  The functions below carry the names of the
C entry points and take torch tensors (CUDA or CPU) or numpy arrays of FP64
values, contiguous, x fastest; CPU arrays are staged by the library.  The
library must have been built (``__graft_entry__.build()`` or
``python paper_1209_5553_gb300/build.py``); importing this package without it
raises ImportError.  There is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liberem.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`"
    )
_lib = ctypes.CDLL(LIB_PATH)

# status codes (erem_status)
EREM_OK, EREM_EINVAL, EREM_ENOMEM, EREM_ENOTCONV, EREM_ETIMEOUT, EREM_ENONFINITE, EREM_ECUDA = range(7)
STATUS_NAMES = {0: "EREM_OK", 1: "EREM_EINVAL", 2: "EREM_ENOMEM", 3: "EREM_ENOTCONV",
                4: "EREM_ETIMEOUT", 5: "EREM_ENONFINITE", 6: "EREM_ECUDA"}
EREM_FP64, EREM_FP32_BULK = 0, 1
EREM_ROSM1, EREM_ROSM_HALF, EREM_ROS2, EREM_ROS3P = 0, 1, 2, 3
EREM_LEJA_EXACT, EREM_LEJA_FAST = 0, 1
EREM_SUBSTEPS_FROM_ONE, EREM_SUBSTEPS_FROM_LAST = 0, 1
EREM_SPLIT_TROTTER, EREM_SPLIT_STRANG = 0, 1


class erem_grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("lx", ctypes.c_double), ("ly", ctypes.c_double),
                ("lz", ctypes.c_double)]


class erem_physics(ctypes.Structure):
    _fields_ = [("rhoc_f", ctypes.c_double), ("rhoc_s", ctypes.c_double),
                ("head_left", ctypes.c_double), ("head_right", ctypes.c_double),
                ("T_inflow", ctypes.c_double), ("fluid_model", ctypes.c_int)]


class erem_leja_opts(ctypes.Structure):
    _fields_ = [("tol_a", ctypes.c_double), ("tol_r", ctypes.c_double),
                ("p_order", ctypes.c_int), ("m_max", ctypes.c_int),
                ("max_doublings", ctypes.c_int), ("avg_window", ctypes.c_int),
                ("replay", ctypes.POINTER(ctypes.c_int)), ("n_replay", ctypes.c_int),
                ("time_terms", ctypes.c_int)]


class erem_stats(ctypes.Structure):
    _fields_ = [("substeps", ctypes.c_int), ("degree_total", ctypes.c_int),
                ("degrees", ctypes.c_int * 64), ("alpha", ctypes.c_double),
                ("beta", ctypes.c_double), ("err_est", ctypes.c_double),
                ("lin_iters", ctypes.c_int), ("lin_resid", ctypes.c_double),
                ("flux_in", ctypes.c_double), ("vmax", ctypes.c_double),
                ("t_ms", ctypes.c_double), ("t_terms_ms", ctypes.c_double),
                ("n_terms_timed", ctypes.c_int), ("launches", ctypes.c_int),
                ("n_launches_timed", ctypes.c_int), ("degree_phi2", ctypes.c_int),
                ("terms_lagged", ctypes.c_int)]

    @property
    def schedule(self):
        return [self.substeps] + [self.degrees[k] for k in range(self.substeps)]

    @property
    def schedule_forced(self):
        """[s, m_1..m_s, m_phi2] of erem_step_forced (its replay format)."""
        return self.schedule + [self.degree_phi2]


class erem_adapt_stats(ctypes.Structure):
    _fields_ = [("accepted", ctypes.c_int), ("rejected", ctypes.c_int), ("lin_iters", ctypes.c_int),
                ("launches", ctypes.c_int), ("t_reached", ctypes.c_double),
                ("dt_min", ctypes.c_double), ("dt_max", ctypes.c_double), ("t_ms", ctypes.c_double)]


class erem_krylov_opts(ctypes.Structure):
    _fields_ = [("tol_a", ctypes.c_double), ("tol_r", ctypes.c_double), ("m", ctypes.c_int),
                ("max_substeps", ctypes.c_int), ("replay", ctypes.POINTER(ctypes.c_double)),
                ("n_replay", ctypes.c_int)]


class erem_krylov_stats(ctypes.Structure):
    _fields_ = [("substeps", ctypes.c_int), ("rejections", ctypes.c_int),
                ("dims", ctypes.c_int * 64), ("deltas", ctypes.c_double * 64),
                ("err", ctypes.c_double * 64), ("t_ms", ctypes.c_double),
                ("launches", ctypes.c_int), ("pad", ctypes.c_int)]

    @property
    def schedule(self):
        """Substep lengths (the first 64), for replay."""
        return [self.deltas[k] for k in range(min(self.substeps, 64))]


EREM_ENS_KEEP_SUBSTEPS, EREM_ENS_RESTART_SUBSTEPS = 0, 1


class erem_ens_config(ctypes.Structure):
    _fields_ = [("substep_policy", ctypes.c_int), ("cluster_ctas", ctypes.c_int),
                ("max_clusters", ctypes.c_int), ("reserved", ctypes.c_int)]


class erem_ens_member_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("steps_done", ctypes.c_int),
                ("substeps", ctypes.c_int), ("degree_total", ctypes.c_int),
                ("degrees", ctypes.c_int * 64), ("terms", ctypes.c_int),
                ("passes", ctypes.c_int), ("attempts", ctypes.c_int),
                ("leja_coefficients", ctypes.c_int),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double)]

    @property
    def schedule(self):
        return [self.substeps] + [self.degrees[k] for k in range(self.substeps)]


class erem_ens_run_stats(ctypes.Structure):
    _fields_ = [("t_ms", ctypes.c_double), ("passes", ctypes.c_longlong),
                ("cells", ctypes.c_longlong), ("cell_terms", ctypes.c_longlong),
                ("cell_passes", ctypes.c_longlong), ("cluster_ctas", ctypes.c_int),
                ("clusters", ctypes.c_int), ("cta_threads", ctypes.c_int),
                ("members_failed", ctypes.c_int), ("graph", ctypes.c_int), ("reserved", ctypes.c_int)]


_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_sigs = {
    "erem_default_leja_opts": (None, [ctypes.POINTER(erem_leja_opts)]),
    "erem_create": (_I, [ctypes.POINTER(erem_grid), ctypes.POINTER(erem_physics), _I,
                         ctypes.POINTER(_P)]),
    "erem_destroy": (_I, [_P]),
    "erem_set_physics": (_I, [_P, ctypes.POINTER(erem_physics)]),
    "pressure_solve": (_I, [_P, _P, _P, _P, _D, _I, ctypes.POINTER(erem_stats), _P]),
    "erem_set_state": (_I, [_P, _P, _P, _P, _P, _P, _D, _P]),
    "phi1_apply": (_I, [_P, _P, _P, ctypes.POINTER(erem_leja_opts), ctypes.POINTER(erem_stats), _P]),
    "erem_step": (_I, [_P, _P, _P, _P, _P, _P, _D, ctypes.POINTER(erem_leja_opts),
                       ctypes.POINTER(erem_stats), _P]),
    "rosm_step": (_I, [_P, _P, _P, _P, _P, _P, _D, _I, _D, _I, ctypes.POINTER(erem_stats), _P]),
    "erem_last_error": (ctypes.c_char_p, [_P]),
    "erem_leja_coefficients": (_I, [_P]),
    "erem_leja_points": (_I, [_I, ctypes.POINTER(_D)]),
    "erem_fast_leja_points": (_I, [_I, ctypes.POINTER(_D)]),
    "erem_phi2_divided_differences": (_I, [_I, ctypes.POINTER(_D), _D, _D, ctypes.POINTER(_D)]),
    "coupled_step": (_I, [_P, _P, _P, _P, _P, _P, _P, _D, _I, _D, _I, ctypes.POINTER(erem_leja_opts),
                          ctypes.POINTER(erem_stats), ctypes.POINTER(erem_stats), _P]),
    "rosm_integrate": (_I, [_P, _P, _D, _D, _I, _D, _D, _D, _I, _I, ctypes.POINTER(_D),
                            ctypes.POINTER(erem_adapt_stats), _P]),
    "erem_step_forced": (_I, [_P, _P, _D, _D, _D, _P, _P, _P, _P, ctypes.POINTER(erem_leja_opts),
                              ctypes.POINTER(erem_stats), _P]),
    "erem_set_leja_points": (_I, [_P, _I]),
    "erem_set_substep_start": (_I, [_P, _I]),
    "erem_phi1_divided_differences": (_I, [_I, ctypes.POINTER(_D), _D, _D, ctypes.POINTER(_D)]),
    "erem_pressure_solve_static": (_I, [ctypes.POINTER(erem_grid), ctypes.POINTER(erem_physics),
                                        _P, _P, _P, _D, _I, ctypes.POINTER(erem_stats), _P]),
    "erem_default_krylov_opts": (None, [ctypes.POINTER(erem_krylov_opts)]),
    "phi1_apply_krylov": (_I, [_P, _P, _P, ctypes.POINTER(erem_krylov_opts),
                               ctypes.POINTER(erem_krylov_stats), _P]),
    "erem_step_krylov": (_I, [_P, _P, _P, _P, _P, _P, _D, ctypes.POINTER(erem_krylov_opts),
                              ctypes.POINTER(erem_krylov_stats), _P]),
    "erem_hold_interval": (_I, [_P, _I, _D, _D]),
    "erem_set_pressure_precond": (_I, [_P, _I]),
    "erem_set_pressure_multigrid": (_I, [_P, _I, _D]),
    "erem_set_stage_precond": (_I, [_P, _I]),
    "erem_set_host_access": (_I, [_P, _I]),
    "erem_adjoint_tape": (_I, [_P, ctypes.c_size_t, _I]),
    "erem_adjoint_begin": (_I, [_P, _P]),
    "erem_adjoint_step": (_I, [_P, _P, _P, ctypes.POINTER(ctypes.c_int), _I, _P]),
    "erem_adjoint_lnk": (_I, [_P, _P, _P, _D, _I, ctypes.POINTER(erem_stats), _P]),
    "erem_ensemble_create": (_I, [_I, ctypes.POINTER(erem_grid), ctypes.POINTER(erem_physics), _I,
                                  ctypes.POINTER(_P)]),
    "erem_ensemble_destroy": (_I, [_P]),
    "erem_ensemble_set_member": (_I, [_P, _I, _P, _P, _P, _P, _P, _D, _P]),
    "erem_ensemble_get_member": (_I, [_P, _I, _P, _P]),
    "erem_ensemble_set_temperature": (_I, [_P, _I, _P, _P]),
    "erem_ensemble_configure": (_I, [_P, ctypes.POINTER(erem_leja_opts),
                                     ctypes.POINTER(erem_ens_config)]),
    "erem_ensemble_autotune": (_I, [_P, _I, _P]),
    "erem_ensemble_run": (_I, [_P, _I, _P]),
    "erem_ensemble_member_stats": (_I, [_P, _I, ctypes.POINTER(erem_ens_member_stats)]),
    "erem_ensemble_run_stats": (_I, [_P, ctypes.POINTER(erem_ens_run_stats)]),
    "erem_ensemble_last_error": (ctypes.c_char_p, [_P]),
}
for _name, (_res, _args) in _sigs.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_sigs)


class EremError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _ptr(x, n: int | None):
    """Raw pointer of an FP64 contiguous array (torch tensor or numpy array)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"]:
            raise TypeError("numpy arrays must be contiguous float64")
        if n is not None and x.size != n:
            raise ValueError(f"array has {x.size} entries, expected {n}")
        return x.ctypes.data
    import torch

    if isinstance(x, torch.Tensor):
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise TypeError("tensors must be contiguous float64")
        if n is not None and x.numel() != n:
            raise ValueError(f"tensor has {x.numel()} entries, expected {n}")
        return x.data_ptr()
    raise TypeError(f"unsupported array type {type(x)}")


def _stream(stream):
    if stream is not None:
        return getattr(stream, "cuda_stream", stream)
    try:
        import torch

        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None


def leja_opts(tol=1e-6, tol_a=None, tol_r=None, p_order=2, m_max=150, max_doublings=6,
              avg_window=5, replay=None, time_terms=False):
    """erem_leja_opts with the given fields (replay = [s, m_1..m_s] or None)."""
    o = erem_leja_opts()
    erem_default_leja_opts(o)
    o.tol_a = tol if tol_a is None else tol_a
    o.tol_r = tol if tol_r is None else tol_r
    o.p_order, o.m_max, o.max_doublings, o.avg_window = p_order, m_max, max_doublings, avg_window
    o.time_terms = 1 if time_terms else 0
    if replay is not None:
        arr = (ctypes.c_int * len(replay))(*[int(v) for v in replay])
        o._replay_keep = arr  # keep alive with the struct
        o.replay = ctypes.cast(arr, ctypes.POINTER(ctypes.c_int))
        o.n_replay = len(replay)
    return o


# ---------------------------------------------------------------------------
# C entry points under their own names
# ---------------------------------------------------------------------------
def erem_default_leja_opts(opts: erem_leja_opts) -> None:
    _lib.erem_default_leja_opts(ctypes.byref(opts))


def erem_create(grid: erem_grid, phys: erem_physics, precision: int = EREM_FP64):
    h = _P()
    st = _lib.erem_create(ctypes.byref(grid), ctypes.byref(phys), int(precision), ctypes.byref(h))
    if st != EREM_OK:
        raise EremError(st, "erem_create failed")
    return h


def erem_destroy(ctx) -> None:
    _lib.erem_destroy(ctx)


def erem_last_error(ctx) -> str:
    r = _lib.erem_last_error(ctx)
    return r.decode() if r else ""


def _check(ctx, st):
    if st != EREM_OK:
        raise EremError(st, erem_last_error(ctx))


def erem_set_physics(ctx, phys: erem_physics) -> None:
    _check(ctx, _lib.erem_set_physics(ctx, ctypes.byref(phys)))


def pressure_solve(ctx, n, lnk, T, p, tol=1e-10, maxit=100000, stream=None) -> erem_stats:
    st = erem_stats()
    _check(ctx, _lib.pressure_solve(ctx, _ptr(lnk, n), _ptr(T, n), _ptr(p, n), float(tol),
                                    int(maxit), ctypes.byref(st), _stream(stream)))
    return st


def erem_set_state(ctx, n, T, p, lnk, phi, lam, dt, stream=None) -> None:
    _check(ctx, _lib.erem_set_state(ctx, _ptr(T, n), _ptr(p, n), _ptr(lnk, n), _ptr(phi, n),
                                    _ptr(lam, n), float(dt), _stream(stream)))


def phi1_apply(ctx, n, v, out, opts: erem_leja_opts | None = None, stream=None) -> erem_stats:
    st = erem_stats()
    _check(ctx, _lib.phi1_apply(ctx, _ptr(v, n), _ptr(out, n),
                                ctypes.byref(opts) if opts is not None else None,
                                ctypes.byref(st), _stream(stream)))
    return st


def erem_step(ctx, n, T, dt, p=None, lnk=None, phi=None, lam=None,
              opts: erem_leja_opts | None = None, stream=None) -> erem_stats:
    st = erem_stats()
    _check(ctx, _lib.erem_step(ctx, _ptr(T, n), _ptr(p, n), _ptr(lnk, n), _ptr(phi, n),
                               _ptr(lam, n), float(dt),
                               ctypes.byref(opts) if opts is not None else None,
                               ctypes.byref(st), _stream(stream)))
    return st


def erem_step_forced(ctx, n, T, dt, T_in, T_in_rate, p=None, lnk=None, phi=None, lam=None,
                     opts: erem_leja_opts | None = None, stream=None) -> erem_stats:
    st = erem_stats()
    _check(ctx, _lib.erem_step_forced(ctx, _ptr(T, n), float(dt), float(T_in), float(T_in_rate),
                                      _ptr(p, n), _ptr(lnk, n), _ptr(phi, n), _ptr(lam, n),
                                      ctypes.byref(opts) if opts is not None else None,
                                      ctypes.byref(st), _stream(stream)))
    return st


def coupled_step(ctx, n, T, p, lnk, phi, lam, dt, splitting=EREM_SPLIT_TROTTER,
                 pressure_tol=1e-10, pressure_maxit=200000, opts=None, stream=None, T_p=None):
    """One split pressure/temperature step; opts: None or a list of one
    (Trotter) or two (Strang) erem_leja_opts; T_p: None or the temperature p
    was solved at (updated to the one the step's pressure was solved at).
    Returns (heat stats list, pressure stats)."""
    nh = 2 if splitting == EREM_SPLIT_STRANG else 1
    if opts is not None:
        if len(opts) != nh:
            raise ValueError(f"opts needs {nh} entries")
        arr = (erem_leja_opts * nh)(*opts)
    st = (erem_stats * nh)()
    pst = erem_stats()
    _check(ctx, _lib.coupled_step(ctx, _ptr(T, n), _ptr(p, n), _ptr(T_p, n), _ptr(lnk, n), _ptr(phi, n),
                                  _ptr(lam, n), float(dt), int(splitting), float(pressure_tol),
                                  int(pressure_maxit),
                                  ctypes.cast(arr, ctypes.POINTER(erem_leja_opts)) if opts is not None
                                  else None, ctypes.cast(st, ctypes.POINTER(erem_stats)),
                                  ctypes.byref(pst), _stream(stream)))
    return list(st), pst


def rosm_integrate(ctx, n, T, t_end, dt0, scheme=EREM_ROS2, tol_a=1e-6, tol_r=1e-6,
                   lin_tol=1e-10, maxit=10000, max_attempts=100000, stream=None):
    """Adaptive ROS2(1)/ROS3p over [0, t_end]; returns (erem_adapt_stats,
    accepted step lengths)."""
    st = erem_adapt_stats()
    dts = np.zeros(max_attempts)
    _check(ctx, _lib.rosm_integrate(ctx, _ptr(T, n), float(t_end), float(dt0), int(scheme),
                                    float(tol_a), float(tol_r), float(lin_tol), int(maxit),
                                    int(max_attempts), dts.ctypes.data_as(ctypes.POINTER(_D)),
                                    ctypes.byref(st), _stream(stream)))
    return st, dts[: st.accepted].copy()


def rosm_step(ctx, n, T, dt, scheme=EREM_ROS2, p=None, lnk=None, phi=None, lam=None,
              lin_tol=1e-10, maxit=10000, stream=None) -> erem_stats:
    st = erem_stats()
    _check(ctx, _lib.rosm_step(ctx, _ptr(T, n), _ptr(p, n), _ptr(lnk, n), _ptr(phi, n),
                               _ptr(lam, n), float(dt), int(scheme), float(lin_tol), int(maxit),
                               ctypes.byref(st), _stream(stream)))
    return st


def erem_leja_points(M: int) -> np.ndarray:
    out = np.zeros(M + 1)
    if _lib.erem_leja_points(int(M), out.ctypes.data_as(ctypes.POINTER(_D))) != 0:
        raise ValueError("bad M")
    return out


def erem_phi2_divided_differences(xi, c: float, gamma: float) -> np.ndarray:
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    d = np.zeros(xi.size)
    if _lib.erem_phi2_divided_differences(xi.size - 1, xi.ctypes.data_as(ctypes.POINTER(_D)),
                                          float(c), float(gamma),
                                          d.ctypes.data_as(ctypes.POINTER(_D))) != 0:
        raise ValueError("bad arguments")
    return d


def erem_fast_leja_points(M: int) -> np.ndarray:
    out = np.zeros(M + 1)
    if _lib.erem_fast_leja_points(int(M), out.ctypes.data_as(ctypes.POINTER(_D))) != 0:
        raise ValueError("bad M")
    return out


def erem_set_leja_points(ctx, kind) -> None:
    """EREM_LEJA_EXACT or EREM_LEJA_FAST (or "exact" / "fast")."""
    kind = {"exact": EREM_LEJA_EXACT, "fast": EREM_LEJA_FAST}.get(kind, kind)
    _check(ctx, _lib.erem_set_leja_points(ctx, int(kind)))


def erem_set_substep_start(ctx, mode) -> None:
    """EREM_SUBSTEPS_FROM_ONE or EREM_SUBSTEPS_FROM_LAST (or "one" / "last")."""
    mode = {"one": EREM_SUBSTEPS_FROM_ONE, "last": EREM_SUBSTEPS_FROM_LAST}.get(mode, mode)
    _check(ctx, _lib.erem_set_substep_start(ctx, int(mode)))


def erem_phi1_divided_differences(xi, c: float, gamma: float) -> np.ndarray:
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    out = np.zeros(xi.size)
    if _lib.erem_phi1_divided_differences(xi.size - 1, xi.ctypes.data_as(ctypes.POINTER(_D)),
                                          float(c), float(gamma),
                                          out.ctypes.data_as(ctypes.POINTER(_D))) != 0:
        raise ValueError("bad arguments")
    return out


def erem_pressure_solve_static(grid: erem_grid, phys: erem_physics, lnk, T, p, tol=1e-10,
                               maxit=100000, stream=None) -> erem_stats:
    """Pressure solve for callers that cannot allocate device memory: no
    context, work space in a static device array (at most 65536 padded
    cells); lnk, T and p must be CUDA tensors."""
    n = grid.nx * grid.ny * grid.nz
    st = erem_stats()
    rc = _lib.erem_pressure_solve_static(ctypes.byref(grid), ctypes.byref(phys), _ptr(lnk, n),
                                         _ptr(T, n), _ptr(p, n), float(tol), int(maxit),
                                         ctypes.byref(st), _stream(stream))
    if rc != EREM_OK:
        raise EremError(rc, "erem_pressure_solve_static failed")
    return st


def krylov_opts(tol=1e-6, tol_a=None, tol_r=None, m=10, max_substeps=1000, replay=None):
    """erem_krylov_opts with the given fields (replay = substep lengths or None)."""
    o = erem_krylov_opts()
    _lib.erem_default_krylov_opts(ctypes.byref(o))
    o.tol_a = tol if tol_a is None else tol_a
    o.tol_r = tol if tol_r is None else tol_r
    o.m, o.max_substeps = int(m), int(max_substeps)
    if replay is not None:
        arr = (ctypes.c_double * len(replay))(*[float(v) for v in replay])
        o._replay_keep = arr
        o.replay = ctypes.cast(arr, ctypes.POINTER(ctypes.c_double))
        o.n_replay = len(replay)
    return o


def erem_default_krylov_opts(opts: erem_krylov_opts) -> None:
    _lib.erem_default_krylov_opts(ctypes.byref(opts))


def phi1_apply_krylov(ctx, n, v, out, opts: erem_krylov_opts | None = None,
                      stream=None) -> erem_krylov_stats:
    st = erem_krylov_stats()
    _check(ctx, _lib.phi1_apply_krylov(ctx, _ptr(v, n), _ptr(out, n),
                                       ctypes.byref(opts) if opts is not None else None,
                                       ctypes.byref(st), _stream(stream)))
    return st


def erem_step_krylov(ctx, n, T, dt, p=None, lnk=None, phi=None, lam=None,
                     opts: erem_krylov_opts | None = None, stream=None) -> erem_krylov_stats:
    st = erem_krylov_stats()
    _check(ctx, _lib.erem_step_krylov(ctx, _ptr(T, n), _ptr(p, n), _ptr(lnk, n), _ptr(phi, n),
                                      _ptr(lam, n), float(dt),
                                      ctypes.byref(opts) if opts is not None else None,
                                      ctypes.byref(st), _stream(stream)))
    return st


def erem_hold_interval(ctx, interval) -> None:
    """Hold the Gershgorin interval (lo, hi) of J for later steps; None
    releases it."""
    if interval is None:
        _check(ctx, _lib.erem_hold_interval(ctx, 0, 0.0, 0.0))
    else:
        lo, hi = interval
        _check(ctx, _lib.erem_hold_interval(ctx, 1, float(lo), float(hi)))


def erem_set_pressure_precond(ctx, degree) -> None:
    """Pressure CG preconditioner: 0 = FP32 multigrid V-cycle (default),
    1 = Jacobi, 2..64 = FP32 Chebyshev polynomial of that degree."""
    _check(ctx, _lib.erem_set_pressure_precond(ctx, int(degree)))


def erem_adjoint_begin(ctx, stream=None) -> None:
    _check(ctx, _lib.erem_adjoint_begin(ctx, _stream(stream)))


def erem_adjoint_step(ctx, n, T, lam, schedule, stream=None) -> None:
    arr = (ctypes.c_int * len(schedule))(*[int(v) for v in schedule])
    _check(ctx, _lib.erem_adjoint_step(ctx, _ptr(T, n), _ptr(lam, n), arr, len(schedule),
                                       _stream(stream)))


def erem_adjoint_lnk(ctx, n, lnk, glnk, tol=1e-12, maxit=200000, stream=None) -> erem_stats:
    st = erem_stats()
    _check(ctx, _lib.erem_adjoint_lnk(ctx, _ptr(lnk, n), _ptr(glnk, n), float(tol), int(maxit),
                                      ctypes.byref(st), _stream(stream)))
    return st


def erem_ensemble_create(grids, physics, precision: int = EREM_FP64):
    n = len(grids)
    ga = (erem_grid * n)(*grids)
    pa = (erem_physics * n)(*physics)
    h = _P()
    st = _lib.erem_ensemble_create(n, ga, pa, int(precision), ctypes.byref(h))
    if st != EREM_OK:
        raise EremError(st, "erem_ensemble_create failed")
    return h


def erem_ensemble_destroy(ens) -> None:
    _lib.erem_ensemble_destroy(ens)


def erem_ensemble_last_error(ens) -> str:
    r = _lib.erem_ensemble_last_error(ens)
    return r.decode() if r else ""


def _echeck(ens, st):
    if st != EREM_OK:
        raise EremError(st, erem_ensemble_last_error(ens))


def erem_ensemble_set_member(ens, e, n, T, p, lnk, phi, lam, dt, stream=None) -> None:
    _echeck(ens, _lib.erem_ensemble_set_member(ens, int(e), _ptr(T, n), _ptr(p, n), _ptr(lnk, n),
                                               _ptr(phi, n), _ptr(lam, n), float(dt),
                                               _stream(stream)))


def erem_ensemble_get_member(ens, e, n, T, stream=None) -> None:
    _echeck(ens, _lib.erem_ensemble_get_member(ens, int(e), _ptr(T, n), _stream(stream)))


def erem_ensemble_set_temperature(ens, e, n, T, stream=None) -> None:
    _echeck(ens, _lib.erem_ensemble_set_temperature(ens, int(e), _ptr(T, n), _stream(stream)))


def erem_ensemble_configure(ens, opts: erem_leja_opts | None = None,
                            cfg: erem_ens_config | None = None) -> None:
    _echeck(ens, _lib.erem_ensemble_configure(ens, ctypes.byref(opts) if opts is not None else None,
                                              ctypes.byref(cfg) if cfg is not None else None))


def erem_ensemble_autotune(ens, probe_steps=1, stream=None) -> None:
    _echeck(ens, _lib.erem_ensemble_autotune(ens, int(probe_steps), _stream(stream)))


def erem_ensemble_run(ens, steps, stream=None) -> None:
    _echeck(ens, _lib.erem_ensemble_run(ens, int(steps), _stream(stream)))


def erem_ensemble_member_stats(ens, e) -> erem_ens_member_stats:
    st = erem_ens_member_stats()
    _echeck(ens, _lib.erem_ensemble_member_stats(ens, int(e), ctypes.byref(st)))
    return st


def erem_ensemble_run_stats(ens) -> erem_ens_run_stats:
    st = erem_ens_run_stats()
    _echeck(ens, _lib.erem_ensemble_run_stats(ens, ctypes.byref(st)))
    return st


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------
@dataclass
class Physics:
    rhoc_f: float = 1.0
    rhoc_s: float = 1.0
    head_left: float = 1.0
    head_right: float = 0.0
    T_inflow: float = 80.0
    fluid_model: int = 0

    def c(self) -> erem_physics:
        return erem_physics(self.rhoc_f, self.rhoc_s, self.head_left, self.head_right,
                            self.T_inflow, self.fluid_model)


class Context:
    """Owns one erem_ctx; methods forward to the C entry points."""

    def __init__(self, dim, nx, ny, nz=1, physics: Physics | None = None, precision="fp64",
                 lx=1.0, ly=1.0, lz=1.0):
        prec = {"fp64": EREM_FP64, "fp32_bulk": EREM_FP32_BULK}[precision] \
            if isinstance(precision, str) else int(precision)
        self.n = nx * ny * nz
        self.grid = erem_grid(dim, nx, ny, nz, lx, ly, lz)
        self.physics = physics or Physics()
        self._h = erem_create(self.grid, self.physics.c(), prec)

    def close(self):
        if getattr(self, "_h", None):
            erem_destroy(self._h)
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

    @property
    def handle(self):
        return self._h

    def set_physics(self, physics: Physics):
        self.physics = physics
        erem_set_physics(self._h, physics.c())

    def pressure_solve(self, lnk, T, p, tol=1e-10, maxit=100000, stream=None):
        return pressure_solve(self._h, self.n, lnk, T, p, tol, maxit, stream)

    @property
    def leja_coefficients(self) -> int:
        """Coefficient arrays per cell of the Leja copy of J (7 or 5 with the
        diagonal, 6 for a diagonal-free FP32-bulk 3D copy; 0 before any
        state)."""
        return int(_lib.erem_leja_coefficients(self._h))

    def set_state(self, T, p, lnk, phi, lam, dt, stream=None):
        erem_set_state(self._h, self.n, T, p, lnk, phi, lam, dt, stream)

    def phi1_apply(self, v, out, opts=None, stream=None):
        return phi1_apply(self._h, self.n, v, out, opts, stream)

    def erem_step(self, T, dt, p=None, lnk=None, phi=None, lam=None, opts=None, stream=None):
        return erem_step(self._h, self.n, T, dt, p, lnk, phi, lam, opts, stream)

    def coupled_step(self, T, p, lnk, phi, lam, dt, splitting=EREM_SPLIT_TROTTER,
                     pressure_tol=1e-10, pressure_maxit=200000, opts=None, stream=None, T_p=None):
        return coupled_step(self._h, self.n, T, p, lnk, phi, lam, dt, splitting, pressure_tol,
                            pressure_maxit, opts, stream, T_p)

    def rosm_integrate(self, T, t_end, dt0, scheme=EREM_ROS2, tol_a=1e-6, tol_r=1e-6,
                       lin_tol=1e-10, maxit=10000, max_attempts=100000, stream=None):
        return rosm_integrate(self._h, self.n, T, t_end, dt0, scheme, tol_a, tol_r, lin_tol, maxit,
                              max_attempts, stream)

    def erem_step_forced(self, T, dt, T_in, T_in_rate, p=None, lnk=None, phi=None, lam=None,
                         opts=None, stream=None):
        return erem_step_forced(self._h, self.n, T, dt, T_in, T_in_rate, p, lnk, phi, lam, opts,
                                stream)

    def rosm_step(self, T, dt, scheme=EREM_ROS2, p=None, lnk=None, phi=None, lam=None,
                  lin_tol=1e-10, maxit=10000, stream=None):
        return rosm_step(self._h, self.n, T, dt, scheme, p, lnk, phi, lam, lin_tol, maxit, stream)

    def set_leja_points(self, kind):
        erem_set_leja_points(self._h, kind)

    def set_substep_start(self, mode):
        erem_set_substep_start(self._h, mode)

    def set_pressure_precond(self, degree):
        erem_set_pressure_precond(self._h, degree)

    def set_host_access(self, mode):
        """erem_step with a pinned host T: 1 = kernels access it in place
        (default), 0 = staged copies."""
        _check(self._h, _lib.erem_set_host_access(self._h, int(mode)))

    def set_stage_precond(self, kind):
        """Rosenbrock stage solves: 0 = Jacobi BiCGSTAB, 1 = multigrid (default)."""
        _check(self._h, _lib.erem_set_stage_precond(self._h, int(kind)))

    def set_pressure_multigrid(self, nu=3, omega=1.8):
        _check(self._h, _lib.erem_set_pressure_multigrid(self._h, int(nu), float(omega)))

    def hold_interval(self, interval):
        erem_hold_interval(self._h, interval)

    def adjoint_tape(self, nbytes, record=True):
        """Reserve the adjoint tape (bytes) and record the following
        erem_steps (record=True), or stop recording (record=False)."""
        _check(self._h, _lib.erem_adjoint_tape(self._h, int(nbytes), 1 if record else 0))

    def adjoint_begin(self, stream=None):
        erem_adjoint_begin(self._h, stream)

    def adjoint_step(self, T, lam, schedule, stream=None):
        erem_adjoint_step(self._h, self.n, T, lam, schedule, stream)

    def adjoint_lnk(self, lnk, glnk, tol=1e-12, maxit=200000, stream=None):
        return erem_adjoint_lnk(self._h, self.n, lnk, glnk, tol, maxit, stream)

    def phi1_apply_krylov(self, v, out, opts=None, stream=None):
        return phi1_apply_krylov(self._h, self.n, v, out, opts, stream)

    def erem_step_krylov(self, T, dt, p=None, lnk=None, phi=None, lam=None, opts=None,
                         stream=None):
        return erem_step_krylov(self._h, self.n, T, dt, p, lnk, phi, lam, opts, stream)


class Ensemble:
    """Owns one erem_ens (a batch of independent 2D members); methods
    forward to the erem_ensemble_* entry points.  members: list of
    (nx, ny, Physics)."""

    def __init__(self, members, precision="fp64", lx=1.0, ly=1.0):
        prec = {"fp64": EREM_FP64, "fp32_bulk": EREM_FP32_BULK}[precision] \
            if isinstance(precision, str) else int(precision)
        self.sizes = [nx * ny for nx, ny, _ in members]
        grids = [erem_grid(2, nx, ny, 1, lx, ly, 1.0) for nx, ny, _ in members]
        phys = [(ph or Physics()).c() for _, _, ph in members]
        self._h = erem_ensemble_create(grids, phys, prec)

    def close(self):
        if getattr(self, "_h", None):
            erem_ensemble_destroy(self._h)
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

    def __len__(self):
        return len(self.sizes)

    def set_member(self, e, T, p, lnk, phi, lam, dt, stream=None):
        erem_ensemble_set_member(self._h, e, self.sizes[e], T, p, lnk, phi, lam, dt, stream)

    def set_temperature(self, e, T, stream=None):
        erem_ensemble_set_temperature(self._h, e, self.sizes[e], T, stream)

    def get_member(self, e, T, stream=None):
        erem_ensemble_get_member(self._h, e, self.sizes[e], T, stream)

    def configure(self, opts=None, policy=EREM_ENS_KEEP_SUBSTEPS, cluster_ctas=0, max_clusters=0):
        cfg = erem_ens_config(int(policy), int(cluster_ctas), int(max_clusters), 0)
        erem_ensemble_configure(self._h, opts, cfg)

    def autotune(self, probe_steps=1, stream=None):
        erem_ensemble_autotune(self._h, probe_steps, stream)

    def run(self, steps, stream=None) -> erem_ens_run_stats:
        erem_ensemble_run(self._h, steps, stream)
        return erem_ensemble_run_stats(self._h)

    def member_stats(self, e) -> erem_ens_member_stats:
        return erem_ensemble_member_stats(self._h, e)

    def run_stats(self) -> erem_ens_run_stats:
        return erem_ensemble_run_stats(self._h)
