"""Reference oracle for the SIMPLE-TS time step: a plain serial FP64 C
implementation (simplets_oracle.c) and its ctypes binding.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  It shares
no code with the CUDA path and imports nothing from it.

State dictionaries hold 2D float64 arrays indexed [j, i]:
    u: (ny, nx+1)   v: (ny+1, nx)   p, T: (ny, nx)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Dict, Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "simplets_oracle.c")
_HDR = os.path.join(_HERE, "simplets_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_ROWS = os.path.join(_HERE, "liboracle_rows.so")

CFLAGS = ["-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-Wall"]


def build(force: bool = False, rows: bool = False) -> str:
    """Compile liboracle.so next to the source (plain gcc, no FMA contraction).

    rows=True compiles the same source with -fopenmp into liboracle_rows.so,
    whose row loops run on all host threads (the multi-core CPU baseline);
    it gives the same bits as the serial build."""
    lib = _LIB_ROWS if rows else _LIB
    stale = (not os.path.exists(lib)
             or os.path.getmtime(lib) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, *(["-fopenmp"] if rows else []), "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, lib)
    return lib


class _Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("lx", ctypes.c_double), ("ly", ctypes.c_double),
        ("dx", ctypes.POINTER(ctypes.c_double)), ("dy", ctypes.POINTER(ctypes.c_double)),
        ("gas_model", ctypes.c_int),
        ("gamma", ctypes.c_double), ("prandtl", ctypes.c_double), ("visc_exp", ctypes.c_double),
        ("mach_in", ctypes.c_double), ("reynolds", ctypes.c_double), ("kn", ctypes.c_double),
        ("gx", ctypes.c_double), ("gy", ctypes.c_double),
        ("side_kind", ctypes.c_int * 4), ("side_vel", ctypes.c_double * 4),
        ("side_T", ctypes.c_double * 4), ("body_T", ctypes.c_double),
        ("n_rect", ctypes.c_int), ("rect", ctypes.POINTER(ctypes.c_int)),
        ("inflow_u", ctypes.POINTER(ctypes.c_double)),
        ("inflow_T", ctypes.POINTER(ctypes.c_double)),
        ("inflow_p", ctypes.POINTER(ctypes.c_double)),
        ("dt", ctypes.c_double), ("cfl", ctypes.c_double),
        ("implicit", ctypes.c_int), ("tvd", ctypes.c_int),
        ("iters", ctypes.c_int), ("tol", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("perturb", ctypes.c_double),
        ("zeta_coef", ctypes.c_double), ("tau_coef", ctypes.c_double),
    ]


class _Coeffs(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("A", "B", "CT1f", "CT2f", "CT3f", "omega", "u_in", "dt")]


_libs: Dict[bool, ctypes.CDLL] = {}
_DP = ctypes.POINTER(ctypes.c_double)


def _load(rows: bool = False):
    if rows not in _libs:
        # SIMPLETS_ORACLE_LIB points the serial binding at another build of the
        # same source (the mutation test compiles deliberately broken copies)
        path = build(rows=True) if rows else (os.environ.get("SIMPLETS_ORACLE_LIB") or build())
        lib = ctypes.CDLL(path)
        lib.orc_coefficients.argtypes = [ctypes.POINTER(_Problem), ctypes.POINTER(_Coeffs)]
        lib.orc_init.argtypes = [ctypes.POINTER(_Problem), _DP, _DP, _DP, _DP]
        lib.orc_run.argtypes = [ctypes.POINTER(_Problem), _DP, _DP, _DP, _DP, ctypes.c_int,
                                _DP, ctypes.POINTER(ctypes.c_int)]
        lib.orc_van_leer.argtypes = [ctypes.c_double] * 2
        lib.orc_van_leer.restype = ctypes.c_double
        lib.orc_psi_s.argtypes = [ctypes.c_double] * 9
        lib.orc_psi_s.restype = ctypes.c_double
        lib.orc_psi_c.argtypes = [ctypes.c_double] * 8
        lib.orc_psi_c.restype = ctypes.c_double
        lib.orc_splitmix_uniform.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.orc_splitmix_uniform.restype = ctypes.c_double
        lib.orc_gam_harmonic.argtypes = [ctypes.c_double] * 4
        lib.orc_gam_harmonic.restype = ctypes.c_double
        lib.orc_threads.argtypes = []
        lib.orc_threads.restype = ctypes.c_int
        _libs[rows] = lib
    return _libs[rows]


def _dptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(_DP)


class _Pinned:
    """Keeps the numpy buffers referenced by a _Problem alive."""

    def __init__(self, case):
        c = case
        self.keep = []

        def arr(x, dtype=np.float64):
            if x is None:
                return None
            a = np.ascontiguousarray(np.asarray(x, dtype=dtype))
            self.keep.append(a)
            return a

        dx, dy = arr(c.dx), arr(c.dy)
        rect = arr(np.asarray(c.rects, dtype=np.int32).reshape(-1), np.int32) if c.rects else None
        iu, iT, ip = arr(c.inflow_u), arr(c.inflow_T), arr(c.inflow_p)
        P = _Problem()
        P.nx, P.ny, P.lx, P.ly = c.nx, c.ny, c.lx, c.ly
        P.dx, P.dy = _dptr(dx), _dptr(dy)
        P.gas_model = c.gas_model
        P.gamma, P.prandtl, P.visc_exp = c.gamma, c.prandtl, c.visc_exp
        P.mach_in, P.reynolds, P.kn = c.mach_in, c.reynolds, c.kn
        P.gx, P.gy = c.gx, c.gy
        for k in range(4):
            P.side_kind[k] = int(c.side_kind[k])
            P.side_vel[k] = float(c.side_vel[k])
            P.side_T[k] = float(c.side_T[k])
        P.body_T = c.body_T
        P.n_rect = len(c.rects)
        P.rect = rect.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) if rect is not None else None
        P.inflow_u, P.inflow_T, P.inflow_p = _dptr(iu), _dptr(iT), _dptr(ip)
        P.dt, P.cfl = c.dt, c.cfl
        P.implicit, P.tvd = int(bool(c.implicit)), int(bool(c.tvd))
        P.iters, P.tol = c.iters, c.tol
        P.seed, P.perturb = c.seed, c.perturb
        P.zeta_coef, P.tau_coef = c.zeta_coef, c.tau_coef
        self.P = P


def coefficients(case) -> Dict[str, float]:
    lib = _load()
    pin = _Pinned(case)
    k = _Coeffs()
    rc = lib.orc_coefficients(ctypes.byref(pin.P), ctypes.byref(k))
    if rc:
        raise ValueError(f"orc_coefficients failed ({rc})")
    return {n: getattr(k, n) for n, _ in _Coeffs._fields_}


def empty_state(case) -> Dict[str, np.ndarray]:
    nx, ny = case.nx, case.ny
    return {"u": np.zeros((ny, nx + 1)), "v": np.zeros((ny + 1, nx)),
            "p": np.zeros((ny, nx)), "T": np.zeros((ny, nx))}


def init(case) -> Dict[str, np.ndarray]:
    """Initial state: inflow state plus the seeded perturbation."""
    lib = _load()
    pin = _Pinned(case)
    s = empty_state(case)
    rc = lib.orc_init(ctypes.byref(pin.P), *(_dptr(s[k]) for k in ("u", "v", "p", "T")))
    if rc:
        raise ValueError(f"orc_init failed ({rc})")
    return s


def run(case, state: Optional[Dict[str, np.ndarray]] = None, nsteps: int = 1,
        allow_diverged: bool = False, rows: bool = False) -> Tuple[Dict[str, np.ndarray], np.ndarray, int]:
    """Advance `nsteps` time steps.  Returns (state, residuals[u, v, p, T], iterations of last step).
    rows=True runs the row-parallel build (same bits, all host threads)."""
    lib = _load(rows)
    pin = _Pinned(case)
    s = init(case) if state is None else {k: np.array(v, dtype=np.float64, copy=True) for k, v in state.items()}
    for k in ("u", "v", "p", "T"):
        s[k] = np.ascontiguousarray(s[k])
    res = np.zeros(4)
    it = ctypes.c_int(0)
    rc = lib.orc_run(ctypes.byref(pin.P), *(_dptr(s[k]) for k in ("u", "v", "p", "T")),
                     int(nsteps), _dptr(res), ctypes.byref(it))
    if rc == 3 and allow_diverged:
        return s, res, it.value
    if rc:
        raise ValueError(f"orc_run failed ({rc})")
    return s, res, it.value


def van_leer(num: float, den: float) -> float:
    return _load().orc_van_leer(num, den)


def psi_s(f1, f2, f3, f4, d1, d2, d3, d4, vel) -> float:
    return _load().orc_psi_s(f1, f2, f3, f4, d1, d2, d3, d4, vel)


def psi_c(f1, f2, f3, f4, d1, d2, d3, vel) -> float:
    return _load().orc_psi_c(f1, f2, f3, f4, d1, d2, d3, vel)


def gam_harmonic(ga: float, gb: float, da: float, db: float) -> float:
    return _load().orc_gam_harmonic(ga, gb, da, db)


def splitmix_uniform(seed: int, field: int, i: int, j: int) -> float:
    return _load().orc_splitmix_uniform(seed, field, i, j)


def threads(rows: bool = False) -> int:
    """Threads the row loops of a run use (1 for the serial build)."""
    return _load(rows).orc_threads()
