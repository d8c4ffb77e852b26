"""Python binding of libsimplets.so, the GB300 implementation of the SIMPLE-TS
time step (K. S. Shterev, arXiv:1802.04243).

The binding only marshals arguments: every step of the sweep runs in the
library's CUDA kernels.  Names follow the C ABI of include/simplets.h.  The
library is built in-tree (``paper_1802_04243_gb300.build.build()``); loading
fails loudly when it is missing -- there is no CPU fallback.

PyTorch supplies the CUDA stream (``torch.cuda.current_stream()``) and views
of borrowed device fields (``Simulation.field_view``).
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsimplets.so")

# status codes, sides, kinds, schemes, fields (include/simplets.h)
SIM_OK, SIM_EINVAL, SIM_ENOMEM, SIM_ECUDA, SIM_EDIVERGED, SIM_ETIMEOUT, SIM_ESTATE = range(7)
SIM_W, SIM_E, SIM_S, SIM_N = range(4)
SIM_BC_WALL, SIM_BC_SYMMETRY, SIM_BC_INFLOW, SIM_BC_OUTFLOW = range(4)
SIM_GAS_IDEAL_RE, SIM_GAS_HARD_SPHERE_KN = range(2)
SIM_EXPLICIT, SIM_IMPLICIT, SIM_UPWIND, SIM_TVD = 0, 1, 0, 2
SIM_FP64, SIM_MIXED, SIM_DF64 = 0, 1, 2
FIELDS = {"u": 0, "v": 1, "p": 2, "T": 3, "rho": 4, "gamma": 5}
KERNELS = {"faces": 0, "assemble": 1, "pressure": 2, "velocity": 3, "ghosts": 4, "explicit": 5}
STATUS = {0: "SIM_OK", 1: "SIM_EINVAL", 2: "SIM_ENOMEM", 3: "SIM_ECUDA", 4: "SIM_EDIVERGED",
          5: "SIM_ETIMEOUT", 6: "SIM_ESTATE"}

_DP = ctypes.POINTER(ctypes.c_double)


class sim_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("lx", ctypes.c_double), ("ly", ctypes.c_double),
                ("dx", _DP), ("dy", _DP)]


class sim_gas(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("gamma", ctypes.c_double), ("prandtl", ctypes.c_double),
                ("visc_exp", ctypes.c_double), ("mach_in", ctypes.c_double), ("reynolds", ctypes.c_double),
                ("kn", ctypes.c_double), ("gx", ctypes.c_double), ("gy", ctypes.c_double)]


class sim_bc(ctypes.Structure):
    _fields_ = [("side_kind", ctypes.c_int * 4), ("side_vel", ctypes.c_double * 4),
                ("side_T", ctypes.c_double * 4), ("body_T", ctypes.c_double),
                ("n_rect", ctypes.c_int), ("rect", ctypes.POINTER(ctypes.c_int)),
                ("inflow_u", _DP), ("inflow_T", _DP), ("inflow_p", _DP),
                ("dt", ctypes.c_double), ("cfl", ctypes.c_double), ("iters", ctypes.c_int),
                ("tol", ctypes.c_double), ("seed", ctypes.c_uint64), ("perturb", ctypes.c_double),
                ("precision", ctypes.c_int), ("zeta_coef", ctypes.c_double), ("tau_coef", ctypes.c_double)]


class SimError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None

# exported symbols and their signatures (the test of the ABI checks this list
# against include/simplets.h)
_SIGNATURES = {
    "sim_create": ([ctypes.POINTER(sim_grid), ctypes.POINTER(sim_gas), ctypes.POINTER(sim_bc), ctypes.c_void_p,
                    ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "sim_step": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "sim_fields": ([ctypes.c_void_p, ctypes.c_int, _DP, ctypes.c_size_t], ctypes.c_int),
    "sim_field_ptr": ([ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                       ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "sim_set_fields": ([ctypes.c_void_p, ctypes.c_int, _DP, ctypes.c_size_t], ctypes.c_int),
    "sim_set_state": ([ctypes.c_void_p, _DP, _DP, _DP, _DP], ctypes.c_int),
    "sim_get_state": ([ctypes.c_void_p, _DP, _DP, _DP, _DP, _DP], ctypes.c_int),
    "sim_residuals": ([ctypes.c_void_p, _DP, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "sim_coefficients": ([ctypes.c_void_p, _DP], ctypes.c_int),
    "sim_set_plan": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "sim_profile": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "sim_profile_read": ([ctypes.c_void_p, ctypes.c_int, _DP, ctypes.POINTER(ctypes.c_longlong)], ctypes.c_int),
    "sim_last_error": ([ctypes.c_void_p], ctypes.c_char_p),
    "simplets_alu_peak": ([ctypes.c_int, ctypes.c_double, ctypes.c_void_p, _DP], ctypes.c_int),
    "simplets_recip_check": ([_DP, ctypes.c_int, _DP], ctypes.c_int),
    "simplets_sqrt_check": ([_DP, ctypes.c_int, _DP], ctypes.c_int),
    "simplets_barrier_check": ([ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
                               ctypes.c_int),
    "sim_destroy": ([ctypes.c_void_p], None),
    "sim_batch_create": ([ctypes.c_int, ctypes.POINTER(sim_grid), ctypes.POINTER(sim_gas), ctypes.POINTER(sim_bc),
                          ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "sim_batch_step": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "sim_batch_fields": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _DP, ctypes.c_size_t], ctypes.c_int),
    "sim_batch_residuals": ([ctypes.c_void_p, ctypes.c_int, _DP], ctypes.c_int),
    "sim_batch_tune": ([ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "sim_batch_set_tiles": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "sim_batch_last_error": ([ctypes.c_void_p], ctypes.c_char_p),
    "sim_batch_set_persistent": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "sim_batch_plan_info": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "sim_batch_destroy": ([ctypes.c_void_p], None),
    "sim_strips_layout": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "sim_strips_create": ([ctypes.POINTER(sim_grid), ctypes.POINTER(sim_gas), ctypes.POINTER(sim_bc), ctypes.c_int,
                           ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "sim_strips_step": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "sim_strips_fields": ([ctypes.c_void_p, ctypes.c_int, _DP, ctypes.c_size_t], ctypes.c_int),
    "sim_strips_residuals": ([ctypes.c_void_p, _DP], ctypes.c_int),
    "sim_strips_last_error": ([ctypes.c_void_p], ctypes.c_char_p),
    "sim_strips_destroy": ([ctypes.c_void_p], None),
    "sim_step_noalloc": ([ctypes.POINTER(sim_grid), ctypes.POINTER(sim_gas), ctypes.POINTER(sim_bc), ctypes.c_int,
                          ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                          ctypes.c_void_p, _DP], ctypes.c_int),
}


def load(path: Optional[str] = None):
    """Load libsimplets.so (built by build.build()).  Raises if it is missing."""
    global _lib
    if _lib is None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build it with paper_1802_04243_gb300.build.build() "
                               "(the CUDA library is required; there is no CPU fallback)")
        lib = ctypes.CDLL(p)
        for name, (args, res) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_DP)


class _Desc:
    """ctypes descriptions of a workload case, with the arrays they point to."""

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
        self.grid = sim_grid(c.nx, c.ny, c.lx, c.ly, _ptr(dx), _ptr(dy))
        self.gas = sim_gas(c.gas_model, c.gamma, c.prandtl, c.visc_exp, c.mach_in, c.reynolds, c.kn, c.gx, c.gy)
        rect = arr(np.asarray(c.rects, dtype=np.int32).reshape(-1), np.int32) if len(c.rects) else None
        iu, iT, ip = arr(c.inflow_u), arr(c.inflow_T), arr(c.inflow_p)
        bc = sim_bc()
        for k in range(4):
            bc.side_kind[k] = int(c.side_kind[k])
            bc.side_vel[k] = float(c.side_vel[k])
            bc.side_T[k] = float(c.side_T[k])
        bc.body_T = c.body_T
        bc.n_rect = len(c.rects)
        bc.rect = rect.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) if rect is not None else None
        bc.inflow_u, bc.inflow_T, bc.inflow_p = _ptr(iu), _ptr(iT), _ptr(ip)
        bc.dt, bc.cfl, bc.iters, bc.tol = c.dt, c.cfl, c.iters, c.tol
        bc.seed, bc.perturb, bc.precision = c.seed, c.perturb, c.precision
        bc.zeta_coef, bc.tau_coef = c.zeta_coef, c.tau_coef
        self.bc = bc


def scheme_of(implicit: bool, tvd: bool) -> int:
    return (SIM_IMPLICIT if implicit else SIM_EXPLICIT) | (SIM_TVD if tvd else SIM_UPWIND)


def alu_peak_gflops(kind: str = "fp64", millis: float = 50.0, stream: Optional[int] = None) -> float:
    """Sustained FMA rate of the device (include/simplets_probe.h), in GFLOP/s."""
    out = ctypes.c_double()
    rc = load().simplets_alu_peak(0 if kind == "fp64" else 1, float(millis), ctypes.c_void_p(stream or 0),
                                  ctypes.byref(out))
    if rc:
        raise SimError(SIM_ECUDA, f"simplets_alu_peak failed ({rc})")
    return out.value


def recip_check(x) -> "tuple[np.ndarray, np.ndarray]":
    """The sweep's FP64 reciprocal of each x and the IEEE quotient 1/x, both
    computed on the device (include/simplets_probe.h)."""
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    out = np.empty(2 * x.size)
    rc = load().simplets_recip_check(x.ctypes.data_as(_DP), int(x.size), out.ctypes.data_as(_DP))
    if rc:
        raise SimError(SIM_ECUDA, f"simplets_recip_check failed ({rc})")
    return out[0::2].copy(), out[1::2].copy()


def sqrt_check(x) -> "tuple[np.ndarray, np.ndarray]":
    """The sweep's FP64 square root of each x (Gamma for omega = 1/2) and the
    IEEE root, both computed on the device (include/simplets_probe.h)."""
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    out = np.empty(2 * x.size)
    rc = load().simplets_sqrt_check(x.ctypes.data_as(_DP), int(x.size), out.ctypes.data_as(_DP))
    if rc:
        raise SimError(SIM_ECUDA, f"simplets_sqrt_check failed ({rc})")
    return out[0::2].copy(), out[1::2].copy()


def barrier_check(extra_blocks: int = 0, rounds: int = 10) -> "tuple[int, int]":
    """(error word, CTAs) of simplets_barrier_check: the persistent step's grid
    barrier crossed `rounds` times by every resident CTA, each barrier expecting
    `extra_blocks` CTAs more than were launched (include/simplets_probe.h)."""
    err, ctas = ctypes.c_int(), ctypes.c_int()
    rc = load().simplets_barrier_check(int(extra_blocks), int(rounds), ctypes.byref(err), ctypes.byref(ctas))
    if rc:
        raise SimError(SIM_ECUDA, f"simplets_barrier_check failed ({rc})")
    return err.value, ctas.value


class _CudaArray:
    """__cuda_array_interface__ view of a borrowed device array."""

    def __init__(self, ptr: int, shape, strides_bytes):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f8", "data": (ptr, False),
                                         "strides": tuple(strides_bytes), "version": 2}


class Simulation:
    """One SIMPLE-TS problem on the GPU (owns a sim_t)."""

    def __init__(self, case, stream: Optional[int] = None):
        self.lib = load()
        self.case = case
        self._desc = _Desc(case)
        h = ctypes.c_void_p()
        st = self.lib.sim_create(ctypes.byref(self._desc.grid), ctypes.byref(self._desc.gas),
                                 ctypes.byref(self._desc.bc), ctypes.c_void_p(stream or 0), ctypes.byref(h))
        if st != SIM_OK:
            raise SimError(st, "sim_create failed (invalid description or no device)")
        self.handle = h
        self._stream = stream or 0
        self.scheme = scheme_of(case.implicit, case.tvd)

    def _check(self, st: int):
        if st != SIM_OK:
            raise SimError(st, self.lib.sim_last_error(self.handle).decode())

    def step(self, n: int = 1, scheme: Optional[int] = None):
        self._check(self.lib.sim_step(self.handle, int(n), self.scheme if scheme is None else int(scheme)))

    def shape(self, name: str):
        nx, ny = self.case.nx, self.case.ny
        return {"u": (ny, nx + 1), "v": (ny + 1, nx)}.get(name, (ny, nx))

    def field(self, name: str, out: Optional[np.ndarray] = None) -> np.ndarray:
        a = np.empty(self.shape(name)) if out is None else out
        self._check(self.lib.sim_fields(self.handle, FIELDS[name], a.ctypes.data_as(_DP), a.size))
        return a

    def fields(self, names: Sequence[str] = ("u", "v", "p", "T")) -> Dict[str, np.ndarray]:
        return {k: self.field(k) for k in names}

    def set_field(self, name: str, values: np.ndarray):
        a = np.ascontiguousarray(values, dtype=np.float64)
        if a.shape != self.shape(name):
            raise ValueError(f"{name}: shape {a.shape} != {self.shape(name)}")
        self._check(self.lib.sim_set_fields(self.handle, FIELDS[name], a.ctypes.data_as(_DP), a.size))

    def set_fields(self, state: Dict[str, np.ndarray]):
        for k in ("u", "v", "p", "T"):
            if k in state:
                self.set_field(k, state[k])

    def set_state(self, state: Dict[str, np.ndarray]):
        """All of u, v, p, T at once (sim_set_state): one synchronisation, checks on the device."""
        arrs = []
        for k in ("u", "v", "p", "T"):
            a = np.ascontiguousarray(state[k], dtype=np.float64)
            if a.shape != self.shape(k):
                raise ValueError(f"{k}: shape {a.shape} != {self.shape(k)}")
            arrs.append(a)
        self._check(self.lib.sim_set_state(self.handle, *[a.ctypes.data_as(_DP) for a in arrs]))

    def get_state(self, out: Optional[Dict[str, np.ndarray]] = None):
        """u, v, p, T and the residuals (sim_get_state), with one synchronisation.
        Returns (fields, residuals, status)."""
        out = out if out is not None else {k: np.empty(self.shape(k)) for k in ("u", "v", "p", "T")}
        res = np.zeros(4)
        st = self.lib.sim_get_state(self.handle, *[out[k].ctypes.data_as(_DP) for k in ("u", "v", "p", "T")],
                                    res.ctypes.data_as(_DP))
        if st not in (SIM_OK, SIM_EDIVERGED):
            self._check(st)
        return out, res, st

    def residuals(self):
        out = np.zeros(4)
        it = ctypes.c_int(0)
        st = self.lib.sim_residuals(self.handle, out.ctypes.data_as(_DP), ctypes.byref(it))
        if st not in (SIM_OK, SIM_EDIVERGED):
            self._check(st)
        return out, it.value, st

    def coefficients(self) -> Dict[str, float]:
        out = np.zeros(9)
        self._check(self.lib.sim_coefficients(self.handle, out.ctypes.data_as(_DP)))
        return dict(zip(("A", "B", "CT1f", "CT2f", "CT3f", "omega", "u_in", "dt", "cells"), out.tolist()))

    def field_view(self, name: str):
        """Zero-copy torch view (including the two ghost layers) of a device field
        of the current state; valid until the next step."""
        import torch
        dev = ctypes.c_void_p()
        pitch = ctypes.c_size_t()
        self._check(self.lib.sim_field_ptr(self.handle, FIELDS[name], ctypes.byref(dev), ctypes.byref(pitch)))
        if self._stream:
            # the handle's stream may still be filling the array (double-float
            # state, the mixed path's FP64 u, v, T, Gamma): torch's current
            # stream waits for it
            torch.cuda.current_stream().wait_stream(torch.cuda.ExternalStream(self._stream))
        ny, nx = self.shape(name)
        base = dev.value - (2 * pitch.value + 2) * 8
        arr = _CudaArray(base, (ny + 4, nx + 4), (pitch.value * 8, 8))
        return torch.as_tensor(arr, device="cuda")

    def set_plan(self, tile_x: int = 32, tile_y: int = 8, ctas: int = 0, asm_ctas: int = 0):
        """Work distribution of the equation kernels (sim_set_plan); the same bits for every choice."""
        self._check(self.lib.sim_set_plan(self.handle, int(tile_x), int(tile_y), int(ctas), int(asm_ctas)))

    def profile(self, enable: bool = True, timing: bool = True):
        """enable=True: clear the launch counters; timing=True also brackets every
        kernel with CUDA events (and launches kernels one by one)."""
        self._check(self.lib.sim_profile(self.handle, (1 if timing else 2) if enable else 0))

    def profile_read(self) -> Dict[str, tuple]:
        out = {}
        for name, k in KERNELS.items():
            ms = ctypes.c_double()
            n = ctypes.c_longlong()
            self._check(self.lib.sim_profile_read(self.handle, k, ctypes.byref(ms), ctypes.byref(n)))
            out[name] = (ms.value, n.value)
        return out

    def close(self):
        if getattr(self, "handle", None):
            self.lib.sim_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Many independent problems advanced together (sim_batch_*): one launch per
    kernel phase over all of them, whole steps replayed as CUDA graphs."""

    def __init__(self, cases, stream: Optional[int] = None):
        self.lib = load()
        self.cases = list(cases)
        n = len(self.cases)
        self._descs = [_Desc(c) for c in self.cases]
        grids, gases, bcs = (sim_grid * n)(), (sim_gas * n)(), (sim_bc * n)()
        for q, d in enumerate(self._descs):
            grids[q], gases[q], bcs[q] = d.grid, d.gas, d.bc
        self._arrays = (grids, gases, bcs)
        h = ctypes.c_void_p()
        st = self.lib.sim_batch_create(n, grids, gases, bcs, ctypes.c_void_p(stream or 0), ctypes.byref(h))
        if st != SIM_OK:
            raise SimError(st, "sim_batch_create failed")
        self.handle = h
        c0 = self.cases[0]
        self.scheme = scheme_of(c0.implicit, c0.tvd)

    def _check(self, st: int):
        if st != SIM_OK:
            raise SimError(st, self.lib.sim_batch_last_error(self.handle).decode())

    def step(self, n: int = 1, scheme: Optional[int] = None):
        self._check(self.lib.sim_batch_step(self.handle, int(n), self.scheme if scheme is None else int(scheme)))

    def tune(self, scheme: Optional[int] = None):
        out = (ctypes.c_int * 3)()
        self._check(self.lib.sim_batch_tune(self.handle, self.scheme if scheme is None else int(scheme), out))
        return tuple(out)

    def set_tiles(self, tile_x: int, tile_y: int, ctas: int = 0):
        """Tiles of tile_x x tile_y threads walked by `ctas` CTAs (0: one per tile), sim_batch_set_tiles."""
        self._check(self.lib.sim_batch_set_tiles(self.handle, int(tile_x), int(tile_y), int(ctas)))

    def set_persistent(self, on: bool = True):
        """Each step as one persistent cooperative kernel (sim_batch_set_persistent)."""
        self._check(self.lib.sim_batch_set_persistent(self.handle, 1 if on else 0))

    def plan_info(self):
        """(tile x, tile y, CTAs, persistent) of the batch's work distribution."""
        out = (ctypes.c_int * 4)()
        self._check(self.lib.sim_batch_plan_info(self.handle, out))
        return tuple(out)

    def field(self, instance: int, name: str) -> np.ndarray:
        c = self.cases[instance]
        shape = {"u": (c.ny, c.nx + 1), "v": (c.ny + 1, c.nx)}.get(name, (c.ny, c.nx))
        a = np.empty(shape)
        self._check(self.lib.sim_batch_fields(self.handle, instance, FIELDS[name], a.ctypes.data_as(_DP), a.size))
        return a

    def fields(self, instance: int, names: Sequence[str] = ("u", "v", "p", "T")) -> Dict[str, np.ndarray]:
        return {k: self.field(instance, k) for k in names}

    def residuals(self, instance: int):
        out = np.zeros(4)
        st = self.lib.sim_batch_residuals(self.handle, instance, out.ctypes.data_as(_DP))
        if st not in (SIM_OK, SIM_EDIVERGED):
            self._check(st)
        return out, st

    @property
    def cells(self) -> int:
        return sum(c.cells for c in self.cases)

    def close(self):
        if getattr(self, "handle", None):
            self.lib.sim_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


STRIP_HALO = 4


def strips_layout(nx: int, n_strips: int, strip: int) -> Dict[str, tuple]:
    """Columns of one strip of an x-decomposed problem (sim_strips_layout, host
    only): owned cell columns, stored columns of the extended grid, computed
    positions, each as a half-open range."""
    out = (ctypes.c_int * 6)()
    st = load().sim_strips_layout(int(nx), int(n_strips), int(strip), out)
    if st != SIM_OK:
        raise SimError(st, f"no layout for strip {strip} of {n_strips} over {nx} columns")
    return {"own": (out[0], out[1]), "store": (out[2], out[3]), "compute": (out[4], out[5])}


class Strips:
    """One problem decomposed into x-strips with halo exchange (sim_strips_*),
    advanced on one device; results equal a whole-problem Simulation's."""

    def __init__(self, case, n_strips: int, stream: Optional[int] = None):
        self.lib = load()
        self.case = case
        self._desc = _Desc(case)
        h = ctypes.c_void_p()
        st = self.lib.sim_strips_create(ctypes.byref(self._desc.grid), ctypes.byref(self._desc.gas),
                                        ctypes.byref(self._desc.bc), int(n_strips), ctypes.c_void_p(stream or 0),
                                        ctypes.byref(h))
        if st != SIM_OK:
            raise SimError(st, "sim_strips_create failed")
        self.handle = h
        self.scheme = scheme_of(case.implicit, case.tvd)

    def _check(self, st: int):
        if st != SIM_OK:
            raise SimError(st, self.lib.sim_strips_last_error(self.handle).decode())

    def step(self, n: int = 1, scheme: Optional[int] = None):
        self._check(self.lib.sim_strips_step(self.handle, int(n), self.scheme if scheme is None else int(scheme)))

    def field(self, name: str) -> np.ndarray:
        c = self.case
        shape = {"u": (c.ny, c.nx + 1), "v": (c.ny + 1, c.nx)}.get(name, (c.ny, c.nx))
        a = np.empty(shape)
        self._check(self.lib.sim_strips_fields(self.handle, FIELDS[name], a.ctypes.data_as(_DP), a.size))
        return a

    def fields(self, names: Sequence[str] = ("u", "v", "p", "T")) -> Dict[str, np.ndarray]:
        return {k: self.field(k) for k in names}

    def residuals(self):
        out = np.zeros(4)
        st = self.lib.sim_strips_residuals(self.handle, out.ctypes.data_as(_DP))
        if st not in (SIM_OK, SIM_EDIVERGED):
            self._check(st)
        return out, st

    def close(self):
        if getattr(self, "handle", None):
            self.lib.sim_strips_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
