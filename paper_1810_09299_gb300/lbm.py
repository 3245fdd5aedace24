"""ctypes binding of the C ABI in include/lbm.h (libaxilbm.so).

Argument marshalling only: every step of the method runs in the CUDA kernels
of the library.  The library is loaded from this package directory; a missing
library raises immediately (there is no fallback path).  PyTorch, when
present, only supplies the CUDA stream (``stream=None`` uses torch's current
stream if torch is importable, else the default stream).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libaxilbm.so")

LBM_OK = 0
LBM_ERR_INVALID_ARG = -1
LBM_ERR_CUDA = -2
LBM_ERR_NONFINITE = -3
LBM_ERR_TIMEOUT = -4
LBM_ERR_OOM = -5
LBM_ERR_STATE = -6

PRECISIONS = {"fp64": 0, "fp32": 1, "mix_fp16": 2, "mix_bf16": 3}
SHAPES = {"flat": 0, "sphere": 1, "ellipsoid": 2, "p2": 3, "thread": 4, "bubble": 5, "host_array": 6}
FIELDS = ("phi", "rho", "uz", "ur", "p")

# Every symbol include/lbm.h declares.
EXPORTS = (
    "lbm_create", "lbm_batch_create", "lbm_num_cases", "lbm_init_phase", "lbm_case_init_phase",
    "lbm_step", "lbm_get_fields", "lbm_case_get_fields", "lbm_diagnostics", "lbm_case_diagnostics",
    "lbm_get_state", "lbm_set_state", "lbm_checkpoint_size", "lbm_checkpoint_save",
    "lbm_checkpoint_load", "lbm_autotune", "lbm_set_variant", "lbm_num_variants",
    "lbm_kernel_launches", "lbm_destroy", "lbm_strerror", "lbm_diag_reduce_noalloc",
    "lbm_selftest_bounded_wait", "lbm_case_diagnostics_enqueue", "lbm_diagnostics_wait", "lbm_init_phase_all",
    "lbm_case_axis_drops", "lbm_measure_fp64_rate",
)
MAX_AXIS_DROPS = 64
DIAG_SLOTS = 4


class LbmParams(ctypes.Structure):
    _fields_ = [
        ("nr", ctypes.c_int32), ("nz", ctypes.c_int32), ("z_periodic", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("p_coupling", ctypes.c_int32), ("collision", ctypes.c_int32),
        ("rho_l", ctypes.c_double), ("rho_g", ctypes.c_double),
        ("nu_l", ctypes.c_double), ("nu_g", ctypes.c_double),
        ("sigma", ctypes.c_double), ("W", ctypes.c_double),
        ("mobility", ctypes.c_double), ("grav_z", ctypes.c_double),
        ("sf", ctypes.c_double * 9), ("sg", ctypes.c_double * 9),
        ("n_eps", ctypes.c_double),
    ]


class LbmDiag(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "step", "mass", "kinetic", "z_centroid", "dp", "umax", "phi_min", "phi_max",
        "axis_half_length", "radial_half_length", "nonfinite")]


class LbmDrop(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("z_start", "z_end", "volume", "radius")]


class LbmError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


_lib = None


def lib():
    """Load libaxilbm.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing (run __graft_entry__.build())")
    L = ctypes.CDLL(LIB_PATH)
    vp, dp, i32, i64 = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.c_int64
    hpp = ctypes.POINTER(ctypes.c_void_p)
    P = ctypes.POINTER(LbmParams)
    sig = {
        "lbm_create": (ctypes.c_int, [P, vp, hpp]),
        "lbm_batch_create": (ctypes.c_int, [P, i32, vp, hpp]),
        "lbm_num_cases": (i32, [vp]),
        "lbm_init_phase": (ctypes.c_int, [vp, i32, dp, i32, dp]),
        "lbm_case_init_phase": (ctypes.c_int, [vp, i32, i32, dp, i32, dp]),
        "lbm_step": (ctypes.c_int, [vp, i64]),
        "lbm_get_fields": (ctypes.c_int, [vp, i32, dp]),
        "lbm_case_get_fields": (ctypes.c_int, [vp, i32, i32, dp]),
        "lbm_diagnostics": (ctypes.c_int, [vp, ctypes.POINTER(LbmDiag)]),
        "lbm_case_diagnostics": (ctypes.c_int, [vp, i32, ctypes.POINTER(LbmDiag)]),
        "lbm_get_state": (ctypes.c_int, [vp, i32, dp, dp, dp]),
        "lbm_set_state": (ctypes.c_int, [vp, i32, dp, dp, dp]),
        "lbm_checkpoint_size": (i64, [vp]),
        "lbm_checkpoint_save": (ctypes.c_int, [vp, vp]),
        "lbm_checkpoint_load": (ctypes.c_int, [vp, vp]),
        "lbm_autotune": (ctypes.c_int, [vp, i32, ctypes.POINTER(i32)]),
        "lbm_set_variant": (ctypes.c_int, [vp, i32]),
        "lbm_num_variants": (i32, []),
        "lbm_kernel_launches": (i64, [vp]),
        "lbm_destroy": (ctypes.c_int, [vp]),
        "lbm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "lbm_diag_reduce_noalloc": (ctypes.c_int, [vp, i32, i32, i32, ctypes.c_double, vp, vp]),
        "lbm_selftest_bounded_wait": (ctypes.c_int, [i32, vp, vp]),
        "lbm_case_diagnostics_enqueue": (ctypes.c_int, [vp, i32, ctypes.POINTER(LbmDiag), i32]),
        "lbm_diagnostics_wait": (ctypes.c_int, [vp, i32]),
        "lbm_init_phase_all": (ctypes.c_int, [vp, dp]),
        "lbm_case_axis_drops": (ctypes.c_int, [vp, i32, i32, ctypes.POINTER(LbmDrop), ctypes.POINTER(i32), dp]),
        "lbm_measure_fp64_rate": (ctypes.c_int, [i32, vp, dp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def strerror(code: int) -> str:
    return lib().lbm_strerror(int(code)).decode()


def _check(code: int, what: str):
    if code != LBM_OK:
        raise LbmError(code, what)


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_params(case: dict) -> LbmParams:
    p = LbmParams()
    p.nr, p.nz = int(case["nr"]), int(case["nz"])
    p.z_periodic = int(case.get("z_periodic", 0))
    prec = case.get("precision", "fp64")
    p.precision = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    p.p_coupling = int(case.get("p_coupling", 0))
    p.collision = int(case.get("collision", 0))
    for k in ("rho_l", "rho_g", "nu_l", "nu_g", "sigma", "W", "mobility"):
        setattr(p, k, float(case[k]))
    p.grav_z = float(case.get("grav_z", 0.0))
    for i in range(9):
        p.sf[i] = float(case["sf"][i])
        p.sg[i] = float(case["sg"][i])
    p.n_eps = float(case.get("n_eps", 1e-12))
    return p


def _stream_ptr(stream) -> int:
    if stream is not None:
        return int(stream)
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return 0


class Simulation:
    """A handle of one or more cases (``cases`` is a dict or a list of dicts)."""

    def __init__(self, cases, stream=None):
        if isinstance(cases, dict):
            cases = [cases]
        self.cases = [dict(c) for c in cases]
        arr = (LbmParams * len(cases))(*[make_params(c) for c in cases])
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(_stream_ptr(stream))
        if len(cases) == 1:
            rc = lib().lbm_create(arr, st, ctypes.byref(h))
        else:
            rc = lib().lbm_batch_create(arr, len(cases), st, ctypes.byref(h))
        _check(rc, "lbm_create")
        self._h = h

    # -- life cycle
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().lbm_destroy(self._h)
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

    @property
    def num_cases(self) -> int:
        return int(lib().lbm_num_cases(self._h))

    # -- initial condition
    def init_phase(self, icase: int = 0, shape: str = "host_array", args: Sequence[float] = (),
                   phi: Optional[np.ndarray] = None):
        c = self.cases[icase]
        a = np.ascontiguousarray(np.asarray(args, dtype=np.float64))
        ph = None
        if shape == "host_array":
            ph = np.ascontiguousarray(phi, dtype=np.float64)
            assert ph.shape == (c["nz"], c["nr"])
        rc = lib().lbm_case_init_phase(self._h, icase, SHAPES[shape], _dp(a) if a.size else None, a.size, _dp(ph))
        _check(rc, "lbm_init_phase")
        return self

    def init_all(self, phi_all: np.ndarray):
        """Every case from host arrays at once: phi_all holds each case's
        [nz][nr] phi0 one after the other (C-contiguous float64)."""
        need = sum(c["nz"] * c["nr"] for c in self.cases)
        assert phi_all.dtype == np.float64 and phi_all.flags["C_CONTIGUOUS"] and phi_all.size == need
        _check(lib().lbm_init_phase_all(self._h, _dp(phi_all)), "lbm_init_phase_all")
        return self

    def init_case(self, icase: int, case: Optional[dict] = None, host_array: bool = True):
        """Initial phi of a workloads.py case dict: from its host array or its shape."""
        from . import workloads
        c = case or self.cases[icase]
        if host_array:
            return self.init_phase(icase, "host_array", phi=workloads.initial_phi(c))
        return self.init_phase(icase, c["shape"], c["shape_args"])

    # -- stepping
    def step(self, n: int = 1):
        _check(lib().lbm_step(self._h, int(n)), "lbm_step")
        return self

    # -- read-back
    def fields(self, icase: int = 0, which=FIELDS) -> dict:
        c = self.cases[icase]
        mask = 0
        for k in which:
            mask |= 1 << FIELDS.index(k)
        order = [k for k in FIELDS if mask & (1 << FIELDS.index(k))]
        out = np.zeros((len(order), c["nz"], c["nr"]))
        _check(lib().lbm_case_get_fields(self._h, icase, mask, _dp(out)), "lbm_get_fields")
        return {k: out[i] for i, k in enumerate(order)}

    def diagnostics(self, icase: int = 0, check: bool = True) -> dict:
        d = LbmDiag()
        rc = lib().lbm_case_diagnostics(self._h, icase, ctypes.byref(d))
        if check:
            _check(rc, "lbm_diagnostics")
        out = {k: getattr(d, k) for k, _ in LbmDiag._fields_}
        out["status"] = rc
        return out

    def axis_drops(self, icase: int = 0, max_drops: int = MAX_AXIS_DROPS):
        """The drops along the axis (lbm_case_axis_drops): a list of dicts
        (z_start, z_end, volume, radius) in scan order, the number of drops
        found, and (least phi on the axis row, its z)."""
        arr = (LbmDrop * max(1, max_drops))()
        n = ctypes.c_int32(0)
        amin = np.zeros(2)
        _check(lib().lbm_case_axis_drops(self._h, icase, max_drops, arr, ctypes.byref(n), _dp(amin)),
               "lbm_case_axis_drops")
        drops = [{k: getattr(arr[i], k) for k, _ in LbmDrop._fields_} for i in range(min(n.value, max_drops))]
        return drops, int(n.value), (float(amin[0]), float(amin[1]))

    def diagnostics_enqueue(self, icase: int, out: "LbmDiag", slot: int):
        """Enqueue case icase's record into `out` (keep it alive, and pinned for
        the copy to be asynchronous, until diagnostics_wait(slot))."""
        _check(lib().lbm_case_diagnostics_enqueue(self._h, icase, ctypes.byref(out), slot), "lbm_diagnostics_enqueue")

    def diagnostics_wait(self, slot: int) -> int:
        """Wait for the record enqueued on `slot`; returns the status code."""
        return int(lib().lbm_diagnostics_wait(self._h, slot))

    def state(self, icase: int = 0):
        c = self.cases[icase]
        f = np.zeros((9, c["nz"], c["nr"]))
        g = np.zeros((9, c["nz"], c["nr"]))
        aux = np.zeros((3, c["nz"], c["nr"]))
        _check(lib().lbm_get_state(self._h, icase, _dp(f), _dp(g), _dp(aux)), "lbm_get_state")
        return f, g, aux

    def set_state(self, icase: int, f=None, g=None, aux=None):
        cv = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)
        f, g, aux = cv(f), cv(g), cv(aux)
        _check(lib().lbm_set_state(self._h, icase, _dp(f), _dp(g), _dp(aux)), "lbm_set_state")

    # -- checkpoints and tuning
    def checkpoint(self) -> bytes:
        n = int(lib().lbm_checkpoint_size(self._h))
        buf = ctypes.create_string_buffer(n)
        _check(lib().lbm_checkpoint_save(self._h, buf), "lbm_checkpoint_save")
        return buf.raw

    def restore(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(lib().lbm_checkpoint_load(self._h, buf), "lbm_checkpoint_load")

    def autotune(self, reps: int = 3) -> int:
        v = ctypes.c_int32(-1)
        _check(lib().lbm_autotune(self._h, int(reps), ctypes.byref(v)), "lbm_autotune")
        return int(v.value)

    def set_variant(self, v: int):
        _check(lib().lbm_set_variant(self._h, int(v)), "lbm_set_variant")

    @property
    def kernel_launches(self) -> int:
        return int(lib().lbm_kernel_launches(self._h))


def measure_fp64_rate(iters: int = 20000, stream=None) -> float:
    """FP64 fused multiply-adds per second the GPU sustains (lbm_measure_fp64_rate)."""
    out = ctypes.c_double(0.0)
    _check(lib().lbm_measure_fp64_rate(int(iters), ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(out)),
           "lbm_measure_fp64_rate")
    return float(out.value)


def num_variants() -> int:
    return int(lib().lbm_num_variants())
