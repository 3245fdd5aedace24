"""FP64 CPU oracle of the axisymmetric Allen-Cahn phase-field MRT lattice Boltzmann step.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It wraps ``axilbm_oracle.c`` (plain C, libm only) through ctypes and
shares no code with the CUDA library in ``paper_1810_09299_gb300``.

Every function here is a thin marshalling layer; the arithmetic lives in the
C file, which cites the paper's equation for each step.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "axilbm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

Q = 9


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("nr", ctypes.c_int32), ("nz", ctypes.c_int32), ("z_periodic", ctypes.c_int32),
        ("p_coupling", ctypes.c_int32), ("collision", ctypes.c_int32),
        ("rho_l", ctypes.c_double), ("rho_g", ctypes.c_double),
        ("nu_l", ctypes.c_double), ("nu_g", ctypes.c_double),
        ("sigma", ctypes.c_double), ("W", ctypes.c_double),
        ("mobility", ctypes.c_double), ("grav_z", ctypes.c_double),
        ("sf", ctypes.c_double * 9), ("sg", ctypes.c_double * 9),
        ("n_eps", ctypes.c_double),
    ]


class OrcDiag(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "step", "mass", "kinetic", "z_centroid", "dp", "umax", "phi_min", "phi_max",
        "axis_half_length", "radial_half_length", "nonfinite")]


def build(force: bool = False, openmp: bool = True) -> str:
    """Compile the oracle with gcc (-O2, no FP contraction).  Returns the .so path."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared",
            _SRC, "-o", _LIB + ".tmp", "-lm"]
    cmds = ([base[:1] + ["-fopenmp"] + base[1:]] if openmp else []) + [base]
    err = ""
    for cmd in cmds:
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(_LIB + ".tmp", _LIB)
            return _LIB
        err = r.stderr
    raise RuntimeError("oracle build failed:\n" + err)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            L.orc_create.restype = ctypes.c_void_p
            L.orc_create.argtypes = [ctypes.POINTER(OrcParams)]
            L.orc_destroy.argtypes = [ctypes.c_void_p]
            L.orc_init.argtypes = [ctypes.c_void_p, dp]
            L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
            L.orc_fields.argtypes = [ctypes.c_void_p, dp, dp, dp, dp, dp]
            L.orc_get_populations.argtypes = [ctypes.c_void_p, dp, dp]
            L.orc_set_populations.argtypes = [ctypes.c_void_p, dp, dp]
            L.orc_get_aux.argtypes = [ctypes.c_void_p, dp, dp, dp]
            L.orc_set_aux.argtypes = [ctypes.c_void_p, dp, dp, dp]
            L.orc_diagnostics.argtypes = [ctypes.c_void_p, ctypes.POINTER(OrcDiag)]
            L.orc_axis_drops.argtypes = [ctypes.c_void_p, ctypes.c_int, dp, ip, dp]
            L.orc_step_count.restype = ctypes.c_int64
            L.orc_step_count.argtypes = [ctypes.c_void_p]
            L.orc_set_threads.argtypes = [ctypes.c_int]
            L.orc_lattice.argtypes = [ip, ip, dp]
            L.orc_matrix_M.argtypes = [dp]
            L.orc_matrix_Minv.argtypes = [dp]
            L.orc_matrix_T.argtypes = [dp]
            L.orc_matrix_Tinv.argtypes = [dp]
            L.orc_raw_collide.argtypes = [dp, dp, dp, dp, dp]
            L.orc_feq.argtypes = [ctypes.c_double] * 5 + [dp]
            L.orc_R.argtypes = [ctypes.c_double] * 6 + [dp]
            L.orc_geq.argtypes = [ctypes.c_double] * 5 + [dp]
            L.orc_T.argtypes = [ctypes.c_double] * 7 + [dp]
            L.orc_mrt_collide.argtypes = [dp, dp, dp, dp, dp]
            L.orc_stencil.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def make_params(case: dict) -> OrcParams:
    """Build the C parameter block from a case dictionary (see paper_1810_09299_gb300.workloads)."""
    p = OrcParams()
    p.nr, p.nz = int(case["nr"]), int(case["nz"])
    p.z_periodic = int(case.get("z_periodic", 0))
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


# ---------------------------------------------------------------- building blocks
def lattice():
    cz = (ctypes.c_int * 9)()
    cr = (ctypes.c_int * 9)()
    w = (ctypes.c_double * 9)()
    lib().orc_lattice(cz, cr, w)
    return np.array(cz[:]), np.array(cr[:]), np.array(w[:])


def matrix_M() -> np.ndarray:
    out = np.zeros(81)
    lib().orc_matrix_M(_p(out))
    return out.reshape(9, 9)


def matrix_Minv() -> np.ndarray:
    out = np.zeros(81)
    lib().orc_matrix_Minv(_p(out))
    return out.reshape(9, 9)


def matrix_T() -> np.ndarray:
    """The raw-moment basis (rows 1, c_z, c_r, c^2, c_z^2 - c_r^2, c_z c_r, c_z^2 c_r, c_z c_r^2, c_z^2 c_r^2)."""
    out = np.zeros(81)
    lib().orc_matrix_T(_p(out))
    return out.reshape(9, 9)


def matrix_Tinv() -> np.ndarray:
    out = np.zeros(81)
    lib().orc_matrix_Tinv(_p(out))
    return out.reshape(9, 9)


def feq(r, phi, uz, ur, mobility) -> np.ndarray:
    out = np.zeros(9)
    lib().orc_feq(r, phi, uz, ur, mobility, _p(out))
    return out


def R_source(r, dchi_z, dchi_r, nz_, nr_, lam) -> np.ndarray:
    out = np.zeros(9)
    lib().orc_R(r, dchi_z, dchi_r, nz_, nr_, lam, _p(out))
    return out


def geq(r, p, rho, uz, ur) -> np.ndarray:
    out = np.zeros(9)
    lib().orc_geq(r, p, rho, uz, ur, _p(out))
    return out


def T_force(rho, uz, ur, Fz, Fr, dz_rrho, dr_rrho) -> np.ndarray:
    out = np.zeros(9)
    lib().orc_T(rho, uz, ur, Fz, Fr, dz_rrho, dr_rrho, _p(out))
    return out


def mrt_collide(x, xeq, src, S) -> np.ndarray:
    x, xeq, src, S = _c(x), _c(xeq), _c(src), _c(S)
    out = np.zeros(9)
    lib().orc_mrt_collide(_p(x), _p(xeq), _p(src), _p(S), _p(out))
    return out


def raw_collide(x, xeq, src, S) -> np.ndarray:
    """The collision of mrt_collide in the raw-moment basis (S: rates of the raw moments)."""
    x, xeq, src, S = _c(x), _c(xeq), _c(src), _c(S)
    out = np.zeros(9)
    lib().orc_raw_collide(_p(x), _p(xeq), _p(src), _p(S), _p(out))
    return out


def stencil(field: np.ndarray, z_periodic: bool):
    """Eq. 39 (gradient) and Eq. 40 (Laplacian) of a [nz][nr] field, ghosts per Sec. 2.3."""
    f = _c(field)
    nz, nr = f.shape
    dz, dr, lap = np.zeros_like(f), np.zeros_like(f), np.zeros_like(f)
    lib().orc_stencil(nr, nz, int(z_periodic), _p(f), _p(dz), _p(dr), _p(lap))
    return dz, dr, lap


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


# ---------------------------------------------------------------- simulation
class Oracle:
    """One FP64 CPU simulation of a case.  Arrays are [nz][nr] / [9][nz][nr]."""

    def __init__(self, case: dict):
        self.case = dict(case)
        self._prm = make_params(case)
        self.nr, self.nz = self._prm.nr, self._prm.nz
        h = lib().orc_create(ctypes.byref(self._prm))
        if not h:
            raise ValueError("orc_create rejected the parameters")
        self._h = ctypes.c_void_p(h)

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, phi0: np.ndarray):
        a = _c(phi0)
        assert a.shape == (self.nz, self.nr)
        lib().orc_init(self._h, _p(a))
        return self

    def step(self, n: int = 1):
        lib().orc_step(self._h, int(n))
        return self

    @property
    def steps(self) -> int:
        return int(lib().orc_step_count(self._h))

    def fields(self) -> dict:
        shp = (self.nz, self.nr)
        out = {k: np.zeros(shp) for k in ("phi", "rho", "uz", "ur", "p")}
        lib().orc_fields(self._h, *(_p(out[k]) for k in ("phi", "rho", "uz", "ur", "p")))
        return out

    def populations(self):
        f = np.zeros((9, self.nz, self.nr))
        g = np.zeros((9, self.nz, self.nr))
        lib().orc_get_populations(self._h, _p(f), _p(g))
        return f, g

    def set_populations(self, f, g):
        f, g = _c(f), _c(g)
        lib().orc_set_populations(self._h, _p(f), _p(g))

    def aux(self):
        shp = (self.nz, self.nr)
        cz, cr, pp = np.zeros(shp), np.zeros(shp), np.zeros(shp)
        lib().orc_get_aux(self._h, _p(cz), _p(cr), _p(pp))
        return cz, cr, pp

    def set_aux(self, chi_z, chi_r, p_prev):
        a, b, c = _c(chi_z), _c(chi_r), _c(p_prev)
        lib().orc_set_aux(self._h, _p(a), _p(b), _p(c))

    def axis_drops(self, max_drops: int = 64):
        """Drops on the axis row: (list of dicts z_start, z_end, volume, radius;
        number found; (least axis phi, its z))."""
        out = np.zeros(4 * max(1, max_drops))
        n = ctypes.c_int(0)
        amin = np.zeros(2)
        lib().orc_axis_drops(self._h, int(max_drops), _p(out), ctypes.byref(n), _p(amin))
        keys = ("z_start", "z_end", "volume", "radius")
        drops = [{k: float(out[4 * m + i]) for i, k in enumerate(keys)} for m in range(min(n.value, max_drops))]
        return drops, int(n.value), (float(amin[0]), float(amin[1]))

    def diagnostics(self) -> dict:
        d = OrcDiag()
        lib().orc_diagnostics(self._h, ctypes.byref(d))
        return {k: getattr(d, k) for k, _ in OrcDiag._fields_}
