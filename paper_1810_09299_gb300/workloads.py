"""Seeded synthetic inputs: case parameter sets and initial phase fields.

This module holds no arithmetic of the lattice Boltzmann method itself.  It
only builds the initial order-parameter field phi0 of the paper's test
problems and the parameter dictionaries of the benchmark cases, so that the
CUDA library and the FP64 oracle can be started from identical inputs.

Coordinates follow the lattice convention of Sec. 2.3: node (k, j) sits at
z = k + 0.5, r = j + 0.5 (first lattice line at r = 0.5).  Arrays are
[nz][nr] (r fastest), float64.

Initial profiles:
  * sphere / bubble: the tanh profile of Eq. 41 (bubble = 1 - sphere)
  * ellipsoid: Eq. 46
  * thread: Eq. 47 with d = amp cos(2 pi z / lambda + theta)
  * p2: drop with radius R0 (1 + eps P2(cos theta)) (n = 2 shape mode)
  * flat: planar tanh interface (the 1-D equilibrium profile)
"""
from __future__ import annotations

import math

import numpy as np

CS2 = 1.0 / 3.0

# MRT rates of the paper's runs (Sec. 3.1): s0=s1=s2=s7=s8=1 and s3..s6 = 1/tau_f
# for f; s = 1 for g except s1 = s7 = s8 = 1/tau_g.  A negative value means
# "derived from the mobility (f) or from the local viscosity (g)".
SF_PAPER = (1.0, 1.0, 1.0, -1.0, -1.0, -1.0, -1.0, 1.0, 1.0)
SG_PAPER = (1.0, -1.0, 1.0, 1.0, 1.0, 1.0, 1.0, -1.0, -1.0)

# The same rate choice for the raw-moment collision (collision = 1), whose
# moments are 1, c_z, c_r, c_z^2 + c_r^2, c_z^2 - c_r^2, c_z c_r, c_z^2 c_r,
# c_z c_r^2, c_z^2 c_r^2: for f the first and third moments relax with
# 1/tau_f; for g the three second moments relax with 1/tau_g.
SF_RAW_PAPER = (1.0, -1.0, -1.0, 1.0, 1.0, 1.0, -1.0, -1.0, 1.0)
SG_RAW_PAPER = (1.0, 1.0, 1.0, -1.0, -1.0, -1.0, 1.0, 1.0, 1.0)
COLLISIONS = {"orthogonal": 0, "raw": 1}

PRECISIONS = {"fp64": 0, "fp32": 1, "mix_fp16": 2, "mix_bf16": 3}


def _coords(nz: int, nr: int):
    z = np.arange(nz, dtype=np.float64)[:, None] + 0.5
    r = np.arange(nr, dtype=np.float64)[None, :] + 0.5
    return z, r


def phi_sphere(nz, nr, zc, R, W):
    z, r = _coords(nz, nr)
    d = np.sqrt((z - zc) ** 2 + r ** 2)
    return 0.5 + 0.5 * np.tanh(2.0 * (R - d) / W)


def phi_bubble(nz, nr, zc, R, W):
    return 1.0 - phi_sphere(nz, nr, zc, R, W)


def phi_ellipsoid(nz, nr, zc, Rz, Rr, W):
    z, r = _coords(nz, nr)
    Re = (Rr * Rr * Rz) ** (1.0 / 3.0)
    q = np.sqrt((z - zc) ** 2 / Rz ** 2 + r ** 2 / Rr ** 2)
    return 0.5 + 0.5 * np.tanh(2.0 * Re * (1.0 - q) / W)


def phi_p2(nz, nr, zc, R0, eps, W):
    z, r = _coords(nz, nr)
    d = np.sqrt((z - zc) ** 2 + r ** 2)
    c = (z - zc) / np.maximum(d, 1e-300)
    Rs = R0 * (1.0 + eps * 0.5 * (3.0 * c * c - 1.0))
    return 0.5 + 0.5 * np.tanh(2.0 * (Rs - d) / W)


def phi_thread(nz, nr, R, amp, lam, theta, W):
    z, r = _coords(nz, nr)
    d = amp * np.cos(2.0 * math.pi * z / lam + theta)
    return 0.5 + 0.5 * np.tanh(2.0 * (R + d - r) / W) + 0.0 * z


def phi_flat(nz, nr, zi, W, axis="z"):
    """Planar interface, liquid (phi=1) below zi along the chosen axis."""
    z, r = _coords(nz, nr)
    x = z if axis == "z" else r
    return (0.5 + 0.5 * np.tanh(2.0 * (zi - x) / W)) + 0.0 * (z + r)


SHAPES = {"flat": 0, "sphere": 1, "ellipsoid": 2, "p2": 3, "thread": 4, "bubble": 5}


def phi_from_shape(nz, nr, shape: str, args):
    a = list(args)
    if shape == "sphere":
        return phi_sphere(nz, nr, a[0], a[1], a[2])
    if shape == "bubble":
        return phi_bubble(nz, nr, a[0], a[1], a[2])
    if shape == "ellipsoid":
        return phi_ellipsoid(nz, nr, a[0], a[1], a[2], a[3])
    if shape == "p2":
        return phi_p2(nz, nr, a[0], a[1], a[2], a[3])
    if shape == "thread":
        return phi_thread(nz, nr, a[0], a[1], a[2], a[3], a[4])
    if shape == "flat":
        return phi_flat(nz, nr, a[0], a[1], "z" if (len(a) < 3 or a[2] == 0) else "r")
    raise ValueError(shape)


# ------------------------------------------------------------------ cases
def base_case(**kw) -> dict:
    c = dict(nr=16, nz=32, z_periodic=0, p_coupling=0, collision=0, precision="fp64",
             rho_l=1.0, rho_g=1e-3, nu_l=0.1, nu_g=0.1, sigma=0.01, W=4.0,
             mobility=0.1, grav_z=0.0, sf=list(SF_PAPER), sg=list(SG_PAPER), n_eps=1e-12)
    c.update(kw)
    return c


def with_raw_collision(case: dict) -> dict:
    """The case with the raw-moment collision and the paper's rate choice in that basis."""
    c = dict(case)
    c.update(collision=1, sf=list(SF_RAW_PAPER), sg=list(SG_RAW_PAPER))
    return c


def static_drop(nr=64, nz=128, R=16.0, zc=None, ratio=1000.0, **kw):
    """Static droplet on the axis: walls elsewhere, rho_l = 1, rho_g = 1/ratio,
    sigma = 0.01, W = 4, M = 0.1, tau_l = tau_g = 0.8 (nu = 0.1)."""
    zc = nz / 2.0 if zc is None else zc
    c = base_case(nr=nr, nz=nz, rho_l=1.0, rho_g=1.0 / ratio, nu_l=0.1, nu_g=0.1,
                  sigma=0.01, W=4.0, mobility=0.1)
    c.update(shape="sphere", shape_args=[zc, R, 4.0], steps=2000)
    c.update(kw)
    c["shape_args"][-1] = c["W"]
    return c


def oscillating_drop(nr=128, nz=256, R0=32.0, eps=0.05, zc=None, ratio=100.0, **kw):
    """P2-perturbed drop: rho_l = 1, rho_g = 1/ratio, nu_l = nu_g = 0.1 (the
    viscosity of the paper's oscillation runs), sigma = 0.005, W = 4, M = 0.05."""
    zc = nz / 2.0 if zc is None else zc
    c = base_case(nr=nr, nz=nz, rho_l=1.0, rho_g=1.0 / ratio, nu_l=0.1, nu_g=0.1,
                  sigma=0.005, W=4.0, mobility=0.05)
    c.update(shape="p2", shape_args=[zc, R0, eps, 4.0], steps=20000)
    c.update(kw)
    c["shape_args"][-1] = c["W"]
    return c


def paper_ellipsoid(Rr=30.0, ratio=100.0, Rz=90.0, **kw):
    """The paper's oscillating ellipsoid (Sec. 3.2, Tables 1 and 2): a 300 x 150
    (z x r) domain, periodic in z, drop centred at (150, 0) with half-axes
    R_z = 90 and R_r, in the paper's density scale rho_g = 1, rho_l = ratio;
    W = 4, sigma = 0.3, M = 0.01, nu_l = nu_g = 0.1, the paper's rates."""
    c = base_case(nr=150, nz=300, z_periodic=1, rho_l=float(ratio), rho_g=1.0, nu_l=0.1, nu_g=0.1,
                  sigma=0.3, W=4.0, mobility=0.01)
    c.update(shape="ellipsoid", shape_args=[150.0, float(Rz), float(Rr), 4.0], steps=60000)
    c.update(kw)
    c["shape_args"][-1] = c["W"]
    return c


def thread_breakup(nr=64, R0=20.0, k_wave=0.7, amp_frac=0.1, seed=None, **kw):
    """Liquid thread on the axis, periodic z of one wavelength lambda = 2 pi R0 / k
    (nz = ceil(lambda)), radius perturbation amp_frac * R0 with a seeded phase."""
    nz = int(math.ceil(2.0 * math.pi * R0 / k_wave))
    theta = 0.0 if seed is None else float(np.random.default_rng(seed).uniform(0.0, 2 * math.pi))
    c = base_case(nr=nr, nz=nz, z_periodic=1, rho_l=1.0, rho_g=1e-3, nu_l=0.1, nu_g=0.1,
                  sigma=0.01, W=4.0, mobility=0.01)
    c.update(shape="thread", shape_args=[R0, amp_frac * R0, float(nz), theta, 4.0],
             steps=30000, precision="mix_fp16")
    c.update(kw)
    c["shape_args"][-1] = c["W"]
    return c


def paper_thread(wavelength=600, ratio=100.0, **kw):
    """The paper's liquid thread (Sec. 3.3): an N_z x N_r = wavelength x 200
    domain, periodic in z as in its static and oscillating drop tests,
    Eq. 47 with R = 60 and d = 0.1 R cos(2 pi z / wavelength); sigma = 0.3,
    W = 4, M = 0.01, nu_l = nu_g = 0.1, the paper's rates, in its density
    scale rho_g = 1, rho_l = ratio.  Wavelengths 600, 1200, 1800 give the wave
    numbers k = 2 pi R / wavelength = 0.63, 0.31, 0.21 whose breakup times the
    paper prints."""
    R = 60.0
    c = base_case(nr=200, nz=int(wavelength), z_periodic=1, rho_l=float(ratio), rho_g=1.0, nu_l=0.1, nu_g=0.1,
                  sigma=0.3, W=4.0, mobility=0.01)
    c.update(shape="thread", shape_args=[R, 0.1 * R, float(wavelength), 0.0, 4.0])
    c.update(kw)
    c["shape_args"][-1] = c["W"]
    return c


def capillary_time(R, rho_l, sigma):
    """sqrt(R^3 rho_l / sigma), the time unit of Sec. 3.3."""
    return math.sqrt(R ** 3 * rho_l / sigma)


def rising_bubble(nr=256, nz=1024, R=32.0, zc=128.0, **kw):
    """Bubble R = 32 on the axis at z = 128: rho ratio 1000, W = 5.
    With nu_l = 0.08: Eo = g drho D^2 / sigma = 10 and
    Mo = g mu_l^4 drho / (rho_l^2 sigma^3) = 1e-3 give sigma = 0.01 and
    g = 2.444e-5.  nu_g = 0.16 (mu_l / mu_g = 500) keeps both relaxation
    rates inside the scheme's stable range, and the mobility is 0.05: with
    M = 0.02 this case turns non-finite after ~7000 steps in every precision."""
    sigma = 0.01
    D = 2.0 * R
    rho_l, rho_g = 1.0, 1e-3
    g = 10.0 * sigma / ((rho_l - rho_g) * D * D)
    c = base_case(nr=nr, nz=nz, rho_l=rho_l, rho_g=rho_g, nu_l=0.08, nu_g=0.16,
                  sigma=sigma, W=5.0, mobility=0.05, grav_z=-g)
    c.update(shape="bubble", shape_args=[zc, R, 5.0], steps=50000, precision="fp32")
    c.update(kw)
    c["shape_args"][-1] = c["W"]
    return c


def batched_cases(n=512, seed=20181022, precision="fp32"):
    """n independent droplet cases: nr ~ U{64..256}, nz ~ U{128..512} (steps of
    16), R ~ U[0.2, 0.35] nr, density ratio in {10, 100, 1000}; half static
    drops, half P2-oscillating drops (amplitude 0.05).  nz is raised, when
    needed, to hold the drop plus two interface widths at each end."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        nr = int(rng.integers(4, 17)) * 16
        nz = int(rng.integers(8, 33)) * 16
        R = float(rng.uniform(0.2, 0.35)) * nr
        ratio = float(rng.choice([10.0, 100.0, 1000.0]))
        kind = "static" if rng.uniform() < 0.5 else "oscillating"
        nz_min = int(math.ceil((2.0 * R * 1.06 + 16.0) / 16.0)) * 16
        nz = max(nz, nz_min)
        if kind == "static":
            c = static_drop(nr=nr, nz=nz, R=R, ratio=ratio)
        else:
            c = oscillating_drop(nr=nr, nz=nz, R0=R, ratio=ratio)
        c["precision"] = precision
        c["kind"] = kind
        out.append(c)
    return out


def initial_phi(case: dict) -> np.ndarray:
    return phi_from_shape(case["nz"], case["nr"], case["shape"], case["shape_args"])


def small_cases():
    """Small grids spanning several tiles with a ragged tail, for parity tests."""
    return {
        "static_walls": static_drop(nr=40, nz=72, R=12.0, steps=50),
        "static_periodic": static_drop(nr=37, nz=66, R=11.0, z_periodic=1, steps=50),
        "oscillating": oscillating_drop(nr=48, nz=90, R0=16.0, steps=50),
        "thread": dict(thread_breakup(nr=33, R0=10.0), precision="fp64", steps=50),
        "bubble": rising_bubble(nr=40, nz=100, R=10.0, zc=30.0, steps=50, precision="fp64",
                                grav_z=-2e-4),
    }
