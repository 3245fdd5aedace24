"""Pins of the oracle's diagnostics record against what the mathematics fixes.

The diagnostics are the quantities Sec. 3.1-3.3 read off the runs: the
conserved sum of r phi (the drop volume over 2 pi), the kinetic energy, the
drop centroid, the pressure jump of Laplace's law, the spurious-velocity
maximum, the extrema of phi and the interface positions on the axis and
along r.  Each test below fixes one field of the record by a closed form of
the initial shapes (Eq. 41, Eq. 46), a symmetry, a textbook flow or the
support of the stencils (Eq. 39-40), so that a dropped r weight, a shifted
node coordinate or a wrong half-cell rule fails a test.  The CUDA
diagnostics are compared with these records in the GPU tests.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1810_09299_gb300 import workloads as W


def _diag(case, phi0, steps=0):
    o = oracle.Oracle(case).init(phi0)
    if steps:
        o.step(steps)
    return o, o.diagnostics()


def _diffuse_sphere_volume(R, Wd):
    """Volume of the tanh drop of Eq. 41: the sharp sphere plus the first
    moment of the odd profile correction, 4/3 pi R^3 + pi^3 R W^2 / 12."""
    return 4.0 / 3.0 * math.pi * R ** 3 + math.pi ** 3 * R * Wd ** 2 / 12.0


@pytest.mark.parametrize("R", [10.0, 16.0])
def test_mass_is_volume_over_two_pi(R):
    """mass = sum r phi, so 2 pi mass is the drop volume (r-weighted sum over
    the meridian plane; the midpoint rule in r leaves an axis term of order
    R / (12 R^3))."""
    case = W.static_drop(nr=48, nz=96, R=R)
    _, d = _diag(case, W.initial_phi(case))
    V = 2.0 * math.pi * d["mass"]
    assert abs(V / _diffuse_sphere_volume(R, 4.0) - 1.0) < 3e-3


def test_z_centroid_of_a_mirror_symmetric_drop():
    """A drop centred at z_c = nz / 2 is mirror-symmetric on the lattice
    (z_k = k + 1/2), so its centroid is z_c up to rounding."""
    case = W.static_drop(nr=40, nz=96, R=14.0)
    _, d = _diag(case, W.initial_phi(case))
    assert abs(d["z_centroid"] - 48.0) < 1e-11


def test_z_centroid_is_volume_weighted():
    """Two separated drops: the centroid is the volume-weighted mean of their
    centres (an unweighted or area-weighted sum would give 78 here)."""
    nz, nr = 128, 40
    phi = W.phi_sphere(nz, nr, 30.0, 8.0, 4.0) + W.phi_sphere(nz, nr, 90.0, 16.0, 4.0)
    _, d = _diag(W.static_drop(nr=nr, nz=nz, R=8.0), phi)
    V1, V2 = _diffuse_sphere_volume(8.0, 4.0), _diffuse_sphere_volume(16.0, 4.0)
    assert abs(d["z_centroid"] - (V1 * 30.0 + V2 * 90.0) / (V1 + V2)) < 0.05


def test_interface_half_lengths_of_an_ellipsoid():
    """Eq. 46 puts phi = 1/2 on the ellipse (z - z_c)^2 / R_z^2 + r^2 / R_r^2 = 1.
    On the axis row (r = 1/2) the phi > 1/2 set has half-length
    R_z sqrt(1 - 1/(4 R_r^2)); on the row nearest the centroid the radial
    crossing is at R_r sqrt(1 - ((z_row - z_c) / R_z)^2)."""
    nz, nr, zc, Rz, Rr = 160, 48, 80.0, 30.0, 18.0
    _, d = _diag(W.static_drop(nr=nr, nz=nz, R=8.0), W.phi_ellipsoid(nz, nr, zc, Rz, Rr, 4.0))
    assert abs(d["axis_half_length"] - Rz * math.sqrt(1.0 - 0.25 / Rr ** 2)) < 0.01
    z_row = math.floor(d["z_centroid"]) + 0.5
    assert abs(d["radial_half_length"] - Rr * math.sqrt(1.0 - ((z_row - zc) / Rz) ** 2)) < 0.01


def test_axis_length_counts_the_half_cell_to_a_wall():
    """Liquid from the wall plane z = 0 up to a flat interface at z = 20: the
    phi > 1/2 set on the axis is 20 long (the first node sits half a cell from
    the wall), half-length 10.  Its extrema are those of the initial profile."""
    nz, nr = 64, 8
    phi = W.phi_flat(nz, nr, 20.0, 4.0)
    _, d = _diag(W.static_drop(nr=nr, nz=nz, R=8.0), phi)
    assert abs(d["axis_half_length"] - 10.0) < 1e-12
    assert d["phi_max"] == pytest.approx(phi.max(), abs=1e-14)
    assert d["phi_min"] == pytest.approx(phi.min(), abs=1e-14)


def test_axis_length_of_a_periodic_thread():
    """An unbroken thread in a z-periodic box is liquid along the whole axis:
    half-length nz / 2."""
    case = W.thread_breakup(nr=24, R0=8.0)
    _, d = _diag(dict(case, precision="fp64"), W.initial_phi(case))
    assert abs(d["axis_half_length"] - case["nz"] / 2.0) < 1e-12


@pytest.fixture(scope="module")
def poiseuille():
    """Uniform fluid in a pipe of radius nr, z-periodic, driven by gravity:
    u_z(r) = G (R^2 - r^2) / (4 rho nu) (Hagen-Poiseuille)."""
    nr, nz, nu, rho = 16, 4, 0.1, 1.0
    c = W.base_case(nr=nr, nz=nz, z_periodic=1, rho_l=2.0, rho_g=rho, nu_l=nu, nu_g=nu, sigma=0.0,
                    mobility=0.1, grav_z=-1e-5)
    o, d = _diag(c, np.zeros((nz, nr)), steps=15000)
    r = np.arange(nr) + 0.5
    G = (rho - 2.0) * -1e-5
    u = G * (nr ** 2 - r ** 2) / (4 * rho * nu)
    return d, u, r, rho, nz


def test_kinetic_energy_of_pipe_flow(poiseuille):
    """kinetic = sum over nodes of r rho |u|^2 / 2, against the analytic profile."""
    d, u, r, rho, nz = poiseuille
    ke = nz * np.sum(0.5 * r * rho * u ** 2)
    assert abs(d["kinetic"] / ke - 1.0) < 0.02


def test_umax_of_pipe_flow(poiseuille):
    d, u, r, rho, nz = poiseuille
    assert abs(d["umax"] / u.max() - 1.0) < 0.01


def test_pressure_jump_is_the_difference_of_r_weighted_phase_means():
    """dp = <p> over phi > 0.99 minus <p> over phi < 0.01, each mean weighted
    by r.  A prescribed pressure field p(k, j) = a + b r_j + c z_k is put into
    the hydrodynamic populations as g = g^eq(p, u = 0) (Eq. 25) with no
    surface tension and no gravity, so the velocity is zero and Eq. 33 gives
    the prescribed p back; dp must then be the difference of the r-weighted
    means of that field over the two phases (its r dependence makes an
    unweighted mean differ).  The lagged coupling with p^{n-1} = 0 keeps the
    pressure term out of u_r (Eq. 32), so u = 0 and Eq. 33 returns p."""
    case = W.static_drop(nr=40, nz=72, R=14.0, sigma=0.0, p_coupling=1)
    phi0 = W.initial_phi(case)
    o = oracle.Oracle(case).init(phi0)
    f, _ = o.populations()
    nz, nr = phi0.shape
    r = np.arange(nr) + 0.5
    z = np.arange(nz) + 0.5
    p = 2e-3 + 1e-4 * r[None, :] - 3e-5 * z[:, None] * np.ones((1, nr))
    rho = phi0 * case["rho_l"] + (1.0 - phi0) * case["rho_g"]
    g = np.zeros((9, nz, nr))
    for k in range(nz):
        for j in range(nr):
            g[:, k, j] = oracle.geq(r[j], p[k, j], rho[k, j], 0.0, 0.0)
    o.set_populations(f, g)
    F = o.fields()
    assert np.max(np.abs(F["p"] - p)) < 1e-15 and np.max(np.abs(F["uz"])) == 0.0
    d = o.diagnostics()
    R2 = np.broadcast_to(r[None, :], p.shape)
    liq, gas = phi0 > 0.99, phi0 < 0.01
    want = np.sum(R2[liq] * p[liq]) / np.sum(R2[liq]) - np.sum(R2[gas] * p[gas]) / np.sum(R2[gas])
    assert d["dp"] == pytest.approx(want, rel=1e-12)
    assert abs(want - (p[liq].mean() - p[gas].mean())) > 1e-3 * abs(want)


def test_nonfinite_nodes_are_counted_and_left_out():
    """A NaN in phi at one interior node reaches u and p through the stencils
    of Eq. 39-40: the node itself and its 16 stencil neighbours (distance 1
    and 2 along the eight lattice directions).  Those 17 nodes are counted and
    left out of every sum, so the mass is that of the other nodes."""
    case = W.static_drop(nr=40, nz=72, R=12.0)
    phi = W.initial_phi(case)
    k0, j0 = 30, 20
    phi[k0, j0] = np.nan
    _, d = _diag(case, phi)
    cz = [1, 0, -1, 0, 1, -1, -1, 1]
    cr = [0, 1, 0, -1, 1, 1, -1, -1]
    support = {(k0, j0)} | {(k0 + s * a, j0 + s * b) for a, b in zip(cz, cr) for s in (1, 2)}
    assert d["nonfinite"] == len(support) == 17
    keep = np.ones_like(phi, dtype=bool)
    for k, j in support:
        keep[k, j] = False
    r = np.arange(case["nr"]) + 0.5
    assert d["mass"] == pytest.approx(np.sum((r[None, :] * phi)[keep]), rel=1e-13)
    for key in ("kinetic", "z_centroid", "dp", "umax", "phi_min", "phi_max"):
        assert math.isfinite(d[key]), key
