"""Pins of the oracle's drops-on-the-axis diagnostic (the bodies a breaking
thread forms, Sec. 3.3) against closed forms of the initial shapes.

Each maximal run of phi > 1/2 on the axis row is one drop; its ends are the
interpolated phi = 1/2 crossings, its volume 2 pi sum r phi over its rows (each
gas gap split at its lightest row).  Separated tanh drops (Eq. 41) must come
out with the volume 4/3 pi R^3 + pi^3 R W^2 / 12 of a diffuse sphere and with
ends at z_c -+ sqrt(R^2 - 1/4) (the axis row lies at r = 1/2); a periodic
unbroken thread is one body; a drop across a periodic boundary is one drop.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1810_09299_gb300 import workloads as W


def _vol(R, Wd=4.0):
    return 4.0 / 3.0 * math.pi * R ** 3 + math.pi ** 3 * R * Wd ** 2 / 12.0


def _drops(case, phi):
    return oracle.Oracle(case).init(phi).axis_drops()


@pytest.mark.parametrize("zper", [0, 1])
def test_two_separated_drops(zper):
    nz, nr = 160, 40
    phi = W.phi_sphere(nz, nr, 40.0, 10.0, 4.0) + W.phi_sphere(nz, nr, 110.0, 16.0, 4.0)
    drops, n, (pmin, zmin) = _drops(W.static_drop(nr=nr, nz=nz, R=8.0, z_periodic=zper), phi)
    assert n == 2
    for d, zc, R in zip(drops, (40.0, 110.0), (10.0, 16.0)):
        half = math.sqrt(R * R - 0.25)
        assert abs(d["z_start"] - (zc - half)) < 0.02 and abs(d["z_end"] - (zc + half)) < 0.02
        assert abs(d["volume"] / _vol(R) - 1.0) < 5e-3
        assert abs(d["radius"] - (3 * d["volume"] / (4 * math.pi)) ** (1 / 3)) < 1e-12
    assert pmin < 1e-6


def test_drop_across_a_periodic_boundary_is_one_drop():
    """A drop centred at z = 0 of a periodic box: one drop from z = nz - R to R."""
    nz, nr, R = 120, 40, 12.0
    z = np.arange(nz) + 0.5
    zz = np.minimum(z, nz - z)  # distance to z = 0 across the boundary
    r = np.arange(nr) + 0.5
    d = np.sqrt(zz[:, None] ** 2 + r[None, :] ** 2)
    phi = 0.5 + 0.5 * np.tanh(2.0 * (R - d) / 4.0)
    drops, n, _ = _drops(W.static_drop(nr=nr, nz=nz, R=8.0, z_periodic=1), phi)
    half = math.sqrt(R * R - 0.25)
    assert n == 1
    assert abs(drops[0]["z_start"] - (nz - half)) < 0.02 and abs(drops[0]["z_end"] - half) < 0.02
    assert abs(drops[0]["volume"] / _vol(R) - 1.0) < 5e-3


def test_unbroken_thread_is_one_body():
    case = dict(W.thread_breakup(nr=24, R0=8.0), precision="fp64")
    phi = W.initial_phi(case)
    drops, n, (pmin, _) = _drops(case, phi)
    assert n == 1 and drops[0]["z_start"] == 0.0 and drops[0]["z_end"] == case["nz"]
    r = np.arange(case["nr"]) + 0.5
    assert drops[0]["volume"] == pytest.approx(2 * math.pi * np.sum(r[None, :] * phi), rel=1e-12)
    assert pmin > 0.5


def test_every_row_belongs_to_one_drop():
    """The drops' volumes add up to the whole 2 pi sum r phi, and each gap is
    cut at its lightest row (three drops of different sizes, walls)."""
    nz, nr = 200, 40
    phi = (W.phi_sphere(nz, nr, 30.0, 8.0, 4.0) + W.phi_sphere(nz, nr, 90.0, 14.0, 4.0)
           + W.phi_sphere(nz, nr, 160.0, 10.0, 4.0))
    case = W.static_drop(nr=nr, nz=nz, R=8.0)
    drops, n, _ = _drops(case, phi)
    r = np.arange(nr) + 0.5
    total = 2 * math.pi * np.sum(r[None, :] * phi)
    assert n == 3
    assert sum(d["volume"] for d in drops) == pytest.approx(total, rel=1e-12)
    # the first drop owns the rows up to the lightest row between 30 + 8 and 90 - 14
    w = np.sum(r[None, :] * phi, axis=1)
    gap = np.arange(int(math.ceil(30 + 8)), int(90 - 14))
    gap = gap[phi[gap, 0] <= 0.5]
    cut = gap[np.argmin(w[gap])]
    assert drops[0]["volume"] == pytest.approx(2 * math.pi * np.sum(w[:cut]), rel=1e-12)


def test_gas_only_axis_has_no_drops():
    nz, nr = 64, 16
    _, n, (pmin, _) = _drops(W.static_drop(nr=nr, nz=nz, R=8.0, z_periodic=1), np.zeros((nz, nr)))
    assert n == 0 and pmin == 0.0
