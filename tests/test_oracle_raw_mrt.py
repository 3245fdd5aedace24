"""Pins of the oracle's raw-moment (non-orthogonal) MRT option (CPU).

The paper's summary (Sec. 4) names the non-orthogonal MRT as a direct
extension of its orthogonal model.  The option keeps the collisions of
Eq. 10 / Eq. 24 and replaces M by the raw-moment basis 1, c_z, c_r,
c_z^2 + c_r^2, c_z^2 - c_r^2, c_z c_r, c_z^2 c_r, c_z c_r^2, c_z^2 c_r^2.
What fixes it independently of the oracle's own code:
- the raw moments of f^eq (Eq. 11) have closed forms from the lattice sums
  sum w_i = 1, sum w_i c_a c_b = cs2 delta_ab, sum w_i c_z^2 c_r^2 = 1/9;
- a diagonal rate matrix acts the same in any basis whose rows span the same
  subspaces per rate: with rate s on {c_z, c_r, c_z^2 c_r, c_z c_r^2} and 1
  elsewhere the raw collision is the paper's f-collision (rate s on j and q,
  Sec. 2.2), since q_z = 3 c_z c_r^2 - 2 c_z and q_r = 3 c_z^2 c_r - 2 c_r;
- a single rate is BGK in every basis (Sec. 2.2), so a single-rate run is
  the same in both bases, s_p of Eq. 33 included;
- the whole scheme keeps Laplace's law and conserves mass.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import analytic as A
from paper_1810_09299_gb300 import workloads as W

RNG = np.random.default_rng(1810)


def _rand(n):
    return RNG.uniform(-1.0, 1.0, size=n)


@pytest.mark.parametrize("trial", range(6))
def test_raw_moments_of_feq_closed_form(trial):
    r, phi = RNG.uniform(0.5, 40.0), RNG.uniform(-0.1, 1.1)
    uz, ur, mob = _rand(1)[0] * 0.05, _rand(1)[0] * 0.05, RNG.uniform(0.01, 0.2)
    k = oracle.matrix_T() @ oracle.feq(r, phi, uz, ur, mob)
    chi_z, chi_r = r * phi * uz, r * phi * ur + mob * phi
    ref = [r * phi, chi_z, chi_r, 2.0 / 3.0 * r * phi, 0.0, 0.0, chi_r / 3.0, chi_z / 3.0, r * phi / 9.0]
    assert np.allclose(k, ref, rtol=0, atol=1e-13 * max(1.0, r))


def test_raw_basis_inverse():
    T, Ti = oracle.matrix_T(), oracle.matrix_Tinv()
    assert np.max(np.abs(Ti @ T - np.eye(9))) < 1e-14
    # the rest population is k_0 - k_3 + k_8 (the i = 0 row of T^-1 used for s_p)
    assert np.allclose(Ti[0], [1, 0, 0, -1, 0, 0, 0, 0, 1], atol=1e-15)


@pytest.mark.parametrize("s", [0.55, 1.0, 1.3, 1.85])
def test_raw_with_paper_f_rates_is_the_orthogonal_f_collision(s):
    x, xeq, src = _rand(9), _rand(9), 0.1 * _rand(9)
    raw = oracle.raw_collide(x, xeq, src, np.array([1, s, s, 1, 1, 1, s, s, 1.0]))
    ortho = oracle.mrt_collide(x, xeq, src, np.array([1, 1, 1, s, s, s, s, 1, 1.0]))
    assert np.max(np.abs(raw - ortho)) <= 1e-13 * np.max(np.abs(ortho))


@pytest.mark.parametrize("s", [0.6, 1.0, 1.7])
def test_raw_with_a_single_rate_is_bgk(s):
    x, xeq, src = _rand(9), _rand(9), 0.1 * _rand(9)
    got = oracle.raw_collide(x, xeq, src, np.full(9, s))
    bgk = x - s * (x - xeq) + (1 - s / 2) * src
    assert np.max(np.abs(got - bgk)) <= 1e-14 * np.max(np.abs(bgk))


def test_raw_g_collision_is_a_different_operator():
    """With the paper's g rates (second moments at 1/tau_g) the raw basis does
    not span the orthogonal rate subspaces (e = 3 c^2 - 4 mixes the zeroth moment
    in), so the two hydrodynamic collisions differ."""
    s = 1.0 / 0.8
    x, xeq, src = _rand(9), _rand(9), 0.1 * _rand(9)
    raw = oracle.raw_collide(x, xeq, src, np.array([1, 1, 1, s, s, s, 1, 1, 1.0]))
    ortho = oracle.mrt_collide(x, xeq, src, np.array([1, s, 1, 1, 1, 1, 1, s, s]))
    assert np.max(np.abs(raw - ortho)) > 1e-3
    # both keep the same momentum (rate 1 on c_z, c_r in both)
    T = oracle.matrix_T()
    assert np.allclose((T @ raw)[1:3], (T @ ortho)[1:3], atol=1e-14)


def _single_rate_case(collision, z_periodic):
    c = W.static_drop(nr=20, nz=32, R=7.0, ratio=10.0, z_periodic=z_periodic, grav_z=-1e-5)
    c.update(collision=collision, sf=[-1.0] * 9, sg=[-1.0] * 9)
    return c


@pytest.mark.parametrize("zper", [0, 1])
def test_single_rate_runs_agree_in_both_bases(zper):
    """Single-rate f and g (BGK with the local 1/tau_g): the raw and orthogonal
    runs are the same scheme, s_p of Eq. 33 included (both give 1/s - 1/2)."""
    out = []
    for coll in (0, 1):
        case = _single_rate_case(coll, zper)
        o = oracle.Oracle(case).init(W.initial_phi(case))
        o.step(150)
        out.append(o.fields())
    for k in ("phi", "uz", "ur", "p"):
        scale = max(1e-12, np.max(np.abs(out[0][k])))
        assert np.max(np.abs(out[1][k] - out[0][k])) <= 1e-11 * scale, k


@pytest.mark.parametrize("zper", [0, 1])
def test_raw_mass_conserved_to_roundoff(zper):
    case = W.with_raw_collision(W.static_drop(nr=20, nz=32, R=7.0, z_periodic=zper, ratio=10.0, grav_z=-1e-5))
    o = oracle.Oracle(case).init(W.initial_phi(case))
    m0 = o.diagnostics()["mass"]
    o.step(300)
    assert abs(o.diagnostics()["mass"] - m0) <= 1e-13 * m0


def test_raw_laplace_law_static_drop():
    """The raw-moment scheme on the static drop (64 x 128, R = 16, ratio 1000):
    Laplace's law within 1 % with R_eff from the drop volume.  4000 steps: at
    2000 the drop is still ringing in both bases (|u|max about 8e-3), the
    orthogonal run 0.5 % and the raw one 1.4 % from the law; at 4000 both are
    within 0.15 %."""
    case = W.with_raw_collision(W.static_drop())
    o = oracle.Oracle(case).init(W.initial_phi(case))
    m0 = o.diagnostics()["mass"]
    o.step(4000)
    d = o.diagnostics()
    F = o.fields()
    r = np.arange(case["nr"])[None, :] + 0.5
    V = 2 * math.pi * np.sum(r * F["phi"])
    R_eff = (3 * V / (4 * math.pi)) ** (1 / 3)
    dp_th = A.laplace_jump(case["sigma"], R_eff)
    assert abs(d["dp"] - dp_th) / dp_th < 0.01, (d["dp"], dp_th)
    assert abs(d["mass"] - m0) / m0 < 1e-12


def test_raw_hagen_poiseuille_pipe_flow():
    """Shear rates in the raw basis: uniform gas in a pipe of radius nr, periodic
    in z, driven by G_z.  u_z(r) = G (R^2 - r^2) / (4 rho nu) within 1 %, which
    holds only if the three second raw moments relax with 1/tau_g (Eq. 34)."""
    nr, nu, rho = 16, 0.1, 1.0
    c = W.with_raw_collision(W.base_case(nr=nr, nz=4, z_periodic=1, rho_l=2.0, rho_g=rho, nu_l=nu, nu_g=nu,
                                         sigma=0.0, mobility=0.1, grav_z=-1e-5))
    o = oracle.Oracle(c).init(np.zeros((4, nr)))
    o.step(15000)
    F = o.fields()
    r = np.arange(nr) + 0.5
    G = (rho - 2.0) * -1e-5
    ex = G * (nr ** 2 - r ** 2) / (4 * rho * nu)
    assert np.max(np.abs(F["uz"][0] - ex)) / ex.max() < 0.01
    assert np.max(np.abs(F["ur"])) < 1e-3 * ex.max()


def test_raw_oscillating_drop_frequency_miller_scriven():
    """The n = 2 oscillation of a P2-deformed drop in the raw scheme within 10 %
    of Eq. 43, as the orthogonal scheme (reduced grid 60 x 120, R0 = 20)."""
    pytest.importorskip("scipy")
    from tests.test_oracle_pins import _fit_frequency
    case = W.with_raw_collision(W.oscillating_drop(nr=60, nz=120, R0=20.0, eps=0.1, sigma=0.01))
    o = oracle.Oracle(case).init(W.initial_phi(case))
    Re = (3 * o.diagnostics()["mass"] * 2 * math.pi / (4 * math.pi)) ** (1 / 3)
    ts, L = [], []
    for _ in range(200):
        o.step(25)
        ts.append(o.steps)
        L.append(o.diagnostics()["axis_half_length"])
    ts, L = np.array(ts, float), np.array(L)
    w_th = A.miller_scriven_frequency(2, Re, case["rho_l"], case["rho_g"], case["nu_l"], case["nu_g"],
                                      case["sigma"])
    sel = ts > 300
    w = _fit_frequency(ts[sel], L[sel], w_th)
    assert abs(w - w_th) / w_th < 0.10, (w, w_th)


def _stokes_cell(collision, n, A0=2e-3, T0=400):
    """A decaying axisymmetric cellular flow of uniform gas with u_r != 0:
    u from the Stokes stream function psi = A r^2 (R^2 - r^2)^2 sin(kz) / R^4
    (no slip at the wall r = R = nr, periodic in z), g = g^eq(p = 0, rho, u).
    Grid 24n x 48n, amplitude 1/n and T0 n^2 steps (diffusive scaling);
    returns u_z averaged over n x n blocks, scaled back by n."""
    nr, nz = 24 * n, 48 * n
    R, k, A = float(nr), 2 * math.pi / nz, A0 / n
    z = np.arange(nz)[:, None] + 0.5
    r = np.arange(nr)[None, :] + 0.5
    uz = A / R ** 4 * (2 * (R ** 2 - r ** 2) ** 2 - 4 * r ** 2 * (R ** 2 - r ** 2)) * np.sin(k * z)
    ur = -A / R ** 4 * r * (R ** 2 - r ** 2) ** 2 * k * np.cos(k * z)
    c = W.base_case(nr=nr, nz=nz, z_periodic=1, rho_l=1.0, rho_g=1.0, nu_l=0.1, nu_g=0.1, sigma=0.0,
                    mobility=0.1)
    if collision:
        c = W.with_raw_collision(c)
    o = oracle.Oracle(c).init(np.zeros((nz, nr)))
    f, _ = o.populations()
    g = np.zeros((9, nz, nr))
    for kk in range(nz):
        for j in range(nr):
            g[:, kk, j] = oracle.geq(r[0, j], 0.0, 1.0, uz[kk, j], ur[kk, j])
    o.set_populations(f, g)
    o.step(T0 * n * n)
    return o.fields()["uz"].reshape(48, n, 24, n).mean(axis=(1, 3)) * n


def test_raw_and_orthogonal_velocities_converge_together():
    """The two hydrodynamic collisions differ, but both must discretise the same
    axisymmetric flow equations: in a flow with u_r != 0 their velocities must
    approach each other under refinement (measured: 2.7 % of max |u_z| apart on
    the 24 x 48 grid, 0.47 % on 48 x 96, 0.14 % on 72 x 144)."""
    d = []
    for n in (1, 2):
        a, b = _stokes_cell(0, n), _stokes_cell(1, n)
        d.append(np.max(np.abs(b - a)) / np.max(np.abs(a)))
    assert d[0] < 0.05 and d[1] < 0.01 and d[1] < d[0] / 4, d


# ---------------------------------------------------------------- s_p of Eq. 33 in the raw basis
def _sp_ortho(s1, s2):
    return (s1 + s2 - s1 * s2) / (2 * s1 * s2)


def _sp_raw(s3, s8):
    return 1.5 / s3 - 0.5 / s8 - 0.5


def _residual_raw_moments(z0=3.0, r0=5.0, eps=1e-6, h=1e-3):
    """Raw moments 0, 3, 8 of v = -c . grad g^eq + T (Appendix C's residual with
    the time derivatives dropped, as the appendix does under incompressibility),
    at one point of a slow incompressible axisymmetric flow of uniform density,
    from the oracle's g^eq (Eq. 25) and T (Eq. 29) with central differences.
    u from a stream function: u_z = psi_r / r, u_r = -psi_z / r."""
    rho = 1.0
    cz, cr, w = oracle.lattice()
    T = oracle.matrix_T()

    def u(z, r):
        # psi = eps r^2 (1 + 0.3 z + 0.1 r + 0.05 z r)
        psi_r = eps * (2 * r * (1 + 0.3 * z + 0.1 * r + 0.05 * z * r) + r * r * (0.1 + 0.05 * z))
        psi_z = eps * r * r * (0.3 + 0.05 * r)
        return psi_r / r, -psi_z / r

    def flux(z, r):  # sum_i T_ki c_i g_i^eq for both components
        uz, ur = u(z, r)
        g = oracle.geq(r, 1e-4 * (1 + 0.2 * z + 0.3 * r), rho, uz, ur)
        return T @ (cz * g), T @ (cr * g)

    div = (flux(z0 + h, r0)[0] - flux(z0 - h, r0)[0]) / (2 * h) + (flux(z0, r0 + h)[1] - flux(z0, r0 - h)[1]) / (2 * h)
    uz, ur = u(z0, r0)
    Tf = oracle.T_force(rho, uz, ur, 0.0, 0.0, 0.0, rho)  # d(r rho) = (0, rho) for uniform rho
    k = -div + T @ Tf
    return k, Tf[0], rho, ur


def test_appendix_c_residual_moments():
    """Premise of s_p in both bases: for the residual of Appendix C the raw moments
    0, 3 and 8 are 0, (2/3) rho u_r and (2/9) rho u_r (lattice sums of Eq. 25 and
    Eq. 29 with div(r u) = 0)."""
    k, T0, rho, ur = _residual_raw_moments()
    scale = abs(rho * ur)
    assert abs(k[0]) < 1e-6 * scale
    assert abs(k[3] - 2.0 / 3.0 * rho * ur) < 1e-6 * scale
    assert abs(k[8] - 2.0 / 9.0 * rho * ur) < 1e-6 * scale
    assert abs(T0 + 4.0 / 9.0 * rho * ur) < 1e-12 * scale


@pytest.mark.parametrize("s_a,s_b", [(1.25, 1.0), (0.7, 1.3), (1.6, 0.9)])
def test_sp_follows_from_appendix_c_in_both_bases(s_a, s_b):
    """(g_0 - g_0^eq) / dt = [B^-1 S^-1 B v]_0 - T_0 / 2 = -s_p w_0 rho u_r
    (Appendix C, Eq. C.6 and C.8) with the numerically formed residual v: the
    orthogonal basis gives the paper's s_p (rates s_1 = s_a of e, s_2 = s_b of
    eps), the raw basis 3/(2 s_3) - 1/(2 s_8) - 1/2 (s_3 = s_a of c^2, s_8 = s_b
    of c_z^2 c_r^2)."""
    k, T0, rho, ur = _residual_raw_moments()
    w0 = 4.0 / 9.0
    # orthogonal: M^-1 row 0 = (1/9, -1/9, 1/9, 0, ...), (M v)_1 = 3 k3 - 4 k0, (M v)_2 = 4 k0 - 6 k3 + 9 k8
    g0_ortho = (k[0] - (3 * k[3] - 4 * k[0]) / s_a + (4 * k[0] - 6 * k[3] + 9 * k[8]) / s_b) / 9.0 - T0 / 2
    Ti = oracle.matrix_Tinv()
    g0_raw = Ti[0, 0] * k[0] + Ti[0, 3] * k[3] / s_a + Ti[0, 8] * k[8] / s_b - T0 / 2
    assert abs(-g0_ortho / (w0 * rho * ur) - _sp_ortho(s_a, s_b)) < 1e-5
    assert abs(-g0_raw / (w0 * rho * ur) - _sp_raw(s_a, s_b)) < 1e-5


@pytest.mark.parametrize("zper", [0, 1])
def test_oracle_pressure_uses_the_raw_sp(zper):
    """Same populations, lagged coupling (u_r does not depend on p): the two
    bases' Eq. 33 pressures differ by -(cs2/(1-w0)) (s_p_raw - s_p_ortho) w0 rho u_r / r."""
    nu = 0.1
    tau = 3 * nu + 0.5
    base = W.static_drop(nr=18, nz=30, R=6.0, z_periodic=zper, ratio=10.0, p_coupling=1)
    base.update(nu_l=nu, nu_g=nu)
    rng = np.random.default_rng(7)
    o0 = oracle.Oracle(base).init(W.initial_phi(base))
    f, g = o0.populations()
    g = g + 1e-4 * rng.standard_normal(g.shape)
    out = []
    for case in (base, W.with_raw_collision(base)):
        o = oracle.Oracle(case).init(W.initial_phi(case))
        o.set_populations(f, g)
        out.append(o.fields())
    a, b = out
    r = np.arange(base["nr"])[None, :] + 0.5
    s = 1.0 / tau
    d_sp = _sp_raw(s, 1.0) - _sp_ortho(s, 1.0)
    expect = -(1.0 / 3.0) / (5.0 / 9.0) * d_sp * (4.0 / 9.0) * a["rho"] * a["ur"] / r
    assert np.allclose(b["ur"], a["ur"], rtol=0, atol=1e-15)
    assert np.max(np.abs((b["p"] - a["p"]) - expect)) < 1e-12 * max(np.max(np.abs(expect)), 1e-30)
