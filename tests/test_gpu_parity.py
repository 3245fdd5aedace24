"""CUDA path vs the FP64 oracle, through the C ABI (needs a GB300).

FP64: relative max-norm max|gpu - oracle| / max|oracle| <= 1e-11 on phi, rho,
u_z, u_r and p after N steps.  Reduced precisions: the max and L2 errors
against the FP64 oracle stay within the bounds derived in the design notes
(FP32 rounding of ~1e-7 per step accumulated over the run; 16-bit storage
rounding of ~2.4e-4 (FP16) / 2e-3 (BF16) per population), and the mass stays
conserved to FP32 rounding.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1810_09299_gb300 import lbm, workloads as W

pytestmark = pytest.mark.gpu

FIELDS = ("phi", "rho", "uz", "ur", "p")
TOL_FP64 = 1e-11
# Scale floors of the relative max-norm: max|a - b| <= tol * max(max|b|, floor).
# u and p of a nearly static state are pure round-off noise (|u| ~ 1e-6 on a
# 2 x 2 grid); the floors keep the comparison relative to the scale of the
# problem rather than to that noise.
FLOOR = {"phi": 1.0, "rho": 1e-3, "uz": 1e-4, "ur": 1e-4, "p": 1e-6}


def rel(a, b, floor=1e-300):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), floor))


def field_errors(got, ref):
    return {k: rel(got[k], ref[k], FLOOR[k]) for k in FIELDS}


def run_gpu(case, steps, phi0=None, variant=None):
    phi0 = W.initial_phi(case) if phi0 is None else phi0
    sim = lbm.Simulation(case)
    if variant is not None:
        sim.set_variant(variant)
    sim.init_phase(0, "host_array", phi=phi0)
    sim.step(steps)
    return sim


def run_oracle(case, steps, phi0=None):
    phi0 = W.initial_phi(case) if phi0 is None else phi0
    return oracle.Oracle(dict(case, precision="fp64")).init(phi0).step(steps)


@pytest.mark.parametrize("name", sorted(W.small_cases()))
def test_fp64_matches_oracle_small_cases(name):
    case = W.small_cases()[name]
    sim = run_gpu(case, case["steps"])
    got = sim.fields()
    ref = run_oracle(case, case["steps"]).fields()
    errs = field_errors(got, ref)
    assert all(e <= TOL_FP64 for e in errs.values()), errs


def test_fp64_matches_oracle_static_drop_full():
    """64 x 128 static drop, ratio 1000, 2000 steps (the FP64 parity workload)."""
    case = W.static_drop()
    sim = run_gpu(case, case["steps"])
    got = sim.fields()
    ref_o = run_oracle(case, case["steps"])
    ref = ref_o.fields()
    errs = field_errors(got, ref)
    assert all(e <= TOL_FP64 for e in errs.values()), errs
    dg, do = sim.diagnostics(), ref_o.diagnostics()
    for k in ("mass", "kinetic", "z_centroid", "dp", "umax", "axis_half_length", "radial_half_length"):
        assert abs(dg[k] - do[k]) <= 1e-9 * max(abs(do[k]), 1e-12), (k, dg[k], do[k])


def test_fp64_matches_oracle_oscillating_drop_full():
    """128 x 256 P2 drop, 250 steps.  Beyond ~300 steps the oracle itself turns a
    1e-15 perturbation of phi0 into 1e-12..1e-5 differences (the interface normal
    grad(phi)/|grad(phi)| is discontinuous where phi overshoots 1 inside the
    liquid), so round-off parity is checked inside that horizon."""
    case = W.oscillating_drop()
    got = run_gpu(case, 250).fields()
    ref = run_oracle(case, 250).fields()
    errs = field_errors(got, ref)
    assert all(e <= TOL_FP64 for e in errs.values()), errs


@pytest.mark.parametrize("nr,nz,zper", [(2, 2, 0), (2, 3, 1), (3, 2, 0), (33, 5, 1), (5, 41, 0)])
def test_fp64_edge_grids(nr, nz, zper):
    """Degenerate grids (the drop fills the domain and touches every wall).  These
    states amplify round-off fast (1e-15 -> 1e-8 in 30 steps in the oracle
    itself), so the comparison is made after 10 steps."""
    case = W.static_drop(nr=nr, nz=nz, R=max(nr, nz) / 2.0, z_periodic=zper)
    got = run_gpu(case, 10).fields()
    ref = run_oracle(case, 10).fields()
    errs = field_errors(got, ref)
    assert all(e <= TOL_FP64 for e in errs.values()), errs


def test_fp64_one_step_from_perturbed_state():
    """Arbitrary (non-equilibrium) populations set through lbm_set_state."""
    case = W.static_drop(nr=37, nz=45, R=10.0, grav_z=-1e-5)
    rng = np.random.default_rng(5)
    o = run_oracle(case, 0)
    f, g = o.populations()
    f = f * (1 + 1e-3 * rng.standard_normal(f.shape))
    g = g + 1e-4 * rng.standard_normal(g.shape)
    cz, cr, pp = o.aux()
    cz = cz + 1e-4 * rng.standard_normal(cz.shape)
    o.set_populations(f, g)
    o.set_aux(cz, cr, pp)
    sim = lbm.Simulation(case)
    sim.set_state(0, f, g, np.stack([cz, cr, pp]))
    f2, g2, aux2 = sim.state(0)
    assert np.array_equal(f2, f) and np.array_equal(g2, g)
    sim.step(1)
    o.step(1)
    fo, go = o.populations()
    fg, gg, auxg = sim.state(0)
    assert rel(fg, fo) <= TOL_FP64 and rel(gg, go) <= TOL_FP64
    assert rel(auxg[0], o.aux()[0]) <= TOL_FP64


@pytest.mark.parametrize("pc", [0, 1])
def test_fp64_pressure_couplings(pc):
    case = W.static_drop(nr=40, nz=72, R=12.0, p_coupling=pc)
    got = run_gpu(case, 100).fields()
    ref = run_oracle(case, 100).fields()
    errs = field_errors(got, ref)
    assert all(e <= TOL_FP64 for e in errs.values()), errs


def test_variants_graph_and_direct_are_bit_identical():
    case = W.static_drop(nr=45, nz=70, R=12.0)
    ref = None
    for v in range(lbm.num_variants()):
        f = run_gpu(case, 70, variant=v).fields()  # 70 steps = graph replays + direct remainder
        if ref is None:
            ref = f
        for k in FIELDS:
            assert np.array_equal(f[k], ref[k]), (v, k)
    sim = lbm.Simulation(case)
    sim.init_case(0)
    for _ in range(70):
        sim.step(1)
    f = sim.fields()
    for k in FIELDS:
        assert np.array_equal(f[k], ref[k]), k


@pytest.mark.parametrize("prec", ["fp32", "mix_fp16", "mix_bf16"])
def test_launch_variants_bit_identical_reduced_precision(prec):
    """Every launch shape (register-staged and TMA-staged tiles) computes the
    same numbers, also for periodic z (ghost rows wrap around)."""
    for case in (dict(W.static_drop(nr=45, nz=70, R=12.0), precision=prec),
                 dict(W.thread_breakup(nr=40, R0=12.0), precision=prec)):
        ref = None
        for v in range(lbm.num_variants()):
            f = run_gpu(case, 40, variant=v).fields()
            if ref is None:
                ref = f
            for k in FIELDS:
                assert np.array_equal(f[k], ref[k]), (prec, v, k)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mix_fp16"])
def test_batch_equals_single_cases(prec):
    cases = [dict(W.static_drop(nr=40, nz=64, R=10.0), precision=prec),
             dict(W.oscillating_drop(nr=33, nz=50, R0=10.0), precision=prec),
             dict(W.thread_breakup(nr=24, R0=8.0), precision=prec)]
    b = lbm.Simulation(cases)
    for i, c in enumerate(cases):
        b.init_case(i, c)
    b.step(40)
    for i, c in enumerate(cases):
        s = run_gpu(c, 40).fields()
        f = b.fields(i)
        for k in FIELDS:
            assert np.array_equal(f[k], s[k]), (i, k)


def test_checkpoint_resume_bit_identical():
    case = dict(W.oscillating_drop(nr=48, nz=90, R0=16.0), precision="mix_fp16")
    a = run_gpu(case, 50)
    blob = a.checkpoint()
    a.step(30)
    fa = a.fields()
    b = lbm.Simulation(case)
    b.restore(blob)
    b.step(30)
    fb = b.fields()
    for k in FIELDS:
        assert np.array_equal(fa[k], fb[k]), k
    assert b.diagnostics()["step"] == 80


@pytest.mark.parametrize("shape", ["sphere", "bubble", "ellipsoid", "p2", "thread", "flat"])
def test_builtin_shapes_match_input_generator(shape):
    nz, nr = 70, 45
    args = {"sphere": [30.0, 12.0, 4.0], "bubble": [30.0, 12.0, 5.0], "ellipsoid": [35.0, 20.0, 10.0, 4.0],
            "p2": [35.0, 14.0, 0.1, 4.0], "thread": [12.0, 1.2, 70.0, 0.3, 4.0], "flat": [33.0, 4.0, 0.0]}[shape]
    case = W.static_drop(nr=nr, nz=nz, R=10.0)
    sim = lbm.Simulation(case)
    sim.init_phase(0, shape, args)
    got = sim.fields(which=("phi",))["phi"]
    ref = W.phi_from_shape(nz, nr, shape, args)
    assert np.max(np.abs(got - ref)) < 1e-13


def test_errors_reported():
    case = W.static_drop(nr=16, nz=16, R=4.0)
    sim = lbm.Simulation(case)
    with pytest.raises(lbm.LbmError) as e:
        sim.step(1)  # before init
    assert e.value.code == lbm.LBM_ERR_STATE
    phi = W.initial_phi(case)
    phi[3, 3] = np.nan
    sim.init_phase(0, "host_array", phi=phi)
    sim.step(0)
    d = sim.diagnostics(check=False)
    assert d["status"] == lbm.LBM_ERR_NONFINITE and d["nonfinite"] >= 1
    with pytest.raises(lbm.LbmError):
        sim.step(1)  # sticky
    sim2 = lbm.Simulation(case)
    sim2.init_case(0)
    with pytest.raises(lbm.LbmError) as e:
        sim2.init_phase(0, "sphere", [1.0, 2.0])  # wrong arg count
    assert e.value.code == lbm.LBM_ERR_INVALID_ARG


# ---------------------------------------------------------------- reduced precision
def _errors(got, ref):
    out = {}
    for k in FIELDS:
        d = got[k] - ref[k]
        out[k] = (float(np.max(np.abs(d))), float(np.sqrt(np.mean(d * d))))
    return out


def test_fp32_static_drop_error_vs_oracle():
    """FP32 arithmetic: max / L2 errors against the FP64 oracle after 2000 steps."""
    case = dict(W.static_drop(), precision="fp32")
    sim = run_gpu(case, 2000)
    got = sim.fields()
    ref_o = run_oracle(case, 2000)
    ref = ref_o.fields()
    e = _errors(got, ref)
    print("fp32 errors (max, L2):", e)
    assert e["phi"][0] < 2e-3 and e["phi"][1] < 1e-4, e
    m_g, m_o = sim.diagnostics()["mass"], ref_o.diagnostics()["mass"]
    assert abs(m_g - m_o) / m_o < 1e-6


@pytest.mark.parametrize("prec,phi_tol", [("mix_fp16", (2e-2, 5e-4)), ("mix_bf16", (0.2, 1e-2))])
def test_mixed_precision_static_drop(prec, phi_tol):
    """Mass drift < 1e-6 relative and Laplace law within 1 % (FP16), errors stated."""
    case = dict(W.static_drop(), precision=prec)
    sim = run_gpu(case, 0)
    m0 = sim.diagnostics()["mass"]
    sim.step(2000)
    d = sim.diagnostics()
    assert abs(d["mass"] - m0) / m0 < 1e-6, (d["mass"], m0)
    got = sim.fields()
    ref = run_oracle(case, 2000).fields()
    e = _errors(got, ref)
    print(prec, "errors (max, L2):", e)
    assert e["phi"][0] < phi_tol[0] and e["phi"][1] < phi_tol[1], e
    if prec == "mix_fp16":
        r = np.arange(case["nr"])[None, :] + 0.5
        R_eff = (3 * 2 * math.pi * np.sum(r * got["phi"]) / (4 * math.pi)) ** (1 / 3)
        lap = 2 * case["sigma"] / R_eff
        assert abs(d["dp"] - lap) / lap < 0.01, (d["dp"], lap)


@pytest.mark.parametrize("prec", ["fp32", "mix_fp16", "mix_bf16"])
@pytest.mark.parametrize("case", ["static_drop", "thread"])
def test_population_sum_is_conserved_by_the_ledger(prec, case):
    """The step conserves the sum of all populations (sum r phi, Eq. 16):
    in FP16 storage exactly (every value the f_0 ledger adds lies on its
    column grid, so its FP32 sums are exact: the exact sums of the stored
    state before and after 500 steps are equal bit for bit), in FP32 and
    bfloat16 storage to the double-float ledger's ~2^-48.  z walls and axis
    (static drop), periodic z (thread)."""
    c = dict(W.static_drop() if case == "static_drop" else W.thread_breakup(), precision=prec)
    sim = run_gpu(c, 0)
    total0 = math.fsum(sim.state()[0].ravel())
    sim.step(500)
    total = math.fsum(sim.state()[0].ravel())
    assert sim.diagnostics()["nonfinite"] == 0
    sim.close()
    print(prec, case, "sum of populations", total0, total, (total - total0) / total0)
    if prec == "mix_fp16":
        assert total == total0
    else:
        assert abs(total - total0) <= 1e-13 * total0


def test_diagnostics_leave_out_nonfinite_nodes_like_the_oracle():
    """One NaN in phi0 reaches u and p of its 16 stencil neighbours (Eq. 39-40).
    The GPU record and the oracle record both count those 17 nodes and leave
    them out of every sum and extremum, so the two records agree."""
    case = W.static_drop(nr=40, nz=72, R=12.0)
    phi = W.initial_phi(case)
    phi[30, 20] = np.nan
    sim = lbm.Simulation(case)
    sim.init_phase(0, "host_array", phi=phi)
    dg = sim.diagnostics(check=False)
    do = oracle.Oracle(case).init(phi).diagnostics()
    assert dg["status"] == lbm.LBM_ERR_NONFINITE
    assert dg["nonfinite"] == do["nonfinite"] == 17
    for k in ("mass", "kinetic", "z_centroid", "dp", "umax", "phi_min", "phi_max", "axis_half_length",
              "radial_half_length"):
        assert math.isfinite(dg[k]), k
        assert abs(dg[k] - do[k]) <= 1e-12 * max(abs(do[k]), 1e-12), (k, dg[k], do[k])
