"""The raw-moment (non-orthogonal) MRT option through the C ABI against the
FP64 oracle's raw-moment option (needs a GB300).  Cases with the paper's rate
choice in the raw basis run the kernels specialised for it; SF_ANY / SG_ANY
and the mixed-basis batch run the general-rate kernels.

The CUDA path keeps the orthogonal moments it already forms and maps their
deviations into the raw basis and back with fixed combinations; the oracle
uses the raw basis matrix and its Gauss-Jordan inverse in velocity space.
FP64 must agree to the same 1e-11 as the orthogonal scheme; FP32 and 16-bit
storage to the bounds of their orthogonal counterparts.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1810_09299_gb300 import lbm, workloads as W
from tests.test_gpu_parity import FIELDS, TOL_FP64, _errors, field_errors, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

# rates of the nine raw moments, none of them the paper's pattern (general kernels)
SF_ANY = [1.0, 0.9, 0.9, 1.2, 1.1, 1.0, 0.8, 0.85, 1.3]
SG_ANY = [1.0, 1.05, 0.95, -1.0, -1.0, -1.0, 1.15, 1.1, 0.9]


def test_raw_fp64_matches_oracle_static_drop_full():
    case = W.with_raw_collision(W.static_drop())
    sim = run_gpu(case, case["steps"])
    ref_o = run_oracle(case, case["steps"])
    errs = field_errors(sim.fields(), ref_o.fields())
    assert all(e <= TOL_FP64 for e in errs.values()), errs
    dg, do = sim.diagnostics(), ref_o.diagnostics()
    for k in ("mass", "kinetic", "dp", "umax"):
        assert abs(dg[k] - do[k]) <= 1e-9 * max(abs(do[k]), 1e-12), (k, dg[k], do[k])


@pytest.mark.parametrize("zper,pc", [(0, 0), (1, 0), (0, 1)])
def test_raw_fp64_general_rates(zper, pc):
    case = W.with_raw_collision(W.static_drop(nr=37, nz=60, R=11.0, z_periodic=zper, p_coupling=pc,
                                              ratio=100.0, grav_z=-2e-6))
    case.update(sf=list(SF_ANY), sg=list(SG_ANY))
    got = run_gpu(case, 300).fields()
    ref = run_oracle(case, 300).fields()
    errs = field_errors(got, ref)
    assert all(e <= TOL_FP64 for e in errs.values()), errs


def test_raw_fp64_oscillating_drop():
    """128 x 256 P2 drop, 10 steps.  In the raw scheme the oracle itself turns a
    1e-15 perturbation of phi0 into relative differences of phi of 1.4e-15 at
    step 10, 6e-13 at step 20 and 2e-10 at step 40 (the orthogonal scheme stays
    near 1e-13 to step 300), so round-off parity is checked inside that
    horizon; the longer static-drop run above is not sensitive that way."""
    case = W.with_raw_collision(W.oscillating_drop())
    got = run_gpu(case, 10).fields()
    ref = run_oracle(case, 10).fields()
    errs = field_errors(got, ref)
    assert all(e <= TOL_FP64 for e in errs.values()), errs


@pytest.mark.parametrize("nr,nz,zper", [(2, 2, 0), (2, 3, 1), (33, 5, 1)])
def test_raw_fp64_edge_grids(nr, nz, zper):
    case = W.with_raw_collision(W.static_drop(nr=nr, nz=nz, R=max(nr, nz) / 2.0, z_periodic=zper))
    got = run_gpu(case, 10).fields()
    ref = run_oracle(case, 10).fields()
    errs = field_errors(got, ref)
    assert all(e <= TOL_FP64 for e in errs.values()), errs


def test_raw_and_orthogonal_cases_in_one_batch():
    """A batch may mix the two bases: each case matches its own oracle run."""
    cases = [W.with_raw_collision(W.static_drop(nr=40, nz=64, R=12.0)),
             W.static_drop(nr=50, nz=48, R=10.0, z_periodic=1)]
    sim = lbm.Simulation(cases)
    for i, c in enumerate(cases):
        sim.init_phase(i, "host_array", phi=W.initial_phi(c))
    sim.step(200)
    for i, c in enumerate(cases):
        errs = field_errors(sim.fields(i), run_oracle(c, 200).fields())
        assert all(e <= TOL_FP64 for e in errs.values()), (i, errs)


@pytest.mark.parametrize("prec,phi_tol", [("fp32", (2e-3, 1e-4)), ("mix_fp16", (2e-2, 5e-4))])
def test_raw_reduced_precision_static_drop(prec, phi_tol):
    """FP32 / 16-bit storage with the raw-moment collision: mass drift below
    1e-6 and the phi errors against the FP64 oracle within the bounds of the
    orthogonal scheme."""
    case = dict(W.with_raw_collision(W.static_drop()), precision=prec)
    sim = run_gpu(case, 0)
    m0 = sim.diagnostics()["mass"]
    sim.step(2000)
    d = sim.diagnostics()
    assert abs(d["mass"] - m0) / m0 < 1e-6, (d["mass"], m0)
    e = _errors(sim.fields(), run_oracle(case, 2000).fields())
    print(prec, "raw errors (max, L2):", e)
    assert e["phi"][0] < phi_tol[0] and e["phi"][1] < phi_tol[1], e


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mix_fp16"])
def test_raw_launch_variants_bit_identical(prec):
    """Every launch shape computes the same numbers with the raw-moment
    collision (its compile-time rate mode; walls and periodic z)."""
    for case in (dict(W.with_raw_collision(W.static_drop(nr=45, nz=70, R=12.0)), precision=prec),
                 dict(W.with_raw_collision(W.thread_breakup(nr=40, R0=12.0)), precision=prec)):
        ref = None
        for v in range(lbm.num_variants()):
            f = run_gpu(case, 40, variant=v).fields()
            if ref is None:
                ref = f
            for k in FIELDS:
                assert np.array_equal(f[k], ref[k]), (prec, v, k)
