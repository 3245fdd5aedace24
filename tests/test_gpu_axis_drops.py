"""Drops along the axis (lbm_case_axis_drops) on the GPU (needs a GB300).

* Parity: the device diagnostic against the oracle's restatement on the same
  states (separated drops, a drop across a periodic boundary, an unbroken
  thread, a walled case, a stepped state): the same drop count, crossings
  to 1e-9 and volumes to 1e-10 relative.
* The paper's thread-breakup experiment (Sec. 3.3) at its own setup: the
  breakup times against the printed ones (a cited fixture under golden/),
  and the main and satellite drop sizes against the trends the paper states
  (its Fig. 7 values are not in the text).  FP32 storage and arithmetic; the
  FP64 path gives the same times (see the design notes).
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1810_09299_gb300 import lbm, workloads as W

pytestmark = pytest.mark.gpu


def _states():
    nz, nr = 160, 40
    two = W.phi_sphere(nz, nr, 40.0, 10.0, 4.0) + W.phi_sphere(nz, nr, 110.0, 16.0, 4.0)
    z = np.arange(120) + 0.5
    zz = np.minimum(z, 120 - z)
    r = np.arange(40) + 0.5
    wrap = 0.5 + 0.5 * np.tanh(2.0 * (12.0 - np.sqrt(zz[:, None] ** 2 + r[None, :] ** 2)) / 4.0)
    three = (W.phi_sphere(200, 40, 30.0, 8.0, 4.0) + W.phi_sphere(200, 40, 90.0, 14.0, 4.0)
             + W.phi_sphere(200, 40, 160.0, 10.0, 4.0))
    thread = dict(W.thread_breakup(nr=24, R0=8.0), precision="fp64")
    return {
        "two_walls": (W.static_drop(nr=nr, nz=nz, R=8.0), two, 0),
        "two_periodic": (W.static_drop(nr=nr, nz=nz, R=8.0, z_periodic=1), two, 0),
        "across_boundary": (W.static_drop(nr=40, nz=120, R=8.0, z_periodic=1), wrap, 0),
        "three_walls": (W.static_drop(nr=40, nz=200, R=8.0), three, 0),
        "thread": (thread, W.initial_phi(thread), 0),
        "stepped_two_periodic": (W.static_drop(nr=nr, nz=nz, R=8.0, z_periodic=1), two, 40),
    }


STATES = _states()


@pytest.mark.parametrize("name", sorted(STATES))
def test_axis_drops_match_oracle(name):
    case, phi, steps = STATES[name]
    sim = lbm.Simulation(case)
    sim.init_phase(0, "host_array", phi=phi)
    sim.step(steps)
    got, n, (pmin, zmin) = sim.axis_drops(0)
    ref, n_ref, (pmin_ref, zmin_ref) = oracle.Oracle(case).init(phi).step(steps).axis_drops()
    assert n == n_ref and len(got) == len(ref)
    assert abs(pmin - pmin_ref) < 1e-12
    if steps == 0:  # (after steps the gas holds near-ties of tiny phi values)
        assert zmin == zmin_ref
    for g, o in zip(got, ref):
        for k in ("z_start", "z_end"):
            assert abs(g[k] - o[k]) < 1e-9, (k, g, o)
        for k in ("volume", "radius"):
            assert abs(g[k] - o[k]) <= 1e-10 * abs(o[k]), (k, g, o)


def test_axis_drops_argument_checks():
    case, phi, _ = STATES["two_walls"]
    sim = lbm.Simulation(case)
    with pytest.raises(lbm.LbmError) as e:
        sim.axis_drops(0)  # before the initial condition
    assert e.value.code == lbm.LBM_ERR_STATE
    sim.init_phase(0, "host_array", phi=phi)
    with pytest.raises(lbm.LbmError):
        sim.axis_drops(0, max_drops=lbm.MAX_AXIS_DROPS + 1)
    drops, n, _ = sim.axis_drops(0, max_drops=1)
    assert n == 2 and len(drops) == 1


# ---------------------------------------------------------------- the paper's thread
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "thread_breakup_times.txt")
R_THREAD = 60.0
# Breakup is detected by polling the axis every POLL steps: a resolution of
# 0.012 (ratio 100) and 0.019 (ratio 10) capillary times.
POLL = {100.0: 100, 10.0: 50}
# Relaxation after the last breakup, in capillary times, before the drop
# sizes are read.
RELAX = 8.0


def _paper_times():
    out = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            ratio, k, lam, t = line.split()
            out[(float(ratio), int(lam))] = (float(k), float(t))
    return out


def _run_threads(ratio, prec):
    """The three wavelengths of one density ratio as one batch: the step at
    which each thread first pinches (least axis phi below 1/2), then the drop
    sizes R*/R after RELAX more capillary times (drops with R*/R > 0.1)."""
    lams = (600, 1200, 1800)
    cases = [dict(W.paper_thread(lam, ratio), precision=prec) for lam in lams]
    sim = lbm.Simulation(cases)
    for i, c in enumerate(cases):
        sim.init_phase(i, "host_array", phi=W.initial_phi(c))
    tc = W.capillary_time(R_THREAD, ratio, 0.3)
    broke, n, end = [None] * 3, 0, None
    most = [0] * 3
    while end is None or n < end:
        sim.step(POLL[ratio])
        n += POLL[ratio]
        for i in range(3):
            drops, nd, (pmin, _) = sim.axis_drops(i)
            if broke[i] is None and pmin < 0.5:
                broke[i] = n
            if broke[i] is not None:
                most[i] = max(most[i], sum(1 for d in drops if d["radius"] / R_THREAD > 0.1))
        if end is None and all(b is not None for b in broke):
            end = n + int(RELAX * tc)
        assert n < 60 * tc, ("no breakup", broke)
    out = {}
    for i, lam in enumerate(lams):
        drops, nd, _ = sim.axis_drops(i)
        sizes = sorted(d["radius"] / R_THREAD for d in drops if d["radius"] / R_THREAD > 0.1)
        vol = sum(d["volume"] for d in drops)
        out[lam] = {"t_break": broke[i] / tc, "sizes": sizes, "most_drops": most[i], "volume": vol,
                    "nonfinite": sim.diagnostics(i)["nonfinite"]}
    sim.close()
    return out


@pytest.fixture(scope="module")
def threads():
    return {ratio: _run_threads(ratio, "fp32") for ratio in (100.0, 10.0)}


def test_breakup_times_match_the_paper(threads):
    """Within 2 % of the printed times (measured: at most 0.8 % off)."""
    for (ratio, lam), (k, t_paper) in _paper_times().items():
        t = threads[ratio][lam]["t_break"]
        print(f"ratio {ratio:g} k {k} breakup {t:.2f} paper {t_paper}")
        assert abs(t - t_paper) / t_paper < 0.02, (ratio, k, t, t_paper)


def test_main_and_satellite_drop_after_breakup(threads):
    """Each thread ends as one main drop and one satellite (one wavelength
    per domain), and the drops hold the thread's volume
    pi R^2 wavelength (1 + 0.005) (Eq. 47 with the 0.1 R cosine)."""
    for ratio, res in threads.items():
        for lam, r in res.items():
            print(f"ratio {ratio:g} wavelength {lam}: drops R*/R {r['sizes']}, most drops at once {r['most_drops']}")
            assert r["nonfinite"] == 0
            assert len(r["sizes"]) == 2, (ratio, lam, r["sizes"])
            v_thread = math.pi * R_THREAD ** 2 * lam * (1.0 + 0.5 * 0.1 ** 2)
            assert abs(r["volume"] / v_thread - 1.0) < 5e-3, (ratio, lam, r["volume"], v_thread)


def test_drop_size_trends_of_sec_3_3(threads):
    """Sec. 3.3: both drops shrink as the wave number grows; the satellite is
    smaller, and the main drop larger, at the larger density ratio."""
    for ratio, res in threads.items():
        sat = [res[lam]["sizes"][0] for lam in (1800, 1200, 600)]   # k = 0.21, 0.31, 0.63
        main = [res[lam]["sizes"][1] for lam in (1800, 1200, 600)]
        assert sat[0] > sat[1] > sat[2] and main[0] > main[1] > main[2], (ratio, sat, main)
    for lam in (600, 1200, 1800):
        s100, s10 = threads[100.0][lam]["sizes"], threads[10.0][lam]["sizes"]
        assert s100[0] < s10[0] and s100[1] > s10[1], (lam, s100, s10)
