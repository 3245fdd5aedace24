"""lbm_init_phase_all through the C ABI (needs a GB300): initialising every case
of a batch from one concatenated host array gives the same state, bit for
bit, as initialising the cases one by one."""
import numpy as np
import pytest

from paper_1810_09299_gb300 import lbm, workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mix_fp16"])
def test_init_all_equals_per_case_init(prec):
    cases = [dict(W.static_drop(nr=40, nz=72, R=10.0), precision=prec),
             dict(W.oscillating_drop(nr=64, nz=96, R0=18.0), precision=prec),
             dict(W.thread_breakup(nr=32, R0=8.0), precision=prec)]
    one = lbm.Simulation(cases)
    for i in range(len(cases)):
        one.init_case(i)
    allc = lbm.Simulation(cases)
    phi_all = np.concatenate([W.initial_phi(c).ravel() for c in cases])
    allc.init_all(np.ascontiguousarray(phi_all))
    for sim in (one, allc):
        sim.step(7)
    for i in range(len(cases)):
        for a, b in zip(one.state(i), allc.state(i)):
            np.testing.assert_array_equal(a, b)
        assert one.diagnostics(i) == allc.diagnostics(i)
    with pytest.raises(AssertionError):
        allc.init_all(phi_all[:-1])  # wrong size is refused before the call
    assert lbm.lib().lbm_init_phase_all(allc.handle, None) == lbm.LBM_ERR_INVALID_ARG
