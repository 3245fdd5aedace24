"""Failure detection without faulting the GPU.

A device wait that cannot complete gives up after a bounded number of polls
and reports through a status word (the host turns it into LBM_ERR_TIMEOUT);
the context stays usable afterwards.  Non-finite states are reported as
LBM_ERR_NONFINITE (see test_gpu_parity.test_errors_reported)."""
import ctypes

import numpy as np
import pytest

from paper_1810_09299_gb300 import lbm, workloads as W

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    torch = pytest.importorskip("torch")
    L = lbm.lib()
    word = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream()
    rc = L.lbm_selftest_bounded_wait(2000, ctypes.c_void_p(st.cuda_stream), ctypes.c_void_p(word.data_ptr()))
    assert rc == lbm.LBM_ERR_TIMEOUT
    assert int(word.item()) == 1
    assert L.lbm_selftest_bounded_wait(0, None, ctypes.c_void_p(word.data_ptr())) == lbm.LBM_ERR_INVALID_ARG
    # the device is still usable
    case = W.static_drop(nr=20, nz=24, R=6.0)
    sim = lbm.Simulation(case)
    sim.init_case(0)
    sim.step(5)
    assert sim.diagnostics()["nonfinite"] == 0


def test_autotune_leaves_the_state_untouched():
    case = dict(W.oscillating_drop(nr=64, nz=96, R0=20.0), precision="mix_fp16")
    a = lbm.Simulation(case)
    a.init_case(0)
    a.step(7)
    v = a.autotune(reps=2)
    assert 0 <= v < lbm.num_variants()
    a.step(5)
    b = lbm.Simulation(case)
    b.init_case(0)
    b.step(12)
    fa, fb = a.fields(), b.fields()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
    assert a.diagnostics()["step"] == 12
