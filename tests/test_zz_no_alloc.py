"""The allocation-free diagnostics reduction (lbm_diag_reduce_noalloc).

Some callers cannot allocate device memory at the moment they want the
diagnostics (their memory is held by their own pool, or they poll inside a
loop that must not allocate).  lbm_diag_reduce_noalloc serves them with a
fixed static scratch array in the library.  Its output must equal the
handle-based lbm_diagnostics for the same fields, call after call.

This file is collected last on purpose: the test must also pass after every
other test has run in the same process (the static scratch keeps the previous
call's contents).
"""
import ctypes

import numpy as np
import pytest

from paper_1810_09299_gb300 import lbm, workloads as W

pytestmark = pytest.mark.gpu

KEYS = ("step", "mass", "kinetic", "z_centroid", "dp", "umax", "phi_min", "phi_max",
        "axis_half_length", "radial_half_length", "nonfinite")


def _reference(case, steps):
    sim = lbm.Simulation(case)
    sim.init_case(0)
    sim.step(steps)
    F = sim.fields()
    d = sim.diagnostics()
    sim.close()
    return np.stack([F[k] for k in ("phi", "rho", "uz", "ur", "p")]), d


def test_noalloc_reduction_matches_lbm_diagnostics_on_two_calls():
    torch = pytest.importorskip("torch")
    L = lbm.lib()
    cases = [W.static_drop(nr=48, nz=80, R=14.0),
             dict(W.oscillating_drop(nr=37, nz=66, R0=12.0), precision="fp32", z_periodic=1)]
    stream = torch.cuda.current_stream()
    for steps, case in zip((30, 45), cases):
        fields, ref = _reference(case, steps)
        d_fields = torch.from_numpy(np.ascontiguousarray(fields)).to("cuda")
        d_out = torch.full((11,), float("nan"), dtype=torch.float64, device="cuda")
        rc = L.lbm_diag_reduce_noalloc(ctypes.c_void_p(d_fields.data_ptr()), case["nz"], case["nr"],
                                       int(case.get("z_periodic", 0)), float(steps),
                                       ctypes.c_void_p(d_out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == lbm.LBM_OK, lbm.strerror(rc)
        torch.cuda.synchronize()
        out = d_out.cpu().numpy()
        for i, k in enumerate(KEYS):
            assert abs(out[i] - ref[k]) <= 1e-12 * max(abs(ref[k]), 1e-300), (k, out[i], ref[k])


def test_noalloc_rejects_bad_sizes_without_device_work():
    L = lbm.lib()
    dummy = ctypes.c_void_p(16)
    assert L.lbm_diag_reduce_noalloc(dummy, 70000, 70000, 0, 0.0, dummy, None) == lbm.LBM_ERR_INVALID_ARG
    assert L.lbm_diag_reduce_noalloc(dummy, 0, 8, 0, 0.0, dummy, None) == lbm.LBM_ERR_INVALID_ARG
    assert L.lbm_diag_reduce_noalloc(None, 8, 8, 0, 0.0, dummy, None) == lbm.LBM_ERR_INVALID_ARG
