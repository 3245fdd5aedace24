"""Pipelined diagnostics (lbm_case_diagnostics_enqueue / lbm_diagnostics_wait)
through the C ABI (needs a GB300).

A loop that reads one record per step enqueues step n + 1 before it waits for
record n, so the GPU never waits for the host.  The records it gets must be
the very records lbm_case_diagnostics returns at the same steps (same kernels,
same summation order), here checked bit for bit on two batched cases.
"""
import ctypes

import numpy as np
import pytest

from paper_1810_09299_gb300 import lbm, workloads as W

pytestmark = pytest.mark.gpu


def _cases():
    return [dict(W.static_drop(nr=48, nz=96, R=12.0), precision="fp32"),
            dict(W.oscillating_drop(nr=64, nz=128, R0=20.0), precision="fp32")]


def _pinned_records(n):
    torch = pytest.importorskip("torch")
    bufs = [torch.zeros(11, dtype=torch.float64).pin_memory() for _ in range(n)]
    return bufs, [lbm.LbmDiag.from_address(b.data_ptr()) for b in bufs]


def _as_tuple(d):
    return tuple(getattr(d, k) for k, _ in lbm.LbmDiag._fields_)


def test_pipelined_records_equal_synchronous_ones():
    steps, case = 12, 1
    # synchronous reference: one record per step
    ref = lbm.Simulation(_cases())
    for i in range(2):
        ref.init_case(i)
    expect = []
    for _ in range(steps):
        ref.step(1)
        d = ref.diagnostics(case)
        expect.append(tuple(d[k] for k, _ in lbm.LbmDiag._fields_))
    # pipelined: record n is waited for after step n + 1 is enqueued
    sim = lbm.Simulation(_cases())
    for i in range(2):
        sim.init_case(i)
    keep, recs = _pinned_records(2)
    got = []
    for n in range(steps):
        sim.step(1)
        sim.diagnostics_enqueue(case, recs[n % 2], n % 2)
        if n > 0:
            assert sim.diagnostics_wait((n - 1) % 2) == lbm.LBM_OK
            got.append(_as_tuple(recs[(n - 1) % 2]))
    assert sim.diagnostics_wait((steps - 1) % 2) == lbm.LBM_OK
    got.append(_as_tuple(recs[(steps - 1) % 2]))
    assert len(got) == steps
    for n, (g, e) in enumerate(zip(got, expect)):
        assert g[0] == n + 1  # the record's step count
        np.testing.assert_array_equal(np.array(g), np.array(e))
    del keep


def test_pipelined_argument_checks():
    sim = lbm.Simulation(_cases()[0])
    L = lbm.lib()
    keep, recs = _pinned_records(1)
    h = sim.handle
    # no initial condition yet
    assert L.lbm_case_diagnostics_enqueue(h, 0, ctypes.byref(recs[0]), 0) == lbm.LBM_ERR_STATE
    sim.init_case(0)
    assert L.lbm_case_diagnostics_enqueue(h, 1, ctypes.byref(recs[0]), 0) == lbm.LBM_ERR_INVALID_ARG
    assert L.lbm_case_diagnostics_enqueue(h, 0, None, 0) == lbm.LBM_ERR_INVALID_ARG
    assert L.lbm_case_diagnostics_enqueue(h, 0, ctypes.byref(recs[0]), lbm.DIAG_SLOTS) == lbm.LBM_ERR_INVALID_ARG
    assert L.lbm_diagnostics_wait(h, -1) == lbm.LBM_ERR_INVALID_ARG
    assert L.lbm_diagnostics_wait(h, 2) == lbm.LBM_ERR_STATE  # nothing pending there
    sim.step(3)
    sim.diagnostics_enqueue(0, recs[0], 3)
    assert sim.diagnostics_wait(3) == lbm.LBM_OK
    assert recs[0].step == 3
    assert sim.diagnostics_wait(3) == lbm.LBM_ERR_STATE  # already collected
    del keep
