"""Failure detection of the fused step kernel, tested without a GPU fault.

The fused kernel's plane waits are bounded (1 s of the device's global timer, and a cap on the
number of polls); a wait that runs out sets a flag that the next synchronising call reports as
LB_ETIMEOUT.  lb_selftest runs that wait against a completion target that nothing reaches, so
the limit is exercised on the device; the context must report it, clear it and keep working.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

LB_ETIMEOUT = 5


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_08923_gb300.build as b
    b.build()
    import paper_1804_08923_gb300 as lbm
    return lbm


def jet(lb, step_kernel=1):
    cfg = workloads.scaled_jet("jet96", 36, 34, 40, D=10)
    lat = lb.Lattice((36, 34, 40), dict(cfg["params"], step_kernel=step_kernel), bc=cfg["bc"])
    lat.init_jet()
    return lat


def test_a_fused_wait_that_runs_out_is_reported_and_the_context_survives(lb):
    lat, ref = jet(lb), jet(lb)
    lat.step(5)
    ref.step(5)
    status, ms = lat.selftest_fused_wait()
    assert status == LB_ETIMEOUT
    assert 900.0 <= ms <= 5000.0, ms  # the 1 s limit of the global timer, not the poll cap
    # the flag was read and cleared: the context steps and reduces as before, bit for bit
    lat.step(5)
    ref.step(5)
    m = lat.mass()
    assert np.all(np.isfinite(m))
    assert np.array_equal(lat.populations(device=False), ref.populations(device=False))
    lat.close()
    ref.close()


def test_selftest_arguments(lb):
    import ctypes as C
    lat = jet(lb, step_kernel=0)
    L = lb.library()
    res, ms = C.c_int32(), C.c_double()
    assert L.lb_selftest(lat._ctx, 99, C.byref(res), C.byref(ms)) == 1  # LB_EINVAL
    assert L.lb_selftest(lat._ctx, 1, None, C.byref(ms)) == 1
    lat.step_gather()
    assert L.lb_selftest(lat._ctx, 1, C.byref(res), C.byref(ms)) == 6  # LB_ESTATE inside a split step
    lat.step_collide()
    lat.close()
