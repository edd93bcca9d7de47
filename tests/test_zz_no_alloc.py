"""lb_mass_noalloc: colour masses with no device allocation, checked against lb_mass.

The entry point serves callers that cannot call cudaMalloc (code that keeps its own
population arrays under a device-memory budget fixed at start-up, with no lb_ctx): its
scratch is a static device array inside the library.  Its result must equal lb_mass's on
the same state within the reduction tolerance of the other mass tests (two FP64 sums of
the same values in different orders), on two calls in a row, after the rest of the suite
and, in a child process, as the library's very first call on its device.  The file name
sorts last so that a run stopping at the first failure has already run every other test.
"""
import ctypes as C
import os
import subprocess
import sys

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_08923_gb300.build as b
    b.build()
    import paper_1804_08923_gb300 as lbm
    return lbm


def noalloc_mass(lb, pops, stream):
    import torch
    out = torch.full((2,), float("nan"), dtype=torch.float64, device=pops.device)
    nodes = pops.numel() // 54
    rc = lb.library().lb_mass_noalloc(C.c_void_p(pops.data_ptr()), C.c_int64(nodes), C.c_void_p(out.data_ptr()),
                                      C.c_void_p(stream.cuda_stream))
    assert rc == 0, lb.library().lb_last_error()
    stream.synchronize()
    return out.cpu().numpy()


def test_noalloc_mass_matches_lb_mass_twice(lb):
    shape = (40, 33, 70)  # 92 400 nodes: two first-stage blocks per colour, ragged tail
    params = dict(rho_r0=1.0, rho_b0=0.5, nu_r=0.02, nu_b=0.05, sigma=0.003)
    lat = lb.Lattice((70, 33, 40), params)
    lat.init_fields(*workloads.random_two_phase_fields(shape, 21, 1.0, 0.5))
    for call in range(2):
        pops = lat.populations(device=True)
        got = noalloc_mass(lb, pops, lat.stream)
        ref = lat.mass()
        assert np.all(np.isfinite(got))
        assert np.allclose(got, ref, rtol=1e-12, atol=0), (call, got, ref)
        lat.step(3)  # a different state for the second call


def test_noalloc_mass_small_then_large(lb):
    """A small input after a larger one: stale partials of the earlier call are never read."""
    import torch
    big = lb.Lattice((64, 64, 40), dict(rho_r0=1.0, rho_b0=1.0))
    big.init_uniform(0.25, 0.75)
    small = lb.Lattice((5, 4, 3), dict(rho_r0=1.0, rho_b0=1.0))
    small.init_uniform(0.5, 0.5)
    for lat in (big, small):
        got = noalloc_mass(lb, lat.populations(device=True), lat.stream)
        assert np.allclose(got, lat.mass(), rtol=1e-12, atol=0)
    assert np.allclose(noalloc_mass(lb, small.populations(device=True), small.stream), [30.0, 30.0], rtol=1e-6)
    del torch


def test_noalloc_rejects_oversized_input(lb):
    L = lb.library()
    too_many = (1 << 28) + 1  # LB_MASS_NOALLOC_MAX_NODES + 1
    rc = L.lb_mass_noalloc(C.c_void_p(16), C.c_int64(too_many), C.c_void_p(16), None)
    assert rc == 1
    assert b"static scratch" in L.lb_last_error()
    assert L.lb_mass_noalloc(C.c_void_p(16), C.c_int64(0), C.c_void_p(16), None) == 1


FIRST_CALL = r"""
import ctypes as C, sys
import numpy as np, torch
sys.path.insert(0, ROOT)
import paper_1804_08923_gb300 as lb
import workloads
L = lb.library()
s = torch.cuda.current_stream()
g = torch.Generator(device="cuda").manual_seed(5)
pops = torch.rand((2, 27, 50000), generator=g, device="cuda", dtype=torch.float32)
out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
# the library's first call in this process: the scratch address is looked up here
rc = L.lb_mass_noalloc(C.c_void_p(pops.data_ptr()), C.c_int64(50000), C.c_void_p(out.data_ptr()),
                       C.c_void_p(s.cuda_stream))
assert rc == 0, L.lb_last_error()
ref = pops.double().sum(dim=(1, 2))
assert torch.allclose(out, ref, rtol=1e-12, atol=0), (out, ref)
lat = lb.Lattice((37, 20, 30), dict(rho_r0=1.0, rho_b0=0.5, nu_r=0.02, nu_b=0.05, sigma=0.003))
lat.init_fields(*workloads.random_two_phase_fields((30, 20, 37), 8, 1.0, 0.5))
p2 = lat.populations(device=True)
rc = L.lb_mass_noalloc(C.c_void_p(p2.data_ptr()), C.c_int64(p2.numel() // 54), C.c_void_p(out.data_ptr()),
                       C.c_void_p(lat.stream.cuda_stream))
assert rc == 0, L.lb_last_error()
lat.stream.synchronize()
assert np.allclose(out.cpu().numpy(), lat.mass(), rtol=1e-12, atol=0)
print("first-call ok")
"""


def test_noalloc_mass_as_the_first_call_of_a_fresh_process(lb):
    """A child process whose first library call is lb_mass_noalloc (the scratch address is
    looked up on a device that has run no library kernel yet): FP64 colour sums of random
    device populations against torch's, then against lb_mass on a lattice."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = "ROOT = " + repr(root) + "\n" + FIRST_CALL
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0 and "first-call ok" in r.stdout, r.stdout + r.stderr
