"""The C-ABI library loads and exports every entry point declared in include/lbcm.h, and
its host-side checks (no GPU work) behave as documented."""
import ctypes as C
import os
import re
import subprocess

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "lbcm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import paper_1804_08923_gb300.build as b
    b.build()
    from paper_1804_08923_gb300 import _abi
    return _abi.library()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 16
    nm = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_1804_08923_gb300", "liblbcm.so")],
                        capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\b(lb_[a-z_0-9]+)\b", nm))
    assert set(names) <= exported, set(names) - exported
    from paper_1804_08923_gb300 import _abi
    assert set(names) == set(_abi.EXPORTS)
    for n in names:
        getattr(lib, n)


def test_only_abi_symbols_are_exported():
    nm = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_1804_08923_gb300", "liblbcm.so")],
                        capture_output=True, text=True, check=True).stdout
    ours = [l.split()[-1] for l in nm.splitlines() if l.split() and l.split()[1] == "T"]
    assert all(s.startswith("lb_") for s in ours), [s for s in ours if not s.startswith("lb_")]


def test_buffer_sizes_and_validation(lib):
    from paper_1804_08923_gb300 import _abi
    g = _abi.make_grid(96, 96, 384, _abi.BC_INLET, _abi.BC_CONVECTIVE)
    p = _abi.make_params(dict(rho_r0=1.0, rho_b0=2 / 3, nu_r=4e-4, nu_b=4e-4, sigma=4e-4, u_in=0.05, d_in=16))
    sizes = (C.c_size_t * _abi.MAX_BUFFERS)()
    n = C.c_int32()
    assert lib.lb_buffer_sizes(C.byref(g), C.byref(p), sizes, C.byref(n)) == 0
    nodes = 96 * 96 * 384
    assert n.value == 6 and sizes[0] >= 54 * 4 * nodes and sizes[1] == sizes[0] and sizes[2] >= 8 * nodes
    assert sizes[5] >= 48 * nodes  # the collision moments written and read within a step
    assert all(int(sizes[j]) % 256 == 0 for j in range(n.value))
    # FP16 storage: 112 B per node per population buffer; the phase buffer holds two float4
    # entries per node (the fitted encoding packs its FP8 fit into them)
    by = {}
    for st in (_abi.STORE_FP16, _abi.STORE_FP16_FIT):
        ps = _abi.make_params(dict(rho_r0=1.0, rho_b0=2 / 3, nu_r=4e-4, nu_b=4e-4, sigma=4e-4, storage=st))
        assert lib.lb_buffer_sizes(C.byref(g), C.byref(ps), sizes, C.byref(n)) == 0
        by[st] = [int(sizes[j]) for j in range(n.value)]
        assert 112 * nodes <= by[st][0] < 112 * nodes + 256
    assert by[_abi.STORE_FP16][2] >= 32 * nodes and by[_abi.STORE_FP16_FIT][2] == by[_abi.STORE_FP16][2]
    bad = [
        (_abi.make_grid(0, 4, 4), p),
        (_abi.make_grid(4, 4, 4, _abi.BC_INLET, _abi.BC_PERIODIC), p),
        (_abi.make_grid(4, 4, 2, _abi.BC_INLET, _abi.BC_CONVECTIVE), p),
        (_abi.make_grid(2048, 2048, 1024), p),
        (g, _abi.make_params(dict(rho_r0=0.5, rho_b0=1.0))),          # gamma < 19/27
        (g, _abi.make_params(dict(nu_r=-1.0))),
        (g, _abi.make_params(dict(s3=2.5))),
        (g, _abi.make_params(dict(storage=9))),
        (g, _abi.make_params(dict(storage=-1))),
    ]
    for gg, pp in bad:
        assert lib.lb_buffer_sizes(C.byref(gg), C.byref(pp), sizes, C.byref(n)) == 1
        assert lib.lb_last_error().decode()


def test_null_handling_without_gpu(lib):
    assert lib.lb_step(None, 1) == 1
    assert lib.lb_mass(None, None) == 1
    assert lib.lb_adjoint(None, 0, 0, None, None, 0) == 1          # LB_EINVAL
    assert lib.lb_adjoint_state(None, None, 0) == 1
    assert lib.lb_set_params(None, None) == 1
    assert lib.lb_step_count(None) == -1
    lib.lb_destroy(None)


def test_defaults_are_the_papers(lib):
    from paper_1804_08923_gb300 import _abi
    p = _abi.Params()
    lib.lb_params_default(C.byref(p))
    assert (p.s0, p.s1) == (0.0, 0.0)
    assert (p.s2b, p.s3, p.s4, p.s5, p.s6) == (1.0,) * 5
    assert p.beta == 0.7 and abs(p.nu_r - 1 / 6) < 1e-16 and p.eps_grad == 1e-6


def test_product_does_not_import_oracle():
    """The CUDA path's package never refers to the oracle."""
    pkg = os.path.join(ROOT, "paper_1804_08923_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in src.lower(), f


def test_selftest_rejects_a_missing_context(lib):
    import ctypes as C
    res, ms = C.c_int32(), C.c_double()
    assert lib.lb_selftest(None, 1, C.byref(res), C.byref(ms)) == 1  # LB_EINVAL, no GPU work
