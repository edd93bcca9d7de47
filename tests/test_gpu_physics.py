"""Physics of the CUDA path against numbers the paper prints (no oracle involved).

Table 1 (Section III): a static red droplet, R = 25, W = 4, in a 100^3 periodic box, A = 0.01,
nu = 1/6 (tau = 1), 1e5 iterations.  The paper reports the pressure jump 2 sigma / R =
3.5556e-4 reproduced within 0.40% and a maximum spurious velocity of 1.22e-4 at gamma = 1.
"""
import os

import numpy as np
import pytest

from conftest import GOLDEN


def table1():
    rows = {}
    for line in open(os.path.join(GOLDEN, "table1_laplace.txt")):
        if line.startswith("#") or not line.strip():
            continue
        g, dth, dnum, e, umax = (float(v) for v in line.split())
        rows[g] = dict(dp_theory=dth, dp_numerical=dnum, E=e, umax=umax)
    return rows


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_08923_gb300.build as b
    b.build()
    import paper_1804_08923_gb300 as lbm
    return lbm


def test_golden_table1_is_eq_sigma():
    """The printed theoretical column equals 2 sigma / R with sigma = (4/9) A tau (Eq. (32))."""
    for row in table1().values():
        assert abs(2 * (4 / 9) * 0.01 * 1.0 / 25 - row["dp_theory"]) < 5e-9


@pytest.mark.gpu
def test_table1_static_droplet_gamma1(lb):
    """gamma = 1: the pressure jump after 1e5 steps is within 1% of 2 sigma / R (the paper
    reaches 0.40%) and the maximum spurious velocity is of the paper's size (1.22e-4)."""
    ref = table1()[1.0]
    n, R, A = 100, 25.0, 0.01
    sigma = 4.0 / 9.0 * A * 1.0
    lat = lb.Lattice((n, n, n), dict(rho_r0=1.0, rho_b0=1.0, nu_r=1 / 6, nu_b=1 / 6, sigma=sigma, check_every=10000))
    lat.init_droplet(R, 4.0)
    m0 = lat.mass()
    lat.step(100000)
    F = lat.fields(device=False)
    c = (n - 1) / 2
    z, y, x = np.meshgrid(*[np.arange(n)] * 3, indexing="ij")
    r = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    dp = F["p"][r < R - 4].mean() - F["p"][r > R + 4].mean()
    assert abs(dp / ref["dp_theory"] - 1) < 0.01, dp
    umax = float(np.sqrt(F["ux"].astype(np.float64) ** 2 + F["uy"] ** 2 + F["uz"] ** 2).max())
    assert 0.5 * ref["umax"] < umax < 2.0 * ref["umax"], umax
    m1 = lat.mass()
    assert np.abs(m1.sum() / m0.sum() - 1) < 1e-5   # total mass (FP32 populations, FP64 sums)
    assert np.all(np.abs(m1 / m0 - 1) < 1e-3)       # per-colour drift over 1e5 FP32 steps


@pytest.mark.gpu
def test_table1_static_droplet_gamma10(lb):
    """gamma = 10 (rho_r0 = gamma, rho_b0 = 1, equal bulk pressures): after 1e5 steps the
    pressure jump is 2 sigma / R within 1% (the paper reaches 0.36%) with R the radius of the
    final droplet's volume (phi > 0), and the droplet keeps its colour masses."""
    n, R = 100, 25.0
    sigma = 4.0 / 9.0 * 0.01 * 1.0
    lat = lb.Lattice((n, n, n), dict(rho_r0=10.0, rho_b0=1.0, nu_r=1 / 6, nu_b=1 / 6, sigma=sigma, check_every=10000))
    lat.init_droplet(R, 4.0)
    m0 = lat.mass()
    lat.step(100000)
    F = lat.fields(device=False)
    c = (n - 1) / 2
    z, y, x = np.meshgrid(*[np.arange(n)] * 3, indexing="ij")
    r = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    Reff = (3 * float((F["phi"] > 0).sum()) / (4 * np.pi)) ** (1 / 3)
    p = F["p"].astype(np.float64)
    dp = p[r < Reff - 6].mean() - p[r > Reff + 6].mean()
    assert abs(dp * Reff / 2 / sigma - 1) < 0.01, (dp, Reff)
    assert np.abs(lat.mass() / m0 - 1).max() < 3e-3


@pytest.mark.gpu
def test_table1_static_droplet_gamma100_mass_fraction_alpha(lb):
    """gamma = 100 under reading R15 (alpha-bar by mass fraction; rho_r0 = gamma, rho_b0 = 1): the
    droplet is stable for 1e5 steps, the pressure jump is 2 sigma / R within 1% (the paper
    reaches 0.32%), and the maximum spurious velocity is the paper's 4.67e-5 within 10%."""
    ref = table1()[100.0]
    n, R = 100, 25.0
    sigma = 4.0 / 9.0 * 0.01 * 1.0
    lat = lb.Lattice((n, n, n), dict(rho_r0=100.0, rho_b0=1.0, nu_r=1 / 6, nu_b=1 / 6, sigma=sigma,
                                     check_every=10000, alpha_mix=1))
    lat.init_droplet(R, 4.0)
    lat.step(100000)
    F = lat.fields(device=False)
    c = (n - 1) / 2
    z, y, x = np.meshgrid(*[np.arange(n)] * 3, indexing="ij")
    r = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    p = F["p"].astype(np.float64)
    dp = p[r < R - 6].mean() - p[r > R + 6].mean()
    assert abs(dp / ref["dp_theory"] - 1) < 0.01, dp
    umax = float(np.sqrt(F["ux"].astype(np.float64) ** 2 + F["uy"] ** 2 + F["uz"] ** 2).max())
    assert abs(umax / ref["umax"] - 1) < 0.1, umax


@pytest.mark.gpu
def test_table1_static_droplet_gamma1000_mass_fraction_alpha(lb):
    """gamma = 1000 under reading R15 (rho_r0 = 1000, rho_b0 = 1): stable for 1e5 steps, the
    maximum spurious velocity is the paper's 6.94e-5 within 10%, each colour's mass holds to
    1e-3 as at gamma = 1 (measured: red -6e-5, blue +1.3e-4), and the pressure jump between the means over r < R - 6 and r > R + 6 is 2 sigma / R
    within 1.5% (the paper's 0.40% came from an averaging procedure it does not specify; with
    this droplet the jump varies with the averaging window by about 3% of itself, from -0.2%
    at R -+ 4 to +2.8% at R -+ 10).  Needs 1 - alpha-bar formed from the colours' 1 - alpha_k:
    alpha_r = 0.9993 leaves 1 - alpha-bar few FP32 digits when taken by subtraction."""
    ref = table1()[1000.0]
    n, R = 100, 25.0
    sigma = 4.0 / 9.0 * 0.01 * 1.0
    lat = lb.Lattice((n, n, n), dict(rho_r0=1000.0, rho_b0=1.0, nu_r=1 / 6, nu_b=1 / 6, sigma=sigma,
                                     check_every=10000, alpha_mix=1))
    lat.init_droplet(R, 4.0)
    m0 = lat.mass()
    lat.step(100000)
    F = lat.fields(device=False)
    c = (n - 1) / 2
    z, y, x = np.meshgrid(*[np.arange(n)] * 3, indexing="ij")
    r = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    p = F["p"].astype(np.float64)
    dp = p[r < R - 6].mean() - p[r > R + 6].mean()
    assert abs(dp / ref["dp_theory"] - 1) < 0.015, dp
    umax = float(np.sqrt(F["ux"].astype(np.float64) ** 2 + F["uy"] ** 2 + F["uz"] ** 2).max())
    assert abs(umax / ref["umax"] - 1) < 0.1, umax
    assert np.abs(lat.mass() / m0 - 1).max() < 1e-3
