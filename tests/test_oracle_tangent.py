"""The oracle's forward-mode tangent (complex step) against what fixes it from outside:
central differences of the FP64 oracle, the FP64 objective itself, and linearity.

Central differences with relative step h have truncation error O(h^2) and roundoff
~ eps_mach |J| / h; with h = 1e-5 of the parameter that is below 1e-5 of the derivative for
these cases, which sets the bar.  The complex-step tangent has no cancellation and is exact to
rounding.
"""
import numpy as np
import pytest

import oracle
import workloads


def jet_setup():
    cfg = workloads.scaled_jet("jet64", 12, 11, 10, D=6)
    p = dict(workloads.CONFIGS["droplet32"]["params"])
    p.update(cfg["params"])
    p["noise_amp"] = 0.02
    p["fourier"] = tuple(0.05 * np.random.default_rng(4).standard_normal(16))
    g = oracle.make_grid(12, 11, 10, *cfg["bc"])
    ref = oracle.Lattice(g, oracle.make_params(p))
    ref.init_jet()
    return g, p, ref.S.copy(), ref.hist.copy()


def J_fp64(g, p, S0, H0, T, kind, args):
    r = oracle.Lattice(g, oracle.make_params(p))
    r.set_state(S0, H0)
    r.step(T)
    return r.objective(kind, args)


@pytest.mark.parametrize("kind,args", [("area", (1e-3,)), ("penetration", (2.0,))])
def test_tangent_matches_central_differences(kind, args):
    g, p, S0, H0 = jet_setup()
    T = 6
    J0 = J_fp64(g, p, S0, H0, T, kind, args)
    for name in ("u_in", "sigma", "nu_r", "nu_b", "a3", "b7"):
        if name[0] in "ab" and name[1:].isdigit():
            k = 2 * (int(name[1:]) - 1) + (name[0] == "b")
            d = [0.0] * 16
            d[k] = 1.0
            dp, h = {"fourier": d}, 1e-5

            def shifted(s, k=k):
                q = dict(p)
                f = list(q["fourier"])
                f[k] += s
                q["fourier"] = tuple(f)
                return q
        else:
            dp, h = {name: 1.0}, 1e-5 * p[name]

            def shifted(s, name=name):
                return dict(p, **{name: p[name] + s})
        J, dJ = oracle.tangent_objective(g, p, S0, H0, T, kind, args, dparams=dp)
        assert J == J0  # the complex build's real part is the FP64 oracle
        fd = (J_fp64(g, shifted(h), S0, H0, T, kind, args) - J_fp64(g, shifted(-h), S0, H0, T, kind, args)) / (2 * h)
        assert abs(dJ - fd) < 1e-5 * abs(fd) + 1e-12, (name, dJ, fd)


def test_state_tangent_and_linearity():
    """Along a state direction the tangent matches central differences; tangents are linear in
    the direction (parameters and state together).  Free-slip walls with gravity and a random
    two-phase state: no outflow clamp, whose kink at a resting outflow has one-sided
    derivatives that central differences average."""
    nx, ny, nz = 10, 9, 8
    p = dict(workloads.CONFIGS["droplet32"]["params"])
    p.update(rho_r0=1.0, rho_b0=0.5, nu_r=0.02, nu_b=0.05, sigma=0.004, g=(0.0, 0.0, 3e-5), u_in=0.0)
    g = oracle.make_grid(nx, ny, nz, oracle.BC_FREESLIP, oracle.BC_FREESLIP)
    ref = oracle.Lattice(g, oracle.make_params(p))
    ref.init_fields(*workloads.random_two_phase_fields((nz, ny, nx), 9, 1.0, 0.5, u_amp=0.03))
    S0, H0 = ref.S.copy(), ref.hist.copy()
    T = 5
    rng = np.random.default_rng(8)
    dS = rng.standard_normal(S0.shape) * 1e-3
    _, d1 = oracle.tangent_objective(g, p, S0, H0, T, "area", (1e-3,), dS=dS)
    h = 1e-4

    def J_at(s):
        r = oracle.Lattice(g, oracle.make_params(p))
        r.set_state(S0 + s * dS, H0)
        r.step(T)
        return r.objective("area", (1e-3,))
    fd = (J_at(h) - J_at(-h)) / (2 * h)
    assert abs(d1 - fd) < 1e-6 * abs(fd)
    _, d2 = oracle.tangent_objective(g, p, S0, H0, T, "area", (1e-3,), dparams={"sigma": 1.0})
    _, d12 = oracle.tangent_objective(g, p, S0, H0, T, "area", (1e-3,), dparams={"sigma": 2.0}, dS=-3.0 * dS)
    assert abs(d12 - (2 * d2 - 3 * d1)) < 1e-9 * (abs(2 * d2) + abs(3 * d1))
