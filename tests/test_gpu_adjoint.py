"""The discrete adjoint of the CUDA step (lb_adjoint) against FP64 central finite differences
of the oracle and against the oracle's forward-mode (complex-step) tangent, same seeded inputs
on both sides; the oracle never sees a GPU value.

Gradient error norms: max over parameters of |g_adjoint - g_fd| / max over parameters of
|g_fd| (the gradient's own scale), bar 1e-4; and every component whose reference exceeds 1e-3
of that scale against its own value, bar 1e-4 as well (check_components).  The directional
derivative along a random state perturbation has the same bar.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-4
NAMES = ("u_in", "sigma", "nu_r", "nu_b") + tuple(f"{ab}{m}" for m in range(1, 9) for ab in "ab")


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1804_08923_gb300.build as b
    b.build()
    import paper_1804_08923_gb300 as lbm
    return lbm


def full_params(p):
    base = dict(workloads.CONFIGS["droplet32"]["params"])
    base.update(p)
    return base


def perturbed(params, name, h):
    p = dict(params)
    if name in ("u_in", "sigma", "nu_r", "nu_b"):
        p[name] = full_params(params)[name] + h
    else:
        m, ab = int(name[1:]), name[0]
        four = list(p.get("fourier", (0.0,) * 16)) + [0.0] * 16
        four = four[:16]
        four[2 * (m - 1) + (ab == "b")] += h
        p["fourier"] = tuple(four)
    return p


def fd_step(params, name):
    """Central-difference step: 1e-5 of the value for the scalars, 1e-4 for profile coefficients."""
    if name in ("u_in", "sigma", "nu_r", "nu_b"):
        return 1e-5 * abs(full_params(params)[name])
    return 1e-4


def oracle_J(grid, bc, params, init, T, objective, args):
    nx, ny, nz = grid
    ref = oracle.Lattice(oracle.make_grid(nx, ny, nz, *bc), oracle.make_params(full_params(params)))
    init(ref)
    ref.step(T)
    return ref.objective(objective, args)


def fd_gradient(grid, bc, params, init, T, objective, args, names):
    g = np.zeros(len(names))
    for k, nm in enumerate(names):
        h = fd_step(params, nm)
        jp = oracle_J(grid, bc, perturbed(params, nm, h), init, T, objective, args)
        jm = oracle_J(grid, bc, perturbed(params, nm, -h), init, T, objective, args)
        g[k] = (jp - jm) / (2 * h)
    return g


def tangent_gradient(grid, bc, params, init, T, objective, args, names):
    """The oracle's complex-step tangent along each parameter direction."""
    nx, ny, nz = grid
    g = oracle.make_grid(nx, ny, nz, *bc)
    ref = oracle.Lattice(g, oracle.make_params(full_params(params)))
    init(ref)
    out = np.zeros(len(names))
    for k, nm in enumerate(names):
        if nm in ("u_in", "sigma", "nu_r", "nu_b"):
            dp = {nm: 1.0}
        else:
            d = [0.0] * 16
            d[2 * (int(nm[1:]) - 1) + (nm[0] == "b")] = 1.0
            dp = {"fourier": d}
        out[k] = oracle.tangent_objective(g, full_params(params), ref.S, ref.hist, T, objective, args, dparams=dp)[1]
    return out


TOL_COMP = 1e-4


def check_components(g, ref, names):
    """Each component whose reference exceeds 1e-3 of the largest, relative to its own value."""
    big = np.abs(ref) > 1e-3 * np.abs(ref).max()
    rel = np.abs(g - ref)[big] / np.abs(ref)[big]
    worst = [(n, float(a), float(b)) for n, a, b, k in zip(names, g, ref, big) if k]
    assert rel.size and rel.max() < TOL_COMP, (float(rel.max()), worst)
    return float(rel.max())


def jet_case():
    cfg = workloads.scaled_jet("jet64", 16, 14, 18, D=8)
    params = dict(cfg["params"])
    params["noise_amp"] = 0.02
    params["fourier"] = tuple(0.05 * np.random.default_rng(4).standard_normal(16))
    return (16, 14, 18), cfg["bc"], params


@pytest.mark.parametrize("objective,args", [("area", (1e-3,)), ("penetration", (2.0,))])
def test_adjoint_jet_parameters_match_finite_differences(lb, objective, args):
    """Inlet disc with noise and a profile, free slip around it, convective outflow: the
    20 parameter gradients after 12 steps against central differences of the oracle."""
    grid, bc, params = jet_case()
    T = 12
    lat = lb.Lattice(grid, params, bc=bc)
    lat.init_jet()
    J, g = lat.adjoint(T, objective, args)
    J_ref = oracle_J(grid, bc, params, lambda r: r.init_jet(), T, objective, args)
    assert abs(J / J_ref - 1) < 1e-5, (J, J_ref)
    g_fd = fd_gradient(grid, bc, params, lambda r: r.init_jet(), T, objective, args, NAMES)
    err = np.abs(g - g_fd).max() / np.abs(g_fd).max()
    assert err < TOL, (err, list(zip(NAMES, g, g_fd)))
    assert np.abs(g_fd[4:]).max() > 1e-3 * np.abs(g_fd).max()  # the profile really matters
    g_tan = tangent_gradient(grid, bc, params, lambda r: r.init_jet(), T, objective, args, NAMES)
    err_t = np.abs(g - g_tan).max() / np.abs(g_tan).max()
    assert err_t < TOL, (err_t, list(zip(NAMES, g, g_tan)))
    check_components(g, g_tan, NAMES)
    check_components(g, g_fd, NAMES)


@pytest.mark.parametrize("bc,g", [((0, 0), (1e-5, 0.0, 2e-5)), ((1, 1), (0.0, 0.0, 3e-5))])
def test_adjoint_state_directional_derivative(lb, bc, g):
    """dJ/dS(0) along a random direction against the oracle's central difference of J(S(0) +
    h dS), on a random two-phase state (periodic, and free-slip walls with gravity), 8 steps."""
    nx, ny, nz = 12, 10, 14
    shape = (nz, ny, nx)
    params = dict(rho_r0=1.0, rho_b0=0.5, nu_r=0.02, nu_b=0.05, sigma=0.004, g=g)
    fields = workloads.random_two_phase_fields(shape, 9, 1.0, 0.5, u_amp=0.03)
    lat = lb.Lattice((nx, ny, nz), params, bc=bc)
    lat.init_fields(*fields)
    T = 8
    J, grad = lat.adjoint(T, "area", (1e-3,), checkpoint=3)
    lS = lat.adjoint_state().astype(np.float64)
    dS = np.random.default_rng(2).standard_normal((2, 27) + shape) * 1e-3
    ref = oracle.Lattice(oracle.make_grid(nx, ny, nz, *bc), oracle.make_params(full_params(params)))
    ref.init_fields(*fields)
    S0, H0 = ref.S.copy(), ref.hist.copy()
    h = 1e-3
    Js = []
    for sgn in (1, -1):
        ref.set_state(S0 + sgn * h * dS, H0)
        ref.step(T)
        Js.append(ref.objective("area", (1e-3,)))
    fd = (Js[0] - Js[1]) / (2 * h)
    ad = float((lS * dS).sum())
    assert abs(ad - fd) < TOL * abs(fd), (ad, fd)
    _, tan = oracle.tangent_objective(oracle.make_grid(nx, ny, nz, *bc), full_params(params), S0, H0, T, "area",
                                      (1e-3,), dS=dS)
    assert abs(ad - tan) < TOL * abs(tan), (ad, tan)
    # sigma and the viscosities against central differences too
    init = lambda r: r.init_fields(*fields)
    g_fd = fd_gradient((nx, ny, nz), bc, params, init, T, "area", (1e-3,), ("sigma", "nu_r", "nu_b"))
    err = np.abs(grad[1:4] - g_fd).max() / np.abs(g_fd).max()
    assert err < TOL, (err, grad[1:4], g_fd)


def test_adjoint_is_independent_of_the_checkpoint_interval(lb):
    """Recomputed segments are bitwise the forward steps, so the gradient does not depend on
    the checkpoint interval; the context ends at S(T), bitwise the state lb_step(T) reaches."""
    grid, bc, params = jet_case()
    T = 9
    res = []
    for k in (0, 1, 4, 9):
        lat = lb.Lattice(grid, params, bc=bc)
        lat.init_jet()
        res.append(lat.adjoint(T, "area", (1e-3,), checkpoint=k))
        if k == 0:
            S_adj = lat.populations(device=False)
            ref = lb.Lattice(grid, params, bc=bc)
            ref.init_jet()
            ref.step(T)
            assert np.array_equal(S_adj, ref.populations(device=False))
            assert lat.step_count == T
    for J, g in res[1:]:
        assert J == res[0][0]
        assert np.array_equal(g, res[0][1])


def test_adjoint_rejects_what_it_does_not_cover(lb):
    grid, bc, params = jet_case()
    lat = lb.Lattice(grid, dict(params, s3=0.9), bc=bc)
    lat.init_jet()
    with pytest.raises(lb.LBError):
        lat.adjoint(3)
    lat16 = lb.Lattice(grid, dict(params, storage=1), bc=bc)
    lat16.init_jet()
    with pytest.raises(lb.LBError):
        lat16.adjoint(3)
    lat = lb.Lattice(grid, params, bc=bc)
    lat.init_jet()
    with pytest.raises(lb.LBError):
        lat.adjoint_state()
    with pytest.raises(lb.LBError):
        lat.adjoint(3, "area", (0.0,))


def test_autograd_function_gives_the_adjoint_gradient(lb):
    """torch.autograd through LatticeObjective: backward returns lb_adjoint's gradient, the
    lattice is restored to the saved state on every call, and a step against the gradient
    lowers the objective as the first-order prediction says."""
    import torch
    from paper_1804_08923_gb300 import autograd as ag
    grid, bc, params = jet_case()
    lat = lb.Lattice(grid, params, bc=bc)
    lat.init_jet()
    state = lat.save()
    theta = ag.theta_of(params).requires_grad_(True)
    J = ag.objective(lat, theta, 6, state, "area", (1e-3,))
    J.backward()
    ref = lb.Lattice(grid, params, bc=bc)
    ref.init_jet()
    J_ref, g_ref = ref.adjoint(6, "area", (1e-3,))
    assert float(J) == J_ref
    assert np.array_equal(theta.grad.numpy(), g_ref)
    g = theta.grad.detach().clone()
    step = -1e-3 * g / g.norm() * theta.detach().norm()
    J2 = ag.objective(lat, theta.detach() + step, 6, state, "area", (1e-3,))
    predicted = float(J) + float(g @ step)
    assert abs(float(J2) - predicted) < 0.05 * abs(float(g @ step))
    assert float(J2) < float(J)


def test_adjoint_full_size_jet_short_horizon(lb):
    """On the full 64x64x256 jet of the adjoint benchmark (D = 12, Re = 500, We = 50) in the
    benchmark's launch configuration: J and the gradients w.r.t. u_in and a_2 after 10 steps
    (checkpoints every 4: segments of 4, 4 and 2) against the oracle's tangent; the oracle at
    this size costs seconds per step, hence the short horizon."""
    cfg = workloads.CONFIGS["jet64"]
    grid, bc, params = cfg["grid"], cfg["bc"], dict(cfg["params"])
    T = 10
    lat = lb.Lattice(grid, params, bc=bc)
    lat.init_jet()
    J, g = lat.adjoint(T, "penetration", (4.0,), checkpoint=4)
    names = ("u_in", "a2")
    g_tan = tangent_gradient(grid, bc, params, lambda r: r.init_jet(), T, "penetration", (4.0,), names)
    J_ref = oracle_J(grid, bc, params, lambda r: r.init_jet(), T, "penetration", (4.0,))
    assert abs(J / J_ref - 1) < 1e-5, (J, J_ref)
    got = np.array([g[NAMES.index(n)] for n in names])
    err = np.abs(got - g_tan).max() / np.abs(g_tan).max()
    assert err < TOL, (err, got, g_tan)
    check_components(got, g_tan, names)


def test_adjoint_with_side_walls(lb):
    """The paper's boundaries (side walls free-slip): gradients against the oracle's tangent and
    central differences."""
    grid, bc, params = jet_case()
    bc = tuple(bc) + (1, 1)
    T = 10
    lat = lb.Lattice(grid, params, bc=bc)
    lat.init_jet()
    J, g = lat.adjoint(T, "area", (1e-3,))
    init = lambda r: r.init_jet()
    names = ("u_in", "sigma", "nu_r", "nu_b", "a1", "b2", "a5")
    idx = [NAMES.index(n) for n in names]
    g_tan = tangent_gradient(grid, bc, params, init, T, "area", (1e-3,), names)
    err = np.abs(g[idx] - g_tan).max() / np.abs(g_tan).max()
    assert err < TOL, (err, g[idx], g_tan)
    check_components(g[idx], g_tan, names)
    g_fd = fd_gradient(grid, bc, params, init, T, "area", (1e-3,), names)
    assert np.abs(g[idx] - g_fd).max() / np.abs(g_fd).max() < TOL


def test_adjoint_state_with_side_walls(lb):
    """dJ/dS(0) along a random direction, closed box (all walls free-slip), gravity."""
    nx, ny, nz = 11, 10, 9
    shape = (nz, ny, nx)
    bc = (1, 1, 1, 1)
    params = dict(rho_r0=1.0, rho_b0=0.5, nu_r=0.02, nu_b=0.05, sigma=0.004, g=(1e-5, -2e-5, 3e-5))
    fields = workloads.random_two_phase_fields(shape, 21, 1.0, 0.5, u_amp=0.03)
    lat = lb.Lattice((nx, ny, nz), params, bc=bc)
    lat.init_fields(*fields)
    T = 6
    lat.adjoint(T, "area", (1e-3,), checkpoint=2)
    lS = lat.adjoint_state().astype(np.float64)
    dS = np.random.default_rng(6).standard_normal((2, 27) + shape) * 1e-3
    ref = oracle.Lattice(oracle.make_grid(nx, ny, nz, *bc), oracle.make_params(full_params(params)))
    ref.init_fields(*fields)
    _, tan = oracle.tangent_objective(oracle.make_grid(nx, ny, nz, *bc), full_params(params), ref.S, ref.hist, T,
                                      "area", (1e-3,), dS=dS)
    ad = float((lS * dS).sum())
    assert abs(ad - tan) < TOL * abs(tan), (ad, tan)


def test_adjoint_with_mass_fraction_alpha(lb):
    """Reading R15 changes d alpha-bar / d rho_k: gradients at density ratio 8 against the oracle's
    tangent."""
    grid, bc, params = jet_case()
    params = dict(params, rho_b0=1 / 8.0, alpha_mix=1)
    T = 8
    lat = lb.Lattice(grid, params, bc=bc)
    lat.init_jet()
    J, g = lat.adjoint(T, "area", (1e-3,))
    names = ("u_in", "sigma", "nu_r", "nu_b", "a2")
    g_tan = tangent_gradient(grid, bc, params, lambda r: r.init_jet(), T, "area", (1e-3,), names)
    got = np.array([g[NAMES.index(n)] for n in names])
    assert np.abs(got - g_tan).max() / np.abs(g_tan).max() < TOL, (got, g_tan)
    check_components(got, g_tan, names)


def test_adjoint_long_horizon_against_the_tangent(lb):
    """100 steps of a 24x24x48 jet (D = 8, inlet noise and profile, convective outflow), the
    default checkpoint interval (10 segments of 10, the last recorded by the forward pass, the
    others recomputed on the second stream): J and six gradients against the oracle's
    complex-step tangent, each component against its own value."""
    cfg = workloads.scaled_jet("jet64", 24, 24, 48, D=8)
    params = dict(cfg["params"])
    params["noise_amp"] = 0.02
    params["fourier"] = tuple(0.05 * np.random.default_rng(5).standard_normal(16))
    grid, bc, T = (24, 24, 48), cfg["bc"], 100
    lat = lb.Lattice(grid, params, bc=bc)
    lat.init_jet()
    J, g = lat.adjoint(T, "area", (1e-3,))
    names = ("u_in", "sigma", "nu_r", "nu_b", "a1", "b2")
    g_tan = tangent_gradient(grid, bc, params, lambda r: r.init_jet(), T, "area", (1e-3,), names)
    J_ref = oracle_J(grid, bc, params, lambda r: r.init_jet(), T, "area", (1e-3,))
    assert abs(J / J_ref - 1) < 1e-5, (J, J_ref)
    got = np.array([g[NAMES.index(n)] for n in names])
    assert np.abs(got - g_tan).max() / np.abs(g_tan).max() < TOL, (got, g_tan)
    check_components(got, g_tan, names)
