"""Parity of the CUDA step (through the C ABI) with the FP64 oracle.

Error norm: max over colours, directions and nodes of |f_gpu - f_oracle| / (w_i max(rho_r0,
rho_b0)); the FP32 bar is 1e-5 after 50 steps on smooth cases.  Sizes span several
32x4 thread blocks with ragged tails in x and y.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

TOL = 1e-5


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


def pair(lb, shape, params, bc=(0, 0)):
    nz, ny, nx = shape
    gpu = lb.Lattice((nx, ny, nz), params, bc=bc)
    ref = oracle.Lattice(oracle.make_grid(nx, ny, nz, *bc), oracle.make_params(full_params(params)))
    return gpu, ref


def norm_err(gpu, ref, params):
    got = gpu.populations(device=False).astype(np.float64)
    w = oracle.weights()[None, :, None, None, None]
    scale = w * max(params["rho_r0"], params["rho_b0"])
    return np.abs(got - ref.S) / scale


def run_both(gpu, ref, steps):
    gpu.step(steps)
    ref.step(steps)


def test_droplet_periodic_parity(lb):
    """Static droplet (Section III physics, tau = 1) on 20^3, 50 steps."""
    shape = (20, 20, 20)
    params = dict(rho_r0=1.0, rho_b0=1.0, nu_r=1 / 6, nu_b=1 / 6, sigma=0.01)
    gpu, ref = pair(lb, shape, params)
    gpu.init_droplet(6.0, 4.0)
    ref.init_droplet(6.0, 4.0)
    run_both(gpu, ref, 50)
    e = norm_err(gpu, ref, params)
    assert e.max() < TOL, e.max()


@pytest.mark.parametrize("seed,gamma,g", [(1, 2.0, (0.0, 0.0, 1e-5)), (2, 8.0, (1e-6, -2e-6, 3e-6))])
def test_random_two_phase_parity(lb, seed, gamma, g):
    """Random smooth two-phase state with density and viscosity contrast and gravity,
    ragged 40x9x12 lattice, 50 steps."""
    shape = (12, 9, 40)
    params = dict(rho_r0=1.0, rho_b0=1.0 / gamma, nu_r=0.02, nu_b=0.08, sigma=0.003, g=g)
    gpu, ref = pair(lb, shape, params)
    fields = workloads.random_two_phase_fields(shape, seed, 1.0, 1.0 / gamma, u_amp=0.03)
    gpu.init_fields(*fields)
    ref.init_fields(*fields)
    run_both(gpu, ref, 50)
    e = norm_err(gpu, ref, params)
    assert e.max() < TOL, e.max()


@pytest.mark.parametrize("storage,bc", [(0, (0, 0)), (0, (1, 1, 1, 1)), (1, (0, 0)), (2, (0, 0)), (2, (1, 1, 1, 1))])
def test_general_relaxation_rates_parity(lb, storage, bc):
    """Every relaxation group with its own rate (s0, s1 and s2b..s6 away from the paper's
    values) exercises each branch of the moment-space relaxation; periodic and closed
    free-slip boxes, every storage."""
    shape = (8, 6, 10)
    params = dict(rho_r0=1.0, rho_b0=0.5, nu_r=0.03, nu_b=0.06, sigma=0.002, s0=0.3, s1=0.6,
                  s2b=1.3, s3=0.9, s4=1.1, s5=1.4, s6=0.8, g=(0.0, 2e-5, 0.0), storage=storage)
    gpu, ref = pair(lb, shape, params, bc=bc)
    fields = workloads.random_two_phase_fields(shape, 5, 1.0, 0.5, u_amp=0.04)
    gpu.init_fields(*fields)
    ref.init_fields(*fields)
    run_both(gpu, ref, 20)
    e = norm_err(gpu, ref, params)
    assert e.max() < (TOL if storage == 0 else TOL16), e.max()


def test_small_jet_parity(lb):
    """Jet with inlet disc, radial noise, free slip around the disc and convective
    outflow (Section IV.A) on 36x34x40 with the 96x96x384 jet's lattice parameters
    (tau -> 0.5012), 50 steps."""
    cfg = workloads.scaled_jet("jet96", 36, 34, 40, D=10)
    params = cfg["params"]
    shape = (40, 34, 36)
    gpu, ref = pair(lb, shape, params, bc=cfg["bc"])
    gpu.init_jet()
    ref.init_jet()
    run_both(gpu, ref, 50)
    e = norm_err(gpu, ref, params)
    assert e.max() < TOL, e.max()
    h = gpu.history().astype(np.float64)
    assert np.abs(h - ref.hist).max() / max(params["rho_r0"], params["rho_b0"]) < TOL
    assert gpu.fields(device=False)["rho_r"].sum() > 0.5  # red has entered


def test_jet_inlet_profile_parity(lb):
    """Inlet with a nonuniform profile 1 + sum_m (a_m cos m theta + b_m sin m theta) over all
    eight modes (the parameters the adjoint differentiates), 40 steps."""
    cfg = workloads.scaled_jet("jet96", 28, 26, 30, D=12)
    params = dict(cfg["params"])
    rng = np.random.default_rng(11)
    params["fourier"] = tuple(0.15 * rng.standard_normal(16) / np.repeat(np.arange(1, 9), 2))
    shape = (30, 26, 28)
    gpu, ref = pair(lb, shape, params, bc=cfg["bc"])
    gpu.init_jet()
    ref.init_jet()
    run_both(gpu, ref, 40)
    e = norm_err(gpu, ref, params)
    assert e.max() < TOL, e.max()


def test_jet_with_gravity_parity(lb):
    """High-Re jet parameters (tau -> 0.5000384) with gravity along +z, 40 steps."""
    cfg = workloads.scaled_jet("jet256", 24, 24, 32, D=8)
    params = dict(cfg["params"])
    params["g"] = (0.0, 0.0, 1e-4)  # stronger than the jet's so the force terms matter
    shape = (32, 24, 24)
    gpu, ref = pair(lb, shape, params, bc=cfg["bc"])
    gpu.init_jet()
    ref.init_jet()
    run_both(gpu, ref, 40)
    e = norm_err(gpu, ref, params)
    assert e.max() < TOL, e.max()


def test_free_slip_box_parity(lb):
    """Free-slip walls at both z ends around a random two-phase state, 30 steps."""
    shape = (10, 8, 12)
    params = dict(rho_r0=1.0, rho_b0=0.5, nu_r=0.05, nu_b=0.05, sigma=0.004)
    gpu, ref = pair(lb, shape, params, bc=(lb.BC_FREESLIP, lb.BC_FREESLIP))
    fields = workloads.random_two_phase_fields(shape, 9, 1.0, 0.5)
    gpu.init_fields(*fields)
    ref.init_fields(*fields)
    run_both(gpu, ref, 30)
    e = norm_err(gpu, ref, params)
    assert e.max() < TOL, e.max()


def test_degenerate_lattices_parity(lb):
    """Degenerate extents: a 1x32x1 shear wave (every neighbour wraps onto itself in x and
    z), a single node, and the smallest convective column (nz = 3)."""
    params = dict(rho_r0=1.0, rho_b0=1.0, nu_r=0.05, nu_b=0.05, sigma=0.0)
    gpu, ref = pair(lb, (1, 32, 1), params)
    f = workloads.shear_wave_fields((1, 32, 1), 1e-3)
    gpu.init_fields(*[a.astype(np.float32) for a in f])
    ref.init_fields(*[a.astype(np.float32) for a in f])
    run_both(gpu, ref, 50)
    assert norm_err(gpu, ref, params).max() < TOL
    gpu, ref = pair(lb, (1, 1, 1), params)
    gpu.init_uniform(0.7, 0.3, (0.01, 0.02, -0.01))
    ref.init_fields(np.full((1, 1, 1), 0.7, np.float32), np.full((1, 1, 1), 0.3, np.float32),
                    np.array([0.01, 0.02, -0.01], np.float32).reshape(3, 1, 1, 1))
    run_both(gpu, ref, 10)
    assert norm_err(gpu, ref, params).max() < TOL
    p2 = dict(params, u_in=0.05, d_in=3.0, rho_b0=0.5)
    gpu, ref = pair(lb, (3, 5, 5), p2, bc=(lb.BC_INLET, lb.BC_CONVECTIVE))
    gpu.init_jet()
    ref.init_jet()
    run_both(gpu, ref, 20)
    assert norm_err(gpu, ref, p2).max() < TOL


def test_full_size_jet_sampled_one_step(lb):
    """At the benchmark's 96x96x384 jet (same launch configuration), one GPU step from the
    GPU's own state matches the oracle's step from that state at sampled nodes: inlet and
    outflow planes, lattice edges, interface and bulk."""
    cfg = workloads.CONFIGS["jet96"]
    nx, ny, nz = cfg["grid"]
    params = cfg["params"]
    gpu = lb.Lattice((nx, ny, nz), params, bc=cfg["bc"])
    gpu.init_jet()
    gpu.step(60)
    S = gpu.populations(device=False).astype(np.float64)
    H = gpu.history().astype(np.float64)
    n0 = gpu.step_count
    gpu.step(1)
    got = gpu.populations(device=False)
    ref = oracle.Lattice(oracle.make_grid(nx, ny, nz, *cfg["bc"]), oracle.make_params(full_params(params)))
    ref.set_state(S, H, n0)
    rng = np.random.default_rng(3)
    mask = np.zeros((nz, ny, nx), np.uint8)
    for z in (0, 1, 2, nz - 2, nz - 1):
        mask[z, rng.integers(0, ny, 40), rng.integers(0, nx, 40)] = 1
    mask[0, ny // 2 - 8:ny // 2 + 8, nx // 2 - 8:nx // 2 + 8] = 1  # inlet disc
    mask[:, 0, 0] = mask[:, ny - 1, nx - 1] = 1
    mask[rng.integers(0, nz, 500), rng.integers(0, ny, 500), rng.integers(0, nx, 500)] = 1
    mask[1:6, ny // 2 - 10:ny // 2 + 10, nx // 2] = 1  # jet interface region
    ref.step(1, mask=mask)
    sel = mask.astype(bool)
    w = oracle.weights()[None, :, None]
    e = np.abs(got[:, :, sel].astype(np.float64) - ref.S[:, :, sel]) / (w * max(params["rho_r0"], params["rho_b0"]))
    assert e.max() < TOL, e.max()
    assert np.isfinite(got).all()


def test_mass_conservation_and_reduction(lb):
    """lb_mass equals an FP64 sum of the populations, and a periodic run conserves the
    colour masses to FP32 round-off."""
    shape = (24, 20, 36)
    params = dict(rho_r0=1.0, rho_b0=0.5, nu_r=0.02, nu_b=0.05, sigma=0.003)
    gpu = lb.Lattice((36, 20, 24), params)
    gpu.init_fields(*workloads.random_two_phase_fields(shape, 4, 1.0, 0.5))
    m0 = gpu.mass()
    S = gpu.populations(device=False).astype(np.float64)
    assert np.allclose(m0, [S[0].sum(), S[1].sum()], rtol=1e-12, atol=0)
    gpu.step(1000)
    m1 = gpu.mass()
    assert np.all(np.abs(m1 - m0) / m0 < 2e-6), (m0, m1)
    m2 = gpu.mass()
    assert np.array_equal(m1, m2)  # deterministic reduction order


def test_save_load_roundtrip_is_bitwise(lb):
    cfg = workloads.scaled_jet("jet96", 32, 32, 24, D=8)
    gpu = lb.Lattice((32, 32, 24), cfg["params"], bc=cfg["bc"])
    gpu.init_jet()
    gpu.step(7)
    blob = gpu.save()
    gpu.step(5)
    a = gpu.populations(device=False)
    gpu.load(blob)
    assert gpu.step_count == 7
    gpu.step(5)
    assert np.array_equal(gpu.populations(device=False), a)


def test_unstable_state_is_reported(lb):
    """Fault injection on the host: a checkpoint carrying a NaN population makes the next
    periodic mass check return LB_EUNSTABLE."""
    shape = (8, 8, 8)
    params = dict(rho_r0=1.0, rho_b0=1.0, nu_r=0.1, nu_b=0.1, sigma=0.001, check_every=2)
    gpu = lb.Lattice((8, 8, 8), params)
    gpu.init_droplet(2.5, 2.0)
    gpu.step(2)
    blob = bytearray(gpu.save())
    hdr = len(blob) - 54 * 512 * 4 - 54 * 64 * 4
    np.frombuffer(blob, dtype=np.float32, count=1, offset=hdr + 4 * 100)[:]  # readable
    view = np.frombuffer(blob, dtype=np.float32, offset=hdr, count=54 * 512)
    view = view.copy()
    view[1234] = np.nan
    blob[hdr:hdr + view.nbytes] = view.tobytes()
    gpu.load(bytes(blob))
    with pytest.raises(lb.LBError) as ei:
        gpu.step(2)
    assert ei.value.status == 4


def test_host_errors(lb):
    g = lb.Lattice((4, 4, 4), dict(rho_r0=1.0, rho_b0=1.0))
    with pytest.raises(lb.LBError) as ei:
        g.step(1)
    assert ei.value.status == 6  # LB_ESTATE before init
    with pytest.raises(lb.LBError):
        g.init_droplet(-1.0, 4.0)
    assert lb.library().lb_adjoint(g._ctx, 0, 10, None, None, 0) == 1  # LB_EINVAL: NULL arguments
    with pytest.raises(lb.LBError) as ei:
        g.adjoint(3)
    assert ei.value.status == 6  # LB_ESTATE before init
    with pytest.raises(lb.LBError) as ei:
        g.set_params(nu_r=-1.0)
    assert ei.value.status == 1 and g.params.get("nu_r") != -1.0
    for st in (1, 2):  # an FP16 state is encoded against the densities' shift weights
        h = lb.Lattice((4, 4, 4), dict(rho_r0=1.0, rho_b0=1.0, storage=st))
        h.set_params(rho_b0=0.5)  # no state yet
        h.init_droplet(1.5, 2.0)
        with pytest.raises(lb.LBError) as ei:
            h.set_params(rho_r0=2.0)
        assert ei.value.status == 1
        h.set_params(sigma=0.02)


# ------------------------------------------------------------------ FP16 storage
# Half precision keeps 11 significant bits: a stored deviation h from the rest equilibrium
# carries a relative rounding of 2^-12, and h is at most a fraction of w_i rho.  The bar for
# populations after 50 steps is therefore 5e-3 of w_i max(rho_k0) (the FP32 bar is 1e-5).
TOL16 = 5e-3


@pytest.mark.parametrize("storage", [1, 2])
@pytest.mark.parametrize("case", ["droplet", "two_phase", "jet"])
def test_fp16_storage_parity(lb, case, storage):
    if case == "droplet":
        shape, bc = (20, 20, 20), (0, 0)
        params = dict(rho_r0=1.0, rho_b0=1.0, nu_r=1 / 6, nu_b=1 / 6, sigma=0.01)
    elif case == "two_phase":
        shape, bc = (12, 9, 40), (0, 0)
        params = dict(rho_r0=1.0, rho_b0=0.5, nu_r=0.02, nu_b=0.08, sigma=0.003, g=(0.0, 0.0, 1e-5))
    else:
        cfg = workloads.scaled_jet("jet96", 36, 34, 40, D=10)
        shape, bc, params = (40, 34, 36), cfg["bc"], dict(cfg["params"])
    gpu, ref = pair(lb, shape, dict(params, storage=storage), bc=bc)
    if case == "droplet":
        gpu.init_droplet(6.0, 4.0)
        ref.init_droplet(6.0, 4.0)
    elif case == "two_phase":
        fields = workloads.random_two_phase_fields(shape, 1, 1.0, 0.5, u_amp=0.03)
        gpu.init_fields(*fields)
        ref.init_fields(*fields)
    else:
        gpu.init_jet()
        ref.init_jet()
    run_both(gpu, ref, 50)
    e = norm_err(gpu, ref, params)
    assert e.max() < TOL16, e.max()
    F = gpu.fields(device=False)
    R = ref.fields()
    assert np.abs(F["phi"] - R["phi"]).max() < 2e-3
    # velocity: half-precision rounding of the stored deviations moves u by ~1e-5 per step,
    # a random walk of ~1e-4 over 50 steps, on top of 2% of the flow's own speed
    u_ref = np.abs(R["u"]).max()
    for d, nm in enumerate(("ux", "uy", "uz")):
        assert np.abs(F[nm] - R["u"][d]).max() < 2e-2 * u_ref + 1e-4


@pytest.mark.parametrize("case", ["two_phase", "jet"])
def test_fitted_fp16_fields_within_1e3_of_the_oracle(lb, case):
    """The fitted half-precision storage against the FP64 oracle after 50 steps: largest
    |phi - phi_oracle| <= 1e-3 and relative L2 error of the velocity <= 1e-3, the precision
    target for FP16 population storage.  (The rest-shift storage, LB_STORE_FP16, does not hold
    1e-3 on longer runs: it is tested with the population bar above only.)"""
    if case == "two_phase":
        shape, bc = (12, 9, 40), (0, 0)
        params = dict(rho_r0=1.0, rho_b0=0.5, nu_r=0.02, nu_b=0.08, sigma=0.003, g=(0.0, 0.0, 1e-5))
    else:
        cfg = workloads.scaled_jet("jet96", 36, 34, 40, D=10)
        shape, bc, params = (40, 34, 36), cfg["bc"], dict(cfg["params"])
    gpu, ref = pair(lb, shape, dict(params, storage=2), bc=bc)
    if case == "two_phase":
        fields = workloads.random_two_phase_fields(shape, 1, 1.0, 0.5, u_amp=0.03)
        gpu.init_fields(*fields)
        ref.init_fields(*fields)
    else:
        gpu.init_jet()
        ref.init_jet()
    run_both(gpu, ref, 50)
    F = gpu.fields(device=False)
    R = ref.fields()
    dphi = np.abs(F["phi"] - R["phi"]).max()
    du = np.stack([F[k].astype(np.float64) - R["u"][d] for d, k in enumerate(("ux", "uy", "uz"))])
    rel_u = np.linalg.norm(du) / np.linalg.norm(R["u"])
    print(f"FP16_FIT vs oracle, {case}: max|dphi| {dphi:.3e}, rel L2 u {rel_u:.3e}")
    assert dphi <= 1e-3 and rel_u <= 1e-3, (dphi, rel_u)


@pytest.mark.parametrize("storage", [1, 2])
def test_fp16_storage_conserves_colour_mass(lb, storage):
    """The FP32 rest population absorbs the half-precision rounding of the moving ones, so
    colour mass moves only by the FP32 rounding of the nodes' density sums (1e-8 per step)."""
    shape = (24, 20, 36)
    params = dict(rho_r0=1.0, rho_b0=0.5, nu_r=0.02, nu_b=0.05, sigma=0.003, storage=storage)
    gpu = lb.Lattice((36, 20, 24), params)
    gpu.init_fields(*workloads.random_two_phase_fields(shape, 4, 1.0, 0.5))
    m0 = gpu.mass()
    gpu.step(1000)
    m1 = gpu.mass()
    assert np.all(np.abs(m1 - m0) / m0 < 1e-5), (m0, m1)


@pytest.mark.parametrize("storage", [1, 2])
def test_fp16_save_load_roundtrip_is_bitwise(lb, storage):
    cfg = workloads.scaled_jet("jet96", 32, 32, 24, D=8)
    gpu = lb.Lattice((32, 32, 24), dict(cfg["params"], storage=storage), bc=cfg["bc"])
    gpu.init_jet()
    gpu.step(7)
    blob = gpu.save()
    gpu.step(5)
    a = gpu.populations(device=False)
    gpu.load(blob)
    gpu.step(5)
    assert np.array_equal(gpu.populations(device=False), a)


# ------------------------------------------------------------ free-slip side walls
def test_side_walls_jet_parity(lb):
    """The paper's jet boundaries (Section IV.A): inlet disc at z = 0, convective outflow, and
    free-slip walls on all four sides, 36x34x40, 50 steps."""
    cfg = workloads.scaled_jet("jet96", 36, 34, 40, D=10)
    params = cfg["params"]
    shape = (40, 34, 36)
    bc = tuple(cfg["bc"]) + (1, 1)
    gpu, ref = pair(lb, shape, params, bc=bc)
    gpu.init_jet()
    ref.init_jet()
    run_both(gpu, ref, 50)
    e = norm_err(gpu, ref, params)
    assert e.max() < TOL, e.max()


@pytest.mark.parametrize("walls", [(1, 0), (0, 1), (1, 1)])
def test_closed_and_side_walled_boxes_with_gravity(lb, walls):
    """Random two-phase state, free-slip z walls, free-slip x and/or y walls, gravity with
    components along every axis, ragged 33x10x9 lattice, 40 steps."""
    shape = (9, 10, 33)
    params = dict(rho_r0=1.0, rho_b0=0.5, nu_r=0.03, nu_b=0.06, sigma=0.003, g=(2e-5, -3e-5, 4e-5))
    gpu, ref = pair(lb, shape, params, bc=(1, 1) + walls)
    fields = workloads.random_two_phase_fields(shape, 13, 1.0, 0.5, u_amp=0.03)
    gpu.init_fields(*fields)
    ref.init_fields(*fields)
    run_both(gpu, ref, 40)
    e = norm_err(gpu, ref, params)
    assert e.max() < TOL, e.max()


@pytest.mark.parametrize("storage", [1, 2])
def test_side_walls_fp16_storage_parity(lb, storage):
    cfg = workloads.scaled_jet("jet96", 36, 34, 40, D=10)
    params = dict(cfg["params"], storage=storage)
    shape = (40, 34, 36)
    gpu, ref = pair(lb, shape, params, bc=tuple(cfg["bc"]) + (1, 1))
    gpu.init_jet()
    ref.init_jet()
    run_both(gpu, ref, 50)
    e = norm_err(gpu, ref, params)
    assert e.max() < TOL16, e.max()


@pytest.mark.parametrize("storage", [0, 1, 2])
def test_mass_fraction_alpha_parity(lb, storage):
    """Reading R15 (alpha-bar by mass fraction) at density ratio 20 with gravity: random
    two-phase state, 30 steps."""
    shape = (10, 9, 34)
    params = dict(rho_r0=20.0, rho_b0=1.0, nu_r=0.03, nu_b=0.06, sigma=0.003, g=(0.0, 1e-5, -2e-5), alpha_mix=1,
                  storage=storage)
    gpu, ref = pair(lb, shape, params)
    fields = workloads.random_two_phase_fields(shape, 17, 20.0, 1.0, u_amp=0.02)
    gpu.init_fields(*fields)
    ref.init_fields(*fields)
    run_both(gpu, ref, 30)
    e = norm_err(gpu, ref, params)
    assert e.max() < (TOL if storage == 0 else TOL16), e.max()
    F = gpu.fields(device=False)
    ar = 1 - (1 - 8 / 27) / 20.0
    add = F["rho_r"] * 9 * (1 - ar) / 19 + F["rho_b"] / 3
    assert np.abs(F["p"] - add).max() < 1e-5 * add.max()  # additive equation of state


@pytest.mark.parametrize("storage,bc", [(0, (1, 3)), (1, (1, 3)), (2, (1, 3)), (0, (1, 3, 1, 1)), (2, (1, 3, 1, 1)),
                                        (0, (0, 0))])
def test_uniform_rest_state_is_a_fixed_point(lb, storage, bc):
    """A uniform resting mixture (gamma = 1.5, the jet's ambient ratio) must stay exactly at rest:
    after the first step the state repeats bit for bit, so the interior cannot drift away from
    a frozen convective plane and set up a spurious outflow velocity."""
    shape = (16, 12, 40)
    params = dict(rho_r0=1.0, rho_b0=2 / 3, nu_r=4e-4, nu_b=4e-4, sigma=4e-4, storage=storage)
    nz, ny, nx = shape
    gpu = lb.Lattice((nx, ny, nz), params, bc=bc)
    for rr, rb in ((0.0, 2 / 3), (0.3, 0.4), (1.0, 0.0)):
        gpu.init_fields(np.full(shape, rr, np.float32), np.full(shape, rb, np.float32), np.zeros((3,) + shape, np.float32))
        gpu.step(1)
        s1 = gpu.populations(device=False).copy()
        gpu.step(40)
        assert np.array_equal(gpu.populations(device=False), s1)
        F = gpu.fields(device=False)
        for k in ("ux", "uy", "uz"):
            assert not F[k].any()
        assert np.unique(F["rho_r"]).size == 1 and np.unique(F["rho_b"]).size == 1


@pytest.mark.parametrize("case", ["two_phase", "jet"])
def test_fitted_fp16_encoding_is_closer_to_the_oracle(lb, case):
    """The fitted prediction leaves smaller deviations to round than the rest shift, most of
    all at interfaces: after 50 steps the populations' RMS error against the oracle must be
    well below that of the rest-shift encoding on the same case."""
    if case == "two_phase":
        shape, bc = (12, 9, 40), (0, 0)
        params = dict(rho_r0=1.0, rho_b0=0.5, nu_r=0.02, nu_b=0.08, sigma=0.003, g=(0.0, 0.0, 1e-5))
    else:
        cfg = workloads.scaled_jet("jet96", 36, 34, 40, D=10)
        shape, bc, params = (40, 34, 36), cfg["bc"], dict(cfg["params"])
    nz, ny, nx = shape
    ref = oracle.Lattice(oracle.make_grid(nx, ny, nz, *bc), oracle.make_params(full_params(params)))
    gpus = {st: lb.Lattice((nx, ny, nz), dict(params, storage=st), bc=bc) for st in (1, 2)}
    if case == "two_phase":
        fields = workloads.random_two_phase_fields(shape, 1, 1.0, 0.5, u_amp=0.03)
        ref.init_fields(*fields)
        for g in gpus.values():
            g.init_fields(*fields)
    else:
        ref.init_jet()
        for g in gpus.values():
            g.init_jet()
    ref.step(50)
    rms = {}
    for st, g in gpus.items():
        g.step(50)
        rms[st] = float(np.sqrt(np.mean(norm_err(g, ref, params) ** 2)))
    assert rms[2] < 0.6 * rms[1], rms


@pytest.mark.parametrize("storage,bc", [(0, None), (1, None), (2, None), (0, (0, 0))])
def test_fused_step_kernel_equals_the_two_launches(lb, storage, bc):
    """The fused step kernel (one cooperative launch, params.step_kernel = 1) computes what the
    two launches compute, node by node with the same device functions; the compiler contracts
    some products into FMAs differently in the two kernels, so the populations agree to FP32
    rounding (the normalised error of the parity tests within 1e-6 after 30 steps; with the
    half-precision storages a last-bit FP32 difference can move a stored deviation by one FP16
    step, so there the FP16 parity bar TOL16 applies), on the small jet (inlet, outflow, every
    storage; nx = 64 drops the moments' L2 lines after use) and a periodic two-phase lattice
    with gravity."""
    if bc is None:
        cfg = workloads.scaled_jet("jet96", 64, 34, 40, D=10)
        grid, bc, params, shape = (64, 34, 40), cfg["bc"], dict(cfg["params"]), None
    else:
        shape = (24, 9, 40)
        grid, params = (40, 9, 24), dict(rho_r0=1.0, rho_b0=0.5, nu_r=0.02, nu_b=0.08, sigma=0.003, g=(0.0, 0.0, 1e-5))
    out = []
    for sk in (0, 1):
        lat = lb.Lattice(grid, dict(params, storage=storage, step_kernel=sk), bc=bc)
        if shape is None:
            lat.init_jet()
        else:
            lat.init_fields(*workloads.random_two_phase_fields(shape, 6, 1.0, 0.5, u_amp=0.03))
        lat.step(30)
        out.append(lat.populations(device=False))
        lat.mass()  # reports a wait of the fused kernel that ran out (LB_ETIMEOUT)
    w = oracle.weights()[None, :, None, None, None]
    err = np.abs(out[0].astype(np.float64) - out[1]) / (w * max(params["rho_r0"], params["rho_b0"]))
    assert err.max() < (1e-6 if storage == 0 else TOL16), err.max()


@pytest.mark.parametrize("storage,walls", [(0, False), (0, True), (1, False), (2, True)])
def test_large_plane_jet_boundaries_parity(lb, storage, walls):
    """The boundary planes on a plane of 160 x 160 = 25 600 columns, which the library treats
    with its thread-per-column kernel (planes of at least 24 576 columns; the other parity cases
    use the warp-per-column kernel): inlet disc with noise and convective outflow, optionally
    free-slip side walls, 6 steps, populations and the outflow history plane against the oracle."""
    cfg = workloads.scaled_jet("jet96", 160, 160, 8, D=40)
    params = dict(cfg["params"], storage=storage)
    shape = (8, 160, 160)
    bc = tuple(cfg["bc"]) + ((1, 1) if walls else ())
    gpu, ref = pair(lb, shape, params, bc=bc)
    gpu.init_jet()
    ref.init_jet()
    run_both(gpu, ref, 6)
    tol = TOL if storage == 0 else TOL16
    e = norm_err(gpu, ref, params)
    assert e.max() < tol, e.max()
    h = gpu.history().astype(np.float64)
    assert np.abs(h - ref.hist).max() / max(params["rho_r0"], params["rho_b0"]) < tol
    assert gpu.fields(device=False)["rho_r"].sum() > 0.5  # red has entered
