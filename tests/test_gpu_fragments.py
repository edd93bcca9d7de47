"""lb_fragments (GPU union-find labelling, volumes, diameters) against the oracle's flood fill
on the same seeded states: components are named by their smallest node index, so the lists
must agree exactly."""
import numpy as np
import pytest

import oracle

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


def fields_of(jet, rho_b0=0.5):
    phi = np.where(jet, 0.9, -0.9)
    return 1.0 * (1 + phi) / 2, rho_b0 * (1 - phi) / 2, np.zeros((3,) + jet.shape)


def both(lb, jet, bc=(0, 0), storage=0):
    nz, ny, nx = jet.shape
    p = dict(rho_r0=1.0, rho_b0=0.5, nu_r=1 / 6, nu_b=1 / 6, sigma=0.0, storage=storage)
    gpu = lb.Lattice((nx, ny, nz), p, bc=bc)
    ref = oracle.Lattice(oracle.make_grid(nx, ny, nz, *bc), oracle.make_params(dict(p, beta=0.7)))
    f = fields_of(jet)
    gpu.init_fields(*f)
    ref.init_fields(*f)
    return gpu, ref


def same(a, b):
    assert np.array_equal(a["roots"], b["roots"])
    assert np.array_equal(a["volumes"], b["volumes"])
    assert np.allclose(a["diameters"], b["diameters"], rtol=1e-14, atol=0)
    assert a["column_volume"] == b["column_volume"] and a["total_volume"] == b["total_volume"]
    assert a["mass_median_diameter"] == pytest.approx(b["mass_median_diameter"], rel=1e-14)


def balls(shape, spec):
    """Union of balls, periodic in x and y (each evaluated on its own z slab)."""
    nz, ny, nx = shape
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    jet = np.zeros(shape, bool)
    for (cx, cy, cz), R in spec:
        dx = (x - cx + nx / 2) % nx - nx / 2
        dy = (y - cy + ny / 2) % ny - ny / 2
        r2 = dx * dx + dy * dy
        for z in range(max(0, int(np.floor(cz - R))), min(nz, int(np.ceil(cz + R)) + 1)):
            jet[z] |= r2 + (z - cz) ** 2 <= R * R
    return jet


@pytest.mark.parametrize("storage", [0, 1, 2])
def test_balls_with_periodic_wrap(lb, storage):
    jet = balls((20, 18, 37), [((4.2, 5.0, 5.0), 2.6), ((30.0, 12.3, 6.0), 3.1), ((0.4, 9.0, 14.5), 3.4)])
    gpu, ref = both(lb, jet, storage=storage)
    for conn in (6, 26):
        same(gpu.fragments(conn), ref.fragments(conn))
    assert len(gpu.fragments(6)["roots"]) == 3


@pytest.mark.parametrize("conn,fill,periodic_z", [(6, 0.32, True), (26, 0.12, True), (6, 0.25, False)])
def test_random_fields_near_percolation(lb, conn, fill, periodic_z):
    """Random fields near the site-percolation threshold: many small clusters and a few large,
    tortuous ones, which stress the concurrent unions."""
    jet = np.random.default_rng(11).random((24, 40, 70)) < fill
    bc = (0, 0) if periodic_z else (1, 1)
    gpu, ref = both(lb, jet, bc=bc)
    g, r = gpu.fragments(conn), ref.fragments(conn)
    same(g, r)
    assert len(r["roots"]) > 50 and r["volumes"].max() > 100


def test_inlet_column_and_degenerate_states(lb):
    shape = (16, 12, 12)
    jet = np.zeros(shape, bool)
    jet[0:7, 5:7, 5:7] = True
    jet |= balls(shape, [((6.0, 6.0, 11.0), 2.2)])
    gpu, ref = both(lb, jet, bc=(2, 3))
    same(gpu.fragments(6), ref.fragments(6))
    same(gpu.fragments(6, exclude_inlet=False), ref.fragments(6, exclude_inlet=False))
    assert gpu.fragments(6)["column_volume"] == 28
    empty, _ = both(lb, np.zeros((6, 5, 7), bool))
    e = empty.fragments(26)
    assert len(e["roots"]) == 0 and e["mass_median_diameter"] == 0.0
    full, _ = both(lb, np.ones((6, 5, 7), bool))
    f = full.fragments(6)
    assert list(f["roots"]) == [0] and list(f["volumes"]) == [210]
    with pytest.raises(lb.LBError):
        full.fragments(18)


def test_full_size_field(lb):
    """The benchmark's 96x96x384 lattice (3.5 M nodes) with 400 random balls: one launch
    configuration at full size, against the oracle."""
    rng = np.random.default_rng(5)
    shape = (384, 96, 96)
    spec = [((rng.uniform(0, 96), rng.uniform(0, 96), rng.uniform(3, 381)), rng.uniform(0.8, 4.0)) for _ in range(400)]
    jet = balls(shape, spec)
    gpu, ref = both(lb, jet, bc=(1, 1))
    same(gpu.fragments(6), ref.fragments(6))


def test_no_fragment_joins_across_a_side_wall(lb):
    """With free-slip side walls a ball cut by the x = 0 plane is two pieces, not one wrapped
    fragment; against the oracle."""
    jet = balls((14, 12, 20), [((0.2, 6.0, 7.0), 3.3), ((10.0, 0.1, 6.0), 2.8)])
    gw, rw = both(lb, jet, bc=(1, 1, 1, 1))
    same(gw.fragments(6), rw.fragments(6))
    gp, rp = both(lb, jet, bc=(1, 1))
    assert len(gw.fragments(6)["roots"]) == len(gp.fragments(6)["roots"]) + 2
