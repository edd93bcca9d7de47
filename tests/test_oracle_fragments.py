"""Pins of the oracle's fragment analysis (Section IV.B diameter procedure, reading R13)
against independent computations: lattice-point counts of balls, scipy's labelling, and
hand-worked diameters."""
import numpy as np
import pytest

import oracle


def lattice_with(jet, bc=(oracle.BC_PERIODIC, oracle.BC_PERIODIC), rho_b0=0.5):
    """An oracle lattice whose state has phi = +0.9 on the jet nodes and -0.9 elsewhere."""
    nz, ny, nx = jet.shape
    p = dict(rho_r0=1.0, rho_b0=rho_b0, nu_r=1 / 6, nu_b=1 / 6, sigma=0.0)
    lat = oracle.Lattice(oracle.make_grid(nx, ny, nz, *bc), oracle.make_params(p))
    phi = np.where(jet, 0.9, -0.9)
    lat.init_fields(1.0 * (1 + phi) / 2, rho_b0 * (1 - phi) / 2, np.zeros((3,) + jet.shape))
    return lat


def periodic_ball(shape, centre, R, periodic_z=False):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    d = [x - centre[0], y - centre[1], z - centre[2]]
    for k, n in enumerate((nx, ny, nz)):
        if k < 2 or periodic_z:
            d[k] = (d[k] + n / 2) % n - n / 2
    return d[0] ** 2 + d[1] ** 2 + d[2] ** 2 <= R * R


def test_separated_balls_and_periodic_wrap():
    shape = (20, 18, 22)
    balls = [((4.2, 5.0, 5.0), 2.6), ((15.0, 12.3, 6.0), 3.1), ((0.4, 9.0, 14.5), 3.4)]  # the last wraps in x
    masks = [periodic_ball(shape, c, R) for c, R in balls]
    jet = np.any(masks, axis=0)
    fr = lattice_with(jet).fragments(6)
    expect_roots = sorted(int(np.flatnonzero(m.ravel())[0]) for m in masks)
    assert list(fr["roots"]) == expect_roots
    by_root = {int(np.flatnonzero(m.ravel())[0]): int(m.sum()) for m in masks}
    assert [by_root[r] for r in fr["roots"]] == list(fr["volumes"])
    assert np.allclose(fr["diameters"], (6 * fr["volumes"] / np.pi) ** (1 / 3))


def test_connectivity_6_and_26():
    """Two cubes touching along an edge: two fragments with faces, one with the full
    neighbourhood; touching at a corner likewise."""
    jet = np.zeros((10, 10, 10), bool)
    jet[2:4, 2:4, 2:4] = True
    jet[4:6, 4:6, 2:4] = True  # shares the edge x = 3|4, y = 3|4
    lat = lattice_with(jet)
    assert len(lat.fragments(6)["roots"]) == 2
    assert len(lat.fragments(26)["roots"]) == 1
    jet2 = np.zeros((10, 10, 10), bool)
    jet2[1:3, 1:3, 1:3] = True
    jet2[3:5, 3:5, 3:5] = True  # corner contact
    lat2 = lattice_with(jet2)
    assert len(lat2.fragments(6)["roots"]) == 2 and len(lat2.fragments(26)["roots"]) == 1


@pytest.mark.parametrize("conn", [6, 26])
def test_random_field_against_scipy_label(conn):
    """A random field with an empty border in x and y (so periodic wrapping joins nothing)
    against scipy.ndimage.label: same components, named by their smallest index."""
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(3)
    jet = rng.random((9, 12, 14)) < 0.3
    jet[:, 0, :] = jet[:, -1, :] = False
    jet[:, :, 0] = jet[:, :, -1] = False
    lat = lattice_with(jet, bc=(oracle.BC_FREESLIP, oracle.BC_FREESLIP))
    fr = lat.fragments(conn)
    lab, n = ndimage.label(jet, structure=ndimage.generate_binary_structure(3, 1 if conn == 6 else 3))
    flat = lab.ravel()
    roots = sorted(int(np.flatnonzero(flat == k)[0]) for k in range(1, n + 1))
    assert list(fr["roots"]) == roots
    assert list(fr["volumes"]) == [int((flat == flat[r]).sum()) for r in roots]


def test_inlet_column_is_excluded():
    """On an inlet lattice the component touching z = 0 (the column from the nozzle) is left
    out and reported as the column volume; a detached droplet stays."""
    shape = (16, 12, 12)
    jet = np.zeros(shape, bool)
    jet[0:7, 5:7, 5:7] = True                       # column from the inlet plane
    drop = periodic_ball(shape, (6.0, 6.0, 11.0), 2.2)
    jet |= drop
    lat = lattice_with(jet, bc=(oracle.BC_INLET, oracle.BC_CONVECTIVE))
    fr = lat.fragments(6)
    assert list(fr["volumes"]) == [int(drop.sum())] and fr["column_volume"] == 7 * 4
    assert lat.fragments(6, exclude_inlet=False)["total_volume"] == int(jet.sum())


def test_mass_median_diameter_by_hand():
    """Volumes 1, 8, 27, 2: the total is 38, half is 19; sorted cumulative 1, 3, 11, 38 reaches
    it at V = 27, so d_m = (6 * 27 / pi)^(1/3)."""
    st = oracle.fragment_stats([0, 10, 20, 30], [1, 8, 27, 2])
    assert st["mass_median_diameter"] == pytest.approx((6 * 27 / np.pi) ** (1 / 3), rel=1e-15)
    st2 = oracle.fragment_stats([0, 1], [5, 5])  # cumulative 5, 10: half = 5 reached at the first
    assert st2["mass_median_diameter"] == pytest.approx((30 / np.pi) ** (1 / 3))
    assert oracle.fragment_stats([], [])["mass_median_diameter"] == 0.0
