"""Seeded synthetic workloads shared by the CUDA path's tests/benchmark and the oracle.

This module holds no arithmetic of the method: only the lattice sizes and parameters
of the benchmark configurations, the map from the jet's dimensionless groups to lattice
parameters (the definitions of Eqs. (1)-(5) of arXiv:1804.08923), and seeded random
field generators.  Both the CUDA binding and the oracle read their inputs from here;
neither imports the other.

The paper runs no public dataset: its jet runs are defined by lattice parameters only.
The configurations below are synthetic lattices of the paper's kind (static droplet of
Section III; liquid-liquid and melt jets of Section IV) at stated sizes.
"""
from __future__ import annotations

import numpy as np

BC_PERIODIC, BC_FREESLIP, BC_INLET, BC_CONVECTIVE = 0, 1, 2, 3
ALPHA_B = 8.0 / 27.0  # Section II: alpha_b = 8/27 (c_s^b = 1/sqrt(3))


def jet_parameters(D, u, gamma, eta, Re, We, Fr=None, rho_j=1.0):
    """Lattice parameters of a jet from Eqs. (1)-(5): gamma = rho_j/rho_c,
    eta = nu_j/nu_c, Re = rho_j u D / mu_j (= u D / nu_j), We = rho_j u^2 D / sigma,
    Fr = u^2 / (g D).  The jet (dispersed phase) is red, the coolant blue."""
    nu_j = u * D / Re
    nu_c = nu_j / eta
    sigma = rho_j * u * u * D / We
    g = 0.0 if Fr is None else u * u / (Fr * D)
    return dict(rho_r0=rho_j, rho_b0=rho_j / gamma, nu_r=nu_j, nu_b=nu_c, sigma=sigma,
                g=(0.0, 0.0, g), u_in=u, d_in=float(D))


def _cfg(name, grid, bc, params, init, steps, text):
    p = dict(beta=0.7, s0=0.0, s1=0.0, s2b=1.0, s3=1.0, s4=1.0, s5=1.0, s6=1.0,
             eps_grad=1e-6, noise_amp=0.0, seed=12345, u_in=0.0, d_in=0.0, g=(0.0, 0.0, 0.0))
    p.update(params)
    return dict(name=name, grid=grid, bc=bc, params=p, init=init, steps=steps, text=text)


CONFIGS = {
    "droplet32": _cfg(
        "droplet32", (32, 32, 32), (BC_PERIODIC, BC_PERIODIC),
        dict(rho_r0=1.0, rho_b0=1.0, nu_r=1.0 / 6.0, nu_b=1.0 / 6.0, sigma=0.01),
        dict(kind="droplet", R=8.0, W=4.0), 200,
        "static droplet R=8 W=4 in 32^3, fully periodic, gamma=1, tau=1, sigma=0.01, beta=0.7"),
    "jet96": _cfg(
        "jet96", (96, 96, 384), (BC_INLET, BC_CONVECTIVE),
        dict(**jet_parameters(D=16, u=0.05, gamma=1.5, eta=1.0, Re=2000, We=100), noise_amp=0.01),
        dict(kind="jet"), 5000,
        "liquid-liquid jet 96x96x384, D=16, u=0.05, gamma=1.5, eta=1, Re=2000, We=100, "
        "no gravity, 1% radial inlet noise, convective outflow, periodic x/y"),
    "jet256": _cfg(
        "jet256", (256, 256, 1024), (BC_INLET, BC_CONVECTIVE),
        dict(**jet_parameters(D=32, u=0.04, gamma=2.0, eta=1.0, Re=1e5, We=1000, Fr=100), noise_amp=0.005),
        dict(kind="jet"), 2000,
        "high-Re jet 256x256x1024, D=32, u=0.04, gamma=2, Re=1e5, We=1000, Fr=100 (gravity +z), 0.5% noise"),
    "jet64": _cfg(
        "jet64", (64, 64, 256), (BC_INLET, BC_CONVECTIVE),
        dict(**jet_parameters(D=12, u=0.05, gamma=1.5, eta=1.0, Re=500, We=50)),
        dict(kind="jet"), 500,
        "jet 64x64x256, D=12, u=0.05, gamma=1.5, Re=500, We=50"),
    "jet384": _cfg(
        "jet384", (384, 384, 1536), (BC_INLET, BC_CONVECTIVE),
        dict(**jet_parameters(D=48, u=0.05, gamma=8.0, eta=0.1, Re=1e6, We=5000), noise_amp=0.01),
        dict(kind="jet"), 1000,
        "atomisation jet 384x384x1536 (226M nodes), D=48, u=0.05, gamma=8, eta=0.1, Re=1e6, We=5000, 1% noise"),
    # The paper's own runs (Section IV): UT melt jets (Table of UT conditions, Cases 1-4) on the
    # 8D x 8D x 40D lattice with D = 30, u_j0 = 0.05, rho_j = 1, rho_c = 1/gamma, free-slip side
    # walls, gravity on the dispersed phase, no inlet disturbance.
    **{f"ut{k}": _cfg(
        f"ut{k}", (240, 240, 1200), (BC_INLET, BC_CONVECTIVE, BC_FREESLIP, BC_FREESLIP),
        dict(**jet_parameters(D=30, u=0.05, gamma=8.3, eta=0.54, Re=Re, We=We, Fr=Fr)),
        dict(kind="jet"), 20000,
        f"UT Case {k}: melt jet 240x240x1200, D=30, u=0.05, gamma=8.3, eta=0.54, Re={Re:g}, We={We:g}, Fr={Fr:g}, "
        "free-slip side walls, gravity +z")
       for k, (Re, We, Fr) in enumerate([(6.1e4, 230, 64), (6.5e4, 180, 24), (1.1e5, 330, 20), (1.5e5, 450, 16)], 1)},
    # FT T1, coarse grid: the lattice parameters printed with its figure (sigma = 1.6e-5 gives
    # We = u^2 D / sigma = 4.7e3, not the 9.3e4 of its table of conditions; the printed lattice
    # values are used).
    "ft_coarse": _cfg(
        "ft_coarse", (240, 240, 600), (BC_INLET, BC_CONVECTIVE, BC_FREESLIP, BC_FREESLIP),
        dict(rho_r0=1.0, rho_b0=0.099, nu_r=1.4e-6, nu_b=9.9e-7, sigma=1.6e-5, g=(0.0, 0.0, 4.1e-7),
             u_in=0.05, d_in=30.0),
        dict(kind="jet"), 20000,
        "FT T1 coarse: UO2 melt into sodium 240x240x600, D=30, u=0.05, gamma=10.1, eta=1.4, Re=1.1e6, "
        "lattice sigma=1.6e-5, g=4.1e-7, free-slip side walls"),
}


def scaled_jet(name: str, nx: int, ny: int, nz: int, D: float | None = None) -> dict:
    """A copy of a jet configuration on a smaller lattice (same lattice parameters)."""
    c = dict(CONFIGS[name])
    c["params"] = dict(c["params"])
    c["grid"] = (nx, ny, nz)
    if D is not None:
        c["params"]["d_in"] = float(D)
    c["name"] = f"{name}@{nx}x{ny}x{nz}"
    return c


def _smooth_noise(rng, shape, modes=3):
    """Sum of a few random low Fourier modes on a periodic lattice, unit max amplitude."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    out = np.zeros(shape)
    for _ in range(modes):
        kx, ky, kz = rng.integers(0, 3, size=3)
        ph = rng.uniform(0, 2 * np.pi)
        amp = rng.uniform(0.5, 1.0)
        out += amp * np.cos(2 * np.pi * (kx * x / nx + ky * y / ny + kz * z / nz) + ph)
    m = np.abs(out).max()
    return out / m if m > 0 else out


def random_two_phase_fields(shape, seed, rho_r0=1.0, rho_b0=1.0, u_amp=0.02, width=3.0, ddens=0.01):
    """Seeded smooth two-phase fields (rho_r, rho_b, u) as float32 arrays.

    A red blob bounded by a smooth random surface (tanh profile of the given width),
    small density fluctuations and a smooth random velocity of amplitude u_amp.
    shape = (nz, ny, nx); u has shape (3, nz, ny, nx) with components x, y, z."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r = np.sqrt(((x - (nx - 1) / 2)) ** 2 + ((y - (ny - 1) / 2)) ** 2 + ((z - (nz - 1) / 2)) ** 2)
    R = 0.3 * min(shape) * (1.0 + 0.15 * _smooth_noise(rng, shape))
    s = np.tanh(2.0 * (r - R) / width)
    dens = 1.0 + ddens * _smooth_noise(rng, shape)
    rho_r = 0.5 * rho_r0 * (1.0 - s) * dens
    rho_b = 0.5 * rho_b0 * (1.0 + s) * dens
    u = np.stack([u_amp * _smooth_noise(rng, shape) for _ in range(3)])
    return rho_r.astype(np.float32), rho_b.astype(np.float32), u.astype(np.float32)


def shear_wave_fields(shape, u0, rho_r=1.0, rho_b=0.0):
    """Single-colour shear wave u_x = u0 sin(2 pi y / ny) at uniform density."""
    nz, ny, nx = shape
    y = np.arange(ny)[None, :, None] * np.ones(shape)
    u = np.zeros((3,) + shape)
    u[0] = u0 * np.sin(2 * np.pi * y / ny)
    return (np.full(shape, rho_r, dtype=np.float64), np.full(shape, rho_b, dtype=np.float64), u)


def random_droplet_fields(shape, n, r_min, r_max, seed, rho_r0=1.0, rho_b0=1.0, phi_abs=0.9):
    """Seeded broken-up state: n red balls with radii uniform in [r_min, r_max) at uniform
    random centres (distances wrap periodically in x, y and z; overlapping balls merge) in
    blue.  Binarised like a settled interface: phi = +phi_abs inside, -phi_abs outside, so
    (rho_r, rho_b) = ((1 + phi)/2 rho_r0, (1 - phi)/2 rho_b0), at rest.  shape = (nz, ny, nx);
    returns float32 rho_r, rho_b, u (3, nz, ny, nx)."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    red = np.zeros(shape, dtype=bool)
    for _ in range(n):
        c = rng.uniform(0.0, 1.0, 3) * np.array([nx, ny, nz])
        r = rng.uniform(r_min, r_max)
        k = int(np.ceil(r))
        ax = [(np.arange(int(np.floor(c[d])) - k, int(np.floor(c[d])) + k + 2)) for d in range(3)]
        dx, dy, dz = (ax[d] - c[d] for d in range(3))
        inside = (dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2) < r * r
        iz, iy, ix = np.nonzero(inside)
        red[ax[2][iz] % nz, ax[1][iy] % ny, ax[0][ix] % nx] = True
    phi = np.where(red, phi_abs, -phi_abs)
    rho_r = (0.5 * rho_r0 * (1.0 + phi)).astype(np.float32)
    rho_b = (0.5 * rho_b0 * (1.0 - phi)).astype(np.float32)
    return rho_r, rho_b, np.zeros((3,) + shape, dtype=np.float32)
