"""Pins of the oracle's convective outflow (Section IV.A, Eqs. (45)-(47)) against the
advection equation it discretises.

At the outflow node N the paper applies df_i/dt + U_c df_i/dz = 0 with the first-order
implicit scheme f_i(N, t+1) = [f_i(N, t) + lambda f_i(N-1, t+1)] / (1 + lambda), where
lambda = U_c(t+1) = u_z(x, y, N-1, t+1).  That is backward Euler in time of the upwind
semi-discretisation df_N/dt = -U (f_N - f_{N-1}); the tests below drive the N-1 plane of a
one-column lattice through the oracle's streaming call and compare the outflow plane with
what the advection equation and its discretisation fix:

* a slow harmonic modulation passes the boundary with gain -> 1 and phase lag -> omega/U,
  the one-cell transit time 1/U of the continuous equation (a swapped blend,
  [lambda f(N, t) + f(N-1, t+1)] / (1 + lambda), lags by omega U instead), and the response
  equals the scheme's transfer function U / (1 + U - exp(-i omega)) exactly;
* after a jump of the convective speed from 0 to U the outflow relaxes towards the new
  inflow as (1 + U)^-m at every step m >= 1, which holds only with lambda taken at the new
  time level t + 1 as Eq. (46) prints (lambda at t leaves the first step frozen).
"""
import numpy as np
import pytest

import oracle

NZ = 4  # planes 0..3: N = 3, N - 1 = 2; the pulls into N - 1 come from planes 1..3


def column_lattice(**params):
    p = dict(rho_r0=1.0, rho_b0=0.5, nu_r=0.01, nu_b=0.01, sigma=0.0)
    p.update(params)
    return oracle.Lattice(oracle.make_grid(1, 1, NZ, oracle.BC_FREESLIP, oracle.BC_CONVECTIVE),
                          oracle.make_params(p))


def red_equilibrium(rho, uz):
    alpha_r = 1.0 - (1.0 - 8.0 / 27.0) / 2.0  # gamma = rho_r0 / rho_b0 = 2
    return oracle.equilibrium(rho, [0.0, 0.0, uz], alpha_r, 0.01, [0.0, 0.0, 0.0])


CZ = oracle.velocity_set()[:, 2]


def drive(lat, inflow, prev=None):
    """Streams once so that the post-stream plane N - 1 holds the red populations `inflow`
    (27) exactly; returns the outflow plane f(N) of that step (27 red values) and keeps the
    history.  The post-collision state S(t) holds `inflow` on planes 1..3, except that the
    moving (c_z != 0) populations of plane N - 1 itself are those of `prev` (the inflow of the
    step before): S(t) at N - 1 then carries the old velocity u_z(N - 1, t), while the pulls
    from N - 2 and N bring in the new one, as in a flow whose speed changes."""
    S = np.zeros_like(lat.S)
    S[0, :, 1:, 0, 0] = inflow[:, None]
    if prev is not None:
        S[0, CZ != 0, NZ - 2, 0, 0] = prev[CZ != 0]
    lat.set_state(S)
    f, h = lat.stream()
    lat.hist = h
    lat.step_count += 1
    assert np.array_equal(f[0, :, NZ - 2, 0, 0], inflow)
    assert np.array_equal(f[0, :, NZ - 1, 0, 0], h[0, :, 0, 0])
    return f[0, :, NZ - 1, 0, 0].copy()


def harmonic_response(U, period, periods=4):
    """Complex ratio of the outflow's and the inflow's Fourier coefficients at omega = 2 pi /
    period, per direction, over the last two periods of a run of `periods` periods."""
    lat = column_lattice()
    e = red_equilibrium(1.0, U)
    lat.hist[0, :, 0, 0] = e  # the outflow starts at the mean inflow
    omega = 2 * np.pi / period
    T = periods * period
    rho = 1.0 + 0.01 * np.sin(omega * np.arange(1, T + 1))
    out = np.array([drive(lat, r * e, r0 * e) for r, r0 in zip(rho, np.r_[1.0, rho[:-1]])])  # f(N, t)
    t = np.arange(1, T + 1)[-2 * period:]
    ph = np.exp(-1j * omega * t)
    a_in = ((rho[-2 * period:] - 1.0) * ph).sum()
    a_out = ((out[-2 * period:] - e[None, :]) * ph[:, None]).sum(0)
    return a_out / (a_in * e), omega


@pytest.mark.parametrize("U", [0.05, 0.2])
def test_slow_modulation_crosses_the_outflow_in_one_cell_transit_time(U):
    H, omega = harmonic_response(U, period=2000)
    assert np.allclose(H, H[0], rtol=1e-12, atol=0)  # every direction is advected alike
    gain, lag = np.abs(H[0]), -np.angle(H[0])
    # continuous advection: unit gain, phase lag omega * (delta z / U)
    assert abs(gain - 1.0) < (omega / U) ** 2
    assert abs(lag / (omega / U) - 1.0) < 0.02
    # the implicit scheme's own transfer function, U / (1 + U - exp(-i omega))
    H_scheme = U / (1.0 + U - np.exp(-1j * omega))
    assert abs(H[0] / H_scheme - 1.0) < 1e-9


def test_fast_modulation_is_damped_as_the_scheme_predicts():
    """Away from the continuum limit (period 20, U = 0.05) the scheme damps strongly; the
    response still equals its transfer function."""
    U = 0.05
    H, omega = harmonic_response(U, period=20, periods=60)
    H_scheme = U / (1.0 + U - np.exp(-1j * omega))
    assert np.abs(H / H_scheme - 1.0).max() < 1e-9
    assert np.abs(H[0]) < 0.2


@pytest.mark.parametrize("U", [0.05, 0.3])
def test_speed_jump_relaxes_with_lambda_at_the_new_time_level(U):
    """The inflow switches from fluid at rest (lambda = 0: the outflow plane is frozen) to
    fluid moving at U; from the first step after the switch the outflow approaches the new
    inflow by the factor 1 / (1 + U) per step."""
    lat = column_lattice()
    g0, g1 = red_equilibrium(1.0, 0.0), red_equilibrium(1.1, U)
    lat.hist[0, :, 0, 0] = 0.9 * g0  # an outflow plane that differs from the inflow
    for _ in range(5):
        out = drive(lat, g0)
        assert np.array_equal(out, 0.9 * g0)  # lambda = u_z(N-1) = 0 freezes the plane
    for m in range(1, 41):
        out = drive(lat, g1, g0 if m == 1 else g1)
        expect = g1 + (0.9 * g0 - g1) * (1.0 + U) ** (-m)
        assert np.abs(out - expect).max() < 1e-13 * np.abs(g1).max(), m


def test_backflow_freezes_the_outflow_plane():
    """Reading of Section IV.A for u_z(N-1) < 0 (the paper is silent): lambda is clamped to
    [0, 1], so inflowing fluid at the outflow leaves f(N) at its history."""
    lat = column_lattice()
    g = red_equilibrium(1.0, -0.03)
    lat.hist[0, :, 0, 0] = red_equilibrium(0.95, 0.0)
    h0 = lat.hist.copy()
    for _ in range(3):
        drive(lat, g)
    assert np.array_equal(lat.hist, h0)
