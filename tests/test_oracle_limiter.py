"""Pins of the flux-limited drag oracle (oracle/limiter.py) against what the mathematics fixes:
the upwind step as the mu = 0 special case, exact transport of quadratic cell averages by the
kappa = 1/3 face values, conservation, positivity and the TVD property under the Courant bound,
the 2D step reducing to the 1D one, and second-order convergence to the exact solution of the
drag equation (characteristics) where the upwind step converges at first order."""
import math

import numpy as np
import pytest

from oracle import lattice as O
from oracle import limiter as K


def test_single_stage_with_mu_zero_is_the_upwind_step():
    rng = np.random.default_rng(1)
    nv, nx, dv, dt, tau_p = 17, 9, 0.2, 0.05, 1.0
    f = rng.random((nv, nx))
    u = rng.uniform(-1.0, 1.0, nx)
    v = O.velocities(nv, dv)
    a = O.drag_acceleration(v[:, None], u[None, :], tau_p) * np.ones_like(f)
    got = K._stage_1d(f, a, dt / dv, 0.0)
    assert np.array_equal(got, O.drag_1d(f, u, tau_p, dt, dv))


@pytest.mark.parametrize("sign", [1.0, -1.0])
@pytest.mark.parametrize("mu", [2.0 / 3.0, 1.0])
def test_face_values_transport_quadratic_cell_averages_exactly(sign, mu):
    """Cell averages of q(s) = 1 + 0.3 s + 0.02 s^2 over unit cells [j - 1/2, j + 1/2]: the limited
    kappa = 1/3 face value equals q at the face, so F = a q(j + 1/2) for a constant speed a.
    (Away from the walls, where the stencil holds real cells; theta stays near 1, unclipped.)"""
    n = 24
    s = np.arange(n, dtype=np.float64)
    q = lambda x: 1.0 + 0.3 * x + 0.02 * x * x  # noqa: E731
    avg = q(s) + 0.02 / 12.0
    a = np.full(n, 0.7 * sign)
    F = K.limited_fluxes(a, avg, mu)
    faces = np.arange(2, n - 3)  # interface j + 1/2 for j = 2 .. n - 4
    np.testing.assert_allclose(F[faces + 1], a[0] * q(faces + 0.5), rtol=1e-13)


@pytest.mark.parametrize("mu", [2.0 / 3.0, 1.0])
def test_mass_is_conserved(mu):
    rng = np.random.default_rng(2)
    f = rng.random((33, 40)) * np.exp(rng.normal(0, 1, (33, 40)))
    u = rng.uniform(-2.0, 2.0, 40)
    g = K.drag_1d(f, u, 1.0, 0.02, 0.25, mu)
    np.testing.assert_allclose(g.sum(axis=0), f.sum(axis=0), rtol=1e-14)
    f2 = rng.random((9, 9, 4, 5))
    g2 = K.drag_2d(f2, rng.uniform(-1, 1, (4, 5)), rng.uniform(-1, 1, (4, 5)), 1.0, 0.05, 0.3, mu)
    np.testing.assert_allclose(g2.sum(axis=(0, 1)), f2.sum(axis=(0, 1)), rtol=1e-14)


@pytest.mark.parametrize("mu", [2.0 / 3.0, 1.0])
@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_stages_are_tvd_and_positive_at_the_courant_bound(mu, sign):
    """Constant speed, nu (1 + mu) = 1, rough nonnegative data kept away from the walls: the total
    variation never grows and no value goes negative (Harten's conditions for psi <= 1,
    psi / theta <= mu)."""
    rng = np.random.default_rng(3)
    n = 80
    f = np.zeros(n)
    f[25:55] = rng.random(30) * (rng.random(30) > 0.3)
    a = np.full(n, sign)
    c = 1.0 / (1.0 + mu)
    tv = lambda x: np.abs(np.diff(np.concatenate([[0.0], x, [0.0]]))).sum()  # noqa: E731
    for _ in range(10):
        g = K._stage_1d(f, a, c, mu)
        assert tv(g) <= tv(f) * (1 + 1e-14)
        assert g.min() >= -1e-15
        f = g


def test_drag_field_stays_positive_over_many_steps():
    rng = np.random.default_rng(4)
    nv, nx, tau_p, mu = 33, 16, 1.0, 2.0 / 3.0
    J = (nv - 1) // 2
    f = rng.random((nv, nx)) * (rng.random((nv, nx)) > 0.5)
    dv = 0.1
    umax = 0.5
    dt = dv * tau_p / ((J * dv + umax) * (1 + mu))  # nu (1 + mu) = 1 at the extreme cell
    for _ in range(50):
        u = rng.uniform(-umax, umax, nx)
        f = K.drag_1d(f, u, tau_p, dt, dv, mu)
        assert f.min() >= -1e-14 * f.max()


def test_2d_step_on_a_single_row_is_the_1d_step():
    """All mass in velocity row jy0 with uy = v_jy0: the vy drag vanishes there and no vy flux
    moves anything, so the unsplit 2D stage is the 1D stage on that row, bit for bit."""
    rng = np.random.default_rng(5)
    nv, nx, ny, dv, dt = 9, 3, 2, 0.3, 0.04
    jy0 = 6
    f = np.zeros((nv, nv, ny, nx))
    f[jy0] = rng.random((nv, ny, nx))
    ux = rng.uniform(-0.5, 0.5, (ny, nx))
    uy = np.full((ny, nx), O.velocities(nv, dv)[jy0])
    g = K.drag_2d(f, ux, uy, 1.0, dt, dv)
    for y in range(ny):
        want = K.drag_1d(f[jy0, :, y, :], ux[y], 1.0, dt, dv)
        assert np.array_equal(g[jy0, :, y, :], want)
    assert not np.any(np.delete(g, jy0, axis=0))


def _exact_averages(nv, vmax, t, tau, v0, sig):
    """Cell averages of the drag equation's solution with u = 0: the mass between v_l and v_r at
    time t is the initial mass between v_l e^{t/tau} and v_r e^{t/tau} (characteristics
    v(t) = v(0) e^{-t/tau}); the initial state is a normalised Gaussian (v0, sig)."""
    J = (nv - 1) // 2
    dv = vmax / J
    edges = (np.arange(nv + 1) - J - 0.5) * dv * math.exp(t / tau)
    cdf = np.array([0.5 * (1 + math.erf((e - v0) / (sig * math.sqrt(2)))) for e in edges])
    return np.diff(cdf) / dv, dv


def test_limited_step_converges_at_second_order_where_upwind_is_first():
    tau, vmax, v0, sig, T, nu = 1.0, 4.0, 1.0, 0.5, 0.5, 0.4
    errs = {"upwind": [], "limited": []}
    sizes = (33, 65, 129, 257)
    for nv in sizes:
        f0, dv = _exact_averages(nv, vmax, 0.0, tau, v0, sig)
        want, _ = _exact_averages(nv, vmax, T, tau, v0, sig)
        n = int(math.ceil(T / (nu * dv * tau / vmax)))
        dt = T / n
        u = np.zeros(1)
        fu = f0[:, None].copy()
        fl = f0[:, None].copy()
        for _ in range(n):
            fu = O.drag_1d(fu, u, tau, dt, dv)
            fl = K.drag_1d(fl, u, tau, dt, dv)
        errs["upwind"].append(np.abs(fu[:, 0] - want).sum() * dv)
        errs["limited"].append(np.abs(fl[:, 0] - want).sum() * dv)
    order = {k: np.log2(np.array(v[:-1]) / np.array(v[1:])) for k, v in errs.items()}
    # observed: upwind 0.75, 0.82, 0.91 (tending to 1); limited 1.46, 2.07, 2.05
    assert 0.8 < order["upwind"][-1] < 1.2, order
    assert np.all(order["limited"][1:] > 1.8), order
    assert errs["limited"][-1] < 0.05 * errs["upwind"][-1]
