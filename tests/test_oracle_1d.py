"""Pins of the 1D FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test states the fact it checks and where it comes from.  Together they are chosen so that
a plausible mistake in the oracle (a reversed shift, a drag sign, a factor 2 in the diffusion, a
missing wall condition, a swapped cos/sin) fails at least one of them; ``test_oracle_mutations``
plants such mistakes and checks exactly that.
"""
import math
import os

import numpy as np
import pytest

from oracle import lattice as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------------------------
# Streaming (Section 2: mass in velocity cell j moves by j grid points; advection is exact)
# ---------------------------------------------------------------------------------------------
def check_unit_mass_moves_by_j(mod=O):
    nx, nv = 11, 7
    J = 3
    for jj in range(nv):
        j = jj - J
        f = np.zeros((nv, nx))
        f[jj, 4] = 1.0
        out = mod.stream_1d(f)
        assert out[jj, (4 + j) % nx] == 1.0, f"velocity {j} must move mass to the right by {j}"
        assert out.sum() == 1.0


def test_unit_mass_moves_by_j():
    check_unit_mass_moves_by_j()


def test_free_streaming_period_is_exact():
    """With no drag (tau_p = inf) and no diffusion, N_x steps return f bit for bit."""
    rng = np.random.default_rng(0)
    nx, nv = 24, 9
    f0 = rng.random((nv, nx))
    f = f0.copy()
    u = np.zeros(nx)
    for _ in range(nx):
        f = O.step_1d(f, u, math.inf, 0.0, 0.1, 0.5)
    assert np.array_equal(f, f0)


# ---------------------------------------------------------------------------------------------
# Hand-derived single steps (golden fixture with its derivation)
# ---------------------------------------------------------------------------------------------
def _golden_1d():
    rows = []
    with open(os.path.join(GOLDEN, "tiny_nv3_1d.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                p = line.split()
                rows.append((p[0], float(p[1]), float(p[2]),
                             np.array([float(x) for x in p[3:6]]),
                             np.array([float(x) for x in p[6:9]])))
    return rows


def check_golden_1d(mod=O):
    for name, u, kappa, fin, fout in _golden_1d():
        got = mod.step_1d(fin.reshape(3, 1), np.array([u]), 2.0, kappa, 0.5, 1.0)[:, 0]
        assert np.array_equal(got, fout), (name, got, fout)


def test_golden_tiny_steps():
    check_golden_1d()


# ---------------------------------------------------------------------------------------------
# Conservation (Section 2: both sub-steps are finite-volume conservation laws, zero wall flux)
# ---------------------------------------------------------------------------------------------
def _random_case(seed, nx=40, nv=17):
    rng = np.random.default_rng(seed)
    f = rng.random((nv, nx)) + 0.05
    dv = 0.25
    vmax = (nv - 1) // 2 * dv
    u = rng.uniform(-vmax, vmax, nx)
    return f, u, dv


def test_mass_conserved_per_cell():
    f, u, dv = _random_case(1)
    fd = O.drag_1d(f, u, 1.3, 0.05, dv)
    fk = O.diffuse_1d(f, 0.02, 0.05, dv)
    np.testing.assert_allclose(fd.sum(axis=0), f.sum(axis=0), rtol=1e-14, atol=0)
    np.testing.assert_allclose(fk.sum(axis=0), f.sum(axis=0), rtol=1e-14, atol=0)


def check_first_moment_drag(mod=O):
    """Identity: with |u| <= V_max the wall terms vanish and one drag sub-step gives
    M1' = M1 - (dt/tau_p)(M1 - u M0) exactly (M_k = sum_j v_j^k f_j)."""
    f, u, dv = _random_case(2)
    tau_p, dt = 1.7, 0.05
    v = O.velocities(f.shape[0], dv)
    fd = mod.drag_1d(f, u, tau_p, dt, dv)
    M0, M1 = f.sum(0), (v[:, None] * f).sum(0)
    want = M1 - (dt / tau_p) * (M1 - u * M0)
    np.testing.assert_allclose((v[:, None] * fd).sum(0), want, rtol=1e-12, atol=1e-12)


def test_first_moment_drag():
    check_first_moment_drag()


def test_second_moment_drag():
    """Identity: M2' = M2 - (2 dt/tau_p)(M2 - u M1) + (dt dv/tau_p) sum_j f_j |v_j - u|.
    The last term is the upwind numerical diffusion (Section 2, kappa_num)."""
    f, u, dv = _random_case(3)
    tau_p, dt = 1.7, 0.05
    v = O.velocities(f.shape[0], dv)
    fd = O.drag_1d(f, u, tau_p, dt, dv)
    M1, M2 = (v[:, None] * f).sum(0), (v[:, None] ** 2 * f).sum(0)
    want = M2 - (2 * dt / tau_p) * (M2 - u * M1) \
        + (dt * dv / tau_p) * (f * np.abs(v[:, None] - u[None, :])).sum(0)
    np.testing.assert_allclose((v[:, None] ** 2 * fd).sum(0), want, rtol=1e-12, atol=1e-12)


def check_diffusion_moments(mod=O):
    """Identities of the zero-flux discrete Laplacian: M1' = M1 - (kappa dt/dv)(f_J - f_-J),
    M2' = M2 + 2 kappa dt M0 - N_v kappa dt (f_J + f_-J)."""
    f, _, dv = _random_case(4)
    nv = f.shape[0]
    kappa, dt = 0.03, 0.05
    v = O.velocities(nv, dv)
    fk = mod.diffuse_1d(f, kappa, dt, dv)
    M0, M1, M2 = f.sum(0), (v[:, None] * f).sum(0), (v[:, None] ** 2 * f).sum(0)
    w1 = M1 - (kappa * dt / dv) * (f[-1] - f[0])
    w2 = M2 + 2 * kappa * dt * M0 - nv * kappa * dt * (f[-1] + f[0])
    np.testing.assert_allclose((v[:, None] * fk).sum(0), w1, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose((v[:, None] ** 2 * fk).sum(0), w2, rtol=1e-12, atol=1e-12)


def test_diffusion_moments():
    check_diffusion_moments()


def test_diffusion_matches_cosine_eigenmodes():
    """The zero-flux discrete Laplacian on N_v points has eigenvectors
    cos(pi k (i + 1/2)/N_v) and one explicit step multiplies mode k by
    1 - 4 r sin^2(pi k / (2 N_v)), r = kappa dt / dv^2 (textbook result)."""
    nv, dv, kappa, dt, n = 21, 0.3, 0.02, 0.4, 60
    r = kappa * dt / dv ** 2
    rng = np.random.default_rng(5)
    f0 = rng.random(nv)
    i = np.arange(nv)
    E = np.array([np.cos(np.pi * k * (i + 0.5) / nv) for k in range(nv)])
    coef = E @ f0 / (E * E).sum(axis=1)
    lam = 1 - 4 * r * np.sin(np.pi * np.arange(nv) / (2 * nv)) ** 2
    want = (coef * lam ** n) @ E
    f = f0.reshape(nv, 1)
    for _ in range(n):
        f = O.diffuse_1d(f, kappa, dt, dv)
    np.testing.assert_allclose(f[:, 0], want, rtol=1e-12, atol=1e-13)


def test_gaussian_spreading():
    """Pure diffusion spreads a centred packet as sigma^2(t) = sigma_0^2 + 2 kappa t
    (continuous Fokker-Planck; exact on the lattice while the walls hold no mass)."""
    nv, dv, kappa, dt, n = 201, 0.05, 0.01, 0.05, 400
    v = O.velocities(nv, dv)
    s0 = 0.3
    f = np.exp(-0.5 * (v / s0) ** 2).reshape(nv, 1)
    var0 = (v ** 2 * f[:, 0]).sum() / f.sum()
    for _ in range(n):
        f = O.diffuse_1d(f, kappa, dt, dv)
    var = (v ** 2 * f[:, 0]).sum() / f.sum()
    assert abs(var - (var0 + 2 * kappa * n * dt)) < 1e-10


# ---------------------------------------------------------------------------------------------
# Relaxation under Stokes drag (Eq. stokes_drag)
# ---------------------------------------------------------------------------------------------
def check_relaxation_to_rest(mod=O):
    """With u = 0 and no diffusion, <v> decays like exp(-t/tau_p) (to O(dt/tau_p))."""
    nx, nv, dv, tau_p, dt = 8, 41, 0.1, 1.0, 0.01
    v = O.velocities(nv, dv)
    g = np.exp(-0.5 * ((v - 0.8) / 0.2) ** 2)
    f = np.repeat(g[:, None], nx, axis=1)
    u = np.zeros(nx)
    m_prev = None
    n = 100  # t = tau_p
    for _ in range(n):
        f = mod.step_1d(f, u, tau_p, 0.0, dt, dv)
    m = (v[:, None] * f).sum(0) / f.sum(0)
    m0 = (v * g).sum() / g.sum()
    want = m0 * math.exp(-n * dt / tau_p)
    np.testing.assert_allclose(m, want, rtol=2 * dt / tau_p)
    del m_prev


def test_relaxation_to_rest():
    check_relaxation_to_rest()


def test_relaxation_toward_constant_flow():
    """Particles in a uniform constant flow u0 acquire <v> -> u0 (Eq. stokes_drag)."""
    nx, nv, dv, tau_p, dt, u0 = 4, 41, 0.1, 0.5, 0.01, 0.7
    v = O.velocities(nv, dv)
    f = np.repeat(np.exp(-0.5 * (v / 0.2) ** 2)[:, None], nx, axis=1)
    u = np.full(nx, u0)
    for _ in range(2000):
        f = O.step_1d(f, u, tau_p, 1e-3, dt, dv)
    m = (v[:, None] * f).sum(0) / f.sum(0)
    np.testing.assert_allclose(m, u0, rtol=1e-6)


def test_stationary_velocity_variance():
    """Stokes drag plus diffusion is an Ornstein-Uhlenbeck velocity process whose stationary
    variance is kappa tau_p (Sec. 3.2, v_d^2 ~ kappa tau_p).  On the lattice the upwind
    numerical diffusion dv |a| / 2 adds (dv/2)<|v|> (identity of test_second_moment_drag)."""
    nx, nv, dv, tau_p, kappa, dt = 2, 101, 0.01, 1.0, 0.01, 0.002
    v = O.velocities(nv, dv)
    f = np.repeat(np.exp(-0.5 * (v / 0.05) ** 2)[:, None], nx, axis=1)
    u = np.zeros(nx)
    for _ in range(5000):  # t = 10 tau_p
        f = O.step_1d(f, u, tau_p, kappa, dt, dv)
    col = f[:, 0] / f[:, 0].sum()
    var = (v ** 2 * col).sum()
    mabs = (np.abs(v) * col).sum()
    assert abs(var - (kappa * tau_p + 0.5 * dv * mabs)) < 0.01 * var
    assert abs(var - kappa * tau_p) < 0.08 * kappa * tau_p


def test_positivity_under_cfl():
    """The upwind and Laplacian steps are positive when Eq. (cfl) and Eq. (stabLapl) hold."""
    rng = np.random.default_rng(6)
    nx, nv, dv, tau_p = 64, 33, 0.2, 1.0
    vmax = 16 * dv
    f = rng.random((nv, nx)) ** 8
    u = rng.uniform(-vmax, vmax, nx)
    dt = 0.95 / (2 * vmax / tau_p / dv)  # CFL 0.95 at the worst |v - u| = 2 V_max
    kappa = 0.49 * dv * dv / dt
    for _ in range(50):
        f = O.step_1d(f, u, tau_p, kappa, dt, dv)
        assert f.min() >= -1e-14 * f.max()


# ---------------------------------------------------------------------------------------------
# Flow and moments
# ---------------------------------------------------------------------------------------------
def check_single_modes(mod=O):
    nx = 16
    x = 2 * math.pi * np.arange(nx) / nx
    k = np.array([3])
    np.testing.assert_allclose(mod.flow1d_u(np.array([1.0, 0.0]), k, nx), np.cos(3 * x),
                               atol=1e-14)
    np.testing.assert_allclose(mod.flow1d_u(np.array([0.0, 1.0]), k, nx), np.sin(3 * x),
                               atol=1e-14)


def test_flow_single_modes():
    """Eq. (u1d): A cos(2 pi k x/L) + B sin(2 pi k x/L) on x_i = i L / N_x."""
    check_single_modes()


def test_ou_statistics():
    """The exact OU update keeps the stationary variance sigma^2 and has lag-one
    autocorrelation exp(-dt/tau_f) (Eq. A1d)."""
    rng = np.random.default_rng(7)
    n, dt, tau_f, sigma = 200000, 0.1, 1.0, 0.7
    a = np.empty(n)
    a[0] = sigma * rng.standard_normal()
    xi = rng.standard_normal(n)
    for t in range(1, n):
        a[t] = O.ou_advance(np.array([a[t - 1]]), xi[t:t + 1], dt, tau_f, sigma)[0]
    assert abs(a.var() / sigma ** 2 - 1) < 0.05
    rho1 = np.corrcoef(a[:-1], a[1:])[0, 1]
    assert abs(rho1 - math.exp(-dt / tau_f)) < 0.01


def test_moments_of_known_distributions():
    nx, nv, dx, dv = 3, 9, 0.5, 0.25
    v = O.velocities(nv, dv)
    f = np.zeros((nv, nx))
    f[6, 0] = 2.0                       # all mass at v = 0.5
    f[1, 1], f[7, 1] = 1.0, 1.0         # two-point distribution at v = -0.75, +0.75
    rho, mv, mv2, glob = O.moments_1d(f, dx, dv)
    assert rho[0] == 2.0 * dv and mv[0] == v[6] and mv2[0] == v[6] ** 2
    assert mv[1] == 0.0 and mv2[1] == 0.75 ** 2
    assert rho[2] == 0.0 and mv[2] == 0.0 and mv2[2] == 0.0
    assert glob[0] == 4.0 * dx * dv
    assert glob[1] == pytest.approx(2.0 * 0.5 * dx * dv)
