"""Pins of the 2D FP64 oracle and of the synthetic 2D flow (no GPU)."""
import math
import os

import numpy as np

from oracle import lattice as O
from paper_1508_02899_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def check_golden_2d(mod=O):
    """Hand-derived unsplit step (fixture tiny_nv3_2d.txt, derivation inside)."""
    f = np.zeros((3, 3, 1, 1))
    f[1, 2, 0, 0] = 1.0  # [jy = 0, jx = +1]
    want = np.zeros((3, 3))
    with open(os.path.join(GOLDEN, "tiny_nv3_2d.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                jx, jy, val = line.split()
                want[int(jy) + 1, int(jx) + 1] = float(val)
    z = np.zeros((1, 1))
    got = mod.step_2d(f, z, z, 2.0, 0.25, 0.5, 1.0)[:, :, 0, 0]
    assert np.array_equal(got, want), (got, want)


def test_golden_tiny_step():
    check_golden_2d()


def check_unit_mass_moves(mod=O):
    """Section 2, d = 2: mass in velocity cell (jx, jy) moves by (jx, jy) grid points."""
    nx, ny, nv = 7, 6, 5
    for jy in range(nv):
        for jx in range(nv):
            f = np.zeros((nv, nv, ny, nx))
            f[jy, jx, 2, 3] = 1.0
            out = mod.stream_2d(f)
            assert out[jy, jx, (2 + jy - 2) % ny, (3 + jx - 2) % nx] == 1.0


def test_unit_mass_moves():
    check_unit_mass_moves()


def test_free_streaming_period():
    rng = np.random.default_rng(0)
    nx, ny, nv = 6, 4, 5
    f0 = rng.random((nv, nv, ny, nx))
    f = f0.copy()
    z = np.zeros((ny, nx))
    for _ in range(12):  # lcm(6, 4)
        f = O.step_2d(f, z, z, math.inf, 0.0, 0.1, 0.5)
    assert np.array_equal(f, f0)


def _case(seed, nx=6, ny=5, nv=9):
    rng = np.random.default_rng(seed)
    f = rng.random((nv, nv, ny, nx)) + 0.05
    dv = 0.25
    vmax = (nv - 1) // 2 * dv
    ux = rng.uniform(-vmax, vmax, (ny, nx))
    uy = rng.uniform(-vmax, vmax, (ny, nx))
    return f, ux, uy, dv


def test_mass_conserved():
    f, ux, uy, dv = _case(1)
    for g in (O.drag_2d(f, ux, uy, 1.1, 0.03, dv), O.diffuse_2d(f, 0.02, 0.03, dv)):
        np.testing.assert_allclose(g.sum(axis=(0, 1)), f.sum(axis=(0, 1)), rtol=1e-14)


def check_first_moments_2d(mod=O):
    """Each velocity component obeys the 1D identity M1' = M1 - (dt/tau_p)(M1 - u M0)."""
    f, ux, uy, dv = _case(2)
    tau_p, dt = 1.1, 0.03
    v = O.velocities(f.shape[0], dv)
    g = mod.drag_2d(f, ux, uy, tau_p, dt, dv)
    M0 = f.sum(axis=(0, 1))
    for comp, u in ((1, ux), (0, uy)):
        w = v[None, :, None, None] if comp == 1 else v[:, None, None, None]
        M1 = (w * f).sum(axis=(0, 1))
        np.testing.assert_allclose((w * g).sum(axis=(0, 1)),
                                   M1 - (dt / tau_p) * (M1 - u * M0), rtol=1e-12, atol=1e-12)


def test_first_moments():
    check_first_moments_2d()


def test_reduces_to_1d():
    """All mass on the v_y = 0 row, u_y = 0, kappa = 0: the y fluxes vanish identically and
    every y row evolves as the 1D scheme."""
    rng = np.random.default_rng(3)
    nx, ny, nv, dv, dt, tau_p = 10, 3, 9, 0.3, 0.05, 0.8
    J = (nv - 1) // 2
    f1 = rng.random((ny, nv, nx))
    f = np.zeros((nv, nv, ny, nx))
    for y in range(ny):
        f[J, :, y, :] = f1[y]
    ux = rng.uniform(-1, 1, (ny, nx))
    g = O.step_2d(f, ux, np.zeros((ny, nx)), tau_p, 0.0, dt, dv)
    for y in range(ny):
        # 2D streaming also moves row y by jy = 0, i.e. not at all
        want = O.step_1d(f1[y], ux[y], tau_p, 0.0, dt, dv)
        np.testing.assert_allclose(g[J, :, y, :], want, rtol=1e-15, atol=1e-16)
    mask = np.ones(nv, bool)
    mask[J] = False
    assert np.all(g[mask] == 0.0)


def test_xy_symmetry():
    """Swapping the roles of x and y (transpose f, swap u components) transposes the result."""
    f, ux, uy, dv = _case(4, nx=5, ny=5)
    g = O.step_2d(f, ux, uy, 0.9, 0.01, 0.03, dv)
    gt = O.step_2d(f.transpose(1, 0, 3, 2).copy(), uy.T.copy(), ux.T.copy(), 0.9, 0.01, 0.03, dv)
    np.testing.assert_allclose(gt.transpose(1, 0, 3, 2), g, rtol=1e-13, atol=1e-15)


def test_gaussian_spreading_each_component():
    """Five-point Laplacian: each velocity component's variance grows by 2 kappa dt per step
    while the walls hold no mass (continuous result sigma^2 = sigma_0^2 + 2 kappa t)."""
    nv, dv, kappa, dt, n = 61, 0.1, 0.01, 0.05, 100
    v = O.velocities(nv, dv)
    g = np.exp(-0.5 * (v / 0.3) ** 2)
    f = (g[:, None] * g[None, :])[:, :, None, None].copy()
    var0 = (v ** 2 * g).sum() / g.sum()
    for _ in range(n):
        f = O.diffuse_2d(f, kappa, dt, dv)
    c = f[:, :, 0, 0]
    vx = (v[None, :] ** 2 * c).sum() / c.sum()
    vy = (v[:, None] ** 2 * c).sum() / c.sum()
    want = var0 + 2 * kappa * n * dt
    assert abs(vx - want) < 1e-10 and abs(vy - want) < 1e-10


def test_relaxation_toward_constant_flow():
    nv, dv, tau_p, dt = 21, 0.1, 0.5, 0.01
    v = O.velocities(nv, dv)
    g = np.exp(-0.5 * (v / 0.2) ** 2)
    f = (g[:, None] * g[None, :])[:, :, None, None].copy()
    ux, uy = np.full((1, 1), 0.4), np.full((1, 1), -0.3)
    for _ in range(1500):
        f = O.step_2d(f, ux, uy, tau_p, 1e-3, dt, dv)
    c = f[:, :, 0, 0]
    assert abs((v[None, :] * c).sum() / c.sum() - 0.4) < 1e-6
    assert abs((v[:, None] * c).sum() / c.sum() + 0.3) < 1e-6


def check_moments_2d_known(mod=O):
    """Per-cell and global 2D moments of hand-built velocity distributions (Sec. 3.2: the mass
    of a cell is f dx^2 dv^2; Sec. 4.2: rho is the sum over both velocity components).

    Cell (y, x) = (0, 0): all mass 2 in velocity cell (jx, jy) = (+3, -1): rho = 2 dv^2, the
    mean velocity is that cell's velocity, <|v|^2> its squared norm.  (0, 1): two points
    (+2, -1) and (-2, +1) of mass 1: mean 0, <|v|^2> = 5 dv^2.  (1, 0): empty: zeros.  (1, 1):
    mass 1 at (+3, 0) and 3 at (0, -1): <v> = (3/4, -3/4) dv, <|v|^2> = (9 + 3)/4 dv^2, which
    tells v_x from v_y and catches a dropped component of |v|^2.  dx and dv are powers of two,
    so every expected value is exact in binary."""
    nv, dx, dv = 9, 0.5, 0.25
    J = (nv - 1) // 2
    f = np.zeros((nv, nv, 2, 2))

    def put(y, x, jx, jy, m):
        f[jy + J, jx + J, y, x] += m

    put(0, 0, 3, -1, 2.0)
    put(0, 1, 2, -1, 1.0)
    put(0, 1, -2, 1, 1.0)
    put(1, 1, 3, 0, 1.0)
    put(1, 1, 0, -1, 3.0)
    rho, mvx, mvy, mv2, glob = mod.moments_2d(f, dx, dv)
    assert rho.shape == (2, 2)
    assert rho[0, 0] == 2.0 * dv * dv and rho[0, 1] == 2.0 * dv * dv
    assert rho[1, 0] == 0.0 and rho[1, 1] == 4.0 * dv * dv
    assert mvx[0, 0] == 3 * dv and mvy[0, 0] == -1 * dv and mv2[0, 0] == 10 * dv * dv
    assert mvx[0, 1] == 0.0 and mvy[0, 1] == 0.0 and mv2[0, 1] == 5 * dv * dv
    assert mvx[1, 0] == 0.0 and mvy[1, 0] == 0.0 and mv2[1, 0] == 0.0
    assert mvx[1, 1] == 0.75 * dv and mvy[1, 1] == -0.75 * dv and mv2[1, 1] == 3 * dv * dv
    w = dx * dx * dv * dv
    # M = 2 + 2 + 4; P_x = 2(3) + (2 - 2) + 1(3) = 9 dv; P_y = 2(-1) + (-1 + 1) + 3(-1) = -5 dv;
    # E = 2(10) + 5 + 5 + (9 + 3) = 42 dv^2
    assert glob[0] == 8.0 * w
    assert glob[1] == 9.0 * dv * w
    assert glob[2] == -5.0 * dv * w
    assert glob[3] == 42.0 * dv * dv * w


def test_moments_2d_known():
    check_moments_2d_known()


def check_moments_2d_reduce_to_1d(mod=O):
    """A 2D state supported on the row jy = 0 (v_y = 0) has the 1D moments of that row for
    rho / dv, <v_x> and <|v|^2>, zero <v_y>; the same state transposed in (jx, jy) swaps
    <v_x> and <v_y> (x <-> y symmetry of the velocity lattice).  The 1D moments are pinned by
    test_oracle_1d.test_moments_of_known_distributions."""
    rng = np.random.default_rng(11)
    nv, ny, nx, dx, dv = 7, 3, 4, 0.3, 0.7
    J = (nv - 1) // 2
    row = rng.random((nv, ny * nx))
    row[:, 5] = 0.0  # one empty cell
    f = np.zeros((nv, nv, ny, nx))
    f[J] = row.reshape(nv, ny, nx)
    rho, mvx, mvy, mv2, glob = mod.moments_2d(f, dx, dv)
    r1, m1, m21, g1 = mod.moments_1d(row, dx, dv)
    np.testing.assert_allclose(rho.ravel(), r1 * dv, rtol=1e-15, atol=0)
    np.testing.assert_allclose(mvx.ravel(), m1, rtol=1e-14, atol=1e-300)
    np.testing.assert_allclose(mv2.ravel(), m21, rtol=1e-14, atol=1e-300)
    assert np.all(mvy == 0.0)
    np.testing.assert_allclose(glob[[0, 1, 3]], np.asarray(g1) * dx * dv, rtol=1e-14)
    assert glob[2] == 0.0
    ft = np.ascontiguousarray(np.swapaxes(f, 0, 1))
    rt, mxt, myt, m2t, gt = mod.moments_2d(ft, dx, dv)
    np.testing.assert_array_equal(rt, rho)
    np.testing.assert_allclose(myt, mvx, rtol=1e-15, atol=0)
    np.testing.assert_allclose(mxt, mvy, rtol=1e-15, atol=0)
    np.testing.assert_allclose(m2t, mv2, rtol=1e-15, atol=0)
    np.testing.assert_allclose(gt[[0, 2, 1, 3]], glob, rtol=1e-15)


def test_moments_2d_reduce_to_1d():
    check_moments_2d_reduce_to_1d()


def check_flow2d_is_perp_gradient(mod=O):
    """u = (d_y psi, -d_x psi) and div u = 0, checked with spectral derivatives of psi."""
    nx = ny = 64
    dx = 2 * math.pi / nx
    fl = I.flow2d_inputs(11, 1, nx, ny, dx, kmax=5)
    ux, uy = mod.flow2d_u(fl.a, fl.kvec, fl.phi0, nx, ny, dx)
    ii = np.arange(nx)[None, :]
    ll = np.arange(ny)[:, None]
    psi = sum(fl.a[m] * np.cos(2 * math.pi * (fl.kvec[m, 0] * ii / nx + fl.kvec[m, 1] * ll / ny)
                               + fl.phi0[m]) for m in range(len(fl.a)))
    kx = np.fft.fftfreq(nx, d=dx) * 2 * math.pi
    ky = np.fft.fftfreq(ny, d=dx) * 2 * math.pi
    P = np.fft.fft2(psi)
    dpsi_dx = np.real(np.fft.ifft2(1j * kx[None, :] * P))
    dpsi_dy = np.real(np.fft.ifft2(1j * ky[:, None] * P))
    np.testing.assert_allclose(ux, dpsi_dy, atol=1e-10)
    np.testing.assert_allclose(uy, -dpsi_dx, atol=1e-10)
    div = np.real(np.fft.ifft2(1j * kx[None, :] * np.fft.fft2(ux) + 1j * ky[:, None] * np.fft.fft2(uy)))
    assert np.abs(div).max() < 1e-10


def test_flow2d_is_perp_gradient():
    check_flow2d_is_perp_gradient()


def test_flow2d_rms_and_spectrum():
    """Recipe check: u_rms = 1 per component on average over phases; |a_k| ~ |k|^-3."""
    nx = ny = 64
    dx = 2 * math.pi / nx
    acc = np.zeros(2)
    for s in range(20):
        fl = I.flow2d_inputs(100 + s, 1, nx, ny, dx)
        ux, uy = O.flow2d_u(fl.a, fl.kvec, fl.phi0, nx, ny, dx)
        acc += [np.mean(ux ** 2), np.mean(uy ** 2)]
    acc /= 20
    assert abs(acc.mean() - 1.0) < 0.15
    kk = np.sqrt((fl.kvec ** 2).sum(1))
    np.testing.assert_allclose(fl.a * kk ** 3, (fl.a * kk ** 3)[0], rtol=1e-12)


def test_phase_walk_decorrelates_like_exp():
    """<cos(phi(t) - phi(0))> = exp(-t/tau_f) for the random-walk phase."""
    rng = np.random.default_rng(9)
    n_real, n_steps, dt, tau_f = 20000, 50, 0.02, 1.0
    phi = np.zeros(n_real)
    for _ in range(n_steps):
        phi = O.phase_advance(phi, rng.standard_normal(n_real), dt, tau_f)
    assert abs(np.mean(np.cos(phi)) - math.exp(-n_steps * dt / tau_f)) < 0.02


def test_cellular_flow_is_the_orthogonal_gradient_of_its_stream_function():
    """inputs.cellular_flow against centred differences of psi = U sin(pi(x+y)/L) sin(pi(x-y)/L)
    (fourth-order stencil) and a spectral divergence of zero."""
    import math
    from paper_1508_02899_gb300 import inputs as I
    L, n, U = 2 * math.pi, 128, 1.3
    ux, uy = I.cellular_flow(n, n, L, U)
    dx = L / n
    x = np.arange(n) * dx
    X, Y = np.meshgrid(x, x)
    psi = U * np.sin(np.pi * (X + Y) / L) * np.sin(np.pi * (X - Y) / L)

    def d(f, axis):
        return (8 * (np.roll(f, -1, axis) - np.roll(f, 1, axis))
                - (np.roll(f, -2, axis) - np.roll(f, 2, axis))) / (12 * dx)
    np.testing.assert_allclose(ux, d(psi, 0), atol=1e-6)
    np.testing.assert_allclose(uy, -d(psi, 1), atol=1e-6)
    kx = np.fft.fftfreq(n, d=dx) * 2 * np.pi
    div = np.fft.ifft2(1j * kx[None, :] * np.fft.fft2(ux) + 1j * kx[:, None] * np.fft.fft2(uy))
    assert np.abs(div).max() < 1e-12
