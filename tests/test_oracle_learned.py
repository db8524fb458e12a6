"""Pins of the learned-closure oracle (oracle/learned.py): the restriction keeps mass, the
features are what they say, a zero network gives the plain coarse step bit for bit, the
corrected step keeps mass for any weights, and the hand-written gradients agree with central
finite differences of the loss."""
import math

import numpy as np
import pytest

from oracle import lattice as O
from oracle import learned as Lr
from paper_1508_02899_gb300 import inputs as I


def test_restriction_keeps_mass_and_centres():
    R = Lr.restrict_matrix(33)
    assert R.shape == (9, 33)
    # each fine cell's weights sum to one coarse cell width: sum_k R[k, j] * 4 = 1
    np.testing.assert_allclose(R.sum(axis=0) * 4, 1.0, rtol=0, atol=1e-15)
    rng = np.random.default_rng(2)
    ff = rng.random((33, 33, 3, 4))
    fc = Lr.restrict(ff)
    dvf = 0.1
    np.testing.assert_allclose(fc.sum(axis=(0, 1)) * (4 * dvf) ** 2, ff.sum(axis=(0, 1)) * dvf**2,
                               rtol=1e-14)
    # interior coarse cells of a state constant in v stay at that constant
    fc1 = Lr.restrict(np.ones((33, 33, 1, 1)))
    np.testing.assert_allclose(fc1[1:-1, 1:-1], 1.0, rtol=1e-15)
    # a fine delta at 4k lands in coarse cell k alone, with 1/16 of its value
    d = np.zeros((33, 33, 1, 1))
    d[16 + 8, 16 - 4] = 1.0
    fcd = Lr.restrict(d)
    assert fcd[4 + 2, 4 - 1, 0, 0] == 1.0 / 16 and fcd.sum() == 1.0 / 16


def test_velocity_gradients_match_the_centred_difference_of_a_sine():
    nx = ny = 16
    dx = 2 * math.pi / nx
    y = (np.arange(ny) * dx)[:, None] * np.ones((1, nx))
    x = np.ones((ny, 1)) * (np.arange(nx) * dx)[None, :]
    ux, uy = np.sin(y), np.cos(2 * x)
    g = Lr.velocity_gradients(ux, uy, dx)
    np.testing.assert_allclose(g[0], 0.0, atol=1e-15)
    np.testing.assert_allclose(g[1], np.cos(y) * math.sin(dx) / dx, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(g[2], -np.sin(2 * x) * math.sin(2 * dx) / dx, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(g[3], 0.0, atol=1e-15)


def _case(seed=0, nv=5, ny=6, nx=7, nsteps=2):
    rng = np.random.default_rng(seed)
    L = 2 * math.pi
    tau_p, kappa = 1.0 * L, 2e-3
    dt = I.choose_dt(2, nx, L, nv, tau_p, kappa)
    dx = L / nx
    dv = dx / dt
    f0 = rng.random((nv, nv, ny, nx)) + 0.1
    fl = I.flow2d_inputs(seed, nsteps, nx, ny, dx, kmax=2)
    flows, phi = [], fl.phi0.copy()
    for n in range(nsteps):
        flows.append(O.flow2d_u(fl.a, fl.kvec, phi, nx, ny, dx))
        phi = O.phase_advance(phi, fl.noise[n], dt, fl.tau_f)
    kw = dict(tau_p=tau_p, kappa=kappa, dt=dt, dv=dv, dx=dx)
    return f0, flows, kw


def test_features_are_the_normalised_neighbourhood():
    f0, flows, kw = _case()
    fs = O.stream_2d(f0)
    X, rho = Lr.features(fs, *flows[0], **{k: kw[k] for k in ("tau_p", "dt", "dv", "dx")})
    np.testing.assert_allclose(rho, fs.sum(axis=(0, 1)), rtol=1e-15)
    np.testing.assert_allclose(X[..., 4].sum(axis=(0, 1)), 1.0, rtol=1e-14)   # centre cell
    np.testing.assert_array_equal(X[0, :, ..., 0], 0.0)                         # below the box
    np.testing.assert_allclose(X[2, 3, ..., 8], fs[3, 4] / rho, rtol=1e-15)     # (dy, dx) = (1, 1)
    assert np.all(X[..., 15] == 1.0)


def test_zero_network_gives_the_plain_step_exactly():
    f0, flows, kw = _case()
    out = Lr.learned_step_2d(f0, *flows[0], Lr.zero_weights(), **kw)
    want = O.step_2d(f0, *flows[0], kw["tau_p"], kw["kappa"], kw["dt"], kw["dv"])
    np.testing.assert_array_equal(out, want)


def test_corrected_step_keeps_mass_for_any_weights():
    f0, flows, kw = _case(seed=4)
    W = Lr.init_weights(7, scale=0.3)
    out = Lr.learned_step_2d(f0, *flows[0], W, **kw)
    plain = O.step_2d(f0, *flows[0], kw["tau_p"], kw["kappa"], kw["dt"], kw["dv"])
    assert np.max(np.abs(out - plain)) > 1e-3           # the correction does something
    np.testing.assert_allclose(out.sum(), f0.sum(), rtol=1e-13)
    np.testing.assert_allclose(out.sum(axis=(0, 1)).sum(), plain.sum(), rtol=1e-13)


def test_mlp_backward_matches_finite_differences():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((11, Lr.NF))
    W = Lr.init_weights(5)
    for k in W:
        W[k] = W[k] + 0.1 * rng.standard_normal(W[k].shape)
    dy = rng.standard_normal((11, Lr.NO))
    y, cache = Lr.mlp_forward(X, W, 0.05)
    g, dX = Lr.mlp_backward(dy, W, cache)
    h = 1e-6
    for k in ("W1", "b2", "W3"):
        idx = tuple(rng.integers(0, s) for s in W[k].shape)
        Wp = {q: v.copy() for q, v in W.items()}
        Wm = {q: v.copy() for q, v in W.items()}
        Wp[k][idx] += h
        Wm[k][idx] -= h
        fd = ((Lr.mlp_forward(X, Wp, 0.05)[0] - Lr.mlp_forward(X, Wm, 0.05)[0]) * dy).sum() / (2 * h)
        assert fd == pytest.approx(g[k][idx], rel=1e-6, abs=1e-9)
    Xp, Xm = X.copy(), X.copy()
    Xp[2, 5] += h
    Xm[2, 5] -= h
    fd = ((Lr.mlp_forward(Xp, W, 0.05)[0] - Lr.mlp_forward(Xm, W, 0.05)[0]) * dy).sum() / (2 * h)
    assert fd == pytest.approx(dX[2, 5], rel=1e-6, abs=1e-9)


def test_rollout_gradient_matches_finite_differences():
    f0, flows, kw = _case(seed=6, nsteps=3)
    W = Lr.init_weights(9, scale=0.5)
    rng = np.random.default_rng(1)
    target = Lr.rollout(f0, Lr.zero_weights(), 3, flows, **kw) * (1 + 0.01 * rng.standard_normal(f0.shape))
    beta = 0.5
    L0, g = Lr.rollout_grad(f0, W, 3, flows, target, rho_weight=beta, **kw)
    h = 1e-6
    checked = 0
    for k, idxs in (("W1", [(0, 3), (4, 10), (13, 60), (15, 1)]), ("b1", [(5,), (40,)]),
                    ("W2", [(3, 7), (60, 2)]), ("b2", [(8,)]), ("W3", [(10, 0), (33, 1)]),
                    ("b3", [(0,), (1,)])):
        for idx in idxs:
            Wp = {q: v.copy() for q, v in W.items()}
            Wm = {q: v.copy() for q, v in W.items()}
            Wp[k][idx] += h
            Wm[k][idx] -= h
            fd = (Lr.loss(f0, Wp, 3, flows, target, beta, **kw)
                  - Lr.loss(f0, Wm, 3, flows, target, beta, **kw)) / (2 * h)
            scale = max(abs(fd), 1e-3 * np.abs(g[k]).max())
            assert abs(fd - g[k][idx]) <= 1e-5 * scale, (k, idx, fd, g[k][idx])
            checked += 1
    assert checked == 13


def test_corrections_are_the_step_difference_on_each_face():
    # the step with corrections minus the plain step is minus the divergence of (Gx, Gy),
    # diffused: check it against the corrections computed on their own
    f0, flows, kw = _case(seed=12)
    W = Lr.init_weights(4, scale=0.5)
    Gx, Gy = Lr.corrections(f0, *flows[0], W, **{k: kw[k] for k in ("tau_p", "dt", "dv", "dx")})
    assert np.all(Gx[:, -1] == 0) and np.all(Gy[-1] == 0)
    fs = O.stream_2d(f0)
    div = np.zeros_like(fs)
    div[:, :] += Gx
    div[:, 1:] -= Gx[:, :-1]
    div[:, :] += Gy
    div[1:] -= Gy[:-1]
    want = O.diffuse_2d(O.drag_2d(fs, *flows[0], kw["tau_p"], kw["dt"], kw["dv"]) - div,
                        kw["kappa"], kw["dt"], kw["dv"])
    got = Lr.learned_step_2d(f0, *flows[0], W, **kw)
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-15 * np.abs(want).max())


def test_outputs_stay_inside_their_bounds():
    # large random weights drive the outputs to their bounds: never more anti-diffusion than
    # THETA times the face's upwind numerical diffusivity, never more diffusion than Y_MAX
    rng = np.random.default_rng(8)
    X = rng.standard_normal((4000, Lr.NF))
    X[:, 13:15] = rng.uniform(-0.6, 0.6, (4000, 2))
    W = Lr.init_weights(2, scale=20.0)
    y, _ = Lr.mlp_forward(X, W, 0.05)
    ca = np.abs(X[:, 13:15] - 0.025)
    assert np.all(y <= Lr.THETA * ca * (1 - ca) / 2 + 1e-15)
    assert np.all(y >= -Lr.Y_MAX)
    assert y.max() > 0.5 * (Lr.THETA * ca * (1 - ca) / 2).max() and y.min() < -0.2
