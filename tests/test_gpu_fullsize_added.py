"""Full-size checks, in the launch configuration bench.py times, of the two rows this library adds:
16-bit storage at 1024^2 x 33^2 and the learned closure at 2048^2 x 9^2.  The oracle recomputes
sampled outputs one by one from the same seeded inputs (it never reads a value the library
produced): a cell's whole velocity column after one 16-bit step, and the correction fluxes of
sampled phase-space cells.  The 16-bit tolerances are those of test_gpu_2d_half.py; the learned
closure's are per output, from the BF16 network's rounding (bf16_bound.py).
"""
import math

import numpy as np
import pytest
import torch

from bf16_bound import output_error_bound
from oracle import lattice as O
from oracle import learned as Lr
from oracle import storage16 as S16
from paper_1508_02899_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L = 2 * math.pi
STEP = {"f16": 2.0**-10, "bf16": 2.0**-7}
SIG = {"f16": 10, "bf16": 7}
TDT = {"f16": torch.float16, "bf16": torch.bfloat16}


def seeded_state(n, nv, dx, dv, seed, device="cuda"):
    """Gaussian velocity column (sigma = 0.3 V_max) times a seeded spatial modulation, on device."""
    J = (nv - 1) // 2
    col = I.gaussian_column(1, nv, dx, dv, 0.3 * J * dv)
    mod = 1 + 0.3 * np.random.default_rng(seed).random((n, n))
    c2 = torch.tensor(np.outer(col, col), dtype=torch.float32, device=device)
    m = torch.tensor(mod, dtype=torch.float32, device=device)
    return c2[:, :, None, None] * m[None, None]


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_16bit_full_size_sampled_columns(lat, fmt):
    n, nv = 1024, 33
    J = (nv - 1) // 2
    tau_p, kappa = L, 1e-3
    dt = I.choose_dt(2, n, L, nv, tau_p, kappa)
    dx = L / n
    dv = dx / dt
    f = seeded_state(n, nv, dx, dv, 5)
    # only the bits each line's scale holds exactly, so that encoding leaves no residual
    mx = f.abs().amax(dim=3, keepdim=True)
    q = torch.exp2(torch.floor(torch.log2(mx)) - SIG[fmt])
    fq = torch.round(f / q) * q
    del f, mx, q
    fl = I.flow2d_inputs(1234 + 11, 2, n, n, dx)
    lt = lat.Lattice(torch.zeros(fq.shape, dtype=TDT[fmt], device="cuda"), d=2, nx=n, ny=n, nv=nv,
                     L=L, tau_p=tau_p, kappa=kappa, dt=dt)
    lt.set_launch(kernel=5, blocks_per_sm=3)
    lt.encode(fq)
    lt.set_flow_modes_2d(fl.kvec, fl.a, fl.phi0, fl.tau_f)
    lt.set_noise(fl.noise)
    lt.step(1)
    assert lt.status() == 0
    _, sc = lt.decode()
    sc = sc.double().cpu().numpy().reshape(nv, nv, n)
    # oracle: scales of the output lines from the input line maxima, then sampled columns
    host = fq.cpu().numpy()
    S = S16.scale_for(S16.diamond_bound(np.abs(host).max(axis=3).astype(np.float64)))
    rng = np.random.default_rng(3)
    rows = rng.integers(0, n, 4)
    np.testing.assert_array_equal(sc[:, :, rows], S[:, :, rows])
    ux, uy = O.flow2d_u(fl.a, fl.kvec, fl.phi0, n, n, dx)
    jy = np.arange(nv)[:, None]
    jx = np.arange(nv)[None, :]
    state = lt.state
    for y in rows:
        for x in rng.integers(0, n, 3):
            fs = host[jy, jx, (y - (jy - J)) % n, (x - (jx - J)) % n].astype(np.float64)
            col = O.diffuse_2d(O.drag_2d(fs[..., None, None], ux[y:y + 1, x:x + 1],
                                         uy[y:y + 1, x:x + 1], tau_p, dt, dv), kappa, dt, dv)
            want, over = S16.encode(col, S[:, :, y:y + 1], fmt)
            assert not over
            want = want[..., 0, 0]
            got = (state[:, :, y, x].double().cpu().numpy() * sc[:, :, y])
            w = np.abs(want).ravel()
            prev = np.concatenate([[0.0], w[:-1]])
            tol = (STEP[fmt] * (w + prev)).reshape(want.shape) + 2.0**-20 * 4096 * S[:, :, y]
            assert np.all(np.abs(got - want) <= tol), (y, x, np.max(np.abs(got - want) / tol))
    lt.close()


def test_learned_full_size_sampled_corrections(lat):
    n, nv = 2048, 9
    J = (nv - 1) // 2
    tau_p, kappa = L, 1e-3
    dt = I.choose_dt(2, n, L, 33, tau_p, kappa) / 4
    dx = L / n
    dv = dx / dt
    f = seeded_state(n, nv, dx, dv, 9)
    fl = I.flow2d_inputs(1234 + 13, 2, n, n, dx)
    W = {k: v.astype(np.float32).astype(np.float64) for k, v in Lr.init_weights(21, 0.5).items()}
    params = np.concatenate([W["W1"].ravel(), W["b1"], W["W2"].ravel(), W["b2"], W["W3"].ravel(),
                             W["b3"]]).astype(np.float32)
    lt = lat.Lattice(f, d=2, nx=n, ny=n, nv=nv, L=L, tau_p=tau_p, kappa=kappa, dt=dt)
    lt.set_flow_modes_2d(fl.kvec, fl.a, fl.phi0, fl.tau_f)
    lt.set_noise(fl.noise)
    lt.learn(params, 2)
    G = torch.empty((2, nv, nv, n, n), dtype=torch.float32, device="cuda")
    lt.learn_corrections(G)
    assert lt.status() == 0
    host = f.cpu().numpy()
    ux, uy = O.flow2d_u(fl.a, fl.kvec, fl.phi0, n, n, dx)
    rng = np.random.default_rng(4)
    got, want, tol = [], [], []
    jy = np.arange(nv)[:, None, None, None]
    jx = np.arange(nv)[None, :, None, None]
    d = np.arange(-1, 2)
    for _ in range(48):
        y, x = int(rng.integers(0, n)), int(rng.integers(0, n))
        ys, xs = (y + d) % n, (x + d) % n
        # streamed state and flow on the 3 x 3 spatial patch around the cell
        fs = host[jy, jx, (ys[None, None, :, None] - (jy - J)) % n,
                  (xs[None, None, None, :] - (jx - J)) % n].astype(np.float64)
        X, _ = Lr.features(fs, ux[np.ix_(ys, xs)], uy[np.ix_(ys, xs)], tau_p=tau_p, dt=dt, dv=dv,
                           dx=dx)
        y_out, _ = Lr.mlp_forward(X[:, :, 1, 1], W, dt / tau_p)
        dy = output_error_bound(X[:, :, 1, 1], W, dt / tau_p)
        c = fs[:, :, 1, 1]
        gx, gy, tx, ty = (np.zeros((nv, nv)) for _ in range(4))
        gx[:, :-1] = y_out[:, :-1, 0] * (c[:, 1:] - c[:, :-1])
        gy[:-1] = y_out[:-1, :, 1] * (c[1:] - c[:-1])
        tx[:, :-1] = dy[:, :-1, 0] * np.abs(c[:, 1:] - c[:, :-1])
        ty[:-1] = dy[:-1, :, 1] * np.abs(c[1:] - c[:-1])
        want.append(np.stack([gx, gy]))
        tol.append(np.stack([tx, ty]))
        got.append(G[:, :, :, y, x].double().cpu().numpy())
    got, want, tol = np.array(got), np.array(want), np.array(tol)
    # element by element, within the BF16 network's rounding tolerance (probabilistic analysis,
    # six standard deviations); FP32 features and products add 1e-5 of each value
    err = np.abs(got - want)
    assert np.all(err <= tol + 1e-5 * np.abs(want) + 1e-30), np.max(err / (tol + 1e-30))
    # and the outputs carry the network's effect: not all inside the tolerance of zero
    assert np.sum(np.abs(want) > tol) > 0.5 * np.sum(want != 0)
    # one full learned step keeps the mass
    m0 = lt.moments(per_cell=False)[4][0]
    lt.step(1)
    code, *_, g = lt.moments(per_cell=False)
    assert code == 0 and abs(g[0] - m0) / m0 < 1e-6
    lt.close()
