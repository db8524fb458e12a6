"""The learned flux closure through the C ABI against the FP64 oracle (oracle/learned.py).

Tolerances.  The FP32 network (mode 1) follows the oracle to FP32 rounding: relative L1 1e-5
after a few steps, like the plain FP32 step.  The BF16 tensor-core network (mode 2) rounds its
inputs, weights and hidden activations to 8 significant bits, so its outputs carry a relative
error of a few times 2^-8; the test bounds the state's distance to the oracle by 3 % of the
correction's own effect (the distance between the learned and the plain oracle states), plus
the FP32 level.  The gradient of a rollout (FP32 arithmetic throughout) must agree with the
oracle's exact adjoint to 1e-5 of its norm.  The network's outputs are bounded (y = tanh/4)
and the corrections are face diffusivities times the density differences across the faces.
"""
import math

import numpy as np
import pytest
import torch

from oracle import lattice as O
from oracle import learned as Lr
from paper_1508_02899_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L = 2 * math.pi


def pack(W):
    return np.concatenate([W["W1"].ravel(), W["b1"], W["W2"].ravel(), W["b2"], W["W3"].ravel(),
                           W["b3"]]).astype(np.float32)


def quantised_weights(seed, scale):
    """Weights exactly representable in FP32 (the GPU's parameters), as float64 for the oracle."""
    W = Lr.init_weights(seed, scale)
    rng = np.random.default_rng(seed + 1)
    W["b1"] = 0.05 * rng.standard_normal(W["b1"].shape)
    W["b2"] = 0.05 * rng.standard_normal(W["b2"].shape)
    W["b3"] = 0.01 * rng.standard_normal(W["b3"].shape)
    return {k: v.astype(np.float32).astype(np.float64) for k, v in W.items()}


def case(nx, ny, nv, nsteps, seed, st=1.0, kappa=2e-3):
    tau_p = st * L
    dt = I.choose_dt(2, nx, L, nv, tau_p, kappa)
    dx = L / nx
    dv = dx / dt
    J = (nv - 1) // 2
    f0 = I.gaussian_initial_2d(nx, ny, nv, dx, dv, 0.3 * J * dv)
    rng = np.random.default_rng(seed)
    f0 = (f0 * (1 + 0.5 * rng.random((1, 1, ny, nx)))).astype(np.float32).astype(np.float64)
    fl = I.flow2d_inputs(seed, nsteps, nx, ny, dx, kmax=3)
    flows, phi = [], fl.phi0.copy()
    for n in range(nsteps):
        flows.append(O.flow2d_u(fl.a, fl.kvec, phi, nx, ny, dx))
        phi = O.phase_advance(phi, fl.noise[n], dt, fl.tau_f)
    kw = dict(tau_p=tau_p, kappa=kappa, dt=dt, dv=dv, dx=dx)
    return dict(nx=nx, ny=ny, nv=nv, f0=f0, fl=fl, flows=flows, kw=kw)


def lattice(lat, c, f0=None):
    kw = c["kw"]
    t = torch.tensor(c["f0"] if f0 is None else f0, dtype=torch.float32, device="cuda")
    lt = lat.Lattice(t, d=2, nx=c["nx"], ny=c["ny"], nv=c["nv"], L=L, tau_p=kw["tau_p"],
                     kappa=kw["kappa"], dt=kw["dt"])
    fl = c["fl"]
    lt.set_flow_modes_2d(fl.kvec, fl.a, fl.phi0, fl.tau_f)
    lt.set_noise(fl.noise)
    return lt


def rel_l1(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


@pytest.mark.parametrize("mode", [1, 2])
def test_zero_network_gives_the_plain_step(lat, mode):
    c = case(40, 24, 9, 6, 1)
    plain = lattice(lat, c)
    plain.set_launch(kernel=1)
    plain.step(6)
    learned = lattice(lat, c)
    learned.learn(np.zeros(lat.LEARN_NPARAM, np.float32), mode)
    learned.step(6)
    assert plain.status() == 0 and learned.status() == 0
    assert np.array_equal(plain.state.cpu().numpy(), learned.state.cpu().numpy())
    plain.close()
    learned.close()


@pytest.mark.parametrize("nx,ny,nv", [(32, 20, 9), (150, 6, 5), (13, 9, 3), (48, 16, 17)])
def test_fp32_network_matches_oracle(lat, nx, ny, nv):
    """Tiles of 128 phase cells with ragged ends, N_v from 3 to 17, four learned steps."""
    c = case(nx, ny, nv, 4, 7 + nx)
    W = quantised_weights(3, 0.4)
    want = Lr.rollout(c["f0"], W, 4, c["flows"], **c["kw"])
    plain = O.run_2d(c["f0"], 4, kvec=c["fl"].kvec, a=c["fl"].a, phi0=c["fl"].phi0,
                     tau_f=c["fl"].tau_f, noise=c["fl"].noise, **c["kw"])[0]
    assert rel_l1(want, plain) > 1e-4  # the correction matters
    lt = lattice(lat, c)
    lt.learn(pack(W), 1)
    lt.step(4)
    assert lt.status() == 0
    got = lt.state.double().cpu().numpy()
    assert rel_l1(got, want) <= 1e-5, rel_l1(got, want)
    lt.close()


@pytest.mark.parametrize("nx,ny,nv", [(32, 20, 9), (150, 6, 5), (48, 16, 17), (256, 12, 9),
                                     (128, 7, 5)])
def test_tensor_core_network_matches_oracle(lat, nx, ny, nv):
    """Ragged 128-cell tiles in storage order (N_x = 128 is below the copy ring's window, so
    its launch keeps plain loads and storage order too), and with N_x = 256 units of 128 x taken
    plane by plane."""
    c = case(nx, ny, nv, 4, 11 + nx)
    W = quantised_weights(5, 0.4)
    want = Lr.rollout(c["f0"], W, 4, c["flows"], **c["kw"])
    plain = O.run_2d(c["f0"], 4, kvec=c["fl"].kvec, a=c["fl"].a, phi0=c["fl"].phi0,
                     tau_f=c["fl"].tau_f, noise=c["fl"].noise, **c["kw"])[0]
    lt = lattice(lat, c)
    lt.learn(pack(W), 2)
    lt.step(4)
    assert lt.status() == 0
    got = lt.state.double().cpu().numpy()
    effect = np.abs(want - plain).sum()
    err = np.abs(got - want).sum()
    assert err <= 0.03 * effect + 1e-5 * np.abs(want).sum(), (err / effect)
    lt.close()


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("nx,ny,nv", [(256, 10, 9), (136, 6, 9), (264, 12, 17)])
def test_corrected_step_on_the_ring_gives_the_plain_bits(lat, mode, nx, ny, nv):
    """The corrected step on the bulk-copy ring (the default where N_x allows it) against the
    plain-load corrected step (launch kernel 1): the same sweep with the same corrections,
    including a ragged last tile."""
    c = case(nx, ny, nv, 3, 31 + nv)
    W = quantised_weights(9, 0.4)
    out = []
    for plain in (True, False):
        lt = lattice(lat, c)
        if plain:
            lt.set_launch(kernel=1)
        lt.learn(pack(W), mode)
        lt.step(3)
        assert lt.status() == 0
        out.append(lt.state.cpu().numpy())
        lt.close()
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("nx,ny,nv", [(256, 10, 9), (512, 7, 3), (384, 9, 5), (256, 12, 17)])
def test_unit_order_network_gives_the_storage_order_bits(lat, nx, ny, nv):
    """Tensor-core network with N_x a multiple of 128: units of 128 x taken plane by plane with
    the velocity neighbourhood slid along each plane row (the default launch) against tiles in
    storage order that gather all nine neighbours (launch kernel 1); the corrections must be the
    same bits, and so must the state after three learned steps."""
    c = case(nx, ny, nv, 3, 41 + nv)
    W = quantised_weights(13, 0.5)
    G, S = [], []
    for plain in (True, False):
        lt = lattice(lat, c)
        if plain:
            lt.set_launch(kernel=1)
        lt.learn(pack(W), 2)
        out = torch.empty((2, nv * nv * ny * nx), dtype=torch.float32, device="cuda")
        lt.learn_corrections(out)
        lt.step(3)
        assert lt.status() == 0
        G.append(out.cpu().numpy())
        S.append(lt.state.cpu().numpy())
        lt.close()
    assert np.abs(G[1]).sum() > 0
    assert np.array_equal(G[0], G[1])
    assert np.array_equal(S[0], S[1])


@pytest.mark.parametrize("mode", [1, 2])
def test_learned_step_keeps_mass(lat, mode):
    c = case(64, 32, 9, 20, 5)
    lt = lattice(lat, c)
    lt.learn(pack(quantised_weights(9, 0.5)), mode)
    m0 = lt.moments(per_cell=False)[4][0]
    lt.step(20)
    code, *_, g = lt.moments(per_cell=False)
    assert code == 0
    assert abs(g[0] - m0) / m0 < 2e-6, abs(g[0] - m0) / m0
    lt.close()


def test_rollout_gradient_matches_oracle(lat):
    c = case(16, 12, 5, 3, 21)
    W = quantised_weights(13, 0.5)
    rng = np.random.default_rng(4)
    target = Lr.rollout(c["f0"], Lr.zero_weights(), 3, c["flows"], **c["kw"])
    target = (target * (1 + 0.02 * rng.standard_normal(target.shape))).astype(np.float32)
    loss_o, g_o = Lr.rollout_grad(c["f0"], W, 3, c["flows"], target.astype(np.float64),
                                  rho_weight=0.7, **c["kw"])
    lt = lattice(lat, c)
    lt.learn(pack(W), 1)
    state0 = lt.state.clone()
    loss, g = lt.learn_grad(3, torch.tensor(target, device="cuda"), 0.7)
    # the state and the step count are untouched
    assert torch.equal(lt.state, state0) and lt.steps_done == 0
    assert loss == pytest.approx(loss_o, rel=1e-5)
    go = pack(g_o).astype(np.float64)
    assert np.linalg.norm(g - go) <= 1e-5 * np.linalg.norm(go), np.linalg.norm(g - go) / np.linalg.norm(go)
    # a second call gives the same numbers (the flow state was restored), up to the order of
    # the FP32 atomic additions that sum the parameter gradients over the cells
    loss2, g2 = lt.learn_grad(3, torch.tensor(target, device="cuda"), 0.7)
    assert loss2 == loss
    assert np.linalg.norm(g2 - g) <= 1e-6 * np.linalg.norm(g)
    lt.close()


def _bf16_weights(W):
    """The weights the tensor-core network multiplies by: W1 with b1 folded into its row 15
    (the constant feature) and every weight rounded to BF16 (8 significant bits, ties to even)."""
    from oracle import storage16 as S16

    def bf(x):
        return S16.round16(np.asarray(x, dtype=np.float64), "bf16")

    We = {k: v.copy() for k, v in W.items()}
    w1 = We["W1"].astype(np.float32)
    w1[15] = w1[15] + We["b1"].astype(np.float32)
    We["W1"] = bf(w1)
    We["b1"] = np.zeros_like(We["b1"])
    for k in ("W2", "b2", "W3", "b3"):
        We[k] = bf(We[k])
    return We


@pytest.mark.parametrize("nx,ny,nv,nsteps", [(16, 12, 5, 3), (40, 24, 9, 2), (136, 8, 9, 2)])
def test_tensor_core_gradient_matches_oracle(lat, nx, ny, nv, nsteps):
    """lat_learn_grad with the BF16 tensor-core network (mode 2): forward rollout on the tensor
    cores, then the network's backward and the weight-gradient sums as tcgen05 MMAs (FP32
    accumulation).  Compared with the oracle's exact adjoint (FP64) of the network with the
    weights it multiplies by (b1 folded into W1's row 15, all rounded to BF16), and with the
    FP64 weights.  The rounding of the weights alone moves the oracle's gradient by 0.7 to 3 %
    on these cases; features, activations and the backward's operands are rounded to 8 bits as
    well.  Measured: 0.9, 2.3 and 0.6 % against the BF16 weights, 1.3, 3.8 and 2.4 % against the
    FP64 weights."""
    c = case(nx, ny, nv, nsteps, 21 + nx)
    W = quantised_weights(13, 0.5)
    rng = np.random.default_rng(4)
    target = Lr.rollout(c["f0"], Lr.zero_weights(), nsteps, c["flows"], **c["kw"])
    target = (target * (1 + 0.02 * rng.standard_normal(target.shape))).astype(np.float32)
    tg = target.astype(np.float64)
    loss_o, g_o = Lr.rollout_grad(c["f0"], W, nsteps, c["flows"], tg, rho_weight=0.7, **c["kw"])
    _, g_e = Lr.rollout_grad(c["f0"], _bf16_weights(W), nsteps, c["flows"], tg, rho_weight=0.7,
                             **c["kw"])
    ge = pack(g_e).astype(np.float64)
    ge[1024:1088] = ge[15 * 64:16 * 64]  # b1 enters like the folded row: the same gradient
    lt = lattice(lat, c)
    lt.learn(pack(W), 2)
    state0 = lt.state.clone()
    loss, g = lt.learn_grad(nsteps, torch.tensor(target, device="cuda"), 0.7)
    assert torch.equal(lt.state, state0) and lt.steps_done == 0
    go = pack(g_o).astype(np.float64)
    err_e = np.linalg.norm(g - ge) / np.linalg.norm(ge)
    err_o = np.linalg.norm(g - go) / np.linalg.norm(go)
    print(f"\n[{nx}x{ny}x{nv}^2, {nsteps} steps] loss rel {abs(loss - loss_o) / loss_o:.3e}, "
          f"gradient rel {err_e:.3e} (BF16 weights), {err_o:.3e} (FP64 weights)", end="")
    assert abs(loss - loss_o) <= 1e-2 * loss_o
    assert err_e <= 3e-2, err_e
    assert err_o <= 5e-2, err_o
    lt.close()


@pytest.mark.parametrize("nx", [72, 256])
@pytest.mark.parametrize("mode,tol", [(1, 1e-5), (2, 0.03)])
def test_corrections_match_oracle(lat, mode, tol, nx):
    """Correction fluxes of one state (128-cell tiles with a ragged end, or row tiles): FP32
    network to 1e-5 of their norm, BF16 tensor-core network to 3 % (inputs, weights, activations
    rounded to 2^-8)."""
    c = case(nx, 30, 9, 1, 17)
    W = quantised_weights(7, 0.5)
    gx, gy = Lr.corrections(c["f0"], *c["flows"][0], W,
                            **{k: c["kw"][k] for k in ("tau_p", "dt", "dv", "dx")})
    want = np.stack([gx, gy])
    lt = lattice(lat, c)
    lt.learn(pack(W), mode)
    out = torch.empty(want.shape, dtype=torch.float32, device="cuda")
    lt.learn_corrections(out)
    assert lt.status() == 0
    got = out.double().cpu().numpy()
    assert np.linalg.norm(got - want) <= tol * np.linalg.norm(want), (
        np.linalg.norm(got - want) / np.linalg.norm(want))
    lt.close()


def test_adam_kernel_matches_the_update_rule(lat):
    """lat_adam against the Adam update written out in FP64 (Kingma and Ba), three steps."""
    rng = np.random.default_rng(9)
    n = 5378
    p = rng.standard_normal(n).astype(np.float32)
    pd = torch.tensor(p, device="cuda")
    m = torch.zeros_like(pd)
    v = torch.zeros_like(pd)
    gd = torch.zeros_like(pd)
    pr, mr, vr = p.astype(np.float64), np.zeros(n), np.zeros(n)
    lr, b1, b2, eps, sc = 1e-3, 0.9, 0.999, 1e-8, 3.0
    for t in (1, 2, 3):
        g = (rng.standard_normal(n) * 1e-3).astype(np.float32)
        gd.copy_(torch.tensor(g))
        lat.adam(pd, m, v, gd, t, lr, b1, b2, eps, sc)
        gg = g.astype(np.float64) * sc
        mr = b1 * mr + (1 - b1) * gg
        vr = b2 * vr + (1 - b2) * gg * gg
        pr = pr - lr * (mr / (1 - b1 ** t)) / (np.sqrt(vr / (1 - b2 ** t)) + eps)
    got = pd.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - pr)) <= 1e-6 * (np.abs(pr).max() + 1), np.max(np.abs(got - pr))
    with pytest.raises(lat.LatError):
        lat.adam(pd, m, v, gd, 0, lr)
