"""Parity of the batched 1D ensemble (one persistent launch per step) with the FP64 oracle."""
import math

import numpy as np
import pytest
import torch

from oracle import lattice as O
from paper_1508_02899_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def rel_l1(got, want):
    return np.abs(got - want).sum() / np.abs(want).sum()


def build(lat, tab, nv, dtype, fl, seed=0, init="gauss", launch=None):
    parts = []
    for i in range(len(tab.nx)):
        nx = int(tab.nx[i])
        dx = tab.L[i] / nx
        dv = dx / tab.dt[i]
        if init == "gauss":
            parts.append(I.gaussian_initial_1d(nx, nv, dx, dv, 0.2 * ((nv - 1) // 2) * dv))
        else:
            parts.append(I.random_initial((nv, nx), seed + i))
    f0 = np.concatenate([p.ravel() for p in parts])
    t = torch.tensor(f0, dtype=dtype, device="cuda")
    ens = lat.Ensemble(t, nv=nv, nx=tab.nx, L=tab.L, tau_p=tab.tau_p, kappa=tab.kappa,
                       dt=tab.dt)
    if launch:
        ens.set_launch(**launch)
    ens.set_flow_modes(fl.k, fl.amp0, fl.tau_f, fl.sigma)
    ens.set_noise(fl.noise)
    return ens, parts


def oracle_instance(tab, i, nv, f0, fl, nsteps):
    nx = int(tab.nx[i])
    dv = (tab.L[i] / nx) / tab.dt[i]
    f, _ = O.run_1d(f0, nsteps, tau_p=tab.tau_p[i], kappa=tab.kappa[i], dt=tab.dt[i], dv=dv,
                    k=fl.k, amp0=fl.amp0[i], tau_f=fl.tau_f, sigma=fl.sigma,
                    noise=fl.noise[:, i, :])
    return f


def small_table():
    tab = I.ensemble_table(6, 5, nv=33, sizes=(100, 256, 37, 512, 8, 300))
    return tab


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_small_ensemble_matches_oracle(lat, dtype):
    nv, nsteps = 33, 120
    tab = small_table()
    fl = I.flow1d_inputs(77, nsteps, n_inst=len(tab.nx))
    ens, parts = build(lat, tab, nv, dtype, fl, init="random")
    ens.step(nsteps)
    assert ens.status() == 0
    for i in range(len(tab.nx)):
        got = ens.instance_view(i).double().cpu().numpy()
        want = oracle_instance(tab, i, nv, parts[i], fl, nsteps)
        assert rel_l1(got, want) <= TOL[dtype], (i, rel_l1(got, want))
    ens.close()


def test_instances_equal_single_runs_bit_for_bit(lat):
    nv, nsteps = 33, 50
    tab = small_table()
    fl = I.flow1d_inputs(78, nsteps, n_inst=len(tab.nx))
    ens, parts = build(lat, tab, nv, torch.float32, fl, init="random")
    ens.step(nsteps)
    for i in range(len(tab.nx)):
        t = torch.tensor(parts[i], dtype=torch.float32, device="cuda")
        lt = lat.Lattice(t, d=1, nx=int(tab.nx[i]), nv=nv, L=tab.L[i], tau_p=tab.tau_p[i],
                         kappa=tab.kappa[i], dt=tab.dt[i])
        lt.set_flow_modes_1d(fl.k, fl.amp0[i], fl.tau_f, fl.sigma)
        lt.set_noise(fl.noise[:, i, :])
        lt.step(nsteps)
        assert np.array_equal(lt.state.cpu().numpy(), ens.instance_view(i).cpu().numpy()), i
        lt.close()
    ens.close()


def test_per_instance_launches_equal_persistent_launch(lat):
    nv, nsteps = 65, 30
    tab = I.ensemble_table(9, 6, nv=nv, sizes=(1024, 2048, 333))
    fl = I.flow1d_inputs(79, nsteps, n_inst=9)
    a, _ = build(lat, tab, nv, torch.float32, fl)
    b, _ = build(lat, tab, nv, torch.float32, fl, launch=dict(mode=1))
    a.step(nsteps)
    b.step(nsteps)
    assert np.array_equal(a.state.cpu().numpy(), b.state.cpu().numpy())
    a.close()
    b.close()


def test_ensemble_moments_match_oracle(lat):
    nv, nsteps = 33, 20
    tab = small_table()
    fl = I.flow1d_inputs(80, nsteps, n_inst=len(tab.nx))
    ens, _ = build(lat, tab, nv, torch.float64, fl, init="random")
    ens.step(nsteps)
    code, rho, mv, mv2, glob = ens.moments(per_cell=True)
    assert code == 0
    for i in range(len(tab.nx)):
        f = ens.instance_view(i).cpu().numpy()
        dx = tab.L[i] / tab.nx[i]
        dv = dx / tab.dt[i]
        r_o, m_o, m2_o, g_o = O.moments_1d(f, dx, dv)
        sl = slice(int(ens.xoff[i]), int(ens.xoff[i + 1]))
        np.testing.assert_allclose(rho[sl].cpu().numpy(), r_o, rtol=1e-13)
        np.testing.assert_allclose(mv2[sl].cpu().numpy(), m2_o, rtol=1e-12)
        np.testing.assert_allclose(glob[i], g_o, rtol=1e-13, atol=1e-15)
    ens.close()


def test_autotune_keeps_state(lat):
    nv, nsteps = 65, 10
    tab = I.ensemble_table(64, 8, nv=nv)
    fl = I.flow1d_inputs(81, 2 * nsteps, n_inst=64)
    a, _ = build(lat, tab, nv, torch.float32, fl)
    b, _ = build(lat, tab, nv, torch.float32, fl)
    best = b.autotune(reps=2)
    assert best["kernel"] in (1, 2, 3, 4, 5, 6, 7) and best["us_per_step"] > 0
    a.step(nsteps)
    b.step(nsteps)
    assert np.array_equal(a.state.cpu().numpy(), b.state.cpu().numpy())
    a.close()
    b.close()


def test_full_size_ensemble_sampled(lat):
    """The benchmark workload: 4096 instances, N_x uniform over {1024..8192}, N_v = 65,
    St cycling {0.1, 1, 10}, FP32, in the launch shape the bench uses (autotuned); eight
    sampled instances are compared with the oracle after 20 steps."""
    nv, nsteps, n = 65, 20, 4096
    tab = I.ensemble_table(n, 2024, nv=nv)
    fl = I.flow1d_inputs(2025, nsteps, n_inst=n)
    f0 = I.ensemble_initial(tab, nv, torch.float32, "cuda")
    ens = lat.Ensemble(f0, nv=nv, nx=tab.nx, L=tab.L, tau_p=tab.tau_p, kappa=tab.kappa,
                       dt=tab.dt)
    ens.set_flow_modes(fl.k, fl.amp0, fl.tau_f, fl.sigma)
    ens.set_noise(fl.noise)
    ens.autotune(reps=2)
    ens.step(nsteps)
    assert ens.status() == 0
    rng = np.random.default_rng(0)
    sample = sorted(int(i) for i in rng.choice(n, 8, replace=False))
    parts = I.ensemble_initial(tab, nv, None, None, instances=sample)
    for i in sample:
        got = ens.instance_view(i).double().cpu().numpy()
        want = oracle_instance(tab, i, nv, parts[i], fl, nsteps)
        assert rel_l1(got, want) <= 1e-5, (i, rel_l1(got, want))
    code, _, _, _, glob = ens.moments()
    assert code == 0
    np.testing.assert_allclose(glob[:, 0], 1.0, rtol=1e-5)
    ens.close()


@pytest.mark.parametrize("kernel", [5, 1])
def test_step_moments_fused_matches_separate_calls(lat, kernel):
    """lat_step_moments (moments fused into the last step of the producer/consumer kernel, or
    the two calls otherwise) equals lat_step + lat_moments: per-cell moments bit for bit, the
    globals to the rounding order of the compensated sums."""
    nv, nsteps = 65, 6
    tab = I.ensemble_table(40, 12, nv=nv, sizes=(1024, 2048, 4096))
    fl = I.flow1d_inputs(83, nsteps, n_inst=40)
    a, _ = build(lat, tab, nv, torch.float32, fl, launch=dict(kernel=kernel))
    b, _ = build(lat, tab, nv, torch.float32, fl, launch=dict(kernel=kernel))
    a.step(nsteps)
    ca, ra, ma, m2a, ga = a.moments(per_cell=True)
    cb, rb, mb, m2b, gb = b.step_moments(nsteps, per_cell=True)
    assert ca == 0 and cb == 0
    assert np.array_equal(a.state.cpu().numpy(), b.state.cpu().numpy())
    assert torch.equal(ra, rb) and torch.equal(ma, mb) and torch.equal(m2a, m2b)
    np.testing.assert_allclose(gb, ga, rtol=1e-14, atol=1e-18)
    a.close()
    b.close()
