"""Parity of the CUDA 1D path (through the C ABI) with the FP64 oracle.

Tolerances: relative L1 error sum|f_gpu - f_oracle| / sum|f_oracle| after the stated number of
steps must be <= 1e-12 for FP64 storage and <= 1e-5 for FP32 storage (the stated targets for
1000 steps of the 1D lattice N_x = 256, N_v = 33).  Integer-like results (pure streaming) are
compared bit for bit.
"""
import math

import numpy as np
import pytest
import torch

from oracle import lattice as O
from paper_1508_02899_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L = 2 * math.pi
TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def rel_l1(got, want):
    return np.abs(got - want).sum() / np.abs(want).sum()


def make_case(nx, nv, st, kappa, nsteps, seed, nmodes=8, init="gauss"):
    tau_p = st * L
    dt = I.choose_dt(1, nx, L, nv, tau_p, kappa)
    dx = L / nx
    dv = dx / dt
    J = (nv - 1) // 2
    if init == "gauss":
        f0 = I.gaussian_initial_1d(nx, nv, dx, dv, 0.2 * max(J, 1) * dv)
    else:
        f0 = I.random_initial((nv, nx), seed)
    fl = I.flow1d_inputs(seed, nsteps, nmodes=nmodes)
    return dict(nx=nx, nv=nv, tau_p=tau_p, kappa=kappa, dt=dt, dx=dx, dv=dv, f0=f0, fl=fl,
                nsteps=nsteps)


def run_gpu(lat, c, dtype, nsteps=None, launch=None):
    nsteps = c["nsteps"] if nsteps is None else nsteps
    t = torch.tensor(c["f0"], dtype=dtype, device="cuda")
    lt = lat.Lattice(t, d=1, nx=c["nx"], nv=c["nv"], L=L, tau_p=c["tau_p"], kappa=c["kappa"],
                     dt=c["dt"])
    if launch:
        lt.set_launch(**launch)
    fl = c["fl"]
    lt.set_flow_modes_1d(fl.k, fl.amp0[0], fl.tau_f, fl.sigma)
    lt.set_noise(fl.noise[:, 0, :])
    lt.step(nsteps)
    assert lt.status() == 0
    out = lt.state.double().cpu().numpy()
    return out, lt


def run_oracle(c, nsteps=None):
    nsteps = c["nsteps"] if nsteps is None else nsteps
    fl = c["fl"]
    f, _ = O.run_1d(c["f0"], nsteps, tau_p=c["tau_p"], kappa=c["kappa"], dt=c["dt"],
                    dv=c["dv"], k=fl.k, amp0=fl.amp0[0], tau_f=fl.tau_f, sigma=fl.sigma,
                    noise=fl.noise[:, 0, :])
    return f


_CONFIG0 = None


def config0():
    """N_x = 256, N_v = 33, St = 1, kappa = 1e-3, 8-mode OU flow, Gaussian f0, 1000 steps."""
    global _CONFIG0
    if _CONFIG0 is None:
        c = make_case(256, 33, 1.0, 1e-3, 1000, 1234)
        _CONFIG0 = (c, run_oracle(c))
    return _CONFIG0


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_config0_1000_steps(lat, dtype):
    c, want = config0()
    got, lt = run_gpu(lat, c, dtype)
    err = rel_l1(got, want)
    assert err <= TOL[dtype], err
    lt.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("nx,nv,steps", [(300, 17, 400), (37, 65, 200), (1000, 7, 300),
                                         (5, 1, 10), (1, 5, 20), (3, 9, 50), (700, 33, 300)])
def test_ragged_and_edge_sizes(lat, dtype, nx, nv, steps):
    """Several tiles with a ragged tail, a single partial tile, the generic-N_v kernel (7),
    N_v = 1 (nothing moves), N_x smaller than J (modular wrap)."""
    c = make_case(nx, nv, 0.5, 2e-3, steps, 7 + nx, init="random")
    want = run_oracle(c)
    got, lt = run_gpu(lat, c, dtype)
    assert rel_l1(got, want) <= TOL[dtype]
    lt.close()


@pytest.mark.parametrize("nv", [9, 33, 65, 11])
def test_free_streaming_is_exact(lat, nv):
    """tau_p = inf, kappa = 0: the step is the exact shift f(x - j, j), bit for bit in FP32."""
    nx = 200
    rng = np.random.default_rng(nv)
    f0 = rng.random((nv, nx)).astype(np.float32)
    t = torch.tensor(f0, device="cuda")
    lt = lat.Lattice(t, d=1, nx=nx, nv=nv, L=L, tau_p=math.inf, kappa=0.0, dt=0.1)
    lt.step(7)
    J = (nv - 1) // 2
    want = np.stack([np.roll(f0[jj], 7 * (jj - J)) for jj in range(nv)])
    assert np.array_equal(lt.state.cpu().numpy(), want)
    lt.step(nx - 7)
    assert np.array_equal(lt.state.cpu().numpy(), f0)
    lt.close()


@pytest.mark.parametrize("launch", [dict(kernel=1, block=128, blocks_per_sm=2),
                                    dict(kernel=1, block=512, blocks_per_sm=1),
                                    dict(kernel=2, blocks_per_sm=1), dict(kernel=4),
                                    dict(kernel=5), dict(kernel=6, blocks_per_sm=1),
                                    dict(kernel=7), dict(kernel=1, mode=2), dict(mode=1)])
def test_launch_shapes_are_bit_identical(lat, launch):
    """Kernel variant (plain loads or bulk-copy ring), tile width, grid size, graph capture or
    direct launches change nothing in the result."""
    c = make_case(1000, 33, 1.0, 1e-3, 40, 99, init="random")
    ref, lt0 = run_gpu(lat, c, torch.float32)
    got, lt1 = run_gpu(lat, c, torch.float32, launch=launch)
    assert np.array_equal(ref, got)
    lt0.close()
    lt1.close()


def test_moments_match_oracle(lat):
    c = make_case(300, 17, 1.0, 1e-3, 30, 5, init="random")
    got, lt = run_gpu(lat, c, torch.float64)
    code, rho, mv, mv2, glob = lt.moments()
    assert code == 0
    rho_o, mv_o, mv2_o, glob_o = O.moments_1d(got, c["dx"], c["dv"])
    np.testing.assert_allclose(rho.cpu().numpy(), rho_o, rtol=1e-13)
    np.testing.assert_allclose(mv.cpu().numpy(), mv_o, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(mv2.cpu().numpy(), mv2_o, rtol=1e-12)
    np.testing.assert_allclose(glob, glob_o, rtol=1e-14, atol=1e-16)
    lt.close()


def test_fp32_moments_within_their_bound(lat):
    """FP32 state: the mass sums are exact up to the roundings of their compensation terms
    (about N_v u^2 per column); the momentum and energy column sums take one FMA per value, so
    their error is at most (N_v - 1) u of the sum of |v^k f| (u = 2^-24), plus the compensated
    cross-column part."""
    c = make_case(300, 33, 1.0, 1e-3, 30, 6, init="random")
    got, lt = run_gpu(lat, c, torch.float32)
    code, rho, mv, mv2, glob = lt.moments()
    assert code == 0
    f = got.astype(np.float64)
    rho_o, mv_o, mv2_o, glob_o = O.moments_1d(f, c["dx"], c["dv"])
    nv = f.shape[0]
    v = (np.arange(nv) - (nv - 1) // 2) * c["dv"]
    u = 2.0**-24
    assert abs(glob[0] - glob_o[0]) <= 1e-12 * glob_o[0]
    for k in (1, 2):
        bound = (nv - 1) * u * math.fsum((np.abs(v[:, None]) ** k * np.abs(f)).ravel())
        bound *= c["dx"] * c["dv"]
        assert abs(glob[k] - glob_o[k]) <= bound + 1e-14 * abs(glob_o[k]), k
    np.testing.assert_allclose(rho.cpu().numpy(), rho_o, rtol=1e-12)
    col = (nv - 1) * u * (np.abs(v[:, None]) ** 2 * f).sum(axis=0) / f.sum(axis=0)
    assert np.all(np.abs(mv2.cpu().numpy() - mv2_o) <= col + 1e-13 * np.abs(mv2_o))
    lt.close()


def test_mass_is_conserved_over_1000_steps(lat):
    c, _ = config0()
    got, lt = run_gpu(lat, c, torch.float32)
    code, _, _, _, glob = lt.moments(per_cell=False)
    assert code == 0
    assert abs(glob[0] - 1.0) < 1e-5  # FP32 storage, FP64 reduction
    lt.close()


def test_cfl_rejected_on_host(lat):
    t = torch.zeros((33, 64), device="cuda")
    with pytest.raises(lat.LatError) as e:
        lat.Lattice(t, d=1, nx=64, nv=33, L=L, tau_p=0.01, kappa=0.0, dt=0.5)
    assert e.value.code == lat.LAT_ECFL
    with pytest.raises(lat.LatError) as e:  # kappa dt / dv^2 = 130 > 1/2, drag off
        lat.Lattice(t, d=1, nx=64, nv=33, L=L, tau_p=math.inf, kappa=10.0, dt=0.5)
    assert e.value.code == lat.LAT_ECFL
    with pytest.raises(lat.LatError) as e:
        lat.Lattice(torch.zeros((32, 64), device="cuda"), d=1, nx=64, nv=32, L=L, tau_p=1.0,
                    kappa=0.0, dt=0.01)
    assert e.value.code == lat.LAT_EINVAL


def test_cfl_flagged_on_device_by_a_strong_flow(lat):
    nx, nv = 64, 9
    dt = 0.05
    t = torch.ones((nv, nx), device="cuda")
    lt = lat.Lattice(t, d=1, nx=nx, nv=nv, L=L, tau_p=1.0, kappa=0.0, dt=dt)
    dv = (L / nx) / dt
    u = torch.full((nx,), 100.0 * dv, device="cuda")  # (dt/tau_p)(J + 100) > 1
    lt.set_flow_field(u)
    lt.step(1)
    assert lt.status() == lat.LAT_ECFL
    assert lt.status() == 0  # cleared
    lt.close()


def test_noise_exhaustion_is_reported(lat):
    c = make_case(128, 9, 1.0, 1e-3, 5, 3)
    t = torch.tensor(c["f0"], dtype=torch.float32, device="cuda")
    lt = lat.Lattice(t, d=1, nx=128, nv=9, L=L, tau_p=c["tau_p"], kappa=c["kappa"], dt=c["dt"])
    fl = c["fl"]
    lt.set_flow_modes_1d(fl.k, fl.amp0[0], fl.tau_f, fl.sigma)
    lt.set_noise(fl.noise[:3, 0, :])
    lt.step(3)
    assert lt.status() == 0
    lt.step(1)
    assert lt.status() == lat.LAT_ENOISE
    lt.close()


def test_noise_refill_per_step_matches_one_table(lat):
    """Uploading one row per step (the end-to-end path) equals uploading the whole table."""
    c = make_case(256, 33, 1.0, 1e-3, 20, 11)
    ref, lt0 = run_gpu(lat, c, torch.float64)
    t = torch.tensor(c["f0"], dtype=torch.float64, device="cuda")
    lt = lat.Lattice(t, d=1, nx=256, nv=33, L=L, tau_p=c["tau_p"], kappa=c["kappa"], dt=c["dt"])
    fl = c["fl"]
    lt.set_flow_modes_1d(fl.k, fl.amp0[0], fl.tau_f, fl.sigma)
    for n in range(20):
        lt.set_noise(fl.noise[n:n + 1, 0, :])
        lt.step(1)
    assert np.array_equal(lt.state.cpu().numpy(), ref)
    lt.close()
    lt0.close()
