"""Parity of the CUDA 2D path (through the C ABI) with the FP64 oracle.

Tolerances as for 1D: relative L1 error <= 1e-12 (FP64 storage) and <= 1e-5 (FP32 storage);
pure streaming and the two load paths (plain loads, bulk-copy ring) are compared bit for bit.
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


def make2d(nx, ny, nv, st, kappa, nsteps, seed, init="random", kmax=4):
    tau_p = st * L
    dt = I.choose_dt(2, nx, L, nv, tau_p, kappa)
    dx = L / nx
    dv = dx / dt
    J = (nv - 1) // 2
    if init == "random":
        f0 = I.random_initial((nv, nv, ny, nx), seed)
    else:
        f0 = I.gaussian_initial_2d(nx, ny, nv, dx, dv, 0.2 * max(J, 1) * dv)
    fl = I.flow2d_inputs(seed, nsteps, nx, ny, dx, kmax=kmax)
    return dict(nx=nx, ny=ny, nv=nv, tau_p=tau_p, kappa=kappa, dt=dt, dx=dx, dv=dv, f0=f0,
                fl=fl, nsteps=nsteps)


def gpu2d(lat, c, dtype, kernel=0, nsteps=None, frozen_field=None):
    nsteps = c["nsteps"] if nsteps is None else nsteps
    t = torch.tensor(c["f0"], dtype=dtype, device="cuda")
    lt = lat.Lattice(t, d=2, nx=c["nx"], ny=c["ny"], nv=c["nv"], L=L, tau_p=c["tau_p"],
                     kappa=c["kappa"], dt=c["dt"])
    if kernel:
        lt.set_launch(kernel=kernel)
    if frozen_field is not None:
        lt.set_flow_field(frozen_field)
    else:
        fl = c["fl"]
        lt.set_flow_modes_2d(fl.kvec, fl.a, fl.phi0, fl.tau_f)
        lt.set_noise(fl.noise)
    lt.step(nsteps)
    assert lt.status() == 0
    return lt.state.double().cpu().numpy(), lt


def oracle2d(c, nsteps=None, field=None):
    nsteps = c["nsteps"] if nsteps is None else nsteps
    fl = c["fl"]
    f, _ = O.run_2d(c["f0"], nsteps, tau_p=c["tau_p"], kappa=c["kappa"], dt=c["dt"],
                    dv=c["dv"], dx=c["dx"], kvec=fl.kvec, a=fl.a, phi0=fl.phi0, tau_f=fl.tau_f,
                    noise=fl.noise, field=field)
    return f


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("nx,ny,nv,steps", [(64, 64, 9, 200), (40, 24, 5, 100), (72, 40, 9, 60),
                                            (9, 7, 3, 30), (3, 2, 5, 10), (5, 4, 1, 5)])
def test_plain_path_matches_oracle(lat, dtype, nx, ny, nv, steps):
    """Several tiles, ragged tails in x, N_x and N_y below J (modular wrap), N_v = 1."""
    c = make2d(nx, ny, nv, 0.5, 2e-3, steps, 11 + nx + nv)
    want = oracle2d(c)
    got, lt = gpu2d(lat, c, dtype, kernel=1)
    assert rel_l1(got, want) <= TOL[dtype], rel_l1(got, want)
    lt.close()


@pytest.mark.parametrize("nx,ny,nv,steps", [(136, 6, 33, 12), (256, 8, 17, 20),
                                            (132, 5, 9, 40), (260, 3, 21, 10)])
def test_ring_path_matches_oracle(lat, nx, ny, nv, steps):
    """The bulk-copy ring path: x windows that wrap, several tiles, a ragged last tile."""
    c = make2d(nx, ny, nv, 1.0, 1e-3, steps, 5 + nx)
    want = oracle2d(c)
    got, lt = gpu2d(lat, c, torch.float32, kernel=2)
    assert rel_l1(got, want) <= 1e-5, rel_l1(got, want)
    plain, lt2 = gpu2d(lat, c, torch.float32, kernel=1)
    assert np.array_equal(got, plain)
    lt.close()
    lt2.close()


def test_gaussian_start_with_flow_1000_steps(lat):
    """64^2 x 9^2, St = 1, Gaussian start, random-phase flow, 1000 steps, FP64 and FP32."""
    c = make2d(64, 64, 9, 1.0, 1e-3, 1000, 21, init="gauss")
    want = oracle2d(c)
    for dtype in (torch.float64, torch.float32):
        got, lt = gpu2d(lat, c, dtype)
        assert rel_l1(got, want) <= TOL[dtype], (dtype, rel_l1(got, want))
        lt.close()


def test_128x128_33x33_100_steps(lat):
    """The 2D size at which the 16-bit forms are validated: 128^2 x 33^2, St = 1, random-phase
    flow, 100 steps, FP64 (1e-12) and FP32 (1e-5) storage in the default launch shape."""
    c = make2d(128, 128, 33, 1.0, 1e-3, 100, 13)
    want = oracle2d(c)
    for dtype in (torch.float64, torch.float32):
        got, lt = gpu2d(lat, c, dtype)
        err = rel_l1(got, want)
        print(f"\n[{dtype}] relative L1 {err:.3e}", end="")
        assert err <= TOL[dtype], (dtype, err)
        lt.close()


@pytest.mark.parametrize("st", [0.1, 10.0])
@pytest.mark.parametrize("kernel", [1, 5])
def test_stokes_numbers_match_oracle(lat, st, kernel):
    """St = 0.1 (smallest tau_p: largest V_max and drag Courant number under Eq. cfl) and
    St = 10 on 136 x 24 x 17^2 (two tiles with a ragged second one), 150 steps, plain loads and
    the producer/consumer ring, FP64 (plain loads only) and FP32."""
    c = make2d(136, 24, 17, st, 1e-3, 150, 31 + int(10 * st))
    want = oracle2d(c)
    for dtype in ((torch.float64, torch.float32) if kernel == 1 else (torch.float32,)):
        got, lt = gpu2d(lat, c, dtype, kernel=kernel)
        assert rel_l1(got, want) <= TOL[dtype], (st, dtype, rel_l1(got, want))
        assert got.min() >= -1e-6 * got.max()
        lt.close()


@pytest.mark.parametrize("kernel", [1, 2, 3, 4, 5, 6, 7, 8, 9, 10])
def test_free_streaming_is_exact(lat, kernel):
    nx, ny, nv = 136, 12, 9
    rng = np.random.default_rng(3)
    f0 = rng.random((nv, nv, ny, nx)).astype(np.float32)
    t = torch.tensor(f0, device="cuda")
    lt = lat.Lattice(t, d=2, nx=nx, ny=ny, nv=nv, L=L, tau_p=math.inf, kappa=0.0, dt=0.1)
    lt.set_launch(kernel=kernel)
    lt.step(5)
    J = (nv - 1) // 2
    want = np.empty_like(f0)
    for jy in range(nv):
        for jx in range(nv):
            want[jy, jx] = np.roll(f0[jy, jx], (5 * (jy - J), 5 * (jx - J)), axis=(0, 1))
    assert np.array_equal(lt.state.cpu().numpy(), want)
    lt.close()


def test_frozen_field_flow(lat):
    c = make2d(48, 40, 9, 1.0, 1e-3, 50, 4)
    rng = np.random.default_rng(4)
    vmax = 4 * c["dv"]
    ux = rng.uniform(-vmax, vmax, (40, 48))
    uy = rng.uniform(-vmax, vmax, (40, 48))
    want = oracle2d(c, field=(ux, uy))
    u = torch.tensor(np.stack([ux, uy]), dtype=torch.float64, device="cuda")
    got, lt = gpu2d(lat, c, torch.float64, frozen_field=u)
    assert rel_l1(got, want) <= 1e-12
    lt.close()


def test_moments_match_oracle(lat):
    c = make2d(40, 24, 9, 1.0, 1e-3, 10, 8)
    got, lt = gpu2d(lat, c, torch.float64)
    code, rho, mv, mv2, glob = lt.moments()
    assert code == 0
    r_o, mvx_o, mvy_o, mv2_o, g_o = O.moments_2d(got, c["dx"], c["dv"])
    np.testing.assert_allclose(rho.cpu().numpy(), r_o.ravel(), rtol=1e-13)
    mvc = mv.cpu().numpy()
    np.testing.assert_allclose(mvc[:40 * 24], mvx_o.ravel(), rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(mvc[40 * 24:], mvy_o.ravel(), rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(mv2.cpu().numpy(), mv2_o.ravel(), rtol=1e-12)
    np.testing.assert_allclose(glob, g_o, rtol=1e-13, atol=1e-15)
    lt.close()


def test_cfl_rejected_on_host_2d(lat):
    t = torch.zeros((9, 9, 8, 8), device="cuda")
    with pytest.raises(lat.LatError) as e:  # 2 (dt/tau_p) J = 2 * 0.3 * 4 > 1
        lat.Lattice(t, d=2, nx=8, ny=8, nv=9, L=L, tau_p=1.0, kappa=0.0, dt=0.3)
    assert e.value.code == lat.LAT_ECFL


def _one_cell_oracle(f0, x, y, ux, uy, tau_p, kappa, dt, dv, gathered=False):
    """Oracle output column of one cell after one step: gather its post-streaming column
    f*(x, y, jx, jy) = f0(x - jx, y - jy, jx, jy) (already done when ``gathered``) and apply the
    oracle's drag and diffusion."""
    nv, _, ny, nx = f0.shape
    J = (nv - 1) // 2
    col = np.empty((nv, nv, 1, 1))
    for jy in range(nv):
        for jx in range(nv):
            col[jy, jx, 0, 0] = (f0[jy, jx, 0, 0] if gathered else
                                 f0[jy, jx, (y - (jy - J)) % ny, (x - (jx - J)) % nx])
    g = O.drag_2d(col, np.array([[ux]]), np.array([[uy]]), tau_p, dt, dv)
    return O.diffuse_2d(g, kappa, dt, dv)[:, :, 0, 0]


@pytest.mark.parametrize("kernel", [1, 2, 3, 4, 5, 6, 7])
def test_many_tiles_per_block_match_oracle(lat, kernel):
    """136 x 200 x 9^2 with one resident block per SM: 400 tiles on at most 152 blocks, so every
    block carries its pipeline across several tiles."""
    c = make2d(136, 200, 9, 1.0, 1e-3, 6, 31)
    want = oracle2d(c)
    t = torch.tensor(c["f0"], dtype=torch.float32, device="cuda")
    lt = lat.Lattice(t, d=2, nx=136, ny=200, nv=9, L=L, tau_p=c["tau_p"], kappa=c["kappa"],
                     dt=c["dt"])
    lt.set_launch(kernel=kernel, blocks_per_sm=1)
    fl = c["fl"]
    lt.set_flow_modes_2d(fl.kvec, fl.a, fl.phi0, fl.tau_f)
    lt.set_noise(fl.noise)
    lt.step(6)
    assert lt.status() == 0
    got = lt.state.double().cpu().numpy()
    assert rel_l1(got, want) <= 1e-5, rel_l1(got, want)
    lt.close()


def test_ring_equals_plain_at_full_size(lat):
    nx = ny = 512
    nv = 33
    gen = torch.Generator(device="cuda")
    gen.manual_seed(9)
    f0 = torch.rand((nv, nv, ny, nx), generator=gen, device="cuda") + 0.1
    dt = I.choose_dt(2, nx, L, nv, L, 1e-3)
    fl = I.flow2d_inputs(10, 3, nx, ny, L / nx)
    outs = []
    # plain loads; ring with 1 and 3 chunks; the five producer/consumer variants
    for kernel, block in ((1, 0), (2, 128), (2, 384), (3, 0), (4, 0), (5, 0), (6, 0), (7, 0)):
        lt = lat.Lattice(f0.clone(), d=2, nx=nx, ny=ny, nv=nv, L=L, tau_p=L, kappa=1e-3, dt=dt)
        lt.set_launch(kernel=kernel, block=block)
        lt.set_flow_modes_2d(fl.kvec, fl.a, fl.phi0, fl.tau_f)
        lt.set_noise(fl.noise)
        lt.step(2)
        assert lt.status() == 0
        outs.append(lt.state.clone())
        lt.close()
    for o in outs[1:]:
        assert torch.equal(outs[0], o)


@pytest.mark.parametrize("flow", ["none", "modes"])
def test_full_size_512_sampled(lat, flow):
    """512^2 x 33^2 FP32 (2.85e8 cells) in the launch shape the bench uses: one step from a
    random state, 24 sampled cells recomputed by the oracle one by one; then 20 more steps
    with mass conservation and positivity checked at full size."""
    nx = ny = 512
    nv = 33
    tau_p = 1.0 * L
    kappa = 1e-3
    dt = I.choose_dt(2, nx, L, nv, tau_p, kappa)
    dx = L / nx
    dv = dx / dt
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    t = torch.rand((nv, nv, ny, nx), generator=gen, device="cuda") + 0.1
    f0 = t.clone()
    fl = I.flow2d_inputs(6, 21, nx, ny, dx)
    lt = lat.Lattice(t, d=2, nx=nx, ny=ny, nv=nv, L=L, tau_p=tau_p, kappa=kappa, dt=dt)
    if flow == "modes":
        lt.set_flow_modes_2d(fl.kvec, fl.a, fl.phi0, fl.tau_f)
        lt.set_noise(fl.noise)
        ux, uy = O.flow2d_u(fl.a, fl.kvec, fl.phi0, nx, ny, dx)
    else:
        ux = uy = np.zeros((ny, nx))
    lt.autotune(reps=2)
    lt.step(1)
    out = lt.state
    rng = np.random.default_rng(7)
    J = (nv - 1) // 2
    jj = np.arange(nv)
    for _ in range(24):
        x, y = int(rng.integers(nx)), int(rng.integers(ny))
        ys = [(y - (jy - J)) % ny for jy in range(nv)]
        xs = [(x - (jx - J)) % nx for jx in range(nv)]
        block = f0[:, :, ys][:, :, :, xs].double().cpu().numpy()   # [jy, jx, a, b]
        col = block[jj[:, None], jj[None, :], jj[:, None], jj[None, :]]  # f*(x, y, jx, jy)
        want = _one_cell_oracle(col[:, :, None, None], 0, 0, ux[y, x], uy[y, x], tau_p, kappa,
                                dt, dv, gathered=True)
        got = out[:, :, y, x].double().cpu().numpy()
        assert rel_l1(got, want) <= 1e-6, (x, y, rel_l1(got, want))
    m0 = f0.double().sum().item()
    lt.step(20)
    assert lt.status() == 0
    s = lt.state
    assert abs(s.double().sum().item() / m0 - 1) < 1e-6
    assert s.min().item() >= -1e-6 * s.max().item()
    lt.close()


@pytest.mark.parametrize("kernel,nv", [(1, 9), (4, 9), (5, 9), (4, 17), (5, 33)])
def test_step_moments_equal_step_then_moments(lat, kernel, nv):
    """lat_step_moments against lat_step + lat_moments from the same start: the state and the
    per-cell moments bit for bit, the globals to the rounding order of the compensated sums.
    Kernels 4 and 5 reduce the moments inside the last step; kernel 1 takes the two calls.
    136 x 23: a ragged last tile (136 = 128 + 8) and several tiles per block."""
    c = make2d(136, 23, nv, 1.0, 1e-3, 5, 40 + nv)
    outs = []
    for fused in (False, True):
        t = torch.tensor(c["f0"], dtype=torch.float32, device="cuda")
        lt = lat.Lattice(t, d=2, nx=136, ny=23, nv=nv, L=L, tau_p=c["tau_p"], kappa=c["kappa"],
                         dt=c["dt"])
        lt.set_launch(kernel=kernel, blocks_per_sm=1)
        fl = c["fl"]
        lt.set_flow_modes_2d(fl.kvec, fl.a, fl.phi0, fl.tau_f)
        lt.set_noise(fl.noise)
        lt.step(1)
        if fused:
            code, rho, mv, mv2, glob = lt.step_moments(4)
        else:
            lt.step(4)
            code, rho, mv, mv2, glob = lt.moments()
        assert code == 0 and lt.status() == 0 and lt.steps_done == 5
        outs.append((lt.state.cpu().numpy().copy(), rho.cpu().numpy(), mv.cpu().numpy(),
                     mv2.cpu().numpy(), glob.copy()))
        lt.close()
    (s0, r0, v0, w0, g0), (s1, r1, v1, w1, g1) = outs
    assert np.array_equal(s0, s1)
    assert np.array_equal(r0, r1) and np.array_equal(v0, v1) and np.array_equal(w0, w1)
    # mass and energy (positive sums) to 1e-12; momentum, a sum of both signs, to 1e-12 of
    # sqrt(M E), which bounds the sum of |v| f by Cauchy-Schwarz
    np.testing.assert_allclose(g1[[0, 3]], g0[[0, 3]], rtol=1e-12)
    np.testing.assert_allclose(g1[1:3], g0[1:3], rtol=0, atol=1e-12 * math.sqrt(g0[0] * g0[3]))


@pytest.mark.parametrize("nv", [9, 13, 17, 19, 21, 33])
def test_packed_sweep_gives_the_scalar_bits(lat, nv):
    """Launch kernels 8..10 (a velocity row as two half-rows in f32x2 register pairs) write the
    bits of the scalar sweep (plain loads, kernel 1; producer/consumer, kernel 5), on a flowing
    random state with ragged tiles, and stay within the FP32 tolerance of the oracle."""
    c = make2d(136, 20, nv, 1.0, 2e-3, 12, 40 + nv)
    plain, lt1 = gpu2d(lat, c, torch.float32, kernel=1)
    lt1.close()
    for k in (5, 8, 9, 10):
        got, lt = gpu2d(lat, c, torch.float32, kernel=k)
        assert np.array_equal(got, plain), (k, np.abs(got - plain).max())
        lt.close()
    want = oracle2d(c)
    assert rel_l1(plain, want) <= 1e-5
