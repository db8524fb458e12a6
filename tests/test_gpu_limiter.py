"""Parity of the flux-limited drag scheme (LAT_SCHEME_KOREN) with the FP64 oracle of
oracle/limiter.py.  1D: single lattices after 1000 steps (1e-12 FP64, 1e-5 FP32), every launch
variant bit for bit, an ensemble with ragged sizes, the benchmark ensemble at full size on sampled
instances, mass and positivity, and the host-side checks.  2D (the scheme of the paper's 2D runs):
random-phase flows on four shapes (the fused kernel, the default), the fused kernel against the
three passes bit for bit, the tilted cellular flow, mass and positivity, and the bench's
1024^2 x 19^2 form at full size on sampled cells."""
import math

import numpy as np
import pytest
import torch

from oracle import lattice as O
from oracle import limiter as K
from paper_1508_02899_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L = 2 * math.pi
MU = 2.0 / 3.0
TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


def rel_l1(got, want):
    return np.abs(got - want).sum() / np.abs(want).sum()


def case(nx, nv, st, kappa, nsteps, seed, mu=MU, init="gauss"):
    tau_p = st * L
    dt = I.choose_dt(1, nx, L, nv, tau_p, kappa, cfl_factor=1 + mu)
    dx = L / nx
    dv = dx / dt
    J = (nv - 1) // 2
    if init == "gauss":
        f0 = I.gaussian_initial_1d(nx, nv, dx, dv, 0.2 * J * dv)
    else:
        f0 = I.random_initial((nv, nx), seed)
    fl = I.flow1d_inputs(seed, nsteps)
    return dict(nx=nx, nv=nv, tau_p=tau_p, kappa=kappa, dt=dt, dv=dv, f0=f0, fl=fl,
                nsteps=nsteps, mu=mu)


def run_gpu(lat, c, dtype, launch=None, nsteps=None):
    nsteps = c["nsteps"] if nsteps is None else nsteps
    t = torch.tensor(c["f0"], dtype=dtype, device="cuda")
    lt = lat.Lattice(t, d=1, nx=c["nx"], nv=c["nv"], L=L, tau_p=c["tau_p"], kappa=c["kappa"],
                     dt=c["dt"])
    lt.set_scheme(lat.SCHEME_KOREN, c["mu"])
    if launch:
        lt.set_launch(**launch)
    fl = c["fl"]
    lt.set_flow_modes_1d(fl.k, fl.amp0[0], fl.tau_f, fl.sigma)
    lt.set_noise(fl.noise[:, 0, :])
    lt.step(nsteps)
    assert lt.status() == 0
    return lt.state.double().cpu().numpy(), lt


def run_oracle(c, nsteps=None):
    nsteps = c["nsteps"] if nsteps is None else nsteps
    fl = c["fl"]
    f, _ = K.run_1d(c["f0"], nsteps, tau_p=c["tau_p"], kappa=c["kappa"], dt=c["dt"], dv=c["dv"],
                    k=fl.k, amp0=fl.amp0[0], tau_f=fl.tau_f, sigma=fl.sigma,
                    noise=fl.noise[:, 0, :], mu=c["mu"])
    return f


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_1000_steps_match_oracle(lat, dtype):
    c = case(256, 33, 1.0, 1e-3, 1000, 11)
    want = run_oracle(c)
    got, lt = run_gpu(lat, c, dtype)
    assert rel_l1(got, want) <= TOL[dtype], rel_l1(got, want)
    lt.close()


@pytest.mark.parametrize("nv,nx,mu", [(3, 40, MU), (9, 137, 1.0), (17, 300, MU), (65, 520, 1.0)])
def test_shapes_and_limiter_bounds_match_oracle(lat, nv, nx, mu):
    c = case(nx, nv, 0.3, 2e-3, 40, nv + nx, mu=mu, init="random")
    want = run_oracle(c)
    got, lt = run_gpu(lat, c, torch.float64)
    assert rel_l1(got, want) <= 1e-12, rel_l1(got, want)
    lt.close()


def test_launch_variants_give_the_same_bits(lat):
    c = case(1000, 33, 1.0, 1e-3, 30, 5, init="random")
    outs = []
    for kernel in (1, 2, 3, 4, 5, 6, 7):
        got, lt = run_gpu(lat, c, torch.float32, launch=dict(kernel=kernel))
        outs.append(got)
        lt.close()
    for k, o in enumerate(outs[1:], start=2):
        assert np.array_equal(outs[0], o), k


def test_ensemble_matches_oracle(lat):
    nv, nsteps = 33, 60
    tab = I.ensemble_table(6, 5, nv=nv, sizes=(100, 256, 37, 512, 8, 300), cfl_factor=1 + MU)
    fl = I.flow1d_inputs(78, nsteps, n_inst=len(tab.nx))
    parts = [I.random_initial((nv, int(n)), 30 + i) for i, n in enumerate(tab.nx)]
    t = torch.tensor(np.concatenate([p.ravel() for p in parts]), dtype=torch.float64,
                     device="cuda")
    ens = lat.Ensemble(t, nv=nv, nx=tab.nx, L=tab.L, tau_p=tab.tau_p, kappa=tab.kappa, dt=tab.dt)
    ens.set_scheme(lat.SCHEME_KOREN, MU)
    ens.set_flow_modes(fl.k, fl.amp0, fl.tau_f, fl.sigma)
    ens.set_noise(fl.noise)
    ens.step(nsteps)
    assert ens.status() == 0
    for i in range(len(tab.nx)):
        nx = int(tab.nx[i])
        dv = (tab.L[i] / nx) / tab.dt[i]
        want, _ = K.run_1d(parts[i], nsteps, tau_p=tab.tau_p[i], kappa=tab.kappa[i],
                           dt=tab.dt[i], dv=dv, k=fl.k, amp0=fl.amp0[i], tau_f=fl.tau_f,
                           sigma=fl.sigma, noise=fl.noise[:, i, :], mu=MU)
        got = ens.instance_view(i).cpu().numpy()
        assert rel_l1(got, want) <= 1e-12, (i, rel_l1(got, want))
    ens.close()


def test_full_size_ensemble_sampled(lat):
    """The benchmark ensemble (4096 instances, N_v = 65, FP32) with the limited scheme, autotuned
    launch shape: eight sampled instances against the oracle after 10 steps; mass and
    positivity of the whole ensemble."""
    nv, nsteps, n = 65, 10, 4096
    tab = I.ensemble_table(n, 2024, nv=nv, cfl_factor=1 + MU)
    fl = I.flow1d_inputs(2025, nsteps, n_inst=n)
    f0 = I.ensemble_initial(tab, nv, torch.float32, "cuda")
    ens = lat.Ensemble(f0, nv=nv, nx=tab.nx, L=tab.L, tau_p=tab.tau_p, kappa=tab.kappa,
                       dt=tab.dt)
    ens.set_scheme(lat.SCHEME_KOREN, MU)
    ens.set_flow_modes(fl.k, fl.amp0, fl.tau_f, fl.sigma)
    ens.set_noise(fl.noise)
    ens.autotune(reps=2)
    ens.step(nsteps)
    assert ens.status() == 0
    rng = np.random.default_rng(1)
    sample = sorted(int(i) for i in rng.choice(n, 8, replace=False))
    parts = I.ensemble_initial(tab, nv, None, None, instances=sample)
    for i in sample:
        nx = int(tab.nx[i])
        dv = (tab.L[i] / nx) / tab.dt[i]
        want, _ = K.run_1d(parts[i], nsteps, tau_p=tab.tau_p[i], kappa=tab.kappa[i],
                           dt=tab.dt[i], dv=dv, k=fl.k, amp0=fl.amp0[i], tau_f=fl.tau_f,
                           sigma=fl.sigma, noise=fl.noise[:, i, :], mu=MU)
        got = ens.instance_view(i).double().cpu().numpy()
        assert rel_l1(got, want) <= 1e-5, (i, rel_l1(got, want))
    code, _, _, _, glob = ens.moments()
    assert code == 0
    np.testing.assert_allclose(glob[:, 0], 1.0, rtol=1e-5)
    assert float(ens.state.min()) >= -1e-6 * float(ens.state.max())
    ens.close()


def test_mass_and_positivity_over_many_steps(lat):
    c = case(512, 65, 0.1, 1e-3, 500, 21)
    got, lt = run_gpu(lat, c, torch.float32)
    code, _, _, _, glob = lt.moments(per_cell=False)
    assert code == 0
    m0 = c["f0"].sum() * (L / c["nx"]) * c["dv"]
    assert abs(glob[0] - m0) <= 1e-5 * m0
    assert got.min() >= -1e-6 * got.max()
    lt.close()


def test_host_checks(lat):
    c = case(64, 33, 1.0, 1e-3, 1, 1)
    t = torch.tensor(c["f0"], dtype=torch.float32, device="cuda")
    # (dt / tau_p) J = 0.8: fine for the upwind step, too long for the limited one (x 5/3)
    dt = 0.1
    lt = lat.Lattice(t.clone(), d=1, nx=64, nv=33, L=L, tau_p=dt * 16 / 0.8, kappa=1e-3, dt=dt)
    with pytest.raises(lat.LatError) as e:
        lt.set_scheme(lat.SCHEME_KOREN, MU)
    assert e.value.code == lat.LAT_ECFL
    with pytest.raises(lat.LatError) as e:
        lt.set_scheme(lat.SCHEME_KOREN, 0.0)
    assert e.value.code == lat.LAT_EINVAL
    lt.set_scheme(lat.SCHEME_UPWIND)
    lt.close()
    f7 = torch.zeros((7, 64), device="cuda")  # N_v = 7 runs in the runtime-N_v kernel only
    lt = lat.Lattice(f7, d=1, nx=64, nv=7, L=L, tau_p=L, kappa=1e-3, dt=c["dt"])
    with pytest.raises(lat.LatError) as e:
        lt.set_scheme(lat.SCHEME_KOREN, MU)
    assert e.value.code == lat.LAT_EINVAL
    lt.close()
    f2 = torch.zeros((9, 9, 16, 16), dtype=torch.float16, device="cuda")
    lt = lat.Lattice(f2, d=2, nx=16, ny=16, nv=9, L=L, tau_p=L, kappa=1e-3, dt=0.05)
    with pytest.raises(lat.LatError) as e:  # 16-bit storage keeps the upwind scheme
        lt.set_scheme(lat.SCHEME_KOREN, MU)
    assert e.value.code == lat.LAT_EINVAL
    lt.close()


# ---- 2D: the scheme of the paper's 2D runs ------------------------------------------------------
def case2d(nx, ny, nv, st, kappa, nsteps, seed, mu=MU):
    tau_p = st * L
    dt = I.choose_dt(2, nx, L, nv, tau_p, kappa, cfl_factor=1 + mu)
    dx = L / nx
    dv = dx / dt
    rng = np.random.default_rng(seed)
    J = (nv - 1) // 2
    f0 = I.gaussian_initial_2d(nx, ny, nv, dx, dv, 0.3 * J * dv)
    f0 = f0 * (1 + 0.5 * rng.random((1, 1, ny, nx)))
    fl = I.flow2d_inputs(seed, nsteps, nx, ny, dx, kmax=3)
    return dict(nx=nx, ny=ny, nv=nv, tau_p=tau_p, kappa=kappa, dt=dt, dx=dx, dv=dv, f0=f0,
                fl=fl, nsteps=nsteps, mu=mu)


def oracle2d(c):
    fl = c["fl"]
    f = c["f0"].copy()
    phi = fl.phi0.copy()
    for n in range(c["nsteps"]):
        ux, uy = O.flow2d_u(fl.a, fl.kvec, phi, c["nx"], c["ny"], c["dx"])
        f = K.step_2d(f, ux, uy, c["tau_p"], c["kappa"], c["dt"], c["dv"], c["mu"])
        phi = O.phase_advance(phi, fl.noise[n], c["dt"], fl.tau_f)
    return f


def gpu2d(lat, c, dtype, launch=None):
    t = torch.tensor(c["f0"], dtype=dtype, device="cuda")
    lt = lat.Lattice(t, d=2, nx=c["nx"], ny=c["ny"], nv=c["nv"], L=L, tau_p=c["tau_p"],
                     kappa=c["kappa"], dt=c["dt"])
    lt.set_scheme(lat.SCHEME_KOREN, c["mu"])
    if launch:
        lt.set_launch(**launch)
    fl = c["fl"]
    lt.set_flow_modes_2d(fl.kvec, fl.a, fl.phi0, fl.tau_f)
    lt.set_noise(fl.noise)
    lt.step(c["nsteps"])
    assert lt.status() == 0
    return lt.state.double().cpu().numpy(), lt


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("nx,ny,nv,mu", [(48, 40, 9, MU), (33, 20, 5, 1.0), (24, 24, 17, MU)])
def test_2d_matches_oracle(lat, dtype, nx, ny, nv, mu):
    c = case2d(nx, ny, nv, 1.0, 2e-3, 30, nx + nv, mu=mu)
    want = oracle2d(c)
    got, lt = gpu2d(lat, c, dtype)
    assert rel_l1(got, want) <= TOL[dtype], rel_l1(got, want)
    lt.close()


def test_2d_33x33_matches_oracle(lat):
    """The velocity lattice of the 2D configurations (33^2), on a ragged 40 x 36 grid."""
    for dtype in (torch.float64, torch.float32):
        c = case2d(40, 36, 33, 1.0, 2e-3, 8, 91)
        want = oracle2d(c)
        got, lt = gpu2d(lat, c, dtype)
        assert rel_l1(got, want) <= TOL[dtype], (dtype, rel_l1(got, want))
        lt.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("nx,ny,nv,st", [(70, 24, 5, 1.0), (100, 31, 9, 0.1), (40, 20, 13, 1.0),
                                         (64, 20, 17, 1.0), (97, 40, 19, 10.0),
                                         (50, 26, 21, 1.0), (45, 34, 33, 0.5)])
def test_2d_fused_gives_the_three_pass_bits(lat, dtype, nx, ny, nv, st):
    """One kernel per step (tiles of 32, or of 16 and 8 cells for the larger FP64 and N_v = 33
    planes; ragged and odd N_x), scalar and on FP32 register pairs, against the three passes:
    the same faces with the same operations, so equal values (a skipped zero part can change
    only the sign of a zero)."""
    c = case2d(nx, ny, nv, st, 2e-3, 12, nx + 7 * nv)
    ref, lt = gpu2d(lat, c, dtype, launch=dict(kernel=1))
    lt.close()
    shapes = [dict(kernel=2, blocks_per_sm=1), dict(kernel=2, blocks_per_sm=2)]
    if dtype == torch.float32:
        shapes.append(dict(kernel=3))  # cell pairs in FP32 register pairs
    for launch in shapes:
        got, lt = gpu2d(lat, c, dtype, launch=launch)
        lt.close()
        assert np.array_equal(got, ref), (launch, np.abs(got - ref).max())


def test_2d_launch_forms(lat):
    c = case2d(48, 40, 3, 1.0, 2e-3, 2, 5)  # N_v = 3: three passes only
    t = torch.tensor(c["f0"], dtype=torch.float32, device="cuda")
    lt = lat.Lattice(t, d=2, nx=48, ny=40, nv=3, L=L, tau_p=c["tau_p"], kappa=c["kappa"],
                     dt=c["dt"])
    lt.set_scheme(lat.SCHEME_KOREN, MU)
    with pytest.raises(lat.LatError) as e:
        lt.set_launch(kernel=2)
    assert e.value.code == lat.LAT_EINVAL
    with pytest.raises(lat.LatError) as e:
        lt.set_launch(kernel=5)
    assert e.value.code == lat.LAT_EINVAL
    with pytest.raises(lat.LatError) as e:
        lt.set_launch(kernel=3)
    assert e.value.code == lat.LAT_EINVAL
    lt.set_launch(kernel=1)
    lt.step(2)
    assert lt.status() == 0
    lt.close()


def test_2d_mass_and_positivity(lat):
    c = case2d(128, 96, 17, 0.5, 1e-3, 200, 3)
    got, lt = gpu2d(lat, c, torch.float32)
    code, *_, g = lt.moments(per_cell=False)
    assert code == 0
    m0 = c["f0"].sum() * c["dx"] ** 2 * c["dv"] ** 2
    assert abs(g[0] - m0) <= 1e-5 * m0
    assert got.min() >= -1e-6 * got.max()
    lt.close()


def test_2d_cellular_flow_limited_matches_oracle(lat):
    """The paper's 2D set-up of Sec. 4.1: tilted cellular flow, 19^2 velocities, limited drag."""
    n, nv = 40, 19
    tau_p, kappa = 1.0, 8 * math.pi * 1e-3
    dt = I.choose_dt(2, n, L, nv, tau_p, kappa, u_rms=0.1, cfl_factor=1 + MU)
    dx = L / n
    dv = dx / dt
    f0 = I.gaussian_initial_2d(n, n, nv, dx, dv, 0.3 * ((nv - 1) // 2) * dv)
    ux, uy = I.cellular_flow(n, n, L, 1.0)
    want = f0.copy()
    for _ in range(25):
        want = K.step_2d(want, ux, uy, tau_p, kappa, dt, dv, MU)
    lt = lat.Lattice(torch.tensor(f0, device="cuda"), d=2, nx=n, ny=n, nv=nv, L=L, tau_p=tau_p,
                     kappa=kappa, dt=dt)
    lt.set_scheme(lat.SCHEME_KOREN, MU)
    u = torch.tensor(np.stack([ux, uy]), device="cuda")
    lt.set_flow_field(u)
    lt.step(25)
    assert lt.status() == 0
    assert rel_l1(lt.state.cpu().numpy(), want) <= 1e-12
    lt.close()


def test_2d_full_size_cellular_sampled(lat):
    """The bench's flux-limited form at full size: 1024^2 x 19^2 FP32 (3.8e8 phase cells), the
    tilted cellular flow, the default launch (the fused kernel on FP32 pairs).  One step from a
    seeded random state; 32 sampled cells recomputed by the oracle one by one from their
    gathered f* (the limited step acts on each cell's velocity plane), with the FP32 flow values
    the kernel reads."""
    n, nv = 1024, 19
    tau_p, kappa = 1.0, 8 * math.pi * 1e-3
    dt = I.choose_dt(2, n, L, nv, tau_p, kappa, u_rms=0.1, cfl_factor=1 + MU)
    dx = L / n
    dv = dx / dt
    gen = torch.Generator(device="cuda")
    gen.manual_seed(17)
    f0 = torch.rand((nv, nv, n, n), generator=gen, device="cuda") + 0.1
    lt = lat.Lattice(f0.clone(), d=2, nx=n, ny=n, nv=nv, L=L, tau_p=tau_p, kappa=kappa, dt=dt)
    lt.set_scheme(lat.SCHEME_KOREN, MU)
    ux, uy = I.cellular_flow(n, n, L, 1.0)
    u = torch.tensor(np.stack([ux, uy]), dtype=torch.float32, device="cuda")
    lt.set_flow_field(u)
    u64 = u.double().cpu().numpy()
    lt.step(1)
    assert lt.status() == 0
    out = lt.state
    rng = np.random.default_rng(23)
    J = (nv - 1) // 2
    jj = np.arange(nv)
    xs0 = list(rng.integers(n, size=28)) + [0, n - 1, 5, n - 3]  # and cells near the wraps
    ys0 = list(rng.integers(n, size=28)) + [n - 1, 0, n - 2, 3]
    for x, y in zip(xs0, ys0):
        x, y = int(x), int(y)
        ys = [(y - (jy - J)) % n for jy in range(nv)]
        xs = [(x - (jx - J)) % n for jx in range(nv)]
        block = f0[:, :, ys][:, :, :, xs].double().cpu().numpy()
        col = block[jj[:, None], jj[None, :], jj[:, None], jj[None, :]]  # f*(x, y; jx, jy)
        uxc = np.array([[u64[0, y, x]]])
        uyc = np.array([[u64[1, y, x]]])
        want = O.diffuse_2d(K.drag_2d(col[:, :, None, None], uxc, uyc, tau_p, dt, dv, MU),
                            kappa, dt, dv)[:, :, 0, 0]
        got = out[:, :, y, x].double().cpu().numpy()
        assert rel_l1(got, want) <= 1e-6, (x, y, rel_l1(got, want))
    lt.close()

