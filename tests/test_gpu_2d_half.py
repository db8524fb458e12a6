"""16-bit (FP16 / BF16) storage of the 2D lattice, through the C ABI, against the storage oracle
(oracle/storage16.py on top of the FP64 step) and against the FP64 GPU run.

Tolerances.  The GPU computes a step in FP32 and the oracle in FP64, so before encoding the two
differ by FP32 rounding, about 2^-21 of the stencil's values.  That can move a value across a
rounding boundary of the 16-bit code: the stored value then differs by one storage step (at most
2^-10 of it in FP16, 2^-7 in BF16), and the different residual shifts the next value of the
column by as much.  So a value may differ by one step of itself and one of its predecessor,
plus the FP32 rounding.  The carry also hands a large line's FP32 rounding (2^-24 of a value)
to the next, possibly much smaller, line of the column, where it can be a visible fraction of
that line's storage step; so a few per cent of the values differ by one step (an FP32 emulation
of the kernel on the CPU gives the same values bit for bit).  Scales are compared exactly: both
sides derive them from the same line maxima with the same integer rule.
"""
import math

import numpy as np
import pytest
import torch

from oracle import lattice as O
from oracle import storage16 as S16
from paper_1508_02899_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L = 2 * math.pi
TDT = {"f16": torch.float16, "bf16": torch.bfloat16}
STEP = {"f16": 2.0**-10, "bf16": 2.0**-7}       # largest storage step relative to the value
SIG = {"f16": 10, "bf16": 7}                     # fraction bits


def quantised(f, fmt):
    """f with, on every x-line, only the significant bits the line's scale can hold exactly
    (multiples of 2^(ilogb(line max) - SIG)), so that encoding it leaves no residual."""
    mx = np.abs(f).max(axis=3, keepdims=True)
    _, e = np.frexp(mx)
    q = np.ldexp(1.0, e - 1 - SIG[fmt])
    return (np.rint(f / q) * q).astype(np.float32)


def setup(nx, ny, nv, st, kappa, nsteps, seed, gauss=True):
    tau_p = st * L
    dt = I.choose_dt(2, nx, L, nv, tau_p, kappa)
    dx = L / nx
    dv = dx / dt
    J = (nv - 1) // 2
    if gauss:
        f0 = I.gaussian_initial_2d(nx, ny, nv, dx, dv, 0.3 * max(J, 1) * dv)
        rng = np.random.default_rng(seed)
        f0 = f0 * (1 + 0.3 * rng.random((1, 1, ny, nx)))  # spatial structure
    else:
        f0 = I.random_initial((nv, nv, ny, nx), seed)
    fl = I.flow2d_inputs(seed, nsteps, nx, ny, dx, kmax=4)
    return dict(nx=nx, ny=ny, nv=nv, tau_p=tau_p, kappa=kappa, dt=dt, dx=dx, dv=dv, f0=f0, fl=fl)


def lattice16(lat, c, fmt, src32, kernel=0):
    buf = torch.zeros(src32.shape, dtype=TDT[fmt], device="cuda")
    lt = lat.Lattice(buf, d=2, nx=c["nx"], ny=c["ny"], nv=c["nv"], L=L, tau_p=c["tau_p"],
                     kappa=c["kappa"], dt=c["dt"])
    if kernel:
        lt.set_launch(kernel=kernel)
    lt.encode(torch.tensor(src32, device="cuda"))
    fl = c["fl"]
    lt.set_flow_modes_2d(fl.kvec, fl.a, fl.phi0, fl.tau_f)
    lt.set_noise(fl.noise)
    return lt


def decoded(lt):
    dec, sc = lt.decode()
    return dec.double().cpu().numpy(), sc.double().cpu().numpy().reshape(lt.nv, lt.nv, lt.ny)


def column_tolerance(want, fmt, scale_of_stencil):
    nv, _, ny, nx = want.shape
    w = np.abs(want).reshape(nv * nv, ny, nx)
    prev = np.concatenate([np.zeros((1, ny, nx)), w[:-1]])
    return (STEP[fmt] * (w + prev)).reshape(want.shape) + 2.0**-20 * scale_of_stencil


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_encode_matches_oracle(lat, fmt):
    c = setup(48, 20, 9, 1.0, 1e-3, 1, 3)
    src = c["f0"].astype(np.float32)
    lt = lattice16(lat, c, fmt, src)
    got, sc = decoded(lt)
    want, S, _ = S16.encode_state(src.astype(np.float64), fmt)
    np.testing.assert_array_equal(sc, S)
    # the GPU forms value + carry in FP32: a rounding may differ at the last bit of the sum
    tol = column_tolerance(want, fmt, np.abs(src).max(axis=3, keepdims=True))
    assert np.all(np.abs(got - want) <= tol)
    assert np.mean(got == want) > 0.9
    lt.close()


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
@pytest.mark.parametrize("kernel", [1, 4, 5, 6, 7])
def test_one_and_two_steps_match_oracle(lat, fmt, kernel):
    """N_x = 144: two tiles, the second ragged; windows that wrap in x; 9 x 9 velocities."""
    c = setup(144, 12, 9, 1.0, 2e-3, 2, 7 + kernel)
    x0 = quantised(c["f0"], fmt)
    lt = lattice16(lat, c, fmt, x0, kernel)
    got0, _ = decoded(lt)
    np.testing.assert_array_equal(got0, x0)  # exact encoding: no residual anywhere
    fl = c["fl"]
    ux, uy = O.flow2d_u(fl.a, fl.kvec, fl.phi0, c["nx"], c["ny"], c["dx"])
    want1, S1, mx1, over = S16.step_2d_stored(x0.astype(np.float64), S16.line_max(x0), ux, uy,
                                              tau_p=c["tau_p"], kappa=c["kappa"], dt=c["dt"],
                                              dv=c["dv"], fmt=fmt)
    assert not over
    lt.step(1)
    assert lt.status() == 0
    got1, sc1 = decoded(lt)
    np.testing.assert_array_equal(sc1, S1)
    tol = column_tolerance(want1, fmt, 4096 * S1[..., None])
    assert np.all(np.abs(got1 - want1) <= tol), np.max(np.abs(got1 - want1) / tol)
    assert np.mean(got1 == want1) > 0.9
    # second step: the scales come from the line maxima the first step recorded
    phi1 = O.phase_advance(fl.phi0, fl.noise[0], c["dt"], fl.tau_f)
    ux, uy = O.flow2d_u(fl.a, fl.kvec, phi1, c["nx"], c["ny"], c["dx"])
    want2, S2, _, _ = S16.step_2d_stored(want1, mx1, ux, uy, tau_p=c["tau_p"],
                                         kappa=c["kappa"], dt=c["dt"], dv=c["dv"], fmt=fmt)
    lt.step(1)
    assert lt.status() == 0
    got2, sc2 = decoded(lt)
    assert np.mean(sc2 == S2) > 0.999
    tol = column_tolerance(want2, fmt, 4096 * S2[..., None]) * 2
    assert np.all(np.abs(got2 - want2) <= tol), np.max(np.abs(got2 - want2) / tol)
    lt.close()


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_launch_variants_give_the_same_bits(lat, fmt):
    c = setup(272, 10, 17, 1.0, 1e-3, 12, 5)
    src = c["f0"].astype(np.float32)
    outs = []
    for kernel in (1, 4, 5, 6, 7):
        lt = lattice16(lat, c, fmt, src, kernel)
        lt.step(12)
        assert lt.status() == 0
        outs.append(lt.state.view(torch.int16).cpu().numpy().copy())
        outs.append(decoded(lt)[1])
        lt.close()
    for k in range(2, len(outs), 2):
        assert np.array_equal(outs[0], outs[k]), k // 2
        assert np.array_equal(outs[1], outs[k + 1]), k // 2


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_free_streaming_is_exact(lat, fmt):
    nx, ny, nv = 144, 10, 9
    rng = np.random.default_rng(4)
    f0 = quantised(rng.random((nv, nv, ny, nx)) + 0.5, fmt)
    buf = torch.zeros(f0.shape, dtype=TDT[fmt], device="cuda")
    for kernel in (1, 5, 7):
        lt = lat.Lattice(buf.clone(), d=2, nx=nx, ny=ny, nv=nv, L=L, tau_p=math.inf, kappa=0.0,
                         dt=0.1)
        lt.set_launch(kernel=kernel)
        lt.encode(torch.tensor(f0, device="cuda"))
        lt.step(5)
        assert lt.status() == 0
        J = (nv - 1) // 2
        want = np.empty_like(f0)
        for jy in range(nv):
            for jx in range(nv):
                want[jy, jx] = np.roll(f0[jy, jx], (5 * (jy - J), 5 * (jx - J)), axis=(0, 1))
        assert np.array_equal(decoded(lt)[0], want.astype(np.float64))
        lt.close()


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_moments_of_the_stored_state(lat, fmt):
    c = setup(64, 32, 9, 1.0, 1e-3, 3, 9)
    lt = lattice16(lat, c, fmt, c["f0"].astype(np.float32))
    lt.step(3)
    dec, _ = decoded(lt)
    code, rho, mv, mv2, glob = lt.moments()
    assert code == 0
    rho_o, mvx_o, mvy_o, mv2_o, glob_o = O.moments_2d(dec, c["dx"], c["dv"])
    # mass compensated; weighted sums one FMA per value: error at most (N_v^2 - 1) u of the sum
    # of |weight f| (u = 2^-24)
    nv = c["nv"]
    u = 2.0**-24
    v = (np.arange(nv) - (nv - 1) // 2) * c["dv"]
    w2 = (v[None, :] ** 2 + v[:, None] ** 2)[:, :, None, None]
    np.testing.assert_allclose(rho.cpu().numpy().reshape(rho_o.shape), rho_o, rtol=1e-12)
    col = (nv * nv - 1) * u * (w2 * dec).sum(axis=(0, 1)) / dec.sum(axis=(0, 1))
    got2 = mv2.cpu().numpy().reshape(mv2_o.shape)
    assert np.all(np.abs(got2 - mv2_o) <= col + 1e-13 * np.abs(mv2_o))
    cell = c["dx"] ** 2 * c["dv"] ** 2
    assert abs(glob[0] - glob_o[0]) <= 1e-12 * abs(glob_o[0])
    for q, w in ((1, np.abs(v)[None, :, None, None]), (2, np.abs(v)[:, None, None, None]), (3, w2)):
        bound = (nv * nv - 1) * u * float((w * np.abs(dec)).sum()) * cell
        assert abs(glob[q] - glob_o[q]) <= bound + 1e-14 * abs(glob_o[q]), q
    lt.close()


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_long_run_against_fp64(lat, fmt):
    """128^2 x 33^2, St = 1, random-phase flow, 100 steps: mass, <|v|^2> and <rho_r^2> of the
    16-bit run against the FP64 run from the same initial values."""
    c = setup(128, 128, 33, 1.0, 1e-3, 100, 13)
    x0 = quantised(c["f0"], fmt)
    lt = lattice16(lat, c, fmt, x0)
    t64 = torch.tensor(x0.astype(np.float64), device="cuda")
    l64 = lat.Lattice(t64, d=2, nx=c["nx"], ny=c["ny"], nv=c["nv"], L=L, tau_p=c["tau_p"],
                      kappa=c["kappa"], dt=c["dt"])
    fl = c["fl"]
    l64.set_flow_modes_2d(fl.kvec, fl.a, fl.phi0, fl.tau_f)
    l64.set_noise(fl.noise)
    m0 = lt.moments(per_cell=False)[4]
    lt.step(100)
    l64.step(100)
    code, rho, _, _, g16 = lt.moments()
    code64, rho64, _, _, g64 = l64.moments()
    assert code == 0 and code64 == 0
    # the FP64 run the 16-bit one is measured against matches the oracle at 1e-12
    want, _ = O.run_2d(x0.astype(np.float64), 100, tau_p=c["tau_p"], kappa=c["kappa"],
                       dt=c["dt"], dv=c["dv"], dx=c["dx"], kvec=fl.kvec, a=fl.a, phi0=fl.phi0,
                       tau_f=fl.tau_f, noise=fl.noise)
    got64 = l64.state.cpu().numpy()
    err64 = np.abs(got64 - want).sum() / np.abs(want).sum()
    assert err64 <= 1e-12, err64
    # mass: the carried residuals keep it at the FP32 arithmetic level (the FP64 run: 1e-15)
    e16, e64 = g16[3] / g16[0], g64[3] / g64[0]
    print(f"\n[{fmt}] mass drift {abs(g16[0] - m0[0]) / m0[0]:.3e}  <|v|^2> rel diff "
          f"{abs(e16 - e64) / e64:.3e}", end="")
    assert abs(g16[0] - m0[0]) / m0[0] < 1e-8, abs(g16[0] - m0[0]) / m0[0]
    assert abs(e16 - e64) / e64 < 2 * STEP[fmt] / 8, (e16, e64)
    r16 = rho.cpu().numpy().reshape(c["ny"], c["nx"])
    r64 = rho64.cpu().numpy().reshape(c["ny"], c["nx"])
    for r in (4, 16):
        a = S16.coarse_density_moment(r16, c["dx"], r)
        b = S16.coarse_density_moment(r64, c["dx"], r)
        print(f"  <rho_{r}^2> rel diff {abs(a - b) / b:.3e}", end="")
        assert abs(a - b) / b < 2 * STEP[fmt] / 8, (r, a, b)
    lt.close()
    l64.close()
