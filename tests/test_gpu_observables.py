"""Parity of the observables (lat_coarse_moment, lat_s1) with oracle/observables.py on states the
GPU lattice produced: FP64 states at 1e-12; FP32 states with S1's velocity sums in FP32 within
their bound; ragged ensembles per instance; 2D lattices with FP64 and 16-bit storage."""
import math

import numpy as np
import pytest
import torch

from oracle import observables as B
from paper_1508_02899_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L = 2 * math.pi
U32 = 2.0**-24


def lattice1d(lat, nx, nv, dtype, seed, nsteps=30):
    tau_p = 0.3 * L
    dt = I.choose_dt(1, nx, L, nv, tau_p, 1e-3)
    f0 = I.random_initial((nv, nx), seed)
    lt = lat.Lattice(torch.tensor(f0, dtype=dtype, device="cuda"), d=1, nx=nx, nv=nv, L=L,
                     tau_p=tau_p, kappa=1e-3, dt=dt)
    fl = I.flow1d_inputs(seed, nsteps)
    lt.set_flow_modes_1d(fl.k, fl.amp0[0], fl.tau_f, fl.sigma)
    lt.set_noise(fl.noise[:, 0, :])
    lt.step(nsteps)
    assert lt.status() == 0
    return lt, L / nx, (L / nx) / dt


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_1d_coarse_moment_and_s1(lat, dtype):
    nx, nv = 300, 33
    lt, dx, dv = lattice1d(lat, nx, nv, dtype, 7)
    f = lt.state.double().cpu().numpy()
    widths = [1, 2, 7, 64, 299, 300]
    got = lt.coarse_moment(widths)[0]
    np.testing.assert_allclose(got, B.coarse_moment(f, dx, dv, widths), rtol=1e-12)
    seps = [0, 1, 5, 150, 299]
    num, den = lt.s1(seps)
    want_n, want_d = B.s1_terms(f, dv, seps)
    np.testing.assert_allclose(den[0], want_d, rtol=1e-12)
    # FP64: 1e-12; FP32: the running sums round at u = 2^-24, about N_v u of the positive terms
    # each, four such sums per pair
    np.testing.assert_allclose(num[0], want_n, rtol=1e-12 if dtype == torch.float64
                               else 4 * nv * U32)
    assert np.all(num[0] / den[0] > 0)
    lt.close()


def test_ensemble_per_instance(lat):
    nv = 17
    tab = I.ensemble_table(5, 3, nv=nv, sizes=(40, 257, 100, 64, 33))
    parts = [I.random_initial((nv, int(n)), 50 + i) for i, n in enumerate(tab.nx)]
    t = torch.tensor(np.concatenate([p.ravel() for p in parts]), dtype=torch.float64,
                     device="cuda")
    ens = lat.Ensemble(t, nv=nv, nx=tab.nx, L=tab.L, tau_p=tab.tau_p, kappa=tab.kappa, dt=tab.dt)
    ens.step(3)
    assert ens.status() == 0
    widths = [1, 4, int(tab.nx.min())]
    seps = [0, 3, int(tab.nx.min()) - 1]
    cm = ens.coarse_moment(widths)
    num, den = ens.s1(seps)
    for i in range(len(tab.nx)):
        f = ens.instance_view(i).cpu().numpy()
        dx = tab.L[i] / tab.nx[i]
        dv = dx / tab.dt[i]
        np.testing.assert_allclose(cm[i], B.coarse_moment(f, dx, dv, widths), rtol=1e-12)
        wn, wd = B.s1_terms(f, dv, seps)
        np.testing.assert_allclose(num[i], wn, rtol=1e-12)
        np.testing.assert_allclose(den[i], wd, rtol=1e-12)
    with pytest.raises(lat.LatError) as e:
        ens.coarse_moment([int(tab.nx.min()) + 1])
    assert e.value.code == lat.LAT_EINVAL
    with pytest.raises(lat.LatError) as e:
        ens.s1([int(tab.nx.min())])
    assert e.value.code == lat.LAT_EINVAL
    ens.close()


def test_2d_coarse_moment(lat):
    nx, ny, nv = 64, 48, 9
    rng = np.random.default_rng(5)
    f0 = rng.random((nv, nv, ny, nx)) ** 2
    dt = I.choose_dt(2, nx, L, nv, L, 1e-3)
    lt = lat.Lattice(torch.tensor(f0, dtype=torch.float64, device="cuda"), d=2, nx=nx, ny=ny,
                     nv=nv, L=L, tau_p=L, kappa=1e-3, dt=dt)
    fl = I.flow2d_inputs(5, 4, nx, ny, L / nx)
    lt.set_flow_modes_2d(fl.kvec, fl.a, fl.phi0, fl.tau_f)
    lt.set_noise(fl.noise)
    lt.step(4)
    assert lt.status() == 0
    f = lt.state.cpu().numpy()
    dx, dv = L / nx, (L / nx) / dt
    widths = [1, 3, 17, 48]
    np.testing.assert_allclose(lt.coarse_moment(widths)[0], B.coarse_moment(f, dx, dv, widths),
                               rtol=1e-12)
    with pytest.raises(lat.LatError) as e:
        lt.s1([1])
    assert e.value.code == lat.LAT_EINVAL
    lt.close()


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_2d_coarse_moment_of_16bit_storage(lat, fmt):
    nx, ny, nv = 144, 16, 9
    rng = np.random.default_rng(6)
    src = torch.tensor(rng.random((nv, nv, ny, nx)) + 0.1, dtype=torch.float32, device="cuda")
    dt = I.choose_dt(2, nx, L, nv, L, 1e-3)
    buf = torch.zeros(src.shape, dtype=torch.float16 if fmt == "f16" else torch.bfloat16,
                      device="cuda")
    lt = lat.Lattice(buf, d=2, nx=nx, ny=ny, nv=nv, L=L, tau_p=L, kappa=1e-3, dt=dt)
    lt.encode(src)
    lt.step(2)
    assert lt.status() == 0
    vals, _ = lt.decode()
    f = vals.double().cpu().numpy()
    dx, dv = L / nx, (L / nx) / dt
    widths = [1, 5, 16]
    np.testing.assert_allclose(lt.coarse_moment(widths)[0], B.coarse_moment(f, dx, dv, widths),
                               rtol=1e-12)
    lt.close()
