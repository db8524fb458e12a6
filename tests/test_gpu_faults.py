"""The device status paths that guard the method's stability and the pipelines' waits, driven
through the C ABI without faulting the GPU.

- LAT_ENUMERIC: a non-finite density value, put into the caller's buffer from the host, is found
  by the moment reduction (lat_moments) and by the moment epilogue of the fused step
  (lat_step_moments), in 1D and 2D.
- LAT_EOVERFLOW: a 16-bit state holding the format's infinity (a line maximum that no scale can
  bring into range), or a host density too large for FP32, is reported by the next step or by
  lat_set_density.
- LAT_ETIMEOUT: with the stall hook on, the producer warps of the bulk-copy pipelines issue no
  copies, so the consumers' bounded waits give up after about a second; the step reports the
  timeout, and the context keeps working once the hook is off.  No copy is in flight when a wait
  gives up.
"""
import math
import time

import numpy as np
import pytest
import torch

from paper_1508_02899_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L = 2 * math.pi


def lattice1d(lat, dtype, nx=264, nv=33):
    tau_p, kappa = L, 1e-3
    dt = I.choose_dt(1, nx, L, nv, tau_p, kappa)
    t = torch.tensor(I.random_initial((nv, nx), 1), dtype=dtype, device="cuda")
    return lat.Lattice(t, d=1, nx=nx, nv=nv, L=L, tau_p=tau_p, kappa=kappa, dt=dt)


def lattice2d(lat, dtype, nx=136, ny=16, nv=17, f0=None):
    tau_p, kappa = L, 1e-3
    dt = I.choose_dt(2, nx, L, nv, tau_p, kappa)
    if f0 is None:
        f0 = torch.tensor(I.random_initial((nv, nv, ny, nx), 2), dtype=dtype, device="cuda")
    return lat.Lattice(f0, d=2, nx=nx, ny=ny, nv=nv, L=L, tau_p=tau_p, kappa=kappa, dt=dt)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("d", [1, 2])
def test_nonfinite_value_gives_enumeric(lat, d, dtype):
    lt = lattice1d(lat, dtype) if d == 1 else lattice2d(lat, dtype)
    lt.step(2)
    assert lt.status() == lat.LAT_OK
    good = lt.state.clone()
    flat = lt.state.view(-1)
    flat[flat.numel() // 3] = float("nan")
    code = lt.moments()[0]
    assert code == lat.LAT_ENUMERIC
    assert lt.status() == lat.LAT_OK  # read and cleared
    flat[flat.numel() // 3] = float("inf")
    assert lt.moments(per_cell=False)[0] == lat.LAT_ENUMERIC
    # the fused epilogue (1D producer/consumer kernel, 2D FP32 launch kernels 4 and 5) sees the
    # non-finite value it writes
    code = lt.step_moments(1)[0]
    assert code == lat.LAT_ENUMERIC
    # a finite state clears it
    lt.state.copy_(good)
    assert lt.moments()[0] == lat.LAT_OK
    lt.step(1)
    assert lt.status() == lat.LAT_OK
    lt.close()


@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16])
def test_infinite_16bit_value_gives_eoverflow(lat, dtype):
    """The caller's initial 16-bit buffer (scale 1) holds the format's infinity in one cell: its
    line maximum is at the overflow, so the next step's scale pass and encoder flag it."""
    nx, ny, nv = 136, 16, 17
    f0 = torch.tensor(I.random_initial((nv, nv, ny, nx), 3), dtype=dtype, device="cuda")
    f0[nv // 2, nv // 2, 5, 17] = float("inf")
    lt = lattice2d(lat, dtype, nx, ny, nv, f0=f0)
    lt.step(1)
    assert lt.status() == lat.LAT_EOVERFLOW
    lt.close()


@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16])
def test_density_beyond_fp32_gives_eoverflow(lat, dtype):
    nx, ny, nv = 136, 16, 17
    lt = lattice2d(lat, dtype, nx, ny, nv,
                   f0=torch.zeros((nv, nv, ny, nx), dtype=dtype, device="cuda"))
    x = I.random_initial((nv, nv, ny, nx), 4).ravel()
    lt.set_density(x)
    x[1234] = 1e300
    with pytest.raises(lat.LatError) as e:
        lt.set_density(x)
    assert e.value.code == lat.LAT_EOVERFLOW
    lt.close()


def _stalled_step_times_out(lat, lt):
    lt.step(2)
    assert lt.status() == lat.LAT_OK
    good = lt.state.clone()
    lt.debug_stall(True)
    t0 = time.perf_counter()
    lt.step(1)
    code = lt.status()
    waited = time.perf_counter() - t0
    lt.debug_stall(False)
    assert code == lat.LAT_ETIMEOUT, code
    assert 0.5 < waited < 30.0, waited
    # the context and the GPU keep working: restore a good state and step on
    lt.state.copy_(good)
    lt.step(3)
    assert lt.status() == lat.LAT_OK
    assert torch.isfinite(lt.state.float()).all()
    return waited


def test_stalled_pipeline_1d_ensemble_times_out(lat):
    tab = I.ensemble_table(4, 3, nv=33, sizes=(256, 512, 1024, 132))
    parts = [I.random_initial((33, int(n)), i) for i, n in enumerate(tab.nx)]
    t = torch.tensor(np.concatenate([p.ravel() for p in parts]), dtype=torch.float32,
                     device="cuda")
    ens = lat.Ensemble(t, nv=33, nx=tab.nx, L=tab.L, tau_p=tab.tau_p, kappa=tab.kappa,
                       dt=tab.dt)
    ens.set_launch(kernel=5)  # producer/consumer, two slots (the default shape)
    _stalled_step_times_out(lat, ens)
    ens.close()


@pytest.mark.parametrize("kernel", [3, 5])
def test_stalled_pipeline_2d_times_out(lat, kernel):
    lt = lattice2d(lat, torch.float32)
    lt.set_launch(kernel=kernel)
    _stalled_step_times_out(lat, lt)
    lt.close()


def test_stalled_pipeline_16bit_times_out(lat):
    nx, ny, nv = 136, 16, 17
    lt = lattice2d(lat, torch.float16, nx, ny, nv,
                   f0=torch.zeros((nv, nv, ny, nx), dtype=torch.float16, device="cuda"))
    lt.encode(torch.tensor(I.random_initial((nv, nv, ny, nx), 5), dtype=torch.float32,
                           device="cuda"))
    lt.set_launch(kernel=6)
    lt.step(2)
    assert lt.status() == lat.LAT_OK
    good = lt.get_state()
    lt.debug_stall(True)
    lt.step(1)
    code = lt.status()
    lt.debug_stall(False)
    assert code == lat.LAT_ETIMEOUT, code
    lt.set_state(good)  # the state, its scales and maxima as they were
    lt.step(3)
    assert lt.status() == lat.LAT_OK
    dec, _ = lt.decode()
    assert torch.isfinite(dec).all()
    lt.close()


def test_plain_loads_ignore_the_stall_hook(lat):
    lt = lattice2d(lat, torch.float32)
    lt.set_launch(kernel=1)
    lt.debug_stall(True)
    lt.step(2)
    assert lt.status() == lat.LAT_OK
    lt.debug_stall(False)
    lt.close()
