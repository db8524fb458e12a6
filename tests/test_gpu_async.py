"""lat_step_moments_async: the steps and the globals of lat_step_moments without the stream
synchronisation.  The same kernels run in the same order, so the states and the globals read
from the caller's pinned buffers equal the synchronous call's bit for bit; the device status of
the steps comes with the next synchronising call."""
import math

import numpy as np
import pytest
import torch

from paper_1508_02899_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L = 2 * math.pi


def ensemble(lat):
    tab = I.ensemble_table(6, 11, nv=33, sizes=(256, 512, 1024, 132))
    parts = [I.random_initial((33, int(n)), i) for i, n in enumerate(tab.nx)]
    t = torch.tensor(np.concatenate([p.ravel() for p in parts]), dtype=torch.float32,
                     device="cuda")
    return lat.Ensemble(t, nv=33, nx=tab.nx, L=tab.L, tau_p=tab.tau_p, kappa=tab.kappa,
                        dt=tab.dt), (6, 3)


def lattice2d(lat, dtype, nv=17, kernel=None):
    nx, ny = 256, 24
    tau_p, kappa = L, 1e-3
    dt = I.choose_dt(2, nx, L, nv, tau_p, kappa)
    f0 = torch.tensor(I.random_initial((nv, nv, ny, nx), 2), dtype=dtype, device="cuda")
    lt = lat.Lattice(f0, d=2, nx=nx, ny=ny, nv=nv, L=L, tau_p=tau_p, kappa=kappa, dt=dt)
    if kernel:
        lt.set_launch(kernel=kernel)
    return lt, (4,)


def run_pair(make, steps=4):
    a, shape = make()
    b, _ = make()
    want = []
    for _ in range(steps):
        code, *_, g = a.step_moments(1, per_cell=False, globals_out=np.zeros(shape))
        assert code == 0
        want.append(g.copy())
    outs = [torch.zeros(shape, dtype=torch.float64).pin_memory() for _ in range(steps)]
    for k in range(steps):
        b.step_moments_async(1, outs[k])
    torch.cuda.synchronize()
    assert b.status() == 0
    assert torch.equal(a.state, b.state)
    for k in range(steps):
        assert np.array_equal(outs[k].numpy(), want[k]), k
    assert a.steps_done == b.steps_done == steps
    a.close()
    b.close()


def test_ensemble_async_equals_sync(lat):
    run_pair(lambda: ensemble(lat))


@pytest.mark.parametrize("kernel", [9, 1])  # fused moments; a separate pass
def test_2d_async_equals_sync(lat, kernel):
    run_pair(lambda: lattice2d(lat, torch.float32, kernel=kernel))


def test_16bit_async_equals_sync(lat):
    run_pair(lambda: lattice2d(lat, torch.float16))


def test_async_arguments_and_status(lat):
    lt, shape = lattice2d(lat, torch.float32)
    out = torch.zeros(shape, dtype=torch.float64).pin_memory()
    with pytest.raises(lat.LatError) as e:
        lt.step_moments_async(0, out)
    assert e.value.code == lat.LAT_EINVAL
    with pytest.raises(ValueError):  # pageable host memory is refused by the binding
        lt.step_moments_async(1, torch.zeros(shape, dtype=torch.float64))
    # a non-finite value met by the fused epilogue is reported by the next synchronising call
    lt.state.view(-1)[1000] = float("nan")
    lt.step_moments_async(1, out)
    torch.cuda.synchronize()
    assert lt.status() == lat.LAT_ENUMERIC
    lt.close()
