"""The allocation-free moment entry point, called through the C ABI.

lat_moments1d_noalloc serves callers that must not allocate device memory: code running inside
another runtime that has reserved the GPU's memory, or latency-critical loops where cudaMalloc
or cudaFree would synchronise the device.  It keeps its scratch in a static device array.  This
test checks that two calls in a row agree with the globals of lat_moments, the entry point
that allocates its scratch in the context, and that oversized inputs are rejected before
anything runs.

The file name makes pytest collect it last.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

from paper_1508_02899_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L = 2 * math.pi


def _noalloc(lat, f, nv, nx, dx, dv, out):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lat._lib.lat_moments1d_noalloc(ctypes.c_void_p(f.data_ptr()), nv, nx, dx, dv,
                                          ctypes.c_void_p(out.data_ptr()), stream)


def test_noalloc_moments_match_context_moments(lat):
    nx, nv = 3000, 33  # 24 tiles, ragged last tile
    tau_p, kappa = L, 1e-3
    dt = I.choose_dt(1, nx, L, nv, tau_p, kappa)
    dx = L / nx
    dv = dx / dt
    f0 = I.gaussian_initial_1d(nx, nv, dx, dv, 0.2 * 16 * dv)
    fl = I.flow1d_inputs(4242, 20)
    lt = lat.Lattice(torch.tensor(f0, dtype=torch.float32, device="cuda"), d=1, nx=nx, nv=nv,
                     L=L, tau_p=tau_p, kappa=kappa, dt=dt)
    lt.set_flow_modes_1d(fl.k, fl.amp0[0], fl.tau_f, fl.sigma)
    lt.set_noise(fl.noise[:, 0, :])
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    for call in range(2):
        lt.step(7)
        code, _, _, _, want = lt.moments(per_cell=False)
        assert code == 0
        out.fill_(float("nan"))
        assert _noalloc(lat, lt.state, nv, nx, dx, dv, out) == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        # Both sides sum every column in the same FP32 order (the mass by TwoSum, the weighted
        # sums by FMA).  They differ in how columns
        # combine: FP64 Neumaier here; FP32 TwoSum merges (exact but for the rounding of the
        # error term, about u^2 = 2^-48 of a partial per merge, five merges per warp) then
        # FP64 in the context.  So |got - want| <= 1e-13 * sum|terms| of each moment.
        fa = np.abs(lt.state.double().cpu().numpy())
        v = (np.arange(nv) - (nv - 1) // 2) * dv
        mag = np.array([fa.sum(), (np.abs(v)[:, None] * fa).sum(), ((v * v)[:, None] * fa).sum()])
        assert np.all(np.abs(got - want) <= 1e-13 * mag * dx * dv), (call, got, want)
    lt.close()


def test_noalloc_rejects_oversized_input(lat):
    f = torch.zeros(16, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    too_big = 8192 * 128 + 1
    assert _noalloc(lat, f, 1, too_big, 1.0, 1.0, out) == lat.LAT_EINVAL
    assert _noalloc(lat, f, 2, 8, 1.0, 1.0, out) == lat.LAT_EINVAL
