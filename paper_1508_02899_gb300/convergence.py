"""Convergence of the lattice with the velocity resolution (Sec. 3.2, the paper's first-order claim).

The paper's one-dimensional set-up: V_max = u_rms = 1, L = 2 pi, tau_f = 1, a fixed time step
dt = dx / dv = 2^-6 pi, N_v = 2^n + 1 discrete velocities and N_x = 2^(n+6) cells, and a start that
is uniform in x with all the mass at v = 0.  Every resolution sees the same random flow: its
Fourier amplitudes are advanced with the same draws at the same dt.  The error of the
coarse-grained density rho_r on the boxes of a tiling of size r = L / 128 is measured against the
finest lattice of the study, in the relative L2 norm of Sec. 3.2 (spatial and time average);
the paper finds it proportional to dv.

This module is host orchestration: the lattices, their steps and the per-cell densities all run
in the library's kernels (lat.Lattice); only the 128 box sums per snapshot are formed here.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import inputs as I
from . import lat

L = 2 * math.pi
DT = math.pi / 64
BOXES = 128


def lattice(n: int, st: float, kappa: float, fl, scheme: int = lat.SCHEME_UPWIND,
            dtype=torch.float32):
    """The resolution-n lattice of the study: N_v = 2^n + 1, N_x = 2^(n+6), V_max = 1."""
    nv, nx = 2 ** n + 1, 2 ** (n + 6)
    dx = L / nx
    dv = dx / DT
    f0 = torch.zeros((nv, nx), dtype=dtype, device="cuda")
    f0[(nv - 1) // 2] = 1.0 / (L * dv)  # all the mass at v = 0, total 1
    lt = lat.Lattice(f0, d=1, nx=nx, nv=nv, L=L, tau_p=st * L, kappa=kappa, dt=DT)
    if scheme != lat.SCHEME_UPWIND:
        lt.set_scheme(scheme)
    lt.set_flow_modes_1d(fl.k, fl.amp0[0], fl.tau_f, fl.sigma)
    lt.set_noise(fl.noise[:, 0, :])
    return lt, dv


def box_density(lt, nx: int) -> np.ndarray:
    """rho_r on the BOXES boxes of width L / BOXES: per-cell densities (library) summed per box."""
    code, rho, _, _, _ = lt.moments()
    if code != 0:
        raise lat.LatError(code, "moments")
    dx = L / nx
    return rho.cpu().numpy().reshape(BOXES, nx // BOXES).sum(axis=1) * dx


def study(levels, st: float, kappa: float = 1e-3, t_end: float = 40.0, snapshots: int = 4,
          seed: int = 8, scheme: int = lat.SCHEME_UPWIND):
    """Relative L2 errors of rho_r (r = L / 128) of every level but the last against the last
    (finest) one, averaged over `snapshots` times evenly spaced up to t_end.
    Returns (dv per level, errors per level except the finest)."""
    nsteps = int(round(t_end / DT))
    fl = I.flow1d_inputs(seed, nsteps)
    marks = sorted({int(round(nsteps * (q + 1) / snapshots)) for q in range(snapshots)})
    series, dvs = [], []
    for n in levels:
        lt, dv = lattice(n, st, kappa, fl, scheme)
        dvs.append(dv)
        snaps, done = [], 0
        for m in marks:
            lt.step(m - done)
            done = m
            snaps.append(box_density(lt, 2 ** (n + 6)))
        series.append(np.array(snaps))
        lt.close()
    ref = series[-1]
    norm = math.sqrt(np.mean(ref ** 2))
    errs = [math.sqrt(np.mean((s - ref) ** 2)) / norm for s in series[:-1]]
    return np.array(dvs), np.array(errs)
