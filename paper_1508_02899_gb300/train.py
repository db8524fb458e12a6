"""Training of the learned flux closure of a coarse 2D lattice against a restricted fine lattice.

A fine lattice (N_v = 4m + 1 per axis, FP32, plain step) and a coarse one (N_v = m + 1, the same
dx and V_max, so dv four times larger and dt four times smaller) are advanced in the same frozen
random-phase flow.  The fine run's states, restricted to the coarse lattice (lat.restrict), are
the training data: from the restricted state at fine step k, four coarse steps of the learned
step should land on the restricted state at fine step k + 1.  Gradients come from
lat_learn_grad (the adjoint of the four coarse steps, on the GPU); Adam updates the 5378
parameters.  The paper proposes large-eddy closures for the lattice (Section 5); the network,
the features and the flux form are this library's choice (include/lat.h, lat_learn).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

from . import inputs as I
from . import lat

COARSE_PER_FINE = 4
NF, NH, NO = 16, 64, 2


def init_params(seed: int, scale: float = 0.1) -> np.ndarray:
    """He-normal weights times `scale`, zero biases, packed like lat_learn expects."""
    rng = np.random.default_rng(seed)
    w1 = rng.standard_normal((NF, NH)) * math.sqrt(2.0 / NF) * scale
    w2 = rng.standard_normal((NH, NH)) * math.sqrt(2.0 / NH) * scale
    w3 = rng.standard_normal((NH, NO)) * math.sqrt(2.0 / NH) * scale
    return np.concatenate([w1.ravel(), np.zeros(NH), w2.ravel(), np.zeros(NH), w3.ravel(),
                           np.zeros(NO)]).astype(np.float32)


class Adam:
    def __init__(self, n: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, p: np.ndarray, g: np.ndarray) -> np.ndarray:
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return (p - self.lr * mh / (np.sqrt(vh) + self.eps)).astype(np.float32)


@dataclass
class Pair:
    fine: lat.Lattice
    coarse: lat.Lattice
    nx: int
    ny: int
    nv_fine: int
    dx: float


def make_pair(nx: int, ny: int, nv_fine: int, st: float, kappa: float, flow_seed: int,
              init_seed: int, device="cuda", kmax: int = 4) -> Pair:
    """Fine and coarse lattices in the same frozen flow, the coarse one starting from the
    restriction of the fine initial state (Gaussian in v, sigma = 0.3 V_max, spatially modulated)."""
    L = 2 * math.pi
    tau_p = st * L
    dt_f = I.choose_dt(2, nx, L, nv_fine, tau_p, kappa)
    dx = L / nx
    dv_f = dx / dt_f
    J = (nv_fine - 1) // 2
    f0 = I.gaussian_initial_2d(nx, ny, nv_fine, dx, dv_f, 0.3 * J * dv_f)
    rng = np.random.default_rng(init_seed)
    f0 = f0 * (1 + 0.5 * rng.random((1, 1, ny, nx)))
    f0 = f0 / (f0.sum() * dx * dx * dv_f * dv_f)
    ff = torch.tensor(f0, dtype=torch.float32, device=device)
    fine = lat.Lattice(ff, d=2, nx=nx, ny=ny, nv=nv_fine, L=L, tau_p=tau_p, kappa=kappa, dt=dt_f)
    fc = lat.restrict(ff, nx, ny)
    nv_c = (nv_fine - 1) // 4 + 1
    coarse = lat.Lattice(fc, d=2, nx=nx, ny=ny, nv=nv_c, L=L, tau_p=tau_p, kappa=kappa,
                         dt=dt_f / COARSE_PER_FINE)
    fl = I.flow2d_inputs(flow_seed, 1, nx, ny, dx, kmax=kmax)
    for lt in (fine, coarse):
        lt.set_flow_modes_2d(fl.kvec, fl.a, fl.phi0, math.inf)  # frozen
    fine.set_launch(kernel=1)
    return Pair(fine, coarse, nx, ny, nv_fine, dx)


def restricted_trajectory(p: Pair, nsteps: int):
    """Restricted fine states at fine steps 0..nsteps (device tensors)."""
    out = [lat.restrict(p.fine.state, p.nx, p.ny)]
    for _ in range(nsteps):
        p.fine.step(1)
        out.append(lat.restrict(p.fine.state, p.nx, p.ny))
    return out


def train(pairs, trajectories, iters: int, lr: float = 1e-3, seed: int = 0, scale: float = 0.1,
          fine_steps: int = 1, rho_weight: float = 0.0, log=None) -> np.ndarray:
    """Adam on the loss of 4 * fine_steps coarse steps from a restricted state at a random fine
    step k of a random trajectory against the restricted state at k + fine_steps, normalised by
    the target's mean square so that every sample weighs alike."""
    params = init_params(seed, scale)
    opt = Adam(params.size, lr)
    rng = np.random.default_rng(seed)
    for p in pairs:
        p.coarse.learn(params, 1)
    for it in range(iters):
        q = int(rng.integers(0, len(pairs)))
        p, states = pairs[q], trajectories[q]
        k = int(rng.integers(0, len(states) - fine_steps))
        c = p.coarse
        c.f[c.current_index].copy_(states[k])
        target = states[k + fine_steps]
        loss, g = c.learn_grad(COARSE_PER_FINE * fine_steps, target, rho_weight)
        w = 1.0 / float((target.double() ** 2).mean())
        params = opt.step(params, g.astype(np.float64) * w)
        for pp in pairs:
            pp.coarse.learn(params, 1)
        if log is not None:
            log(it, loss * w)
    return params


def observables(lt: lat.Lattice, dx: float, r: int):
    """<|v|^2> = E / M and <rho_r^2> (mass in r x r boxes, mean square) of a lattice."""
    code, rho, _, _, g = lt.moments()
    rho = rho.cpu().numpy().reshape(lt.ny, lt.nx)
    boxes = rho.reshape(lt.ny // r, r, lt.nx // r, r).sum(axis=(1, 3)) * dx * dx
    return g[3] / g[0], float(np.mean(boxes * boxes)), code
