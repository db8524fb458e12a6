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
    """Adam with its moments and the parameters on the device; each step is lat_adam (the
    gradient comes back from lat_learn_grad as host floats and goes up once)."""

    def __init__(self, params: np.ndarray, lr: float, b1: float = 0.9, b2: float = 0.999,
                 eps: float = 1e-8, device="cuda"):
        self.p = torch.tensor(np.asarray(params, dtype=np.float32), device=device)
        self.m = torch.zeros_like(self.p)
        self.v = torch.zeros_like(self.p)
        self.g = torch.zeros_like(self.p)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, g: np.ndarray, scale: float = 1.0) -> np.ndarray:
        """Apply the gradient g (times scale); returns the new parameters (host float32)."""
        self.t += 1
        self.g.copy_(torch.from_numpy(np.asarray(g, dtype=np.float32)))
        lat.adam(self.p, self.m, self.v, self.g, self.t, self.lr, self.b1, self.b2, self.eps,
                 scale)
        return self.p.cpu().numpy()


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
    # f0 = G(vx) G(vy) m(x, y) with unit mass, built on the device one velocity row at a time
    v = np.arange(-J, J + 1, dtype=np.float64) * dv_f
    g = np.exp(-0.5 * (v / (0.3 * J * dv_f)) ** 2)
    col = np.outer(g, g)
    m = 1 + 0.5 * np.random.default_rng(init_seed).random((ny, nx))
    colt = torch.tensor(col / col.sum(), dtype=torch.float64, device=device)
    mt = torch.tensor(m / (m.sum() * dx * dx * dv_f * dv_f), dtype=torch.float64, device=device)
    ff = torch.empty((nv_fine, nv_fine, ny, nx), dtype=torch.float32, device=device)
    for jy in range(nv_fine):
        ff[jy] = (colt[jy][:, None, None] * mt[None]).float()
    del mt
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
          fine_steps: int = 1, rho_weight: float = 0.0, log=None, mode: int = 1) -> np.ndarray:
    """Adam on the loss of 4 * fine_steps coarse steps from a restricted state at a random fine
    step k of a random trajectory against the restricted state at k + fine_steps, normalised by
    the target's mean square so that every sample weighs alike.  mode: the network whose
    gradient lat_learn_grad takes (1: FP32 on CUDA cores; 2: BF16 on the tensor cores, forward
    and backward)."""
    params = init_params(seed, scale)
    opt = Adam(params, lr)
    rng = np.random.default_rng(seed)
    for p in pairs:
        p.coarse.learn(params, mode)
    for it in range(iters):
        q = int(rng.integers(0, len(pairs)))
        p, states = pairs[q], trajectories[q]
        k = int(rng.integers(0, len(states) - fine_steps))
        c = p.coarse
        c.f[c.current_index].copy_(states[k])
        target = states[k + fine_steps]
        loss, g = c.learn_grad(COARSE_PER_FINE * fine_steps, target, rho_weight)
        w = 1.0 / float((target.double() ** 2).mean())
        params = opt.step(g, w)
        for pp in pairs:
            pp.coarse.learn(params, mode)
        if log is not None:
            log(it, loss * w)
    return params


def observables(lt: lat.Lattice, dx: float, r: int):
    """<|v|^2> = E / M (lat_moments) and <rho_r^2> of Eq. (def_coarse) for windows of r x r cells,
    averaged over every position (lat_coarse_moment); dx is unused (kept for callers)."""
    code, _, _, _, g = lt.moments(per_cell=False)
    rho2 = float(lt.coarse_moment([r])[0, 0])
    return g[3] / g[0], rho2, code


def evaluate(params, n: int, nv_fine: int, st: float, kappa: float, flow_seed: int,
             init_seed: int, times, r: int, kmax: int = 4, mode: int = 2):
    """Relative errors of <|v|^2> and <rho_r^2> of the plain coarse lattice and of the coarse
    lattice with the closure (network mode `mode`) against the fine lattice, in one frozen flow,
    at the fine steps `times`.  Returns {"plain": [(ev, er), ...], "learned": [...]}."""
    base = make_pair(n, n, nv_fine, st, kappa, flow_seed=flow_seed, init_seed=init_seed,
                     kmax=kmax)
    learned = make_pair(n, n, nv_fine, st, kappa, flow_seed=flow_seed, init_seed=init_seed,
                        kmax=kmax)
    learned.fine.close()
    learned.coarse.learn(params, mode)
    base.fine.set_launch(kernel=0)
    base.fine.autotune(reps=2)
    out = {"plain": [], "learned": []}
    done = 0
    for k in sorted(times):
        base.fine.step(k - done)
        base.coarse.step(COARSE_PER_FINE * (k - done))
        learned.coarse.step(COARSE_PER_FINE * (k - done))
        done = k
        vf, rf, cf = observables(base.fine, base.dx, r)
        if cf != 0:
            raise lat.LatError(cf, "fine lattice")
        for name, lt in (("plain", base.coarse), ("learned", learned.coarse)):
            v, rr, code = observables(lt, base.dx, r)
            if code != 0:
                raise lat.LatError(code, name)
            out[name].append((abs(v - vf) / vf, abs(rr - rf) / rf))
    for lt in (base.fine, base.coarse, learned.coarse):
        lt.close()
    return out


def save_params(path: str, params: np.ndarray, **recipe):
    np.savez(path, params=np.asarray(params, dtype=np.float32),
             recipe=np.array(repr(sorted(recipe.items()))))


def load_params(path: str) -> np.ndarray:
    with np.load(path) as z:
        p = np.asarray(z["params"], dtype=np.float32)
    if p.size != lat.LEARN_NPARAM:
        raise ValueError(f"{path}: {p.size} parameters, expected {lat.LEARN_NPARAM}")
    return p


def main(argv=None):
    """Train the closure on GPU fine runs and write its parameters (np.savez); optionally
    evaluate them.  Pairs of every listed grid size and flow seed (frozen random-phase flows,
    N_v 33 -> 9, St = 1, kappa = 1e-3) supply restricted fine trajectories; each Adam iteration
    takes one pair and one start at random."""
    import argparse
    import json
    import time
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--sizes", default="128,256")
    ap.add_argument("--seeds", default="101,102")
    ap.add_argument("--iters", type=int, default=400)
    ap.add_argument("--kmax", type=int, default=8)
    ap.add_argument("--fine-steps", type=int, default=4)
    ap.add_argument("--traj", type=int, default=40)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--rho-weight", type=float, default=0.3)
    ap.add_argument("--mode", type=int, default=1, help="1: FP32 network, 2: tensor cores")
    ap.add_argument("--out", required=True)
    ap.add_argument("--eval", default="",
                    help="evaluations n:times:r[;...] after training, e.g. 2048:100,400:16")
    a = ap.parse_args(argv)
    sizes = [int(v) for v in a.sizes.split(",")]
    seeds = [int(v) for v in a.seeds.split(",")]
    t0 = time.time()
    pairs = [make_pair(n, n, 33, 1.0, 1e-3, flow_seed=s + n, init_seed=s + n + 7, kmax=a.kmax)
             for n in sizes for s in seeds]
    trajs = [restricted_trajectory(p, a.traj) for p in pairs]
    for p in pairs:
        p.fine.close()

    def log(it, loss):
        if it % 50 == 0:
            print(f"iter {it} loss {loss:.4e} ({time.time() - t0:.0f} s)", flush=True)

    params = train(pairs, trajs, a.iters, lr=a.lr, seed=1, fine_steps=a.fine_steps,
                   rho_weight=a.rho_weight, log=log, mode=a.mode)
    save_params(a.out, params, sizes=sizes, seeds=seeds, iters=a.iters, kmax=a.kmax, mode=a.mode,
                fine_steps=a.fine_steps, traj=a.traj, lr=a.lr, rho_weight=a.rho_weight)
    print(f"wrote {a.out} after {time.time() - t0:.0f} s", flush=True)
    for p in pairs:
        p.coarse.close()
    del pairs, trajs
    torch.cuda.empty_cache()
    for spec in filter(None, a.eval.split(";")):
        n, times, r = spec.split(":")
        times = [int(v) for v in times.split(",")]
        e = evaluate(params, int(n), 33, 1.0, 1e-3, flow_seed=505, init_seed=506, times=times,
                     r=int(r), kmax=a.kmax, mode=2)
        print(json.dumps({"n": int(n), "r_cells": int(r), "fine_steps": times,
                          "plain": e["plain"], "learned": e["learned"]}), flush=True)
        torch.cuda.empty_cache()


if __name__ == "__main__":
    main()
