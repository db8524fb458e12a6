"""Flux-limited drag sub-step of the phase-space lattice: plain FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or execute this
module: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the CUDA library.

Section 2 of the paper offers, besides the first-order upwind drag step, a flux-limiter scheme
after Hundsdorfer et al. (1995): a higher-order interface flux where f is smooth, lowered towards
upwind near strong gradients by a nonlinear function of the ratio of consecutive differences,
total-variation diminishing (TVD) so that it stays stable; the limiter is Koren's (1993) "with
parameter 2/3".  Readings K1-K3, taken here:

* K1  Koren's limiter in Hundsdorfer et al.'s form.  The value carried through interface
      j+1/2 from its upwind side is q_j + psi(theta_j) (q_{j+1} - q_j), with
      theta_j = (q_j - q_{j-1}) / (q_{j+1} - q_j) and
          psi(theta) = max(0, min(1, 1/3 + theta/6, mu theta)),
      the limited kappa = 1/3 scheme.  mu bounds psi(theta)/theta; the paper's "parameter 2/3"
      is read as mu = 2/3 (mu = 1 is the limiter's usual form; both are accepted).  Where
      q_{j+1} = q_j the increment is zero (psi is bounded).
* K2  With the cell-centre force of reading R3 the upwind flux is a flux-vector splitting,
      F_{j+1/2} = P_j + M_{j+1} with P = a^+ f, M = a^- f.  The limiter acts on each split
      flux from its own upwind side:
          F_{j+1/2} = P_j + psi(theta^P_j) (P_{j+1} - P_j)
                    + M_{j+1} + psi(theta^M_{j+1}) (M_j - M_{j+1}),
          theta^P_j = (P_j - P_{j-1}) / (P_{j+1} - P_j),
          theta^M_{j+1} = (M_{j+1} - M_{j+2}) / (M_j - M_{j+1}).
      Cells beyond the walls count as empty (P, M = 0 there); the wall fluxes stay zero.
* K3  The limited sub-step is integrated by Heun's two-stage method (the explicit trapezoidal
      rule, which Hundsdorfer et al. pair with the limited scheme):
          f1 = f + dt L(f),  f2 = f1 + dt L(f1),  f_new = (f + f2) / 2,
      L(f) = -(F_{j+1/2} - F_{j-1/2}) / dv, with u frozen at t_n (reading R4).  Each stage is a
      forward-Euler step, positive when the Courant number nu = (dt/dv) max|a| obeys
      nu (1 + mu) <= 1 (psi <= 1 and psi/theta <= mu), so the average is positive too.

Layouts are the lattice oracle's: 1D f[j, x]; 2D f[jy, jx, y, x].
"""
from __future__ import annotations

import numpy as np

from . import lattice as O

MU_DEFAULT = 2.0 / 3.0


def koren_psi(theta: np.ndarray, mu: float) -> np.ndarray:
    """psi(theta) = max(0, min(1, 1/3 + theta/6, mu theta))  (K1)."""
    return np.maximum(0.0, np.minimum(np.minimum(1.0, 1.0 / 3.0 + theta / 6.0), mu * theta))


def _increment(q_up2: np.ndarray, q_up: np.ndarray, q_down: np.ndarray, mu: float) -> np.ndarray:
    """psi(theta) (q_down - q_up), theta = (q_up - q_up2) / (q_down - q_up); zero where
    q_down = q_up."""
    dp = q_down - q_up
    dm = q_up - q_up2
    nz = dp != 0.0
    theta = np.divide(dm, dp, out=np.zeros_like(dp), where=nz)
    return np.where(nz, koren_psi(theta, mu) * dp, 0.0)


def limited_fluxes(a: np.ndarray, f: np.ndarray, mu: float) -> np.ndarray:
    """Interface fluxes of d_t f + d_v (a f) = 0 along axis 0 (K1, K2).

    a, f: (N, ...) cell-centre speeds and densities.  Returns F (N + 1, ...): F[k] is the flux
    through the interface below cell k, zero at both walls.
    """
    n = f.shape[0]
    P = np.maximum(a, 0.0) * f
    M = np.minimum(a, 0.0) * f
    pad = [(2, 2)] + [(0, 0)] * (f.ndim - 1)
    Pp = np.pad(P, pad)  # Pp[k + 2] = P_k, zero beyond the walls
    Mp = np.pad(M, pad)
    F = np.zeros((n + 1,) + f.shape[1:])
    for j in range(n - 1):  # interior interface j + 1/2 = F[j + 1]
        k = j + 2
        pos = Pp[k] + _increment(Pp[k - 1], Pp[k], Pp[k + 1], mu)
        neg = Mp[k + 1] + _increment(Mp[k + 2], Mp[k + 1], Mp[k], mu)
        F[j + 1] = pos + neg
    return F


def _stage_1d(f, a, c, mu):
    F = limited_fluxes(a, f, mu)
    return f - c * (F[1:] - F[:-1])


def drag_1d(f: np.ndarray, u: np.ndarray, tau_p: float, dt: float, dv: float,
            mu: float = MU_DEFAULT) -> np.ndarray:
    """Limited drag sub-step (K1-K3) of f (N_v, N_x) with fluid velocity u (N_x,)."""
    nv = f.shape[0]
    v = O.velocities(nv, dv)
    a = O.drag_acceleration(v[:, None], u[None, :], tau_p) * np.ones_like(f)
    c = dt / dv
    f1 = _stage_1d(f, a, c, mu)
    f2 = _stage_1d(f1, a, c, mu)
    return 0.5 * (f + f2)


def step_1d(f, u, tau_p, kappa, dt, dv, mu=MU_DEFAULT):
    """Stream, limited drag, diffusion (reading R4 with K1-K3)."""
    return O.diffuse_1d(drag_1d(O.stream_1d(f), u, tau_p, dt, dv, mu), kappa, dt, dv)


def run_1d(f0, nsteps, *, tau_p, kappa, dt, dv, k, amp0, tau_f, sigma, noise, field=None,
           mu=MU_DEFAULT):
    """lattice.run_1d with the limited drag sub-step."""
    f = np.array(f0, dtype=np.float64, copy=True)
    amp = np.array(amp0, dtype=np.float64, copy=True)
    nx = f.shape[1]
    for n in range(nsteps):
        u = field if field is not None else O.flow1d_u(amp, k, nx)
        f = step_1d(f, u, tau_p, kappa, dt, dv, mu)
        if field is None:
            amp = O.ou_advance(amp, noise[n], dt, tau_f, sigma)
    return f, amp


def drag_2d(f: np.ndarray, ux: np.ndarray, uy: np.ndarray, tau_p: float, dt: float, dv: float,
            mu: float = MU_DEFAULT) -> np.ndarray:
    """Unsplit limited drag sub-step in 2D (reading R5 with K1-K3): each stage applies the
    limited flux differences of both velocity axes to the same state."""
    nv = f.shape[0]
    v = O.velocities(nv, dv)
    ax = O.drag_acceleration(v[None, :, None, None], ux[None, None], tau_p) * np.ones_like(f)
    ay = O.drag_acceleration(v[:, None, None, None], uy[None, None], tau_p) * np.ones_like(f)
    c = dt / dv

    def stage(g):
        Fy = limited_fluxes(ay, g, mu)
        Fx = np.moveaxis(limited_fluxes(np.moveaxis(ax, 1, 0), np.moveaxis(g, 1, 0), mu), 0, 1)
        return g - c * (Fx[:, 1:] - Fx[:, :-1]) - c * (Fy[1:] - Fy[:-1])

    f1 = stage(f)
    f2 = stage(f1)
    return 0.5 * (f + f2)


def step_2d(f, ux, uy, tau_p, kappa, dt, dv, mu=MU_DEFAULT):
    return O.diffuse_2d(drag_2d(O.stream_2d(f), ux, uy, tau_p, dt, dv, mu), kappa, dt, dv)
