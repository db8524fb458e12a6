"""Plain FP64 CPU oracle of the phase-space lattice method for heavy inertial particles.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or execute this
module: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the CUDA library.

What it computes (Laenen, Krstulovic & Bec, "A lattice model for the Eulerian description of
heavy particle suspensions", arXiv:1508.02899):

* the phase-space density f(x, v, t) is piecewise constant on a lattice of N_x^d spatial cells
  times N_v^d velocity cells, every particle of a cell sitting at its centre (Section 2);
* the lattice obeys dx = dv * dt, so velocity index j moves mass by exactly j cells per step
  (Section 2);
* one time step is an operator splitting: exact streaming in x, then a finite-volume step of
  the force term, then a finite-volume step of the velocity diffusion, with zero flux through
  the walls of the velocity box (Section 2);
* the force is the Stokes drag of Eq. (stokes_drag): a = F/m_p = -(v - u(x, t)) / tau_p,
  evaluated at the cell-centre velocities; the drag step is first-order upwind, stable when the
  CFL number of Eq. (cfl) is below one; the diffusion step is the finite-difference interface
  flux kappa (f_{j+1} - f_j)/dv, stable when kappa dt / dv^2 < 1/2 (Eq. stabLapl).

Readings R1-R6, taken where the paper is silent or ambiguous:

* R1  dv = 2 V_max / (N_v - 1): cell centres j*dv, j = -J..J, J = (N_v-1)/2 (Section 2 and the
      caption of Fig. 14 disagree; this is the reading that reproduces the time step of Sec. 3.2).
* R2  the sign of the force term: Eq. (conslaw) prints it with a minus sign; the particle
      dynamics of Eq. (stokes_drag) fixes d_t f + d_v (a f) = kappa d_v^2 f, which is used here.
* R3  upwinding with the cell-centre force: flux through interface j+1/2 is
      a_j^+ f_j + a_{j+1}^- f_{j+1}  (x^+ = max(x,0), x^- = min(x,0)).
* R4  Lie splitting in the order stream -> drag -> diffusion, the drag using u at the
      post-stream position and the pre-step time t_n.
* R5  in two dimensions both velocity components are updated in one unsplit sub-step (drag),
      and the diffusion is the unsplit five-point Laplacian in (jx, jy).
* R6  positions x_i = i dx, i = 0..N_x-1, periodic.

The flows are the synthetic stand-ins for the paper's carrier flows (Sec. 3.1 Eq. u1d/A1d, in an
8-mode generalisation; Sec. 4.2 replaced by an incompressible random-phase flow).  Their random
draws are inputs; the Ornstein-Uhlenbeck updates and the field evaluation are computed here.

Array layouts (identical to the CUDA library's, so results compare element by element):
    1D  f[j, x]           shape (N_v, N_x)
    2D  f[jy, jx, y, x]   shape (N_v, N_v, N_y, N_x)
"""
from __future__ import annotations

import math

import numpy as np


# --------------------------------------------------------------------------------------------
# Velocity lattice (Section 2, reading R1)
# --------------------------------------------------------------------------------------------
def velocities(nv: int, dv: float) -> np.ndarray:
    """Cell-centre velocities v_j = j dv, j = -J..J (Section 2)."""
    if nv < 1 or nv % 2 == 0:
        raise ValueError("N_v must be odd")
    J = (nv - 1) // 2
    return np.arange(-J, J + 1, dtype=np.float64) * dv


def drag_acceleration(v: np.ndarray, u: np.ndarray, tau_p: float) -> np.ndarray:
    """Deterministic part of Eq. (stokes_drag): a = -(v - u) / tau_p (broadcasting)."""
    return -(v - u) / tau_p


# --------------------------------------------------------------------------------------------
# One dimension
# --------------------------------------------------------------------------------------------
def stream_1d(f: np.ndarray) -> np.ndarray:
    """Exact lattice advection (Section 2): the mass of velocity cell j moves j cells in x.

    out[j, x] = f[j, (x - j) mod N_x].
    """
    nv, _ = f.shape
    J = (nv - 1) // 2
    out = np.empty_like(f)
    for jj in range(nv):
        out[jj] = np.roll(f[jj], jj - J)  # np.roll(a, s)[i] = a[(i - s) mod n]
    return out


def drag_1d(f: np.ndarray, u: np.ndarray, tau_p: float, dt: float, dv: float) -> np.ndarray:
    """First-order upwind finite-volume step of d_t f + d_v (a f) = 0 (Section 2, R2, R3).

    f: (N_v, N_x) after streaming; u: (N_x,) fluid velocity at the cell positions.
    Interface fluxes F_{j+1/2} = a_j^+ f_j + a_{j+1}^- f_{j+1}; zero at both walls.
    f_j <- f_j - (dt/dv) (F_{j+1/2} - F_{j-1/2}).
    """
    nv, nx = f.shape
    v = velocities(nv, dv)
    a = drag_acceleration(v[:, None], u[None, :], tau_p)
    ap = np.maximum(a, 0.0)
    am = np.minimum(a, 0.0)
    F = np.zeros((nv + 1, nx))  # F[k] is the flux through the interface below cell k
    F[1:-1] = ap[:-1] * f[:-1] + am[1:] * f[1:]
    return f - (dt / dv) * (F[1:] - F[:-1])


def diffuse_1d(f: np.ndarray, kappa: float, dt: float, dv: float) -> np.ndarray:
    """Finite-volume velocity diffusion (Section 2, Eq. stabLapl).

    Interface flux D_{j+1/2} = kappa (f_{j+1} - f_j) / dv, zero at both walls;
    f_j <- f_j + (dt/dv) (D_{j+1/2} - D_{j-1/2}): a discrete Laplacian in v.
    """
    nv, nx = f.shape
    D = np.zeros((nv + 1, nx))
    D[1:-1] = kappa * (f[1:] - f[:-1]) / dv
    return f + (dt / dv) * (D[1:] - D[:-1])


def step_1d(f: np.ndarray, u: np.ndarray, tau_p: float, kappa: float, dt: float,
            dv: float) -> np.ndarray:
    """One lattice time step (Section 2, R4): stream, then drag, then diffusion."""
    fs = stream_1d(f)
    fd = drag_1d(fs, u, tau_p, dt, dv)
    return diffuse_1d(fd, kappa, dt, dv)


def moments_1d(f: np.ndarray, dx: float, dv: float):
    """Velocity moments of f (Sec. 3.2 normalisation, Sec. 4.2 density by summing over v).

    Returns per-cell rho = sum_j f dv, <v> = sum_j v_j f / sum_j f, <v^2> likewise (0 where
    rho = 0), and the global sums [M, P, E] = sum f dx dv * [1, v, v^2], each formed with
    math.fsum (correctly rounded) over the products.
    """
    nv, nx = f.shape
    v = velocities(nv, dv)
    rho = np.array([math.fsum(f[:, i]) for i in range(nx)]) * dv
    m1 = np.array([math.fsum(v * f[:, i]) for i in range(nx)]) * dv
    m2 = np.array([math.fsum(v * v * f[:, i]) for i in range(nx)]) * dv
    with np.errstate(invalid="ignore", divide="ignore"):
        mean_v = np.where(rho != 0.0, m1 / rho, 0.0)
        mean_v2 = np.where(rho != 0.0, m2 / rho, 0.0)
    glob = np.array([
        math.fsum(f.ravel()) * dx * dv,
        math.fsum((v[:, None] * f).ravel()) * dx * dv,
        math.fsum((v[:, None] * v[:, None] * f).ravel()) * dx * dv,
    ])
    return rho, mean_v, mean_v2, glob


# --------------------------------------------------------------------------------------------
# Two dimensions (Section 4; readings R5, R6)
# --------------------------------------------------------------------------------------------
def stream_2d(f: np.ndarray) -> np.ndarray:
    """out[jy, jx, y, x] = f[jy, jx, (y - jy) mod N_y, (x - jx) mod N_x] (Section 2, d = 2)."""
    nv = f.shape[0]
    J = (nv - 1) // 2
    out = np.empty_like(f)
    for jy in range(nv):
        for jx in range(nv):
            out[jy, jx] = np.roll(f[jy, jx], (jy - J, jx - J), axis=(0, 1))
    return out


def drag_2d(f: np.ndarray, ux: np.ndarray, uy: np.ndarray, tau_p: float, dt: float,
            dv: float) -> np.ndarray:
    """Unsplit first-order upwind drag step in (vx, vy) (Section 2, R3, R5).

    f: (N_v, N_v, N_y, N_x) indexed [jy, jx, y, x]; ux, uy: (N_y, N_x).
    The vx fluxes run along axis 1 with a_x = -(v_jx - ux)/tau_p, the vy fluxes along axis 0
    with a_y = -(v_jy - uy)/tau_p; both flux differences are applied to the same f.
    """
    nv = f.shape[0]
    v = velocities(nv, dv)
    ax = drag_acceleration(v[None, :, None, None], ux[None, None], tau_p)  # varies with jx
    ay = drag_acceleration(v[:, None, None, None], uy[None, None], tau_p)  # varies with jy
    axp = np.broadcast_to(np.maximum(ax, 0.0), f.shape)
    axm = np.broadcast_to(np.minimum(ax, 0.0), f.shape)
    ayp = np.broadcast_to(np.maximum(ay, 0.0), f.shape)
    aym = np.broadcast_to(np.minimum(ay, 0.0), f.shape)
    shp = f.shape
    Fx = np.zeros((shp[0], shp[1] + 1) + shp[2:])
    Fx[:, 1:-1] = axp[:, :-1] * f[:, :-1] + axm[:, 1:] * f[:, 1:]
    Fy = np.zeros((shp[0] + 1,) + shp[1:])
    Fy[1:-1] = ayp[:-1] * f[:-1] + aym[1:] * f[1:]
    c = dt / dv
    return f - c * (Fx[:, 1:] - Fx[:, :-1]) - c * (Fy[1:] - Fy[:-1])


def diffuse_2d(f: np.ndarray, kappa: float, dt: float, dv: float) -> np.ndarray:
    """Unsplit five-point velocity Laplacian with zero-flux walls (Section 2, R5)."""
    shp = f.shape
    Dx = np.zeros((shp[0], shp[1] + 1) + shp[2:])
    Dx[:, 1:-1] = kappa * (f[:, 1:] - f[:, :-1]) / dv
    Dy = np.zeros((shp[0] + 1,) + shp[1:])
    Dy[1:-1] = kappa * (f[1:] - f[:-1]) / dv
    c = dt / dv
    return f + c * (Dx[:, 1:] - Dx[:, :-1]) + c * (Dy[1:] - Dy[:-1])


def step_2d(f: np.ndarray, ux: np.ndarray, uy: np.ndarray, tau_p: float, kappa: float,
            dt: float, dv: float) -> np.ndarray:
    """One 2D lattice time step: stream, drag, diffusion (Section 2, R4, R5)."""
    return diffuse_2d(drag_2d(stream_2d(f), ux, uy, tau_p, dt, dv), kappa, dt, dv)


def moments_2d(f: np.ndarray, dx: float, dv: float):
    """Per-cell rho = sum f dv^2, <vx>, <vy>, <|v|^2>; globals [M, Px, Py, E] (fsum)."""
    nv, _, ny, nx = f.shape
    v = velocities(nv, dv)
    vx = np.broadcast_to(v[None, :, None, None], f.shape)
    vy = np.broadcast_to(v[:, None, None, None], f.shape)
    s0 = f.sum(axis=(0, 1))
    s1x = (vx * f).sum(axis=(0, 1))
    s1y = (vy * f).sum(axis=(0, 1))
    s2 = ((vx * vx + vy * vy) * f).sum(axis=(0, 1))
    rho = s0 * dv * dv
    with np.errstate(invalid="ignore", divide="ignore"):
        mvx = np.where(s0 != 0.0, s1x / s0, 0.0)
        mvy = np.where(s0 != 0.0, s1y / s0, 0.0)
        mv2 = np.where(s0 != 0.0, s2 / s0, 0.0)
    w = dx * dx * dv * dv
    glob = np.array([
        math.fsum(f.ravel()) * w,
        math.fsum((vx * f).ravel()) * w,
        math.fsum((vy * f).ravel()) * w,
        math.fsum(((vx * vx + vy * vy) * f).ravel()) * w,
    ])
    return rho, mvx, mvy, mv2, glob


# --------------------------------------------------------------------------------------------
# Synthetic carrier flows (Sec. 3.1 Eq. u1d/A1d generalised to M modes; 2D random-phase flow)
# --------------------------------------------------------------------------------------------
def flow1d_u(amp: np.ndarray, k: np.ndarray, nx: int) -> np.ndarray:
    """u(x_i) = sum_m A_m cos(2 pi k_m x_i / L) + B_m sin(2 pi k_m x_i / L), x_i = i L / N_x.

    amp = [A_0..A_{M-1}, B_0..B_{M-1}] (Eq. u1d, with M modes instead of one).
    """
    M = len(k)
    i = np.arange(nx, dtype=np.float64)
    u = np.zeros(nx)
    for m in range(M):
        th = 2.0 * math.pi * k[m] * i / nx
        u += amp[m] * np.cos(th) + amp[M + m] * np.sin(th)
    return u


def ou_advance(amp: np.ndarray, xi: np.ndarray, dt: float, tau_f: float,
               sigma: float) -> np.ndarray:
    """Exact one-step transition of the Ornstein-Uhlenbeck amplitudes of Eq. (A1d).

    A(t+dt) = A(t) e^{-dt/tau_f} + sigma sqrt(1 - e^{-2 dt/tau_f}) xi, xi ~ N(0,1),
    sigma^2 being the stationary variance of each amplitude.  tau_f = inf freezes the flow.
    """
    if math.isinf(tau_f):
        return amp.copy()
    e = math.exp(-dt / tau_f)
    return amp * e + sigma * math.sqrt(1.0 - e * e) * xi


def flow2d_u(a: np.ndarray, kvec: np.ndarray, phi: np.ndarray, nx: int, ny: int, dx: float):
    """Incompressible flow u = (d_y psi, -d_x psi) of psi = sum_m a_m cos(theta_m).

    theta_m(x_i, y_l) = 2 pi (kx_m i / N_x + ky_m l / N_y) + phi_m on the periodic
    (N_x dx) x (N_y dx) domain.  Returns (ux, uy), each (N_y, N_x).
    """
    Lx, Ly = nx * dx, ny * dx
    ii = np.arange(nx, dtype=np.float64)[None, :]
    ll = np.arange(ny, dtype=np.float64)[:, None]
    ux = np.zeros((ny, nx))
    uy = np.zeros((ny, nx))
    for m in range(len(a)):
        kx, ky = float(kvec[m, 0]), float(kvec[m, 1])
        th = 2.0 * math.pi * (kx * ii / nx + ky * ll / ny) + phi[m]
        s = np.sin(th)
        ux += -a[m] * (2.0 * math.pi * ky / Ly) * s
        uy += a[m] * (2.0 * math.pi * kx / Lx) * s
    return ux, uy


def phase_advance(phi: np.ndarray, xi: np.ndarray, dt: float, tau_f: float) -> np.ndarray:
    """Random-walk phases phi <- phi + sqrt(2 dt / tau_f) xi: <e^{i(phi(t)-phi(0))}> = e^{-t/tau_f}."""
    if math.isinf(tau_f):
        return phi.copy()
    return phi + math.sqrt(2.0 * dt / tau_f) * xi


# --------------------------------------------------------------------------------------------
# Drivers
# --------------------------------------------------------------------------------------------
def run_1d(f0, nsteps, *, tau_p, kappa, dt, dv, k, amp0, tau_f, sigma, noise, field=None):
    """Advance f0 by nsteps (R4: step n uses u at t_n, then the amplitudes move to t_{n+1}).

    noise[n] holds the 2M standard normal draws of the update after step n.  When ``field`` is
    given it is a frozen u(x) and the modal flow is ignored.  Returns (f, amp).
    """
    f = np.array(f0, dtype=np.float64, copy=True)
    amp = np.array(amp0, dtype=np.float64, copy=True)
    nx = f.shape[1]
    for n in range(nsteps):
        u = field if field is not None else flow1d_u(amp, k, nx)
        f = step_1d(f, u, tau_p, kappa, dt, dv)
        if field is None:
            amp = ou_advance(amp, noise[n], dt, tau_f, sigma)
    return f, amp


def run_2d(f0, nsteps, *, tau_p, kappa, dt, dv, dx, kvec=None, a=None, phi0=None, tau_f=math.inf,
           noise=None, field=None):
    """2D analogue of run_1d; ``field`` = (ux, uy) frozen, else the random-phase flow."""
    f = np.array(f0, dtype=np.float64, copy=True)
    _, _, ny, nx = f.shape
    phi = None if phi0 is None else np.array(phi0, dtype=np.float64, copy=True)
    for n in range(nsteps):
        if field is not None:
            ux, uy = field
        else:
            ux, uy = flow2d_u(a, kvec, phi, nx, ny, dx)
        f = step_2d(f, ux, uy, tau_p, kappa, dt, dv)
        if field is None:
            phi = phase_advance(phi, noise[n], dt, tau_f)
    return f, phi
