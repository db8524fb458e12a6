"""Seeded synthetic inputs shared by the tests, the bench and the CPU oracle.

This module holds only input recipes: random draws, mode tables, initial densities and
parameter choices.  It performs none of the lattice method's arithmetic (no streaming, no flux,
no flow evolution) and imports neither the oracle nor the CUDA library.

Recipes (stand-ins for the paper's flows, whose realisations are not available):

* 1D flow: M Fourier modes k = 1..M of u = sum A_m cos(k_m x) + B_m sin(k_m x) whose amplitudes
  are Ornstein-Uhlenbeck processes (Sec. 3.1 Eq. u1d/A1d has M = 1); each amplitude has
  stationary variance u_rms^2 / M so that <u^2> = u_rms^2.  Initial amplitudes are drawn from
  the stationary law; every later step consumes 2M standard normal draws.
* 2D flow: stream function psi = sum_m a_m cos(k_m . x + phi_m) over one wave vector of each
  +-k pair with 0 < |k| <= k_max, |a_m| proportional to |k|^-3 (shell energy spectrum k^-3),
  normalised to u_rms per component; phases start uniform and every step consumes one standard
  normal draw per mode.
* initial density: uniform in x, Gaussian in v with standard deviation 0.2 V_max sampled at the
  cell centres, normalised to unit mass sum f dx^d dv^d = 1 (Sec. 3.2 normalises to N_p).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


# --------------------------------------------------------------------------------------------
# Initial densities
# --------------------------------------------------------------------------------------------
def gaussian_column(nx: int, nv: int, dx: float, dv: float, sigma_v: float) -> np.ndarray:
    """Velocity column of the uniform-in-x Gaussian initial density, normalised so that N_x
    copies of it carry unit mass (sum f dx dv = 1)."""
    J = (nv - 1) // 2
    v = np.arange(-J, J + 1, dtype=np.float64) * dv
    g = np.exp(-0.5 * (v / sigma_v) ** 2)
    return g / (nx * g.sum() * dx * dv)


def gaussian_initial_1d(nx: int, nv: int, dx: float, dv: float, sigma_v: float) -> np.ndarray:
    return np.repeat(gaussian_column(nx, nv, dx, dv, sigma_v)[:, None], nx, axis=1)


def ensemble_initial(tab: "EnsembleTable", nv: int, dtype, device, instances=None):
    """Concatenated 1D initial densities (sigma_v = 0.2 V_max per instance) as one torch
    tensor built on ``device``; with ``instances`` given, only those (numpy, float64)."""
    J = (nv - 1) // 2

    def col(i):
        nx = int(tab.nx[i])
        dx = tab.L[i] / nx
        dv = dx / tab.dt[i]
        return gaussian_column(nx, nv, dx, dv, 0.2 * max(J, 1) * dv)

    if instances is not None:
        return {int(i): np.repeat(col(i)[:, None], int(tab.nx[i]), axis=1) for i in instances}
    import torch
    total = int((tab.nx * nv).sum())
    out = torch.empty(total, dtype=dtype, device=device)
    off = 0
    cache = {}
    for i in range(len(tab.nx)):
        nx = int(tab.nx[i])
        key = (nx, float(tab.dt[i]), float(tab.L[i]))
        if key not in cache:
            c = torch.tensor(col(i), dtype=dtype, device=device)
            cache[key] = c[:, None].expand(nv, nx).contiguous().view(-1)
        out[off:off + nv * nx].copy_(cache[key])
        off += nv * nx
    return out


def gaussian_initial_2d(nx: int, ny: int, nv: int, dx: float, dv: float,
                        sigma_v: float) -> np.ndarray:
    J = (nv - 1) // 2
    v = np.arange(-J, J + 1, dtype=np.float64) * dv
    g = np.exp(-0.5 * (v / sigma_v) ** 2)
    col = g[:, None] * g[None, :]
    f = np.broadcast_to(col[:, :, None, None], (nv, nv, ny, nx)).copy()
    return f / (f.sum() * dx * dx * dv * dv)


def random_initial(shape, seed: int) -> np.ndarray:
    """Positive random density (uniform in [0.1, 1.1)) for parity tests that need structure."""
    rng = np.random.default_rng(seed)
    return rng.random(shape) + 0.1


# --------------------------------------------------------------------------------------------
# Flows
# --------------------------------------------------------------------------------------------
@dataclass
class Flow1D:
    k: np.ndarray        # (M,) integer wavenumbers
    amp0: np.ndarray     # (n_inst, 2M) initial [A_0..A_{M-1}, B_0..B_{M-1}]
    noise: np.ndarray    # (nsteps, n_inst, 2M) standard normal draws
    sigma: float         # stationary std of each amplitude
    tau_f: float


def flow1d_inputs(seed: int, nsteps: int, nmodes: int = 8, u_rms: float = 1.0,
                  tau_f: float = 1.0, n_inst: int = 1) -> Flow1D:
    rng = np.random.default_rng(seed)
    sigma = u_rms / math.sqrt(nmodes)
    k = np.arange(1, nmodes + 1, dtype=np.int32)
    amp0 = sigma * rng.standard_normal((n_inst, 2 * nmodes))
    noise = rng.standard_normal((nsteps, n_inst, 2 * nmodes))
    return Flow1D(k=k, amp0=amp0, noise=noise, sigma=sigma, tau_f=tau_f)


@dataclass
class Flow2D:
    kvec: np.ndarray     # (M, 2) integer wave vectors (kx, ky)
    a: np.ndarray        # (M,) stream-function amplitudes
    phi0: np.ndarray     # (M,) initial phases
    noise: np.ndarray    # (nsteps, M) standard normal draws
    tau_f: float


def wave_vectors(kmax: int) -> np.ndarray:
    """One wave vector of each +-k pair with 0 < |k| <= kmax (kx > 0, or kx == 0 and ky > 0)."""
    out = []
    for kx in range(0, kmax + 1):
        for ky in range(-kmax, kmax + 1):
            if kx == 0 and ky <= 0:
                continue
            if kx * kx + ky * ky <= kmax * kmax:
                out.append((kx, ky))
    return np.array(out, dtype=np.int32)


def flow2d_inputs(seed: int, nsteps: int, nx: int, ny: int, dx: float, kmax: int = 8,
                  u_rms: float = 1.0, tau_f: float = 1.0) -> Flow2D:
    rng = np.random.default_rng(seed)
    kvec = wave_vectors(kmax)
    kk = np.sqrt((kvec.astype(np.float64) ** 2).sum(axis=1))
    a = kk ** -3.0
    Lx, Ly = nx * dx, ny * dx
    # <u_x^2> = sum a^2 (2 pi ky / Ly)^2 / 2 and <u_y^2> = sum a^2 (2 pi kx / Lx)^2 / 2
    vx = 0.5 * np.sum(a * a * (2 * math.pi * kvec[:, 1] / Ly) ** 2)
    vy = 0.5 * np.sum(a * a * (2 * math.pi * kvec[:, 0] / Lx) ** 2)
    a = a * (u_rms / math.sqrt(0.5 * (vx + vy)))
    phi0 = rng.uniform(0.0, 2.0 * math.pi, size=len(a))
    noise = rng.standard_normal((nsteps, len(a)))
    return Flow2D(kvec=kvec, a=a, phi0=phi0, noise=noise, tau_f=tau_f)


def cellular_flow(nx: int, ny: int, L: float, U: float = 1.0):
    """The tilted cellular flow of Sec. 4.1: u = (d_y psi, -d_x psi) of the stationary stream
    function psi = U sin(pi (x + y) / L) sin(pi (x - y) / L), at the cell positions x_i = i dx,
    y_k = k dx (dx = L / nx, ny dx = L).  Returns (ux, uy), each (ny, nx), FP64."""
    dx = L / nx
    x = np.arange(nx) * dx
    y = np.arange(ny) * dx
    X, Y = np.meshgrid(x, y)
    a = math.pi * (X + Y) / L
    b = math.pi * (X - Y) / L
    k = math.pi / L
    # d_x psi = U k (cos a sin b + sin a cos b),  d_y psi = U k (cos a sin b - sin a cos b)
    dpsi_dx = U * k * (np.cos(a) * np.sin(b) + np.sin(a) * np.cos(b))
    dpsi_dy = U * k * (np.cos(a) * np.sin(b) - np.sin(a) * np.cos(b))
    return dpsi_dy, -dpsi_dx


# --------------------------------------------------------------------------------------------
# Parameter choices
# --------------------------------------------------------------------------------------------
def choose_dt(d: int, nx: int, L: float, nv: int, tau_p: float, kappa: float,
              u_rms: float = 1.0, cfl_factor: float = 1.0) -> float:
    """Largest dt (bisection) such that, with dv = dx / dt and V_max = J dv:

    (i)   V_max >= 3 u_rms                      (Section 2: Gaussian flows, V_max = 3 u_rms),
    (ii)  d (dt/dv)(V_max + 5 u_rms)/tau_p * cfl_factor <= 0.9
          (Eq. cfl with |u| <= 5 u_rms, d components; cfl_factor = 1 + mu for the limited
          drag scheme, whose stages are positive for nu (1 + mu) <= 1),
    (iii) 2 d kappa dt / dv^2 <= 0.9               (Eq. stabLapl, d dimensions).
    """
    dx = L / nx
    J = (nv - 1) // 2

    def ok(dt):
        dv = dx / dt
        vmax = J * dv
        if J > 0 and vmax < 3.0 * u_rms * (1 - 1e-12):
            return False
        if d * (dt / dv) * (vmax + 5.0 * u_rms) / tau_p * cfl_factor > 0.9:
            return False
        if 2 * d * kappa * dt / (dv * dv) > 0.9:
            return False
        return True

    lo, hi = 0.0, (J * dx / (3.0 * u_rms)) if J > 0 else 1.0
    if ok(hi):
        return hi
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if ok(mid):
            lo = mid
        else:
            hi = mid
    return lo


@dataclass
class EnsembleTable:
    nx: np.ndarray      # (n,) int
    L: np.ndarray       # (n,) float
    tau_p: np.ndarray
    kappa: np.ndarray
    dt: np.ndarray
    st: np.ndarray


def ensemble_table(n_inst: int, seed: int, nv: int = 65,
                   sizes=(1024, 2048, 4096, 8192), stokes=(0.1, 1.0, 10.0),
                   kappa: float = 1e-3, L: float = 2 * math.pi,
                   u_rms: float = 1.0, cfl_factor: float = 1.0) -> EnsembleTable:
    """Instances with N_x drawn uniformly from ``sizes`` and St cycling through ``stokes``.

    St = tau_p u_rms / L (Sec. 3.1) fixes tau_p; dt follows ``choose_dt`` (with ``cfl_factor``
    = 1 + mu for the limited drag scheme).
    """
    rng = np.random.default_rng(seed)
    nx = rng.choice(np.array(sizes, dtype=np.int64), size=n_inst)
    st = np.array([stokes[i % len(stokes)] for i in range(n_inst)], dtype=np.float64)
    tau_p = st * L / u_rms
    cache = {}
    dts = np.empty(n_inst)
    for i in range(n_inst):
        key = (int(nx[i]), float(tau_p[i]))
        if key not in cache:
            cache[key] = choose_dt(1, int(nx[i]), L, nv, float(tau_p[i]), kappa, u_rms,
                                   cfl_factor)
        dts[i] = cache[key]
    return EnsembleTable(nx=nx.astype(np.int64), L=np.full(n_inst, L), tau_p=tau_p,
                         kappa=np.full(n_inst, kappa), dt=dts, st=st)
