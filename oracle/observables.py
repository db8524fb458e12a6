"""Observables of the phase-space density used by the paper to benchmark the method: plain FP64
CPU oracle.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or execute this
module: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the CUDA library.

* The coarse-grained density of Eq. (def_coarse): rho_r(x) is the mass within a window of width
  r around x, the integral of f over that window and over all velocities.  Its second moment
  <rho_r^2> (the average over positions) scales as r^(D_2 - 1) (Sec. 3.2).
* The Eulerian first-order velocity structure function of Eq. (def_eulS1):
      S1(r) = < int dv int dv' f(x, v) f(x + r, v') |v - v'| > / < int dv int dv' f(x, v) f(x + r, v') >,
  the averages taken over positions x.

Lattice readings O1-O2:

* O1  r = w dx for a whole number w of cells; the window of cell i covers cells i .. i + w - 1
      (periodic).  The average over every cell of the domain does not depend on where the
      window sits relative to x_i.  In 2D the window is the w x w square of cells (i..i+w-1) x
      (k..k+w-1), of area r^2.
* O2  The velocity integrals are sums over velocity cells times dv (dv^2 in 2D), the velocity
      difference of cells j and j' is |j - j'| dv, and the separation r = s dx is a whole number
      s of cells.  S1 is formed in 1D only, the geometry of the paper's figures.

Layouts are the lattice oracle's: 1D f[j, x]; 2D f[jy, jx, y, x].
"""
from __future__ import annotations

import math

import numpy as np


def density(f: np.ndarray, dv: float) -> np.ndarray:
    """rho(x) = int dv f: the sum over the velocity cells times dv (dv^2 in 2D)."""
    if f.ndim == 2:
        return f.sum(axis=0) * dv
    return f.sum(axis=(0, 1)) * dv * dv


def coarse_density_1d(f: np.ndarray, dx: float, dv: float, w: int) -> np.ndarray:
    """rho_r(x_i) for r = w dx (Eq. def_coarse, O1): the mass in cells i .. i + w - 1."""
    rho = density(f, dv)
    n = rho.shape[0]
    out = np.zeros(n)
    for q in range(w):
        out += np.roll(rho, -q)
    return out * dx


def coarse_density_2d(f: np.ndarray, dx: float, dv: float, w: int) -> np.ndarray:
    """rho_r over the w x w square of cells starting at (y, x) (Eq. def_coarse in 2D, O1)."""
    rho = density(f, dv)
    out = np.zeros_like(rho)
    for qy in range(w):
        for qx in range(w):
            out += np.roll(rho, (-qy, -qx), axis=(0, 1))
    return out * dx * dx


def coarse_moment(f: np.ndarray, dx: float, dv: float, widths) -> np.ndarray:
    """<rho_r^2> for each window width in cells: the mean of rho_r^2 over all positions."""
    fn = coarse_density_1d if f.ndim == 2 else coarse_density_2d
    ncell = f.shape[1] if f.ndim == 2 else f.shape[2] * f.shape[3]
    return np.array([math.fsum((fn(f, dx, dv, int(w)) ** 2).ravel()) / ncell
                     for w in widths])


def s1_terms(f: np.ndarray, dv: float, seps):
    """Numerator and denominator of Eq. (def_eulS1) in 1D (O2), averaged over positions:
        num(s) = (1/N_x) sum_i sum_j sum_j' f_j(i) f_j'(i + s) |v_j - v_j'| dv^2,
        den(s) = (1/N_x) sum_i sum_j sum_j' f_j(i) f_j'(i + s) dv^2.
    S1(s dx) = num / den.  Direct double sums, as written."""
    nv, nx = f.shape
    J = (nv - 1) // 2
    v = (np.arange(nv) - J) * dv
    dist = np.abs(v[:, None] - v[None, :])
    num, den = [], []
    for s in seps:
        g = np.roll(f, -int(s), axis=1)  # g[:, i] = f[:, i + s]
        pair = np.einsum("ji,ki,jk->i", f, g, dist) * dv * dv
        mass = f.sum(axis=0) * g.sum(axis=0) * dv * dv
        num.append(math.fsum(pair) / nx)
        den.append(math.fsum(mass) / nx)
    return np.array(num), np.array(den)
