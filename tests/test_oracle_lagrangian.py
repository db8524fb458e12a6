"""Whole-step pin: the oracle against brute-force Lagrangian Stokes-drag particles (no GPU).

Eq. (stokes_drag) is integrated for N_p particles in a frozen periodic flow u(x) = U sin(x) on
a tiny grid; the lattice run starts from the same distribution.  The two are independent
discretisations, so the comparison is loose by design: Monte-Carlo noise plus the lattice's
first-order error in dv (Sec. 3.2, Fig. 5).  It fails on gross mistakes (drag sign, diffusion
factor, streaming direction), which ``test_oracle_mutations`` checks.
"""
import math

import numpy as np

from oracle import lattice as O

L = 2 * math.pi
VMAX = 3.0
TAU_P, KAPPA, U0 = 1.0, 0.2, 1.0
T_END = 300 * (L / 1024) / (VMAX / 16)  # 300 steps of the N_v = 33 lattice, ~9.8 tau_p
NBOX = 32
SIG0 = 0.3


def lattice_run(nx, nv, mod=O):
    J = (nv - 1) // 2
    dv, dx = VMAX / J, L / nx
    dt = dx / dv
    v = O.velocities(nv, dv)
    f = np.repeat(np.exp(-0.5 * (v / SIG0) ** 2)[:, None], nx, axis=1)
    f /= f.sum() * dx * dv
    u = U0 * np.sin(np.arange(nx) * dx)
    for _ in range(int(round(T_END / dt))):
        f = mod.step_1d(f, u, TAU_P, KAPPA, dt, dv)
    rho = f.sum(0) * dv
    rho_box = rho.reshape(NBOX, -1).sum(1) * dx
    m1 = (v[:, None] * f).sum() * dx * dv
    m2 = (v[:, None] ** 2 * f).sum() * dx * dv
    return rho_box, m1, m2


def lagrangian_run(n_p=100_000, seed=0, nsub=1200):
    """Exact OU velocity update over sub-steps h with u frozen at the particle position,
    trapezoidal position update, periodic x."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, L, n_p)
    v = SIG0 * rng.standard_normal(n_p)
    h = T_END / nsub
    e = math.exp(-h / TAU_P)
    s = math.sqrt(KAPPA * TAU_P * (1 - e * e))
    for _ in range(nsub):
        u = U0 * np.sin(x)
        vn = u + (v - u) * e + s * rng.standard_normal(n_p)
        x = np.mod(x + 0.5 * h * (v + vn), L)
        v = vn
    counts = np.bincount((x / (L / NBOX)).astype(int) % NBOX, minlength=NBOX)
    return counts / n_p, v.mean(), (v * v).mean()


_LAG = None


def _lag():
    global _LAG
    if _LAG is None:
        _LAG = lagrangian_run()
    return _LAG


def check_against_particles(mod=O):
    """Lattice at N_v = 17 and 33 (dv = 0.375, 0.1875) against 10^5 particles.

    The paper finds the lattice error first order in dv (Sec. 3.2, Fig. 5), so halving dv
    must roughly halve the error of the coarse-grained density and of <v^2>; at N_v = 33 the
    errors must also be small in absolute terms.  Monte-Carlo noise: ~2 % per density box,
    ~0.5 % on <v^2>.
    """
    rho_l, m1_l, m2_l = _lag()
    errs = []
    for nx, nv in ((512, 17), (1024, 33)):
        rho_e, m1_e, m2_e = lattice_run(nx, nv, mod)
        e_rho = np.linalg.norm(rho_e - rho_l) / np.linalg.norm(rho_l)
        e_m2 = abs(m2_e - m2_l) / m2_l
        assert abs(m1_e - m1_l) < 0.02, (nv, m1_e, m1_l)
        errs.append((e_rho, e_m2))
    (r17, v17), (r33, v33) = errs
    assert r33 < 0.08 and v33 < 0.3, errs
    assert r33 < 0.65 * r17 and v33 < 0.65 * v17, errs
    return errs


def test_lattice_matches_lagrangian_particles():
    check_against_particles()
