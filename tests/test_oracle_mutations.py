"""Plant plausible mistakes in a copy of the oracle (on the CPU) and check that a pin fails.

Each mutation is a textual edit of ``oracle/lattice.py`` loaded as a fresh module; the real
oracle is untouched.  A mutation that no pin catches would mean the pins leave that part of the
oracle unchecked.
"""
import math
import os
import types

import numpy as np
import pytest

import test_oracle_1d as P1
import test_oracle_2d as P2
import test_oracle_lagrangian as PL

SRC = os.path.join(os.path.dirname(os.path.dirname(__file__)), "oracle", "lattice.py")


def mutant(old: str, new: str):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
    src = src.replace(old, new, 1)
    mod = types.ModuleType("oracle_mutant")
    mod.__dict__["__name__"] = "oracle_mutant"
    exec(compile(src, "oracle_mutant", "exec"), mod.__dict__)
    return mod


MUTATIONS = [
    ("stream direction reversed", "np.roll(f[jj], jj - J)", "np.roll(f[jj], J - jj)",
     [P1.check_unit_mass_moves_by_j, PL.check_against_particles]),
    ("drag sign flipped", "return -(v - u) / tau_p", "return (v - u) / tau_p",
     [P1.check_first_moment_drag, P1.check_relaxation_to_rest]),
    ("downwind instead of upwind",
     "F[1:-1] = ap[:-1] * f[:-1] + am[1:] * f[1:]",
     "F[1:-1] = ap[1:] * f[1:] + am[:-1] * f[:-1]",
     [P1.check_golden_1d]),
    ("drag step missing 1/dv", "return f - (dt / dv) * (F[1:] - F[:-1])",
     "return f - dt * (F[1:] - F[:-1])", [P1.check_first_moment_drag]),
    ("diffusion factor two", "D[1:-1] = kappa * (f[1:] - f[:-1]) / dv",
     "D[1:-1] = 2 * kappa * (f[1:] - f[:-1]) / dv",
     [P1.check_diffusion_moments, P1.check_golden_1d, PL.check_against_particles]),
    ("flow cos and sin swapped", "u += amp[m] * np.cos(th) + amp[M + m] * np.sin(th)",
     "u += amp[m] * np.sin(th) + amp[M + m] * np.cos(th)", [P1.check_single_modes]),
    ("2D drag axes transposed",
     "ax = drag_acceleration(v[None, :, None, None], ux[None, None], tau_p)",
     "ax = drag_acceleration(v[:, None, None, None], ux[None, None], tau_p)",
     [P2.check_golden_2d, P2.check_first_moments_2d]),
    ("2D stream axes swapped", "np.roll(f[jy, jx], (jy - J, jx - J), axis=(0, 1))",
     "np.roll(f[jy, jx], (jx - J, jy - J), axis=(0, 1))", [P2.check_unit_mass_moves]),
    ("2D flow sign of u_x", "ux += -a[m] * (2.0 * math.pi * ky / Ly) * s",
     "ux += a[m] * (2.0 * math.pi * ky / Ly) * s", [P2.check_flow2d_is_perp_gradient]),
    ("2D diffusion drops the vy direction",
     "return f + c * (Dx[:, 1:] - Dx[:, :-1]) + c * (Dy[1:] - Dy[:-1])",
     "return f + c * (Dx[:, 1:] - Dx[:, :-1])", [P2.check_golden_2d]),
    ("2D energy drops v_y^2", "s2 = ((vx * vx + vy * vy) * f).sum(axis=(0, 1))",
     "s2 = ((vx * vx) * f).sum(axis=(0, 1))",
     [P2.check_moments_2d_known, P2.check_moments_2d_reduce_to_1d]),
    ("2D density missing one dv", "rho = s0 * dv * dv", "rho = s0 * dv",
     [P2.check_moments_2d_known, P2.check_moments_2d_reduce_to_1d]),
    ("2D moment velocity axes transposed",
     "vx = np.broadcast_to(v[None, :, None, None], f.shape)",
     "vx = np.broadcast_to(v[:, None, None, None], f.shape)",
     [P2.check_moments_2d_known, P2.check_moments_2d_reduce_to_1d]),
    ("2D global energy drops v_y^2", "math.fsum(((vx * vx + vy * vy) * f).ravel()) * w",
     "math.fsum(((vx * vx) * f).ravel()) * w", [P2.check_moments_2d_known]),
]


@pytest.mark.parametrize("name,old,new,checks", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_mutation_is_caught(name, old, new, checks):
    mod = mutant(old, new)
    for check in checks:
        with np.errstate(all="ignore"):
            try:
                check(mod)
            except (AssertionError, FloatingPointError, ValueError):
                continue
        raise AssertionError(f"pin {check.__name__} did not catch: {name}")


def test_unmutated_copy_passes():
    mod = mutant("import math", "import math")
    for check in (P1.check_golden_1d, P1.check_first_moment_drag, P2.check_golden_2d):
        check(mod)
    assert math.isfinite(1.0)
