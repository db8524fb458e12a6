"""Reduced-precision (FP16 / BF16) storage of the 2D lattice state: plain CPU reference.

TEST INFRASTRUCTURE ONLY, like ``oracle/lattice.py``: nothing on the product path imports it,
and it shares no code with the CUDA library.

The paper computes in double precision and has no reduced-precision storage.  This module states
the storage scheme that the library's 16-bit path follows, in its plainest form, on top of the
FP64 step of Section 2 (``lattice.step_2d``):

* a stored value is a 16-bit floating-point code h (IEEE binary16, or bfloat16: the upper half
  of an IEEE binary32) times a power-of-two scale S shared by one x-line, i.e. one velocity plane
  (jx, jy) at one row y;
* codes are the round-to-nearest, ties-to-even values of t / S;
* S = 2^(ilogb(B) - 12) for a bound B of the line's values (S = 1 when B = 0): when the state
  is encoded from given values, B is the line's largest |value|; in a step, B is the largest
  line maximum of the input over the 13 velocity cells |djx| + |djy| <= 2 around the output
  line's plane, each taken at the row the streaming brings to y (row y - (jy' - J));
* the rounding residual of each value, t - h S, is carried to the next value of the same spatial
  cell's velocity column, the column taken in (jy, jx) order; a value takes at most
  CARRY_LIM * S of the carry (its own line's scale), the rest stays in the carry; the carry left
  after the last value is dropped.  So the stored column sum equals the given one up to that
  last carry, and |t / S| < 3 * 2^13 + 2^14 < 65504 whatever the neighbouring lines hold.

Why that bound (R-S1).  With g (J + |w_x|) + g (J + |w_y|) <= 1 and 4 r <= 1, the drag output
f** at a velocity cell is a combination of f* at that cell and its four neighbours with
non-negative weights summing to at most 3, and the diffusion output a combination of f** with
weights summing to at most 1; so |output| <= 3 B and |output| / S < 3 * 2^13 < 2^15.
"""
from __future__ import annotations

import numpy as np

from . import lattice as _lat

SCALE_DROP = 12
FORMATS = ("f16", "bf16")


def carry_lim(fmt: str) -> float:
    """Largest part of the carry one value takes, in units of its line's scale."""
    return 2.0**14 if fmt == "f16" else 2.0**100


def round16(q: np.ndarray, fmt: str) -> np.ndarray:
    """Nearest representable value of the 16-bit format to q (ties to even), as float64.

    f16: IEEE binary16 (numpy's correctly rounded conversion, subnormals included, overflow to
    inf).  bf16: 8 significant bits and binary32's exponent range; q = m 2^e with m in
    [1/2, 1) rounds m 2^8 to the nearest integer, ties to even (normal range only).
    """
    q = np.asarray(q, dtype=np.float64)
    if fmt == "f16":
        return q.astype(np.float16).astype(np.float64)
    if fmt == "bf16":
        m, e = np.frexp(q)
        return np.ldexp(np.rint(m * 256.0), e - 8)
    raise ValueError(fmt)


def max_code(fmt: str) -> float:
    """Largest finite value of the format."""
    return 65504.0 if fmt == "f16" else float(np.ldexp(255.0, 120))


def scale_for(bound: np.ndarray) -> np.ndarray:
    """S = 2^(ilogb(B) - 12), clamped to 2^[-120, 120]; 1 where B = 0."""
    b = np.asarray(bound, dtype=np.float64)
    _, e = np.frexp(b)           # b = m 2^e, m in [1/2, 1): ilogb(b) = e - 1
    E = np.clip(e - 1 - SCALE_DROP, -120, 120)
    return np.where(b > 0, np.ldexp(1.0, E), 1.0)


def line_max(f: np.ndarray) -> np.ndarray:
    """Largest |f| over x of every line: f[jy, jx, y, x] -> [jy, jx, y]."""
    return np.abs(f).max(axis=3)


def diamond_bound(mx: np.ndarray) -> np.ndarray:
    """Bound B of every output line of a step from the input line maxima mx[jy, jx, y]:
    max over |djx| + |djy| <= 2 of mx[jy', jx', (y - (jy' - J)) mod N_y]."""
    nv, _, ny = mx.shape
    J = (nv - 1) // 2
    out = np.zeros_like(mx)
    for jy in range(nv):
        for jx in range(nv):
            b = np.zeros(ny)
            for dy in range(-2, 3):
                jy2 = jy + dy
                if not 0 <= jy2 < nv:
                    continue
                for dx in range(-(2 - abs(dy)), 3 - abs(dy)):
                    jx2 = jx + dx
                    if not 0 <= jx2 < nv:
                        continue
                    # value at output row y came from input row y - (jy2 - J)
                    b = np.maximum(b, np.roll(mx[jy2, jx2], jy2 - J))
            out[jy, jx] = b
    return out


def encode(t: np.ndarray, S: np.ndarray, fmt: str):
    """Codes of the values t[jy, jx, y, x] with line scales S[jy, jx, y], residual carried along
    each cell's column in (jy, jx) order.  Returns (decoded stored values, overflow flag)."""
    nv, _, ny, nx = t.shape
    out = np.empty_like(t, dtype=np.float64)
    carry = np.zeros((ny, nx))
    over = False
    for jy in range(nv):
        for jx in range(nv):
            s = S[jy, jx][:, None]
            lim = carry_lim(fmt) * s
            used = np.clip(carry, -lim, lim)
            v = t[jy, jx] + used
            h = round16(v / s, fmt)
            over |= bool(np.any(~(np.abs(h) <= max_code(fmt))))
            back = h * s
            carry = (v - back) + (carry - used)
            out[jy, jx] = back
    return out, over


def encode_state(f: np.ndarray, fmt: str):
    """Encode given values with fresh scales from their own line maxima.
    Returns (decoded stored values, scales, line maxima of the stored values)."""
    S = scale_for(line_max(f))
    dec, _ = encode(np.asarray(f, dtype=np.float64), S, fmt)
    return dec, S, line_max(dec)


def step_2d_stored(dec: np.ndarray, mx: np.ndarray, ux, uy, *, tau_p, kappa, dt, dv, fmt):
    """One step of the stored state: FP64 step of Section 2 on the decoded values, then the
    encoding with the output scales of ``diamond_bound``.
    Returns (decoded output, output scales, output line maxima, overflow flag)."""
    f_new = _lat.step_2d(dec, ux, uy, tau_p, kappa, dt, dv)
    S = scale_for(diamond_bound(mx))
    out, over = encode(f_new, S, fmt)
    return out, S, line_max(out), over


def coarse_density_moment(rho: np.ndarray, dx: float, r: int) -> float:
    """<rho_r^2> of Eq. (def_coarse) in 2D: rho_r is the mass in an r x r box of cells (the
    integral of f over the box and over v), averaged in square over a tiling of the domain.
    rho: per-cell density sum_j f dv^2, shape (N_y, N_x), both divisible by r."""
    ny, nx = rho.shape
    boxes = rho.reshape(ny // r, r, nx // r, r).sum(axis=(1, 3)) * dx * dx
    return float(np.mean(boxes * boxes))
