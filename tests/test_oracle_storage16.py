"""Pins of the 16-bit storage oracle (oracle/storage16.py) against definitions that do not go
through it: the IEEE rounding rule on hand-picked ties, a bit-level bfloat16 rounding, the
exact column-sum identity of the residual carry, the growth bound of the step, and streaming as
an exact permutation of stored values."""
import math

import numpy as np
import pytest

from oracle import lattice as L
from oracle import storage16 as S16


def test_fp16_rounding_on_ties_and_limits():
    r = lambda x: float(S16.round16(np.array([x]), "f16")[0])
    assert r(1 + 2.0**-11) == 1.0                      # tie -> even mantissa
    assert r(1 + 3 * 2.0**-11) == 1 + 2.0**-9          # tie -> even mantissa
    assert r(1 + 2.0**-11 + 2.0**-30) == 1 + 2.0**-10  # above the tie
    assert r(65504.0) == 65504.0
    assert r(65519.0) == 65504.0 and math.isinf(r(65520.0))
    assert r(2.0**-24) == 2.0**-24                     # smallest subnormal
    assert r(2.0**-25) == 0.0 and r(3 * 2.0**-25) == 2.0**-23


def test_bf16_rounding_matches_bit_level_definition():
    assert S16.round16(np.array([1 + 2.0**-8]), "bf16")[0] == 1.0
    assert S16.round16(np.array([1 + 3 * 2.0**-8]), "bf16")[0] == 1 + 2.0**-6
    rng = np.random.default_rng(5)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-30, 30, 20000))).astype(np.float32)
    bits = x.view(np.uint32).astype(np.uint64)
    rnd = ((bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    want = rnd.view(np.float32).astype(np.float64)
    np.testing.assert_array_equal(S16.round16(x.astype(np.float64), "bf16"), want)


def test_scale_rule():
    s = S16.scale_for(np.array([1.0, 1.5, 1.999, 2.0, 0.0, 2.0**-200, 3 * 2.0**40]))
    np.testing.assert_array_equal(s, [2.0**-12, 2.0**-12, 2.0**-12, 2.0**-11, 1.0, 2.0**-120,
                                      2.0**29])


@pytest.mark.parametrize("fmt", S16.FORMATS)
def test_encode_keeps_each_column_sum_up_to_the_last_residual(fmt):
    rng = np.random.default_rng(11)
    nv, ny, nx = 5, 4, 6
    # neighbouring lines within a factor e^2 of each other: every carry is taken in full
    t = rng.gamma(2.0, 1.0, (nv, nv, ny, nx)) * np.exp(rng.uniform(-1, 1, (nv, nv, 1, 1)))
    dec, Sc, mx = S16.encode_state(t, fmt)
    h = dec / Sc[..., None]
    np.testing.assert_array_equal(S16.round16(h, fmt), h)  # codes are representable
    assert np.all(np.abs(h) < 2.0**13 + 2.0**14)
    # column sum identity: sum(t) - sum(dec) is the last residual alone, at most half a
    # storage step of the corner value (2^-11 of it in FP16, 2^-8 in BF16), up to FP64 rounding
    step = 2.0**-11 if fmt == "f16" else 2.0**-8
    last_res = t.sum(axis=(0, 1)) - dec.sum(axis=(0, 1))
    assert np.all(np.abs(last_res) <= step * np.abs(dec[-1, -1]) + 1e-14 * t.sum(axis=(0, 1)))
    # the error of each value: its own residual minus the one it received, each at most half a
    # storage step of its value
    prev = np.concatenate([np.zeros((1, ny, nx)), dec.reshape(nv * nv, ny, nx)[:-1]])
    err = np.abs(dec - t).reshape(nv * nv, ny, nx)
    assert np.all(err <= step * (np.abs(dec.reshape(nv * nv, ny, nx)) + np.abs(prev)) + 1e-300)


def test_encode_bounds_the_carry_next_to_much_smaller_lines():
    # lines 2^20 apart: a large line's residual exceeds what the next small line can hold
    nv, ny, nx = 3, 2, 4
    t = np.ones((nv, nv, ny, nx)) * (1 + 2.0**-12)
    t[0::2] *= 2.0**20
    t[:, :, :, 1] *= 1.3
    dec, Sc, mx = S16.encode_state(t, "f16")
    h = dec / Sc[..., None]
    assert np.all(np.isfinite(h)) and np.all(np.abs(h) < 3 * 2.0**13 + 2.0**14)
    # the column sum still holds up to the final carry, which is at most the residuals' sum
    lost = np.abs(t.sum(axis=(0, 1)) - dec.sum(axis=(0, 1)))
    assert np.all(lost <= 2.0**-11 * np.abs(dec).sum(axis=(0, 1)))
    # without the limit the small lines would have overflowed FP16
    S_small = Sc[1, 0, 0]
    assert 2.0**-11 * t[0, 2, 0, 1] / S_small > 65504


def _random_case(rng, nv=9, ny=8, nx=10):
    f = rng.gamma(1.5, 1.0, (nv, nv, ny, nx)) * np.exp(rng.uniform(-6, 6, (nv, nv, ny, 1)))
    J = (nv - 1) // 2
    dt, dv = 0.05, 0.5
    # CFL of the unsplit drag and 4 r <= 1
    tau_p = 1.02 * dt * (2 * J + 2 * 0.4)
    kappa = 0.24 * dv * dv / dt
    ux = rng.uniform(-0.4, 0.4, (ny, nx)) * dv
    uy = rng.uniform(-0.4, 0.4, (ny, nx)) * dv
    return f, ux, uy, tau_p, kappa, dt, dv


def test_step_growth_is_bounded_by_three_times_the_diamond_maximum():
    rng = np.random.default_rng(3)
    ratios = []
    for _ in range(20):
        f, ux, uy, tau_p, kappa, dt, dv = _random_case(rng)
        g = dt / tau_p
        J = (f.shape[0] - 1) // 2
        assert g * (J + 0.4) * 2 <= 1.0 and 4 * kappa * dt / dv**2 <= 1.0
        out = L.step_2d(f, ux, uy, tau_p, kappa, dt, dv)
        B = S16.diamond_bound(S16.line_max(f))
        assert np.all(S16.line_max(out) <= 3 * B)
        ratios.append(float(np.max(S16.line_max(out) / B)))
    assert max(ratios) > 0.25  # the bound is not vacuous


def test_diamond_bound_reads_the_streamed_rows():
    # a single nonzero line: its bound must land on the rows the streaming moves it to
    nv, ny = 5, 7
    J = (nv - 1) // 2
    mx = np.zeros((nv, nv, ny))
    mx[4, 2, 1] = 1.0          # plane jy = 4 (vy index +2), input row 1 -> output row 3
    B = S16.diamond_bound(mx)
    assert B[4, 2, 3] == 1.0 and B[4, 2, 1] == 0.0
    assert B[2, 2, 3] == 1.0   # two planes down, same source line, same output row
    assert B[1, 2].max() == 0.0  # outside the diamond


@pytest.mark.parametrize("fmt", S16.FORMATS)
def test_pure_streaming_moves_stored_values_exactly(fmt):
    rng = np.random.default_rng(8)
    nv, ny, nx = 5, 6, 8
    f = rng.gamma(2.0, 1.0, (nv, nv, ny, nx))
    dec, Sc, mx = S16.encode_state(f, fmt)
    z = np.zeros((ny, nx))
    out, S2, mx2, over = S16.step_2d_stored(dec, mx, z, z, tau_p=math.inf, kappa=0.0, dt=0.1,
                                            dv=1.0, fmt=fmt)
    assert not over
    np.testing.assert_array_equal(out, L.stream_2d(dec))


@pytest.mark.parametrize("fmt", S16.FORMATS)
def test_stored_step_conserves_mass_up_to_the_dropped_residuals(fmt):
    rng = np.random.default_rng(21)
    f, ux, uy, tau_p, kappa, dt, dv = _random_case(rng)
    dec, Sc, mx = S16.encode_state(f, fmt)
    exact = L.step_2d(dec, ux, uy, tau_p, kappa, dt, dv)
    out, S2, mx2, over = S16.step_2d_stored(dec, mx, ux, uy, tau_p=tau_p, kappa=kappa, dt=dt,
                                            dv=dv, fmt=fmt)
    assert not over
    step = 2.0**-11 if fmt == "f16" else 2.0**-8
    # per cell: only the corner cell's last residual is lost
    lost = np.abs(out.sum(axis=(0, 1)) - exact.sum(axis=(0, 1)))
    assert np.all(lost <= step * np.abs(out[-1, -1]) + 1e-12 * exact.sum(axis=(0, 1)))
    assert np.all(np.abs(out / S2[..., None]) < 3 * 2.0**13)


def test_coarse_density_moment_of_a_uniform_field():
    rho = np.full((8, 8), 2.0)
    # boxes of 4 x 4 cells of area dx^2 each: mass 2 * 16 dx^2
    assert S16.coarse_density_moment(rho, 0.5, 4) == pytest.approx((2 * 16 * 0.25) ** 2)
