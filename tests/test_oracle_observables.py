"""Pins of the observables oracle (oracle/observables.py): closed forms of the coarse-grained
density for uniform states and for the whole-domain window, the second moment against the
density's autocorrelation (FFT), and the Eulerian structure function S1 against a brute-force
average over particle pairs (Eq. def_lagS1) for a lattice built from particles."""
import numpy as np
import pytest

from oracle import observables as B


def test_uniform_state_closed_forms():
    nv, nx, dx, dv = 9, 40, 0.1, 0.3
    col = np.linspace(0.5, 1.5, nv)
    f = np.repeat(col[:, None], nx, axis=1)
    n = col.sum() * dv  # rho, the same in every cell
    widths = [1, 3, 8, 40]
    np.testing.assert_allclose(B.coarse_moment(f, dx, dv, widths),
                               [(w * dx * n) ** 2 for w in widths], rtol=1e-14)
    f2 = np.ones((5, 5, 6, 6)) * 0.25
    n2 = 25 * 0.25 * dv * dv
    np.testing.assert_allclose(B.coarse_moment(f2, dx, dv, [1, 2, 6]),
                               [(w * w * dx * dx * n2) ** 2 for w in (1, 2, 6)], rtol=1e-14)


def test_whole_domain_window_holds_the_total_mass():
    rng = np.random.default_rng(1)
    f = rng.random((17, 31))
    dx, dv = 0.2, 0.1
    M = f.sum() * dx * dv
    np.testing.assert_allclose(B.coarse_moment(f, dx, dv, [31]), [M * M], rtol=1e-13)
    f2 = rng.random((5, 5, 7, 7))
    M2 = f2.sum() * dx * dx * dv * dv
    np.testing.assert_allclose(B.coarse_moment(f2, dx, dv, [7]), [M2 * M2], rtol=1e-13)


def test_second_moment_equals_the_summed_autocorrelation():
    """<rho_r^2> = dx^2 sum_{q, q' < w} C(q - q'), C(s) = mean_i rho_i rho_{i+s} (periodic), with
    C taken from the FFT of rho; in 2D the same with the 2D autocorrelation."""
    rng = np.random.default_rng(2)
    dx, dv = 0.05, 0.2
    f = rng.random((9, 64)) ** 3
    rho = f.sum(axis=0) * dv
    C = np.fft.ifft(np.abs(np.fft.fft(rho)) ** 2).real / rho.size
    for w in (1, 2, 5, 17, 63):
        want = dx * dx * sum(C[(q - p) % 64] for q in range(w) for p in range(w))
        np.testing.assert_allclose(B.coarse_moment(f, dx, dv, [w])[0], want, rtol=1e-12)
    f2 = rng.random((3, 3, 12, 10)) ** 3
    rho2 = f2.sum(axis=(0, 1)) * dv * dv
    C2 = np.fft.ifft2(np.abs(np.fft.fft2(rho2)) ** 2).real / rho2.size
    for w in (1, 3, 4):
        want = dx ** 4 * sum(C2[(qy - py) % 12, (qx - px) % 10]
                             for qy in range(w) for py in range(w)
                             for qx in range(w) for px in range(w))
        np.testing.assert_allclose(B.coarse_moment(f2, dx, dv, [w])[0], want, rtol=1e-12)


def test_s1_equals_the_pair_average_of_particles():
    """A lattice built from particles (each adds 1 / (dx dv) to its cell): S1(s dx) is the mean
    |v_p - v_q| over the ordered particle pairs whose cells are s apart (Eq. def_lagS1)."""
    rng = np.random.default_rng(3)
    nv, nx, dx, dv = 11, 23, 0.1, 0.25
    J = (nv - 1) // 2
    npart = 400
    xi = rng.integers(0, nx, npart)
    vj = rng.integers(0, nv, npart)
    f = np.zeros((nv, nx))
    np.add.at(f, (vj, xi), 1.0 / (dx * dv))
    v = (vj - J) * dv
    seps = [0, 1, 4, 11, 22]
    num, den = B.s1_terms(f, dv, seps)
    for k, s in enumerate(seps):
        close = (xi[None, :] - xi[:, None]) % nx == s  # ordered pairs (p, q), q s cells after p
        want = np.abs(v[:, None] - v[None, :])[close].mean()
        assert num[k] / den[k] == pytest.approx(want, rel=1e-12)
        # den is the mean pair count over cells, per dx^2
        assert den[k] == pytest.approx(close.sum() / nx / dx / dx, rel=1e-12)


def test_s1_of_a_separable_state_does_not_depend_on_the_separation():
    rng = np.random.default_rng(4)
    g = rng.random(15)
    rho = rng.random(30) + 0.5
    f = g[:, None] * rho[None, :]
    num, den = B.s1_terms(f, 0.2, [0, 1, 7, 29])
    s1 = num / den
    np.testing.assert_allclose(s1, s1[0], rtol=1e-13)
