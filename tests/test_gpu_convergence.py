"""The paper's first-order convergence claim (Sec. 3.2): on its 1D set-up (V_max = u_rms = 1,
dt = 2^-6 pi, N_v = 2^n + 1, N_x = 2^(n+6)), the relative L2 error of the coarse-grained density
on boxes of L / 128, against the finest lattice of the study, shrinks in proportion to dv."""
import numpy as np
import pytest

from paper_1508_02899_gb300 import convergence as C
from paper_1508_02899_gb300 import lat as _lat

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("st", [4.0, 8.0])
def test_upwind_lattice_converges_at_first_order_in_dv(lat, st):
    levels = [2, 3, 4, 5, 6, 7]  # N_v = 5 .. 129; N_v = 129 is the reference
    dvs, errs = C.study(levels, st)
    print(f"\n[St {st}] dv {dvs[:-1]} errors {errs}", end="")
    assert np.all(np.diff(errs) < 0)
    # the reference carries its own first-order error: compare e_n with dv_n - dv_ref.  The
    # coarsest lattices (N_v = 5, 9) are far from the asymptotic range; the local order rises
    # with the resolution (measured 0.33, 0.52, 0.68, 0.85 at St = 4 and 0.35, 0.74, 0.82, 0.90
    # at St = 8) and is checked on the finest pair
    x = dvs[:-1] - dvs[-1]
    order = np.log(errs[:-1] / errs[1:]) / np.log(x[:-1] / x[1:])
    print(f" local orders {order}", end="")
    assert np.all(np.diff(order) > 0), order
    assert 0.75 < order[-1] < 1.25, order


def test_limited_scheme_is_more_accurate(lat):
    levels = [2, 3, 4, 5, 6]
    _, e_up = C.study(levels, 8.0)
    _, e_lim = C.study(levels, 8.0, scheme=_lat.SCHEME_KOREN)
    print(f"\n[upwind] {e_up} [limited] {e_lim}", end="")
    # on the coarsest lattices (N_v = 5, 9) the limiter has too few cells to help; from N_v = 17
    # on its errors are smaller and fall faster (measured: 0.042 vs 0.053, 0.010 vs 0.020)
    assert np.all(e_lim[-2:] < e_up[-2:])
    assert e_lim[-2] / e_lim[-1] > e_up[-2] / e_up[-1]
