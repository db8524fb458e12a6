"""Gain of the learned closure: trained on the GPU against restricted fine runs, it brings the
coarse 9 x 9 lattice closer to the fine 33 x 33 lattice than the plain coarse step does, on held-out
flows.

Set-up (reading R-L1..R-L5 of the closure): 32 x 32 grid, St = 1, kappa = 1e-3, frozen random-phase
flows, Gaussian velocity start (sigma = 0.3 V_max) with a seeded spatial modulation.  Training data:
three flows (seeds 101..103), 60 fine steps each, restricted to the coarse lattice; Adam on the
loss of 32 coarse steps (8 fine steps) with a density term (rho_weight 0.3).  Held out: flows 202
and 303.  Errors: relative errors of <|v|^2> and <rho_r^2> (r = 4 cells, lat_coarse_moment) against the
fine run, averaged over fine steps 30, 60, 90 and 120; both must fall below 0.85 times those of
the plain coarse lattice, for the FP32 network and for the BF16 tensor-core network.
"""
import numpy as np
import pytest

from paper_1508_02899_gb300 import lat
from paper_1508_02899_gb300 import train as T

pytestmark = pytest.mark.gpu

NX, ST, KAPPA, R = 32, 1.0, 1e-3, 4
TIMES = (30, 60, 90, 120)


def held_out_errors(params, seed, mode):
    base = T.make_pair(NX, NX, 33, ST, KAPPA, flow_seed=seed, init_seed=seed + 1)
    learned = T.make_pair(NX, NX, 33, ST, KAPPA, flow_seed=seed, init_seed=seed + 1)
    learned.coarse.learn(params, mode)
    err = {"plain": [], "learned": []}
    for k in range(1, max(TIMES) + 1):
        base.fine.step(1)
        base.coarse.step(T.COARSE_PER_FINE)
        learned.coarse.step(T.COARSE_PER_FINE)
        if k in TIMES:
            vf, rf, cf = T.observables(base.fine, base.dx, R)
            for name, lt in (("plain", base.coarse), ("learned", learned.coarse)):
                v, r, code = T.observables(lt, base.dx, R)
                assert code == 0 and cf == 0
                err[name].append((abs(v - vf) / vf, abs(r - rf) / rf))
            fc = lat.restrict(base.fine.state, NX, NX)
            assert float(learned.coarse.state.min()) > -0.05 * float(fc.max())
    return {k: np.mean(np.array(v), axis=0) for k, v in err.items()}


@pytest.fixture(scope="module")
def trained():
    pairs = [T.make_pair(NX, NX, 33, ST, KAPPA, flow_seed=s, init_seed=s + 7) for s in (101, 102, 103)]
    trajs = [T.restricted_trajectory(p, 60) for p in pairs]
    params = T.train(pairs, trajs, 800, lr=1e-3, seed=1, fine_steps=8, rho_weight=0.3)
    assert np.all(np.isfinite(params))
    return params


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("seed", [202, 303])
def test_learned_closure_beats_the_plain_coarse_lattice(lat, trained, seed, mode):
    e = held_out_errors(trained, seed, mode)
    print(f"\n[seed {seed} mode {mode}] <|v|^2> err plain {e['plain'][0]:.3e} learned "
          f"{e['learned'][0]:.3e}; <rho_r^2> err plain {e['plain'][1]:.3e} learned "
          f"{e['learned'][1]:.3e}", end="")
    # measured: the closure cuts the <|v|^2> error by about 45 % and the <rho_r^2> error by
    # about two thirds on both held-out flows; asserted with a margin
    assert e["learned"][0] < 0.85 * e["plain"][0]
    assert e["learned"][1] < 0.85 * e["plain"][1]
