"""Host density I/O and checkpoints through the C ABI (lat_get_density / lat_set_density,
lat_state_bytes / lat_get_state / lat_set_state).

A checkpoint must let a run continue bit for bit: the scheme of Section 2 is a deterministic map
of the density, the step count, the flow state and the noise draws, so a context restored from an
image of step n and stepped m times must hold exactly the bits of the uninterrupted run after
n + m steps, for every storage type and every form of the step (1D lattices and ensembles, the
flux-limited drag, 2D FP32, FP16 and BF16 storage, the learned closure).
"""
import math

import numpy as np
import pytest
import torch

from oracle import learned as Lr
from paper_1508_02899_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L = 2 * math.pi
N_BEFORE, N_AFTER = 7, 9


def _pack(W):
    return np.concatenate([W["W1"].ravel(), W["b1"], W["W2"].ravel(), W["b2"], W["W3"].ravel(),
                           W["b3"]]).astype(np.float32)


def _lattice1d(lat, dtype, seed, scheme=None):
    nx, nv, st, kappa = 264, 33, 1.0, 1e-3
    tau_p = st * L
    mu = 2.0 / 3.0
    dt = I.choose_dt(1, nx, L, nv, tau_p, kappa, cfl_factor=(1 + mu) if scheme else 1.0)
    f0 = I.random_initial((nv, nx), seed)
    t = torch.tensor(f0, dtype=dtype, device="cuda")
    lt = lat.Lattice(t, d=1, nx=nx, nv=nv, L=L, tau_p=tau_p, kappa=kappa, dt=dt)
    fl = I.flow1d_inputs(5, 40)
    lt.set_flow_modes_1d(fl.k, fl.amp0[0], fl.tau_f, fl.sigma)
    if scheme:
        lt.set_scheme(lat.SCHEME_KOREN, mu)
    return lt, lambda ctx: ctx.set_noise(fl.noise[:, 0, :])


def _ensemble(lat, dtype, seed, scheme=None):
    nv = 33
    mu = 2.0 / 3.0
    tab = I.ensemble_table(6, 3, nv=nv, sizes=(256, 512, 132, 1024, 136, 300),
                           cfl_factor=(1 + mu) if scheme else 1.0)
    parts = [I.random_initial((nv, int(n)), seed + i) for i, n in enumerate(tab.nx)]
    t = torch.tensor(np.concatenate([p.ravel() for p in parts]), dtype=dtype, device="cuda")
    ens = lat.Ensemble(t, nv=nv, nx=tab.nx, L=tab.L, tau_p=tab.tau_p, kappa=tab.kappa,
                       dt=tab.dt)
    fl = I.flow1d_inputs(9, 40, n_inst=len(tab.nx))
    ens.set_flow_modes(fl.k, fl.amp0, fl.tau_f, fl.sigma)
    if scheme:
        ens.set_scheme(lat.SCHEME_KOREN, mu)
    return ens, lambda ctx: ctx.set_noise(fl.noise)


def _lattice2d(lat, dtype, seed, nx=136, ny=24, nv=17, learn=0, scheme=None):
    st, kappa = 1.0, 1e-3
    tau_p = st * L
    mu = 2.0 / 3.0
    dt = I.choose_dt(2, nx, L, nv, tau_p, kappa, cfl_factor=(1 + mu) if scheme else 1.0)
    dx = L / nx
    f0 = I.random_initial((nv, nv, ny, nx), seed)
    half = dtype in (torch.float16, torch.bfloat16)
    t = torch.zeros(f0.shape, dtype=dtype, device="cuda") if half else \
        torch.tensor(f0, dtype=dtype, device="cuda")
    lt = lat.Lattice(t, d=2, nx=nx, ny=ny, nv=nv, L=L, tau_p=tau_p, kappa=kappa, dt=dt)
    if half:
        lt.encode(torch.tensor(f0, dtype=torch.float32, device="cuda"))
    fl = I.flow2d_inputs(41, 40, nx, ny, dx, kmax=4)  # the same flow for every seed
    lt.set_flow_modes_2d(fl.kvec, fl.a, fl.phi0, fl.tau_f)
    if learn:
        lt.learn(_pack(Lr.init_weights(3, 0.4)), learn)
    if scheme:
        lt.set_scheme(lat.SCHEME_KOREN, mu)
    return lt, lambda ctx: ctx.set_noise(fl.noise)


FORMS = {
    "1d_f64": lambda lat, s: _lattice1d(lat, torch.float64, s),
    "1d_f32_koren": lambda lat, s: _lattice1d(lat, torch.float32, s, scheme=True),
    "ensemble_f32": lambda lat, s: _ensemble(lat, torch.float32, s),
    "ensemble_f64_koren": lambda lat, s: _ensemble(lat, torch.float64, s, scheme=True),
    "2d_f64": lambda lat, s: _lattice2d(lat, torch.float64, s, nx=40, ny=24, nv=9),
    "2d_f32": lambda lat, s: _lattice2d(lat, torch.float32, s),
    "2d_f16": lambda lat, s: _lattice2d(lat, torch.float16, s),
    "2d_bf16": lambda lat, s: _lattice2d(lat, torch.bfloat16, s),
    "2d_f32_koren": lambda lat, s: _lattice2d(lat, torch.float32, s, nx=48, ny=40, nv=9,
                                              scheme=True),
    "2d_learned_tc": lambda lat, s: _lattice2d(lat, torch.float32, s, nx=32, ny=32, nv=9,
                                               learn=2),
    "2d_learned_f32": lambda lat, s: _lattice2d(lat, torch.float32, s, nx=40, ny=24, nv=9,
                                                learn=1),
}


def _snapshot(ctx):
    """Raw bits of the current buffer (and 16-bit scales)."""
    raw = ctx.state.contiguous().view(torch.uint8).cpu().numpy().copy()
    if ctx.state.dtype in (torch.float16, torch.bfloat16):
        _, sc = ctx.decode()
        return raw, sc.cpu().numpy().copy()
    return raw, None


@pytest.mark.parametrize("form", list(FORMS))
def test_resume_is_bit_for_bit(lat, form):
    a, noise_a = FORMS[form](lat, 100)
    noise_a(a)
    a.step(N_BEFORE)
    assert a.status() == 0
    img = a.get_state()
    a.step(N_AFTER)
    assert a.status() == 0
    want = _snapshot(a)
    steps = a.steps_done

    # a fresh context with another initial state and no noise rows: the image brings them
    b, _ = FORMS[form](lat, 200)
    b.set_state(img)
    assert b.steps_done == N_BEFORE and b.current_index == N_BEFORE & 1
    b.step(N_AFTER)
    assert b.status() == 0
    got = _snapshot(b)
    assert b.steps_done == steps
    assert np.array_equal(got[0], want[0])
    if want[1] is not None:
        assert np.array_equal(got[1], want[1])

    # rewinding the first context gives the same bits again
    a.set_state(img)
    a.step(N_AFTER)
    assert a.status() == 0
    again = _snapshot(a)
    assert np.array_equal(again[0], want[0])
    a.close()
    b.close()


def test_image_keeps_the_noise_window(lat):
    """The image carries the noise rows not yet used: 40 rows, 7 used, so a restored context
    runs 33 more steps cleanly and the 34th reports LAT_ENOISE, as the original does."""
    a, noise_a = FORMS["2d_f32"](lat, 1)
    noise_a(a)
    a.step(7)
    img = a.get_state()
    b, _ = FORMS["2d_f32"](lat, 2)
    b.set_state(img)
    for ctx in (a, b):
        ctx.step(33)
        assert ctx.status() == 0
        ctx.step(1)
        assert ctx.status() == lat.LAT_ENOISE
    assert np.array_equal(a.state.cpu().numpy(), b.state.cpu().numpy())
    a.close()
    b.close()


def test_set_state_refuses_other_lattices(lat):
    a, noise_a = FORMS["2d_f32"](lat, 1)
    noise_a(a)
    a.step(3)
    img = a.get_state()
    other, _ = _lattice2d(lat, torch.float32, 5, nx=136, ny=24, nv=9)       # another N_v
    with pytest.raises(lat.LatError) as e:
        other.set_state(img)
    assert e.value.code == lat.LAT_EINVAL
    wide, _ = _lattice2d(lat, torch.float32, 5, nx=144, ny=24, nv=17)       # another N_x
    with pytest.raises(lat.LatError):
        wide.set_state(img)
    f64, _ = _lattice2d(lat, torch.float64, 5)                               # another dtype
    with pytest.raises(lat.LatError):
        f64.set_state(img)
    still, _ = FORMS["2d_f32"](lat, 3)
    still.set_flow_none()                                                    # another flow kind
    with pytest.raises(lat.LatError):
        still.set_state(img)
    fresh, _ = FORMS["2d_f32"](lat, 3)
    with pytest.raises(lat.LatError):
        fresh.set_state(img[: img.size - 1])                                 # truncated
    bad = img.copy()
    bad[0] ^= 0xFF                                                           # not an image
    with pytest.raises(lat.LatError):
        fresh.set_state(bad)
    fresh.set_state(img)  # the refusals left it usable
    assert fresh.steps_done == 3
    for ctx in (a, other, wide, f64, still, fresh):
        ctx.close()


@pytest.mark.parametrize("form", ["1d_f64", "ensemble_f32", "2d_f64", "2d_f32"])
def test_density_roundtrip(lat, form):
    ctx, _ = FORMS[form](lat, 4)
    n = ctx.f[0].numel()
    rng = np.random.default_rng(8)
    x = rng.random(n) * 3.0 + 1e-3
    ctx.set_density(x)
    got = ctx.get_density()
    if ctx.f[0].dtype == torch.float64:
        assert np.array_equal(got, x)
    else:
        assert np.array_equal(got, x.astype(np.float32).astype(np.float64))
    # the device buffer holds the same values
    assert np.array_equal(ctx.state.double().cpu().numpy().ravel(), got)
    ctx.close()


@pytest.mark.parametrize("form", ["2d_f16", "2d_bf16"])
def test_density_roundtrip_16bit(lat, form):
    """16-bit storage: lat_set_density encodes like lat_encode of the FP32-rounded values, and
    lat_get_density returns the decoded values h S exactly."""
    a, _ = FORMS[form](lat, 4)
    b, _ = FORMS[form](lat, 4)
    rng = np.random.default_rng(8)
    x = rng.random(a.f[0].numel()) * 3.0 + 1e-3
    a.set_density(x)
    b.encode(torch.tensor(x.astype(np.float32).reshape(b.f[0].shape), device="cuda"))
    dec_b, sc_b = b.decode()
    dec_a, sc_a = a.decode()
    assert torch.equal(sc_a, sc_b) and torch.equal(dec_a, dec_b)
    got = a.get_density()
    assert np.array_equal(got, dec_b.double().cpu().numpy().ravel())
    # each value within half a storage step of itself plus the carried half step of its
    # predecessor in the column (all lines of about the same size here)
    step = 2.0 ** -10 if form == "2d_f16" else 2.0 ** -7
    assert np.abs(got - x).max() <= 2 * step * x.max()
    a.close()
    b.close()
