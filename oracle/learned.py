"""Learned flux correction on a coarse velocity lattice: plain FP64 CPU reference.

TEST INFRASTRUCTURE ONLY, like ``oracle/lattice.py``: nothing on the product path imports it,
and it shares no code with the CUDA library.

The paper stops at suggesting large-eddy (subgrid) models for the lattice, since its
conservation law is linear in f (Section 5, Conclusions).  This module states the learned
closure the library implements, in plain numpy:

* Coarse and fine lattices (reading R-L1).  At equal dx and V_max, a coarse lattice with
  N_c = (N_f - 1)/4 + 1 velocities per axis has dv_c = 4 dv_f, hence dt_c = dt_f / 4
  (dx = dv dt): four coarse steps span one fine step.  ``restrict`` maps a fine state to the
  coarse lattice per velocity axis: coarse cell k collects fine cells j = 4k-2 .. 4k+2 with
  weights (1/2, 1, 1, 1, 1/2), divided by 4 (the ratio of cell widths), so that the mass
  sum f dv^2 is kept.
* Features of phase-space cell (x, v_j) after streaming (reading R-L2), 16 in all:
  f*(x, v_{j+d}) / rho*(x) for the 3 x 3 velocity neighbourhood d (0 outside the box; rho* the
  streamed density sum_j f*), dt_c times the four velocity gradients (du_x/dx, du_x/dy, du_y/dx,
  du_y/dy, centred differences on the grid), the two drag Courant numbers c a_x, c a_y of the
  cell, and the constant 1.  Every feature is dimensionless.
* Network (reading R-L3): 16 -> 64 -> 64 -> 2, ReLU on both hidden layers, biases on all three,
  outputs bounded by y = b tanh(z) with b = Y_MAX = 1/4 for z <= 0 (extra diffusion) and
  b = THETA D_num for z > 0 (anti-diffusion), D_num = |ca| (1 - |ca|) / 2 the numerical
  diffusivity of the upwind flux at the face (ca the face's drag Courant number, the mean of the
  two cells'), THETA = 0.9: the learned flux never takes back all of the scheme's own diffusion.
* Correction (flux form, reading R-L5): the drag fluxes of Section 2 (reading R3) get
  c F_{jx+1/2} += y_0(jx, jy) (f*_{jx+1} - f*_{jx}) and c F_{jy+1/2} += y_1 (f*_{jy+1} - f*_{jy})
  on every interior face: a learned face diffusivity in lattice units (y > 0 moves mass up the
  gradient, i.e. takes back numerical diffusion); faces on the walls stay at zero flux.  Mass is
  kept exactly, a network with zero output gives back the plain coarse step, and the correction
  of a face is proportional to the densities next to it, so the sparse tails of f are not
  flooded by corrections sized for the bulk.
* Training loss (reading R-L4): mean square difference between the coarse state after n_c
  coarse steps and the target (the restricted fine state at the same time), plus rho_weight
  times the mean square of the density difference sum_j (f - target) per spatial cell.
  ``rollout_grad`` is its exact gradient with respect to the weights, by the adjoint of every
  step.
"""
from __future__ import annotations

import math

import numpy as np

from . import lattice as _lat

NF = 16       # features
NH = 64       # hidden units per layer
NO = 2        # outputs
Y_MAX = 0.25  # bound of the outputs towards extra diffusion
THETA = 0.9   # share of the upwind numerical diffusivity the outputs may take back


# --------------------------------------------------------------------------------------------
# coarse <-> fine
# --------------------------------------------------------------------------------------------
def restrict_matrix(nv_fine: int) -> np.ndarray:
    """R[k, j]: weight of fine velocity cell j in coarse cell k, per axis (reading R-L1)."""
    assert (nv_fine - 1) % 4 == 0
    nc = (nv_fine - 1) // 4 + 1
    Jf, Jc = (nv_fine - 1) // 2, (nc - 1) // 2
    R = np.zeros((nc, nv_fine))
    for k in range(-Jc, Jc + 1):
        for d, w in zip(range(-2, 3), (0.5, 1.0, 1.0, 1.0, 0.5)):
            j = 4 * k + d
            if -Jf <= j <= Jf:
                R[k + Jc, j + Jf] += w / 4.0
    return R


def restrict(f_fine: np.ndarray) -> np.ndarray:
    """Fine 2D state [jy, jx, y, x] -> coarse state, per axis with restrict_matrix."""
    R = restrict_matrix(f_fine.shape[0])
    return np.einsum("ab,cd,bdyx->acyx", R, R, f_fine)


# --------------------------------------------------------------------------------------------
# features, network
# --------------------------------------------------------------------------------------------
def velocity_gradients(ux: np.ndarray, uy: np.ndarray, dx: float):
    """Centred differences on the periodic grid: (du_x/dx, du_x/dy, du_y/dx, du_y/dy)."""
    def ddx(u):
        return (np.roll(u, -1, axis=1) - np.roll(u, 1, axis=1)) / (2 * dx)

    def ddy(u):
        return (np.roll(u, -1, axis=0) - np.roll(u, 1, axis=0)) / (2 * dx)

    return ddx(ux), ddy(ux), ddx(uy), ddy(uy)


def courant(ux, uy, nv, tau_p, dt, dv):
    """c a_x (varies with jx) and c a_y (varies with jy) at every phase-space cell."""
    v = _lat.velocities(nv, dv)
    c = dt / dv
    ax = c * _lat.drag_acceleration(v[None, :, None, None], ux[None, None], tau_p)
    ay = c * _lat.drag_acceleration(v[:, None, None, None], uy[None, None], tau_p)
    shp = (nv, nv) + ux.shape
    return np.broadcast_to(ax, shp), np.broadcast_to(ay, shp)


def features(fs: np.ndarray, ux, uy, *, tau_p, dt, dv, dx):
    """X[jy, jx, y, x, 16] of the streamed state fs (reading R-L2) and rho*[y, x]."""
    nv = fs.shape[0]
    rho = fs.sum(axis=(0, 1))
    inv = np.where(rho != 0.0, 1.0 / np.where(rho != 0.0, rho, 1.0), 0.0)
    X = np.zeros(fs.shape + (NF,))
    pad = np.zeros((nv + 2, nv + 2) + fs.shape[2:])
    pad[1:-1, 1:-1] = fs
    q = 0
    for dy in (-1, 0, 1):
        for dxv in (-1, 0, 1):
            X[..., q] = pad[1 + dy:1 + dy + nv, 1 + dxv:1 + dxv + nv] * inv
            q += 1
    g = velocity_gradients(ux, uy, dx)
    for i in range(4):
        X[..., 9 + i] = dt * g[i]
    cax, cay = courant(ux, uy, nv, tau_p, dt, dv)
    X[..., 13] = cax
    X[..., 14] = cay
    X[..., 15] = 1.0
    return X, rho


def init_weights(seed: int, scale: float = 1.0):
    """He-normal weights times `scale`, zero biases: W1 [16, 64], W2 [64, 64], W3 [64, 2]."""
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.standard_normal((NF, NH)) * math.sqrt(2.0 / NF) * scale,
        "b1": np.zeros(NH),
        "W2": rng.standard_normal((NH, NH)) * math.sqrt(2.0 / NH) * scale,
        "b2": np.zeros(NH),
        "W3": rng.standard_normal((NH, NO)) * math.sqrt(2.0 / NH) * scale,
        "b3": np.zeros(NO),
    }


def zero_weights():
    return {k: np.zeros_like(v) for k, v in init_weights(0).items()}


def output_bounds(X: np.ndarray, g: float):
    """Bounds b of the two outputs for z > 0: THETA |ca| (1 - |ca|) / 2 at the +jx and +jy faces,
    with ca = c a_j - g / 2 the face value of the drag Courant numbers (features 13 and 14)."""
    out = []
    for q in (13, 14):
        ca = np.abs(X[..., q] - 0.5 * g)
        out.append(THETA * np.maximum(ca * (1.0 - ca), 0.0) * 0.5)
    return np.stack(out, axis=-1)


def mlp_forward(X: np.ndarray, W, g: float = 0.0):
    """y = b tanh(relu(relu(X W1 + b1) W2 + b2) W3 + b3), b from output_bounds for z > 0 and
    Y_MAX otherwise (reading R-L3); returns y and the cache.  g = dt / tau_p."""
    z1 = X @ W["W1"] + W["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W["W2"] + W["b2"]
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ W["W3"] + W["b3"]
    t = np.tanh(z3)
    b = np.where(z3 > 0.0, output_bounds(X, g), Y_MAX)
    return b * t, (X, z1, h1, z2, h2, t, b)


def mlp_backward(dy: np.ndarray, W, cache):
    """Gradients of sum(dy * y) with respect to the weights and to X (chain rule by hand).
    The bounds depend on the flow features only, which no weight and no density moves."""
    X, z1, h1, z2, h2, t, b = cache
    rows = (dy * b * (1.0 - t * t)).reshape(-1, NO)   # through the bounded tanh
    g = {"W3": h2.reshape(-1, NH).T @ rows, "b3": rows.sum(axis=0)}
    dz2 = (rows @ W["W3"].T) * (z2.reshape(-1, NH) > 0)
    g["W2"] = h1.reshape(-1, NH).T @ dz2
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ W["W2"].T) * (z1.reshape(-1, NH) > 0)
    g["W1"] = X.reshape(-1, NF).T @ dz1
    g["b1"] = dz1.sum(axis=0)
    dX = (dz1 @ W["W1"].T).reshape(X.shape)
    return g, dX


# --------------------------------------------------------------------------------------------
# learned coarse step
# --------------------------------------------------------------------------------------------
def _drag_parts(fs, ux, uy, tau_p, dt, dv):
    cax, cay = courant(ux, uy, fs.shape[0], tau_p, dt, dv)
    return np.maximum(cax, 0.0), np.minimum(cax, 0.0), np.maximum(cay, 0.0), np.minimum(cay, 0.0)


def corrections(f, ux, uy, W, *, tau_p, dt, dv, dx):
    """Correction fluxes of one step from state f: Gx[jy, jx] through face jx + 1/2 and
    Gy[jy, jx] through face jy + 1/2 (zero on the walls), at every spatial cell."""
    fs = _lat.stream_2d(f)
    X, _ = features(fs, ux, uy, tau_p=tau_p, dt=dt, dv=dv, dx=dx)
    y, _ = mlp_forward(X, W, dt / tau_p)
    Gx = np.zeros_like(fs)
    Gx[:, :-1] = y[:, :-1, ..., 0] * (fs[:, 1:] - fs[:, :-1])
    Gy = np.zeros_like(fs)
    Gy[:-1] = y[:-1, :, ..., 1] * (fs[1:] - fs[:-1])
    return Gx, Gy


def learned_step_2d(f, ux, uy, W, *, tau_p, kappa, dt, dv, dx, keep=False):
    """Stream, corrected upwind drag, diffusion (Section 2 with the learned flux correction)."""
    fs = _lat.stream_2d(f)
    X, rho = features(fs, ux, uy, tau_p=tau_p, dt=dt, dv=dv, dx=dx)
    y, cache = mlp_forward(X, W, dt / tau_p)
    axp, axm, ayp, aym = _drag_parts(fs, ux, uy, tau_p, dt, dv)
    shp = fs.shape
    # correction fluxes y (f*_{j+1} - f*_j) on the interior faces, added to the plain drag step
    Gx = np.zeros((shp[0], shp[1] + 1) + shp[2:])
    Gx[:, 1:-1] = y[:, :-1, ..., 0] * (fs[:, 1:] - fs[:, :-1])
    Gy = np.zeros((shp[0] + 1,) + shp[1:])
    Gy[1:-1] = y[:-1, :, ..., 1] * (fs[1:] - fs[:-1])
    fss = _lat.drag_2d(fs, ux, uy, tau_p, dt, dv) - (Gx[:, 1:] - Gx[:, :-1]) - (Gy[1:] - Gy[:-1])
    out = _lat.diffuse_2d(fss, kappa, dt, dv)
    if keep:
        return out, (fs, X, rho, y, cache, axp, axm, ayp, aym)
    return out


def _diffuse_adjoint(lam, kappa, dt, dv):
    # the zero-flux five-point Laplacian step is a symmetric linear map
    return _lat.diffuse_2d(lam, kappa, dt, dv)


def _stream_adjoint(lam):
    nv = lam.shape[0]
    J = (nv - 1) // 2
    out = np.empty_like(lam)
    for jy in range(nv):
        for jx in range(nv):
            out[jy, jx] = np.roll(lam[jy, jx], (-(jy - J), -(jx - J)), axis=(0, 1))
    return out


def learned_step_adjoint(lam_out, W, saved, *, kappa, dt, dv):
    """Given dL/d(out) of one learned step, return dL/d(f) and the weight gradients."""
    fs, X, rho, y, cache, axp, axm, ayp, aym = saved
    lss = _diffuse_adjoint(lam_out, kappa, dt, dv)          # dL/df**
    lfs = lss.copy()                                         # identity part of f** = fs - ...
    # interior x faces: Fx_{j+1/2} enters f**_j with -1 and f**_{j+1} with +1
    lFx = lss[:, 1:] - lss[:, :-1]                           # dL/dFx at faces 1/2 .. J-1/2
    lFy = lss[1:] - lss[:-1]
    lfs[:, :-1] += axp[:, :-1] * lFx
    lfs[:, 1:] += axm[:, 1:] * lFx
    lfs[:-1] += ayp[:-1] * lFy
    lfs[1:] += aym[1:] * lFy
    # correction G_{j+1/2} = y_j (f*_{j+1} - f*_j)
    yx, yy = y[:, :-1, ..., 0], y[:-1, :, ..., 1]
    lfs[:, 1:] += yx * lFx
    lfs[:, :-1] -= yx * lFx
    lfs[1:] += yy * lFy
    lfs[:-1] -= yy * lFy
    dy = np.zeros_like(y)
    dy[:, :-1, ..., 0] = (fs[:, 1:] - fs[:, :-1]) * lFx
    dy[:-1, :, ..., 1] = (fs[1:] - fs[:-1]) * lFy
    lrho = np.zeros(fs.shape[2:])
    g, dX = mlp_backward(dy, W, cache)
    # neighbour features f*(v + d) / rho*
    nv = fs.shape[0]
    inv = np.where(rho != 0.0, 1.0 / np.where(rho != 0.0, rho, 1.0), 0.0)
    pad = np.zeros((nv + 2, nv + 2) + fs.shape[2:])
    q = 0
    for d_y in (-1, 0, 1):
        for d_x in (-1, 0, 1):
            pad[1 + d_y:1 + d_y + nv, 1 + d_x:1 + d_x + nv] += dX[..., q] * inv
            lrho -= (dX[..., q] * X[..., q]).sum(axis=(0, 1)) * inv
            q += 1
    lfs += pad[1:-1, 1:-1]
    lfs += lrho  # rho* = sum_j f*_j
    return _stream_adjoint(lfs), g


def rollout(f0, W, nsteps, flows, *, tau_p, kappa, dt, dv, dx, keep=False):
    """nsteps learned coarse steps; flows[n] = (ux, uy) of step n."""
    f = np.array(f0, dtype=np.float64, copy=True)
    saved = []
    for n in range(nsteps):
        ux, uy = flows[n]
        if keep:
            f, s = learned_step_2d(f, ux, uy, W, tau_p=tau_p, kappa=kappa, dt=dt, dv=dv, dx=dx,
                                   keep=True)
            saved.append(s)
        else:
            f = learned_step_2d(f, ux, uy, W, tau_p=tau_p, kappa=kappa, dt=dt, dv=dv, dx=dx)
    return (f, saved) if keep else f


def loss_value(f, target, rho_weight=0.0):
    """mean (f - target)^2 + rho_weight mean_x (sum_j (f - target))^2 (reading R-L4)."""
    d = f - target
    r = d.sum(axis=(0, 1))
    return float(np.mean(d * d) + rho_weight * np.mean(r * r))


def loss(f0, W, nsteps, flows, target, rho_weight=0.0, **kw):
    """The training loss after nsteps learned steps."""
    return loss_value(rollout(f0, W, nsteps, flows, **kw), target, rho_weight)


def rollout_grad(f0, W, nsteps, flows, target, *, tau_p, kappa, dt, dv, dx, rho_weight=0.0):
    """Loss and its exact gradient with respect to every weight (adjoint of every step)."""
    f, saved = rollout(f0, W, nsteps, flows, tau_p=tau_p, kappa=kappa, dt=dt, dv=dv, dx=dx,
                       keep=True)
    L = loss_value(f, target, rho_weight)
    d = f - target
    r = d.sum(axis=(0, 1))
    lam = 2.0 * d / f.size + rho_weight * 2.0 * r / r.size
    grads = {k: np.zeros_like(v) for k, v in W.items()}
    for n in reversed(range(nsteps)):
        lam, g = learned_step_adjoint(lam, W, saved[n], kappa=kappa, dt=dt, dv=dv)
        for k in grads:
            grads[k] += g[k]
    return L, grads
