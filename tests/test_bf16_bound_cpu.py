"""The BF16 output-error bound used by the tensor-core closure tests holds for a CPU emulation of
that network: inputs, weights (biases folded into the row of the constant feature or of a constant
activation, as the tensor-core kernel packs them) and activations rounded to BF16, products
accumulated in FP32.  Inputs: the oracle's features of seeded states, and hidden weights scaled so
that many outputs sit near z = 0, where the bound switches from the relative to the crossing form."""
import math

import numpy as np
import torch

from bf16_bound import output_error_bound
from oracle import learned as Lr


def bf(a):
    return torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).float()


def emulated_forward(X, W, g):
    """BF16 operands, FP32 accumulation; the tanh itself exact."""
    x = bf(X.reshape(-1, X.shape[-1]))
    W1 = W["W1"].copy()
    W1[15] += W["b1"]
    z = x @ bf(W1)
    for k in (2, 3):
        h = bf(torch.relu(z).numpy())
        z = h @ bf(W[f"W{k}"]) + bf(W[f"b{k}"])
    z3 = z.double().numpy().reshape(X.shape[:-1] + (2,))
    b = np.where(z3 > 0.0, Lr.output_bounds(X, g), Lr.Y_MAX)
    return b * np.tanh(z3)


def seeded_features(seed, n=12, nv=9):
    rng = np.random.default_rng(seed)
    J = (nv - 1) // 2
    v = np.arange(-J, J + 1)
    col = np.exp(-0.5 * (v / (0.3 * J)) ** 2)
    fs = col[:, None, None, None] * col[None, :, None, None] * (1 + 0.5 * rng.random((1, 1, n, n)))
    k = 2 * math.pi / n
    xx = np.arange(n)
    ux = 0.3 * np.sin(k * xx)[None, :] * np.cos(2 * k * xx)[:, None]
    uy = -0.2 * np.cos(k * xx)[None, :] * np.sin(3 * k * xx)[:, None]
    X, _ = Lr.features(fs, ux, uy, tau_p=1.0, dt=0.05, dv=0.1, dx=0.005)
    return X


def test_bound_holds_for_the_emulated_network():
    g = 0.05
    worst = 0.0
    for seed in range(6):
        X = seeded_features(seed)
        for scale in (0.5, 1.0, 2.0):
            W = Lr.init_weights(100 + seed, scale)
            rng = np.random.default_rng(seed)
            W["b1"] = 0.05 * rng.standard_normal(W["b1"].shape)
            W["b3"] = 0.01 * rng.standard_normal(W["b3"].shape)
            W = {k: v.astype(np.float32).astype(np.float64) for k, v in W.items()}
            y, _ = Lr.mlp_forward(X, W, g)
            err = np.abs(emulated_forward(X, W, g) - y)
            bound = output_error_bound(X, W, g)
            assert np.all(err <= bound)
            worst = max(worst, float(np.max(err / bound)))
    # the bound is not vacuous: the worst case comes within a factor 20 of it
    assert worst > 0.05


def test_bound_is_a_few_roundings_where_nothing_cancels():
    X = seeded_features(1)
    W = {k: v.astype(np.float32).astype(np.float64) for k, v in Lr.init_weights(3, 1.0).items()}
    y, _ = Lr.mlp_forward(X, W, 0.05)
    bound = output_error_bound(X, W, 0.05)
    big = np.abs(y) > 0.1 * np.abs(y).max()
    assert np.median(bound[big] / np.abs(y[big])) < 0.1
