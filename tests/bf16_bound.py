"""Tolerance on the BF16 tensor-core closure network's outputs, per output.

The tensor-core network rounds its inputs X, its weights and biases, and both hidden activations
to BF16 (8 significant bits, unit roundoff u = 2^-8) and accumulates in FP32.  A worst-case bound
on that arithmetic grows by sum_i |W_ij| per layer while the outputs grow by about
sqrt(sum_i W_ij^2), so after three layers it exceeds the outputs themselves.  The tolerance
therefore follows probabilistic rounding-error analysis instead.  Each rounding of a value a is
an independent, zero-mean error, uniform on [-u|a|, u|a|] (variance u^2 a^2 / 3).  Variances then
propagate through the layers:

    V(z1_j) = sum_i (u^2/3) (2 X_i^2 W1_ij^2) + (u^2/3) b1_j^2
    V(h_k)  = m_k V(z_k) + (u^2/3) h_k^2    m_k = 1 where the unit may be active (z_k + lam s > 0)
    V(z_k+1_j) = sum_i W_ij^2 V(h_k,i) + (u^2/3) sum_i (h_k,i^2 + V(h_k,i)) W_ij^2 + (u^2/3) b_j^2

z3 then lies within E = lam sqrt(V(z3)) of the exact value, with lam = 6, plus the worst case of
FP32 accumulation.  The output is y = b(z) tanh(z), with the bound b chosen by the sign of z.
Where |z3| > E both sides take the same b, and |dy| <= b (E + the tanh approximation's error).
Elsewhere either b may be taken, and |dy| <= |y| + |y^|, each below max(b) (|z3| + E).
"""
import numpy as np

from oracle import learned as Lr

U = 2.0**-8
R = U * U / 3.0          # variance of one BF16 rounding, per unit squared value
U32 = 2.0**-22           # FP32 accumulation over at most 80 terms, worst case, with margin
TANH_REL = 2.0**-10      # relative error of the hardware tanh approximation, with margin
LAM = 6.0


def z_tolerance(X, W):
    """(z3, E): the oracle's last pre-activation and the tolerance on its BF16 counterpart."""
    z = X @ W["W1"] + W["b1"]
    V = R * (2 * (X * X) @ (W["W1"] ** 2) + W["b1"] ** 2)
    A = np.abs(X) @ np.abs(W["W1"]) + np.abs(W["b1"])
    for k in (2, 3):
        Wk, bk = W[f"W{k}"], W[f"b{k}"]
        s = np.sqrt(V)
        h = np.maximum(z, 0.0)
        Vh = np.where(z + LAM * s > 0.0, V, 0.0) + R * h * h
        A = np.abs(h) @ np.abs(Wk) + np.abs(bk)
        z = h @ Wk + bk
        V = Vh @ (Wk ** 2) + R * ((h * h + Vh) @ (Wk ** 2)) + R * bk ** 2
    return z, LAM * np.sqrt(V) + U32 * A


def output_error_bound(X, W, g):
    """Tolerance on |y_bf16 - y_exact|, same shape as the oracle's y (..., 2)."""
    z3, E = z_tolerance(X, W)
    bpos = Lr.output_bounds(X, g)
    bmax = np.maximum(bpos, Lr.Y_MAX)
    b = np.where(z3 > 0.0, bpos, Lr.Y_MAX)
    same = np.abs(z3) > E
    t = np.abs(np.tanh(z3))
    near = b * (E + TANH_REL * (t + E))
    cross = bmax * (2 * np.abs(z3) + E) * (1 + TANH_REL)
    return np.where(same, near, cross)
