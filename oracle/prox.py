"""Losses, regularisers and their proximal operators, row-wise, in float64.

Test infrastructure (see the package header): never imported by the product.

Definition (Sec. 2.3, Proximity Operator): prox_f[v] = argmin_o 1/2 |v - o|^2 + f(o).
The ADMM wrapper touches the loss V and the regulariser r only through
prox_{tV} and prox_{tau r} (Sec. 3, "Modularity", which lists squared, l1,
hinge and multinomial logistic losses).

Readings (the paper fixes neither constants nor the multiclass hinge):
* squared loss  V(y, o) = |y - o|^2 and r(W) = |W|_F^2, no factor 1/2: the only
  constants for which the minimiser is the ridge solution (Z^T Z + n lam I)^-1 Z^T Y
  of Sec. 2.2.
* hinge, m = 1: max(0, 1 - y o), y in {-1, +1}; m > 1: one-vs-rest,
  sum_k max(0, 1 - y_k o_k) with +-1 one-hot targets.
* logistic, m = 1: log(1 + exp(-y o)), y in {-1, +1}.
* multinomial logistic: log sum_k exp(o_k) - o_c with c = argmax_k y_k (first).
* l1 regulariser r(W) = sum |W_ij|.

Methods: closed forms where they exist (squared, hinge, l2, l1); the binary
logistic prox by bisection of its monotone optimality condition to 1e-15; the
multinomial prox by damped Newton on its strictly convex objective until
the gradient is below 1e-14 (relative).

Pins: brute-force minimisation of the prox objective on random tiny inputs,
the t -> 0 limit (prox -> identity), kink cases of the hinge.
"""
import numpy as np

LOSSES = ("squared", "hinge", "logistic", "multinomial")
REGS = ("l2", "l1")


# ----------------------------------------------------------------- values
def loss_value(loss, Y, O):
    """Sum over rows of V(y_i, o_i)."""
    Y = np.asarray(Y, dtype=np.float64)
    O = np.asarray(O, dtype=np.float64)
    if loss == "squared":
        return float(((Y - O) ** 2).sum())
    if loss == "hinge":
        return float(np.maximum(0.0, 1.0 - Y * O).sum())
    if loss == "logistic":
        return float(np.logaddexp(0.0, -Y * O).sum())
    if loss == "multinomial":
        c = np.argmax(Y, axis=1)
        mx = O.max(axis=1)
        lse = mx + np.log(np.exp(O - mx[:, None]).sum(axis=1))
        return float((lse - O[np.arange(O.shape[0]), c]).sum())
    raise ValueError(loss)


def reg_value(reg, W):
    W = np.asarray(W, dtype=np.float64)
    if reg == "l2":
        return float((W * W).sum())
    if reg == "l1":
        return float(np.abs(W).sum())
    raise ValueError(reg)


# ----------------------------------------------------------------- proxes
def prox_loss(loss, V, Y, t):
    """Row-wise prox_{t V(y_i, .)}[v_i] for all rows of V (n x m)."""
    V = np.asarray(V, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    if loss == "squared":
        # stationarity: o - v - 2 t (y - o) = 0
        return (V + 2.0 * t * Y) / (1.0 + 2.0 * t)
    if loss == "hinge":
        # per entry, with u = y v (y^2 = 1): argmin_p 1/2 (p - u)^2 + t max(0, 1 - p)
        u = Y * V
        return np.where(u > 1.0, V, np.where(u < 1.0 - t, V + t * Y, Y))
    if loss == "logistic":
        return _prox_logistic(V, Y, t)
    if loss == "multinomial":
        return _prox_multinomial(V, Y, t)
    raise ValueError(loss)


def _sigmoid_neg(u):
    """1 / (1 + exp(u)) without overflow."""
    return np.where(u > 0, np.exp(-u) / (1.0 + np.exp(-u)), 1.0 / (1.0 + np.exp(np.minimum(u, 0.0))))


def _prox_logistic(V, Y, t):
    # In p = y o and a = y v the condition is p - a - t / (1 + e^p) = 0, whose
    # left side is strictly increasing in p and changes sign on [a, a + t].
    a = Y * V
    lo = a.copy()
    hi = a + t
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        f = mid - a - t * _sigmoid_neg(mid)
        lo = np.where(f < 0, mid, lo)
        hi = np.where(f < 0, hi, mid)
        if np.max(hi - lo) < 1e-15 * max(1.0, float(np.max(np.abs(a)))):
            break
    return Y * (0.5 * (lo + hi))


def _prox_multinomial(V, Y, t):
    # minimise phi(o) = 1/2 |o - v|^2 + t (lse(o) - o_c): gradient
    # g = o - v + t (softmax(o) - e_c), Hessian H = I + t (diag p - p p^T).
    # Newton steps H^-1 g by the Sherman-Morrison formula for the rank-one term
    # (H = D - t p p^T with D = I + t diag p), with a backtracking line search.
    n, m = V.shape
    c = np.argmax(Y, axis=1)
    E = np.zeros_like(V)
    E[np.arange(n), c] = 1.0
    O = V.copy()

    def phi(O):
        mx = O.max(axis=1, keepdims=True)
        lse = mx[:, 0] + np.log(np.exp(O - mx).sum(axis=1))
        return 0.5 * ((O - V) ** 2).sum(1) + t * (lse - (O * E).sum(1))

    for _ in range(200):
        mx = O.max(axis=1, keepdims=True)
        Pm = np.exp(O - mx)
        Pm /= Pm.sum(axis=1, keepdims=True)
        g = O - V + t * (Pm - E)
        if np.max(np.abs(g)) < 1e-14 * max(1.0, float(np.max(np.abs(V)))):
            break
        Dinv = 1.0 / (1.0 + t * Pm)
        Dg, Dp = Dinv * g, Dinv * Pm
        step = Dg + t * Dp * ((Pm * Dg).sum(1) / (1.0 - t * (Pm * Dp).sum(1)))[:, None]
        f0 = phi(O)
        alpha = np.ones(n)
        for _ in range(60):
            # Armijo test with a rounding allowance, so that full Newton steps
            # are taken once phi no longer changes measurably
            bad = (phi(O - alpha[:, None] * step)
                   > f0 - 1e-4 * alpha * (g * step).sum(1) + 1e-13 * np.abs(f0))
            if not bad.any():
                break
            alpha = np.where(bad, 0.5 * alpha, alpha)
        O = O - alpha[:, None] * step
    return O


def prox_reg(reg, V, tau):
    """prox_{tau r}[V], entrywise."""
    V = np.asarray(V, dtype=np.float64)
    if reg == "l2":
        # stationarity: w - v + 2 tau w = 0
        return V / (1.0 + 2.0 * tau)
    if reg == "l1":
        return np.sign(V) * np.maximum(np.abs(V) - tau, 0.0)
    raise ValueError(reg)
