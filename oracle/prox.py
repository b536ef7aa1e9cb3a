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
* l1 loss: |y - o|_1 = sum_k |y_k - o_k| (real targets).
* multiclass hinge (Crammer and Singer): max_k (Delta_k + o_k - o_c) with
  Delta_k = 1 - [k = c] and c = argmax_k y_k (first); zero when o_c beats every
  other output by a margin of 1.
* l1 regulariser r(W) = sum |W_ij|.

Methods: closed forms where they exist (squared, hinge, l1 loss, l2, l1); the
binary logistic prox by bisection of its monotone optimality condition to 1e-15;
the multinomial prox by damped Newton on its strictly convex objective until
the gradient is below 1e-14 (relative); the multiclass hinge prox through its
dual, a Euclidean projection onto the probability simplex computed by sorting.

Pins: brute-force minimisation of the prox objective on random tiny inputs,
the t -> 0 limit (prox -> identity), kink cases of the hinge, the optimality
(subgradient) conditions of the multiclass hinge and its two-class reduction to
the binary hinge of the output difference (tests/test_oracle_prox.py).  The values
(loss_value, reg_value): every loss and regulariser written from its definition in
40-digit arithmetic, special values (log 2, log m, unit margins), the two-class
reductions of the multinomial and multiclass hinge losses to the binary ones, shift
invariance, the logistic asymptotes, the Moreau-envelope gradient identity that ties
each value to its prox, and the converged ADMM iterate minimising the objective they
compose (tests/test_oracle_values.py).
"""
import numpy as np

LOSSES = ("squared", "hinge", "logistic", "multinomial", "l1", "crammer_singer")
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
    if loss == "l1":
        return float(np.abs(Y - O).sum())
    if loss == "crammer_singer":
        n, m = O.shape
        c = np.argmax(Y, axis=1)
        Delta = np.ones((n, m))
        Delta[np.arange(n), c] = 0.0
        return float((Delta + O - O[np.arange(n), c][:, None]).max(axis=1).sum())
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
    if loss == "l1":
        # per entry: argmin_o 1/2 (o - v)^2 + t |y - o| is v - y soft-thresholded by t, about y
        Dv = V - Y
        return Y + np.sign(Dv) * np.maximum(np.abs(Dv) - t, 0.0)
    if loss == "crammer_singer":
        return _prox_crammer_singer(V, Y, t)
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


def _project_simplex(U):
    """Row-wise Euclidean projection onto {a >= 0, sum a = 1}, by sorting.

    With the entries sorted decreasingly, u_(1) >= ... >= u_(m), the projection is
    max(u - tau, 0) where tau = (sum_{i <= r} u_(i) - 1) / r and r is the largest j
    with u_(j) > (sum_{i <= j} u_(i) - 1) / j (Held, Wolfe and Crowder 1974; Duchi,
    Shalev-Shwartz, Singer and Chandra 2008).
    """
    n, m = U.shape
    S = -np.sort(-U, axis=1)
    cs = np.cumsum(S, axis=1)
    j = np.arange(1, m + 1)
    ok = S - (cs - 1.0) / j > 0
    r = m - np.argmax(ok[:, ::-1], axis=1)          # last j where ok holds (j = 1 always does)
    tau = (cs[np.arange(n), r - 1] - 1.0) / r
    return np.maximum(U - tau[:, None], 0.0)


def _prox_crammer_singer(V, Y, t):
    # V(y, o) = max_k (Delta_k + o_k - o_c) = max over the probability simplex of
    # a^T Delta + (a - e_c)^T o (sum a = 1).  Exchanging min over o and max over a
    # (the objective is convex in o, concave in a), the inner minimiser of
    # 1/2 |o - v|^2 + t (a - e_c)^T o is o = v - t (a - e_c); what is left to
    # maximise over a is, up to constants, -t^2/2 |a - e_c - (Delta + v)/t|^2, so a is
    # the projection of e_c + (Delta + v)/t onto the simplex.
    n, m = V.shape
    if t <= 0.0:
        return V.copy()
    c = np.argmax(Y, axis=1)
    E = np.zeros((n, m))
    E[np.arange(n), c] = 1.0
    Delta = 1.0 - E
    A = _project_simplex(E + (Delta + V) / t)
    return V - t * (A - E)


def prox_reg(reg, V, tau):
    """prox_{tau r}[V], entrywise."""
    V = np.asarray(V, dtype=np.float64)
    if reg == "l2":
        # stationarity: w - v + 2 tau w = 0
        return V / (1.0 + 2.0 * tau)
    if reg == "l1":
        return np.sign(V) * np.maximum(np.abs(V) - tau, 0.0)
    raise ValueError(reg)
