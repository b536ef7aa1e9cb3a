"""Pins for the oracle's proximal operators: brute-force minimisation of the definition."""
import numpy as np
import pytest
from scipy import optimize

from oracle import prox as P


mp = pytest.importorskip("mpmath").mp
mp.dps = 40
from loss_definitions import row_loss_mp  # noqa: E402  (the losses from their definitions)


def _golden(f, a, b, tol=1e-25):
    """Golden-section minimisation of a unimodal f on [a, b], in 40-digit arithmetic.

    Function values limit a value-based search to sqrt(precision) in position,
    so the search runs in mpmath: ~1e-20 in position, far below float64 rounding.
    """
    a, b = mp.mpf(a), mp.mpf(b)
    g = (mp.sqrt(5) - 1) / 2
    c, d = b - g * (b - a), a + g * (b - a)
    fc, fd = f(c), f(d)
    while b - a > tol * max(1, abs(a) + abs(b)):
        if fc < fd:
            b, d, fd = d, c, fc
            c = b - g * (b - a)
            fc = f(c)
        else:
            a, c, fc = c, d, fd
            d = a + g * (b - a)
            fd = f(d)
    return float((a + b) / 2)


def _loss_mp(loss, y, o):
    """V(y, o) for scalars, written from its definition in mpmath."""
    if loss == "squared":
        return (y - o) ** 2
    if loss == "hinge":
        return mp.mpf(0) if 1 - y * o < 0 else 1 - y * o
    if loss == "logistic":
        return mp.log(1 + mp.exp(-y * o))
    if loss == "l1":
        return abs(y - o)
    raise ValueError(loss)


def _brute_scalar(loss, v, y, t):
    v, y, t = mp.mpf(v), mp.mpf(y), mp.mpf(t)
    f = lambda o: (o - v) ** 2 / 2 + t * _loss_mp(loss, y, o)
    span = abs(v) + abs(y) + t + 2
    return _golden(f, v - span, v + span)


@pytest.mark.parametrize("loss", ["squared", "hinge", "logistic", "l1"])
def test_scalar_losses_brute_force(loss):
    rng = np.random.default_rng(1)
    for _ in range(150):
        t = float(10 ** rng.uniform(-3, 1.5))
        v = float(rng.normal() * 3)
        y = float(rng.normal()) if loss == "squared" else float(rng.choice([-1.0, 1.0]))
        got = P.prox_loss(loss, np.array([[v]]), np.array([[y]]), t)[0, 0]
        ref = _brute_scalar(loss, v, y, t)
        assert abs(got - ref) < 1e-12 * max(1.0, abs(ref)), (loss, v, y, t, got, ref)


def test_hinge_one_vs_rest_is_entrywise():
    rng = np.random.default_rng(2)
    V = rng.normal(size=(7, 5)) * 2
    Y = np.where(rng.random((7, 5)) < 0.5, -1.0, 1.0)
    t = 0.7
    got = P.prox_loss("hinge", V, Y, t)
    for r in range(7):
        for k in range(5):
            assert abs(got[r, k] - _brute_scalar("hinge", V[r, k], Y[r, k], t)) < 1e-12


def test_hinge_kinks():
    t = 0.5
    # y v > 1: untouched; y v < 1 - t: shifted by t y; in between: clamped to y
    V = np.array([[1.5, -1.5, 0.2, -0.8, 0.75]])
    Y = np.array([[1.0, -1.0, 1.0, -1.0, 1.0]])
    got = P.prox_loss("hinge", V, Y, t)
    assert np.allclose(got, [[1.5, -1.5, 0.7, -1.0, 1.0]], atol=0, rtol=0)


@pytest.mark.parametrize("m", [2, 3, 6])
def test_multinomial_brute_force(m):
    rng = np.random.default_rng(3 + m)
    for _ in range(30):
        t = float(10 ** rng.uniform(-2, 1))
        v = rng.normal(size=m) * 2
        c = int(rng.integers(m))
        y = -np.ones(m)
        y[c] = 1.0
        # the objective from the loss's own definition, not from the oracle's loss_value
        f = lambda o: 0.5 * np.sum((o - v) ** 2) + t * float(row_loss_mp("multinomial", y, o))
        res = optimize.minimize(f, v, method="BFGS", options=dict(gtol=1e-13, maxiter=5000))
        got = P.prox_loss("multinomial", v[None], y[None], t)[0]
        assert np.max(np.abs(got - res.x)) < 1e-6
        # and the oracle's answer is at least as good as the generic minimiser's
        assert f(got) <= f(res.x) + 1e-12


@pytest.mark.parametrize("loss", ["squared", "hinge", "logistic", "multinomial", "l1", "crammer_singer"])
def test_small_step_is_identity(loss):
    rng = np.random.default_rng(4)
    V = rng.normal(size=(5, 3)) * 2
    Y = -np.ones((5, 3))
    Y[np.arange(5), rng.integers(0, 3, 5)] = 1.0
    if loss == "logistic":
        V, Y = V[:, :1], Y[:, :1]
    got = P.prox_loss(loss, V, Y, 1e-12)
    assert np.max(np.abs(got - V)) < 1e-10


def test_squared_large_step_goes_to_target():
    V = np.array([[3.0, -2.0]])
    Y = np.array([[0.5, 0.25]])
    assert np.allclose(P.prox_loss("squared", V, Y, 1e9), Y, atol=1e-8)


@pytest.mark.parametrize("reg", ["l2", "l1"])
def test_regulariser_brute_force(reg):
    rng = np.random.default_rng(5)
    for _ in range(150):
        tau = float(10 ** rng.uniform(-3, 1))
        v = float(rng.normal() * 2)
        vm, tm = mp.mpf(v), mp.mpf(tau)
        r = (lambda w: w * w) if reg == "l2" else (lambda w: abs(w))
        f = lambda w: (w - vm) ** 2 / 2 + tm * r(w)
        ref = _golden(f, vm - abs(vm) - 1, vm + abs(vm) + 1)
        got = P.prox_reg(reg, np.array([[v]]), tau)[0, 0]
        assert abs(got - ref) < 1e-12 * max(1.0, abs(ref))


def test_l1_loss_kinks():
    t = 0.5
    # |v - y| <= t: the output sits on the target; otherwise it moves t towards it
    V = np.array([[1.2, 0.9, -3.0, 2.0]])
    Y = np.array([[1.0, 1.5, -1.0, 2.0]])
    got = P.prox_loss("l1", V, Y, t)
    assert np.allclose(got, [[1.0, 1.4, -2.5, 2.0]], atol=0, rtol=1e-15)


def _cs_problem(rng, m):
    t = float(10 ** rng.uniform(-2, 1))
    v = rng.normal(size=m) * rng.choice([0.3, 1.0, 3.0])
    c = int(rng.integers(m))
    y = -np.ones(m)
    y[c] = 1.0
    return v, y, c, t


@pytest.mark.parametrize("m", [2, 3, 5, 10, 147])
def test_crammer_singer_optimality_conditions(m):
    """o = prox_{tV}(v) iff (v - o)/t is a subgradient of V at o.

    V(o) = max_k (Delta_k + o_k - o_c) has subdifferential conv{e_k - e_c : k active},
    active = the maximising k.  So g = (v - o)/t must be a - e_c with a >= 0,
    sum a = 1 and a_k = 0 off the active set (this reads the definition of the
    subdifferential, not the projection the oracle uses).
    """
    rng = np.random.default_rng(40 + m)
    for _ in range(200):
        v, y, c, t = _cs_problem(rng, m)
        o = P.prox_loss("crammer_singer", v[None], y[None], t)[0]
        a = (v - o) / t
        a[c] += 1.0
        scale = 1e-9 * (1.0 + np.abs(v).max() / t)
        assert a.min() > -scale
        assert abs(a.sum() - 1.0) < scale
        delta = np.ones(m)
        delta[c] = 0.0
        margin = delta + o - o[c]
        active = margin >= margin.max() - 1e-9 * (1.0 + np.abs(o).max())
        assert np.all(a[~active] < scale), (a, margin)


def test_crammer_singer_two_classes_is_binary_hinge_of_difference():
    """m = 2: V = max(0, 1 - (o_c - o_k)); the mean of o is free and stays at the mean
    of v, and the difference d = o_c - o_k minimises (d - e)^2/4 + t max(0, 1 - d),
    e = v_c - v_k: the binary hinge prox with step 2t and y = 1."""
    rng = np.random.default_rng(7)
    for _ in range(500):
        t = float(10 ** rng.uniform(-2, 1))
        v = rng.normal(size=2) * 2
        c = int(rng.integers(2))
        k = 1 - c
        y = np.array([-1.0, -1.0])
        y[c] = 1.0
        o = P.prox_loss("crammer_singer", v[None], y[None], t)[0]
        e = v[c] - v[k]
        d = e if e > 1.0 else (e + 2 * t if e < 1.0 - 2 * t else 1.0)
        assert abs((o[c] - o[k]) - d) < 1e-12 * (1 + abs(d))
        assert abs(o.sum() - v.sum()) < 1e-12 * (1 + np.abs(v).sum())


@pytest.mark.parametrize("m", [3, 4])
def test_crammer_singer_brute_force(m):
    """Against a generic constrained minimiser of the epigraph form
    min 1/2 |o - v|^2 + t s  subject to  s >= Delta_k + o_k - o_c for every k."""
    rng = np.random.default_rng(60 + m)
    for _ in range(25):
        v, y, c, t = _cs_problem(rng, m)
        delta = np.ones(m)
        delta[c] = 0.0
        f = lambda z: 0.5 * np.sum((z[:m] - v) ** 2) + t * z[m]
        cons = [{"type": "ineq", "fun": (lambda z, k=k: z[m] - (delta[k] + z[k] - z[c]))} for k in range(m)]
        z0 = np.concatenate([v, [np.max(delta + v - v[c])]])
        res = optimize.minimize(f, z0, method="SLSQP", constraints=cons,
                                options=dict(ftol=1e-15, maxiter=1000))
        got = P.prox_loss("crammer_singer", v[None], y[None], t)[0]
        obj = lambda o: 0.5 * np.sum((o - v) ** 2) + t * float(row_loss_mp("crammer_singer", y, o))
        assert np.max(np.abs(got - res.x[:m])) < 1e-6
        assert obj(got) <= obj(res.x[:m]) + 1e-12
