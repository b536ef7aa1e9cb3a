"""Pins for the oracle's loss and regulariser values (oracle/prox.py loss_value, reg_value)
and for the objective they compose (oracle/admm.py Problem.objective).

Four kinds of evidence, none of which calls the function under test to make its own
expected value:
* every loss and regulariser written entry by entry from its definition in 40-digit
  mpmath (tests/loss_definitions.py) and compared on random inputs, ties in the targets and large outputs included;
* values fixed by the mathematics: special points (log 2, log m, margins of exactly one),
  reductions of the multiclass losses to binary ones at m = 2, shift invariance, the
  asymptotes of the logistic loss;
* the Moreau-envelope identity that ties each value to its proximal operator (Sec. 2.3):
  with p = prox_{tV}(v), the envelope e(v) = V(p) + |p - v|^2 / (2t) is differentiable
  with gradient (v - p)/t; the proxes are pinned by brute force elsewhere, so a wrong
  term in a value breaks the identity;
* the objective's minimiser: the converged ADMM iterate (whose steps use only the pinned
  proxes) must not be beaten by any nearby point of objective(), so a wrong weight of the
  regulariser or a wrong loss term shows up.
"""
import numpy as np
import pytest

import synth
from oracle import admm
from oracle import prox as P

pytest.importorskip("mpmath")
from loss_definitions import loss_mp as _loss_mp, reg_mp as _reg_mp  # noqa: E402


def _targets(rng, loss, n, m, ties=False):
    if loss in ("squared", "l1"):
        return rng.normal(size=(n, m))
    if loss in ("hinge", "logistic"):
        return np.where(rng.random((n, m)) < 0.5, -1.0, 1.0)
    Y = -np.ones((n, m))
    Y[np.arange(n), rng.integers(0, m, n)] = 1.0
    if ties:
        # rows with several equal maxima: the first one is the class
        Y[: n // 2] = 1.0
    return Y


ALL = ["squared", "hinge", "logistic", "multinomial", "l1", "crammer_singer"]


def _m_of(loss, m):
    return 1 if loss == "logistic" else m


@pytest.mark.parametrize("loss", ALL)
def test_loss_value_matches_definition(loss):
    rng = np.random.default_rng(11)
    for m in (1, 2, 3, 7):
        if loss in ("multinomial", "crammer_singer") and m == 1:
            continue
        mm = _m_of(loss, m)
        for scale in (0.1, 1.0, 30.0):
            for ties in (False, True):
                Y = _targets(rng, loss, 6, mm, ties)
                O = rng.normal(size=(6, mm)) * scale
                got = P.loss_value(loss, Y, O)
                ref = _loss_mp(loss, Y, O)
                assert abs(got - float(ref)) <= 1e-13 * max(1.0, float(abs(ref))), (loss, m, scale, ties)


@pytest.mark.parametrize("reg", ["l2", "l1"])
def test_reg_value_matches_definition(reg):
    rng = np.random.default_rng(12)
    for shape in ((1, 1), (5, 3), (40, 7)):
        W = rng.normal(size=shape) * rng.choice([1e-3, 1.0, 1e3])
        got = P.reg_value(reg, W)
        ref = float(_reg_mp(reg, W))
        assert abs(got - ref) <= 1e-14 * max(1.0, abs(ref))


def test_special_values():
    # logistic at a zero output is log 2, whatever the label
    assert P.loss_value("logistic", [[1.0], [-1.0]], [[0.0], [0.0]]) == pytest.approx(2 * np.log(2), rel=1e-15)
    # multinomial with all outputs equal: log m (the class does not matter)
    for m in (2, 5, 147):
        Y = -np.ones((1, m))
        Y[0, m // 3] = 1.0
        assert P.loss_value("multinomial", Y, np.full((1, m), 3.25)) == pytest.approx(np.log(m), rel=1e-14)
    # hinge: zero at a margin of exactly one, one at a zero output, linear below
    assert P.loss_value("hinge", [[1.0, -1.0]], [[1.0, -1.0]]) == 0.0
    assert P.loss_value("hinge", [[1.0, -1.0]], [[0.0, 0.0]]) == 2.0
    assert P.loss_value("hinge", [[1.0]], [[-2.5]]) == 3.5
    # Crammer-Singer: all outputs equal gives the margin 1; a winning margin of one gives 0
    assert P.loss_value("crammer_singer", [[-1.0, 1.0, -1.0]], [[0.3, 0.3, 0.3]]) == 1.0
    assert P.loss_value("crammer_singer", [[-1.0, 1.0, -1.0]], [[0.0, 1.0, -4.0]]) == 0.0
    # squared and l1 on a known residual (3, -4): 25 and 7
    assert P.loss_value("squared", [[1.0, 2.0]], [[-2.0, 6.0]]) == 25.0
    assert P.loss_value("l1", [[1.0, 2.0]], [[-2.0, 6.0]]) == 7.0
    assert P.reg_value("l2", [[3.0, -4.0]]) == 25.0
    assert P.reg_value("l1", [[3.0, -4.0]]) == 7.0


def test_two_class_reductions():
    """At m = 2 the multinomial loss is the binary logistic loss of the margin o_c - o_k and
    the Crammer-Singer loss the binary hinge of that margin (each branch checked against
    another one, through an identity of the mathematics)."""
    rng = np.random.default_rng(13)
    for _ in range(200):
        o = rng.normal(size=2) * rng.choice([0.5, 5.0, 50.0])
        c = int(rng.integers(2))
        y = -np.ones(2)
        y[c] = 1.0
        margin = o[c] - o[1 - c]
        mult = P.loss_value("multinomial", y[None], o[None])
        logi = P.loss_value("logistic", [[1.0]], [[margin]])
        assert abs(mult - logi) <= 1e-12 * max(1.0, abs(logi))
        cs = P.loss_value("crammer_singer", y[None], o[None])
        hin = P.loss_value("hinge", [[1.0]], [[margin]])
        assert abs(cs - hin) <= 1e-12 * max(1.0, abs(hin))


def test_shift_invariance_and_logistic_asymptotes():
    rng = np.random.default_rng(14)
    for _ in range(50):
        m = int(rng.integers(2, 9))
        O = rng.normal(size=(3, m))
        Y = _targets(rng, "multinomial", 3, m)
        s = float(rng.normal() * 10)
        for loss in ("multinomial", "crammer_singer"):
            a, b = P.loss_value(loss, Y, O), P.loss_value(loss, Y, O + s)
            assert abs(a - b) <= 1e-12 * max(1.0, abs(a))
    # log(1 + e^-u): -u + e^u for u -> -inf, e^-u for u -> +inf (no overflow either way)
    for u in (-800.0, -60.0):
        assert P.loss_value("logistic", [[1.0]], [[u]]) == pytest.approx(-u, rel=1e-15)
    for u in (40.0, 700.0):
        assert P.loss_value("logistic", [[1.0]], [[u]]) == pytest.approx(np.exp(-u), rel=1e-12)


@pytest.mark.parametrize("loss", ALL)
def test_moreau_envelope_gradient(loss):
    """e(v) = V(p(v)) + |p(v) - v|^2 / (2t), p = prox_{tV}: grad e = (v - p)/t, checked by
    central differences of e built from loss_value and prox_loss."""
    rng = np.random.default_rng(15)
    m = 1 if loss == "logistic" else 4
    h = 1e-6
    for _ in range(20):
        t = float(10 ** rng.uniform(-1, 0.5))
        Y = _targets(rng, loss, 1, m)
        v = rng.normal(size=(1, m)) * 2

        def env(v):
            p = P.prox_loss(loss, v, Y, t)
            return P.loss_value(loss, Y, p) + float(np.sum((p - v) ** 2)) / (2 * t)

        p = P.prox_loss(loss, v, Y, t)
        grad = (v - p) / t
        for k in range(m):
            e = np.zeros((1, m))
            e[0, k] = h
            fd = (env(v + e) - env(v - e)) / (2 * h)
            assert abs(fd - grad[0, k]) < 2e-6 * max(1.0, abs(grad[0, k])), (loss, k, fd, grad[0, k])


@pytest.mark.parametrize("reg", ["l2", "l1"])
def test_moreau_envelope_gradient_reg(reg):
    rng = np.random.default_rng(16)
    h = 1e-6
    for _ in range(50):
        tau = float(10 ** rng.uniform(-2, 0.5))
        v = float(rng.normal() * 2)
        env = lambda v: (P.reg_value(reg, P.prox_reg(reg, np.array([[v]]), tau))
                         + (P.prox_reg(reg, np.array([[v]]), tau)[0, 0] - v) ** 2 / (2 * tau))
        p = P.prox_reg(reg, np.array([[v]]), tau)[0, 0]
        fd = (env(v + h) - env(v - h)) / (2 * h)
        assert abs(fd - (v - p) / tau) < 2e-6 * max(1.0, abs((v - p) / tau))


@pytest.mark.parametrize("loss,reg", [("logistic", "l2"), ("multinomial", "l2"), ("hinge", "l2"),
                                      ("squared", "l1"), ("crammer_singer", "l2"), ("l1", "l2")])
def test_converged_iterate_minimises_objective(loss, reg):
    """objective(W) = sum_i V(y_i, (Z W)_i) + n lambda r(W) (sum-scaled reading of rho):
    the ADMM fixed point reached from the pinned proxes is its minimiser, so no nearby
    point of the objective as the oracle writes it may be lower (beyond the iterate's
    residual).  A factor n dropped from the regulariser or a wrong loss term moves the
    objective's minimiser away from the fixed point and fails this."""
    if loss == "logistic":
        X, Y = synth.binary(n=240, d=5, seed=21)
    else:
        X, Y = synth.multiclass(n=240, d=5, m=3, seed=21)
    p = admm.Problem(X, Y, loss, reg, lam=3e-3, sigma=2.0, rho=1.0, D=32, R=1, C=1, seed=4)
    W = admm.admm(p, 4000)["Wbar"]
    f0 = p.objective(W)
    rng = np.random.default_rng(17)
    worst = 0.0
    for _ in range(60):
        dW = rng.normal(size=W.shape)
        dW *= 1e-3 * np.linalg.norm(W) / np.linalg.norm(dW)
        worst = min(worst, p.objective(W + dW) - f0, p.objective(W - dW) - f0)
    assert worst > -1e-7 * abs(f0), (loss, reg, worst, f0)
    if loss in ("hinge", "crammer_singer", "l1"):
        return
    # smooth losses: the same check finds the fixed point off the minimiser of an objective
    # whose regulariser lacks the factor n (scaling W up moves that objective down)
    wrong = lambda W: P.loss_value(loss, p.Y, p.Z() @ W) + p.lam * P.reg_value(reg, W)
    g0 = wrong(W)
    assert min(wrong((1.0 + s) * W) - g0 for s in (1e-2, -1e-2)) < -1e-7 * abs(g0)
