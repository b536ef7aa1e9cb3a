"""The losses and regularisers written entry by entry from their definitions in 40-digit
mpmath (Sec. 3 "Modularity" lists the losses; squared and l2 carry no factor 1/2, the
multiclass losses take the class c as the first maximum of the +-1 targets).  Test-only
reference values for the oracle's pins: independent of oracle/prox.py, which they check.
"""
import mpmath
import numpy as np

mp = mpmath.mp
mp.dps = 40


def _first_argmax(y):
    c = 0
    for k in range(1, len(y)):
        if y[k] > y[c]:
            c = k
    return c


def row_loss_mp(loss, y, o):
    """V(y, o) of one row, from the definition of each loss."""
    y = [mp.mpf(float(v)) for v in y]
    o = [mp.mpf(float(v)) for v in o]
    m = len(o)
    if loss == "squared":
        return mp.fsum((y[k] - o[k]) ** 2 for k in range(m))
    if loss == "hinge":
        return mp.fsum(max(mp.mpf(0), 1 - y[k] * o[k]) for k in range(m))
    if loss == "logistic":
        return mp.fsum(mp.log(1 + mp.exp(-y[k] * o[k])) for k in range(m))
    if loss == "l1":
        return mp.fsum(abs(y[k] - o[k]) for k in range(m))
    c = _first_argmax(y)
    if loss == "multinomial":
        return mp.log(mp.fsum(mp.exp(o[k]) for k in range(m))) - o[c]
    if loss == "crammer_singer":
        return max((0 if k == c else 1) + o[k] - o[c] for k in range(m))
    raise ValueError(loss)


def loss_mp(loss, Y, O):
    return mp.fsum(row_loss_mp(loss, Y[i], O[i]) for i in range(len(O)))


def reg_mp(reg, W):
    w = [mp.mpf(float(v)) for v in np.ravel(W)]
    if reg == "l2":
        return mp.fsum(v * v for v in w)
    if reg == "l1":
        return mp.fsum(abs(v) for v in w)
    raise ValueError(reg)
