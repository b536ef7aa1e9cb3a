"""Cached-Z precision: Z materialised once and streamed through the chained products.

The oracle parity of this path runs in test_gpu_solver.py (every grid, loss and
regulariser, 1e-4).  Here: agreement with the implicit split-BF16 path, which
regenerates the same Z every pass; bit-identical resume and repeat runs; memory
accounting and refusal when Z does not fit the budget."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import synth  # noqa: E402


@pytest.fixture(scope="module")
def rff():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1409_0940_gb300
    return paper_1409_0940_gb300


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _slots(total, parts):
    q, r = divmod(total, parts)
    return sum(-(-(q + (i < r)) // 128) * 128 for i in range(parts))


@pytest.mark.parametrize("loss,reg,m,R,C,D", [("squared", "l2", 3, 2, 2, 512), ("hinge", "l1", 5, 3, 2, 300),
                                             ("logistic", "l2", 1, 1, 3, 384)])
def test_cached_equals_implicit_split(rff, loss, reg, m, R, C, D):
    n, d = 1500, 21
    if loss == "squared":
        X, y = synth.ridge(n=n, d=d, seed=4)
        Y = np.ascontiguousarray(np.repeat(y, m, axis=1))
    elif m == 1:
        X, Y = synth.binary(n=n, d=d, seed=4)
    else:
        X, Y = synth.multiclass(n=n, d=d, m=m, seed=4)
    out = {}
    for prec in ("split_bf16", "cached_z"):
        s = rff.Solver(prec=prec, loss=loss, reg=reg, lam=1e-3, sigma=3.0, D=D, R=R, C=C, seed=6, m=m)
        s.set_data(X, Y)
        st = s.solve(25)
        out[prec] = (s.weights(), st["objective"], s.predict(X[:64]))
        s.close()
    (Wa, fa, pa), (Wb, fb, pb) = out["split_bf16"], out["cached_z"]
    # the two differ only in where sqrt(2/D) meets the rounding of Z to hi/lo BF16
    assert rel(Wb, Wa) < 2e-5, rel(Wb, Wa)
    assert abs(fb - fa) < 2e-5 * abs(fa)
    assert rel(pb, pa) < 2e-5


def test_cached_resume_and_repeat_are_bit_identical(rff):
    X, Y = synth.multiclass(n=900, d=10, m=4, seed=3)
    kw = dict(prec="cached_z", loss="hinge", reg="l2", lam=1e-3, sigma=2.0, D=256, R=2, C=2, seed=4, m=4)
    a = rff.Solver(**kw)
    a.set_data(X, Y)
    a.solve(11, stats=False)
    b = rff.Solver(**kw)
    b.set_data(X, Y)
    b.solve(11, stats=False)
    assert np.array_equal(a.weights(), b.weights())
    c = rff.Solver(**kw)
    c.set_data(X, Y)
    c.solve(4, stats=False)
    state = c.get_state()
    c.close()
    e = rff.Solver(**kw)
    e.set_data(X, Y)
    e.set_state(state)
    e.solve(7, stats=False)
    assert np.array_equal(e.weights(), a.weights())
    for s in (a, b, e):
        s.close()


def test_cached_memory_accounting_and_refusal(rff):
    n, d, D, R, C, m = 20000, 50, 4096, 3, 2, 7
    kw = dict(loss="squared", reg="l2", lam=1e-3, sigma=3.0, D=D, R=R, C=C, seed=1, m=m)
    _, peak_split = rff.rff_admm_estimate_bytes(rff.make_params(prec="split_bf16", **kw), n, d)
    res_c, peak_c = rff.rff_admm_estimate_bytes(rff.make_params(prec="cached_z", **kw), n, d)
    zbytes = _slots(n, R) * _slots(D, C) * 8          # Z and Z^T, hi and lo BF16
    assert zbytes <= peak_c - peak_split <= zbytes * 1.1
    X, y = synth.ridge(n=n, d=d, seed=2)
    Y = np.ascontiguousarray(np.repeat(y, m, axis=1))
    s = rff.Solver(prec="cached_z", **kw)
    rff.rff_admm_set_memory_limit(s.h, peak_split)   # enough for the implicit path, not for Z
    with pytest.raises(rff.RffError) as e:
        s.set_data(X, Y)
    assert e.value.status == rff.RFF_ENOMEM
    rff.rff_admm_set_memory_limit(s.h, 0)
    s.set_data(X, Y)
    s.solve(3, stats=False)
    assert np.isfinite(s.weights()).all()
    s.close()
