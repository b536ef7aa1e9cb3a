"""Model-selection sweep: lambda columns sharing one factor, solves run side by side."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import admm  # noqa: E402

TOL = {"fp32": 1e-5, "split_bf16": 1e-4, "cached_z": 1e-4}


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


@pytest.mark.parametrize("prec", list(TOL))
@pytest.mark.parametrize("loss,reg", [("logistic", "l2"), ("squared", "l1"), ("hinge", "l2")])
def test_lambda_columns_equal_separate_solves(rff, prec, loss, reg):
    """Each output column with its own lambda is the solve of that lambda alone (same Z, same factor)."""
    n, d, D, iters = 700, 9, 256, 20
    if loss == "squared":
        X, y = synth.ridge(n=n, d=d, seed=5)
    else:
        X, y = synth.binary(n=n, d=d, seed=5)
    lams = [3e-2, 1e-3, 1e-4, 1e-5]
    m = len(lams)
    Y = np.ascontiguousarray(np.repeat(y, m, axis=1))
    s = rff.Solver(prec=prec, loss=loss, reg=reg, lam=lams[0], sigma=2.0, rho=1.0, D=D, R=2, C=2, seed=3, m=m)
    s.set_lambdas(lams)
    s.set_data(X, Y)
    st = s.solve(iters)
    W = s.weights()
    f_total = 0.0
    for c, lam in enumerate(lams):
        p = admm.Problem(X, y, loss, reg, lam, 2.0, 1.0, D, 2, 2, seed=3)
        Wc = admm.admm(p, iters)["Wbar"]
        assert rel(W[:, c:c + 1], Wc) < TOL[prec], (c, rel(W[:, c:c + 1], Wc))
        f_total += p.objective(Wc)
    # the reported objective is the sum of the columns' objectives
    assert abs(st["objective"] - f_total) < TOL[prec] * abs(f_total)
    s.close()


def test_sweep_run_equals_individual_solves(rff):
    """rff_sweep_run overlaps solves on their own streams; each result equals the solve run alone."""
    groups = [(600, 2.0, 256, 2, 2), (900, 8.0, 384, 1, 3), (450, 0.5, 128, 3, 1)]
    kw = dict(loss="logistic", reg="l2", lam=1e-3, rho=1.0, m=3)
    lams = [1e-2, 1e-3, 1e-4]
    alone, mixed = [], []
    for k, (n, sigma, D, R, C) in enumerate(groups):
        X, y = synth.binary(n=n, d=12, seed=k)
        Y = np.ascontiguousarray(np.repeat(y, 3, axis=1))
        for bucket in (alone, mixed):
            s = rff.Solver(prec="split_bf16" if k % 2 == 0 else "fp32", sigma=sigma, D=D, R=R, C=C, seed=k, **kw)
            s.set_lambdas(lams)
            s.set_data(X, Y)
            bucket.append(s)
    for s in alone:
        s.solve(15, stats=False)
    rff.rff_sweep_run([s.h for s in mixed], 15)
    for a, b in zip(alone, mixed):
        assert np.array_equal(a.weights(), b.weights())
        a.close()
        b.close()


def test_enqueue_then_wait_equals_solve(rff):
    X, Y = synth.multiclass(n=500, d=7, m=3, seed=9)
    kw = dict(loss="hinge", reg="l2", lam=1e-3, sigma=2.0, D=200, R=2, C=2, seed=2, m=3, prec="split_bf16")
    a = rff.Solver(**kw)
    a.set_data(X, Y)
    a.solve(9, stats=False)
    b = rff.Solver(**kw)
    b.set_data(X, Y)
    b.enqueue(4)
    b.enqueue(5)
    b.wait()
    assert np.array_equal(a.weights(), b.weights())
    a.close()
    b.close()


def test_autotuner_choice_is_reported(rff):
    X, Y = synth.multiclass(n=2000, d=30, m=4, seed=1)
    s = rff.Solver(prec="split_bf16", loss="squared", lam=1e-3, sigma=4.0, D=1024, R=2, C=2, seed=1, m=4)
    s.set_data(X, Y)
    s.solve(1, stats=False)
    p = s.profile()
    assert p["tc_kchunk"] in (32, 64) and p["nsplit"] >= 1
    s.close()


@pytest.mark.parametrize("shape", [dict(n=1500, D=640, R=2, C=2), dict(n=1111, D=900, R=3, C=2),
                                   dict(n=700, D=384, R=1, C=3), dict(n=600, D=1024, R=5, C=2)])
def test_every_tile_geometry_gives_identical_results(rff, monkeypatch, shape):
    """The twelve geometries of the regeneration kernels (ring K chunk 64 or 32; Z tile in shared
    or tensor memory, the latter with one or two X.G accumulators; one CTA or a CTA pair per
    MMA; X.G products 128 or 256 wide) issue the same products in the same order
    for every output element: weights and scores agree bitwise.  The shapes give row blocks and
    column blocks with an odd number of 128-slot tiles (a CTA pair then computes and discards a
    tile past the block), an odd number of query tiles, and blocks of fewer rows than features
    (the outer form, whose set-up materialises Z through the same kernel)."""
    X, Y = synth.multiclass(n=shape["n"], d=30, m=5, seed=2)
    kw = dict(prec="split_bf16", loss="hinge", reg="l2", lam=1e-3, sigma=3.0, D=shape["D"], R=shape["R"],
              C=shape["C"], seed=3, m=5)
    out = []
    for g in ("64,0", "64,1", "32,0", "32,1", "64,1,2", "32,1,2", "64,2", "32,2", "64,2,2", "32,2,2", "64,3",
              "32,3"):
        monkeypatch.setenv("RFF_TC_GEOMETRY", g)
        s = rff.Solver(**kw)
        s.set_data(X, Y)
        s.solve(8, stats=False)
        p = s.profile()
        f = [int(x) for x in g.split(",")] + [1]
        assert (p["tc_kchunk"], p["tc_z_tmem"], p["tc_cta_pair"] + 1) == (f[0], f[1], f[2])
        out.append((s.weights(), s.predict(X[:200]), s.predict(X[:333])))
        s.close()
    for W, P, P2 in out[1:]:
        assert np.array_equal(W, out[0][0])
        assert np.array_equal(P, out[0][1])
        assert np.array_equal(P2, out[0][2])


def test_sweep_graph_continues_and_keeps_masks(rff):
    """Repeated sweep calls replay one graph for all solves (no eager iteration after the
    first); a stochastic solve in the mix keeps drawing the masks of its own iterations."""
    X, y = synth.binary(n=700, d=10, seed=5)
    Y = np.ascontiguousarray(np.repeat(y, 2, axis=1))
    specs = [dict(prec="split_bf16", sigma=2.0, D=256, R=2, C=2, seed=1, frac=None),
             dict(prec="split_bf16", sigma=4.0, D=384, R=1, C=3, seed=2, frac=0.5),
             dict(prec="fp32", sigma=1.0, D=128, R=2, C=1, seed=3, frac=None)]
    alone, mixed = [], []
    for sp in specs:
        for bucket in (alone, mixed):
            s = rff.Solver(prec=sp["prec"], loss="logistic", reg="l2", lam=1e-3, rho=1.0, sigma=sp["sigma"],
                           D=sp["D"], R=sp["R"], C=sp["C"], seed=sp["seed"], m=2)
            if sp["frac"]:
                s.set_block_fraction(sp["frac"])
            s.set_data(X, Y)
            bucket.append(s)
    for s in alone:
        s.solve(6, stats=False)
        s.solve(7, stats=False)
    rff.rff_sweep_run([s.h for s in mixed], 6)
    rff.rff_sweep_run([s.h for s in mixed], 7)
    for a, b in zip(alone, mixed):
        assert np.array_equal(a.weights(), b.weights())
        a.close()
        b.close()
