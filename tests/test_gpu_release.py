"""Feature parameters given back and drawn again on demand (Sec. 4: omega kept implicit as
the generator's state): scores and iterates are bit-identical to a model that kept them."""
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


@pytest.mark.parametrize("prec,fmap", [("split_bf16", "fourier"), ("fp32", "fourier"), ("cached_z", "fourier"),
                                       ("split_bf16", "fastfood"), ("fp32", "laplace")])
def test_release_and_regenerate_are_invisible(rff, prec, fmap):
    if fmap == "laplace":
        X, Y = synth.histograms(n=700, d=24, m=3, seed=3)
    else:
        X, Y = synth.multiclass(n=700, d=24, m=3, seed=3)
    kw = dict(prec=prec, loss="hinge", reg="l2", lam=1e-3, sigma=3.0, D=384, R=2, C=2, seed=9, m=3,
              feature_map=fmap)
    Xq = np.abs(np.random.default_rng(4).standard_normal((300, 24))).astype(np.float32)
    a, b = rff.Solver(**kw), rff.Solver(**kw)
    for s in (a, b):
        s.set_data(X, Y)
        s.solve(6, stats=False)
    freed = b.release_features()
    assert freed >= 384 * 64 * (4 if prec == "fp32" else 4)
    assert b.release_features() == 0                      # nothing left to give back
    assert np.array_equal(b.predict(Xq), a.predict(Xq))  # drawn for the call, given back again
    assert np.array_equal(b.predict(Xq), a.predict(Xq))
    if prec == "split_bf16":
        out = torch.zeros((300, 3), dtype=torch.float32, device="cuda")
        with pytest.raises(rff.RffError):
            rff.rff_admm_predict_noalloc(b.h, torch.from_numpy(Xq).cuda(), out)
    sa, sb = a.solve(5), b.solve(5)                      # resident again for the iterations
    assert np.array_equal(b.weights(), a.weights())
    assert sa["objective"] == sb["objective"]
    a.close()
    b.close()


def test_release_needs_a_solve(rff):
    s = rff.Solver(prec="fp32", loss="squared", reg="l2", lam=1e-3, sigma=2.0, D=64, seed=1, m=1)
    X, Y = synth.ridge(n=100, d=4, seed=1)
    s.set_data(X, Y)
    with pytest.raises(rff.RffError):
        s.release_features()
    s.close()
