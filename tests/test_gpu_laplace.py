"""The random Laplace feature map on the GPU against the oracle: its parameters, the map
itself, and whole solves on histogram inputs (FP32 and cached-Z precisions)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import admm, philox, rff as orff  # noqa: E402

PRECS = {"fp32": 1e-5, "cached_z": 1e-4}


@pytest.fixture(scope="module")
def rff():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1409_0940_gb300
    return paper_1409_0940_gb300


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def test_parameters_match_oracle(rff):
    """W = 1/(2 sigma^2 g^2) from the Philox normals: equal to the oracle's float32 values except
    rare one-ulp ties of the float64 libraries (log, cos, sin differ in their last bit)."""
    d, k_lo, k_hi, seed, sigma = 37, 100, 4200, 77, 1.7
    W = torch.zeros((d, k_hi - k_lo), dtype=torch.float32, device="cuda")
    rff.rff_laplace_params(seed, sigma, d, k_lo, k_hi, W)
    got = W.cpu().numpy()
    ref = philox.laplace_params(seed, sigma, d, k_hi, k_lo, k_hi)
    diff = got != ref
    assert diff.mean() <= 1e-4
    if diff.any():
        ulps = np.abs(got.view(np.int32)[diff].astype(np.int64) - ref.view(np.int32)[diff].astype(np.int64))
        assert ulps.max() <= 2


@pytest.mark.parametrize("k_lo,k_hi", [(0, 300), (513, 1100)])
def test_features_match_oracle(rff, k_lo, k_hi):
    X, _ = synth.histograms(n=333, d=40, m=3, seed=6)
    D, seed, sigma = 2000, 5, 3.0
    Z = torch.zeros((X.shape[0], k_hi - k_lo), dtype=torch.float32, device="cuda")
    rff.rff_laplace_features(dev(X), seed, sigma, D, k_lo, k_hi, Z)
    ref = orff.features_block(X.astype(np.float64), seed, sigma, D, k_lo, k_hi, "laplace")
    assert np.abs(Z.cpu().numpy() - ref).max() <= 2e-6 / np.sqrt(D)


def test_negative_inputs_are_refused(rff):
    X, Y = synth.histograms(n=300, d=16, m=2, seed=7)
    Xn = X.copy()
    Xn[5, 3] = -1e-3
    Z = torch.zeros((300, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(rff.RffError):
        rff.rff_laplace_features(dev(Xn), 1, 1.0, 64, 0, 64, Z)
    s = rff.Solver(prec="fp32", loss="squared", reg="l2", lam=1e-3, sigma=2.0, D=128, R=1, C=1, seed=1, m=2,
                   feature_map="laplace")
    with pytest.raises(rff.RffError):
        s.set_data(Xn, Y)
    s.set_data(X, Y)
    s.solve(2, stats=False)
    with pytest.raises(rff.RffError):
        s.predict(Xn[:10])
    s.close()


def test_split_precision_is_refused(rff):
    with pytest.raises(rff.RffError):
        rff.Solver(prec="split_bf16", loss="squared", reg="l2", lam=1e-3, sigma=2.0, D=128, seed=1, m=1,
                   feature_map="laplace")


CASES = [
    # (loss, reg, n, d, m, D, R, C, iters): Gram form with ragged blocks, and the outer form
    ("squared", "l2", 900, 32, 4, 384, 3, 2, 25),
    ("hinge", "l2", 700, 24, 5, 512, 2, 2, 25),
    ("crammer_singer", "l1", 600, 20, 3, 2048, 2, 2, 20),
]


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("case", CASES, ids=lambda c: "%s-%dx%d-D%d" % (c[0], c[6], c[7], c[5]))
def test_solver_matches_oracle(rff, prec, case):
    loss, reg, n, d, m, D, R, C, iters = case
    if prec == "cached_z" and D // C > n // R:
        pytest.skip("the cached-Z precision takes the Gram form only")
    X, Y = synth.histograms(n=n, d=d, m=m, seed=n + d)
    sigma, lam = 4.0, 1e-3
    prob = admm.Problem(X, Y, loss, reg, lam, sigma, 1.0, D, R, C, seed=23, feature_map="laplace")
    out = admm.admm(prob, iters, history=True)
    s = rff.Solver(prec=prec, loss=loss, reg=reg, lam=lam, sigma=sigma, rho=1.0, D=D, R=R, C=C, seed=23, m=m,
                   feature_map="laplace")
    s.set_data(X, Y)
    st = s.solve(iters)
    W = s.weights()
    tol = PRECS[prec]
    assert rel(W, out["Wbar"]) < tol, rel(W, out["Wbar"])
    f_ref = prob.objective(out["Wbar"])
    assert abs(st["objective"] - f_ref) < tol * abs(f_ref)
    Xq, _ = synth.histograms(n=257, d=d, m=m, seed=99)
    got = s.predict(Xq)
    ref = prob.predict(Xq, out["Wbar"])
    assert np.abs(got - ref).max() < 10 * tol * np.abs(ref).max()
    s.close()
