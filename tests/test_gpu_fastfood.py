"""The Fastfood feature map on the GPU against the oracle: the structured projection V and
whole solves on every precision path."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import admm, fastfood  # noqa: E402

PRECS = {"fp32": 1e-5, "split_bf16": 1e-4, "cached_z": 1e-4}


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


@pytest.mark.parametrize("d,k_lo,k_hi", [(13, 0, 700), (440, 300, 1400), (1, 5, 9)])
def test_projection_matches_oracle(rff, d, k_lo, k_hi):
    """V from one Walsh-Hadamard transform per row in float64 on the device; the oracle
    multiplies the factors as matrices.  Equal after rounding to float32 except rare ties
    (the two float64 results differ in their last bits)."""
    seed, sigma = 31, 1.9
    nk = k_hi - k_lo
    Vt = torch.zeros((nk, d), dtype=torch.float32, device="cuda")
    b = torch.zeros(nk, dtype=torch.float32, device="cuda")
    rff.rff_fastfood_params(seed, sigma, d, k_lo, k_hi, Vt, b)
    G, bref = fastfood.fastfood_params(seed, sigma, d, k_hi, k_lo, k_hi)
    got, ref = Vt.cpu().numpy(), np.ascontiguousarray(G.T)
    diff = got != ref
    assert diff.mean() <= 1e-3
    if diff.any():
        ulps = np.abs(got.view(np.int32)[diff].astype(np.int64) - ref.view(np.int32)[diff].astype(np.int64))
        assert ulps.max() <= 2
    assert np.array_equal(b.cpu().numpy(), bref)


CASES = [
    # (loss, reg, n, d, m, D, R, C, iters): Gram form (d' = 16, D not a multiple of d'), a wider
    # input (d' = 64), and the outer form
    ("squared", "l2", 777, 13, 2, 300, 3, 2, 30),
    ("hinge", "l2", 900, 40, 5, 512, 2, 2, 25),
    ("multinomial", "l2", 500, 9, 4, 2048, 2, 2, 15),
]


def _data(loss, n, d, m, seed):
    if loss == "squared":
        X, y = synth.ridge(n=n, d=d, seed=seed)
        return X, np.ascontiguousarray(np.repeat(y, m, axis=1), dtype=np.float32)
    return synth.multiclass(n=n, d=d, m=m, seed=seed)


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("case", CASES, ids=lambda c: "%s-%dx%d-d%d" % (c[0], c[6], c[7], c[3]))
def test_solver_matches_oracle(rff, prec, case):
    loss, reg, n, d, m, D, R, C, iters = case
    if prec == "cached_z" and D // C > n // R:
        pytest.skip("the cached-Z precision takes the Gram form only")
    X, Y = _data(loss, n, d, m, seed=n + d)
    prob = admm.Problem(X, Y, loss, reg, 1e-3, 2.5, 1.0, D, R, C, seed=41, feature_map="fastfood")
    out = admm.admm(prob, iters, history=True)
    s = rff.Solver(prec=prec, loss=loss, reg=reg, lam=1e-3, sigma=2.5, rho=1.0, D=D, R=R, C=C, seed=41, m=m,
                   feature_map="fastfood")
    s.set_data(X, Y)
    st = s.solve(iters)
    W = s.weights()
    tol = PRECS[prec]
    assert rel(W, out["Wbar"]) < tol, rel(W, out["Wbar"])
    f_ref = prob.objective(out["Wbar"])
    assert abs(st["objective"] - f_ref) < tol * abs(f_ref)
    Xq = np.random.default_rng(5).standard_normal((129, d)).astype(np.float32)
    got = s.predict(Xq)
    ref = prob.predict(Xq, out["Wbar"])
    assert np.abs(got - ref).max() < 10 * tol * np.abs(ref).max()
    s.close()


def test_wide_inputs_are_refused(rff):
    s = rff.Solver(prec="fp32", loss="squared", reg="l2", lam=1e-3, sigma=2.0, D=64, seed=1, m=1,
                   feature_map="fastfood")
    X = np.zeros((10, 4097), dtype=np.float32)
    with pytest.raises(rff.RffError):
        s.set_data(X, np.zeros((10, 1), dtype=np.float32))
    s.close()
