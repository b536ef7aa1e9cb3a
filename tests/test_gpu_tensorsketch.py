"""TensorSketch features (Sec. 4 lists the map; Pham and Pagh 2013) on the GPU against the
oracle: the sketches themselves, whole cached-Z solves, scoring, determinism, refusals."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import admm, rff as orff, tensorsketch as ots  # noqa: E402


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


@pytest.mark.parametrize("q,D,C,d", [(1, 300, 2, 13), (2, 1000, 3, 20), (3, 640, 1, 7), (2, 256, 4, 64)])
def test_features_match_oracle(rff, q, D, C, d):
    """Every block's sketch (ragged block sizes, one to four blocks, degrees 1 to 3) equals the
    oracle's FFT form within FP32 rounding of its sums."""
    rng = np.random.default_rng(q * 100 + d)
    X = rng.standard_normal((257, d)).astype(np.float32)
    seed, sigma, c = 9 + q, 1.7, 0.5
    Z = torch.zeros((X.shape[0], D), dtype=torch.float32, device="cuda")
    rff.rff_tensorsketch_features(dev(X), seed, sigma, c, q, D, C, Z)
    ref = ots.features(X.astype(np.float64), seed, sigma, c, q, orff.partition(D, C))
    got = Z.cpu().numpy()
    assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max(), np.abs(got - ref).max() / np.abs(ref).max()


def test_sparse_rows_and_zero_rows(rff):
    """Rows with many zeros skip them (the same sums), and a zero row sketches (0.., sqrt(c))."""
    X, _ = synth.sparse01(n=200, d=50, m=2, seed=4)
    X[7] = 0.0
    Z = torch.zeros((200, 512), dtype=torch.float32, device="cuda")
    rff.rff_tensorsketch_features(dev(X), 3, 1.0, 2.0, 2, 512, 2, Z)
    ref = ots.features(X.astype(np.float64), 3, 1.0, 2.0, 2, orff.partition(512, 2))
    got = Z.cpu().numpy()
    assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max()
    assert np.abs(got[7] - ref[7]).max() <= 1e-6 * np.abs(ref[7]).max()


def test_refusals(rff):
    X = torch.zeros((4, 3), dtype=torch.float32, device="cuda")
    Z = torch.zeros((4, 64), dtype=torch.float32, device="cuda")
    for bad in (dict(degree=0), dict(degree=9), dict(coef0=-1.0)):
        kw = dict(seed=1, sigma=1.0, coef0=1.0, degree=2, D=64, C=1)
        kw.update(bad)
        with pytest.raises(rff.RffError):
            rff.rff_tensorsketch_features(X, kw["seed"], kw["sigma"], kw["coef0"], kw["degree"], kw["D"], kw["C"], Z)
    for prec in ("fp32", "split_bf16"):
        with pytest.raises(rff.RffError):
            rff.Solver(prec=prec, feature_map="tensorsketch", D=128, m=1)
    with pytest.raises(rff.RffError):
        rff.Solver(prec="cached_z", feature_map="tensorsketch", D=20000, C=2, m=1)


CASES = [
    # (loss, reg, n, d, m, D, R, C, degree, coef0, iters)
    ("squared", "l2", 1200, 16, 2, 512, 2, 2, 2, 1.0, 25),
    ("hinge", "l2", 1500, 24, 1, 384, 3, 1, 3, 0.5, 25),
    ("multinomial", "l1", 1000, 12, 3, 768, 2, 3, 2, 2.0, 20),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%s-q%d-%dx%d" % (c[0], c[8], c[6], c[7]))
def test_solver_matches_oracle(rff, case):
    loss, reg, n, d, m, D, R, C, q, c, iters = case
    if loss == "squared":
        X, y = synth.ridge(n=n, d=d, seed=n)
        Y = np.ascontiguousarray(np.repeat(y, m, axis=1))
    elif m == 1:
        X, Y = synth.binary(n=n, d=d, seed=n)
    else:
        X, Y = synth.multiclass(n=n, d=d, m=m, seed=n)
    sigma, lam = 4.0, 1e-3
    prob = admm.Problem(X, Y, loss, reg, lam, sigma, 1.0, D, R, C, seed=31, feature_map="tensorsketch", degree=q,
                        coef0=c)
    out = admm.admm(prob, iters, history=True)
    kw = dict(prec="cached_z", loss=loss, reg=reg, lam=lam, sigma=sigma, rho=1.0, D=D, R=R, C=C, seed=31, m=m,
              feature_map="tensorsketch", degree=q, coef0=c)
    s = rff.Solver(**kw)
    s.set_data(X, Y)
    st = s.solve(iters)
    W = s.weights()
    assert rel(W, out["Wbar"]) < 1e-4, rel(W, out["Wbar"])
    f_ref = prob.objective(out["Wbar"])
    assert abs(st["objective"] - f_ref) < 1e-4 * abs(f_ref)
    Xq = np.random.default_rng(5).standard_normal((2500, d)).astype(np.float32)   # two scoring chunks
    got = s.predict(Xq)
    ref = prob.predict(Xq, out["Wbar"])
    assert np.abs(got - ref).max() < 1e-3 * np.abs(ref).max()
    # bit-reproducible: the same solve again
    s2 = rff.Solver(**kw)
    s2.set_data(X, Y)
    s2.solve(iters, stats=False)
    assert np.array_equal(s2.weights(), W)
    s.close()
    s2.close()


def test_largest_block_and_degree(rff):
    """The largest column block (8192 features) at degree 4, and degree 8 on a small block:
    the shared-memory layouts at their limits, still equal to the oracle."""
    rng = np.random.default_rng(11)
    for q, D, C, d in ((4, 8192, 1, 300), (8, 96, 1, 5)):
        X = (rng.standard_normal((64, d)) * 0.3).astype(np.float32)
        Z = torch.zeros((64, D), dtype=torch.float32, device="cuda")
        rff.rff_tensorsketch_features(dev(X), 2, 3.0, 0.7, q, D, C, Z)
        ref = ots.features(X.astype(np.float64), 2, 3.0, 0.7, q, orff.partition(D, C))
        got = Z.cpu().numpy()
        assert np.abs(got - ref).max() <= 5e-5 * np.abs(ref).max(), (q, np.abs(got - ref).max() / np.abs(ref).max())


def test_shared_memory_limit_is_refused(rff):
    """Degree x (d + 1) hash tables plus a block of 8192 features beyond the kernel's shared
    memory: refused before any launch, by the step call and by set_data."""
    X = torch.zeros((4, 5000), dtype=torch.float32, device="cuda")
    Z = torch.zeros((4, 8192), dtype=torch.float32, device="cuda")
    with pytest.raises(rff.RffError):
        rff.rff_tensorsketch_features(X, 1, 1.0, 1.0, 8, 8192, 1, Z)
    s = rff.Solver(prec="cached_z", feature_map="tensorsketch", degree=8, D=8192, C=1, m=1, loss="squared")
    with pytest.raises(rff.RffError):
        s.set_data(np.zeros((300, 5000), np.float32), np.zeros((300, 1), np.float32))
    s.close()


def test_full_size_sampled_rows(rff):
    """At the benchmark's size (200,000 x 440 rows, D = 16384 in 4 blocks: Z has 3.3e9 entries,
    past 32-bit indexing), sampled rows of the device sketches equal the oracle's."""
    n, d, D, C = 200_000, 440, 16384, 4
    X = np.random.default_rng(8).standard_normal((n, d)).astype(np.float32)
    Z = torch.empty((n, D), dtype=torch.float32, device="cuda")
    rff.rff_tensorsketch_features(dev(X), 17, 10.0, 1.0, 2, D, C, Z)
    rows = np.array([0, 1, 4097, 65535, 131071, 131072, 150000, 199998, 199999])
    got = Z[torch.from_numpy(rows).cuda()].cpu().numpy()
    del Z
    ref = ots.features(X[rows].astype(np.float64), 17, 10.0, 1.0, 2, orff.partition(D, C))
    assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max()
