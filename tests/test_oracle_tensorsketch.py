"""Pins of the oracle's TensorSketch map (Sec. 4 lists it; Pham and Pagh 2013) against the
definition and the mathematics, independent of the FFT code path it uses."""
import itertools

import numpy as np
import pytest

from oracle import rff, tensorsketch as ts


@pytest.mark.parametrize("q,S", [(2, 7), (2, 8), (3, 5), (1, 6)])
def test_fft_form_is_the_countsketch_of_the_tensor_power(q, S):
    """TS(x) equals the CountSketch of x'^(tensor q) under H = sum_p h_p(i_p) mod S and the
    sign prod_p g_p(i_p), accumulated entry by entry over all (d+1)^q index tuples."""
    rng = np.random.default_rng(q * 10 + S)
    X = rng.standard_normal((3, 3))
    sigma, c, seed, j = 1.7, 0.6, 11, 2
    got = ts.sketch_block(X, seed, sigma, c, q, S, j)
    h, g = ts.hashes(seed, j, S, X.shape[1], q)
    Xp = ts.augment(X, sigma, c)
    want = np.zeros((X.shape[0], S))
    for tup in itertools.product(range(X.shape[1] + 1), repeat=q):
        bucket = sum(int(h[p, i]) for p, i in enumerate(tup)) % S
        sign = np.prod([g[p, i] for p, i in enumerate(tup)])
        want[:, bucket] += sign * np.prod([Xp[:, i] for i in tup], axis=0)
    assert np.allclose(got, want, rtol=0, atol=1e-12 * max(1.0, np.abs(want).max()))


def test_sum_of_sketch_is_product_of_signed_sums():
    """The entries of a circular convolution sum to the product of the factors' sums:
    sum_t TS(x)[t] = prod_p sum_i g_p(i) x'_i (exact up to rounding, any d and S)."""
    rng = np.random.default_rng(3)
    X = rng.standard_normal((5, 40))
    sigma, c, q, S, seed, j = 2.0, 1.5, 3, 96, 4, 1
    T = ts.sketch_block(X, seed, sigma, c, q, S, j)
    h, g = ts.hashes(seed, j, S, X.shape[1], q)
    Xp = ts.augment(X, sigma, c)
    want = np.prod([Xp @ g[p] for p in range(q)], axis=0)
    assert np.allclose(T.sum(axis=1), want, rtol=1e-11, atol=1e-11)


def test_kernel_estimate_is_unbiased():
    """Over independent seeds, <z(x), z(y)> averages to (<x, y>/sigma^2 + c)^q: the mean lies
    within five standard errors of the kernel value (a dropped augmentation entry, a wrong
    block scale or a sign error biases it by many)."""
    rng = np.random.default_rng(7)
    X = rng.standard_normal((2, 6)) * 0.7
    sigma, c, q = 1.3, 0.8, 2
    cols = rff.partition(48, 3)
    k = ts.polynomial_kernel(X[:1], X[1:], sigma, c, q)[0, 0]
    kxx = ts.polynomial_kernel(X[:1], X[:1], sigma, c, q)[0, 0]
    est, norms = [], []
    for seed in range(600):
        Z = ts.features(X, seed, sigma, c, q, cols)
        est.append(Z[0] @ Z[1])
        norms.append(Z[0] @ Z[0])
    for vals, target in ((np.array(est), k), (np.array(norms), kxx)):
        se = vals.std(ddof=1) / np.sqrt(len(vals))
        assert abs(vals.mean() - target) < 5 * se, (vals.mean(), target, se)


def test_hashes_uniform_and_signs_balanced():
    """h uniform on {0..S-1} (chi-square, 9 degrees of freedom, far below its 0.1 % point
    27.9), signs +-1 with mean near zero."""
    S, d, q = 10, 999, 4
    h, g = ts.hashes(5, 0, S, d, q)
    counts = np.bincount(h.ravel(), minlength=S)
    assert h.min() >= 0 and h.max() < S
    exp = h.size / S
    assert ((counts - exp) ** 2 / exp).sum() < 27.9
    assert set(np.unique(g)) == {-1.0, 1.0}
    assert abs(g.mean()) < 4 / np.sqrt(g.size)


def test_blocks_are_independent_and_scaled():
    """With one column block the map is sqrt(1) TS_0; with several, block j is
    sqrt(s_j / D) TS_j with its own hashes (blocks 0 and 1 of the same size differ)."""
    rng = np.random.default_rng(1)
    X = rng.standard_normal((4, 5))
    Z1 = ts.features(X, 3, 1.0, 1.0, 2, rff.partition(32, 1))
    assert np.allclose(Z1, ts.sketch_block(X, 3, 1.0, 1.0, 2, 32, 0), rtol=0, atol=1e-14)
    Z2 = ts.features(X, 3, 1.0, 1.0, 2, rff.partition(32, 2))
    assert np.allclose(Z2[:, :16], np.sqrt(0.5) * ts.sketch_block(X, 3, 1.0, 1.0, 2, 16, 0), atol=1e-14)
    assert not np.allclose(Z2[:, :16], Z2[:, 16:])


def test_admm_with_sketches_reaches_ridge_closed_form():
    """The solver over TensorSketch features (Z assembled from per-block sketches) converges to
    the ridge minimiser (Z^T Z + n lam I)^-1 Z^T Y of that Z (Sec. 2.2); the sketches' larger
    scale slows the linear rate at rho = 1, so 6000 iterations reach 1e-6."""
    import synth
    from oracle import admm
    X, Y = synth.ridge(n=300, d=5, seed=4)
    p = admm.Problem(X, Y, "squared", "l2", lam=1e-3, sigma=2.0, rho=1.0, D=96, R=2, C=3, seed=7,
                     feature_map="tensorsketch", degree=2, coef0=1.0)
    out = admm.admm(p, 6000)
    W = admm.ridge_closed_form(p.Z(), p.Y, p.lam)
    assert np.linalg.norm(out["Wbar"] - W) / np.linalg.norm(W) < 1e-6


def test_sketch_ridge_tends_to_polynomial_kernel_ridge():
    """With the exact polynomial kernel the ridge minimiser predicts f = K(Xq, X) (K + n lam I)^-1 Y
    (eq. (krr)); the sketched ridge's predictions approach it as D grows (d = 30: the tensor
    square has 961 entries, so the sketches keep colliding over this range of D)."""
    rng = np.random.default_rng(5)
    X = rng.standard_normal((60, 30)) / np.sqrt(30)
    Y = np.tanh(X[:, :1] * X[:, 1:2])
    Xq = rng.standard_normal((30, 30)) / np.sqrt(30)
    sigma, c, q, lam, n = 1.0, 1.0, 2, 1e-3, 60
    K = ts.polynomial_kernel(X, X, sigma, c, q)
    f = ts.polynomial_kernel(Xq, X, sigma, c, q) @ np.linalg.solve(K + n * lam * np.eye(n), Y)
    errs = []
    Ds = [64, 256, 1024, 4096]
    for D in Ds:
        e = []
        for seed in range(3):
            cols = rff.partition(D, 2)
            Z = ts.features(X, 60 + seed, sigma, c, q, cols)
            W = Z.T @ np.linalg.solve(Z @ Z.T + n * lam * np.eye(n), Y)
            e.append(np.abs(ts.features(Xq, 60 + seed, sigma, c, q, cols) @ W - f).mean())
        errs.append(np.mean(e))
    slope = np.polyfit(np.log(Ds), np.log(errs), 1)[0]
    assert errs[-1] < 0.25 * errs[0], errs
    assert -0.8 < slope < -0.25, (slope, errs)
