"""Pins for the random Laplace feature map of the oracle (Sec. 4 lists it among the
solver's maps): its parameters against the Levy law, its inner products against the
exponential semigroup kernel, block independence, and the ridge closed form."""
import numpy as np
import pytest
from scipy import special, stats

import synth
from oracle import admm, philox, rff


def levy_cdf(t, sigma):
    """P(W <= t) for W = c / g^2, g ~ N(0, 1), c = 1 / (2 sigma^2): P(|g| >= sqrt(c / t))."""
    return special.erfc(np.sqrt(1.0 / (2.0 * sigma * sigma) / (2.0 * t)))


@pytest.mark.parametrize("sigma", [0.5, 3.0])
def test_parameters_follow_the_levy_law(sigma):
    W = philox.laplace_params(5, sigma, 12, 20000).ravel().astype(np.float64)
    assert W.min() > 0
    res = stats.kstest(W, lambda t: levy_cdf(t, sigma))
    assert res.pvalue > 1e-3, res


def test_laplace_transform_of_the_parameters():
    """E[exp(-t W)] = exp(-sqrt(t) / sigma); each sample lies in [0, 1] (Hoeffding)."""
    sigma = 0.7
    W = philox.laplace_params(9, sigma, 8, 30000).ravel().astype(np.float64)
    delta = 1e-6
    bound = np.sqrt(np.log(2.0 / delta) / (2.0 * W.size))
    for t in [1e-3, 0.05, 0.5, 3.0]:
        assert abs(np.exp(-t * W).mean() - np.exp(-np.sqrt(t) / sigma)) <= bound


def test_kernel_approximation_hoeffding():
    """E[z(x)^T z(x')] = exp(-sum_r sqrt(x_r + x'_r) / sigma); each of the D products lies
    in [0, 1/D], so |Z Z^T - K| <= sqrt(ln(2/delta) / (2 D)) except with probability delta."""
    X, _ = synth.histograms(n=30, d=16, m=3, seed=2)
    sigma, D = 1.0, 8192
    Z = rff.features_block(X, 13, sigma, D, 0, D, "laplace")
    K = rff.semigroup_kernel(X, X, sigma)
    delta = 1e-6
    assert np.abs(Z @ Z.T - K).max() <= np.sqrt(np.log(2.0 / delta) / (2.0 * D))
    # a kernel with a spread of values, and not the Gaussian kernel's estimate
    assert K.min() < 0.5 * K.max()
    assert np.abs(K - rff.gaussian_kernel(X, X, sigma)).max() > 0.1


def test_block_map_independent_of_C():
    X, _ = synth.histograms(n=20, d=9, m=2, seed=3)
    D = 200
    Z1 = rff.features_block(X, 3, 1.5, D, 0, D, "laplace")
    cols = rff.partition(D, 16)
    Z16 = np.concatenate([rff.features_block(X, 3, 1.5, D, cols[j], cols[j + 1], "laplace")
                          for j in range(16)], axis=1)
    assert np.array_equal(Z1, Z16)


def test_ridge_closed_form_with_laplace_features():
    """The solver never looks inside T: with the Laplace map the iterates reach the same
    closed form (Z^T Z + n lam I)^-1 Z^T Y of Sec. 2.2."""
    X, Y = synth.histograms(n=400, d=12, m=2, seed=4)
    p = admm.Problem(X, Y, "squared", "l2", lam=1e-3, sigma=2.0, rho=1.0, D=256, R=1, C=1, seed=8,
                     feature_map="laplace")
    W = admm.ridge_closed_form(p.Z(), p.Y, p.lam)
    out = admm.admm(p, 300)
    assert np.linalg.norm(out["Wbar"] - W) / np.linalg.norm(W) < 1e-9


def test_negative_inputs_are_refused():
    X, Y = synth.histograms(n=50, d=4, m=2, seed=5)
    X[3, 1] = -0.1
    with pytest.raises(ValueError):
        admm.Problem(X, Y, feature_map="laplace")
