"""Pins for the oracle's Fastfood map (Sec. 4 lists it; Le, Sarlos and Smola 2013): its rows
follow the Gaussian kernel's spectral law, the dense block equals the product of its
factors applied by fast transforms, and its features estimate the Gaussian kernel."""
import numpy as np
import pytest
from scipy import stats

import synth
from oracle import admm, fastfood, rff


def fwht(y):
    """Unnormalised Walsh-Hadamard transform along the last axis (Sylvester order)."""
    y = np.array(y, dtype=np.float64)
    n = y.shape[-1]
    h = 1
    while h < n:
        y = y.reshape(*y.shape[:-1], n // (2 * h), 2, h)
        a, b = y[..., 0, :].copy(), y[..., 1, :].copy()
        y[..., 0, :], y[..., 1, :] = a + b, a - b
        y = y.reshape(*y.shape[:-3], n)
        h *= 2
    return y


def test_block_is_the_product_applied_by_transforms():
    """V x = (1/(sigma sqrt d')) S H g * (P (H (B x))) evaluated right to left, with
    (P y)[m] = y[pi(m)]."""
    seed, sigma, dp = 4, 1.3, 64
    rng = np.random.default_rng(0)
    x = rng.standard_normal((5, dp))
    for beta in (0, 3):
        V = fastfood.block_matrix(seed, sigma, dp, beta)
        B, g, perm = fastfood.block_params(seed, dp, beta)
        s = fastfood.chi_scales(seed, dp, beta * dp + np.arange(dp))
        y = fwht(x * B)[:, perm] * g
        y = fwht(y) * (s / np.linalg.norm(g)) / (sigma * np.sqrt(dp))
        assert np.abs(x @ V.T - y).max() < 1e-12 * np.abs(y).max()


def test_parameters_are_signs_and_permutations():
    for beta in range(5):
        B, g, perm = fastfood.block_params(9, 128, beta)
        assert set(np.unique(B)) <= {-1.0, 1.0} and abs(B.mean()) < 0.5
        assert np.array_equal(np.sort(perm), np.arange(128))
        assert not np.array_equal(perm, np.arange(128))


def test_rows_follow_the_gaussian_spectral_law():
    """One row per block (blocks are independent): projections on a fixed unit vector are
    N(0, 1/sigma^2) and row lengths are chi(d') / sigma."""
    seed, sigma, d = 12, 0.8, 16
    nblk = 3000
    G, _ = fastfood.fastfood_params(seed, sigma, d, nblk * 16, 0, nblk * 16)
    rows = G.T.astype(np.float64)[::16]
    u = np.random.default_rng(1).standard_normal(d)
    u /= np.linalg.norm(u)
    assert stats.kstest(rows @ u * sigma, "norm").pvalue > 1e-3
    assert stats.kstest(np.linalg.norm(rows, axis=1) * sigma, stats.chi(16).cdf).pvalue > 1e-3


def test_features_estimate_the_gaussian_kernel():
    """Mean kernel error well inside the Monte Carlo scale and falling like D^-1/2."""
    rng = np.random.default_rng(10)
    X = rng.random((40, 7))
    K = rff.gaussian_kernel(X, X, 0.7)
    errs = []
    Ds = [256, 1024, 4096]
    for D in Ds:
        e = []
        for seed in range(3):
            Z = rff.features_block(X, 50 + seed, 0.7, D, 0, D, "fastfood")
            e.append(np.abs(Z @ Z.T - K).mean())
        errs.append(np.mean(e))
    slope = np.polyfit(np.log(Ds), np.log(errs), 1)[0]
    assert -0.75 < slope < -0.3
    assert errs[-1] < 2.0 / np.sqrt(Ds[-1])


def test_block_map_independent_of_C():
    rng = np.random.default_rng(11)
    X = rng.random((20, 9))
    D = 200
    Z1 = rff.features_block(X, 3, 1.5, D, 0, D, "fastfood")
    cols = rff.partition(D, 16)
    Z16 = np.concatenate([rff.features_block(X, 3, 1.5, D, cols[j], cols[j + 1], "fastfood")
                          for j in range(16)], axis=1)
    assert np.array_equal(Z1, Z16)


def test_ridge_closed_form_with_fastfood_features():
    X, Y = synth.ridge(n=300, d=5, seed=4)
    p = admm.Problem(X, Y, "squared", "l2", lam=1e-3, sigma=2.0, rho=1.0, D=96, R=1, C=1, seed=7,
                     feature_map="fastfood")
    W = admm.ridge_closed_form(p.Z(), p.Y, p.lam)
    out = admm.admm(p, 300)
    assert np.linalg.norm(out["Wbar"] - W) / np.linalg.norm(W) < 1e-9
