"""Pins for the oracle's block-splitting ADMM, graph projection and RFF maps."""
import numpy as np
import pytest

import synth
from oracle import admm, memory, philox, rff


@pytest.fixture(scope="module")
def ridge_problem():
    X, Y = synth.ridge(seed=1)
    return X, Y


def test_partition():
    assert list(rff.partition(10, 3)) == [0, 4, 7, 10]
    assert list(rff.partition(8, 4)) == [0, 2, 4, 6, 8]
    assert list(rff.partition(2, 4)) == [0, 1, 2, 2, 2]


def test_ridge_closed_form_1x1(ridge_problem):
    """Ridge of Sec. 2.2 at the smallest workload: n=2000, d=16, D=512, sigma=4, lam=1e-4, rho=1."""
    X, Y = ridge_problem
    p = admm.Problem(X, Y, "squared", "l2", lam=1e-4, sigma=4.0, rho=1.0, D=512, R=1, C=1, seed=2)
    out = admm.admm(p, 200)
    W = admm.ridge_closed_form(p.Z(), p.Y, p.lam)
    assert np.linalg.norm(out["Wbar"] - W) / np.linalg.norm(W) < 1e-10


def test_ridge_closed_form_grid_converged():
    """Any grid: run to convergence and compare with the closed form."""
    X, Y = synth.ridge(n=300, d=5, seed=4)
    p = admm.Problem(X, Y, "squared", "l2", lam=1e-3, sigma=2.0, rho=1.0, D=96, R=2, C=3, seed=7)
    out = admm.admm(p, 6000)
    W = admm.ridge_closed_form(p.Z(), p.Y, p.lam)
    assert np.linalg.norm(out["Wbar"] - W) / np.linalg.norm(W) < 1e-8


def test_reorganised_equals_equation_form():
    """Sec. 3: the U_ij / Delta rewrite changes memory, not the iterates."""
    X, Y = synth.multiclass(n=600, d=7, m=4, seed=5)
    for loss in ["squared", "hinge", "multinomial"]:
        p = admm.Problem(X, Y, loss, "l2", lam=1e-3, sigma=3.0, rho=0.5, D=80, R=3, C=4, seed=9)
        a = admm.admm(p, 25, variant="equation")
        b = admm.admm(p, 25, variant="reorganised")
        for key in ["Wbar", "O", "Obar", "nu", "mu"]:
            scale = max(1.0, np.abs(a[key]).max())
            assert np.abs(a[key] - b[key]).max() < 1e-12 * scale, (loss, key)


def test_incremental_equals_equation_form():
    """The projection taken from the previous (What_ij, O_ij) gives the same iterates, in the
    Gram form (s_j <= n_i) and in the outer form (n_i < s_j)."""
    X, Y = synth.multiclass(n=600, d=7, m=4, seed=5)
    for D, R, C in [(80, 3, 4), (600, 3, 2)]:
        for loss in ["squared", "hinge", "multinomial"]:
            p = admm.Problem(X, Y, loss, "l2", lam=1e-3, sigma=3.0, rho=0.5, D=D, R=R, C=C, seed=9)
            a = admm.admm(p, 25, variant="equation")
            b = admm.admm(p, 25, variant="incremental")
            for key in ["Wbar", "O", "Obar", "nu", "mu"]:
                scale = max(1.0, np.abs(a[key]).max())
                assert np.abs(a[key] - b[key]).max() < 1e-12 * scale, (D, loss, key)


def test_algorithm1_as_printed_stalls(ridge_problem):
    """Reading 1: the printed pseudo-code (no Z^T nu, stale Wbar) does not reach the minimiser."""
    X, Y = ridge_problem
    p = admm.Problem(X, Y, "squared", "l2", lam=1e-4, sigma=4.0, rho=1.0, D=512, R=1, C=1, seed=2)
    W = admm.ridge_closed_form(p.Z(), p.Y, p.lam)
    lit = admm.admm(p, 200, variant="algorithm1_literal")
    assert np.linalg.norm(lit["Wbar"] - W) / np.linalg.norm(W) > 0.5


def test_rho_scales_are_one_method():
    """Reading 2: 'mean' scaling with rho/n reproduces 'sum' scaling with rho."""
    X, Y = synth.ridge(n=200, d=4, seed=3)
    a = admm.admm(admm.Problem(X, Y, "squared", "l2", 1e-3, 2.0, 2.0, 64, 2, 2, 1, "sum"), 30)
    b = admm.admm(admm.Problem(X, Y, "squared", "l2", 1e-3, 2.0, 2.0 / 200, 64, 2, 2, 1, "mean"), 30)
    assert np.abs(a["Wbar"] - b["Wbar"]).max() < 1e-12 * np.abs(a["Wbar"]).max()


@pytest.mark.parametrize("form", ["gram", "outer"])
def test_graph_projection_kkt(form):
    """eq. (graphU)/(graphV): V = A U and (U - X) + A^T (V - Y) = 0."""
    rng = np.random.default_rng(6)
    for n, d in [(30, 7), (7, 30), (12, 12)]:
        A = rng.normal(size=(n, d))
        Xi, Yi = rng.normal(size=(d, 3)), rng.normal(size=(n, 3))
        U, V = admm.graph_projection(A, Xi, Yi, form)
        assert np.abs(V - A @ U).max() < 1e-12
        assert np.abs((U - Xi) + A.T @ (V - Yi)).max() < 1e-11


def test_graph_projection_is_the_argmin():
    """The projection beats every other point of the graph it is compared with."""
    rng = np.random.default_rng(7)
    A = rng.normal(size=(9, 4))
    Xi, Yi = rng.normal(size=(4, 2)), rng.normal(size=(9, 2))
    U, V = admm.graph_projection(A, Xi, Yi)
    f = lambda U: 0.5 * np.sum((A @ U - Yi) ** 2) + 0.5 * np.sum((U - Xi) ** 2)
    for _ in range(200):
        assert f(U) <= f(U + 1e-3 * rng.normal(size=U.shape))


@pytest.mark.parametrize("loss,reg", [("hinge", "l2"), ("squared", "l1"), ("logistic", "l2"),
                                      ("multinomial", "l2"), ("l1", "l2"), ("crammer_singer", "l2")])
def test_residuals_go_to_zero(loss, reg):
    if loss == "logistic":
        X, Y = synth.binary(n=400, d=6, seed=8)
    else:
        X, Y = synth.multiclass(n=400, d=6, m=3, seed=8)
    p = admm.Problem(X, Y, loss, reg, lam=1e-3, sigma=3.0, rho=1.0, D=64, R=2, C=2, seed=3)
    h = admm.admm(p, 600, history=True)["history"]
    assert h[-1, 0] < 1e-2 * h[5, 0] and h[-1, 1] < 1e-2 * h[5, 1]


def test_objective_decreases_to_minimum():
    X, Y = synth.ridge(n=300, d=5, seed=4)
    p = admm.Problem(X, Y, "squared", "l2", lam=1e-3, sigma=2.0, rho=1.0, D=96, R=2, C=2, seed=7)
    W = admm.ridge_closed_form(p.Z(), p.Y, p.lam)
    fmin = p.objective(W)
    f = [p.objective(admm.admm(p, k)["Wbar"]) for k in (10, 100, 3000)]
    assert f[0] > f[1] > f[2] >= fmin - 1e-9 * abs(fmin)
    assert f[2] - fmin < 1e-8 * abs(fmin)


def test_kernel_approximation_hoeffding():
    """Sec. 4: E[z(x)^T z(x')] = exp(-|x-x'|^2 / 2 sigma^2); each sample is bounded by 2/D."""
    rng = np.random.default_rng(9)
    X = rng.random((40, 6))
    sigma, D = 0.8, 8192
    Z = rff.features_block(X, 21, sigma, D, 0, D)
    K = rff.gaussian_kernel(X, X, sigma)
    delta = 1e-6
    # |2 cos cos| <= 2, Hoeffding: |mean - E| <= 2 sqrt(2 ln(2/delta) / D)
    bound = 2.0 * np.sqrt(2.0 * np.log(2.0 / delta) / D)
    assert np.abs(Z @ Z.T - K).max() <= bound


def test_kernel_error_slope():
    """Mean kernel error falls like D^-1/2 (slope of log-log fit near -1/2)."""
    rng = np.random.default_rng(10)
    X = rng.random((60, 5))
    K = rff.gaussian_kernel(X, X, 1.0)
    Ds = [2 ** k for k in range(9, 16)]
    errs = []
    for D in Ds:
        e = []
        for seed in range(4):
            Z = rff.features_block(X, 100 + seed, 1.0, D, 0, D)
            e.append(np.abs(Z @ Z.T - K).mean())
        errs.append(np.mean(e))
    slope = np.polyfit(np.log(Ds), np.log(errs), 1)[0]
    assert -0.65 < slope < -0.35


def test_block_map_independent_of_C():
    """Sec. 4 block-wise maps with global feature counters: Z_ij are columns of Z for any C."""
    rng = np.random.default_rng(11)
    X = rng.random((20, 9))
    D = 200
    Z1 = rff.features_block(X, 3, 1.5, D, 0, D)
    cols = rff.partition(D, 16)
    Z16 = np.concatenate([rff.features_block(X, 3, 1.5, D, cols[j], cols[j + 1]) for j in range(16)], axis=1)
    assert np.array_equal(Z1, Z16)


def test_memory_model_reproduces_paper_figures():
    """eq. (mem) with 8-byte values in GiB: ~6.2 GB (triloka, 1 node) and ~2.4 GB (BG/Q, 32 nodes)."""
    g1 = memory.bytes_per_node(n=200_000, d=784, m=10, s=100_000, R=1, C=200, N=1, t=6) / 2 ** 30
    g2 = memory.bytes_per_node(n=250_000, d=784, m=10, s=100_000, R=32, C=200, N=32, t=64) / 2 ** 30
    assert round(g1, 1) == 6.2
    assert round(g2, 1) == 2.4


def test_predict_is_features_times_weights():
    X, Y = synth.ridge(n=50, d=3, seed=2)
    p = admm.Problem(X, Y, "squared", "l2", 1e-3, 1.0, 1.0, 32, 1, 1, 5)
    W = np.random.default_rng(0).normal(size=(32, 1))
    Xq = X[:7]
    G, b = philox.rff_params(5, 1.0, 3, 32)
    assert np.allclose(p.predict(Xq, W), rff.features(Xq, G, b, 32) @ W, rtol=0, atol=1e-14)


# ----------------------------------------------------------------- stochastic block subsets
def test_block_mask_frequency_and_full_fraction():
    """Each block is active with probability p, independently across blocks and iterations
    (binomial bounds at 6 sigma); p = 1 keeps every block active."""
    R, C, K = 4, 4, 400
    for p in (0.25, 0.5, 0.8):
        M = np.array([admm.block_mask(11, R, C, k, p) for k in range(K)])
        n = M.size
        assert abs(M.mean() - p) < 6 * np.sqrt(p * (1 - p) / n)
        per_block = M.reshape(K, R * C).mean(axis=0)
        assert np.all(np.abs(per_block - p) < 6 * np.sqrt(p * (1 - p) / K))
        # successive iterations are not copies of each other
        assert np.mean([np.array_equal(M[k], M[k + 1]) for k in range(K - 1)]) < 0.2
    assert all(admm.block_mask(3, 5, 3, k, 1.0).all() for k in range(50))


def test_stochastic_equation_equals_reorganised():
    X, Y = synth.multiclass(n=300, d=5, m=3, seed=12)
    p = admm.Problem(X, Y, "hinge", "l2", lam=1e-3, sigma=2.0, rho=1.0, D=120, R=3, C=2, seed=5)
    a = admm.admm(p, 40, variant="equation", block_fraction=0.5)
    b = admm.admm(p, 40, variant="reorganised", block_fraction=0.5)
    assert np.abs(a["Wbar"] - b["Wbar"]).max() < 1e-12 * max(1.0, np.abs(a["Wbar"]).max())


def test_stochastic_equation_equals_incremental():
    """An inactive block keeps What_ij and O_ij, from which its next projection starts."""
    X, Y = synth.multiclass(n=300, d=5, m=3, seed=12)
    p = admm.Problem(X, Y, "hinge", "l2", lam=1e-3, sigma=2.0, rho=1.0, D=120, R=3, C=2, seed=5)
    a = admm.admm(p, 40, variant="equation", block_fraction=0.5)
    b = admm.admm(p, 40, variant="incremental", block_fraction=0.5)
    assert np.abs(a["Wbar"] - b["Wbar"]).max() < 1e-12 * max(1.0, np.abs(a["Wbar"]).max())


def test_stochastic_keeps_consensus_duals_summing_to_zero():
    """mu_j + sum_i mu_ij = 0 after every iteration, as in the full method."""
    X, Y = synth.ridge(n=240, d=4, seed=13)
    p = admm.Problem(X, Y, "squared", "l2", lam=1e-3, sigma=2.0, rho=1.0, D=90, R=3, C=3, seed=8)
    for it in (1, 7, 30):
        o = admm.admm(p, it, block_fraction=0.4)
        s = o["mu"] + sum(o["muij"])
        assert np.abs(s).max() < 1e-12 * max(1.0, np.abs(o["mu"]).max())


def test_stochastic_reaches_ridge_closed_form():
    """With half of the blocks updated per iteration the iterates still reach the
    minimiser (Sec. 2.2 closed form), at about half the rate of the full method."""
    X, Y = synth.ridge(n=300, d=5, seed=4)
    p = admm.Problem(X, Y, "squared", "l2", lam=1e-3, sigma=2.0, rho=1.0, D=96, R=2, C=2, seed=7)
    W = admm.ridge_closed_form(p.Z(), p.Y, p.lam)
    o = admm.admm(p, 6000, variant="reorganised", block_fraction=0.5)
    assert np.linalg.norm(o["Wbar"] - W) / np.linalg.norm(W) < 1e-5


def test_stochastic_residuals_go_to_zero():
    X, Y = synth.multiclass(n=400, d=6, m=3, seed=8)
    p = admm.Problem(X, Y, "hinge", "l2", lam=1e-3, sigma=3.0, rho=1.0, D=64, R=2, C=2, seed=3)
    h = admm.admm(p, 1200, variant="reorganised", history=True, block_fraction=0.5)["history"]
    assert h[-1, 0] < 1e-2 * h[5, 0] and h[-1, 1] < 1e-2 * h[5, 1]


def test_random_feature_ridge_tends_to_kernel_ridge():
    """Sec. 2.2: with the exact kernel the minimiser is f(x) = sum_i alpha_i k(x, x_i),
    (K + n lam I) alpha = Y (eq. (krr)); the random-feature ridge solution's predictions
    approach it as D grows (error falling roughly like D^-1/2)."""
    rng = np.random.default_rng(21)
    X = rng.random((80, 3))
    Y = np.sin(3 * X.sum(1, keepdims=True))
    Xq = rng.random((40, 3))
    sigma, lam, n = 0.7, 1e-3, 80
    alpha = np.linalg.solve(rff.gaussian_kernel(X, X, sigma) + n * lam * np.eye(n), Y)
    f_krr = rff.gaussian_kernel(Xq, X, sigma) @ alpha
    errs = []
    Ds = [256, 1024, 4096, 16384]
    for D in Ds:
        e = []
        for seed in range(3):
            Z = rff.features_block(X, 40 + seed, sigma, D, 0, D)
            # (Z^T Z + n lam I)^-1 Z^T Y = Z^T (Z Z^T + n lam I)^-1 Y: the n x n form, same W
            W = Z.T @ np.linalg.solve(Z @ Z.T + n * lam * np.eye(n), Y)
            e.append(np.abs(rff.features_block(Xq, 40 + seed, sigma, D, 0, D) @ W - f_krr).mean())
        errs.append(np.mean(e))
    slope = np.polyfit(np.log(Ds), np.log(errs), 1)[0]
    assert errs[-1] < 0.25 * errs[0]
    assert -0.8 < slope < -0.25, (slope, errs)
