"""Explicit random Fourier feature matrix, block partitions, Gaussian kernel.

Test infrastructure (see the package header): never imported by the product.

Sec. 4 (Random Fourier Features): z(x) = cos(omega^T x + b) scaled, omega an
appropriately scaled Gaussian, b uniform on [0, pi), approximating the Gaussian
kernel k(x, x') = exp(-|x - x'|^2 / (2 sigma^2)).

Reading of the scale (the printed 1/sqrt(s) gives E[z(x)^T z(x')] = k/2): this
build uses sqrt(2/D), so that Z Z^T -> K.  With b ~ U[0, pi), 2b is uniform on
[0, 2 pi) and the estimator stays unbiased: E[2 cos(a+b) cos(c+b)] = cos(a-c).

Sec. 4 (block-wise maps): z(x) = s^-1/2 [sqrt(s_1) z_1(x) ... sqrt(s_C) z_C(x)]
with z_j independent maps of s_j features each.  Drawing every feature from a
counter indexed by its GLOBAL feature number makes this identical to one map of
D features, for every C: block j of Z is simply columns of the full Z.

Sec. 3 (partition): n = sum n_i over R row blocks, s = sum s_j over C column
blocks; sizes may be uneven.  Reading: the leading (n mod R) blocks get one
extra row, likewise for features, and blocks are contiguous ranges.

Random Laplace features (Sec. 4 lists them among the solver's other maps; Yang,
Sindhwani, Fan, Avron and Mahoney 2014): for nonnegative inputs (histograms),
z(x) = exp(-W^T x) / sqrt(D) with W[r, k] i.i.d. Levy(0, 1/(2 sigma^2)), whose
inner products estimate the exponential semigroup kernel
k(x, x') = exp(-sum_r sqrt(x_r + x'_r) / sigma).  Same operator T[X_i, j] and
block structure; only the nonlinearity and the parameter law change.

Pins: Z Z^T against the Gaussian kernel within a Hoeffding bound; the slope of
the mean kernel error against D; Z block (C = 16) == columns of Z (C = 1),
bitwise; partition sizes against their definition; the Laplace map against the
semigroup kernel within a Hoeffding bound, its parameters against the Levy CDF.
"""

MAPS = ("fourier", "laplace", "fastfood", "tensorsketch")
import numpy as np

from . import philox


def partition(total, parts):
    """Block boundaries [start_0, ..., start_parts]: leading blocks one larger."""
    if parts <= 0 or total < 0:
        raise ValueError("bad partition")
    q, rem = divmod(total, parts)
    sizes = [q + 1 if p < rem else q for p in range(parts)]
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def features(X, G, b, D):
    """Z = sqrt(2/D) cos(X G + b) in float64 (rows of X, columns of G)."""
    X = np.asarray(X, dtype=np.float64)
    A = X @ np.asarray(G, dtype=np.float64) + np.asarray(b, dtype=np.float64)[None, :]
    return np.sqrt(2.0 / D) * np.cos(A)


def laplace_features(X, W, D):
    """Z = exp(-X W) / sqrt(D) in float64."""
    A = np.asarray(X, dtype=np.float64) @ np.asarray(W, dtype=np.float64)
    return np.exp(-A) / np.sqrt(D)


def features_block(X, seed, sigma, D, k_lo, k_hi, feature_map="fourier"):
    """Z restricted to global features k_lo..k_hi-1 (the operator T[X_i, j])."""
    if feature_map == "laplace":
        return laplace_features(X, philox.laplace_params(seed, sigma, X.shape[1], D, k_lo, k_hi), D)
    if feature_map == "fastfood":
        from . import fastfood
        G, b = fastfood.fastfood_params(seed, sigma, X.shape[1], D, k_lo, k_hi)
        return features(X, G, b, D)
    if feature_map != "fourier":
        raise ValueError(feature_map)
    G, b = philox.rff_params(seed, sigma, X.shape[1], D, k_lo, k_hi)
    return features(X, G, b, D)


def semigroup_kernel(X1, X2, sigma):
    """k(x, x') = exp(-sum_r sqrt(x_r + x'_r) / sigma) for nonnegative x, x'."""
    X1 = np.asarray(X1, dtype=np.float64)
    X2 = np.asarray(X2, dtype=np.float64)
    return np.exp(-np.sqrt(X1[:, None, :] + X2[None, :, :]).sum(-1) / sigma)


def gaussian_kernel(X1, X2, sigma):
    """k(x, x') = exp(-|x - x'|^2 / (2 sigma^2)) (Sec. 4)."""
    X1 = np.asarray(X1, dtype=np.float64)
    X2 = np.asarray(X2, dtype=np.float64)
    d2 = (X1 * X1).sum(1)[:, None] + (X2 * X2).sum(1)[None, :] - 2.0 * X1 @ X2.T
    return np.exp(-np.maximum(d2, 0.0) / (2.0 * sigma * sigma))
