"""Fastfood feature parameters (Sec. 4 lists Fastfood among the solver's maps; Le, Sarlos
and Smola, "Fastfood: approximating kernel expansions in loglinear time", ICML 2013).

Test infrastructure (see the package header): never imported by the product.

The map is the random Fourier map z(x) = sqrt(2/D) cos(V x + b) with a structured V in place
of a dense Gaussian G^T.  With d' the smallest power of two >= d (inputs zero-padded to d'),
the features come in blocks of d' rows,

    V_block = (1 / (sigma sqrt(d'))) S H diag(g) P H diag(B),

H the d' x d' Walsh-Hadamard matrix (Sylvester order, H[i, j] = (-1)^popcount(i & j)),
B random signs, P a random permutation ((P y)[m] = y[pi(m)]), g standard normals, and
S = diag(s_i / |g|) with s_i chi-distributed with d' degrees of freedom.  Each row of H diag(g) P
H diag(B) is an N(0, d' I) vector of length sqrt(d') |g|, so every row of V is distributed as
N(0, I / sigma^2), the spectral law of the Gaussian kernel: the estimator stays unbiased while
V x costs O(d' log d') per block instead of O(d'^2).

Stream layout (a reading: the paper fixes none of it), key as in philox.py, block beta =
k // d' for global feature k, row i = k mod d' inside it:
  B[beta, j]  counter (beta, j, 3, 0), word 0: -1 if its top bit is set, else +1
  g[beta, m]  counter (beta, m, 4, 0): the first Box-Muller normal of words 0, 1
  pi[beta]    Fisher-Yates from the identity: for i = d'-1 down to 1, word 0 w of counter
              (beta, i, 5, 0) gives j = floor(w (i + 1) / 2^32); swap pi[i], pi[j]
  s[k]        counter (k, q, 6, 0) for q < d'/2 (d' = 1: q = 0): both Box-Muller normals of
              words 0, 1; s = sqrt(sum of the d' squares)
  b[k]        as for the random Fourier map (counter (k, 0, 1, 0))
V is formed in float64 and rounded to float32 once.

Pins: rows Gaussian with the right norm law (Kolmogorov-Smirnov), the dense V against the
same product evaluated by fast transforms, the Gaussian kernel estimate, block independence.
"""
import numpy as np
import scipy.linalg

from . import philox


def padded_dim(d):
    """d' = the smallest power of two >= d."""
    p = 1
    while p < d:
        p *= 2
    return p


def _words(c0, c1, tag, key):
    c0 = np.asarray(c0, dtype=np.uint64)
    c1 = np.asarray(c1, dtype=np.uint64)
    z = np.zeros(np.broadcast(c0, c1).shape, dtype=np.uint64)
    return philox.philox4x32_10(c0 + z, c1 + z, z + np.uint64(tag), z, key[0], key[1])


def block_params(seed, dp, beta):
    """(B, g, perm) of block beta: signs, normals and the permutation pi as an index array."""
    key = philox.seed_key(seed)
    j = np.arange(dp, dtype=np.uint64)
    wb = _words(beta, j, 3, key)[0]
    B = np.where((wb >> np.uint64(31)) != 0, -1.0, 1.0)
    wg = _words(beta, j, 4, key)
    g, _ = philox.box_muller(philox.uniform_from_word(wg[0]), philox.uniform_from_word(wg[1]))
    perm = list(range(dp))
    for i in range(dp - 1, 0, -1):
        w = int(_words(beta, i, 5, key)[0])
        jj = (w * (i + 1)) >> 32
        perm[i], perm[jj] = perm[jj], perm[i]
    return B, g, np.array(perm, dtype=np.int64)


def chi_scales(seed, dp, ks):
    """s[k] for the global features ks: the length of a d'-dimensional standard normal vector."""
    key = philox.seed_key(seed)
    q = np.arange(max(dp // 2, 1), dtype=np.uint64)[None, :]
    w = _words(np.asarray(ks, dtype=np.uint64)[:, None], q, 6, key)
    a, c = philox.box_muller(philox.uniform_from_word(w[0]), philox.uniform_from_word(w[1]))
    n = np.stack([a, c], axis=2).reshape(len(ks), -1)[:, :dp]     # normals 2q, 2q+1 in order
    return np.sqrt(np.sum(n * n, axis=1))


def block_matrix(seed, sigma, dp, beta):
    """The d' x d' block V_block in float64, written as the product of its factors."""
    B, g, perm = block_params(seed, dp, beta)
    H = scipy.linalg.hadamard(dp).astype(np.float64)
    P = np.zeros((dp, dp))
    P[np.arange(dp), perm] = 1.0
    s = chi_scales(seed, dp, beta * dp + np.arange(dp))
    S = np.diag(s / np.linalg.norm(g))
    return (S @ H @ np.diag(g) @ P @ H @ np.diag(B)) / (float(sigma) * np.sqrt(dp))


def fastfood_params(seed, sigma, d, D, k_lo=0, k_hi=None):
    """(G, b) for global features k_lo..k_hi-1: G = V[k_lo:k_hi, :d]^T in float32 (d x nk),
    b as for the random Fourier map, so that z = sqrt(2/D) cos(x^T G + b)."""
    if k_hi is None:
        k_hi = D
    dp = padded_dim(d)
    rows = []
    for beta in range(k_lo // dp, (k_hi - 1) // dp + 1 if k_hi > k_lo else k_lo // dp):
        V = block_matrix(seed, sigma, dp, beta)
        lo, hi = max(k_lo, beta * dp), min(k_hi, (beta + 1) * dp)
        rows.append(V[lo - beta * dp:hi - beta * dp, :d])
    G = (np.concatenate(rows, axis=0) if rows else np.zeros((0, d))).T.astype(np.float32)
    _, b = philox.rff_params(seed, sigma, 1, D, k_lo, k_hi)
    return np.ascontiguousarray(G), b
