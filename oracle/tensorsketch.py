"""TensorSketch features for the polynomial kernel (Sec. 4 lists TensorSketch among the
solver's maps; Pham and Pagh, "Fast and scalable polynomial kernels via explicit feature
maps", KDD 2013).

Test infrastructure (see the package header): never imported by the product.

Kernel: k(x, y) = (<x, y> / sigma^2 + c)^q, degree q >= 1, offset c >= 0.  With the
augmented input x' = (x / sigma, sqrt(c)) (d + 1 entries), k(x, y) = <x', y'>^q.

Sketch of length S: q independent CountSketches CS_p(x')[t] = sum over the entries i with
h_p(i) = t of g_p(i) x'_i (h_p uniform on {0..S-1}, g_p uniform signs), combined by circular
convolution,
    TS(x) = CS_1(x') * CS_2(x') * ... * CS_q(x')   (length S, indices mod S),
which is the CountSketch of the tensor power x'^(tensor q) under the hash
H(i_1..i_q) = (h_1(i_1) + ... + h_q(i_q)) mod S and the sign g_1(i_1) ... g_q(i_q); so
E[<TS(x), TS(y)>] = <x', y'>^q.  Computed here with the FFT: TS = ifft(prod_p fft(CS_p)).

Blocks (Sec. 4: a map that must produce its whole transformed vector is assembled from
independent maps z_j of s_j features each, z(x) = s^-1/2 [sqrt(s_1) z_1(x) ... sqrt(s_C)
z_C(x)]): column block j carries its own sketch of length s_j, and Z[:, block j] =
sqrt(s_j / D) TS_j(X).  Unlike the random Fourier map, Z therefore depends on the column
partition.

Stream layout (a reading: the paper fixes none of it), key as in philox.py: for block j,
degree p (0-based) and augmented entry i, counter (j, p (d + 1) + i, 7, 0) gives
h = floor(w0 s_j / 2^32) and g = -1 if the top bit of w1 is set, else +1.

Pins: the FFT form against the CountSketch of the explicit tensor power (brute force), the
kernel estimate's mean over independent seeds against (<x, y>/sigma^2 + c)^q, the block
scaling identity, the hash and sign distributions.
"""
import numpy as np

from . import philox


def hashes(seed, j, S, d, q):
    """(h, g) of block j, each q x (d + 1): bucket in [0, S) and sign +-1 per augmented entry."""
    key = philox.seed_key(seed)
    c1 = np.arange(q * (d + 1), dtype=np.uint64)
    z = np.zeros_like(c1)
    w = philox.philox4x32_10(z + np.uint64(j), c1, z + np.uint64(7), z, key[0], key[1])
    h = ((w[0] * np.uint64(S)) >> np.uint64(32)).astype(np.int64).reshape(q, d + 1)
    g = np.where((w[1] >> np.uint64(31)) != 0, -1.0, 1.0).reshape(q, d + 1)
    return h, g


def augment(X, sigma, c):
    """x' = (x / sigma, sqrt(c)) for every row of X, float64."""
    X = np.asarray(X, dtype=np.float64)
    return np.concatenate([X / float(sigma), np.full((X.shape[0], 1), np.sqrt(float(c)))], axis=1)


def count_sketch(Xp, h, g, S):
    """CS(x')[t] = sum over i with h(i) = t of g(i) x'_i, for every row of Xp (n x (d+1))."""
    out = np.zeros((Xp.shape[0], S))
    for i in range(Xp.shape[1]):
        out[:, h[i]] += g[i] * Xp[:, i]
    return out


def sketch_block(X, seed, sigma, c, q, S, j):
    """TS_j(X): n x S, the block's sketch of every row (without the block scale)."""
    Xp = augment(X, sigma, c)
    h, g = hashes(seed, j, S, Xp.shape[1] - 1, q)
    F = np.ones((Xp.shape[0], S), dtype=np.complex128)
    for p in range(q):
        F *= np.fft.fft(count_sketch(Xp, h[p], g[p], S), axis=1)
    return np.real(np.fft.ifft(F, axis=1))


def features(X, seed, sigma, c, q, cols):
    """Z = [sqrt(s_j / D) TS_j(X)] over the column blocks with boundaries cols (float64)."""
    D = int(cols[-1])
    blocks = []
    for j in range(len(cols) - 1):
        S = int(cols[j + 1] - cols[j])
        blocks.append(np.sqrt(S / D) * sketch_block(X, seed, sigma, c, q, S, j))
    return np.concatenate(blocks, axis=1)


def polynomial_kernel(X1, X2, sigma, c, q):
    """k(x, y) = (<x, y> / sigma^2 + c)^q."""
    X1 = np.asarray(X1, dtype=np.float64)
    X2 = np.asarray(X2, dtype=np.float64)
    return (X1 @ X2.T / (float(sigma) ** 2) + float(c)) ** int(q)
