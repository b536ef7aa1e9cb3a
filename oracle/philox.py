"""Philox4x32-10 and the random Fourier feature parameters drawn from it.

Test infrastructure (see the package header): never imported by the product.

The paper keeps the Gaussian projection omega implicit, as the state of a
pseudo-random generator from which parts of omega are regenerated on demand
(Sec. 4, the paragraph on the O(sd) memory of omega). It names no generator.
This build fixes it to Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11), a counter-based generator, so that
any entry of omega can be produced from its index alone.

Generator definition (Salmon et al., Sec. 3 / Random123 reference):
  round:  (c0,c1,c2,c3), key (k0,k1)
          hi0:lo0 = 0xD2511F53 * c0   (32x32 -> 64-bit product)
          hi1:lo1 = 0xCD9E8D57 * c2
          -> (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
  key bump between rounds: k0 += 0x9E3779B9, k1 += 0xBB67AE85 (mod 2^32)
  10 rounds; the first round uses the unbumped key.

Stream layout (a reading: the paper leaves it open):
  key      = (seed mod 2^32, seed >> 32)
  G[r, k]  : counter (k, r // 4, 0, 0); its 4 words give two Box-Muller pairs
             for rows 4q, 4q+1 (words 0,1) and 4q+2, 4q+3 (words 2,3)
  b[k]     : counter (k, 0, 1, 0), word 0
  uniform  : u = ((w >> 8) + 0.5) * 2^-24, exact in float64, inside (0, 1)
  normal   : Box-Muller, rho = sqrt(-2 ln u1), theta = 2 pi u2,
             (rho cos theta, rho sin theta), in float64
  G = float32(normal / sigma)  so that omega ~ N(0, sigma^-2 I), the spectral
      measure of the Gaussian kernel exp(-|x-x'|^2 / (2 sigma^2)) (Sec. 4)
  b = float32(u * pi)          b ~ U[0, pi) as Sec. 4 states

Pins: published known-answer vectors, an independent Philox implementation
(the Triton language's, run in its CPU interpreter), moments of the outputs.
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on broadcastable uint32 arrays (as uint64 holders).

    Returns four uint64 arrays holding the 32-bit output words.
    """
    c0 = np.asarray(c0, dtype=np.uint64) & MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & MASK32
    k0 = np.asarray(k0, dtype=np.uint64) & MASK32
    k1 = np.asarray(k1, dtype=np.uint64) & MASK32
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * c0          # < 2^64, exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return c0, c1, c2, c3


def seed_key(seed):
    """Split a 64-bit seed into the Philox key (k0, k1)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.uint64(seed & 0xFFFFFFFF), np.uint64(seed >> 32)


def uniform_from_word(w):
    """u = ((w >> 8) + 0.5) / 2^24 in float64: 2^24 equally spaced points in (0,1)."""
    w = np.asarray(w, dtype=np.uint64)
    return ((w >> np.uint64(8)).astype(np.float64) + 0.5) * (2.0 ** -24)


def box_muller(u1, u2):
    """Two independent standard normals from two uniforms, in float64."""
    rho = np.sqrt(-2.0 * np.log(u1))
    theta = (2.0 * np.pi) * u2
    return rho * np.cos(theta), rho * np.sin(theta)


def g_words(seed, d, k_lo, k_hi):
    """Raw Philox words behind G[:, k_lo:k_hi]: array (4, ceil(d/4), k_hi-k_lo)."""
    k0, k1 = seed_key(seed)
    nq = (d + 3) // 4
    kk = np.arange(k_lo, k_hi, dtype=np.uint64)[None, :]
    qq = np.arange(nq, dtype=np.uint64)[:, None]
    return np.stack(philox4x32_10(kk, qq, 0, 0, k0, k1))


def _gauss(seed, d, k_lo, k_hi):
    """The float64 standard normals behind G[:, k_lo:k_hi], shape (d, k_hi-k_lo)."""
    w = g_words(seed, d, k_lo, k_hi)                     # (4, nq, nk)
    u = uniform_from_word(w)
    a0, a1 = box_muller(u[0], u[1])                      # rows 4q, 4q+1
    a2, a3 = box_muller(u[2], u[3])                      # rows 4q+2, 4q+3
    nq, nk = u.shape[1], u.shape[2]
    z = np.empty((nq, 4, nk), dtype=np.float64)
    z[:, 0], z[:, 1], z[:, 2], z[:, 3] = a0, a1, a2, a3
    return z.reshape(4 * nq, nk)[:d]


def laplace_params(seed, sigma, d, D, k_lo=0, k_hi=None):
    """Random Laplace feature parameters for global features k_lo..k_hi-1.

    W float32 (d, k_hi-k_lo), W[r, k] = 1 / (2 sigma^2 g^2) with g the standard normal
    the Fourier map would use for G[r, k]: a Levy(0, c) draw with c = 1 / (2 sigma^2)
    (c / g^2 is Levy-distributed), whose Laplace transform is E[exp(-t W)] =
    exp(-sqrt(2 c t)) = exp(-sqrt(t) / sigma).
    """
    if k_hi is None:
        k_hi = D
    g = _gauss(seed, d, k_lo, k_hi)
    return (1.0 / (2.0 * float(sigma) * float(sigma) * g * g)).astype(np.float32)


def rff_params(seed, sigma, d, D, k_lo=0, k_hi=None):
    """Random Fourier feature parameters for global features k_lo..k_hi-1.

    Returns (G, b): G float32 (d, k_hi-k_lo) with G[r, k] ~ N(0, sigma^-2),
    b float32 (k_hi-k_lo,) with b ~ U[0, pi).  Any column range gives the same
    values as slicing the full (d, D) matrix: the block-wise construction of
    Sec. 4 is exact and independent of the column split C.
    """
    if k_hi is None:
        k_hi = D
    G = (_gauss(seed, d, k_lo, k_hi) / float(sigma)).astype(np.float32)
    k0, k1 = seed_key(seed)
    kk = np.arange(k_lo, k_hi, dtype=np.uint64)
    wb = philox4x32_10(kk, 0, 1, 0, k0, k1)[0]
    b = (uniform_from_word(wb) * np.pi).astype(np.float32)
    return G, b
