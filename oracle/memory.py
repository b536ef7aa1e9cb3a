"""The per-node memory model of Sec. 3 ("Memory Requirements"), eq. (mem).

Test infrastructure (see the package header): never imported by the product.

Floats held per node when R processes run on N nodes, each with t threads,
s_j = s/C and n_i = n/R:
    4nm/N + 5smR/N + nd/N + nm/N + tns/(CN) + tsmR/(CN) + nmt/N + nm/N + s^2 R/(CN)
(terms: O, Obar, nu, Delta-bar; Wbar, W', mu', mu, U; X_i and Y_i; the
materialised Z_ij of the t threads; temporaries A, O' and Delta; the factor cache.)

Pin: with 8-byte values and GiB units it reproduces the two figures the
experiments section quotes (about 6.2 GB for MNIST, n = 200K, s = 100K, C = 200
on one node with t = 6; about 2.4 GB for n = 250K on 32 BG/Q nodes, t = 64).
"""


def floats_per_node(n, d, m, s, R, C, N, t):
    """Eq. (mem): number of floating-point values held by one node."""
    return (4 * n * m / N + 5 * s * m * R / N + n * d / N + n * m / N
            + t * n * s / (C * N) + t * s * m * R / (C * N) + n * m * t / N + n * m / N
            + s * s * R / (C * N))


def bytes_per_node(n, d, m, s, R, C, N, t, value_bytes=8):
    return value_bytes * floats_per_node(n, d, m, s, R, C, N, t)
