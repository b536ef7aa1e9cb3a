"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds NO arithmetic of the method (no features, no proxes, no ADMM):
it only draws data matrices X (n x d, float32) and targets Y (n x m, float32)
with numpy's PCG64 generator, so that the GPU library, the oracle, the tests and
the benchmark all see identical inputs.  The random numbers the METHOD draws
(the Gaussian projection G and the phases b) are not made here: each side
produces them from the Philox4x32-10 definition.

The paper's data sets (MNIST-8M, TIMIT) are not available; these recipes stand
in for them with matching shapes and value ranges (Sec. 5, "Datasets"):

* ``ridge``       n=2000, d=16, X ~ U[0,1], y = sin(2 pi x.u) + 0.1 N(0,1),
                  u ~ N(0, I/d); real-valued single output.
* ``multiclass``  Gaussian mixture with one class per component (TIMIT-like:
                  d=440, 147 classes): means ~ N(0, I), within-class N(0, 4 I),
                  every feature then standardised; +-1 one-hot targets.
* ``sparse01``    MNIST-like: d=784 values in [0,1], about 20% non-zero; each
                  of the classes has a random support template (35% of the
                  coordinates) and a mean intensity pattern, each row keeps its
                  template entries with probability 0.57 and jitters them;
                  +-1 one-hot targets.  Drawn in independent chunks (threads), so
                  the 8.1M-row MNIST-8M stand-in takes seconds.
* ``binary``      two Gaussians N(+-mu, I), mu ~ 2 N(0, I/d), labels +-1.
* ``histograms``  bag-of-words style histograms for the random Laplace map
                  (nonnegative rows summing to 1): each class draws a Dirichlet
                  weight over the d bins with most mass on a random 20% of them;
                  a row is a normalised Gamma draw around its class weights
                  (concentration 50); +-1 one-hot targets.
"""
import numpy as np


def _rng(seed):
    return np.random.default_rng(int(seed))


def ridge(n=2000, d=16, seed=0):
    rng = _rng(seed)
    X = rng.random((n, d))
    u = rng.standard_normal(d) / np.sqrt(d)
    y = np.sin(2.0 * np.pi * (X @ u)) + 0.1 * rng.standard_normal(n)
    return X.astype(np.float32), y.reshape(n, 1).astype(np.float32)


def onehot_pm1(labels, m):
    Y = -np.ones((labels.shape[0], m), dtype=np.float32)
    Y[np.arange(labels.shape[0]), labels] = 1.0
    return Y


def multiclass(n=200_000, d=440, m=147, seed=0, chunk=50_000):
    rng = _rng(seed)
    means = rng.standard_normal((m, d)).astype(np.float32)
    labels = rng.integers(0, m, size=n)
    X = np.empty((n, d), dtype=np.float32)
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        X[r0:r1] = means[labels[r0:r1]] + 2.0 * rng.standard_normal((r1 - r0, d), dtype=np.float32)
    mu = X.mean(axis=0, dtype=np.float64).astype(np.float32)
    sd = X.std(axis=0, dtype=np.float64).astype(np.float32)
    X -= mu
    X /= np.maximum(sd, 1e-6)
    return X, onehot_pm1(labels, m)


def sparse01(n=20_000, d=784, m=10, seed=0, chunk=65_536, out=None, threads=None):
    """Rows in chunks of `chunk`, chunk c drawn from its own PCG64 stream (spawn key c + 1)
    and the class templates from spawn key 0, so the chunks can be drawn by several
    threads and every full chunk is the same whatever n.  `out` (n x d float32, e.g. pinned host
    memory) receives X when given."""
    import concurrent.futures
    import os
    tmpl = np.random.default_rng(np.random.SeedSequence(int(seed), spawn_key=(0,)))
    support = tmpl.random((m, d)) < 0.35
    level = tmpl.random((m, d)).astype(np.float32)
    X = np.empty((n, d), dtype=np.float32) if out is None else out
    labels = np.empty(n, dtype=np.int64)

    def fill(c):
        r0, r1 = c * chunk, min(n, (c + 1) * chunk)
        rng = np.random.default_rng(np.random.SeedSequence(int(seed), spawn_key=(c + 1,)))
        lab = rng.integers(0, m, size=r1 - r0)
        keep = support[lab] & (rng.random((r1 - r0, d), dtype=np.float32) < np.float32(0.57))
        val = level[lab] + np.float32(0.25) * rng.standard_normal((r1 - r0, d), dtype=np.float32)
        np.clip(val, 0.0, 1.0, out=val)
        X[r0:r1] = np.where(keep, val, np.float32(0.0))
        labels[r0:r1] = lab

    nchunks = -(-n // chunk)
    workers = threads or min(nchunks, os.cpu_count() or 1, 32)
    if workers <= 1:
        for c in range(nchunks):
            fill(c)
    else:
        with concurrent.futures.ThreadPoolExecutor(workers) as ex:
            list(ex.map(fill, range(nchunks)))
    return X, onehot_pm1(labels, m)


def binary(n=10_000, d=128, seed=0):
    rng = _rng(seed)
    mu = 2.0 * rng.standard_normal(d) / np.sqrt(d)
    y = np.where(rng.random(n) < 0.5, 1.0, -1.0)
    X = y[:, None] * mu[None, :] + rng.standard_normal((n, d))
    return X.astype(np.float32), y.reshape(n, 1).astype(np.float32)


def histograms(n=20_000, d=256, m=10, seed=0):
    rng = _rng(seed)
    boost = np.where(rng.random((m, d)) < 0.2, 5.0, 0.2)
    weights = rng.dirichlet(np.ones(d), size=m) * boost
    weights /= weights.sum(axis=1, keepdims=True)
    labels = rng.integers(0, m, size=n)
    X = rng.gamma(50.0 * weights[labels] + 1e-3)
    X /= X.sum(axis=1, keepdims=True)
    return X.astype(np.float32), onehot_pm1(labels, m)
