"""Writes the FP64 oracle iterates of the seeded 20,000-row sample of the large implicit
workload, the stored values that tests/test_gpu_large.py (and the benchmark's "large"
leg) compare the GPU paths with.

Workload: synth.sparse01(n=20,000, d=784, m=10, seed=3) (MNIST-8M-shaped rows, ~20 %
non-zero), sigma = 9, D = 65,536 Philox features (seed 4), one-vs-rest hinge loss + l2,
lambda = 1e-6, rho = 1 (sum-scaled), 50 iterations of the equation form of block-splitting
ADMM (Sec. 3), on two grids:
  32 x 16  the full workload's grid: 625-row blocks, fewer rows than the 4,096 features of
           a column block, so the oracle projects with I + Z_ij Z_ij^T (the outer form);
  2 x 16   10,000-row blocks, so it projects with I + Z_ij^T Z_ij (the Gram form of the
           full-size solve, whose blocks have 253,125 rows).

Only oracle/ computes (Z is an explicit 20,000 x 65,536 float64 matrix, 10.5 GB, formed in
row chunks).  Output: large_20k_32x16_wbar50.npz and large_20k_2x16_wbar50.npz, each with
a seeded sample of 32,768 entries of Wbar (flat indices `idx`, float64 values `w`), the
Frobenius norm of the whole Wbar (`fro`), the objective at Wbar (`objective`) and the row
count (`n`).

    python tests/golden/make_large_sample_reference.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import admm, philox, rff  # noqa: E402

N, DIN, M, SIGMA, D, LAM, RHO, ITERS = 20_000, 784, 10, 9.0, 65536, 1e-6, 1.0, 50
DATA_SEED, PHILOX_SEED = 3, 4
GRIDS = [(32, 16), (2, 16)]
SAMPLE, SAMPLE_SEED = 32768, 0


def main():
    t0 = time.time()
    X, Y = synth.sparse01(n=N, d=DIN, m=M, seed=DATA_SEED)
    G, b = philox.rff_params(PHILOX_SEED, SIGMA, DIN, D, 0, D)
    Z = np.empty((N, D))
    for r0 in range(0, N, 1000):
        Z[r0:r0 + 1000] = rff.features(X[r0:r0 + 1000], G, b, D)
    del G, b
    print("Z %.0f s" % (time.time() - t0), flush=True)
    for R, C in GRIDS:
        p = admm.Problem(X, Y, "hinge", "l2", LAM, SIGMA, RHO, D, R, C, seed=PHILOX_SEED)
        p._Z = Z                   # the same matrix Problem.Z() would form, built in chunks
        W = admm.admm(p, ITERS)["Wbar"]
        idx = np.sort(np.random.default_rng(SAMPLE_SEED).choice(W.size, SAMPLE, replace=False)).astype(np.int64)
        out = os.path.join(HERE, "large_20k_%dx%d_wbar50.npz" % (R, C))
        np.savez(out, idx=idx, w=W.ravel()[idx], fro=np.linalg.norm(W), objective=p.objective(W), n=N)
        print("wrote %s (%.0f s)" % (out, time.time() - t0), flush=True)


if __name__ == "__main__":
    main()
