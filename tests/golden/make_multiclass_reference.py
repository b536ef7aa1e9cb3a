"""Writes the FP64 oracle iterate of the full multiclass workload, the stored value that
tests/test_gpu_full_size.py compares the GPU paths with.

Workload (the benchmark's): synth.multiclass(n=200,000, d=440, m=147, seed=1), sigma = 10,
D = 16,384 Philox features (seed 2), 4 x 4 blocks, squared loss + l2, lambda = 1e-5,
rho = 1 (sum-scaled), 23 iterations of the equation form of block-splitting ADMM (Sec. 3).

Only oracle/ computes: Z is formed in row chunks by oracle.rff.features (an explicit
n x D float64 matrix, 26 GB) so that no temporary of that size is needed beside it, and
oracle.admm.admm runs the iterations.  About 10 minutes and 40 GB of host memory on an
8-core machine.  Output: multiclass_200k_wbar23_sample.npz, a seeded random sample of
32,768 entries of Wbar (flat indices `idx`, float64 values `w`), the Frobenius norm of
the whole Wbar (`fro`) and the objective at Wbar (`objective`); the relative error on the
sample estimates the relative error of the whole matrix.

With --stochastic the same workload runs the stochastic block-subset variant with half of
the blocks active per iteration (block fraction 0.5, masks from Philox as oracle.admm
draws them) and writes multiclass_200k_p05_wbar23_sample.npz.

    python tests/golden/make_multiclass_reference.py [--stochastic]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import admm, philox, rff  # noqa: E402

N, DIN, M, SIGMA, D, R, C, LAM, RHO, ITERS = 200_000, 440, 147, 10.0, 16384, 4, 4, 1e-5, 1.0, 23
DATA_SEED, PHILOX_SEED = 1, 2
FRACTION = 0.5 if "--stochastic" in sys.argv[1:] else 1.0
OUT = os.path.join(HERE, "multiclass_200k_p05_wbar23_sample.npz" if FRACTION < 1.0 else
                   "multiclass_200k_wbar23_sample.npz")
SAMPLE, SAMPLE_SEED = 32768, 0


def main():
    t0 = time.time()
    X, Y = synth.multiclass(n=N, d=DIN, m=M, seed=DATA_SEED)
    G, b = philox.rff_params(PHILOX_SEED, SIGMA, DIN, D, 0, D)
    Z = np.empty((N, D))
    for r0 in range(0, N, 5000):
        Z[r0:r0 + 5000] = rff.features(X[r0:r0 + 5000], G, b, D)
    print("Z %.0f s" % (time.time() - t0), flush=True)
    p = admm.Problem(X, Y, "squared", "l2", LAM, SIGMA, RHO, D, R, C, seed=PHILOX_SEED)
    p._Z = Z                       # the same matrix Problem.Z() would form, built in chunks
    W = admm.admm(p, ITERS, block_fraction=FRACTION)["Wbar"]
    idx = np.sort(np.random.default_rng(SAMPLE_SEED).choice(W.size, SAMPLE, replace=False)).astype(np.int64)
    # the objective sum_i V(y_i, (Z Wbar)_i) + n lambda r(Wbar) at the stored iterate
    np.savez(OUT, idx=idx, w=W.ravel()[idx], fro=np.linalg.norm(W), objective=p.objective(W))
    print("wrote %s (%.0f s)" % (OUT, time.time() - t0), flush=True)


if __name__ == "__main__":
    main()
