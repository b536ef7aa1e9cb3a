"""The three precisions at the full multiclass workload (n = 200,000, d = 440, m = 147,
D = 16,384, 4 x 4 blocks, squared loss + l2, lambda = 1e-5) against the FP64 oracle's
iterate after 23 iterations, stored as a seeded sample of Wbar by
tests/golden/make_multiclass_reference.py (calls only oracle/).

Tolerances: 1e-5 relative for the FP32 path, 1e-4 for the split and cached-Z paths, on the
weights (the stored sample) and on the objective.  Measured: FP32 path 3.0e-6 (its pass-1
sums in chains of at most ~1,600 rows and a compensated projection; 5.3e-5 with whole-block
FP32 sums), split and cached-Z paths 4.5e-5.  The tensor-core paths reach it with the
separate accumulator of the projection's dominant products (without it they were at 2.2e-4
to 2.9e-4); their Gram matrices on the tensor cores (512-row pieces, a separate accumulator
for the dominant products) left it at 4.5e-5.  The stochastic variant (block fraction 0.5):
7.4e-5 on both tensor-core paths."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import synth  # noqa: E402

REF = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "multiclass_200k_wbar23_sample.npz")
KW = dict(loss="squared", reg="l2", lam=1e-5, sigma=10.0, rho=1.0, D=16384, R=4, C=4, seed=2, m=147)


@pytest.fixture(scope="module")
def rff():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1409_0940_gb300
    return paper_1409_0940_gb300


@pytest.fixture(scope="module")
def data():
    return synth.multiclass(n=200_000, d=440, m=147, seed=1)


TOL = {"split_bf16": 1e-4, "cached_z": 1e-4, "fp32": 1e-5}


@pytest.mark.parametrize("prec", ["split_bf16", "cached_z", "fp32"])
def test_full_workload_matches_fp64_oracle(rff, data, prec):
    ref = np.load(REF)
    X, Y = data
    s = rff.Solver(prec=prec, **KW)
    s.set_data(X, Y)
    st = s.solve(23)
    W = s.weights().astype(np.float64).ravel()
    s.close()
    err = np.linalg.norm(W[ref["idx"]] - ref["w"]) / np.linalg.norm(ref["w"])
    assert err < TOL[prec], (prec, err)
    obj = float(ref["objective"])
    assert abs(st["objective"] - obj) / abs(obj) < TOL[prec], (prec, st["objective"], obj)
    # the sample stands for the whole matrix: its norm scales with the sampled fraction
    frac = np.sqrt(ref["idx"].size / W.size)
    assert abs(np.linalg.norm(ref["w"]) / (float(ref["fro"]) * frac) - 1.0) < 0.1


REF_P05 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "multiclass_200k_p05_wbar23_sample.npz")


@pytest.mark.parametrize("prec", ["split_bf16", "cached_z"])
def test_full_workload_stochastic_matches_fp64_oracle(rff, data, prec):
    """The stochastic block-subset variant (half of the 16 blocks active per iteration) at the
    full size, against the oracle's stochastic iterate (make_multiclass_reference.py
    --stochastic): the same Philox masks on both sides."""
    ref = np.load(REF_P05)
    X, Y = data
    s = rff.Solver(prec=prec, **KW)
    s.set_block_fraction(0.5)
    s.set_data(X, Y)
    s.solve(23, stats=False)
    W = s.weights().astype(np.float64).ravel()
    s.close()
    err = np.linalg.norm(W[ref["idx"]] - ref["w"]) / np.linalg.norm(ref["w"])
    assert err < 1e-4, (prec, err)
    # and it is a different iterate from the full method's
    full = np.load(REF)
    assert np.linalg.norm(ref["w"] - full["w"]) / np.linalg.norm(full["w"]) > 1e-2
