"""The large implicit workload (n = 8.1M, d = 784, D = 65,536, 32 x 16 blocks, one-vs-rest
hinge + l2, lambda = 1e-6) on its seeded 20,000-row sample, against the FP64 oracle's
iterate after 50 iterations (stored by tests/golden/make_large_sample_reference.py, which
calls only oracle/): at the full workload's 32 x 16 grid (625-row blocks: the outer form
I + Z_ij Z_ij^T) and at 2 x 16 (10,000-row blocks: the Gram form I + Z_ij^T Z_ij of the
full-size solve).  Weights and objective within 1e-4 relative on the split path and 1e-5
on the FP32 path."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
KW = dict(loss="hinge", reg="l2", lam=1e-6, sigma=9.0, rho=1.0, D=65536, seed=4, m=10)
TOL = {"split_bf16": 1e-4, "fp32": 1e-5}


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
    return synth.sparse01(n=20_000, d=784, m=10, seed=3)


@pytest.mark.parametrize("grid", [(32, 16), (2, 16)])
@pytest.mark.parametrize("prec", ["split_bf16", "fp32"])
def test_large_sample_matches_fp64_oracle(rff, data, grid, prec):
    R, C = grid
    ref = np.load(os.path.join(HERE, "golden", "large_20k_%dx%d_wbar50.npz" % grid))
    X, Y = data
    s = rff.Solver(prec=prec, R=R, C=C, **KW)
    s.set_data(X, Y)
    st = s.solve(50)
    W = s.weights().astype(np.float64).ravel()
    s.close()
    err = np.linalg.norm(W[ref["idx"]] - ref["w"]) / np.linalg.norm(ref["w"])
    obj_err = abs(st["objective"] - float(ref["objective"])) / abs(float(ref["objective"]))
    assert err < TOL[prec], (grid, prec, err)
    assert obj_err < TOL[prec], (grid, prec, obj_err)
    # the sample stands for the whole matrix: its norm scales with the sampled fraction
    frac = np.sqrt(ref["idx"].size / W.size)
    assert abs(np.linalg.norm(ref["w"]) / (float(ref["fro"]) * frac) - 1.0) < 0.1
