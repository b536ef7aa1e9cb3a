"""Allocation-free scoring (rff_admm_predict_noalloc) against rff_admm_predict.

For callers that cannot call cudaMalloc when they score (CUDA-graph capture,
serving loops that must not allocate on the request path), the library offers a
scoring entry point whose scratch is one fixed array in device memory.  Its
results must equal those of the ordinary entry point, call after call (the
shared array keeps the previous call's contents), and a batch too large for
the array must be refused with a clear error.  This file is collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import synth  # noqa: E402


@pytest.fixture(scope="module")
def rff():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1409_0940_gb300
    return paper_1409_0940_gb300


@pytest.mark.parametrize("prec", ["fp32", "split_bf16"])
def test_noalloc_scores_equal_predict_on_two_calls(rff, prec):
    X, Y = synth.multiclass(n=900, d=21, m=5, seed=4)
    s = rff.Solver(prec=prec, loss="hinge", reg="l2", lam=1e-3, sigma=3.0, D=384, R=2, C=3, seed=6, m=5)
    s.set_data(X, Y)
    s.solve(6, stats=False)
    rng = np.random.default_rng(7)
    for q in (300, 129):                      # two calls in a row, different batch sizes
        Xq = torch.from_numpy(rng.standard_normal((q, 21)).astype(np.float32)).cuda()
        ref = torch.empty((q, 5), dtype=torch.float32, device="cuda")
        got = torch.full((q, 5), float("nan"), dtype=torch.float32, device="cuda")
        rff.rff_admm_predict(s.h, Xq, ref)
        rff.rff_admm_predict_noalloc(s.h, Xq, got)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(g))
        # same kernels on the same inputs: the tolerance of the path is a loose upper bound
        assert np.abs(g - r).max() <= 1e-5 * max(1.0, np.abs(r).max())
    s.close()


def test_noalloc_refuses_batches_beyond_its_scratch(rff):
    X, Y = synth.ridge(n=300, d=440, seed=2)
    s = rff.Solver(loss="squared", lam=1e-3, sigma=10.0, D=256, seed=1, m=1)
    s.set_data(X, Y)
    s.solve(2, stats=False)
    q = 40_000                                 # 40k x (4 x 448 + 4 x 16) bytes > 32 MiB
    Xq = torch.zeros((q, 440), dtype=torch.float32, device="cuda")
    out = torch.empty((q, 1), dtype=torch.float32, device="cuda")
    with pytest.raises(rff.RffError) as e:
        rff.rff_admm_predict_noalloc(s.h, Xq, out)
    assert e.value.status == rff.RFF_EINVAL
    assert "smaller batches" in str(e.value)
    # a batch that fits still works after the refusal
    small = Xq[:1000].contiguous()
    out2 = torch.empty((1000, 1), dtype=torch.float32, device="cuda")
    rff.rff_admm_predict_noalloc(s.h, small, out2)
    ref = torch.empty((1000, 1), dtype=torch.float32, device="cuda")
    rff.rff_admm_predict(s.h, small, ref)
    assert torch.allclose(out2, ref, rtol=1e-5, atol=1e-6)
    s.close()
