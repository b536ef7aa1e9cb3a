"""Allocation-free scoring (rff_admm_predict_noalloc) against rff_admm_predict.

Some callers cannot call cudaMalloc when they score: a serving loop whose device
memory is handed out entirely by another allocator's pool, or one that must not take
the device-wide synchronisation of an allocation in the middle of a request.  The
library offers them a scoring entry point whose scratch is one fixed array in device
memory.  Its results must equal those of the ordinary entry point bit for bit, call
after call (the shared array keeps the previous call's contents), it must leave the
device's free memory and torch's allocator where they were, and a batch too large for
the array must be refused with a clear error.  This file is collected last, and each
test also passes alone in a fresh process.
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


def _memory():
    torch.cuda.synchronize()
    free, _ = torch.cuda.mem_get_info()
    return free, torch.cuda.memory_allocated(), torch.cuda.memory_reserved()


@pytest.mark.parametrize("prec", ["fp32", "split_bf16"])
def test_noalloc_scores_equal_predict_on_consecutive_calls(rff, prec):
    X, Y = synth.multiclass(n=900, d=21, m=5, seed=4)
    s = rff.Solver(prec=prec, loss="hinge", reg="l2", lam=1e-3, sigma=3.0, D=384, R=2, C=3, seed=6, m=5)
    s.set_data(X, Y)
    s.solve(6, stats=False)
    rng = np.random.default_rng(7)
    # one batch per call, shrinking, so later calls find the larger earlier batches' rows
    # still in the shared array; the first call on the device also looks up its address
    batches = [torch.from_numpy(rng.standard_normal((q, 21)).astype(np.float32)).cuda() for q in (300, 129, 5)]
    refs = [torch.empty((b.shape[0], 5), dtype=torch.float32, device="cuda") for b in batches]
    outs = [torch.full((b.shape[0], 5), float("nan"), dtype=torch.float32, device="cuda") for b in batches]
    for b, r in zip(batches, refs):
        rff.rff_admm_predict(s.h, b, r)
    for k, (b, o) in enumerate(zip(batches, outs)):
        before = _memory()
        rff.rff_admm_predict_noalloc(s.h, b, o)
        after = _memory()
        if k > 0:
            # no device allocation: free memory does not fall (a stream-ordered pool of
            # another caller may give memory back meanwhile, so it may rise) and torch's
            # allocator is untouched
            assert after[0] >= before[0], (before, after)
            assert after[1:] == before[1:], (before, after)
    for r, o in zip(refs, outs):
        # same kernels on the same padded layout: bit for bit
        assert np.array_equal(o.cpu().numpy(), r.cpu().numpy())
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
    # a batch that fits still works after the refusal, twice
    for q2 in (1000, 1000):
        small = Xq[:q2].contiguous()
        out2 = torch.empty((q2, 1), dtype=torch.float32, device="cuda")
        rff.rff_admm_predict_noalloc(s.h, small, out2)
        ref = torch.empty((q2, 1), dtype=torch.float32, device="cuda")
        rff.rff_admm_predict(s.h, small, ref)
        assert torch.equal(out2, ref)
    s.close()
