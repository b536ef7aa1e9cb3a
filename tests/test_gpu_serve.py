"""Serving loop: admission by memory budget, requests overlapping on the device, and
every result equal to the same request served alone."""
import time

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


def _requests():
    """A seeded mix of solves of different sizes, losses, regularisers and paths."""
    out = []
    specs = [("squared", "l2", "split_bf16", 3000, 20, 1, 512, 2, 2),
             ("hinge", "l2", "fp32", 2500, 33, 4, 384, 1, 3),
             ("logistic", "l1", "split_bf16", 4000, 12, 1, 1024, 2, 4),
             ("hinge", "l1", "split_bf16", 1800, 64, 3, 256, 3, 1),
             ("squared", "l2", "fp32", 1200, 7, 2, 128, 1, 1)]
    for k, (loss, reg, prec, n, d, m, D, R, C) in enumerate(specs):
        if loss == "squared":
            X, y = synth.ridge(n=n, d=d, seed=k)
            Y = np.ascontiguousarray(np.repeat(y, m, axis=1))
        elif m == 1:
            X, Y = synth.binary(n=n, d=d, seed=k)
        else:
            X, Y = synth.multiclass(n=n, d=d, m=m, seed=k)
        out.append((dict(loss=loss, reg=reg, prec=prec, lam=1e-3, sigma=3.0, D=D, R=R, C=C, seed=k, m=m), X, Y))
    return out


def _wait_all(rff, srv, ids, timeout=300):
    got = {}
    t0 = time.time()
    while len(got) < len(ids) and time.time() - t0 < timeout:
        for c in rff.rff_server_poll(srv, 64, 200):
            got[c["id"]] = c
    assert len(got) == len(ids), "requests did not complete"
    return got


def test_results_equal_alone_and_in_the_mix(rff):
    reqs = _requests()
    rng = np.random.default_rng(0)
    queries = [rng.standard_normal((int(q), X.shape[1])).astype(np.float32) for q, (_, X, _) in
               zip([1, 4096, 77, 300, 129], reqs)]
    # alone: one request at a time through the solver API
    alone_w, alone_s = [], []
    for (kw, X, Y), Xq in zip(reqs, queries):
        s = rff.Solver(**kw)
        s.set_data(X, Y)
        s.solve(12, stats=False)
        alone_w.append(s.weights())
        alone_s.append(s.predict(Xq))
        s.close()
    # in the mix: everything submitted at once to a server running 4 requests at a time
    srv = rff.rff_server_create(0, 4)
    ids, scores = [], []
    for (kw, X, Y) in reqs:
        ids.append(rff.rff_server_submit_solve(srv, rff.make_params(**kw), X, Y, 12))
    sids = []
    for mid, Xq, (kw, _, _) in zip(ids, queries, reqs):
        out = np.full((Xq.shape[0], kw["m"]), np.nan, dtype=np.float32)
        scores.append(out)
        sids.append(rff.rff_server_submit_score(srv, mid, Xq, out))
    got = _wait_all(rff, srv, ids + sids)
    assert all(c["status"] == rff.RFF_OK for c in got.values()), got
    for k, (mid, (kw, X, Y)) in enumerate(zip(ids, reqs)):
        W = np.empty((kw["D"], kw["m"]), dtype=np.float32)
        rff.rff_server_get_weights(srv, mid, W)
        assert np.array_equal(W, alone_w[k]), k
        assert np.array_equal(scores[k], alone_s[k]), k
    for c in got.values():
        assert c["latency_ms"] >= c["run_ms"] >= 0 and c["queue_ms"] >= 0
    rff.rff_server_destroy(srv)


def test_admission_keeps_within_budget(rff):
    reqs = _requests()[:3]
    peaks = [rff.rff_admm_estimate_bytes(rff.make_params(**kw), X.shape[0], X.shape[1])[1] for kw, X, _ in reqs]
    budget = int(max(peaks) * 1.2)              # one solve at a time fits
    srv = rff.rff_server_create(budget, 3)
    ids = [rff.rff_server_submit_solve(srv, rff.make_params(**kw), X, Y, 8) for kw, X, Y in reqs]
    seen = 0
    t0 = time.time()
    got = {}
    while len(got) < len(ids) and time.time() - t0 < 300:
        used, b = rff.rff_server_memory(srv)
        assert used <= b == budget
        seen = max(seen, used)
        for c in rff.rff_server_poll(srv, 16, 50):
            got[c["id"]] = c
        # release finished models so the next solve can be admitted
        for i in ids:
            if i in got and got[i].get("released") is None:
                rff.rff_server_release(srv, i)
                got[i]["released"] = True
    assert len(got) == len(ids) and all(c["status"] == rff.RFF_OK for c in got.values())
    assert 0 < seen <= budget
    rff.rff_server_destroy(srv)


def test_refusals(rff):
    srv = rff.rff_server_create(64 << 20, 2)         # 64 MiB
    X, Y = synth.multiclass(n=20000, d=100, m=10, seed=1)
    with pytest.raises(rff.RffError) as e:
        rff.rff_server_submit_solve(srv, rff.make_params(loss="squared", D=8192, R=2, C=2, m=10), X, Y, 5)
    assert e.value.status == rff.RFF_ENOMEM
    with pytest.raises(rff.RffError):
        rff.rff_server_submit_score(srv, 12345, X[:3], np.empty((3, 10), np.float32))
    rff.rff_server_destroy(srv)


def test_cancel_queued_request(rff):
    """With one worker busy on a long solve, a queued solve and the score waiting for it can be
    cancelled: the solve completes at once with RFF_ECANCELLED, the score then fails, and the
    running solve cannot be cancelled and finishes normally."""
    srv = rff.rff_server_create(0, 1)
    XA, YA = synth.multiclass(n=20000, d=32, m=3, seed=3)
    XB, YB = synth.binary(n=2000, d=16, seed=4)
    a = rff.rff_server_submit_solve(srv, rff.make_params(loss="hinge", prec="fp32", D=4096, R=2, C=2, m=3,
                                                         sigma=3.0, lam=1e-3), XA, YA, 300)
    b = rff.rff_server_submit_solve(srv, rff.make_params(loss="hinge", D=256, R=1, C=1, m=1, sigma=3.0,
                                                         lam=1e-3), XB, YB, 5)
    out = np.full((7, 1), np.nan, dtype=np.float32)
    sc = rff.rff_server_submit_score(srv, b, XB[:7], out)
    assert rff.rff_server_cancel(srv, b)
    assert not rff.rff_server_cancel(srv, b)          # already completed (cancelled)
    with pytest.raises(rff.RffError) as e:
        rff.rff_server_cancel(srv, 10 ** 9)
    assert e.value.status == rff.RFF_EINVAL
    got = _wait_all(rff, srv, [a, b, sc])
    assert got[b]["status"] == rff.RFF_ECANCELLED
    assert got[sc]["status"] == rff.RFF_EINVAL and np.isnan(out).all()
    assert got[a]["status"] == rff.RFF_OK
    assert not rff.rff_server_cancel(srv, a)          # done
    with pytest.raises(rff.RffError):
        rff.rff_server_get_weights(srv, b, np.empty((256, 1), np.float32))
    rff.rff_server_destroy(srv)
