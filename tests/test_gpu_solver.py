"""GPU parity of the whole solver (C ABI) against the FP64 oracle, iterate for iterate."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import admm  # noqa: E402

PRECS = {"fp32": 1e-5, "split_bf16": 1e-4, "cached_z": 1e-4}   # relative weight / objective tolerance per path


@pytest.fixture(scope="module")
def rff():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1409_0940_gb300
    return paper_1409_0940_gb300


def run_gpu(rff, X, Y, iters, prec, **kw):
    s = rff.Solver(prec=prec, **kw)
    s.set_data(X, Y)
    st = s.solve(iters)
    W = s.weights()
    return s, st, W


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def ridge_ref():
    """The n=2000, d=16, D=512 ridge workload: oracle iterates and the closed form."""
    X, Y = synth.ridge(seed=1)
    p = admm.Problem(X, Y, "squared", "l2", 1e-4, 4.0, 1.0, 512, 1, 1, 2)
    out = admm.admm(p, 200, history=True)
    return X, Y, p, out, admm.ridge_closed_form(p.Z(), p.Y, p.lam)


@pytest.mark.parametrize("prec", list(PRECS))
def test_ridge_1x1_matches_oracle_and_closed_form(rff, ridge_ref, prec):
    X, Y, p, out, Wcf = ridge_ref
    s, st, W = run_gpu(rff, X, Y, 200, prec, loss="squared", reg="l2", lam=1e-4, sigma=4.0, rho=1.0, D=512,
                       R=1, C=1, seed=2, m=1)
    tol = PRECS[prec]
    assert rel(W, out["Wbar"]) < tol
    assert rel(W, Wcf) < tol
    assert abs(st["objective"] - p.objective(out["Wbar"])) < tol * abs(p.objective(out["Wbar"]))
    # predictions on fresh points
    Xq = np.random.default_rng(5).random((333, 16)).astype(np.float32)
    got = s.predict(Xq)
    ref = p.predict(Xq, out["Wbar"])
    assert np.abs(got - ref).max() < tol * np.abs(ref).max()
    s.close()


GRIDS = [
    # (loss, reg, n, d, m, D, R, C, iters, lam, rho, sigma)
    ("squared", "l2", 777, 13, 1, 300, 3, 2, 30, 1e-3, 1.0, 2.0),
    ("squared", "l1", 640, 9, 2, 256, 2, 2, 25, 1e-4, 1.0, 2.0),
    ("hinge", "l2", 900, 11, 5, 384, 2, 3, 25, 1e-3, 1.0, 3.0),
    ("hinge", "l2", 500, 7, 1, 200, 1, 2, 25, 1e-3, 0.5, 2.0),
    ("logistic", "l2", 600, 8, 1, 256, 2, 1, 25, 1e-3, 1.0, 2.5),
    ("multinomial", "l2", 700, 10, 4, 320, 2, 2, 25, 1e-3, 1.0, 3.0),
    ("l1", "l2", 640, 9, 2, 256, 2, 2, 25, 1e-4, 1.0, 2.0),
    ("crammer_singer", "l2", 700, 10, 6, 320, 2, 2, 25, 1e-3, 1.0, 3.0),
    ("crammer_singer", "l1", 600, 12, 147, 384, 2, 2, 15, 1e-4, 1.0, 3.0),
    # wide outputs: unequal column blocks (301 + 300 features, three 128-row tiles with a
    # ragged last one) and the widest output block the tensor-core passes take (m_pad = 256)
    ("squared", "l2", 900, 12, 150, 601, 2, 2, 20, 1e-3, 1.0, 3.0),
    ("squared", "l1", 500, 8, 250, 384, 1, 2, 15, 1e-3, 1.0, 2.0),
    # fewer rows than features in every block: the outer form (I + Z Z^T)^-1 of the projection,
    # with ragged row blocks (167/167/166) and a multinomial loss
    ("hinge", "l2", 500, 7, 3, 2048, 2, 2, 20, 1e-3, 1.0, 3.0),
    ("logistic", "l1", 500, 12, 1, 1536, 3, 1, 20, 1e-3, 1.0, 2.5),
    ("multinomial", "l2", 400, 9, 4, 1200, 2, 2, 15, 1e-3, 1.0, 3.0),
    ("crammer_singer", "l2", 400, 9, 5, 1200, 2, 2, 15, 1e-3, 1.0, 3.0),
    ("l1", "l2", 500, 8, 3, 1536, 3, 1, 15, 1e-4, 1.0, 2.0),
]


def _data(loss, n, d, m, seed):
    if loss in ("squared", "l1"):
        X, y = synth.ridge(n=n, d=d, seed=seed)
        Y = np.repeat(y, m, axis=1) * np.linspace(1, 0.5, m, dtype=np.float32)[None]
        return X, np.ascontiguousarray(Y, dtype=np.float32)
    if m == 1:
        return synth.binary(n=n, d=d, seed=seed)
    return synth.multiclass(n=n, d=d, m=m, seed=seed)


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("case", GRIDS, ids=lambda c: "%s-%s-%dx%d-m%d" % (c[0], c[1], c[6], c[7], c[4]))
def test_grids_and_losses_match_oracle(rff, prec, case):
    loss, reg, n, d, m, D, R, C, iters, lam, rho, sigma = case
    X, Y = _data(loss, n, d, m, seed=n + m)
    p = admm.Problem(X, Y, loss, reg, lam, sigma, rho, D, R, C, seed=31)
    out = admm.admm(p, iters, history=True)
    s, st, W = run_gpu(rff, X, Y, iters, prec, loss=loss, reg=reg, lam=lam, sigma=sigma, rho=rho, D=D, R=R, C=C,
                       seed=31, m=m)
    tol = PRECS[prec]
    assert rel(W, out["Wbar"]) < tol, rel(W, out["Wbar"])
    f_ref = p.objective(out["Wbar"])
    assert abs(st["objective"] - f_ref) < tol * abs(f_ref)
    pr, du = out["history"][-1]
    assert abs(st["primal_res"] - pr) < 1e-2 * pr + 1e-6
    assert abs(st["dual_res"] - du) < 1e-2 * du + 1e-6
    s.close()


def test_resume_from_checkpoint_is_bit_identical(rff):
    X, Y = synth.multiclass(n=500, d=6, m=3, seed=2)
    kw = dict(loss="hinge", reg="l2", lam=1e-3, sigma=2.0, rho=1.0, D=256, R=2, C=2, seed=4, m=3)
    a = rff.Solver(**kw)
    a.set_data(X, Y)
    a.solve(12, stats=False)
    Wa = a.weights()
    b = rff.Solver(**kw)
    b.set_data(X, Y)
    b.solve(5, stats=False)
    state = b.get_state()
    b.close()
    c = rff.Solver(**kw)
    c.set_data(X, Y)
    c.set_state(state)
    c.solve(7, stats=False)
    assert np.array_equal(c.weights(), Wa)
    a.close()
    c.close()


def test_runs_are_deterministic(rff):
    X, Y = synth.ridge(n=400, d=5, seed=9)
    kw = dict(loss="squared", reg="l2", lam=1e-3, sigma=1.0, D=200, R=2, C=2, seed=1, m=1)
    Ws = []
    for _ in range(2):
        s = rff.Solver(**kw)
        s.set_data(X, Y)
        s.solve(10, stats=False)
        Ws.append(s.weights())
        s.close()
    assert np.array_equal(Ws[0], Ws[1])


def test_invalid_inputs_are_rejected(rff):
    X, Y = synth.binary(n=100, d=4, seed=1)
    s = rff.Solver(loss="hinge", D=64, m=1)
    with pytest.raises(rff.RffError) as e:
        s.predict(X[:3])
    assert e.value.status == rff.RFF_ENOTREADY
    bad = X.copy()
    bad[3, 2] = np.nan
    with pytest.raises(rff.RffError) as e:
        s.set_data(bad, Y)
    assert e.value.status == rff.RFF_EINVAL
    with pytest.raises(rff.RffError) as e:
        s.set_data(X, Y * 0.5)          # hinge targets must be +-1
    assert e.value.status == rff.RFF_EINVAL
    s.set_data(X, Y)
    s.solve(2, stats=False)
    q = X[:5].copy()
    q[0, 0] = np.inf
    with pytest.raises(rff.RffError):
        s.predict(q)
    assert s.predict(X[:0]).shape == (0, 1)
    s.close()


def test_device_pointers_match_host_pointers(rff):
    X, Y = synth.ridge(n=300, d=4, seed=3)
    kw = dict(loss="squared", lam=1e-3, sigma=1.0, D=128, R=1, C=2, seed=8, m=1)
    a = rff.Solver(**kw)
    a.set_data(X, Y)
    a.solve(5, stats=False)
    b = rff.Solver(**kw)
    b.set_data(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda())
    b.solve(5, stats=False)
    out = torch.empty((128, 1), dtype=torch.float32, device="cuda")
    b.weights(out)
    assert np.array_equal(out.cpu().numpy(), a.weights())
    sq = torch.empty((50, 1), dtype=torch.float32, device="cuda")
    b.predict(torch.from_numpy(X[:50]).cuda(), sq)
    assert np.array_equal(sq.cpu().numpy(), a.predict(X[:50]))
    a.close()
    b.close()


@pytest.mark.parametrize("prec", ["split_bf16", "cached_z"])
def test_split_path_query_range(rff, prec):
    """The split path scales X into the FP16 range from the training data: queries up to 128x the
    largest training |x| score (and agree with the FP32 path's features to the split precision);
    larger ones are refused instead of overflowing.  The FP32 path takes any finite query."""
    X, y = synth.ridge(n=600, d=7, seed=4)
    xmax = float(np.abs(X).max())
    kw = dict(loss="squared", reg="l2", lam=1e-3, sigma=50.0, D=256, R=1, C=2, seed=5, m=1)
    s = rff.Solver(prec=prec, **kw)
    s.set_data(X, y)
    s.solve(5, stats=False)
    f = rff.Solver(prec="fp32", **kw)
    f.set_data(X, y)
    f.solve(5, stats=False)
    big = (X[:40] / xmax * 100.0 * xmax).astype(np.float32)
    a, b = s.predict(big), f.predict(big)
    assert np.isfinite(a).all()
    assert np.abs(a - b).max() < 1e-3 * max(np.abs(b).max(), 1e-6)
    with pytest.raises(rff.RffError) as e:
        s.predict((X[:4] * 1000.0).astype(np.float32))
    assert e.value.status == rff.RFF_EINVAL
    assert np.isfinite(f.predict((X[:4] * 1000.0).astype(np.float32))).all()
    s.close()
    f.close()


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("shape", ["gram", "outer", "stochastic"])
def test_solve_in_pieces_with_statistics_is_one_solve(rff, prec, shape):
    """The statistics a solve call reports (residuals, the objective's scoring pass) leave the
    iterates alone: 10 iterations in calls of 3, 3 and 4 are those of one call, bit for bit,
    in the Gram form, in the outer form (whose O'_ij carries over from one iteration to the
    next) and in a stochastic solve (whose inactive blocks keep O'_ij)."""
    if prec == "cached_z" and shape == "outer":
        pytest.skip("the cached-Z precision takes the Gram form only")
    X, Y = synth.multiclass(n=640, d=9, m=3, seed=6)
    D = 2048 if shape == "outer" else 256
    kw = dict(prec=prec, loss="hinge", reg="l2", lam=1e-3, sigma=2.0, D=D, R=2, C=2, seed=1, m=3)
    a = rff.Solver(**kw)
    b = rff.Solver(**kw)
    for s in (a, b):
        s.set_data(X, Y)
        if shape == "stochastic":
            s.set_block_fraction(0.5)
    a.solve(10)
    for k in (3, 3, 4):
        b.solve(k)
    assert np.array_equal(a.weights(), b.weights())
    a.close()
    b.close()


def test_set_stream_mid_solve_keeps_results(rff):
    X, Y = synth.multiclass(n=700, d=9, m=3, seed=6)
    kw = dict(prec="split_bf16", loss="hinge", reg="l2", lam=1e-3, sigma=2.0, D=256, R=2, C=2, seed=1, m=3)
    a = rff.Solver(**kw)
    a.set_data(X, Y)
    a.solve(10, stats=False)
    b = rff.Solver(**kw)
    b.set_data(X, Y)
    b.solve(4, stats=False)
    hp = torch.cuda.Stream(priority=-1)
    rff.rff_admm_set_stream(b.h, hp)
    b.solve(6, stats=False)
    assert np.array_equal(a.weights(), b.weights())
    assert np.array_equal(a.predict(X[:50]), b.predict(X[:50]))
    a.close()
    b.close()


@pytest.fixture(scope="module")
def config3_shape():
    """The large implicit workload's shape at a size the oracle runs in seconds: d = 784 sparse
    inputs in [0, 1], 10-class one-vs-rest hinge + l2, sigma = 9, 4 x 8 blocks of 500 rows x
    1024 features (every block takes the outer form, as the 20k-row subsample of the
    8.1M-row workload does at 32 x 16).  The oracle runs once for both paths."""
    X, Y = synth.sparse01(n=2000, d=784, m=10, seed=3)
    kw = dict(loss="hinge", reg="l2", lam=1e-6, sigma=9.0, rho=1.0, D=8192, R=4, C=8)
    p = admm.Problem(X, Y, kw["loss"], kw["reg"], kw["lam"], kw["sigma"], kw["rho"], kw["D"], kw["R"], kw["C"], seed=7)
    out = admm.admm(p, 10)
    return X, Y, kw, out["Wbar"], p


@pytest.mark.parametrize("prec", ["fp32", "split_bf16"])
def test_outer_form_config3_shape(rff, config3_shape, prec):
    X, Y, kw, W_ref, p = config3_shape
    s, st, W = run_gpu(rff, X, Y, 10, prec, seed=7, m=10, **kw)
    assert rel(W, W_ref) < PRECS[prec], rel(W, W_ref)
    # the reported objective against the oracle's at the GPU's own weights and at the oracle's
    f_at_W = p.objective(np.asarray(W, np.float64))
    assert abs(st["objective"] - f_at_W) < PRECS[prec] * abs(f_at_W)
    f_ref = p.objective(W_ref)
    assert abs(st["objective"] - f_ref) < PRECS[prec] * abs(f_ref), abs(st["objective"] - f_ref) / abs(f_ref)
    s.close()


@pytest.mark.parametrize("prec", ["split_bf16", "fp32"])
def test_predict_labels(rff, prec):
    """Labels decide on the GPU's own float32 scores: argmax with the lowest index among equal
    scores (numpy's argmax returns the first maximum), or the sign for one output."""
    X, Y = synth.multiclass(n=800, d=9, m=5, seed=6)
    s = rff.Solver(prec=prec, loss="hinge", reg="l2", lam=1e-3, sigma=3.0, D=256, R=2, C=2, seed=4, m=5)
    s.set_data(X, Y)
    s.solve(10, stats=False)
    Xq = np.random.default_rng(1).standard_normal((333, 9)).astype(np.float32)
    scores = s.predict(Xq)
    assert np.array_equal(s.predict_labels(Xq), np.argmax(scores, axis=1).astype(np.int32))
    out = torch.zeros(333, dtype=torch.int32, device="cuda")
    s.predict_labels(torch.from_numpy(Xq).cuda(), out)
    assert np.array_equal(out.cpu().numpy(), np.argmax(scores, axis=1))
    s.close()
    Xb, yb = synth.binary(n=600, d=7, seed=2)
    b = rff.Solver(prec=prec, loss="logistic", reg="l2", lam=1e-3, sigma=2.0, D=128, R=1, C=1, seed=1, m=1)
    b.set_data(Xb, yb)
    b.solve(8, stats=False)
    sb = b.predict(Xb[:100])[:, 0]
    assert np.array_equal(b.predict_labels(Xb[:100]), np.where(sb >= 0, 1, -1).astype(np.int32))
    b.close()


@pytest.mark.parametrize("prec", list(PRECS))
@pytest.mark.parametrize("shape", [
    # (n, d, m, D, R, C): one row per row block, one feature per column block, d = 1
    (3, 1, 1, 2, 3, 2),
    # a single feature, a single input dimension, many rows
    (300, 1, 2, 1, 2, 1),
    # blocks of 129 rows and 129 features: one full 128-slot tile plus one live row/feature
    (258, 5, 3, 258, 2, 2),
])
def test_degenerate_shapes_match_oracle(rff, prec, shape):
    n, d, m, D, R, C = shape
    if prec == "cached_z" and D // C > n // R:
        pytest.skip("the cached-Z precision takes the Gram form only")
    rng = np.random.default_rng(n + D)
    X = rng.random((n, d)).astype(np.float32)
    Y = rng.standard_normal((n, m)).astype(np.float32)
    p = admm.Problem(X, Y, "squared", "l2", 1e-3, 1.5, 1.0, D, R, C, seed=13)
    out = admm.admm(p, 12)
    s, st, W = run_gpu(rff, X, Y, 12, prec, loss="squared", reg="l2", lam=1e-3, sigma=1.5, rho=1.0, D=D, R=R, C=C,
                       seed=13, m=m)
    assert rel(W, out["Wbar"]) < PRECS[prec], rel(W, out["Wbar"])
    s.close()
