"""Sparse (CSR) inputs (Sec. 4: sparse inputs enter only through T): the same iterates as the
dense rows they encode, malformed structures refused."""
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


def to_csr(X):
    rows, cols = np.nonzero(X)
    indptr = np.zeros(X.shape[0] + 1, dtype=np.int64)
    np.add.at(indptr, rows + 1, 1)
    return np.cumsum(indptr).astype(np.int64), cols.astype(np.int32), X[rows, cols].astype(np.float32)


@pytest.mark.parametrize("prec", ["split_bf16", "fp32", "cached_z"])
@pytest.mark.parametrize("device", [False, True])
def test_csr_equals_dense(rff, prec, device):
    X, Y = synth.sparse01(n=900, d=60, m=4, seed=2)
    assert (X == 0).mean() > 0.5
    indptr, indices, values = to_csr(X)
    kw = dict(prec=prec, loss="hinge", reg="l2", lam=1e-3, sigma=3.0, D=384, R=2, C=2, seed=5, m=4)
    a, b = rff.Solver(**kw), rff.Solver(**kw)
    a.set_data(X, Y)
    if device:
        b.set_data_csr(*(torch.from_numpy(v).cuda() for v in (indptr, indices, values, Y)), d=60)
    else:
        b.set_data_csr(indptr, indices, values, Y, d=60)
    a.solve(8, stats=False)
    b.solve(8, stats=False)
    assert np.array_equal(a.weights(), b.weights())
    a.close()
    b.close()


def test_repeated_columns_add_up(rff):
    X, Y = synth.sparse01(n=300, d=20, m=2, seed=3)
    indptr, indices, values = to_csr(X)
    # split every entry in two halves stored as two entries of the same column
    rows = np.repeat(np.arange(300), np.diff(indptr))
    order = np.argsort(np.concatenate([rows, rows]), kind="stable")
    ind2 = np.concatenate([indices, indices])[order]
    val2 = np.concatenate([values * 0.5, values * 0.5])[order].astype(np.float32)
    ptr2 = indptr * 2
    kw = dict(prec="fp32", loss="squared", reg="l2", lam=1e-3, sigma=2.0, D=128, R=1, C=1, seed=1, m=2)
    a, b = rff.Solver(**kw), rff.Solver(**kw)
    a.set_data(X, Y)
    b.set_data_csr(ptr2, ind2, val2, Y, d=20)
    a.solve(5, stats=False)
    b.solve(5, stats=False)
    assert np.array_equal(a.weights(), b.weights())
    a.close()
    b.close()


def test_malformed_structures_are_refused(rff):
    X, Y = synth.sparse01(n=50, d=10, m=2, seed=4)
    indptr, indices, values = to_csr(X)
    s = rff.Solver(prec="fp32", loss="squared", reg="l2", lam=1e-3, sigma=2.0, D=64, seed=1, m=2)
    bad_col = indices.copy()
    bad_col[3] = 10
    bad_ptr = indptr.copy()
    bad_ptr[7], bad_ptr[8] = bad_ptr[8], bad_ptr[7] - 1
    short = indptr.copy()
    short[-1] -= 1
    nan = values.copy()
    nan[0] = np.nan
    for args in [(indptr, bad_col, values), (bad_ptr, indices, values), (short, indices, values),
                 (indptr, indices, nan)]:
        with pytest.raises(rff.RffError):
            s.set_data_csr(*args, Y, d=10)
    s.set_data_csr(indptr, indices, values, Y, d=10)
    s.close()
