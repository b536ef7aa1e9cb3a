"""Small solves on every path of the library, run in a process of its own by
test_gpu_checked_build.py: once with the ordinary library and once with the bounds-checked
build (environment RFF_ADMM_CHECK=1).  Writes the weights and scores of every case, and the
bounds-check report, to the .npz file named on the command line."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import paper_1409_0940_gb300 as rff  # noqa: E402
import synth  # noqa: E402

# (name, solver keywords, data, rows, block fraction, CSR input)
CASES = [
    ("fp32_gram", dict(prec="fp32", loss="squared", D=384, R=3, C=2, m=1), "ridge", 900, 1.0, False),
    ("fp32_outer", dict(prec="fp32", loss="hinge", D=2048, R=2, C=2, m=3), "multiclass", 500, 1.0, False),
    ("split_gram", dict(prec="split_bf16", loss="multinomial", D=1024, R=2, C=2, m=3), "multiclass", 3000, 1.0,
     False),
    ("split_outer", dict(prec="split_bf16", loss="logistic", D=2048, R=2, C=1, m=1), "binary", 600, 1.0, False),
    ("cached_z", dict(prec="cached_z", loss="hinge", D=512, R=2, C=2, m=1), "binary", 4000, 1.0, False),
    ("split_stochastic", dict(prec="split_bf16", loss="crammer_singer", D=768, R=3, C=3, m=4), "multiclass", 2500,
     0.5, False),
    ("fp32_csr", dict(prec="fp32", loss="l1", D=256, R=2, C=2, m=2), "sparse", 700, 1.0, True),
    ("fastfood_split", dict(prec="split_bf16", loss="squared", D=512, R=2, C=2, m=1, feature_map="fastfood"),
     "ridge", 1500, 1.0, False),
    ("tensorsketch_cz", dict(prec="cached_z", loss="hinge", D=640, R=2, C=3, m=1, feature_map="tensorsketch"),
     "binary", 2000, 1.0, False),
]


def data(kind, n, m, seed):
    if kind == "ridge":
        X, y = synth.ridge(n=n, d=24, seed=seed)
        return X, np.ascontiguousarray(np.repeat(y, m, axis=1))
    if kind == "binary":
        return synth.binary(n=n, d=31, seed=seed)
    if kind == "sparse":
        return synth.sparse01(n=n, d=50, m=m, seed=seed)
    return synth.multiclass(n=n, d=40, m=m, seed=seed)


def to_csr(X):
    rows, cols = np.nonzero(X)
    indptr = np.zeros(X.shape[0] + 1, dtype=np.int64)
    np.add.at(indptr, rows + 1, 1)
    return np.cumsum(indptr).astype(np.int64), cols.astype(np.int32), X[rows, cols].astype(np.float32)


def main(path):
    out = {"enabled": np.array(rff.rff_check_enabled())}
    rff.rff_check_report()   # start from a clear record
    for k, (name, kw, kind, n, frac, csr) in enumerate(CASES):
        X, Y = data(kind, n, kw["m"], seed=k)
        s = rff.Solver(reg="l2", lam=1e-3, sigma=3.0, seed=k + 1, **kw)
        if csr:
            s.set_data_csr(*to_csr(X), Y, d=X.shape[1])
        else:
            s.set_data(X, Y)
        if frac < 1.0:
            s.set_block_fraction(frac)
        s.solve(10, stats=False)
        out[name + "_W"] = s.weights()
        Xq = np.random.default_rng(k).standard_normal((257, X.shape[1])).astype(np.float32)
        out[name + "_S"] = s.predict(np.abs(Xq) if kind == "sparse" else Xq)
        s.close()
    rep = rff.rff_check_report()
    out["report"] = np.array([rep[k] for k in ("count", "unit", "line", "index", "bound")], dtype=np.int64)
    np.savez(path, **out)


if __name__ == "__main__":
    main(sys.argv[1])
