"""Pins for the oracle's Philox4x32-10 stream and the RFF parameters drawn from it."""
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(w, 16) for w in line.split()])
    return rows


def test_known_answer_vectors():
    rows = _kat_rows()
    assert len(rows) == 3
    for r in rows:
        out = philox.philox4x32_10(r[0], r[1], r[2], r[3], r[4], r[5])
        assert [int(x) for x in out] == r[6:10]


_TRITON_PROBE = r"""
import os, sys
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def _k(out_ptr, seed, N: tl.constexpr):
    i = tl.arange(0, N)
    c0 = i.to(tl.uint32) * 2654435761
    c1 = (i * 7 + 3).to(tl.uint32)
    c2 = (i ^ 5).to(tl.uint32)
    c3 = (i * 0 + 11).to(tl.uint32)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
    tl.store(out_ptr + i * 4 + 0, a.to(tl.int32, bitcast=True))
    tl.store(out_ptr + i * 4 + 1, b.to(tl.int32, bitcast=True))
    tl.store(out_ptr + i * 4 + 2, c.to(tl.int32, bitcast=True))
    tl.store(out_ptr + i * 4 + 3, d.to(tl.int32, bitcast=True))

out = torch.zeros(64 * 4, dtype=torch.int32)
_k[(1,)](out, int(sys.argv[1]), 64)
np.save(sys.argv[2], out.numpy().view(np.uint32).reshape(64, 4))
"""


def test_against_independent_implementation(tmp_path):
    """Triton's own Philox (key = seed lo/hi, 10 rounds), run in its CPU interpreter."""
    pytest.importorskip("triton")
    seed = 0x0123456789ABCDEF
    path = str(tmp_path / "tri.npy")
    env = dict(os.environ, TRITON_INTERPRET="1")
    res = subprocess.run([sys.executable, "-c", _TRITON_PROBE, str(seed), path],
                         env=env, capture_output=True, text=True, timeout=300)
    if res.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + res.stderr[-300:])
    tri = np.load(path)
    i = np.arange(64, dtype=np.uint64)
    k0, k1 = philox.seed_key(seed)
    c0 = (i * np.uint64(2654435761)) & np.uint64(0xFFFFFFFF)
    ours = np.stack(philox.philox4x32_10(c0, i * 7 + 3, i ^ 5, 11, k0, k1), axis=1)
    assert np.array_equal(ours.astype(np.uint32), tri)


def test_uniform_mapping_exact_and_open():
    w = np.array([0, 255, 256, 0xFFFFFFFF, 0x80000000], dtype=np.uint64)
    u = philox.uniform_from_word(w)
    assert u[0] == 0.5 * 2.0 ** -24 and u[1] == u[0]
    assert u[2] == 1.5 * 2.0 ** -24
    assert u[3] == 1.0 - 0.5 * 2.0 ** -24
    assert u[4] == 0.5 + 0.5 * 2.0 ** -24
    assert np.all((u > 0) & (u < 1))


def test_params_moments_and_ranges():
    sigma, d, D = 4.0, 37, 4096
    G, b = philox.rff_params(11, sigma, d, D)
    assert G.shape == (d, D) and G.dtype == np.float32 and b.shape == (D,)
    g = G.astype(np.float64).ravel() * sigma
    n = g.size
    # standard normal: mean 0, variance 1, 4th moment 3, within ~5 standard errors
    assert abs(g.mean()) < 5 / np.sqrt(n)
    assert abs(g.var() - 1) < 5 * np.sqrt(2.0 / n)
    assert abs((g ** 4).mean() - 3) < 5 * np.sqrt(96.0 / n)
    assert np.all((b >= 0) & (b < np.float32(np.pi)))
    # b / pi uniform on [0, 1): chi-square over 16 bins
    h, _ = np.histogram(b / np.pi, bins=16, range=(0, 1))
    chi2 = ((h - D / 16) ** 2 / (D / 16)).sum()
    assert chi2 < 45.0   # P(chi2_15 > 45) ~ 1e-4


def test_block_columns_equal_full_matrix():
    """Sec. 4 block-wise maps: any column range equals the slice of the full draw."""
    G, b = philox.rff_params(5, 2.5, 19, 1000)
    for lo, hi in [(0, 1), (333, 667), (999, 1000), (128, 256)]:
        Gb, bb = philox.rff_params(5, 2.5, 19, 1000, lo, hi)
        assert np.array_equal(Gb, G[:, lo:hi]) and np.array_equal(bb, b[lo:hi])


def test_rows_are_stream_prefix():
    """Rows come from counters (k, r // 4): a shorter d is a prefix of a longer one."""
    G1, _ = philox.rff_params(9, 1.0, 6, 50)
    G2, _ = philox.rff_params(9, 1.0, 13, 50)
    assert np.array_equal(G1, G2[:6])
