"""GPU parity of each step of the iteration against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle import philox, prox as P, rff as orff  # noqa: E402


@pytest.fixture(scope="module")
def rff():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1409_0940_gb300
    torch.cuda.init()
    return paper_1409_0940_gb300


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


# ----------------------------------------------------------------- Philox
def test_philox_words_bit_exact(rff):
    rng = np.random.default_rng(0)
    n = 1 << 20
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64)
    ctr[:4] = [[0, 0, 0, 0], [2 ** 32 - 1] * 4, [1, 2, 3, 4], [0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344]]
    seed = 0x299F31D0A4093822
    out = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
    rff.rff_philox4x32_10(dev(ctr.astype(np.uint32).view(np.int32)), seed, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32)
    k0, k1 = philox.seed_key(seed)
    ref = np.stack(philox.philox4x32_10(ctr[:, 0], ctr[:, 1], ctr[:, 2], ctr[:, 3], k0, k1), axis=1)
    assert np.array_equal(got, ref.astype(np.uint32))
    # the published known-answer vector, run on the device
    ctr1 = np.array([[0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344]], dtype=np.uint32)
    out1 = torch.zeros((1, 4), dtype=torch.int32, device="cuda")
    rff.rff_philox4x32_10(dev(ctr1.view(np.int32)), 0x299F31D0A4093822, out1)
    assert [int(x) for x in out1.cpu().numpy().view(np.uint32)[0]] == [0xD16CFE09, 0x94FDCCEB, 0x5001E420,
                                                                        0x24126EA1]


def _ulp_diff(a, b):
    ai = a.view(np.int32).astype(np.int64)
    bi = b.view(np.int32).astype(np.int64)
    ai = np.where(ai < 0, -(ai & 0x7FFFFFFF), ai)
    bi = np.where(bi < 0, -(bi & 0x7FFFFFFF), bi)
    return np.abs(ai - bi)


@pytest.mark.parametrize("d,k_lo,k_hi,sigma", [(37, 0, 1000, 4.0), (440, 5000, 9096, 10.0), (1, 7, 8, 0.5),
                                              (784, 65000, 65536, 9.0)])
def test_rff_params_match_oracle(rff, d, k_lo, k_hi, sigma):
    seed = 12345
    nk = k_hi - k_lo
    G = torch.empty((d, nk), dtype=torch.float32, device="cuda")
    b = torch.empty((nk,), dtype=torch.float32, device="cuda")
    rff.rff_rff_params(seed, sigma, d, k_lo, k_hi, G, b)
    torch.cuda.synchronize()
    Gr, br = philox.rff_params(seed, sigma, d, k_hi, k_lo, k_hi)
    g, bb = G.cpu().numpy(), b.cpu().numpy()
    # values equal except rare 1-ulp ties of the float64 libraries on each side
    ug, ub = _ulp_diff(g, Gr), _ulp_diff(bb, br)
    assert ug.max() <= 1 and ub.max() <= 1
    assert (ug > 0).sum() <= max(1, int(1e-6 * ug.size)) and (ub > 0).sum() <= 1


# ----------------------------------------------------------------- features
@pytest.mark.parametrize("n,d,D,k_lo,k_hi", [(300, 16, 512, 0, 512), (257, 37, 1000, 333, 667),
                                             (129, 440, 4096, 4000, 4096)])
def test_features_fp32_match_oracle(rff, n, d, D, k_lo, k_hi):
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n, d)).astype(np.float32)
    seed, sigma = 77, 3.0
    Z = torch.empty((n, k_hi - k_lo), dtype=torch.float32, device="cuda")
    rff.rff_features(dev(X), seed, sigma, D, k_lo, k_hi, "fp32", Z)
    torch.cuda.synchronize()
    ref = orff.features_block(X, seed, sigma, D, k_lo, k_hi)
    err = np.abs(Z.cpu().numpy() - ref).max() / np.sqrt(2.0 / D)
    # float32 dot products of length d and the float32 cosine: |error| <= 1e-5 of the scale
    assert err < 1e-5 * max(1.0, np.sqrt(d / 16)), err


@pytest.mark.parametrize("n,d,D,k_lo,k_hi", [(300, 16, 512, 0, 512), (257, 37, 1000, 333, 667),
                                             (129, 440, 4096, 4000, 4096), (1000, 784, 2048, 0, 2048)])
def test_features_split_bf16_match_oracle(rff, n, d, D, k_lo, k_hi):
    """Tensor-core path: X.G as three BF16 products, FP32 accumulate, FP32 cosine."""
    rng = np.random.default_rng(n + 1)
    X = rng.standard_normal((n, d)).astype(np.float32)
    seed, sigma = 78, 3.0
    Z = torch.empty((n, k_hi - k_lo), dtype=torch.float32, device="cuda")
    rff.rff_features(dev(X), seed, sigma, D, k_lo, k_hi, "split_bf16", Z)
    torch.cuda.synchronize()
    ref = orff.features_block(X, seed, sigma, D, k_lo, k_hi)
    err = np.abs(Z.cpu().numpy() - ref).max() / np.sqrt(2.0 / D)
    # split products carry ~2^-16 relative error per term of the length-d dot product
    assert err < 2e-4 * max(1.0, np.sqrt(d / 64)), err


def test_features_independent_of_block_split(rff):
    """Sec. 4 block-wise maps: any feature range is the slice of the full map, bit for bit."""
    rng = np.random.default_rng(3)
    X = rng.random((200, 21)).astype(np.float32)
    D = 700
    full = torch.empty((200, D), dtype=torch.float32, device="cuda")
    rff.rff_features(dev(X), 9, 1.5, D, 0, D, "fp32", full)
    for lo, hi in [(0, 1), (100, 357), (512, 700)]:
        part = torch.empty((200, hi - lo), dtype=torch.float32, device="cuda")
        rff.rff_features(dev(X), 9, 1.5, D, lo, hi, "fp32", part)
        assert torch.equal(part, full[:, lo:hi].contiguous())


# ----------------------------------------------------------------- proxes
@pytest.mark.parametrize("loss,m", [("squared", 3), ("hinge", 1), ("hinge", 7), ("logistic", 1),
                                    ("multinomial", 5), ("multinomial", 147), ("l1", 1), ("l1", 6),
                                    ("crammer_singer", 2), ("crammer_singer", 10), ("crammer_singer", 147),
                                    ("crammer_singer", 256)])
def test_prox_loss_matches_oracle(rff, loss, m):
    rng = np.random.default_rng(m)
    n = 3000
    V = (rng.standard_normal((n, m)) * 2).astype(np.float32)
    if loss in ("squared", "l1"):
        Y = rng.standard_normal((n, m)).astype(np.float32)
    elif loss in ("hinge", "logistic") and m == 1:
        Y = np.where(rng.random((n, 1)) < 0.5, -1.0, 1.0).astype(np.float32)
    else:
        Y = synth.onehot_pm1(rng.integers(0, m, n), m)
    for t in [1e-3, 0.3, 1.0, 7.0]:
        out = torch.empty((n, m), dtype=torch.float32, device="cuda")
        rff.rff_prox_loss(loss, dev(V), dev(Y), t, 8, out)
        torch.cuda.synchronize()
        ref = P.prox_loss(loss, V.astype(np.float64), Y.astype(np.float64), t)
        err = np.abs(out.cpu().numpy() - ref).max() / max(1.0, np.abs(ref).max())
        assert err < 2e-6, (loss, m, t, err)


@pytest.mark.parametrize("reg", ["l2", "l1"])
def test_prox_reg_matches_oracle(rff, reg):
    rng = np.random.default_rng(1)
    V = (rng.standard_normal(10007) * 3).astype(np.float32)
    for tau in [1e-4, 0.5, 2.0]:
        out = torch.empty_like(dev(V))
        rff.rff_prox_reg(reg, dev(V), tau, out)
        ref = P.prox_reg(reg, V.astype(np.float64), tau)
        assert np.abs(out.cpu().numpy() - ref).max() < 1e-6 * max(1.0, np.abs(ref).max())


# ----------------------------------------------------------------- Cholesky
@pytest.mark.parametrize("s", [1, 5, 63, 64, 65, 200, 513, 1100, 2048])
def test_cholesky_f64_matches_numpy(rff, s):
    rng = np.random.default_rng(s)
    batch = 3
    A = np.empty((batch, s, s))
    for b in range(batch):
        M = rng.standard_normal((s, s + 3))
        A[b] = M @ M.T / s + np.eye(s)
    At = dev(A)
    info = torch.zeros(batch, dtype=torch.int32, device="cuda")
    rff.rff_cholesky_f64(At, info)
    torch.cuda.synchronize()
    assert info.cpu().numpy().tolist() == [0] * batch
    L = At.cpu().numpy()
    for b in range(batch):
        ref = np.linalg.cholesky(A[b])
        assert np.abs(L[b] - ref).max() < 1e-12 * np.abs(ref).max()


def test_cholesky_reports_non_positive_pivot(rff):
    s = 100
    A = np.eye(s)[None].repeat(2, 0)
    A[1, 70, 70] = -1.0
    At = dev(A)
    info = torch.zeros(2, dtype=torch.int32, device="cuda")
    rff.rff_cholesky_f64(At, info)
    assert info.cpu().numpy().tolist() == [0, 71]


# ----------------------------------------------------------------- measured SIMT peaks
def test_fma_peaks_are_plausible(rff):
    """FFMA and DFMA throughput from the library's own chains: FP32 between a quarter of and
    just above the derived peak (152 SMs x 128 lanes x 2 flop x 2.07 GHz = 80.5 TFLOP/s), FP64
    far below FP32 on this part."""
    fp32, fp64 = rff.rff_measure_fma_peaks()
    assert 20.0 < fp32 < 1.1 * 80.5, fp32
    assert 0.05 < fp64 < fp32 / 2, (fp32, fp64)


# ----------------------------------------------------------------- failure path
def test_bounded_wait_times_out_and_the_context_survives(rff):
    """A wait that nothing ends (a probe on an mbarrier nobody arrives on) runs out after its
    bound, reports RFF_ETIMEOUT through the device error word, and the GPU stays usable: the
    tensor-core passes run and report success right after."""
    assert rff.rff_selftest_wait_timeout() == rff.RFF_ETIMEOUT
    X, Y = synth.ridge(n=600, d=6, seed=2)
    s = rff.Solver(prec="split_bf16", loss="squared", reg="l2", lam=1e-3, sigma=2.0, D=256, R=2, C=2, seed=3, m=1)
    s.set_data(X, Y)
    st = s.solve(4)
    assert np.isfinite(st["objective"])
    s.close()
    assert rff.rff_selftest_wait_timeout() == rff.RFF_ETIMEOUT   # and again
