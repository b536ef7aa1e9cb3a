"""CPU checks of the C ABI: the library builds for sm_103a, loads without a GPU,
exports every entry point the header declares, and validates arguments on the host."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rff_admm.h")


@pytest.fixture(scope="module")
def rff():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1409_0940_gb300
    return paper_1409_0940_gb300


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rff_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for core in ["rff_admm_create", "rff_admm_set_data", "rff_admm_solve", "rff_admm_predict",
                 "rff_admm_get_weights", "rff_admm_get_state", "rff_admm_set_state", "rff_admm_destroy",
                 "rff_admm_last_error"]:
        assert core in names


def test_every_declared_symbol_is_exported_and_bound(rff):
    lib = ctypes.CDLL(rff.LIB_PATH)
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in rff.PROTOTYPES, name
        assert hasattr(rff, name), name


def test_parameter_validation_on_host(rff):
    bad = [dict(lam=0.0), dict(sigma=-1.0), dict(rho=0.0), dict(D=0), dict(R=0), dict(C=0),
           dict(C=10, D=5), dict(m=0), dict(m=300), dict(prec="split_bf16", C=65, D=1000),
           dict(prec="cached_z", C=65, D=1000)]
    for kw in bad:
        p = rff.make_params(**kw)
        h = ctypes.c_void_p()
        assert rff.lib.rff_admm_create(ctypes.byref(p), None, ctypes.byref(h)) == rff.RFF_EINVAL, kw
        assert not h.value
    p = rff.make_params()
    p.loss = 9
    h = ctypes.c_void_p()
    assert rff.lib.rff_admm_create(ctypes.byref(p), None, ctypes.byref(h)) == rff.RFF_EINVAL
    assert rff.lib.rff_admm_create(None, None, ctypes.byref(h)) == rff.RFF_EINVAL


def test_null_handle_calls_are_rejected(rff):
    assert rff.lib.rff_admm_solve(None, 1, None) == rff.RFF_EINVAL
    assert rff.lib.rff_admm_set_data(None, None, None, 1, 1, 0) == rff.RFF_EINVAL
    assert rff.lib.rff_admm_predict(None, None, 1, None, 0) == rff.RFF_EINVAL
    rff.lib.rff_admm_destroy(None)


def test_step_entry_points_validate_sizes(rff):
    assert rff.lib.rff_philox4x32_10(None, 0, -1, None, None) == rff.RFF_EINVAL
    assert rff.lib.rff_rff_params(0, -1.0, 4, 0, 8, None, None, None) == rff.RFF_EINVAL
    assert rff.lib.rff_features(None, 4, 0, 0, 1.0, 8, 0, 8, 0, None, None) == rff.RFF_EINVAL
    assert rff.lib.rff_prox_loss(7, None, None, 1, 1, 1.0, 8, None, None) == rff.RFF_EINVAL
    assert rff.lib.rff_prox_reg(5, None, 1, 1.0, None, None) == rff.RFF_EINVAL
    assert rff.lib.rff_cholesky_f64(None, 1, 0, None, None) == rff.RFF_EINVAL


def test_noalloc_binding_checks_shapes_before_any_call(rff):
    """rff_admm_predict_noalloc takes bare device pointers, so the binding checks the
    buffers' shapes against the handle's (q, d) and (q, m) before marshalling anything;
    a handle it did not create (or without data) is refused the same way."""
    import numpy as np
    fake = ctypes.c_void_p(0x1000)
    with pytest.raises(TypeError, match="no data"):
        rff.rff_admm_predict_noalloc(fake, np.zeros((4, 3), np.float32), np.zeros((4, 2), np.float32))
    rff._dims[fake.value] = [2, 3]
    try:
        with pytest.raises(TypeError, match="queries of shape"):
            rff.rff_admm_predict_noalloc(fake, np.zeros((4, 5), np.float32), np.zeros((4, 2), np.float32))
        with pytest.raises(TypeError, match="scores of shape"):
            rff.rff_admm_predict_noalloc(fake, np.zeros((4, 3), np.float32), np.zeros((4, 3), np.float32))
        with pytest.raises(TypeError, match="scores of shape"):
            rff.rff_admm_predict_noalloc(fake, np.zeros((4, 3), np.float32), np.zeros((5, 2), np.float32))
        # right shapes on host arrays: refused for not being device memory, still before the call
        with pytest.raises(TypeError, match="device tensors"):
            rff.rff_admm_predict_noalloc(fake, np.zeros((4, 3), np.float32), np.zeros((4, 2), np.float32))
    finally:
        rff._dims.pop(fake.value, None)
