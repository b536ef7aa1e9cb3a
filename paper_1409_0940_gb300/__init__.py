"""Python binding of librff_admm.so: block-splitting ADMM over implicit random
Fourier features on a GB300 (sm_103a).

Argument marshalling only.  Every step of the solver runs in the CUDA library;
this module converts numpy arrays / torch tensors to pointers and sizes, calls
the C ABI of include/rff_admm.h under the same function names, and turns error
codes into exceptions.  There is no CPU fallback: importing fails loudly when
the library has not been built (``paper_1409_0940_gb300.build.build()``).
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# RFF_ADMM_CHECK=1 loads the bounds-checked build of the library (built by build(check=True))
CHECKED = os.environ.get("RFF_ADMM_CHECK") == "1"
LIB_PATH = os.path.join(_HERE, "librff_admm_check.so" if CHECKED else "librff_admm.so")

RFF_OK, RFF_EINVAL, RFF_ENOMEM, RFF_ECUDA, RFF_ETIMEOUT, RFF_ENOTREADY, RFF_ENUMERIC, RFF_ECANCELLED = range(8)
_STATUS = {0: "RFF_OK", 1: "RFF_EINVAL", 2: "RFF_ENOMEM", 3: "RFF_ECUDA", 4: "RFF_ETIMEOUT",
           5: "RFF_ENOTREADY", 6: "RFF_ENUMERIC", 7: "RFF_ECANCELLED"}
LOSSES = {"squared": 0, "hinge": 1, "logistic": 2, "multinomial": 3, "l1": 4, "crammer_singer": 5}
FEATURE_MAPS = {"fourier": 0, "laplace": 1, "fastfood": 2, "tensorsketch": 3}
REGS = {"l2": 0, "l1": 1}
PRECS = {"fp32": 0, "split_bf16": 1, "cached_z": 2}
RHO_SCALES = {"sum": 0, "mean": 1}


class RffError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (_STATUS.get(status, status), message))
        self.status = status


class rff_admm_params(ctypes.Structure):
    _fields_ = [("loss", ctypes.c_int32), ("reg", ctypes.c_int32), ("lambda_", ctypes.c_double),
                ("sigma", ctypes.c_double), ("rho", ctypes.c_double), ("D", ctypes.c_int64),
                ("R", ctypes.c_int32), ("C", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("prec", ctypes.c_int32), ("m", ctypes.c_int32), ("rho_scale", ctypes.c_int32),
                ("newton_iters", ctypes.c_int32), ("feature_map", ctypes.c_int32), ("degree", ctypes.c_int32),
                ("coef0", ctypes.c_double)]


class rff_admm_stats(ctypes.Structure):
    _fields_ = [("iters_done", ctypes.c_int32), ("primal_res", ctypes.c_double), ("dual_res", ctypes.c_double),
                ("objective", ctypes.c_double), ("ms_setup", ctypes.c_double), ("ms_iterations", ctypes.c_double)]


class rff_admm_profile(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("launches", ctypes.c_int64), ("ms_prox_reg", ctypes.c_double),
                ("ms_pass1", ctypes.c_double), ("ms_project", ctypes.c_double), ("ms_pass2", ctypes.c_double),
                ("ms_exchange", ctypes.c_double), ("ms_average", ctypes.c_double), ("tc_kchunk", ctypes.c_int32),
                ("nsplit", ctypes.c_int32), ("tc_z_tmem", ctypes.c_int32), ("tc_cta_pair", ctypes.c_int32)]


class rff_completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("kind", ctypes.c_int32), ("status", ctypes.c_int32),
                ("queue_ms", ctypes.c_double), ("run_ms", ctypes.c_double), ("latency_ms", ctypes.c_double)]


RFF_REQ_SOLVE, RFF_REQ_SCORE = 0, 1


# every entry point of include/rff_admm.h: name -> (restype, argtypes)
_P, _I32, _I64, _U64, _D, _SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, \
    ctypes.c_size_t
PROTOTYPES = {
    "rff_admm_create": (_I32, [ctypes.POINTER(rff_admm_params), _P, ctypes.POINTER(_P)]),
    "rff_admm_set_data": (_I32, [_P, _P, _P, _I64, _I64, ctypes.c_int]),
    "rff_admm_set_data_csr": (_I32, [_P, _P, _P, _P, _I64, _P, _I64, _I64, ctypes.c_int]),
    "rff_admm_solve": (_I32, [_P, _I32, ctypes.POINTER(rff_admm_stats)]),
    "rff_admm_predict": (_I32, [_P, _P, _I64, _P, ctypes.c_int]),
    "rff_admm_predict_noalloc": (_I32, [_P, _P, _I64, _P]),
    "rff_admm_predict_labels": (_I32, [_P, _P, _I64, _P, ctypes.c_int]),
    "rff_admm_get_weights": (_I32, [_P, _P, ctypes.c_int]),
    "rff_admm_get_state": (_I32, [_P, _P, ctypes.POINTER(_SZ)]),
    "rff_admm_set_state": (_I32, [_P, _P, _SZ]),
    "rff_admm_set_profiling": (_I32, [_P, ctypes.c_int]),
    "rff_admm_get_profile": (_I32, [_P, ctypes.POINTER(rff_admm_profile)]),
    "rff_admm_set_memory_limit": (_I32, [_P, _SZ]),
    "rff_admm_set_stream": (_I32, [_P, _P]),
    "rff_admm_estimate_bytes": (_I32, [ctypes.POINTER(rff_admm_params), _I64, _I64, ctypes.POINTER(_SZ),
                                       ctypes.POINTER(_SZ)]),
    "rff_admm_set_lambdas": (_I32, [_P, _P, _I32]),
    "rff_admm_set_block_fraction": (_I32, [_P, _D]),
    "rff_admm_release_features": (_I32, [_P, ctypes.POINTER(_SZ)]),
    "rff_measure_fma_peaks": (_I32, [ctypes.POINTER(_D), ctypes.POINTER(_D), _P]),
    "rff_selftest_wait_timeout": (_I32, [_P]),
    "rff_admm_enqueue": (_I32, [_P, _I32]),
    "rff_admm_wait": (_I32, [_P]),
    "rff_sweep_run": (_I32, [_P, _I32, _I32]),
    "rff_admm_destroy": (None, [_P]),
    "rff_admm_last_error": (ctypes.c_char_p, [_P]),
    "rff_philox4x32_10": (_I32, [_P, _U64, _I64, _P, _P]),
    "rff_rff_params": (_I32, [_U64, _D, _I64, _I64, _I64, _P, _P, _P]),
    "rff_features": (_I32, [_P, _I64, _I64, _U64, _D, _I64, _I64, _I64, _I32, _P, _P]),
    "rff_laplace_params": (_I32, [_U64, _D, _I64, _I64, _I64, _P, _P]),
    "rff_fastfood_params": (_I32, [_U64, _D, _I64, _I64, _I64, _P, _P, _P]),
    "rff_laplace_features": (_I32, [_P, _I64, _I64, _U64, _D, _I64, _I64, _I64, _P, _P]),
    "rff_tensorsketch_features": (_I32, [_P, _I64, _I64, _U64, _D, _D, _I32, _I64, _I32, _P, _P]),
    "rff_prox_loss": (_I32, [_I32, _P, _P, _I64, _I32, _D, _I32, _P, _P]),
    "rff_prox_reg": (_I32, [_I32, _P, _I64, _D, _P, _P]),
    "rff_cholesky_f64": (_I32, [_P, _I32, _I32, _P, _P]),
    "rff_server_create": (_I32, [_SZ, _I32, ctypes.POINTER(_P)]),
    "rff_server_submit_solve": (_I32, [_P, ctypes.POINTER(rff_admm_params), _P, _P, _I64, _I64, _I32,
                                       ctypes.POINTER(_I64)]),
    "rff_server_submit_score": (_I32, [_P, _I64, _P, _I64, _P, ctypes.POINTER(_I64)]),
    "rff_server_poll": (_I32, [_P, ctypes.POINTER(rff_completion), _I32, ctypes.POINTER(_I32), _I32]),
    "rff_server_get_weights": (_I32, [_P, _I64, _P]),
    "rff_server_release": (_I32, [_P, _I64]),
    "rff_server_cancel": (_I32, [_P, _I64]),
    "rff_check_enabled": (_I32, []),
    "rff_check_report": (_I32, [_P]),
    "rff_server_memory": (_I32, [_P, ctypes.POINTER(_SZ), ctypes.POINTER(_SZ)]),
    "rff_server_destroy": (None, [_P]),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("%s is not built; run paper_1409_0940_gb300.build.build(%s) "
                          "(needs nvcc) -- there is no CPU fallback"
                          % (os.path.basename(LIB_PATH), "check=True" if CHECKED else ""))
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


# ----------------------------------------------------------------- marshalling
def _is_torch_cuda(x):
    return type(x).__module__.startswith("torch") and getattr(x, "is_cuda", False)


def _ptr(x, dtype=np.float32):
    """(pointer, is_device) of a contiguous numpy array or torch tensor of `dtype`."""
    if x is None:
        return None, 0
    if _is_torch_cuda(x) or type(x).__module__.startswith("torch"):
        import torch
        tdt = {np.float32: torch.float32, np.float64: torch.float64, np.uint32: torch.int32,
               np.int32: torch.int32, np.int64: torch.int64}[dtype]
        if x.dtype != tdt or not x.is_contiguous():
            raise TypeError("expected a contiguous %s tensor" % tdt)
        if x.is_cuda:
            torch.cuda.synchronize(x.device)
        return ctypes.c_void_p(x.data_ptr()), 1 if x.is_cuda else 0
    if not isinstance(x, np.ndarray) or x.dtype != dtype or not x.flags.c_contiguous:
        raise TypeError("expected a C-contiguous numpy array of %s" % np.dtype(dtype))
    return ctypes.c_void_p(x.ctypes.data), 0


def _check(status, h=None, what=""):
    if status != RFF_OK:
        msg = lib.rff_admm_last_error(h).decode() if h else what
        raise RffError(status, msg or what)


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(stream)
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


def make_params(loss="squared", reg="l2", lam=1e-4, sigma=1.0, rho=1.0, D=512, R=1, C=1, seed=0,
                prec="fp32", m=1, rho_scale="sum", newton_iters=0, feature_map="fourier", degree=2, coef0=1.0):
    return rff_admm_params(LOSSES[loss], REGS[reg], lam, sigma, rho, D, R, C, seed, PRECS[prec], m,
                           RHO_SCALES[rho_scale], newton_iters, FEATURE_MAPS[feature_map], degree, coef0)


# ----------------------------------------------------------------- C ABI, same names
# (m, d) of every handle this binding created, for the shape checks of the calls that take
# bare device pointers (the library cannot see how large a caller's buffer is)
_dims = {}


def rff_admm_create(params, stream=None):
    h = ctypes.c_void_p()
    _check(lib.rff_admm_create(ctypes.byref(params), _stream(stream), ctypes.byref(h)), None,
           "rff_admm_create rejected the parameters")
    _dims[h.value] = [int(params.m), None]
    return h


def rff_admm_set_data(h, X, Y):
    n, d = X.shape
    px, dx = _ptr(X)
    py, dy = _ptr(Y)
    if dx != dy:
        raise TypeError("X and Y must both be host or both be device arrays")
    _check(lib.rff_admm_set_data(h, px, py, n, d, dx), h)
    if h.value in _dims:
        _dims[h.value][1] = int(d)


def rff_admm_set_data_csr(h, indptr, indices, values, Y, d):
    """X in CSR form: indptr (n + 1, int64), indices (int32), values (float32)."""
    n = Y.shape[0]
    pp, dp = _ptr(indptr, np.int64)
    pi, di = _ptr(indices, np.int32)
    pv, dv = _ptr(values, np.float32)
    py, dy = _ptr(Y)
    if len({dp, di, dv, dy}) != 1:
        raise TypeError("the CSR arrays and Y must all be host or all be device arrays")
    _check(lib.rff_admm_set_data_csr(h, pp, pi, pv, values.shape[0], py, n, d, dy), h)
    if h.value in _dims:
        _dims[h.value][1] = int(d)


def rff_admm_solve(h, iters, stats=True):
    st = rff_admm_stats() if stats else None
    _check(lib.rff_admm_solve(h, iters, ctypes.byref(st) if stats else None), h)
    if not stats:
        return None
    return {k: getattr(st, k) for k, _ in rff_admm_stats._fields_}


def rff_admm_predict(h, Xq, out):
    pq, dq = _ptr(Xq)
    po, do = _ptr(out)
    if dq != do:
        raise TypeError("Xq and scores must both be host or both be device arrays")
    _check(lib.rff_admm_predict(h, pq, Xq.shape[0], po, dq), h)
    return out


def rff_admm_predict_labels(h, Xq, out):
    px, dx = _ptr(Xq)
    po, do = _ptr(out, np.int32)
    if dx != do:
        raise TypeError("Xq and the labels must both be host or both be device arrays")
    _check(lib.rff_admm_predict_labels(h, px, Xq.shape[0], po, dx), h)
    return out


def rff_admm_predict_noalloc(h, Xq, out):
    """Scores into `out` without any device allocation (device tensors only).  The
    shapes are checked against the handle first: the library reads q x d queries and
    writes q x m scores through bare device pointers."""
    m, d = _dims.get(getattr(h, "value", h), (None, None))
    if m is None or d is None:
        raise TypeError("rff_admm_predict_noalloc: the handle has no data set through this binding")
    if len(Xq.shape) != 2 or Xq.shape[1] != d:
        raise TypeError("rff_admm_predict_noalloc: queries of shape %s, the model takes (q, %d)"
                        % (tuple(Xq.shape), d))
    if tuple(out.shape) != (Xq.shape[0], m):
        raise TypeError("rff_admm_predict_noalloc: scores of shape %s, expected (%d, %d)"
                        % (tuple(out.shape), Xq.shape[0], m))
    pq, dq = _ptr(Xq)
    po, do = _ptr(out)
    if not (dq and do):
        raise TypeError("rff_admm_predict_noalloc takes device tensors")
    _check(lib.rff_admm_predict_noalloc(h, pq, Xq.shape[0], po), h)
    return out


def rff_admm_get_weights(h, out):
    po, do = _ptr(out)
    _check(lib.rff_admm_get_weights(h, po, do), h)
    return out


def rff_admm_get_state(h):
    n = ctypes.c_size_t(0)
    _check(lib.rff_admm_get_state(h, None, ctypes.byref(n)), h)
    buf = ctypes.create_string_buffer(n.value)
    _check(lib.rff_admm_get_state(h, buf, ctypes.byref(n)), h)
    return buf.raw[:n.value]


def rff_admm_set_state(h, state):
    buf = ctypes.create_string_buffer(state, len(state))
    _check(lib.rff_admm_set_state(h, buf, len(state)), h)


def rff_admm_set_profiling(h, enable):
    _check(lib.rff_admm_set_profiling(h, 1 if enable else 0), h)


def rff_admm_get_profile(h):
    p = rff_admm_profile()
    _check(lib.rff_admm_get_profile(h, ctypes.byref(p)), h)
    return {k: getattr(p, k) for k, _ in rff_admm_profile._fields_}


def rff_admm_set_memory_limit(h, nbytes):
    _check(lib.rff_admm_set_memory_limit(h, nbytes), h)


def rff_admm_set_stream(h, stream):
    """Move the handle's work to `stream` (a torch.cuda.Stream or a raw cudaStream_t)."""
    _check(lib.rff_admm_set_stream(h, getattr(stream, "cuda_stream", stream)), h)


def rff_admm_estimate_bytes(params, n, d):
    """(resident, peak) device bytes of a solve; no device work."""
    r, p = ctypes.c_size_t(0), ctypes.c_size_t(0)
    _check(lib.rff_admm_estimate_bytes(ctypes.byref(params), n, d, ctypes.byref(r), ctypes.byref(p)), None,
           "rff_admm_estimate_bytes")
    return r.value, p.value


def rff_admm_set_lambdas(h, lambdas):
    if lambdas is None:
        _check(lib.rff_admm_set_lambdas(h, None, 0), h)
        return
    arr = np.ascontiguousarray(lambdas, dtype=np.float64)
    _check(lib.rff_admm_set_lambdas(h, ctypes.c_void_p(arr.ctypes.data), arr.size), h)


def rff_admm_enqueue(h, iters):
    _check(lib.rff_admm_enqueue(h, iters), h)


def rff_admm_wait(h):
    _check(lib.rff_admm_wait(h), h)


def rff_sweep_run(handles, iters):
    arr = (ctypes.c_void_p * len(handles))(*[hh.value for hh in handles])
    st = lib.rff_sweep_run(arr, len(handles), iters)
    if st != RFF_OK:
        msgs = [lib.rff_admm_last_error(hh).decode() for hh in handles]
        raise RffError(st, "; ".join(m for m in msgs if m) or "rff_sweep_run failed")


def rff_admm_destroy(h):
    _dims.pop(getattr(h, "value", h), None)
    lib.rff_admm_destroy(h)


def rff_admm_last_error(h):
    return lib.rff_admm_last_error(h).decode()


def rff_philox4x32_10(ctr, seed, out, stream=None):
    pc, _ = _ptr(ctr, np.uint32)
    po, _ = _ptr(out, np.uint32)
    _check(lib.rff_philox4x32_10(pc, seed, ctr.numel() // 4, po, _stream(stream)), None, "rff_philox4x32_10")
    return out


def rff_rff_params(seed, sigma, d, k_lo, k_hi, G, b, stream=None):
    pg, _ = _ptr(G)
    pb, _ = _ptr(b)
    _check(lib.rff_rff_params(seed, sigma, d, k_lo, k_hi, pg, pb, _stream(stream)), None, "rff_rff_params")
    return G, b


def rff_features(X, seed, sigma, D, k_lo, k_hi, prec, Z, stream=None):
    px, _ = _ptr(X)
    pz, _ = _ptr(Z)
    _check(lib.rff_features(px, X.shape[0], X.shape[1], seed, sigma, D, k_lo, k_hi, PRECS.get(prec, prec), pz,
                            _stream(stream)), None, "rff_features")
    return Z


def rff_laplace_params(seed, sigma, d, k_lo, k_hi, W, stream=None):
    pw, _ = _ptr(W)
    _check(lib.rff_laplace_params(seed, sigma, d, k_lo, k_hi, pw, _stream(stream)), None, "rff_laplace_params")
    return W


def rff_fastfood_params(seed, sigma, d, k_lo, k_hi, Vt, b, stream=None):
    pv, _ = _ptr(Vt)
    pb, _ = _ptr(b)
    _check(lib.rff_fastfood_params(seed, sigma, d, k_lo, k_hi, pv, pb, _stream(stream)), None, "rff_fastfood_params")
    return Vt, b


def rff_laplace_features(X, seed, sigma, D, k_lo, k_hi, Z, stream=None):
    px, _ = _ptr(X)
    pz, _ = _ptr(Z)
    _check(lib.rff_laplace_features(px, X.shape[0], X.shape[1], seed, sigma, D, k_lo, k_hi, pz, _stream(stream)),
           None, "rff_laplace_features")
    return Z


def rff_tensorsketch_features(X, seed, sigma, coef0, degree, D, C, Z, stream=None):
    px, _ = _ptr(X)
    pz, _ = _ptr(Z)
    _check(lib.rff_tensorsketch_features(px, X.shape[0], X.shape[1], seed, sigma, coef0, degree, D, C, pz,
                                         _stream(stream)), None, "rff_tensorsketch_features")
    return Z


def rff_prox_loss(loss, V, Y, t, newton_iters, out, stream=None):
    pv, _ = _ptr(V)
    py, _ = _ptr(Y)
    po, _ = _ptr(out)
    _check(lib.rff_prox_loss(LOSSES.get(loss, loss), pv, py, V.shape[0], V.shape[1], t, newton_iters, po,
                             _stream(stream)), None, "rff_prox_loss")
    return out


def rff_prox_reg(reg, V, tau, out, stream=None):
    pv, _ = _ptr(V)
    po, _ = _ptr(out)
    _check(lib.rff_prox_reg(REGS.get(reg, reg), pv, V.numel(), tau, po, _stream(stream)), None, "rff_prox_reg")
    return out


def rff_cholesky_f64(A, info, stream=None):
    pa, _ = _ptr(A, np.float64)
    pi, _ = _ptr(info, np.int32)
    _check(lib.rff_cholesky_f64(pa, A.shape[0], A.shape[1], pi, _stream(stream)), None, "rff_cholesky_f64")
    return A


def rff_server_create(budget_bytes=0, max_active=4):
    s = ctypes.c_void_p()
    _check(lib.rff_server_create(budget_bytes, max_active, ctypes.byref(s)), None, "rff_server_create")
    return s


def rff_server_submit_solve(srv, params, X, Y, iters):
    px, _ = _ptr(X)
    py, _ = _ptr(Y)
    rid = ctypes.c_int64(0)
    _check(lib.rff_server_submit_solve(srv, ctypes.byref(params), px, py, X.shape[0], X.shape[1], iters,
                                       ctypes.byref(rid)), None, "rff_server_submit_solve")
    return rid.value


def rff_server_submit_score(srv, model, Xq, out):
    pq, _ = _ptr(Xq)
    po, _ = _ptr(out)
    rid = ctypes.c_int64(0)
    _check(lib.rff_server_submit_score(srv, model, pq, Xq.shape[0], po, ctypes.byref(rid)), None,
           "rff_server_submit_score")
    return rid.value


def rff_server_poll(srv, max_count=64, wait_ms=0):
    buf = (rff_completion * max_count)()
    n = ctypes.c_int32(0)
    _check(lib.rff_server_poll(srv, buf, max_count, ctypes.byref(n), wait_ms), None, "rff_server_poll")
    return [{k: getattr(buf[i], k) for k, _ in rff_completion._fields_} for i in range(n.value)]


def rff_server_get_weights(srv, model, out):
    po, _ = _ptr(out)
    _check(lib.rff_server_get_weights(srv, model, po), None, "rff_server_get_weights")
    return out


def rff_server_release(srv, model):
    _check(lib.rff_server_release(srv, model), None, "rff_server_release")


def rff_server_cancel(srv, request_id):
    """True if the request left the queue (it completes with RFF_ECANCELLED), False if it had
    already started or finished."""
    st = lib.rff_server_cancel(srv, request_id)
    if st == RFF_ENOTREADY:
        return False
    _check(st, None, "rff_server_cancel")
    return True


def rff_check_enabled():
    return bool(lib.rff_check_enabled())


def rff_check_report():
    """Failed bounds checks since the last report: dict(count, unit, line, index, bound)."""
    out = (ctypes.c_int64 * 5)()
    _check(lib.rff_check_report(out), None, "rff_check_report")
    return dict(zip(("count", "unit", "line", "index", "bound"), list(out)))


def rff_server_memory(srv):
    u, b = ctypes.c_size_t(0), ctypes.c_size_t(0)
    _check(lib.rff_server_memory(srv, ctypes.byref(u), ctypes.byref(b)), None, "rff_server_memory")
    return u.value, b.value


def rff_server_destroy(srv):
    lib.rff_server_destroy(srv)


# ----------------------------------------------------------------- convenience
def rff_admm_set_block_fraction(h, p):
    _check(lib.rff_admm_set_block_fraction(h, float(p)), h)


def rff_selftest_wait_timeout(stream=None):
    """Status of the bounded-wait probe: RFF_ETIMEOUT when the bound fired (the expected outcome)."""
    return lib.rff_selftest_wait_timeout(_stream(stream))


def rff_measure_fma_peaks(stream=None):
    """(FP32, FP64) FMA throughput of the GPU's SIMT pipes in TFLOP/s, measured."""
    a, b = _D(0), _D(0)
    _check(lib.rff_measure_fma_peaks(ctypes.byref(a), ctypes.byref(b), _stream(stream)), None,
           "rff_measure_fma_peaks")
    return a.value, b.value


def rff_admm_release_features(h):
    n = _SZ(0)
    _check(lib.rff_admm_release_features(h, ctypes.byref(n)), h)
    return n.value


class Solver:
    """Owns one rff_admm_t handle."""

    def __init__(self, stream=None, **kw):
        self.params = make_params(**kw)
        self.m = self.params.m
        self.D = self.params.D
        self.h = rff_admm_create(self.params, stream)

    def set_data(self, X, Y):
        rff_admm_set_data(self.h, X, Y)

    def set_data_csr(self, indptr, indices, values, Y, d):
        rff_admm_set_data_csr(self.h, indptr, indices, values, Y, d)

    def solve(self, iters, stats=True):
        return rff_admm_solve(self.h, iters, stats)

    def predict(self, Xq, out=None):
        if out is None:
            out = np.empty((Xq.shape[0], self.m), dtype=np.float32)
        return rff_admm_predict(self.h, Xq, out)

    def predict_labels(self, Xq, out=None):
        if out is None:
            out = np.empty(Xq.shape[0], dtype=np.int32)
        return rff_admm_predict_labels(self.h, Xq, out)

    def weights(self, out=None):
        if out is None:
            out = np.empty((self.D, self.m), dtype=np.float32)
        return rff_admm_get_weights(self.h, out)

    def get_state(self):
        return rff_admm_get_state(self.h)

    def set_state(self, state):
        rff_admm_set_state(self.h, state)

    def set_lambdas(self, lambdas):
        rff_admm_set_lambdas(self.h, lambdas)

    def set_block_fraction(self, p):
        rff_admm_set_block_fraction(self.h, p)

    def release_features(self):
        return rff_admm_release_features(self.h)

    def enqueue(self, iters):
        rff_admm_enqueue(self.h, iters)

    def wait(self):
        rff_admm_wait(self.h)

    def profiling(self, enable=True):
        rff_admm_set_profiling(self.h, enable)

    def profile(self):
        return rff_admm_get_profile(self.h)

    def close(self):
        if self.h:
            rff_admm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
