"""Thin ctypes binding of include/sqsm.h.

Argument marshalling only: tensors are checked for device, dtype and
contiguity and passed as raw pointers together with the current CUDA stream.
Every computation happens in libsqsm.so; there is no CPU fallback, and
importing this module fails if the library has not been built.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsqsm.so")

OK = 0
ERR_INVALID_ARG = 1
ERR_UNSUPPORTED = 2
ERR_NOT_PD = 4
ERR_NONFINITE = 8
ERR_CUDA = 16
ERR_NO_MEMORY = 32
ERR_TOO_LARGE = 64
ERR_NOT_CONVERGED = 128
F32, F64 = 0, 1
CUBATURE, EXTENDED, UNSCENTED, GAUSS_HERMITE = 0, 1, 2, 3
MODEL_CT_BEARINGS = 1
MODEL_POPULATION = 2
MODEL_CT_BEARINGS_R = 3

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with "
                      "`python -m paper_2207_00426_gb300.build` (needs nvcc)")

lib = ctypes.CDLL(LIB_PATH)

_p = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int


class Options(ctypes.Structure):
    _fields_ = [("leaf_chunk", _int), ("radix", _int), ("use_graph", _int), ("autotune", _int),
                ("absolute", _int), ("prior_covariance", _int), ("refine", _int),
                ("textbook_slr", _int), ("max_group_steps", _int)]


class Model(ctypes.Structure):
    _fields_ = [("kind", _int), ("dt", ctypes.c_double), ("sensors", ctypes.c_double * 4)]


lib.sqsm_create.argtypes = [ctypes.POINTER(_p), _int, ctypes.POINTER(Options)]
lib.sqsm_create.restype = _int
lib.sqsm_destroy.argtypes = [_p]
lib.sqsm_destroy.restype = _int
lib.sqsm_last_error.argtypes = [_p]
lib.sqsm_last_error.restype = ctypes.c_char_p
lib.sqsm_get_status.argtypes = [_p, ctypes.POINTER(_int)]
lib.sqsm_get_status.restype = _int
lib.sqsm_supported_shape.argtypes = [_int, _int]
lib.sqsm_supported_shape.restype = _int
lib.sqsm_lgssm_smooth.argtypes = ([_p, _int, _int, _int, _i64] + [_p, _i64] * 6
                                  + [_p] * 3 + [_p] * 4 + [_p, _p])
lib.sqsm_lgssm_smooth.restype = _int
lib.sqsm_ipls_smooth.argtypes = [_p, _int, ctypes.POINTER(Model), ctypes.POINTER(ctypes.c_double),
                                 _int, _int, _i64, ctypes.POINTER(_i64)] + [_p] * 8 + [_p]
lib.sqsm_ipls_smooth.restype = _int
lib.sqsm_ipls_smooth_tol.argtypes = ([_p, _int, ctypes.POINTER(Model),
                                      ctypes.POINTER(ctypes.c_double), _int, _int,
                                      ctypes.c_double, _i64, ctypes.POINTER(_i64)]
                                     + [_p] * 9 + [_p])
lib.sqsm_ipls_smooth_tol.restype = _int
lib.sqsm_ipls_smooth_std.argtypes = ([_p, _int, ctypes.POINTER(Model),
                                      ctypes.POINTER(ctypes.c_double), _int, _int, _i64,
                                      ctypes.POINTER(_i64)] + [_p] * 6 + [_p])
lib.sqsm_ipls_smooth_std.restype = _int
lib.sqsm_ct_linearize.argtypes = [_p, _int, ctypes.POINTER(Model), ctypes.POINTER(ctypes.c_double),
                                  _int, _i64, ctypes.POINTER(_i64)] + [_p] * 9 + [_p]
lib.sqsm_ct_linearize.restype = _int

lib.sqsm_ipls_nll_grad.argtypes = [_p, _int, ctypes.POINTER(Model), ctypes.POINTER(ctypes.c_double),
                                   _int, _int, _int, ctypes.c_double, _i64,
                                   ctypes.POINTER(_i64)] + [_p] * 11 + [_p]
lib.sqsm_ipls_nll_grad.restype = _int
lib.sqsm_lgssm_smooth_noalloc.argtypes = ([_int, _int, _int, _i64] + [_p, _i64] * 6
                                          + [_p] * 3 + [_p] * 4 + [_p, _p])
lib.sqsm_lgssm_smooth_noalloc.restype = _int
lib.sqsm_profile_enable.argtypes = [_p, _int]
lib.sqsm_profile_enable.restype = _int
lib.sqsm_profile_read.argtypes = [_p, _int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_int),
                                  ctypes.POINTER(_int)]
lib.sqsm_profile_read.restype = _int
lib.sqsm_kernel_name.argtypes = [_int]
lib.sqsm_kernel_name.restype = ctypes.c_char_p
lib.sqsm_scan_shape.argtypes = [_p, _int, _int, _i64, ctypes.POINTER(_i64), ctypes.POINTER(_int),
                                ctypes.POINTER(_int)]
lib.sqsm_scan_shape.restype = _int
lib.sqsm_fp32_fma_probe.argtypes = [_int, _int, _int, _p, ctypes.POINTER(ctypes.c_double), _p]
lib.sqsm_fp32_fma_probe.restype = _int

EXPORTED = ["sqsm_create", "sqsm_destroy", "sqsm_last_error", "sqsm_get_status",
            "sqsm_supported_shape", "sqsm_lgssm_smooth", "sqsm_ipls_smooth",
            "sqsm_ct_linearize", "sqsm_profile_enable", "sqsm_profile_read",
            "sqsm_kernel_name", "sqsm_lgssm_smooth_noalloc", "sqsm_ipls_nll_grad",
            "sqsm_scan_shape", "sqsm_ipls_smooth_tol", "sqsm_ipls_smooth_std",
            "sqsm_fp32_fma_probe"]


class SqsmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"sqsm error {code}: {msg}")
        self.code = code


def _dtype_code(t):
    if t == torch.float32:
        return F32
    if t == torch.float64:
        return F64
    raise TypeError(f"unsupported dtype {t}")


def _ptr(t, dtype=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} has dtype {t.dtype}, expected {dtype}")
    return t.data_ptr()


def _stream():
    return torch.cuda.current_stream().cuda_stream


class Context:
    """Owns an sqsm_ctx (workspaces, plans, graphs) on one device."""

    def __init__(self, device=None, leaf_chunk=0, radix=0, use_graph=True, autotune=False,
                 absolute=False, prior_covariance=False, refine=0, textbook_slr=False,
                 max_group_steps=0):
        if device is None:
            device = torch.cuda.current_device()
        self.device = int(device)
        h = _p()
        opt = Options(leaf_chunk, radix, 1 if use_graph else 0, 1 if autotune else 0,
                      1 if absolute else 0, 1 if prior_covariance else 0, int(refine),
                      1 if textbook_slr else 0, int(max_group_steps))
        rc = lib.sqsm_create(ctypes.byref(h), self.device, ctypes.byref(opt))
        if rc != OK:
            raise SqsmError(rc, "sqsm_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib.sqsm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, rc):
        if rc != OK:
            raise SqsmError(rc, lib.sqsm_last_error(self.h).decode())

    def profile(self, on=True):
        """Enable / disable per-kernel event timing of subsequent calls."""
        self.check(lib.sqsm_profile_enable(self.h, 1 if on else 0))

    def profile_read(self):
        """{kernel family: (total ms, launches)} of the last profiled call."""
        n = 32
        ms = (ctypes.c_double * n)()
        cnt = (_int * n)()
        nf = _int(0)
        self.check(lib.sqsm_profile_read(self.h, n, ms, cnt, ctypes.byref(nf)))
        return {lib.sqsm_kernel_name(k).decode(): (ms[k], cnt[k])
                for k in range(nf.value) if cnt[k] > 0}

    def status(self):
        v = _int(0)
        self.check(lib.sqsm_get_status(self.h, ctypes.byref(v)))
        return v.value

    def scan_shape(self, offsets, dtype=torch.float32, linearization=0):
        """(leaf_chunk, radix) that IPLS calls with these sequence offsets use."""
        off = (_i64 * len(offsets))(*[int(v) for v in offsets])
        leaf, radix = _int(0), _int(0)
        self.check(lib.sqsm_scan_shape(self.h, _dtype_code(dtype), int(linearization),
                                       len(offsets) - 1, off, ctypes.byref(leaf),
                                       ctypes.byref(radix)))
        return leaf.value, radix.value


def supported_shape(nx, ny):
    return bool(lib.sqsm_supported_shape(nx, ny))


def sqsm_lgssm_smooth(ctx, F, c, SQ, H, d, SR, m0, N0, y, mf=None, Nf=None, ms=None, Ns=None,
                      loglik=None, strides=None):
    """Call sqsm_lgssm_smooth.  Per-step arrays have a leading time axis of
    length n, or none (time-invariant, stride 0).  Outputs are allocated if
    not given; returns (mf, Nf, ms, Ns, loglik)."""
    dt = y.dtype
    code = _dtype_code(dt)
    n, ny = y.shape
    nx = m0.shape[0]
    dev = y.device

    def stride(a, per):
        return 0 if a.dim() == per else a[0].numel()

    if strides is None:
        strides = (stride(F, 2), stride(c, 1), stride(SQ, 2), stride(H, 2), stride(d, 1), stride(SR, 2))
    if mf is None:
        mf = torch.empty((n + 1, nx), dtype=dt, device=dev)
    if Nf is None:
        Nf = torch.empty((n + 1, nx, nx), dtype=dt, device=dev)
    if ms is None:
        ms = torch.empty((n + 1, nx), dtype=dt, device=dev)
    if Ns is None:
        Ns = torch.empty((n + 1, nx, nx), dtype=dt, device=dev)
    if loglik is None:
        loglik = torch.empty(1, dtype=torch.float64, device=dev)
    args = []
    for name, a, s in zip("F c SQ H d SR".split(), (F, c, SQ, H, d, SR), strides):
        args += [_ptr(a, dt, name), s]
    rc = lib.sqsm_lgssm_smooth(ctx.h, code, nx, ny, n, *args, _ptr(m0, dt, "m0"), _ptr(N0, dt, "N0"),
                               _ptr(y, dt, "y"), _ptr(mf, dt, "mf"), _ptr(Nf, dt, "Nf"),
                               _ptr(ms, dt, "ms"), _ptr(Ns, dt, "Ns"),
                               _ptr(loglik, torch.float64, "loglik"), _stream())
    ctx.check(rc)
    return mf, Nf, ms, Ns, loglik


def _ct_model(theta, dt, sensors):
    """Model struct and host theta array of the CT bearings model: three
    parameters (log sigma, log q_c, log q_omega) give both sensors one noise
    level (MODEL_CT_BEARINGS); four (log sqrt(R_11), log q_c, log q_omega,
    log sqrt(R_22)) give one per sensor (MODEL_CT_BEARINGS_R)."""
    import numpy as np
    th = [float(v) for v in np.asarray(theta, dtype=np.float64).reshape(-1)]
    if len(th) not in (3, 4):
        raise ValueError("CT theta has 3 or 4 entries")
    s = (ctypes.c_double * 4)(*[float(v) for v in np.asarray(sensors).reshape(-1)])
    kind = MODEL_CT_BEARINGS if len(th) == 3 else MODEL_CT_BEARINGS_R
    return Model(kind, float(dt), s), (ctypes.c_double * len(th))(*th)


def _offsets(offsets):
    off = [int(v) for v in offsets]
    return (_i64 * len(off))(*off), len(off) - 1


def sqsm_ipls_smooth(ctx, theta, y, offsets, m0, N0, M, linearization=CUBATURE, dt=0.01,
                     sensors=None, init_ms=None, init_Ns=None, ms=None, Ns=None, loglik=None):
    """Call sqsm_ipls_smooth for the CT bearings model.  offsets is a host
    sequence of batch+1 ints; m0 [batch, 5], N0 [batch, 5, 5]."""
    import numpy as np
    dtp = y.dtype
    code = _dtype_code(dtp)
    if sensors is None:
        sensors = np.array([[-1.5, 0.5], [1.0, 1.0]])
    off, batch = _offsets(offsets)
    rows = int(off[batch]) + batch
    dev = y.device
    if ms is None:
        ms = torch.empty((rows, 5), dtype=dtp, device=dev)
    if Ns is None:
        Ns = torch.empty((rows, 5, 5), dtype=dtp, device=dev)
    if loglik is None:
        loglik = torch.empty(batch, dtype=torch.float64, device=dev)
    mdl, th = _ct_model(theta, dt, sensors)
    rc = lib.sqsm_ipls_smooth(ctx.h, code, ctypes.byref(mdl), th, int(linearization), int(M),
                              batch, off, _ptr(y, dtp, "y"), _ptr(m0, dtp, "m0"),
                              _ptr(N0, dtp, "N0"), _ptr(init_ms, dtp, "init_ms"),
                              _ptr(init_Ns, dtp, "init_Ns"), _ptr(ms, dtp, "ms"),
                              _ptr(Ns, dtp, "Ns"), _ptr(loglik, torch.float64, "loglik"),
                              _stream())
    ctx.check(rc)
    return ms, Ns, loglik


def sqsm_ipls_smooth_tol(ctx, theta, y, offsets, m0, N0, max_iters, tol, linearization=CUBATURE,
                         dt=0.01, sensors=None, init_ms=None, init_Ns=None):
    """Call sqsm_ipls_smooth_tol (iterate until the largest change of a
    smoothing mean is below tol, at most max_iters times).  Returns (ms, Ns,
    loglik, iters_done) as device tensors (iters_done int32 [1])."""
    import numpy as np
    dtp = y.dtype
    code = _dtype_code(dtp)
    if sensors is None:
        sensors = np.array([[-1.5, 0.5], [1.0, 1.0]])
    off, batch = _offsets(offsets)
    rows = int(off[batch]) + batch
    dev = y.device
    ms = torch.empty((rows, 5), dtype=dtp, device=dev)
    Ns = torch.empty((rows, 5, 5), dtype=dtp, device=dev)
    loglik = torch.empty(batch, dtype=torch.float64, device=dev)
    iters = torch.zeros(1, dtype=torch.int32, device=dev)
    mdl, th = _ct_model(theta, dt, sensors)
    rc = lib.sqsm_ipls_smooth_tol(ctx.h, code, ctypes.byref(mdl), th, int(linearization),
                                  int(max_iters), float(tol), batch, off, _ptr(y, dtp, "y"),
                                  _ptr(m0, dtp, "m0"), _ptr(N0, dtp, "N0"),
                                  _ptr(init_ms, dtp, "init_ms"), _ptr(init_Ns, dtp, "init_Ns"),
                                  _ptr(ms, dtp, "ms"), _ptr(Ns, dtp, "Ns"),
                                  _ptr(loglik, torch.float64, "loglik"),
                                  _ptr(iters, torch.int32, "iters_done"), _stream())
    ctx.check(rc)
    return ms, Ns, loglik, iters


def sqsm_ipls_smooth_std(ctx, theta, y, offsets, m0, P0, M, linearization=CUBATURE, dt=0.01,
                         sensors=None):
    """Call sqsm_ipls_smooth_std (standard covariance form).  P0 [batch, 5, 5]
    prior covariances.  Returns (ms, Ps, loglik)."""
    import numpy as np
    dtp = y.dtype
    code = _dtype_code(dtp)
    if sensors is None:
        sensors = np.array([[-1.5, 0.5], [1.0, 1.0]])
    off, batch = _offsets(offsets)
    rows = int(off[batch]) + batch
    dev = y.device
    ms = torch.empty((rows, 5), dtype=dtp, device=dev)
    Ps = torch.empty((rows, 5, 5), dtype=dtp, device=dev)
    loglik = torch.empty(batch, dtype=torch.float64, device=dev)
    mdl, th = _ct_model(theta, dt, sensors)
    rc = lib.sqsm_ipls_smooth_std(ctx.h, code, ctypes.byref(mdl), th, int(linearization), int(M),
                                  batch,
                                  off, _ptr(y, dtp, "y"), _ptr(m0, dtp, "m0"),
                                  _ptr(P0, dtp, "P0"), _ptr(ms, dtp, "ms"), _ptr(Ps, dtp, "Ps"),
                                  _ptr(loglik, torch.float64, "loglik"), _stream())
    ctx.check(rc)
    return ms, Ps, loglik


def sqsm_ipls_smooth_population(ctx, theta, y, offsets, m0, N0, M, linearization=CUBATURE,
                                tol=None, max_iters=None):
    """Alg. 3 on the Ricker population model (n_x = n_y = 1), theta =
    (log a, log b, log Q); y [sum n, 1] counts, m0 [B, 1], N0 [B, 1, 1] (0 for
    a known initial state).  With tol set, iterate until convergence (at
    most max_iters, default M).  Returns (ms, Ns, loglik) or, with tol,
    (ms, Ns, loglik, iters_done)."""
    dtp = y.dtype
    code = _dtype_code(dtp)
    off, batch = _offsets(offsets)
    rows = int(off[batch]) + batch
    dev = y.device
    ms = torch.empty((rows, 1), dtype=dtp, device=dev)
    Ns = torch.empty((rows, 1, 1), dtype=dtp, device=dev)
    loglik = torch.empty(batch, dtype=torch.float64, device=dev)
    th = (ctypes.c_double * 3)(*[float(v) for v in theta])
    mdl = Model(MODEL_POPULATION, 1.0, (ctypes.c_double * 4)())
    args = (batch, off, _ptr(y, dtp, "y"), _ptr(m0, dtp, "m0"), _ptr(N0, dtp, "N0"), None, None,
            _ptr(ms, dtp, "ms"), _ptr(Ns, dtp, "Ns"), _ptr(loglik, torch.float64, "loglik"))
    if tol is None:
        ctx.check(lib.sqsm_ipls_smooth(ctx.h, code, ctypes.byref(mdl), th, int(linearization),
                                       int(M), *args, _stream()))
        return ms, Ns, loglik
    iters = torch.zeros(1, dtype=torch.int32, device=dev)
    ctx.check(lib.sqsm_ipls_smooth_tol(ctx.h, code, ctypes.byref(mdl), th, int(linearization),
                                       int(max_iters or M), float(tol), *args,
                                       _ptr(iters, torch.int32, "iters_done"), _stream()))
    return ms, Ns, loglik, iters


def sqsm_ct_linearize(ctx, theta, y, offsets, ms, Ns, linearization=CUBATURE, dt=0.01,
                      sensors=None):
    """Call sqsm_ct_linearize; returns (F, c, SQ, H, d, SR) with a leading
    axis over observation rows."""
    import numpy as np
    dtp = y.dtype
    code = _dtype_code(dtp)
    if sensors is None:
        sensors = np.array([[-1.5, 0.5], [1.0, 1.0]])
    off, batch = _offsets(offsets)
    n = int(off[batch])
    dev = y.device
    out = [torch.empty(s, dtype=dtp, device=dev) for s in
           ((n, 5, 5), (n, 5), (n, 5, 5), (n, 2, 5), (n, 2), (n, 2, 2))]
    mdl, th = _ct_model(theta, dt, sensors)
    rc = lib.sqsm_ct_linearize(ctx.h, code, ctypes.byref(mdl), th, int(linearization), batch, off,
                               _ptr(y, dtp, "y"), _ptr(ms, dtp, "ms"), _ptr(Ns, dtp, "Ns"),
                               *[_ptr(o, dtp) for o in out], _stream())
    ctx.check(rc)
    return tuple(out)


def sqsm_ipls_nll_grad(ctx, theta, y, offsets, m0, N0, M, adj_iters, dt=0.01, sensors=None,
                       init_ms=None, init_Ns=None, ms=None, Ns=None, nll=None, grad=None,
                       change=None, tol=0.0, ipls_change=None, linearization=CUBATURE):
    """Call sqsm_ipls_nll_grad (any SLR rule).  Returns (nll, grad, change, ms,
    Ns) as device tensors (nll [1], grad [len(theta)], change [1] float64).
    tol > 0 sets ERR_NOT_CONVERGED in the status word when a fixed point has
    not settled; ipls_change (float64 [1], optional) receives the relative
    change of the trajectory in one more iteration of Alg. 3."""
    import numpy as np
    dtp = y.dtype
    code = _dtype_code(dtp)
    if sensors is None:
        sensors = np.array([[-1.5, 0.5], [1.0, 1.0]])
    off, batch = _offsets(offsets)
    rows = int(off[batch]) + batch
    dev = y.device
    if ms is None:
        ms = torch.empty((rows, 5), dtype=dtp, device=dev)
    if Ns is None:
        Ns = torch.empty((rows, 5, 5), dtype=dtp, device=dev)
    f64 = torch.float64
    nll = torch.empty(1, dtype=f64, device=dev) if nll is None else nll
    change = torch.empty(1, dtype=f64, device=dev) if change is None else change
    mdl, th = _ct_model(theta, dt, sensors)
    grad = torch.empty(len(th), dtype=f64, device=dev) if grad is None else grad
    rc = lib.sqsm_ipls_nll_grad(ctx.h, code, ctypes.byref(mdl), th, int(linearization), int(M),
                                int(adj_iters),
                                float(tol), batch, off, _ptr(y, dtp, "y"), _ptr(m0, dtp, "m0"),
                                _ptr(N0, dtp, "N0"), _ptr(init_ms, dtp, "init_ms"),
                                _ptr(init_Ns, dtp, "init_Ns"), _ptr(ms, dtp, "ms"),
                                _ptr(Ns, dtp, "Ns"), _ptr(nll, f64, "nll"), _ptr(grad, f64, "grad"),
                                _ptr(change, f64, "change"), _ptr(ipls_change, f64, "ipls_change"),
                                _stream())
    ctx.check(rc)
    return nll, grad, change, ms, Ns


def fp32_fma_probe(iters, blocks, threads, out):
    """Enqueue the FP32 FMA-pipe probe on the current stream; out is a
    float32 CUDA tensor of blocks * threads elements.  Returns the probe's
    floating-point operation count."""
    if out.numel() < blocks * threads:
        raise ValueError("out holds fewer than blocks * threads floats")
    fl = ctypes.c_double(0.0)
    rc = lib.sqsm_fp32_fma_probe(int(iters), int(blocks), int(threads),
                                 _ptr(out, torch.float32, "out"), ctypes.byref(fl), _stream())
    if rc != OK:
        raise SqsmError(rc, "sqsm_fp32_fma_probe failed")
    return fl.value
