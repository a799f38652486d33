"""Thin ctypes binding of liblsgcpd (include/lsgcpd.h).

Argument marshalling only: every step of the method runs in the CUDA library.
Functions carry the C names; ``Context`` bundles them for convenience.  Device
arrays are torch CUDA tensors (float32, contiguous); host arrays may be numpy
arrays or CPU tensors (``lsgcpd_register`` accepts either for X and Y).
There is no CPU fallback: if the library cannot be built or loaded, the first
call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

MOMENTS = 76
TRACE_WIDTH = 8
PER_N_WIDTH = 16

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ENUMERIC"}


class LsgcpdError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Params(C.Structure):
    _fields_ = [
        ("w", C.c_double), ("alpha_max", C.c_double), ("lam", C.c_double), ("tol", C.c_double),
        ("volume", C.c_double), ("sigma2_init", C.c_double), ("init_R", C.c_double * 9),
        ("init_t", C.c_double * 3), ("newton_tol", C.c_double), ("sigma2_floor_rel", C.c_double),
        ("knn_k", C.c_int32), ("max_iters", C.c_int32), ("include_alpha_norm", C.c_int32),
        ("newton_max", C.c_int32), ("precision", C.c_int32), ("knn_method", C.c_int32),
        ("eta", C.c_double), ("cf_threshold", C.c_double), ("nll_tol", C.c_double),
        ("phi_x", C.c_void_p), ("phi_y", C.c_void_p),
    ]


class Result(C.Structure):
    _fields_ = [("R", C.c_double * 9), ("t", C.c_double * 3), ("sigma2", C.c_double),
                ("iters", C.c_int32), ("mode", C.c_int32), ("ms_estep", C.c_double),
                ("ms_total", C.c_double)]


_lib = None


def lib():
    """Load (building first if needed) the CUDA library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp, dp, fp, ip = C.c_void_p, C.POINTER(C.c_double), C.c_void_p, C.c_void_p
        i64 = C.c_int64
        L.lsgcpd_params_default.argtypes = [C.POINTER(Params)]
        L.lsgcpd_params_default.restype = None
        L.lsgcpd_create.argtypes = [C.POINTER(vp), C.c_int, i64, i64]
        L.lsgcpd_create.restype = C.c_int
        L.lsgcpd_destroy.argtypes = [vp]
        L.lsgcpd_destroy.restype = None
        L.lsgcpd_last_error.argtypes = [vp]
        L.lsgcpd_last_error.restype = C.c_char_p
        L.lsgcpd_set_timing.argtypes = [vp, C.c_int]
        L.lsgcpd_set_timing.restype = C.c_int
        L.lsgcpd_last_timing.argtypes = [vp, dp]
        L.lsgcpd_last_timing.restype = C.c_int
        L.lsgcpd_preprocess.argtypes = [vp, fp, i64, C.POINTER(Params), fp, fp, fp, ip, vp]
        L.lsgcpd_preprocess.restype = C.c_int
        L.lsgcpd_estep.argtypes = [vp, fp, i64, fp, fp, fp, i64, C.POINTER(Params), dp, dp, C.c_double,
                                   C.c_double, dp, fp, vp]
        L.lsgcpd_estep.restype = C.c_int
        L.lsgcpd_mstep.argtypes = [vp, dp, dp, dp, C.POINTER(Params), dp, dp, dp, C.POINTER(C.c_int32), vp]
        L.lsgcpd_mstep.restype = C.c_int
        L.lsgcpd_register.argtypes = [vp, fp, i64, fp, i64, C.POINTER(Params), C.POINTER(Result), dp, vp]
        L.lsgcpd_register.restype = C.c_int
        L.lsgcpd_register_batch.argtypes = [vp, C.c_int32, fp, C.POINTER(i64), fp, C.POINTER(i64),
                                            C.POINTER(Params), dp, dp, dp, C.POINTER(C.c_int32), dp, vp]
        L.lsgcpd_register_batch.restype = C.c_int
        L.lsgcpd_posteriors.argtypes = [vp, fp, i64, fp, fp, fp, i64, C.POINTER(Params), dp, dp, C.c_double,
                                        C.c_double, fp, vp]
        L.lsgcpd_posteriors.restype = C.c_int
        L.lsgcpd_selftest_timeout.argtypes = [vp, i64]
        L.lsgcpd_selftest_timeout.restype = C.c_int
        L.lsgcpd_set_autotune.argtypes = [vp, C.c_int]
        L.lsgcpd_set_autotune.restype = C.c_int
        L.lsgcpd_plan_info.argtypes = [vp, C.POINTER(C.c_int32), dp]
        L.lsgcpd_plan_info.restype = C.c_int
        L.lsgcpd_autotune_save.argtypes = [vp, C.c_char_p]
        L.lsgcpd_autotune_save.restype = C.c_int
        L.lsgcpd_autotune_load.argtypes = [vp, C.c_char_p, C.POINTER(C.c_int32)]
        L.lsgcpd_autotune_load.restype = C.c_int
        L.lsgcpd_estep_noalloc.argtypes = [fp, i64, fp, fp, fp, i64, C.POINTER(Params), dp, dp, C.c_double,
                                           C.c_double, dp, fp, vp]
        L.lsgcpd_estep_noalloc.restype = C.c_int
        _lib = L
    return _lib


def library_path():
    return os.path.abspath(_build.LIB)


def default_params(**kw) -> Params:
    p = Params()
    lib().lsgcpd_params_default(C.byref(p))
    for key, val in kw.items():
        if key in ("init_R", "init_t"):
            arr = np.asarray(val, dtype=np.float64).ravel()
            dst = getattr(p, key)
            for i, v in enumerate(arr):
                dst[i] = float(v)
        elif key == "lambda":
            p.lam = float(val)
        else:
            setattr(p, key, val)
    return p


def _dev_ptr(t, name, shape=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32 and t.dtype != torch.int32:
        raise TypeError(f"{name} must be float32 (or int32 for indices)")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return C.c_void_p(t.data_ptr())


def _any_ptr(a, name):
    """Pointer to a float32 N x 3 array on host (numpy / CPU tensor) or device (CUDA tensor)."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float32 or not a.is_contiguous() or a.dim() != 2 or a.shape[1] != 3:
                raise ValueError(f"{name} must be a contiguous float32 n x 3 tensor")
            return C.c_void_p(a.data_ptr()), a.shape[0], a
    except ImportError:  # pragma: no cover
        pass
    arr = np.ascontiguousarray(a, dtype=np.float32)
    if arr.ndim != 2 or arr.shape[1] != 3:
        raise ValueError(f"{name} must be n x 3")
    return C.c_void_p(arr.ctypes.data), arr.shape[0], arr


def _vec_ptr(a, name, n):
    """Pointer to a float32 vector of n values on host (numpy / CPU tensor) or device (CUDA tensor)."""
    if a is None:
        return None, None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float32 or not a.is_contiguous() or a.numel() != n:
                raise ValueError(f"{name} must be a contiguous float32 tensor of {n} values")
            return a.data_ptr(), a
    except ImportError:  # pragma: no cover
        pass
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float32).ravel())
    if arr.size != n:
        raise ValueError(f"{name} must have {n} values")
    return arr.ctypes.data, arr


class _Confidences:
    """Sets params.phi_x / phi_y for the duration of one call (and keeps the arrays alive)."""

    def __init__(self, params, phi_x, n, phi_y, m):
        self.params = params
        self.px, self.kx = _vec_ptr(phi_x, "phi_x", n)
        self.py, self.ky = _vec_ptr(phi_y, "phi_y", m)

    def __enter__(self):
        self.old = (self.params.phi_x, self.params.phi_y)
        self.params.phi_x = self.px
        self.params.phi_y = self.py
        return self.params

    def __exit__(self, *exc):
        self.params.phi_x, self.params.phi_y = self.old
        return False


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(int(stream))


def _d(arr, n):
    a = np.ascontiguousarray(np.asarray(arr, dtype=np.float64).ravel())
    if a.size != n:
        raise ValueError(f"expected {n} values")
    return a


def _check(ctx, rc):
    if rc != 0:
        msg = lib().lsgcpd_last_error(ctx).decode(errors="replace")
        raise LsgcpdError(rc, msg)


def lsgcpd_create(device=0, max_N=1, max_M=1):
    h = C.c_void_p()
    rc = lib().lsgcpd_create(C.byref(h), int(device), int(max_N), int(max_M))
    if rc != 0:
        raise LsgcpdError(rc, "lsgcpd_create failed")
    return h


def lsgcpd_destroy(ctx):
    lib().lsgcpd_destroy(ctx)


def lsgcpd_preprocess(ctx, Y, params, want_idx=False, stream=None):
    import torch
    M = Y.shape[0]
    _dev_ptr(Y, "Y", (M, 3))
    dev = Y.device
    normals = torch.empty((M, 3), dtype=torch.float32, device=dev)
    kappa = torch.empty(M, dtype=torch.float32, device=dev)
    alpha = torch.empty(M, dtype=torch.float32, device=dev)
    idx = torch.empty((M, params.knn_k), dtype=torch.int32, device=dev) if want_idx else None
    rc = lib().lsgcpd_preprocess(ctx, C.c_void_p(Y.data_ptr()), M, C.byref(params),
                                 C.c_void_p(normals.data_ptr()), C.c_void_p(kappa.data_ptr()),
                                 C.c_void_p(alpha.data_ptr()),
                                 C.c_void_p(idx.data_ptr()) if idx is not None else None, _stream(stream))
    _check(ctx, rc)
    return dict(normals=normals, kappa=kappa, alpha=alpha, idx=idx)


def lsgcpd_estep(ctx, X, Y, normals, alpha, R, t, sigma2, volume, params, per_n=False, stream=None, phi_x=None,
                 phi_y=None):
    import torch
    N, M = X.shape[0], Y.shape[0]
    with _Confidences(params, phi_x, N, phi_y, M) as params:
        return _estep(ctx, X, Y, normals, alpha, R, t, sigma2, volume, params, per_n, stream, N, M)


def _estep(ctx, X, Y, normals, alpha, R, t, sigma2, volume, params, per_n, stream, N, M):
    import torch
    _dev_ptr(X, "X", (N, 3))
    _dev_ptr(Y, "Y", (M, 3))
    _dev_ptr(normals, "normals", (M, 3))
    _dev_ptr(alpha, "alpha", (M,))
    Rd, td = _d(R, 9), _d(t, 3)
    mom = np.zeros(MOMENTS)
    pn = torch.empty((N, PER_N_WIDTH), dtype=torch.float32, device=X.device) if per_n else None
    dpp = C.POINTER(C.c_double)
    rc = lib().lsgcpd_estep(ctx, C.c_void_p(X.data_ptr()), N, C.c_void_p(Y.data_ptr()),
                            C.c_void_p(normals.data_ptr()), C.c_void_p(alpha.data_ptr()), M,
                            C.byref(params), Rd.ctypes.data_as(dpp), td.ctypes.data_as(dpp), float(sigma2),
                            float(volume), mom.ctypes.data_as(dpp),
                            C.c_void_p(pn.data_ptr()) if pn is not None else None, _stream(stream))
    _check(ctx, rc)
    return dict(moments=mom, per_n=pn)


def lsgcpd_estep_noalloc(X, Y, normals, alpha, R, t, sigma2, volume, params, per_n=False, stream=None):
    """The E step without a context and without any device allocation by the library
    (fixed-size static scratch; see lsgcpd.h).  `per_n`, if requested, is allocated
    here by torch, i.e. by the caller."""
    import torch
    N, M = X.shape[0], Y.shape[0]
    _dev_ptr(X, "X", (N, 3))
    _dev_ptr(Y, "Y", (M, 3))
    _dev_ptr(normals, "normals", (M, 3))
    _dev_ptr(alpha, "alpha", (M,))
    Rd, td = _d(R, 9), _d(t, 3)
    mom = np.zeros(MOMENTS)
    pn = torch.empty((N, PER_N_WIDTH), dtype=torch.float32, device=X.device) if per_n else None
    dpp = C.POINTER(C.c_double)
    rc = lib().lsgcpd_estep_noalloc(C.c_void_p(X.data_ptr()), N, C.c_void_p(Y.data_ptr()),
                                    C.c_void_p(normals.data_ptr()), C.c_void_p(alpha.data_ptr()), M,
                                    C.byref(params), Rd.ctypes.data_as(dpp), td.ctypes.data_as(dpp),
                                    float(sigma2), float(volume), mom.ctypes.data_as(dpp),
                                    C.c_void_p(pn.data_ptr()) if pn is not None else None, _stream(stream))
    if rc != 0:
        raise LsgcpdError(rc, "lsgcpd_estep_noalloc failed")
    return dict(moments=mom, per_n=pn)


def lsgcpd_mstep(ctx, moments, R, t, params, stream=None):
    m = _d(moments, MOMENTS)
    Rd, td = _d(R, 9), _d(t, 3)
    Ro = np.zeros(9)
    to = np.zeros(3)
    s2 = C.c_double(0)
    info = (C.c_int32 * 4)()
    dpp = C.POINTER(C.c_double)
    rc = lib().lsgcpd_mstep(ctx, m.ctypes.data_as(dpp), Rd.ctypes.data_as(dpp), td.ctypes.data_as(dpp),
                            C.byref(params), Ro.ctypes.data_as(dpp), to.ctypes.data_as(dpp), C.byref(s2),
                            info, _stream(stream))
    _check(ctx, rc)
    return dict(R=Ro.reshape(3, 3), t=to, sigma2=s2.value, newton_iters=info[0], damped=info[1],
                halvings=info[2])


def lsgcpd_register(ctx, X, Y, params, trace=False, stream=None, phi_x=None, phi_y=None):
    """phi_x / phi_y: optional confidences (Sec. 3.3), in the same memory (host / device) as X / Y."""
    xp, N, _xk = _any_ptr(X, "X")
    yp, M, _yk = _any_ptr(Y, "Y")
    res = Result()
    tr = np.zeros((max(params.max_iters, 1), TRACE_WIDTH)) if trace else None
    with _Confidences(params, phi_x, N, phi_y, M) as pp:
        rc = lib().lsgcpd_register(ctx, xp, N, yp, M, C.byref(pp), C.byref(res),
                                   tr.ctypes.data_as(C.POINTER(C.c_double)) if tr is not None else None,
                                   _stream(stream))
    _check(ctx, rc)
    out = dict(R=np.array(res.R[:]).reshape(3, 3), t=np.array(res.t[:]), sigma2=res.sigma2,
               iters=res.iters, mode=res.mode, ms_estep=res.ms_estep, ms_total=res.ms_total)
    if tr is not None:
        out["trace"] = tr[: res.iters]
    return out


def lsgcpd_register_batch(ctx, X, n_off, Y, m_off, params, trace=False, stream=None, phi_x=None, phi_y=None):
    """Register every pair i: X[n_off[i]:n_off[i+1]] onto Y[m_off[i]:m_off[i+1]].
    phi_x / phi_y: optional confidences with the same offsets and memory as X / Y."""
    xp, _N, _xk = _any_ptr(X, "X")
    yp, _M, _yk = _any_ptr(Y, "Y")
    no = np.ascontiguousarray(np.asarray(n_off, dtype=np.int64))
    mo = np.ascontiguousarray(np.asarray(m_off, dtype=np.int64))
    P = no.size - 1
    if P < 1 or mo.size != P + 1:
        raise ValueError("n_off and m_off need num_pairs + 1 entries each")
    if no[-1] != _N or mo[-1] != _M:
        raise ValueError("the last offsets must equal the row counts of X and Y")
    R = np.zeros((P, 3, 3))
    t = np.zeros((P, 3))
    s2 = np.zeros(P)
    it = np.zeros(P, dtype=np.int32)
    tr = np.zeros((P, max(params.max_iters, 1), TRACE_WIDTH)) if trace else None
    dptr = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    with _Confidences(params, phi_x, int(_N), phi_y, int(_M)) as pp:
        rc = lib().lsgcpd_register_batch(ctx, P, xp, no.ctypes.data_as(C.POINTER(C.c_int64)), yp,
                                         mo.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(pp), dptr(R),
                                         dptr(t), dptr(s2), it.ctypes.data_as(C.POINTER(C.c_int32)),
                                         dptr(tr) if tr is not None else None, _stream(stream))
    _check(ctx, rc)
    out = dict(R=R, t=t, sigma2=s2, iters=it)
    if tr is not None:
        out["trace"] = tr
    return out


def lsgcpd_posteriors(ctx, X, Y, normals, alpha, R, t, sigma2, volume, params, stream=None, phi_x=None,
                      phi_y=None):
    """Dense posteriors (M + 1) x N of one E step (outlier row last), as a CUDA tensor."""
    import torch
    N, M = X.shape[0], Y.shape[0]
    _dev_ptr(X, "X", (N, 3))
    _dev_ptr(Y, "Y", (M, 3))
    _dev_ptr(normals, "normals", (M, 3))
    _dev_ptr(alpha, "alpha", (M,))
    Rd, td = _d(R, 9), _d(t, 3)
    P = torch.empty((M + 1, N), dtype=torch.float32, device=X.device)
    dpp = C.POINTER(C.c_double)
    with _Confidences(params, phi_x, N, phi_y, M) as pp:
        rc = lib().lsgcpd_posteriors(ctx, C.c_void_p(X.data_ptr()), N, C.c_void_p(Y.data_ptr()),
                                     C.c_void_p(normals.data_ptr()), C.c_void_p(alpha.data_ptr()), M, C.byref(pp),
                                     Rd.ctypes.data_as(dpp), td.ctypes.data_as(dpp), float(sigma2), float(volume),
                                     C.c_void_p(P.data_ptr()), _stream(stream))
    _check(ctx, rc)
    return P


def lsgcpd_selftest_timeout(ctx, budget_cycles):
    """Status code of the bounded-wait diagnostic (LSGCPD_ETIMEOUT = 4 is the expected result)."""
    return int(lib().lsgcpd_selftest_timeout(ctx, int(budget_cycles)))


def lsgcpd_set_autotune(ctx, enable):
    _check(ctx, lib().lsgcpd_set_autotune(ctx, 1 if enable else 0))


def lsgcpd_autotune_save(ctx, path):
    _check(ctx, lib().lsgcpd_autotune_save(ctx, str(path).encode()))


def lsgcpd_autotune_load(ctx, path):
    """Entries of a saved autotune file (this device) added to the context; returns their count."""
    n = C.c_int32(0)
    _check(ctx, lib().lsgcpd_autotune_load(ctx, str(path).encode(), C.byref(n)))
    return int(n.value)


def lsgcpd_plan_info(ctx):
    info = np.zeros(4, dtype=np.int32)
    ms = np.zeros(3)
    _check(ctx, lib().lsgcpd_plan_info(ctx, info.ctypes.data_as(C.POINTER(C.c_int32)),
                                       ms.ctypes.data_as(C.POINTER(C.c_double))))
    return dict(sources_per_thread=int(info[0]), block=int(info[1]), ctas=int(info[2]), tuned=bool(info[3]),
                tune_ms={4: ms[0], 2: ms[1], 1: ms[2]})


def lsgcpd_set_timing(ctx, enable):
    lib().lsgcpd_set_timing(ctx, 1 if enable else 0)


def lsgcpd_last_timing(ctx):
    out = np.zeros(8)
    lib().lsgcpd_last_timing(ctx, out.ctypes.data_as(C.POINTER(C.c_double)))
    return dict(ms_total=out[0], ms_estep=out[1], ms_combine=out[2], ms_mstep=out[3], ms_prep=out[4],
                launches=int(out[5]), h2d_bytes=int(out[6]), d2h_bytes=int(out[7]))


class Context:
    """One device context of the library (scratch memory, graphs, events)."""

    def __init__(self, device=0, max_n=1, max_m=1):
        self.handle = lsgcpd_create(device, max_n, max_m)

    def close(self):
        if self.handle:
            lsgcpd_destroy(self.handle)
            self.handle = None

    def __del__(self):  # pragma: no cover - interpreter shutdown order
        try:
            self.close()
        except Exception:
            pass

    def preprocess(self, Y, params, want_idx=False, stream=None):
        return lsgcpd_preprocess(self.handle, Y, params, want_idx, stream)

    def estep(self, X, Y, normals, alpha, R, t, sigma2, volume, params, per_n=False, stream=None, phi_x=None,
              phi_y=None):
        return lsgcpd_estep(self.handle, X, Y, normals, alpha, R, t, sigma2, volume, params, per_n, stream,
                            phi_x, phi_y)

    def mstep(self, moments, R, t, params, stream=None):
        return lsgcpd_mstep(self.handle, moments, R, t, params, stream)

    def register(self, X, Y, params, trace=False, stream=None, phi_x=None, phi_y=None):
        return lsgcpd_register(self.handle, X, Y, params, trace, stream, phi_x, phi_y)

    def register_batch(self, X, n_off, Y, m_off, params, trace=False, stream=None, phi_x=None, phi_y=None):
        return lsgcpd_register_batch(self.handle, X, n_off, Y, m_off, params, trace, stream, phi_x, phi_y)

    def posteriors(self, X, Y, normals, alpha, R, t, sigma2, volume, params, stream=None, phi_x=None, phi_y=None):
        return lsgcpd_posteriors(self.handle, X, Y, normals, alpha, R, t, sigma2, volume, params, stream, phi_x,
                                 phi_y)

    def selftest_timeout(self, budget_cycles):
        return lsgcpd_selftest_timeout(self.handle, budget_cycles)

    def set_autotune(self, enable):
        lsgcpd_set_autotune(self.handle, enable)

    def plan_info(self):
        return lsgcpd_plan_info(self.handle)

    def autotune_save(self, path):
        lsgcpd_autotune_save(self.handle, path)

    def autotune_load(self, path):
        return lsgcpd_autotune_load(self.handle, path)

    def set_timing(self, enable):
        lsgcpd_set_timing(self.handle, enable)

    def last_timing(self):
        return lsgcpd_last_timing(self.handle)
