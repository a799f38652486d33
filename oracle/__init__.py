"""ctypes access to the FP64 LSG-CPD oracle (TEST INFRASTRUCTURE ONLY).

The oracle is a plain CPU restatement of the paper's method (see
``lsgcpd_oracle.cpp`` for the equations and the readings of ambiguous
passages).  Only the test suite, the smoke check and the benchmark's CPU
baseline may import this package; the product path never does.

All inputs are FP32 clouds (the values the GPU sees), up-cast to double
inside.  Arrays are numpy, C-contiguous.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

STAT_WIDTH = 15  # Pbar, ybar[3], W[6], b[3], f, Pout


class OracleParams(C.Structure):
    _fields_ = [
        ("w", C.c_double), ("alpha_max", C.c_double), ("lam", C.c_double), ("tol", C.c_double),
        ("volume", C.c_double), ("sigma2_init", C.c_double), ("init_R", C.c_double * 9),
        ("init_t", C.c_double * 3), ("newton_tol", C.c_double), ("sigma2_floor_rel", C.c_double),
        ("knn_k", C.c_int32), ("max_iters", C.c_int32), ("include_alpha_norm", C.c_int32),
        ("newton_max", C.c_int32), ("threads", C.c_int32), ("pad_", C.c_int32),
        ("eta", C.c_double), ("cf_threshold", C.c_double), ("nll_tol", C.c_double),
        ("phi_x", C.POINTER(C.c_float)), ("phi_y", C.POINTER(C.c_float)),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        fp = C.POINTER(C.c_float)
        ip = C.POINTER(C.c_int32)
        i64 = C.c_int64
        L.oracle_knn.argtypes = [fp, i64, C.c_int32, C.c_int32, ip]
        L.oracle_knn_grid.argtypes = [fp, i64, C.c_int32, C.c_int32, ip]
        L.oracle_knn_subset.argtypes = [fp, i64, C.POINTER(C.c_int64), i64, C.c_int32, C.c_int32, ip]
        L.oracle_jacobi3.argtypes = [dp, dp, dp]
        L.oracle_penalty.argtypes = [C.c_double] * 3
        L.oracle_penalty.restype = C.c_double
        L.oracle_local_geometry.argtypes = [fp, i64, ip, C.c_int32, C.c_double, C.c_double, dp, dp, dp]
        L.oracle_volume.argtypes = [fp, i64, dp]
        L.oracle_volume.restype = C.c_double
        L.oracle_sigma2_init.argtypes = [fp, i64, fp, i64, dp, dp]
        L.oracle_sigma2_init.restype = C.c_double
        L.oracle_estep.argtypes = [fp, i64, fp, i64, dp, dp, dp, dp, C.c_double, C.c_double, dp, dp,
                                   C.c_double, C.c_int32, C.c_int32, dp, dp, dp]
        L.oracle_objective.argtypes = [dp, fp, i64, dp, dp]
        L.oracle_objective.restype = C.c_double
        L.oracle_grad_hess.argtypes = [dp, fp, i64, dp, dp, dp, dp]
        L.oracle_grad_hess_direct.argtypes = [fp, i64, fp, i64, dp, dp, dp, dp, dp, C.c_double, dp, dp]
        L.oracle_se3_exp.argtypes = [dp, dp]
        L.oracle_mstep.argtypes = [dp, fp, i64, dp, dp, C.c_int32, C.c_double, dp, dp, dp, dp, ip]
        L.oracle_register.argtypes = [fp, i64, fp, i64, C.POINTER(OracleParams), dp, dp, dp, ip, dp,
                                      dp, dp]
        L.oracle_w_from_eta.argtypes = [C.c_double, C.c_double, C.c_double, dp, dp, i64, C.c_int32]
        L.oracle_w_from_eta.restype = C.c_double
        _lib = L
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a, t):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(t))


def knn(Y, k, threads=0, method="auto"):
    """k nearest targets of every target (self included, ties to the lower index).
    method: "brute" (O(M^2)), "grid" (exact uniform-grid search, same result) or
    "auto" (grid above 20,000 points)."""
    Y = _f32(Y)
    M = len(Y)
    idx = np.empty((M, k), dtype=np.int32)
    use_grid = method == "grid" or (method == "auto" and M > 20000)
    fn = lib().oracle_knn_grid if use_grid else lib().oracle_knn
    rc = fn(_p(Y, C.c_float), M, k, threads, _p(idx, C.c_int32))
    if rc:
        raise ValueError("oracle_knn: invalid arguments")
    return idx


def knn_rows(Y, queries, k, threads=0):
    """Brute-force k nearest targets of the listed queries (the corresponding rows of knn)."""
    Y = _f32(Y)
    q = np.ascontiguousarray(queries, dtype=np.int64)
    idx = np.empty((len(q), k), dtype=np.int32)
    rc = lib().oracle_knn_subset(_p(Y, C.c_float), len(Y), _p(q, C.c_int64), len(q), k, threads,
                                 _p(idx, C.c_int32))
    if rc:
        raise ValueError("oracle_knn_subset: invalid arguments")
    return idx


def jacobi3(Cm):
    Cm = _f64(Cm).reshape(3, 3)
    ev = np.empty(3)
    vec = np.empty((3, 3))
    lib().oracle_jacobi3(_p(Cm, C.c_double), _p(ev, C.c_double), _p(vec, C.c_double))
    return ev, vec


def penalty(kappa, alpha_max, lam):
    return lib().oracle_penalty(float(kappa), float(alpha_max), float(lam))


def local_geometry(Y, idx, alpha_max, lam):
    Y = _f32(Y)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    M, k = idx.shape
    nrm = np.empty((M, 3))
    kap = np.empty(M)
    alp = np.empty(M)
    rc = lib().oracle_local_geometry(_p(Y, C.c_float), M, _p(idx, C.c_int32), k, float(alpha_max),
                                     float(lam), _p(nrm, C.c_double), _p(kap, C.c_double),
                                     _p(alp, C.c_double))
    if rc:
        raise ValueError("oracle_local_geometry: invalid arguments")
    return nrm, kap, alp


def preprocess(Y, k, alpha_max, lam, threads=0):
    idx = knn(Y, k, threads)  # grid search above 20,000 targets (same result)
    nrm, kap, alp = local_geometry(Y, idx, alpha_max, lam)
    return dict(idx=idx, normals=nrm, kappa=kap, alpha=alp)


def volume(Y):
    Y = _f32(Y)
    d = C.c_double(0)
    V = lib().oracle_volume(_p(Y, C.c_float), len(Y), C.byref(d))
    return V, d.value


def sigma2_init(X, Y, R, t):
    X, Y = _f32(X), _f32(Y)
    R, t = _f64(R).ravel(), _f64(t).ravel()
    return lib().oracle_sigma2_init(_p(X, C.c_float), len(X), _p(Y, C.c_float), len(Y),
                                    _p(R, C.c_double), _p(t, C.c_double))


def estep(X, Y, normals, alpha, R, t, sigma2, w, V, pi_m=None, w_n=None, include_alpha_norm=False,
          dense=False, threads=0):
    """Returns dict(stats [N x 15], nll, P [M x N] if dense)."""
    X, Y = _f32(X), _f32(Y)
    nrm, alp = _f64(normals), _f64(alpha)
    R, t = _f64(R).ravel(), _f64(t).ravel()
    N, M = len(X), len(Y)
    stats = np.empty((N, STAT_WIDTH))
    P = np.empty((M, N)) if dense else None
    nll = C.c_double(0)
    pi_a = _f64(pi_m) if pi_m is not None else None
    w_a = _f64(w_n) if w_n is not None else None
    rc = lib().oracle_estep(_p(X, C.c_float), N, _p(Y, C.c_float), M, _p(nrm, C.c_double),
                            _p(alp, C.c_double), _p(pi_a, C.c_double), _p(w_a, C.c_double), float(w),
                            float(V), _p(R, C.c_double), _p(t, C.c_double), float(sigma2),
                            int(include_alpha_norm), threads, _p(stats, C.c_double),
                            _p(P, C.c_double), C.byref(nll))
    if rc:
        raise ValueError("oracle_estep: invalid arguments")
    out = dict(stats=stats, nll=nll.value)
    if dense:
        out["P"] = P
    return out


def objective(stats, X, R, t):
    stats, X = _f64(stats), _f32(X)
    R, t = _f64(R).ravel(), _f64(t).ravel()
    return lib().oracle_objective(_p(stats, C.c_double), _p(X, C.c_float), len(X), _p(R, C.c_double),
                                  _p(t, C.c_double))


def grad_hess(stats, X, R, t):
    stats, X = _f64(stats), _f32(X)
    R, t = _f64(R).ravel(), _f64(t).ravel()
    g = np.empty(6)
    H = np.empty((6, 6))
    lib().oracle_grad_hess(_p(stats, C.c_double), _p(X, C.c_float), len(X), _p(R, C.c_double),
                           _p(t, C.c_double), _p(g, C.c_double), _p(H, C.c_double))
    return g, H


def grad_hess_direct(X, Y, normals, alpha, P, R, t, sigma2):
    X, Y = _f32(X), _f32(Y)
    nrm, alp, P = _f64(normals), _f64(alpha), _f64(P)
    R, t = _f64(R).ravel(), _f64(t).ravel()
    g = np.empty(6)
    H = np.empty((6, 6))
    lib().oracle_grad_hess_direct(_p(X, C.c_float), len(X), _p(Y, C.c_float), len(Y),
                                  _p(nrm, C.c_double), _p(alp, C.c_double), _p(P, C.c_double),
                                  _p(R, C.c_double), _p(t, C.c_double), float(sigma2),
                                  _p(g, C.c_double), _p(H, C.c_double))
    return g, H


def se3_exp(xi):
    xi = _f64(xi).ravel()
    T = np.empty((4, 4))
    lib().oracle_se3_exp(_p(xi, C.c_double), _p(T, C.c_double))
    return T


def mstep(stats, X, R, t, newton_max=20, newton_tol=1e-12):
    stats, X = _f64(stats), _f32(X)
    R, t = _f64(R).ravel(), _f64(t).ravel()
    Ro = np.empty(9)
    to = np.empty(3)
    s2 = C.c_double(0)
    Q = C.c_double(0)
    info = np.zeros(4, dtype=np.int32)
    rc = lib().oracle_mstep(_p(stats, C.c_double), _p(X, C.c_float), len(X), _p(R, C.c_double),
                            _p(t, C.c_double), int(newton_max), float(newton_tol),
                            _p(Ro, C.c_double), _p(to, C.c_double), C.byref(s2), C.byref(Q),
                            _p(info, C.c_int32))
    return dict(R=Ro.reshape(3, 3), t=to, sigma2=s2.value, Q=Q.value, newton_iters=int(info[0]),
                damped=int(info[1]), halvings=int(info[2]), rc=rc)


def default_params(**kw):
    """Parameter block with the defaults used across the repository."""
    p = OracleParams()
    p.w = 0.1
    p.alpha_max = 2.0
    p.lam = 0.2
    p.tol = 0.0
    p.volume = 0.0
    p.sigma2_init = 0.0
    for i in range(9):
        p.init_R[i] = 1.0 if i % 4 == 0 else 0.0
    for i in range(3):
        p.init_t[i] = 0.0
    p.newton_tol = 1e-12
    p.sigma2_floor_rel = 1e-10
    p.knn_k = 10
    p.max_iters = 50
    p.include_alpha_norm = 0
    p.newton_max = 20
    p.threads = 0
    p.eta = 0.0
    p.cf_threshold = 0.0
    p.nll_tol = 0.0
    for key, val in kw.items():
        if key == "init_R":
            for i, v in enumerate(np.asarray(val, dtype=np.float64).ravel()):
                p.init_R[i] = v
        elif key == "init_t":
            for i, v in enumerate(np.asarray(val, dtype=np.float64).ravel()):
                p.init_t[i] = v
        else:
            setattr(p, key, val)
    return p


def w_from_eta(eta, V, sigma2, alpha=None, pi_m=None, M=None, include_alpha_norm=False):
    """w_max of Sec. 3.2 (reading R14)."""
    a = None if alpha is None else _f64(alpha)
    pi = None if pi_m is None else _f64(pi_m)
    M = M if M is not None else len(a if a is not None else pi)
    return lib().oracle_w_from_eta(float(eta), float(V), float(sigma2), _p(a, C.c_double), _p(pi, C.c_double),
                                   int(M), int(include_alpha_norm))


def register(X, Y, params=None, phi_x=None, phi_y=None, **kw):
    """Full LSG-CPD registration; returns dict(R, t, sigma2, iters, trace, normals, alpha, rc).
    phi_x / phi_y: optional per-point confidences of Sec. 3.3 (with cf_threshold, eta in kw)."""
    p = params if params is not None else default_params(**kw)
    X, Y = _f32(X), _f32(Y)
    keep = []
    if phi_x is not None:
        keep.append(_f32(phi_x))
        p.phi_x = _p(keep[-1], C.c_float)
    if phi_y is not None:
        keep.append(_f32(phi_y))
        p.phi_y = _p(keep[-1], C.c_float)
    Ro = np.empty(9)
    to = np.empty(3)
    s2 = C.c_double(0)
    it = C.c_int32(0)
    trace = np.zeros((max(p.max_iters, 1), 8))
    nrm = np.empty((len(Y), 3))
    alp = np.empty(len(Y))
    rc = lib().oracle_register(_p(X, C.c_float), len(X), _p(Y, C.c_float), len(Y), C.byref(p),
                               _p(Ro, C.c_double), _p(to, C.c_double), C.byref(s2), C.byref(it),
                               _p(trace, C.c_double), _p(nrm, C.c_double), _p(alp, C.c_double))
    if rc == 1:
        raise ValueError("oracle_register: invalid arguments")
    return dict(R=Ro.reshape(3, 3), t=to, sigma2=s2.value, iters=it.value, trace=trace[: it.value],
                normals=nrm, alpha=alp, rc=rc)


def rotation_error(Ra, Rb):
    """Angle (rad) of the relative rotation Ra^T Rb, in the asin form accurate at small angles."""
    d = np.linalg.norm(np.asarray(Ra) - np.asarray(Rb))
    return float(2.0 * np.arcsin(min(1.0, d / (2.0 * np.sqrt(2.0)))))


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return os.uname().machine
