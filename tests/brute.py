"""Independent NumPy brute-force formulas used to pin the oracle.

Nothing here imports the oracle or the CUDA library.  Each function writes a
definition from the paper (or a textbook special case) in the most literal form
available, without the log-domain, statistics or factorisations the oracle uses.
Only for tiny inputs.
"""
from __future__ import annotations

import numpy as np


def component_precisions(normals, alpha, sigma2):
    """Sigma_m^{-1} = (alpha_m n_m n_m^T + I) / sigma^2   (Eq. (2))."""
    n = np.asarray(normals, dtype=np.float64)
    a = np.asarray(alpha, dtype=np.float64)
    return (a[:, None, None] * n[:, :, None] * n[:, None, :] + np.eye(3)[None]) / sigma2


def posterior_bayes(X, Y, normals, alpha, R, t, sigma2, w, V, pi_m=None, w_n=None,
                    gaussian_constant=False):
    """Eq. (5) with Eq. (1) evaluated literally (no log domain).

    Component density of Eq. (2): c_m exp(-1/2 r^T Sigma_m^{-1} r).  With
    ``gaussian_constant`` c_m = 1/sqrt(det(2 pi Sigma_m)) computed from the explicit
    covariance (inverse of the precision); otherwise Eq. (9)'s (2 pi sigma^2)^(-3/2).
    Returns (P [M x N], P_out [N]).
    """
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    N, M = len(X), len(Y)
    pi = np.full(M, 1.0 / M) if pi_m is None else np.asarray(pi_m, dtype=np.float64)
    wn = np.full(N, w) if w_n is None else np.asarray(w_n, dtype=np.float64)
    Sinv = component_precisions(normals, alpha, sigma2)
    Sigma = np.linalg.inv(Sinv)
    if gaussian_constant:
        c = 1.0 / np.sqrt(np.linalg.det(2.0 * np.pi * Sigma))
    else:
        c = np.full(M, (2.0 * np.pi * sigma2) ** -1.5)
    Z = X @ np.asarray(R).T + np.asarray(t)
    dens = np.empty((M, N))
    for m in range(M):
        for n in range(N):
            r = Z[n] - Y[m]
            dens[m, n] = c[m] * np.exp(-0.5 * r @ Sinv[m] @ r)
    p_o = 1.0 / V
    mix = wn * p_o + (1.0 - wn) * (pi[:, None] * dens).sum(axis=0)
    P = (1.0 - wn)[None, :] * pi[:, None] * dens / mix[None, :]
    P_out = wn * p_o / mix
    return P, P_out


def posterior_matrix_form(X, Y, normals, alpha, R, t, sigma2, w, V):
    """Eqs. (9)-(10): P = K / (1^T K + gamma), K = C (.) exp(-(D A + B) / (2 sigma^2)).

    The matrix written as ``t^T t I`` in Eq. (10) is read as t^T t times the all-ones
    M x N matrix (the only reading that makes B the squared distance).
    """
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    Nm = np.asarray(normals, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64).reshape(3, 1)
    N, M = len(X), len(Y)
    one_M = np.ones((M, 1))
    one_N = np.ones((N, 1))
    s = np.einsum("ij,ij->i", Y, Nm).reshape(M, 1)
    A = (Nm @ R @ X.T + Nm @ t @ one_N.T - s @ one_N.T) ** 2
    Qm = (X ** 2).sum(axis=1)[None, :] + (Y ** 2).sum(axis=1)[:, None]
    B = Qm + float((t.T @ t).item()) * np.ones((M, N)) + 2.0 * (one_M @ t.T @ R @ X.T - Y @ R @ X.T
                                                       - Y @ t @ one_N.T)
    D = np.diag(np.asarray(alpha, dtype=np.float64))
    Cm = np.full((M, N), (1.0 - w) / w * (1.0 / M))
    K = Cm * np.exp(-(D @ A + B) / (2.0 * sigma2))
    gamma = (2.0 * np.pi * sigma2) ** 1.5 / V
    return K / (K.sum(axis=0, keepdims=True) + gamma)


def weighted_squared_distances(X, Y, normals, alpha, R, t):
    """d_mn = (z_n - y_m)^T (I + alpha_m n_m n_m^T)(z_n - y_m)  [M x N]."""
    Z = np.asarray(X, dtype=np.float64) @ np.asarray(R).T + np.asarray(t)
    Y = np.asarray(Y, dtype=np.float64)
    r = Z[None, :, :] - Y[:, None, :]
    s = np.einsum("mnk,mk->mn", r, np.asarray(normals, dtype=np.float64))
    return (r ** 2).sum(axis=2) + np.asarray(alpha, dtype=np.float64)[:, None] * s ** 2


def cpd_estep(X, Y, R, t, sigma2, w, V):
    """Isotropic CPD posterior (Myronenko and Song) with the outlier density 1/V:
    P_mn = exp(-|z_n - y_m|^2 / 2 sigma^2) / (sum_k exp(...) + (2 pi sigma^2)^{3/2} w/(1-w) M / V)."""
    Z = np.asarray(X, dtype=np.float64) @ np.asarray(R).T + np.asarray(t)
    Y = np.asarray(Y, dtype=np.float64)
    M = len(Y)
    d2 = ((Z[None, :, :] - Y[:, None, :]) ** 2).sum(axis=2)
    E = np.exp(-d2 / (2.0 * sigma2))
    c = (2.0 * np.pi * sigma2) ** 1.5 * w / (1.0 - w) * M / V
    return E / (E.sum(axis=0, keepdims=True) + c)


def weighted_procrustes(X, Y, P):
    """Rigid (R, t) minimising sum_mn P_mn |R x_n + t - y_m|^2 (Kabsch / Umeyama, no scale)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    NP = P.sum()
    mu_x = (P.sum(axis=0) @ X) / NP
    mu_y = (P.sum(axis=1) @ Y) / NP
    A = (Y - mu_y).T @ P @ (X - mu_x)
    U, _, Vt = np.linalg.svd(A)
    Dg = np.diag([1.0, 1.0, np.linalg.det(U @ Vt)])
    R = U @ Dg @ Vt
    return R, mu_y - R @ mu_x


def hat(w):
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def twist_matrix(xi):
    T = np.zeros((4, 4))
    T[:3, :3] = hat(xi[:3])
    T[:3, 3] = xi[3:]
    return T


def expm_twist(xi):
    """Matrix exponential of the 4x4 twist (scipy.linalg.expm)."""
    from scipy.linalg import expm
    return expm(twist_matrix(np.asarray(xi, dtype=np.float64)))
