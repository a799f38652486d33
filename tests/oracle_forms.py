"""Test-side conversions of the oracle's E-step statistics into the quantities the
CUDA library reports.  FP64 numpy; shares nothing with the CUDA path.

The oracle gives, per source n, Pbar, ybar = sum P y, W = sum P alpha n n^T,
b = sum P alpha (n.y) n, f = sum P (|y|^2 + alpha (n.y)^2), Pout.  With
z = R x + t, A = Pbar I + W, e = ybar + b and Lambda_m = I + alpha_m n_m n_m^T:
  h = sum P Lambda_m (z - y_m)  = A z - e
  D = sum P d(z)                = z^T A z - 2 e^T z + f
"""
import numpy as np

W_IDX = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
XT_PAIRS = [(k, l) for k in range(4) for l in range(k, 4)]


def per_source(stats, X, R, t):
    """Per-source layout of the library: Pbar, h (3), W (6), D, Pout, 0 x 4."""
    s = np.asarray(stats, dtype=np.float64)
    Z = np.asarray(X, dtype=np.float64) @ np.asarray(R).reshape(3, 3).T + np.asarray(t).ravel()
    N = len(Z)
    out = np.zeros((N, 16))
    Pb = s[:, 0]
    W = np.zeros((N, 3, 3))
    for j, (a, b) in enumerate(W_IDX):
        W[:, a, b] = s[:, 4 + j]
        W[:, b, a] = s[:, 4 + j]
    A = W + Pb[:, None, None] * np.eye(3)[None]
    e = s[:, 1:4] + s[:, 10:13]
    out[:, 0] = Pb
    out[:, 1:4] = np.einsum("nij,nj->ni", A, Z) - e
    out[:, 4:10] = s[:, 4:10]
    out[:, 10] = np.einsum("ni,nij,nj->n", Z, A, Z) - 2 * np.einsum("ni,ni->n", e, Z) + s[:, 13]
    out[:, 11] = s[:, 14]
    return out


def global_moments(per_n, X, nll):
    """The 76 global moments from per-source residual-form moments (caller's frame)."""
    p = np.asarray(per_n, dtype=np.float64)
    Xt = np.concatenate([np.asarray(X, dtype=np.float64), np.ones((len(p), 1))], axis=1)
    h = p[:, 1:4]
    Avals = [p[:, 0] + p[:, 4], p[:, 5], p[:, 6], p[:, 0] + p[:, 7], p[:, 8], p[:, 0] + p[:, 9]]
    m = np.zeros(76)
    m[0] = p[:, 0].sum()
    m[1] = p[:, 10].sum()
    m[2:14] = np.einsum("ni,nk->ik", h, Xt).ravel()
    j = 14
    for a in Avals:
        for (k, l) in XT_PAIRS:
            m[j] = (a * Xt[:, k] * Xt[:, l]).sum()
            j += 1
    m[74] = p[:, 11].sum()
    m[75] = nll
    return m


def moment_magnitudes(per_n, X, nll):
    """Sum of |term| for every global moment: the scale of its rounding error."""
    return global_moments(np.abs(per_n), np.abs(np.asarray(X, dtype=np.float64)), abs(nll))
