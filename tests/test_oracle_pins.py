"""Pins of the FP64 oracle to things other than itself: brute-force definitions on
tiny inputs, closed forms, textbook special cases, library routines, finite
differences and invariants.  CPU only."""
import math

import numpy as np
import pytest

import oracle
from brute import (cpd_estep, expm_twist, posterior_bayes, posterior_matrix_form,
                   weighted_procrustes, weighted_squared_distances)
from paper_2103_15039_gb300 import synth


def _tiny(seed, n=6, m=7, alpha_max=2.0, spread=1.0, sigma2=None):
    c = synth.estep_case(seed, n, m, alpha_max=alpha_max, spread=spread, sigma2=sigma2)
    nrm = c["normals"].astype(np.float64)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    c["normals64"] = nrm
    c["alpha64"] = c["alpha"].astype(np.float64)
    return c


# ---------------------------------------------------------------------------
# E step (Eq. (5) with Eqs. (1)-(2))
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("alpha_norm", [False, True])
def test_estep_matches_bruteforce_bayes(seed, alpha_norm):
    c = _tiny(seed)
    rng = np.random.default_rng(seed)
    pi = rng.random(7) + 0.1
    pi /= pi.sum()
    w_n = rng.uniform(0.0, 0.6, 6)
    V = 3.0
    P_ref, Po_ref = posterior_bayes(c["X"], c["Y"], c["normals64"], c["alpha64"], c["R"], c["t"],
                                    c["sigma2"], None, V, pi_m=pi, w_n=w_n,
                                    gaussian_constant=alpha_norm)
    o = oracle.estep(c["X"], c["Y"], c["normals64"], c["alpha64"], c["R"], c["t"], c["sigma2"], 0.0,
                     V, pi_m=pi, w_n=w_n, include_alpha_norm=alpha_norm, dense=True)
    np.testing.assert_allclose(o["P"], P_ref, rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(o["stats"][:, 14], Po_ref, rtol=1e-12)


def test_posterior_rows_sum_to_one_with_outlier_term():
    c = _tiny(11, n=8, m=8)
    o = oracle.estep(c["X"], c["Y"], c["normals64"], c["alpha64"], c["R"], c["t"], c["sigma2"], 0.3,
                     2.0, dense=True)
    np.testing.assert_allclose(o["P"].sum(axis=0) + o["stats"][:, 14], 1.0, rtol=0, atol=1e-14)
    np.testing.assert_allclose(o["stats"][:, 0], o["P"].sum(axis=0), rtol=1e-14)


def test_no_outlier_term_when_w_is_zero():
    c = _tiny(12, n=5, m=9)
    o = oracle.estep(c["X"], c["Y"], c["normals64"], c["alpha64"], c["R"], c["t"], c["sigma2"], 0.0,
                     2.0, dense=True)
    np.testing.assert_allclose(o["P"].sum(axis=0), 1.0, rtol=0, atol=1e-14)
    assert np.all(o["stats"][:, 14] == 0.0)


def test_single_component_closed_form():
    """M = 1: P_1n = K / (K + gamma) with gamma = (2 pi s2)^{3/2} / V and
    K = (1-w)/w exp(-d / (2 s2))  (Eq. (9) with one component)."""
    c = _tiny(13, n=5, m=1)
    w, V, s2 = 0.2, 4.0, c["sigma2"]
    o = oracle.estep(c["X"], c["Y"], c["normals64"], c["alpha64"], c["R"], c["t"], s2, w, V, dense=True)
    d = weighted_squared_distances(c["X"], c["Y"], c["normals64"], c["alpha64"], c["R"], c["t"])[0]
    K = (1 - w) / w * np.exp(-d / (2 * s2))
    gamma = (2 * np.pi * s2) ** 1.5 / V
    np.testing.assert_allclose(o["P"][0], K / (K + gamma), rtol=1e-13)


@pytest.mark.parametrize("seed", [4, 5])
def test_matrix_form_of_eq9_eq10_equals_direct_form(seed):
    c = _tiny(seed, n=7, m=6)
    w, V = 0.15, 2.5
    P_mat = posterior_matrix_form(c["X"], c["Y"], c["normals64"], c["alpha64"], c["R"], c["t"],
                                  c["sigma2"], w, V)
    o = oracle.estep(c["X"], c["Y"], c["normals64"], c["alpha64"], c["R"], c["t"], c["sigma2"], w, V,
                     dense=True)
    np.testing.assert_allclose(o["P"], P_mat, rtol=1e-11)


def test_normal_sign_flip_changes_nothing():
    c = _tiny(14, n=9, m=8)
    a = oracle.estep(c["X"], c["Y"], c["normals64"], c["alpha64"], c["R"], c["t"], c["sigma2"], 0.1, 2.0)
    b = oracle.estep(c["X"], c["Y"], -c["normals64"], c["alpha64"], c["R"], c["t"], c["sigma2"], 0.1, 2.0)
    np.testing.assert_array_equal(a["stats"], b["stats"])


def test_statistics_identity():
    """sum_m P_mn d_mn(z) = z^T A_n z - 2 e_n^T z + f_n at any z, A = Pbar I + W, e = ybar + b."""
    c = _tiny(15, n=6, m=8)
    o = oracle.estep(c["X"], c["Y"], c["normals64"], c["alpha64"], c["R"], c["t"], c["sigma2"], 0.1,
                     2.0, dense=True)
    rng = np.random.default_rng(3)
    R2 = synth.random_rotation(rng, 0.4)
    t2 = rng.standard_normal(3) * 0.2
    d = weighted_squared_distances(c["X"], c["Y"], c["normals64"], c["alpha64"], R2, t2)
    lhs = (o["P"] * d).sum(axis=0)
    Z = c["X"].astype(np.float64) @ R2.T + t2
    s = o["stats"]
    rhs = []
    for n in range(len(Z)):
        W = np.array([[s[n, 4], s[n, 5], s[n, 6]], [s[n, 5], s[n, 7], s[n, 8]],
                      [s[n, 6], s[n, 8], s[n, 9]]])
        A = s[n, 0] * np.eye(3) + W
        e = s[n, 1:4] + s[n, 10:13]
        rhs.append(Z[n] @ A @ Z[n] - 2 * e @ Z[n] + s[n, 13])
    np.testing.assert_allclose(lhs, rhs, rtol=1e-11)
    np.testing.assert_allclose(oracle.objective(s, c["X"], R2, t2), lhs.sum(), rtol=1e-11)


# ---------------------------------------------------------------------------
# alpha = 0 reduces to isotropic CPD (Sec. 3.1: closed form for isotropic covariances)
# ---------------------------------------------------------------------------

def test_alpha_zero_reduces_to_cpd_estep_and_procrustes_mstep():
    c = synth.sphere_plane_pair(seed=7, n=60, m=50)
    X, Y = c["X"], c["Y"]
    M = len(Y)
    R0 = np.eye(3)
    t0 = np.zeros(3)
    s2 = oracle.sigma2_init(X, Y, R0, t0)
    w, V = 0.1, 5.0
    nrm = np.tile([0.0, 0.0, 1.0], (M, 1))
    alpha = np.zeros(M)
    o = oracle.estep(X, Y, nrm, alpha, R0, t0, s2, w, V, dense=True)
    P_cpd = cpd_estep(X, Y, R0, t0, s2, w, V)
    np.testing.assert_allclose(o["P"], P_cpd, rtol=1e-12)
    ms = oracle.mstep(o["stats"], X, R0, t0)
    R_k, t_k = weighted_procrustes(X, Y, P_cpd)
    assert oracle.rotation_error(ms["R"], R_k) < 1e-10
    np.testing.assert_allclose(ms["t"], t_k, atol=1e-10)
    d_new = ((X.astype(np.float64) @ R_k.T + t_k)[None, :, :] - Y.astype(np.float64)[:, None, :]) ** 2
    s2_cpd = (P_cpd * d_new.sum(axis=2)).sum() / (3 * P_cpd.sum())
    np.testing.assert_allclose(ms["sigma2"], s2_cpd, rtol=1e-10)


# ---------------------------------------------------------------------------
# M step: Eqs. (11)-(13)
# ---------------------------------------------------------------------------

def _qd(P, X, Y, nrm, alpha, T):
    return float((P * weighted_squared_distances(X, Y, nrm, alpha, T[:3, :3], T[:3, 3])).sum())


def test_gradient_and_hessian_match_finite_differences():
    c = _tiny(21, n=7, m=9)
    X, Y, nrm, alp = c["X"], c["Y"], c["normals64"], c["alpha64"]
    o = oracle.estep(X, Y, nrm, alp, c["R"], c["t"], c["sigma2"], 0.1, 2.0, dense=True)
    P = o["P"]
    rng = np.random.default_rng(5)
    g = np.eye(4)
    g[:3, :3] = synth.random_rotation(rng, 0.3)
    g[:3, 3] = rng.standard_normal(3) * 0.1
    grad, H = oracle.grad_hess(o["stats"], X, g[:3, :3], g[:3, 3])
    h = 1e-4
    E = np.eye(6)
    fd_g = np.zeros(6)
    for i in range(6):
        fd_g[i] = (_qd(P, X, Y, nrm, alp, g @ expm_twist(h * E[i]))
                   - _qd(P, X, Y, nrm, alp, g @ expm_twist(-h * E[i]))) / (2 * h)
    np.testing.assert_allclose(grad, fd_g, rtol=1e-6, atol=1e-7 * np.abs(fd_g).max())
    # Eq. (12): H_ij is the mixed derivative of Q(g o exp(s E_j) o exp(t E_i)) at s = t = 0
    fd_H = np.zeros((6, 6))
    for i in range(6):
        for j in range(6):
            acc = 0.0
            for si, sj, sg in ((1, 1, 1), (1, -1, -1), (-1, 1, -1), (-1, -1, 1)):
                T = g @ expm_twist(sj * h * E[j]) @ expm_twist(si * h * E[i])
                acc += sg * _qd(P, X, Y, nrm, alp, T)
            fd_H[i, j] = acc / (4 * h * h)
    np.testing.assert_allclose(H, fd_H, rtol=1e-4, atol=1e-5 * np.abs(fd_H).max())
    assert np.abs(H - H.T).max() > 1e-8  # the Hessian of Eq. (12) is asymmetric in general


def test_direct_double_sum_matches_statistics_form():
    c = _tiny(22, n=6, m=8)
    X, Y, nrm, alp = c["X"], c["Y"], c["normals64"], c["alpha64"]
    s2 = c["sigma2"]
    o = oracle.estep(X, Y, nrm, alp, c["R"], c["t"], s2, 0.1, 2.0, dense=True)
    g1, H1 = oracle.grad_hess(o["stats"], X, c["R"], c["t"])
    g2, H2 = oracle.grad_hess_direct(X, Y, nrm, alp, o["P"], c["R"], c["t"], s2)
    np.testing.assert_allclose(g2 * s2, g1, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(H2 * s2, H1, rtol=1e-10, atol=1e-12)


def test_se3_exponential_matches_matrix_exponential():
    rng = np.random.default_rng(9)
    for scale in (1e-9, 1e-5, 1e-3, 0.3, 2.0):
        for _ in range(5):
            xi = rng.standard_normal(6) * scale
            np.testing.assert_allclose(oracle.se3_exp(xi), expm_twist(xi), rtol=1e-12, atol=1e-15)


def test_newton_converges_and_decreases_q():
    c = synth.sphere_plane_pair(seed=8, n=200, m=180)
    X, Y = c["X"], c["Y"]
    pre = oracle.preprocess(Y, 10, 2.0, 0.2)
    R0, t0 = np.eye(3), np.zeros(3)
    s2 = oracle.sigma2_init(X, Y, R0, t0) * 0.2
    V, _ = oracle.volume(Y)
    o = oracle.estep(X, Y, pre["normals"], pre["alpha"], R0, t0, s2, 0.1, V)
    q0 = oracle.objective(o["stats"], X, R0, t0)
    ms = oracle.mstep(o["stats"], X, R0, t0)
    assert ms["Q"] < q0
    g, _ = oracle.grad_hess(o["stats"], X, ms["R"], ms["t"])
    assert np.abs(g).max() < 1e-8 * q0
    np.testing.assert_allclose(ms["R"] @ ms["R"].T, np.eye(3), atol=1e-12)


# ---------------------------------------------------------------------------
# Local surface geometry (Sec. 3.1, Eq. (3)) and preprocessing
# ---------------------------------------------------------------------------

def test_jacobi_matches_numpy_eigh():
    rng = np.random.default_rng(1)
    for _ in range(2000):
        A = rng.standard_normal((3, 3))
        S = A @ A.T * rng.uniform(1e-6, 1e3)
        ev, vec = oracle.jacobi3(S)
        ev_ref = np.linalg.eigvalsh(S)
        np.testing.assert_allclose(ev, ev_ref, rtol=1e-12, atol=1e-13 * ev_ref.max())
        np.testing.assert_allclose(S @ vec, vec * ev, atol=1e-12 * ev_ref.max())
        np.testing.assert_allclose(vec.T @ vec, np.eye(3), atol=1e-13)


def test_penalty_equation3_limits_and_tanh_form():
    """Eq. (3) equals alpha_max tanh(lambda (1/kappa - 3) / 2); alpha -> 0 at kappa = 1/3
    and alpha -> alpha_max as kappa -> 0 (Sec. 3.1)."""
    import os
    fx = os.path.join(os.path.dirname(__file__), "golden", "eq3_limits.txt")
    rows = [ln.split() for ln in open(fx) if ln.strip() and not ln.startswith("#")]
    for kappa_s, ratio_s in rows:
        kappa = eval(kappa_s, {"__builtins__": {}})  # fractions such as 1/3
        assert oracle.penalty(kappa, 2.5, 0.7) == pytest.approx(2.5 * float(ratio_s), abs=1e-15)
    for kappa in (0.01, 0.05, 0.1, 0.2, 0.25, 0.3, 0.333):
        for lam in (0.2, 1.0, 3.0):
            ref = 1.7 * math.tanh(lam * (1.0 / kappa - 3.0) / 2.0)
            assert oracle.penalty(kappa, 1.7, lam) == pytest.approx(ref, rel=1e-13, abs=1e-16)


def test_knn_matches_bruteforce_sort():
    rng = np.random.default_rng(2)
    Y = rng.random((400, 3)).astype(np.float32)
    idx = oracle.knn(Y, 10)
    Yd = Y.astype(np.float64)
    d = ((Yd[:, None, :] - Yd[None, :, :]) ** 2).sum(axis=2)
    ref = np.argsort(d, axis=1, kind="stable")[:, :10]
    assert np.all(idx[:, 0] == np.arange(len(Y)))  # self first
    mism = np.nonzero(np.any(np.sort(idx, 1) != np.sort(ref, 1), axis=1))[0]
    for q in mism:  # only FP32 near-ties at the k-th place may differ
        kth = np.sort(d[q])[9]
        diffset = set(idx[q]) ^ set(ref[q])
        assert all(abs(d[q, j] - kth) < 1e-6 * kth for j in diffset)
    assert len(mism) <= 2


def test_knn_ties_go_to_lower_index():
    Y = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [5, 5, 5]], dtype=np.float32)
    idx = oracle.knn(Y, 3)
    assert list(idx[0]) == [0, 1, 2]


@pytest.mark.parametrize("shape", ["uniform", "lattice", "plane", "clusters", "duplicates"])
def test_grid_knn_equals_bruteforce(shape):
    """The grid search is only a faster route to the brute-force result: every
    row, including exact ties on a lattice and duplicated points, is identical."""
    rng = np.random.default_rng(11)
    Y = {"uniform": rng.uniform(-1, 1, (2500, 3)),
         "lattice": np.stack(np.meshgrid(*[np.arange(11)] * 3), -1).reshape(-1, 3) * 0.25,
         "plane": np.c_[rng.uniform(0, 1, (2000, 2)), np.zeros(2000)],
         "clusters": np.concatenate([rng.normal(c, 0.01, (400, 3)) for c in rng.uniform(-5, 5, (5, 3))]),
         "duplicates": np.repeat(rng.uniform(0, 1, (250, 3)), 4, axis=0)}[shape].astype(np.float32)
    for k in (1, 10, 32):
        np.testing.assert_array_equal(oracle.knn(Y, k, method="grid"), oracle.knn(Y, k, method="brute"))


def test_grid_knn_rows_on_a_large_scan():
    """100k-point LiDAR-shaped cloud: sampled rows of the grid search against
    brute force over all points."""
    c = synth.lidar_pair()
    Y = c["Y"]
    g = oracle.knn(Y, 10, method="grid")
    q = np.random.default_rng(5).choice(len(Y), 60, replace=False)
    np.testing.assert_array_equal(g[q], oracle.knn_rows(Y, q, 10))


def test_planar_neighbourhood_gives_zero_variation_and_max_penalty():
    rng = np.random.default_rng(4)
    pts = np.zeros((300, 3))
    pts[:, :2] = rng.random((300, 2))
    R = synth.random_rotation(rng, 0.7)
    Y = (pts @ R.T).astype(np.float32)
    pre = oracle.preprocess(Y, 10, 2.0, 0.2)
    assert np.all(pre["kappa"] < 1e-6)
    np.testing.assert_allclose(pre["alpha"], 2.0, rtol=1e-12)
    normal = R[:, 2]
    assert np.all(np.abs(np.abs(pre["normals"] @ normal) - 1.0) < 1e-6)


def test_isotropic_neighbourhood_gives_one_third_and_zero_penalty():
    # centre plus the 6 vertices of a regular octahedron: covariance is isotropic
    Y = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]],
                 dtype=np.float32)
    idx = oracle.knn(Y, 7)
    _, kap, alp = oracle.local_geometry(Y, idx, 2.0, 0.2)
    assert kap[0] == pytest.approx(1.0 / 3.0, abs=1e-15)
    assert alp[0] == pytest.approx(0.0, abs=1e-14)


def test_variation_range_and_penalty_falls_with_noise():
    """kappa in [0, 1/3] (Sec. 3.1); the mean penalty decreases as noise grows (Sec. 4.1)."""
    means = []
    for noise in (0.0005, 0.005, 0.02, 0.05):
        c = synth.sphere_plane_pair(seed=3, n=10, m=2000, noise=noise)
        pre = oracle.preprocess(c["Y"], 10, 2.0, 1.0)
        assert np.all(pre["kappa"] >= 0) and np.all(pre["kappa"] <= 1.0 / 3.0 + 1e-15)
        means.append(pre["alpha"].mean())
    assert all(a > b for a, b in zip(means, means[1:]))


def test_sigma2_init_closed_form_matches_double_sum():
    c = synth.estep_case(31, 40, 30, offset=(3.0, -2.0, 1.0))
    X, Y, R, t = c["X"], c["Y"], c["R"], c["t"]
    Z = X.astype(np.float64) @ R.T + t
    brute = ((Z[None, :, :] - Y.astype(np.float64)[:, None, :]) ** 2).sum() / (3 * len(X) * len(Y))
    assert oracle.sigma2_init(X, Y, R, t) == pytest.approx(brute, rel=1e-12)


def test_volume_rule_clamps_flat_boxes():
    Y = np.array([[0, 0, 0], [2, 0, 0], [0, 1, 0], [2, 1, 0]], dtype=np.float32)
    V, diag = oracle.volume(Y)
    assert diag == pytest.approx(math.sqrt(5.0))
    assert V == pytest.approx(2.0 * 1.0 * 1e-2 * math.sqrt(5.0))


# ---------------------------------------------------------------------------
# Full EM
# ---------------------------------------------------------------------------

def test_exact_recovery_of_known_rigid_transform():
    c = synth.sphere_plane_pair(seed=41, n=10, m=600)
    Y = c["Y"]
    rng = np.random.default_rng(41)
    R0 = synth.random_rotation(rng, 0.5)
    t0 = np.array([0.05, -0.02, 0.03])
    X = ((Y.astype(np.float64) - t0) @ R0).astype(np.float32)  # x = R0^T (y - t0)
    r = oracle.register(X, Y, w=0.01, max_iters=100)
    # limited by the FP32 rounding of the moved source (about 1e-7 relative)
    assert oracle.rotation_error(r["R"], R0) < 3e-7
    assert np.linalg.norm(r["t"] - t0) < 3e-7


def test_em_negative_log_likelihood_is_monotone():
    c = synth.sphere_plane_pair(seed=42, n=300, m=300)
    r = oracle.register(c["X"], c["Y"], max_iters=30)
    nll = r["trace"][:, 6]
    assert np.all(np.diff(nll) <= 1e-10 * np.abs(nll[1:]))


def test_equivariance_under_exact_rotation_of_the_target_frame():
    c = synth.sphere_plane_pair(seed=43, n=300, m=300)
    T = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])  # exact in FP32
    r1 = oracle.register(c["X"], c["Y"], max_iters=20)
    Y2 = (c["Y"].astype(np.float64) @ T.T).astype(np.float32)
    r2 = oracle.register(c["X"], Y2, max_iters=20, init_R=T)
    assert oracle.rotation_error(r2["R"], T @ r1["R"]) < 1e-9
    np.testing.assert_allclose(r2["t"], T @ r1["t"], atol=1e-9)


def test_permutation_invariance():
    c = synth.sphere_plane_pair(seed=44, n=300, m=300)
    rng = np.random.default_rng(1)
    r1 = oracle.register(c["X"], c["Y"], max_iters=15)
    px, py = rng.permutation(300), rng.permutation(300)
    r2 = oracle.register(c["X"][px], c["Y"][py], max_iters=15)
    assert oracle.rotation_error(r1["R"], r2["R"]) < 1e-9
    np.testing.assert_allclose(r1["t"], r2["t"], atol=1e-9)
    assert r1["sigma2"] == pytest.approx(r2["sigma2"], rel=1e-8)


# ---------------------------------------------------------------------------
# Sec. 3.2 (outlier weight from the outlier ratio), Sec. 3.3 (confidence
# filtering), termination on the log-likelihood of Eq. (4)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("alpha_norm", [False, True])
def test_w_from_eta_makes_the_expected_outlier_count_eta(alpha_norm):
    """With every component density at its peak c_m, the outlier posterior of
    each source equals eta exactly at w = w_max (the defining equation)."""
    rng = np.random.default_rng(21)
    M = 50
    alpha = rng.uniform(0, 3, M)
    pi = rng.uniform(0.5, 2, M)
    pi /= pi.sum()
    s2, V = 0.013, 2.7
    for eta in (0.01, 0.2, 0.6):
        w = oracle.w_from_eta(eta, V, s2, alpha, pi, include_alpha_norm=alpha_norm)
        c = (2 * math.pi * s2) ** -1.5 * (np.sqrt(1 + alpha) if alpha_norm else 1.0)
        S = float((pi * c).sum())
        A = w / (1 - w) / V
        assert A / (A + S) == pytest.approx(eta, rel=1e-12)
    assert oracle.w_from_eta(0.0, V, s2, alpha, pi) == 0.0


def test_w_from_eta_closed_form_for_uniform_priors():
    s2, V, eta = 0.02, 1.3, 0.1
    c = (2 * math.pi * s2) ** -1.5
    ref = eta * V * c / ((1 - eta) + eta * V * c)
    assert oracle.w_from_eta(eta, V, s2, np.zeros(7)) == pytest.approx(ref, rel=1e-13)


def test_register_with_eta_uses_w_max_at_the_initial_variance():
    c = synth.sphere_plane_pair(seed=23, n=200, m=300)
    X, Y = c["X"], c["Y"]
    s20 = oracle.sigma2_init(X, Y, np.eye(3), np.zeros(3))
    V, _ = oracle.volume(Y)
    w = oracle.w_from_eta(0.15, V, s20, np.zeros(len(Y)))
    a = oracle.register(X, Y, eta=0.15, max_iters=6)
    b = oracle.register(X, Y, w=w, max_iters=6)
    np.testing.assert_array_equal(a["R"], b["R"])
    np.testing.assert_array_equal(a["t"], b["t"])


def test_confidence_special_cases_reduce_to_uniform_weights():
    """phi = 1 everywhere is the uniform setting; a constant target confidence
    gives pi = 1/M; a constant source confidence phi0 gives w = 1 - (1 - w0) phi0."""
    c = synth.sphere_plane_pair(seed=24, n=150, m=250)
    X, Y = c["X"], c["Y"]
    base = oracle.register(X, Y, max_iters=5)
    ones = oracle.register(X, Y, phi_x=np.ones(len(X)), phi_y=np.ones(len(Y)), max_iters=5)
    np.testing.assert_allclose(ones["R"], base["R"], rtol=0, atol=1e-13)
    const_y = oracle.register(X, Y, phi_y=np.full(len(Y), 0.37), max_iters=5)
    np.testing.assert_allclose(const_y["R"], base["R"], rtol=0, atol=1e-13)
    phi0 = float(np.float32(0.8))  # confidences are FP32 inputs
    cx = oracle.register(X, Y, phi_x=np.full(len(X), phi0, dtype=np.float32), max_iters=5)
    ref = oracle.register(X, Y, w=1 - (1 - 0.1) * phi0, max_iters=5)
    np.testing.assert_allclose(cx["R"], ref["R"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(cx["t"], ref["t"], rtol=0, atol=1e-13)


def test_confidence_truncation_is_removal_before_everything():
    c = synth.sphere_plane_pair(seed=25, n=300, m=400)
    X, Y = c["X"], c["Y"]
    rng = np.random.default_rng(25)
    px = rng.uniform(0.2, 1.0, len(X)).astype(np.float32)
    py = rng.uniform(0.2, 1.0, len(Y)).astype(np.float32)
    tau = 0.45
    a = oracle.register(X, Y, phi_x=px, phi_y=py, cf_threshold=tau, max_iters=5)
    kx, ky = px >= tau, py >= tau
    b = oracle.register(X[kx], Y[ky], phi_x=px[kx], phi_y=py[ky], max_iters=5)
    np.testing.assert_array_equal(a["R"], b["R"])
    np.testing.assert_array_equal(a["t"], b["t"])
    assert np.all(np.isnan(a["alpha"][~ky])) and np.all(np.isfinite(a["alpha"][ky]))


def test_nll_termination_stops_at_the_first_small_change():
    c = synth.sphere_plane_pair(seed=26, n=300, m=300)
    X, Y = c["X"], c["Y"]
    full = oracle.register(X, Y, max_iters=40)
    nll = full["trace"][:, 6]
    change = np.abs(np.diff(nll)) / np.abs(nll[1:])
    tol = float(np.median(change))
    rel = change <= tol
    i = int(np.argmax(rel)) + 1  # first iteration whose E step changed the NLL by <= tol
    assert rel.any()
    got = oracle.register(X, Y, max_iters=40, nll_tol=tol)
    assert got["iters"] == i + 1
    same = oracle.register(X, Y, max_iters=i + 1)
    np.testing.assert_array_equal(got["R"], same["R"])
