"""Parity at the full sizes of the large workloads, through the C ABI.

* LiDAR-shaped pair (64 x 1,563 = 100,032 points per scan): every neighbour
  list bit-exact, normals / kappa / alpha for every target, the per-source and
  global moments of one full E step against the oracle's full E step, and a
  two-iteration registration against the oracle's.
* Superquadric range scan (500,000 x 500,000): every neighbour list bit-exact
  (the oracle's exact grid search), one full E step (2.5e11 pairs) checked on
  sampled sources, which the oracle evaluates one by one against all targets,
  and a full 50-iteration registration checked by the properties EM has at any
  size (the negative log-likelihood of Eq. 4 never rises, the posteriors are
  normalised, the ground-truth motion is recovered).

Tolerances are those of the E-step parity tests (FP32 exponent rounding and
partial sums of at most 8,192 terms); the registration bar is the task's
(rotation < 1e-4 rad, translation < 1e-5 of the target diagonal).
"""
import numpy as np
import pytest

import oracle
from oracle_forms import global_moments, moment_magnitudes, per_source
from paper_2103_15039_gb300 import binding, synth

pytestmark = pytest.mark.gpu

RTOL = 2e-4


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _diag(Y):
    Y = np.asarray(Y, dtype=np.float64)
    return float(np.linalg.norm(Y.max(0) - Y.min(0)))


def _check_preprocess(g, ref):
    np.testing.assert_array_equal(g["idx"].cpu().numpy(), ref["idx"])
    np.testing.assert_allclose(g["kappa"].cpu().numpy(), ref["kappa"], rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(g["alpha"].cpu().numpy(), ref["alpha"], rtol=1e-5, atol=1e-6)
    n_g = g["normals"].cpu().numpy().astype(np.float64)
    dots = np.abs(np.einsum("ij,ij->i", n_g, ref["normals"]))
    assert np.all(dots[ref["kappa"] < 0.2] > 1 - 1e-5)


def _per_source_close(got, ref):
    scale = np.abs(ref).max(axis=0) + 1e-30
    err = np.abs(got[:, :12] - ref[:, :12]) / (scale[:12] + np.abs(ref[:, :12]))
    assert err.max() < RTOL, (err.max(axis=0), np.unravel_index(err.argmax(), err.shape))


@pytest.fixture(scope="module")
def lidar():
    c = synth.lidar_pair()
    pre = oracle.preprocess(c["Y"], 10, 2.0, 0.2)
    ctx = binding.Context(0, len(c["X"]), len(c["Y"]))
    yield c, pre, ctx
    ctx.close()


def test_lidar_preprocess_every_target(lidar):
    c, pre, ctx = lidar
    g = ctx.preprocess(_cuda(c["Y"]), binding.default_params(), want_idx=True)
    _check_preprocess(g, pre)


def test_lidar_full_estep(lidar):
    c, pre, ctx = lidar
    X, Y = c["X"], c["Y"]
    R0, t0 = np.eye(3), np.zeros(3)
    s2 = oracle.sigma2_init(X, Y, R0, t0)
    V, _ = oracle.volume(Y)
    nrm32 = pre["normals"].astype(np.float32)
    alpha32 = pre["alpha"].astype(np.float32)
    p = binding.default_params(w=0.1)
    g = ctx.estep(_cuda(X), _cuda(Y), _cuda(nrm32), _cuda(alpha32), R0, t0, s2, V, p, per_n=True)
    o = oracle.estep(X, Y, nrm32.astype(np.float64), alpha32.astype(np.float64), R0, t0, s2, 0.1, V)
    ref_n = per_source(o["stats"], X, R0, t0)
    got_n = g["per_n"].cpu().numpy().astype(np.float64)
    _per_source_close(got_n, ref_n)
    ref_m = global_moments(ref_n, X, o["nll"])
    mag = moment_magnitudes(ref_n, X, o["nll"])
    gerr = np.abs(g["moments"] - ref_m) / (mag + 1e-300)
    assert gerr.max() < RTOL / 2, (gerr.argmax(), gerr.max())


def test_lidar_two_iteration_registration(lidar):
    """Both E-step precisions against the oracle: FP32 at the task's bar, the
    f16x2-exponential variant at its stated bound (1e-3 rad, 1e-4 of the diagonal)."""
    c, _, ctx = lidar
    ref = oracle.register(c["X"], c["Y"], max_iters=2)
    got = ctx.register(c["X"], c["Y"], binding.default_params(max_iters=2))
    assert oracle.rotation_error(got["R"], ref["R"]) < 1e-4
    assert np.linalg.norm(got["t"] - ref["t"]) / _diag(c["Y"]) < 1e-5
    assert got["sigma2"] == pytest.approx(ref["sigma2"], rel=1e-3)
    half = ctx.register(c["X"], c["Y"], binding.default_params(max_iters=2, precision=1))
    assert oracle.rotation_error(half["R"], ref["R"]) < 1e-3
    assert np.linalg.norm(half["t"] - ref["t"]) / _diag(c["Y"]) < 1e-4


@pytest.fixture(scope="module")
def superquadrics():
    c = synth.superquadric_pair()
    pre = oracle.preprocess(c["Y"], 10, 2.0, 0.2)
    ctx = binding.Context(0, len(c["X"]), len(c["Y"]))
    yield c, pre, ctx
    ctx.close()


def test_superquadric_preprocess_every_target(superquadrics):
    c, pre, ctx = superquadrics
    g = ctx.preprocess(_cuda(c["Y"]), binding.default_params(), want_idx=True)
    _check_preprocess(g, pre)


def test_superquadric_full_estep_sampled_sources(superquadrics):
    c, pre, ctx = superquadrics
    X, Y = c["X"], c["Y"]
    R0, t0 = np.eye(3), np.zeros(3)
    s2 = oracle.sigma2_init(X, Y, R0, t0) * 0.01  # sharper posteriors than the start of EM
    V, _ = oracle.volume(Y)
    nrm32 = pre["normals"].astype(np.float32)
    alpha32 = pre["alpha"].astype(np.float32)
    p = binding.default_params(w=0.1)
    g = ctx.estep(_cuda(X), _cuda(Y), _cuda(nrm32), _cuda(alpha32), R0, t0, s2, V, p, per_n=True)
    got_n = g["per_n"].cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(7)
    pick = np.sort(np.concatenate([rng.choice(len(X), 96, replace=False), [0, len(X) - 1]]))
    o = oracle.estep(X[pick], Y, nrm32.astype(np.float64), alpha32.astype(np.float64), R0, t0, s2, 0.1, V)
    ref_n = per_source(o["stats"], X[pick], R0, t0)
    _per_source_close(got_n[pick], ref_n)
    # every source's posteriors (with the outlier term) sum to one
    np.testing.assert_allclose(got_n[:, 0] + got_n[:, 11], 1.0, atol=1e-5)
    assert g["moments"][0] == pytest.approx(got_n[:, 0].sum(), rel=1e-5)


def test_superquadric_registration_properties(superquadrics):
    c, _, ctx = superquadrics
    p = binding.default_params(max_iters=50)
    got = ctx.register(c["X"], c["Y"], p, trace=True)
    tr = got["trace"]
    assert got["iters"] == 50 and np.all(np.isfinite(tr))
    nll = tr[:, 6]
    # EM never raises the negative log-likelihood (FP32 E step: 1e-6 relative slack)
    assert np.all(np.diff(nll) <= 1e-6 * np.abs(nll[1:])), np.diff(nll).max()
    assert np.all(tr[:, 0] > 0)
    # the known motion is recovered (not a parity criterion: EM's own optimum)
    R_gt, t_gt = c["R_gt"], c["t_gt"]
    assert oracle.rotation_error(got["R"], R_gt) < 1e-2
    assert np.linalg.norm(got["t"] - t_gt) / _diag(c["Y"]) < 1e-2

