"""Parity of the CUDA library (through the C ABI) with the FP64 oracle.

Tolerances follow from the FP32 arithmetic of the E step: each exponent
l_m - c (d + kappa_n) carries an absolute rounding error of a few units of
FP32 roundoff times its magnitude (|L| + c d <= ~200), i.e. a relative error of
at most ~2e-5 per exponential; FP32 partial sums are at most 8192 terms long
(about 1e-5 relative at worst for unbiased rounding).  Per-source moments are
compared with rtol = atol = 2e-4 relative to each moment's scale over all
sources; global FP64 moments with 1e-4 of the sum of |terms|.  The M step is
FP64 on both sides (1e-9).  Neighbour indices are compared exactly (both sides
decide in FP32 with the same operation order).
"""
import math

import numpy as np
import pytest

import oracle
from oracle_forms import global_moments, moment_magnitudes, per_source
from paper_2103_15039_gb300 import binding, synth

pytestmark = pytest.mark.gpu

RTOL = 2e-4


@pytest.fixture(scope="module")
def ctx():
    c = binding.Context(0, 4096, 4096)
    yield c
    c.close()


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _run_estep(ctx, case, w, V, alpha_norm=False):
    X, Y = case["X"], case["Y"]
    nrm = case["normals"].astype(np.float64)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    nrm32 = nrm.astype(np.float32)
    alpha = case["alpha"]
    p = binding.default_params(w=w, include_alpha_norm=int(alpha_norm))
    g = ctx.estep(_cuda(X), _cuda(Y), _cuda(nrm32), _cuda(alpha), case["R"], case["t"], case["sigma2"], V, p,
                  per_n=True)
    o = oracle.estep(X, Y, nrm32.astype(np.float64), alpha.astype(np.float64), case["R"], case["t"],
                     case["sigma2"], w, V, include_alpha_norm=alpha_norm)
    ref_n = per_source(o["stats"], X, case["R"], case["t"])
    ref_m = global_moments(ref_n, X, o["nll"])
    mag = moment_magnitudes(ref_n, X, o["nll"])
    return g["per_n"].cpu().numpy().astype(np.float64), g["moments"], ref_n, ref_m, mag


def _compare(got_n, got_m, ref_n, ref_m, mag, rtol=RTOL):
    scale = np.abs(ref_n).max(axis=0) + 1e-30
    err = np.abs(got_n[:, :12] - ref_n[:, :12]) / (scale[:12] + np.abs(ref_n[:, :12]))
    assert err.max() < rtol, (err.max(axis=0), np.unravel_index(err.argmax(), err.shape))
    gerr = np.abs(got_m - ref_m) / (mag + 1e-300)
    assert gerr.max() < rtol / 2, (gerr.argmax(), gerr.max(), got_m[gerr.argmax()], ref_m[gerr.argmax()])


SIZES = [(1, 1), (2, 3), (31, 33), (129, 257), (700, 1000), (2049, 1500)]


@pytest.mark.parametrize("n,m", SIZES)
def test_estep_fixed_shift_mode(ctx, n, m):
    case = synth.estep_case(100 + n + m, n, m)
    _compare(*_run_estep(ctx, case, w=0.1, V=1.0))


@pytest.mark.parametrize("n,m", [(1, 1), (31, 33), (700, 1000)])
def test_estep_without_outlier_term(ctx, n, m):
    """w = 0: no outlier component; the library switches to the per-source max shift."""
    case = synth.estep_case(200 + n, n, m)
    got_n, got_m, ref_n, ref_m, mag = _run_estep(ctx, case, w=0.0, V=1.0)
    _compare(got_n, got_m, ref_n, ref_m, mag)
    np.testing.assert_allclose(got_n[:, 0], 1.0, atol=1e-5)
    assert np.all(got_n[:, 11] == 0.0)


def test_estep_tiny_outlier_weight_uses_max_shift(ctx):
    case = synth.estep_case(301, 300, 400, sigma2=1e-6)
    _compare(*_run_estep(ctx, case, w=1e-35, V=1e6))


@pytest.mark.parametrize("alpha_norm", [False, True])
def test_estep_gaussian_constant_option(ctx, alpha_norm):
    case = synth.estep_case(401, 500, 600, alpha_max=10.0)
    _compare(*_run_estep(ctx, case, w=0.2, V=2.0, alpha_norm=alpha_norm))


def test_estep_far_from_origin_and_sharp_posteriors(ctx):
    case = synth.estep_case(501, 800, 900, offset=(60.0, -35.0, 12.0), sigma2=2e-4)
    _compare(*_run_estep(ctx, case, w=0.1, V=1.0))


def test_estep_posteriors_sum_to_one(ctx):
    case = synth.estep_case(601, 1000, 1200)
    got_n, _, _, _, _ = _run_estep(ctx, case, w=0.3, V=1.0)
    np.testing.assert_allclose(got_n[:, 0] + got_n[:, 11], 1.0, atol=1e-6)


def test_mstep_matches_oracle_newton(ctx):
    c = synth.sphere_plane_pair(seed=77, n=600, m=500)
    X, Y = c["X"], c["Y"]
    pre = oracle.preprocess(Y, 10, 2.0, 0.2)
    R0 = synth.random_rotation(np.random.default_rng(3), 0.2)
    t0 = np.array([0.02, -0.01, 0.03])
    s2 = oracle.sigma2_init(X, Y, R0, t0) * 0.3
    V, _ = oracle.volume(Y)
    o = oracle.estep(X, Y, pre["normals"], pre["alpha"], R0, t0, s2, 0.1, V)
    mom = global_moments(per_source(o["stats"], X, R0, t0), X, o["nll"])
    ref = oracle.mstep(o["stats"], X, R0, t0)
    got = ctx.mstep(mom, R0, t0, binding.default_params())
    assert oracle.rotation_error(got["R"], ref["R"]) < 1e-9
    np.testing.assert_allclose(got["t"], ref["t"], atol=1e-9)
    assert got["sigma2"] == pytest.approx(ref["sigma2"], rel=1e-9)
    # the Newton direction is solved in FP32 (FP64 residual): the path may take one more step
    assert abs(got["newton_iters"] - ref["newton_iters"]) <= 1


@pytest.mark.parametrize("which", ["sphere_plane", "random", "rgbd_full"])
def test_preprocess_matches_oracle(ctx, which):
    if which == "sphere_plane":
        Y = synth.sphere_plane_pair(seed=5, n=10, m=1000)["Y"]
    elif which == "random":
        Y = synth.estep_case(9, 1, 777, offset=(3.0, 4.0, -5.0))["Y"]
    else:
        Y = synth.rgbd_room_pair()["Y"]
    p = binding.default_params()
    g = ctx.preprocess(_cuda(Y), p, want_idx=True)
    ref = oracle.preprocess(Y, 10, 2.0, 0.2)
    np.testing.assert_array_equal(g["idx"].cpu().numpy(), ref["idx"])
    np.testing.assert_allclose(g["kappa"].cpu().numpy(), ref["kappa"], rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(g["alpha"].cpu().numpy(), ref["alpha"], rtol=1e-5, atol=1e-6)
    # the normal's sign is free: compare alpha n n^T where the eigen-gap makes n unique
    n_g = g["normals"].cpu().numpy().astype(np.float64)
    dots = np.abs(np.einsum("ij,ij->i", n_g, ref["normals"]))
    C_ok = ref["kappa"] < 0.2
    assert np.all(dots[C_ok] > 1 - 1e-5)


def test_invalid_arguments_report_einval(ctx):
    import torch
    p = binding.default_params(knn_k=20)
    with pytest.raises(binding.LsgcpdError) as e:
        ctx.preprocess(_cuda(np.zeros((5, 3))), p)
    assert e.value.status == 1
    bad = np.zeros((10, 3), dtype=np.float32)
    bad[3, 1] = np.nan
    with pytest.raises(binding.LsgcpdError) as e:
        ctx.register(bad, np.random.rand(50, 3).astype(np.float32), binding.default_params())
    assert e.value.status == 1
    with pytest.raises(binding.LsgcpdError):
        ctx.register(np.zeros((0, 3), np.float32), np.random.rand(50, 3).astype(np.float32),
                     binding.default_params())
    with pytest.raises(binding.LsgcpdError):
        ctx.register(np.random.rand(5, 3).astype(np.float32), np.random.rand(50, 3).astype(np.float32),
                     binding.default_params(w=1.0))
    # beyond the 2^30-unit limit of the plan tables (4.2e6 targets in 128 x 128 tiles): rejected
    # before any work, and the context stays usable
    big = torch.zeros((4_200_000, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(binding.LsgcpdError) as e:
        ctx.preprocess(big, binding.default_params())
    assert e.value.status == 1 and "too large" in str(e.value)
    del big
    Y = synth.sphere_plane_pair(seed=3, n=10, m=200)["Y"]
    assert ctx.preprocess(_cuda(Y), binding.default_params())["normals"].shape[0] == 200
    torch.cuda.synchronize()


@pytest.mark.parametrize("k", [1, 4, 16, 20, 32])
def test_knn_other_neighbourhood_sizes(ctx, k):
    """Exact neighbour lists for compile-time (k <= 16) and runtime (k > 16) kernels."""
    Y = synth.sphere_plane_pair(seed=6, n=10, m=1500)["Y"]
    p = binding.default_params(knn_k=k)
    g = ctx.preprocess(_cuda(Y), p, want_idx=True)
    np.testing.assert_array_equal(g["idx"].cpu().numpy(), oracle.knn(Y, k))


def test_knn_exact_ties_keep_the_lower_index(ctx):
    """A lattice has many exactly equal FP32 distances; ties must go to the lower index."""
    g1 = np.arange(6, dtype=np.float32)
    Y = np.stack(np.meshgrid(g1, g1, g1, indexing="ij"), axis=-1).reshape(-1, 3).astype(np.float32)
    p = binding.default_params(knn_k=7)
    g = ctx.preprocess(_cuda(Y), p, want_idx=True)
    np.testing.assert_array_equal(g["idx"].cpu().numpy(), oracle.knn(Y, 7))


@pytest.mark.parametrize("shape", ["uniform", "lattice", "plane", "clusters", "duplicates"])
@pytest.mark.parametrize("k", [1, 4, 10, 16, 20, 32])
def test_grid_knn_equals_bruteforce(ctx, shape, k):
    """The uniform-grid search returns the brute-force lists, ties included."""
    rng = np.random.default_rng(31)
    Y = {"uniform": rng.uniform(-1, 1, (3000, 3)),
         "lattice": np.stack(np.meshgrid(*[np.arange(13)] * 3), -1).reshape(-1, 3) * 0.25,
         "plane": np.c_[rng.uniform(0, 1, (2500, 2)), np.zeros(2500)],
         "clusters": np.concatenate([rng.normal(c, 0.01, (500, 3)) for c in rng.uniform(-5, 5, (5, 3))]),
         "duplicates": np.repeat(rng.uniform(0, 1, (300, 3)), 4, axis=0)}[shape].astype(np.float32)
    p = binding.default_params(knn_k=k, knn_method=2)
    g = ctx.preprocess(_cuda(Y), p, want_idx=True)
    np.testing.assert_array_equal(g["idx"].cpu().numpy(), oracle.knn(Y, k, method="brute"))


def test_grid_and_bruteforce_knn_agree_on_the_rgbd_target(ctx):
    Y = synth.rgbd_room_pair()["Y"]
    a = ctx.preprocess(_cuda(Y), binding.default_params(knn_method=1), want_idx=True)
    b = ctx.preprocess(_cuda(Y), binding.default_params(knn_method=2), want_idx=True)
    np.testing.assert_array_equal(a["idx"].cpu().numpy(), b["idx"].cpu().numpy())
    np.testing.assert_array_equal(a["alpha"].cpu().numpy(), b["alpha"].cpu().numpy())


def test_grid_knn_in_a_batch(ctx):
    """Per-pair grids: lists never cross pairs and equal each pair's own search."""
    pairs = synth.batch_pairs(num_pairs=6, n_lo=40, n_hi=3000)
    X = np.concatenate([q["X"] for q in pairs])
    Y = np.concatenate([q["Y"] for q in pairs])
    n_off = np.concatenate([[0], np.cumsum([len(q["X"]) for q in pairs])])
    m_off = np.concatenate([[0], np.cumsum([len(q["Y"]) for q in pairs])])
    a = ctx.register_batch(X, n_off, Y, m_off, binding.default_params(max_iters=3, knn_method=1))
    b = ctx.register_batch(X, n_off, Y, m_off, binding.default_params(max_iters=3, knn_method=2))
    np.testing.assert_array_equal(a["R"], b["R"])
    np.testing.assert_array_equal(a["t"], b["t"])
