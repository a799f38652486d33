"""Full registrations on the GPU against the FP64 oracle from the same start.

The bar for FP32 E steps: rotation error < 1e-4 rad and translation error
< 1e-5 of the target's bounding-box diagonal relative to the oracle's result.
"""
import numpy as np
import pytest

import oracle
from paper_2103_15039_gb300 import binding, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = binding.Context(0, 25000, 25000)
    yield c
    c.close()


def _diag(Y):
    Y = np.asarray(Y, dtype=np.float64)
    return float(np.linalg.norm(Y.max(0) - Y.min(0)))


def _check(got, ref, Y, rot_tol=1e-4, trans_tol=1e-5):
    rot = oracle.rotation_error(got["R"], ref["R"])
    tr = np.linalg.norm(got["t"] - ref["t"]) / _diag(Y)
    assert rot < rot_tol and tr < trans_tol, (rot, tr)
    return rot, tr


def test_register_sphere_plane_1000(ctx):
    c = synth.sphere_plane_pair()
    p = binding.default_params()
    got = ctx.register(c["X"], c["Y"], p, trace=True)
    ref = oracle.register(c["X"], c["Y"])
    _check(got, ref, c["Y"])
    assert got["iters"] == ref["iters"] == 50
    assert got["sigma2"] == pytest.approx(ref["sigma2"], rel=1e-3)
    np.testing.assert_allclose(got["trace"][:, 0], ref["trace"][:, 0], rtol=2e-3)
    np.testing.assert_allclose(got["trace"][:, 6], ref["trace"][:, 6], rtol=1e-4)


def test_register_host_and_device_inputs_agree(ctx):
    import torch
    c = synth.sphere_plane_pair(seed=9, n=700, m=900)
    p = binding.default_params(max_iters=20)
    a = ctx.register(c["X"], c["Y"], p)
    b = ctx.register(torch.from_numpy(c["X"]).cuda(), torch.from_numpy(c["Y"]).cuda(), p)
    np.testing.assert_array_equal(a["R"], b["R"])
    np.testing.assert_array_equal(a["t"], b["t"])


def test_register_is_deterministic(ctx):
    c = synth.sphere_plane_pair(seed=10, n=1500, m=1300)
    p = binding.default_params(max_iters=15)
    a = ctx.register(c["X"], c["Y"], p)
    b = ctx.register(c["X"], c["Y"], p)
    np.testing.assert_array_equal(a["R"], b["R"])
    assert a["sigma2"] == b["sigma2"]


def test_register_exact_recovery(ctx):
    c = synth.sphere_plane_pair(seed=41, n=10, m=1000)
    Y = c["Y"]
    rng = np.random.default_rng(41)
    R0 = synth.random_rotation(rng, 0.5)
    t0 = np.array([0.05, -0.02, 0.03])
    X = ((Y.astype(np.float64) - t0) @ R0).astype(np.float32)
    got = ctx.register(X, Y, binding.default_params(w=0.01, max_iters=100))
    assert oracle.rotation_error(got["R"], R0) < 1e-5
    assert np.linalg.norm(got["t"] - t0) < 1e-5


@pytest.mark.parametrize("w", [0.0, 0.3])
def test_register_outlier_weights(ctx, w):
    c = synth.sphere_plane_pair(seed=12, n=800, m=900)
    got = ctx.register(c["X"], c["Y"], binding.default_params(w=w, max_iters=30))
    ref = oracle.register(c["X"], c["Y"], w=w, max_iters=30)
    _check(got, ref, c["Y"])
    assert got["mode"] == (1 if w == 0.0 else 0)


def test_register_batch_shapes(ctx):
    """Uneven pairs shaped like the batched workload (first 6 pairs, sizes capped)."""
    pairs = synth.batch_pairs(num_pairs=6, n_hi=6000)
    for pr in pairs:
        got = ctx.register(pr["X"], pr["Y"], binding.default_params(max_iters=20))
        ref = oracle.register(pr["X"], pr["Y"], max_iters=20)
        _check(got, ref, pr["Y"])


def test_alternating_shapes_reuse_the_loop_graph_with_identical_results():
    """Consecutive registrations of other shapes update the captured EM loop in place (or
    rebuild it when the kernel sequence changes, e.g. the per-source shift mode of w = 0):
    every result equals, bit for bit, the same registration in a fresh context."""
    shapes = [(800, 900, 0.1), (1000, 1000, 0.1), (1200, 700, 0.1), (900, 1100, 0.0), (800, 900, 0.1)]
    pairs = [synth.sphere_plane_pair(seed=40 + i, n=n, m=m) for i, (n, m, _) in enumerate(shapes)]
    fresh = []
    for (n, m, w), c in zip(shapes, pairs):
        ctx1 = binding.Context(0, 2000, 2000)
        ctx1.set_autotune(False)
        fresh.append(ctx1.register(c["X"], c["Y"], binding.default_params(w=w)))
        ctx1.close()
    shared = binding.Context(0, 2000, 2000)
    shared.set_autotune(False)
    for rep in range(2):
        for (n, m, w), c, ref in zip(shapes, pairs, fresh):
            got = shared.register(c["X"], c["Y"], binding.default_params(w=w))
            np.testing.assert_array_equal(got["R"], ref["R"])
            np.testing.assert_array_equal(got["t"], ref["t"])
            assert got["sigma2"] == ref["sigma2"] and got["iters"] == ref["iters"]
    shared.close()


def test_register_rgbd_full_size(ctx):
    """The benchmark's workload (20,000 x 20,000, RGBD room), first 8 iterations."""
    c = synth.rgbd_room_pair()
    p = binding.default_params(max_iters=8)
    got = ctx.register(c["X"], c["Y"], p, trace=True)
    ref = oracle.register(c["X"], c["Y"], max_iters=8)
    _check(got, ref, c["Y"])
    np.testing.assert_allclose(got["trace"][:, 1], ref["trace"][:, 1], rtol=1e-4)


def test_timing_enabled_calls_report_kernel_times_and_leave_no_error(ctx):
    c = synth.sphere_plane_pair(seed=13, n=900, m=800)
    p = binding.default_params(max_iters=10)
    ctx.set_timing(True)
    try:
        a = ctx.register(c["X"], c["Y"], p)
        t = ctx.last_timing()
        assert 0 < t["ms_estep"] < t["ms_total"]
        assert t["ms_combine"] > 0 and t["ms_mstep"] > 0 and t["launches"] > 30
        b = ctx.register(c["X"], c["Y"], p)  # the next call must not see a stale error
        np.testing.assert_array_equal(a["R"], b["R"])
    finally:
        ctx.set_timing(False)


def test_resume_from_a_saved_state_continues_the_same_run(ctx):
    """Checkpoint / resume: the EM state is (R, t, sigma^2).  25 iterations, then 25 more
    started from the first run's result (init_R, init_t, sigma2_init), end where 50
    iterations in one call end (the pose passes once through the caller's frame in FP64)."""
    c = synth.sphere_plane_pair(seed=71, n=1100, m=1000)
    full = ctx.register(c["X"], c["Y"], binding.default_params(max_iters=50))
    first = ctx.register(c["X"], c["Y"], binding.default_params(max_iters=25))
    second = ctx.register(c["X"], c["Y"], binding.default_params(max_iters=25, init_R=first["R"], init_t=first["t"],
                                                                  sigma2_init=first["sigma2"]))
    assert oracle.rotation_error(second["R"], full["R"]) < 1e-9
    assert np.linalg.norm(second["t"] - full["t"]) / _diag(c["Y"]) < 1e-9
    assert second["sigma2"] == pytest.approx(full["sigma2"], rel=1e-9)


def test_log_environment_variable_prints_the_trace(tmp_path):
    """LSGCPD_LOG=1 prints one line per pair and iteration to stderr."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2103_15039_gb300 import binding, synth\n"
            "c = synth.sphere_plane_pair(n=300, m=300)\n"
            "ctx = binding.Context(0, 300, 300)\n"
            "r = ctx.register(c['X'], c['Y'], binding.default_params(max_iters=7))\n"
            "print('iters', r['iters'])\n" % root)
    env = dict(os.environ, LSGCPD_LOG="1")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stderr.splitlines() if ln.startswith("lsgcpd pair 0 iter ")]
    assert len(lines) == 7 and "sigma2" in lines[0] and "newton" in lines[0]
    assert "iters 7" in out.stdout
