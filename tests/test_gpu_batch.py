"""Batched registration (many independent pairs in one pass) on the GPU.

Each pair of a batch must get the computation a registration of that pair
alone gets: the bar against the FP64 oracle is the one of the single-pair
tests (rotation < 1e-4 rad, translation < 1e-5 of the target diagonal), and
against the single-pair GPU path the same bar (only the FP32 summation order of
the E step differs, through the work split).
"""
import numpy as np
import pytest

import oracle
from paper_2103_15039_gb300 import binding, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = binding.Context(0, 4096, 4096)
    yield c
    c.close()


def _diag(Y):
    Y = np.asarray(Y, dtype=np.float64)
    return float(np.linalg.norm(Y.max(0) - Y.min(0)))


def _close(R, t, ref, Y, rot_tol=1e-4, trans_tol=1e-5):
    rot = oracle.rotation_error(R, ref["R"])
    tr = np.linalg.norm(t - ref["t"]) / _diag(Y)
    assert rot < rot_tol and tr < trans_tol, (rot, tr)


def _concat(pairs):
    X = np.concatenate([p["X"] for p in pairs]).astype(np.float32)
    Y = np.concatenate([p["Y"] for p in pairs]).astype(np.float32)
    n_off = np.concatenate([[0], np.cumsum([len(p["X"]) for p in pairs])])
    m_off = np.concatenate([[0], np.cumsum([len(p["Y"]) for p in pairs])])
    return X, n_off, Y, m_off


def test_batch_of_one_is_the_single_registration(ctx):
    c = synth.sphere_plane_pair(seed=31, n=900, m=1100)
    p = binding.default_params(max_iters=25)
    single = ctx.register(c["X"], c["Y"], p, trace=True)
    X, n_off, Y, m_off = _concat([c])
    batch = ctx.register_batch(X, n_off, Y, m_off, p, trace=True)
    # a batch of one pair has the same plan, hence the same bits
    np.testing.assert_array_equal(batch["R"][0], single["R"])
    np.testing.assert_array_equal(batch["t"][0], single["t"])
    assert batch["sigma2"][0] == single["sigma2"]
    assert batch["iters"][0] == single["iters"]
    np.testing.assert_array_equal(batch["trace"][0, : single["iters"]], single["trace"])


def test_uneven_batch_matches_oracle_and_single(ctx):
    pairs = synth.batch_pairs(num_pairs=6, n_lo=60, n_hi=1500)
    p = binding.default_params(max_iters=20)
    X, n_off, Y, m_off = _concat(pairs)
    got = ctx.register_batch(X, n_off, Y, m_off, p, trace=True)
    assert got["R"].shape == (6, 3, 3) and got["trace"].shape == (6, 20, binding.TRACE_WIDTH)
    for i, c in enumerate(pairs):
        ref = oracle.register(c["X"], c["Y"], max_iters=20)
        _close(got["R"][i], got["t"][i], ref, c["Y"])
        assert got["iters"][i] == ref["iters"] == 20
        assert got["sigma2"][i] == pytest.approx(ref["sigma2"], rel=1e-3)
        one = ctx.register(c["X"], c["Y"], p)
        _close(got["R"][i], got["t"][i], one, c["Y"])


def test_batch_with_degenerate_pairs(ctx):
    """A one-source pair and a pair with exactly k targets beside a larger one."""
    rng = np.random.default_rng(5)
    big = synth.sphere_plane_pair(seed=32, n=700, m=800)
    tiny_y = rng.normal(size=(10, 3)).astype(np.float32)
    tiny = dict(X=tiny_y[:1] + np.float32(0.01), Y=tiny_y)
    few = synth.sphere_plane_pair(seed=33, n=130, m=10)
    pairs = [tiny, big, few]
    p = binding.default_params(max_iters=10)
    X, n_off, Y, m_off = _concat(pairs)
    got = ctx.register_batch(X, n_off, Y, m_off, p)
    refs = [oracle.register(c["X"], c["Y"], max_iters=10) for c in pairs]
    # one source: the pose is not unique, the image of the source is
    x = tiny["X"][0].astype(np.float64)
    z_gpu = got["R"][0] @ x + got["t"][0]
    z_ref = refs[0]["R"] @ x + refs[0]["t"]
    assert np.linalg.norm(z_gpu - z_ref) < 1e-4 * _diag(tiny["Y"])
    for i in (1, 2):
        _close(got["R"][i], got["t"][i], refs[i], pairs[i]["Y"], rot_tol=1e-3, trans_tol=1e-4)


def test_batch_is_deterministic_and_order_free(ctx):
    pairs = synth.batch_pairs(num_pairs=5, n_lo=100, n_hi=2000)
    p = binding.default_params(max_iters=12)
    X, n_off, Y, m_off = _concat(pairs)
    a = ctx.register_batch(X, n_off, Y, m_off, p)
    b = ctx.register_batch(X, n_off, Y, m_off, p)
    np.testing.assert_array_equal(a["R"], b["R"])
    np.testing.assert_array_equal(a["t"], b["t"])
    # reversing the pairs changes only the work split
    Xr, nr, Yr, mr = _concat(pairs[::-1])
    r = ctx.register_batch(Xr, nr, Yr, mr, p)
    for i, c in enumerate(pairs):
        j = len(pairs) - 1 - i
        _close(r["R"][j], r["t"][j], dict(R=a["R"][i], t=a["t"][i]), c["Y"])


def test_batch_device_inputs(ctx):
    import torch
    pairs = synth.batch_pairs(num_pairs=4, n_lo=200, n_hi=1200)
    p = binding.default_params(max_iters=8)
    X, n_off, Y, m_off = _concat(pairs)
    a = ctx.register_batch(X, n_off, Y, m_off, p)
    b = ctx.register_batch(torch.from_numpy(X).cuda(), n_off, torch.from_numpy(Y).cuda(), m_off, p)
    np.testing.assert_array_equal(a["R"], b["R"])


def test_batch_rejects_bad_offsets(ctx):
    c = synth.sphere_plane_pair(seed=34, n=100, m=100)
    X, Y = c["X"], c["Y"]
    p = binding.default_params(max_iters=2)
    with pytest.raises(binding.LsgcpdError) as e:  # empty pair
        ctx.register_batch(X, [0, 0, 100], Y, [0, 50, 100], p)
    assert e.value.status == 1
    with pytest.raises(binding.LsgcpdError):  # k larger than a pair's target count
        ctx.register_batch(X, [0, 50, 100], Y, [0, 95, 100], binding.default_params(max_iters=2, knn_k=10))


def test_full_size_batch_sampled_pairs(ctx):
    """256 uneven pairs (500..20,000 points each): sampled pairs against the
    single-pair GPU path, the smallest against the oracle."""
    pairs = synth.batch_pairs()
    p = binding.default_params(max_iters=50)
    X, n_off, Y, m_off = _concat(pairs)
    big = binding.Context(0, 20000, 20000)
    try:
        got = big.register_batch(X, n_off, Y, m_off, p)
        sizes = np.array([len(c["X"]) * len(c["Y"]) for c in pairs])
        picks = [int(np.argmin(sizes)), int(np.argmax(sizes)), 17, 128, 255]
        for i in picks:
            one = big.register(pairs[i]["X"], pairs[i]["Y"], p)
            _close(got["R"][i], got["t"][i], one, pairs[i]["Y"])
            assert abs(int(got["iters"][i]) - one["iters"]) <= 1
        i = picks[0]
        ref = oracle.register(pairs[i]["X"], pairs[i]["Y"], max_iters=50)
        _close(got["R"][i], got["t"][i], ref, pairs[i]["Y"])
    finally:
        big.close()


def test_thousands_of_tiny_pairs(ctx):
    """3000 pairs of 10-40 points (grids with P in the thousands, many partial
    tiles and blocks): sampled pairs against the oracle."""
    rng = np.random.default_rng(91)
    pairs = []
    for i in range(3000):
        n, m = int(rng.integers(10, 41)), int(rng.integers(10, 41))
        Y = rng.normal(size=(m, 3)).astype(np.float32)
        R0 = synth.random_rotation(rng, 0.3)
        X = ((Y[rng.integers(0, m, n)] @ R0.T) + 0.02 * rng.normal(size=(n, 3))).astype(np.float32)
        pairs.append(dict(X=X, Y=Y))
    X, n_off, Y, m_off = _concat(pairs)
    p = binding.default_params(max_iters=5, knn_k=5)
    got = ctx.register_batch(X, n_off, Y, m_off, p)
    assert np.all(np.isfinite(got["R"])) and np.all(got["iters"] == 5)
    for i in (0, 1, 777, 2048, 2999):
        ref = oracle.register(pairs[i]["X"], pairs[i]["Y"], max_iters=5, knn_k=5)
        _close(got["R"][i], got["t"][i], ref, pairs[i]["Y"], rot_tol=1e-3, trans_tol=1e-4)


def test_batch_pairs_finish_at_their_own_iteration(ctx):
    """With a motion tolerance pairs stop at different iterations; a finished pair is
    no longer computed while the others continue, and each matches its own run."""
    pairs = synth.batch_pairs(num_pairs=6, n_lo=200, n_hi=2500)
    X, n_off, Y, m_off = _concat(pairs)
    p = binding.default_params(max_iters=60, tol=1e-6)
    got = ctx.register_batch(X, n_off, Y, m_off, p)
    assert len(set(got["iters"].tolist())) > 1  # they really stop at different iterations
    for i, c in enumerate(pairs):
        one = ctx.register(c["X"], c["Y"], p)
        assert abs(int(got["iters"][i]) - one["iters"]) <= 1
        _close(got["R"][i], got["t"][i], one, c["Y"])
