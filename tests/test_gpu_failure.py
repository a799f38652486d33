"""The failure path of the E step's copy pipeline, exercised without a fault:
a bounded wait on a barrier that nothing completes must give up, report
LSGCPD_ETIMEOUT through the status word and leave the context usable."""
import time

import numpy as np
import pytest

from paper_2103_15039_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_the_context_survives():
    ctx = binding.Context(0, 1024, 1024)
    try:
        t0 = time.perf_counter()
        assert ctx.selftest_timeout(2_000_000) == 4  # ~1 ms of GPU clocks -> ETIMEOUT
        assert time.perf_counter() - t0 < 5.0
        c = synth.sphere_plane_pair(seed=71, n=300, m=400)
        got = ctx.register(c["X"], c["Y"], binding.default_params(max_iters=5))
        assert np.all(np.isfinite(got["R"])) and got["iters"] == 5
        assert ctx.selftest_timeout(0) == 1  # out-of-range budget: EINVAL, nothing launched
    finally:
        ctx.close()
