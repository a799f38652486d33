"""lsgcpd_estep_noalloc: the E step for callers that cannot allocate device
memory (its scratch is a fixed static arena).  It must give the results of
lsgcpd_estep, call after call, although the arena keeps each call's leftovers.
This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2103_15039_gb300 import binding, synth

pytestmark = pytest.mark.gpu

RTOL = 2e-4  # the per-source / global tolerance of the E-step parity tests


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _case(seed, n, m):
    c = synth.estep_case(seed, n, m)
    nrm = c["normals"].astype(np.float64)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    return c, nrm.astype(np.float32)


def _close(a, b):
    scale = np.abs(b).max(axis=0) + 1e-30
    return np.max(np.abs(a - b) / (scale + np.abs(b)))


@pytest.mark.parametrize("order", ["first", "second"])
def test_noalloc_matches_the_context_estep_on_consecutive_calls(order):
    ctx = binding.Context(0, 4096, 4096)
    try:
        p = binding.default_params(w=0.15)
        # two calls in a row with different shapes: the second reuses a dirty arena
        shapes = [(3000, 2500, 11), (1000, 4096, 12)] if order == "first" else [(4096, 700, 13), (2049, 1999, 14)]
        for n, m, seed in shapes:
            c, nrm = _case(seed, n, m)
            args = (_cuda(c["X"]), _cuda(c["Y"]), _cuda(nrm), _cuda(c["alpha"]), c["R"], c["t"], c["sigma2"], 1.5)
            ref = ctx.estep(*args, p, per_n=True)
            got = binding.lsgcpd_estep_noalloc(*args, p, per_n=True)
            assert _close(got["per_n"].cpu().numpy().astype(np.float64),
                          ref["per_n"].cpu().numpy().astype(np.float64)) < RTOL
            g, r = got["moments"], ref["moments"]
            assert np.max(np.abs(g - r) / (np.abs(r) + 1e-12 * np.abs(r).max())) < RTOL
    finally:
        ctx.close()


def test_noalloc_rejects_sizes_beyond_its_arena():
    c, nrm = _case(15, 4097, 10)
    p = binding.default_params()
    with pytest.raises(binding.LsgcpdError) as e:
        binding.lsgcpd_estep_noalloc(_cuda(c["X"]), _cuda(c["Y"]), _cuda(nrm), _cuda(c["alpha"]), c["R"], c["t"],
                                     c["sigma2"], 1.0, p)
    assert e.value.status == 1
