"""The mixed-precision E step (precision = 1: FP32 residuals and accumulation,
exponentials as packed f16x2) against the FP64 oracle, with its stated bound.

Bound: -q is rounded to f16 (relative error <= 2^-12), so the exponent carries
an absolute error of <= 2.4e-4 |q| and each term e = 2^-q a relative error of
<= 1.7e-4 |q| plus that of the f16 EX2 itself (about 1e-3).  The terms that
carry the posterior mass have q of a few units, so moments agree with FP64 to
about 2e-3 of their scale (tested at 5e-3); the normalisation is exact, so the
posteriors with the outlier term still sum to one in FP32.  A registration then
ends within about 1e-3 rad and 1e-4 of the diagonal of the FP64 result.
"""
import numpy as np
import pytest

import oracle
from oracle_forms import per_source
from paper_2103_15039_gb300 import binding, synth

pytestmark = pytest.mark.gpu

BOUND = 5e-3


@pytest.fixture(scope="module")
def ctx():
    c = binding.Context(0, 4096, 4096)
    yield c
    c.close()


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _diag(Y):
    Y = np.asarray(Y, dtype=np.float64)
    return float(np.linalg.norm(Y.max(0) - Y.min(0)))


@pytest.mark.parametrize("n,m", [(129, 257), (700, 1000)])
@pytest.mark.parametrize("w", [0.0, 0.1])
def test_half_exponential_estep_within_bound(ctx, n, m, w):
    case = synth.estep_case(801 + n, n, m)
    X, Y = case["X"], case["Y"]
    nrm = case["normals"].astype(np.float64)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    nrm32 = nrm.astype(np.float32)
    p = binding.default_params(w=w, precision=1)
    g = ctx.estep(_cuda(X), _cuda(Y), _cuda(nrm32), _cuda(case["alpha"]), case["R"], case["t"], case["sigma2"], 1.0, p,
                  per_n=True)
    o = oracle.estep(X, Y, nrm32.astype(np.float64), case["alpha"].astype(np.float64), case["R"], case["t"],
                     case["sigma2"], w, 1.0)
    ref = per_source(o["stats"], X, case["R"], case["t"])
    got = g["per_n"].cpu().numpy().astype(np.float64)
    scale = np.abs(ref).max(axis=0) + 1e-30
    err = np.abs(got[:, :12] - ref[:, :12]) / (scale[:12] + np.abs(ref[:, :12]))
    assert err.max() < BOUND, err.max(axis=0)
    np.testing.assert_allclose(got[:, 0] + got[:, 11], 1.0, atol=1e-5)


def test_half_exponential_registration_within_bound(ctx):
    c = synth.sphere_plane_pair()
    ref = oracle.register(c["X"], c["Y"])
    full = ctx.register(c["X"], c["Y"], binding.default_params())
    half = ctx.register(c["X"], c["Y"], binding.default_params(precision=1))
    assert oracle.rotation_error(full["R"], ref["R"]) < 1e-4
    assert oracle.rotation_error(half["R"], ref["R"]) < 1e-3
    assert np.linalg.norm(half["t"] - ref["t"]) / _diag(c["Y"]) < 1e-4
    assert half["mode"] == 1  # the f16 range needs the per-source shift
