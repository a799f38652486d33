"""Element-by-element parity of the posteriors P_mn of Eq. (5) with the FP64
oracle's literal E step, through lsgcpd_posteriors.

Tolerance: each exponent q = c d + lambda (+ L_n) is formed in FP32 from
magnitudes up to ~200, an absolute error of ~1e-5 in log2 units, plus 2^-22
for ex2.approx: ~2e-5 relative per element; tested at 1e-4 relative (+1e-9
absolute for underflowing tails).  The f16x2-exponential variant is held to its
stated bound (5e-3 relative to the largest posterior of the source).
"""
import numpy as np
import pytest

import oracle
from paper_2103_15039_gb300 import binding, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = binding.Context(0, 2048, 2048)
    yield c
    c.close()


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _case(seed, n, m, alpha_max=2.0):
    case = synth.estep_case(seed, n, m, alpha_max=alpha_max)
    nrm = case["normals"].astype(np.float64)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    case["nrm32"] = nrm.astype(np.float32)
    return case


def _dense(ctx, case, w, V, **kw):
    phi_x = kw.pop("phi_x", None)
    phi_y = kw.pop("phi_y", None)
    p = binding.default_params(w=w, **kw)
    P = ctx.posteriors(_cuda(case["X"]), _cuda(case["Y"]), _cuda(case["nrm32"]), _cuda(case["alpha"]), case["R"],
                       case["t"], case["sigma2"], V, p,
                       phi_x=None if phi_x is None else _cuda(phi_x), phi_y=None if phi_y is None else _cuda(phi_y))
    return P.cpu().numpy().astype(np.float64)


def _ref(case, w, V, **kw):
    o = oracle.estep(case["X"], case["Y"], case["nrm32"].astype(np.float64), case["alpha"].astype(np.float64),
                     case["R"], case["t"], case["sigma2"], w, V, dense=True, **kw)
    return np.vstack([o["P"], o["stats"][:, 14][None, :]])


@pytest.mark.parametrize("n,m", [(1, 1), (31, 33), (129, 257), (700, 1000)])
@pytest.mark.parametrize("w", [0.0, 0.1])
def test_dense_posteriors_match_oracle(ctx, n, m, w):
    case = _case(900 + n + m, n, m)
    got, ref = _dense(ctx, case, w, 1.0), _ref(case, w, 1.0)
    np.testing.assert_allclose(got, ref, rtol=1e-4, atol=1e-9)
    np.testing.assert_allclose(got.sum(axis=0), 1.0, atol=1e-5)


def test_dense_posteriors_with_gaussian_constant_and_confidences(ctx):
    case = _case(951, 300, 400, alpha_max=10.0)
    rng = np.random.default_rng(951)
    px = rng.uniform(0.1, 1.0, 300).astype(np.float32)
    py = rng.uniform(0.1, 1.0, 400).astype(np.float32)
    got = _dense(ctx, case, 0.2, 2.0, include_alpha_norm=1, phi_x=px, phi_y=py)
    pi = py.astype(np.float64) / py.astype(np.float64).sum()
    wn = 1.0 - 0.8 * px.astype(np.float64)
    ref = _ref(case, 0.2, 2.0, include_alpha_norm=True, pi_m=pi, w_n=wn)
    np.testing.assert_allclose(got, ref, rtol=1e-4, atol=1e-9)


def test_dense_posteriors_half_exponentials_within_bound(ctx):
    case = _case(961, 200, 300)
    got = _dense(ctx, case, 0.1, 1.0, precision=1)
    ref = _ref(case, 0.1, 1.0)
    scale = ref.max(axis=0, keepdims=True)
    assert (np.abs(got - ref) / scale).max() < 5e-3
