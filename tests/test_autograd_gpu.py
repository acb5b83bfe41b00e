"""The differentiable ln psi (torch.autograd.Function over the hand-written
adjoint kernel) against FP64 central differences (step 1e-6, relative 1e-6)
and the oracle's analytic gradient."""
import numpy as np
import pytest
import torch

import oracle
from paper_2112_10526_gb300 import autograd as ag
from paper_2112_10526_gb300 import inputs as I
from paper_2112_10526_gb300 import nk

from gpu_util import cu, vec_rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    with nk.Ctx() as c:
        yield c


@pytest.mark.parametrize("N,M,B,sig", [(6, 5, 7, 0.5), (16, 16, 64, 0.3), (37, 45, 33, 0.2)])
def test_backward_matches_oracle_and_finite_differences(ctx, N, M, B, sig):
    p = I.rbm_params(N, M, 31, sig)
    s = I.random_configs(B, N, 2)
    w = np.random.default_rng(3).normal(size=B)
    pd = cu(p).requires_grad_(True)
    sd = cu(s)
    y = ag.logpsi(pd, sd, N, M, ctx)
    (y * cu(w)).sum().backward()
    got = pd.grad.detach().cpu().numpy()
    ref = oracle.jacobian(p, N, M, s).T @ w
    assert vec_rel_err(got, ref) < 1e-12
    # central differences of the GPU forward itself, FP64, step 1e-6
    if N * M <= 100:
        h = 1e-6
        with torch.no_grad():
            for k in range(p.size):
                pp, pm = p.copy(), p.copy()
                pp[k] += h
                pm[k] -= h
                fp = (ag.logpsi(cu(pp), sd, N, M, ctx).cpu().numpy() * w).sum()
                fm = (ag.logpsi(cu(pm), sd, N, M, ctx).cpu().numpy() * w).sum()
                fd = (fp - fm) / (2 * h)
                assert abs(got[k] - fd) <= 1e-6 * max(1.0, abs(fd))


def test_per_sample_gradients(ctx):
    N, M, B = 10, 12, 25
    p = I.rbm_params(N, M, 4, 0.4)
    s = I.random_configs(B, N, 5)
    O = ag.per_sample_grad(cu(p), cu(s), N, M, ctx)
    np.testing.assert_allclose(O.cpu().numpy(), oracle.jacobian(p, N, M, s), rtol=1e-13, atol=1e-14)


def test_mixed_backward(ctx):
    N, M, B = 100, 200, 300
    p = I.rbm_params(N, M, 6, 0.01)
    s = I.random_configs(B, N, 6)
    w = np.random.default_rng(1).normal(size=B)
    pd = cu(p).requires_grad_(True)
    y = ag.logpsi(pd, cu(s), N, M, ctx, precision="mixed")
    (y * cu(w)).sum().backward()
    ref = oracle.jacobian(p, N, M, s).T @ w
    assert vec_rel_err(pd.grad.detach().cpu().numpy(), ref) < 1e-8
