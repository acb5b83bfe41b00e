"""GPU parity of the SVD solvers of the SR system (Sec. 3.5, "Solving linear
systems": non-iterative solvers whose stability is controlled by dropping
small singular values) against the oracle's solve_svd (parameter space) and
solve_svd_samplespace (Ns x Ns Gram), through the C ABI.

The truncated pseudo-inverse is unique, so the solutions are compared, not
the eigenvectors.  Every case keeps its smallest kept eigenvalue well above
the cutoff and its dropped ones at the rounding level, so that rounding
cannot move an eigenvalue across the cutoff; the tolerance is 1e-8 in norm
for spectra whose kept part spans up to ~1e5 (the rounding of FP64 Jacobi
rotations times that condition number is far below it).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2112_10526_gb300 import inputs as I
from paper_2112_10526_gb300 import nk

from gpu_util import cu, dev, ham_to_device, vec_rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    with nk.Ctx() as c:
        yield c


def _solve(ctx, p, N, M, s, F, solver, eps, rcond, prec):
    d = torch.full((F.size,), np.nan, dtype=torch.float64, device=dev())
    info = nk.nk_sr_solve(ctx, cu(p), N, M, cu(s), cu(F), d, solver=solver, diag_shift=eps, cg_tol=rcond,
                          precision=prec)
    assert info["converged"] and info["iters"] >= 1
    return d.cpu().numpy(), info


# (N, M, Ns, sigma, eps): Ns < Np gives a rank-deficient S (eps = 0 drops the
# null space), Ns > Np a full-rank one
PARAM_CASES = [(8, 8, 40, 0.3, 0.0), (8, 8, 256, 0.3, 0.0), (8, 8, 256, 0.3, 0.01), (7, 9, 61, 0.3, 0.0),
               (16, 16, 300, 0.3, 0.001)]


@pytest.mark.parametrize("N,M,Ns,sig,eps", PARAM_CASES)
@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_parameter_space_svd_matches_oracle(ctx, N, M, Ns, sig, eps, prec):
    p = I.rbm_params(N, M, 3, sig)
    s = I.random_configs(Ns, N, 4)
    O = oracle.jacobian(p, N, M, s)
    F = oracle.force(O, np.random.default_rng(5).normal(size=Ns))
    got, info = _solve(ctx, p, N, M, s, F, "svd", eps, 1e-12, prec)
    ref = oracle.solve_svd(oracle.qgt_dense(O), F, eps, 1e-12)
    assert vec_rel_err(got, ref) < 1e-8, info


SS_CASES = [(8, 8, 40, 0.3), (16, 32, 200, 0.3), (37, 45, 129, 0.3), (100, 200, 1024, 0.01)]


@pytest.mark.parametrize("N,M,Ns,sig", SS_CASES)
@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_sample_space_svd_matches_oracle(ctx, N, M, Ns, sig, prec):
    p = I.rbm_params(N, M, 3, sig)
    s = I.random_configs(Ns, N, 4)
    O = oracle.jacobian(p, N, M, s)
    F = oracle.force(O, np.random.default_rng(6).normal(size=Ns))
    got, info = _solve(ctx, p, N, M, s, F, "svd_samplespace", 0.0, 1e-12, prec)
    ref = oracle.solve_svd_samplespace(O, F, 1e-12)
    assert vec_rel_err(got, ref) < 1e-8, info
    if Ns < N + M + M * N <= 2000:
        # the two spaces give the same truncated solve (the dense Np x Np
        # check only where the oracle's host SVD of S stays small)
        assert vec_rel_err(got, oracle.solve_svd(oracle.qgt_dense(O), F, 0.0, 1e-12)) < 1e-8


def test_cutoff_drops_a_gap(ctx):
    """A cutoff between the kept and the dropped part of the spectrum: with
    rcond just above the smallest kept eigenvalue of S, that direction is
    dropped too, and the GPU follows the oracle."""
    N, M, Ns = 8, 8, 40
    p = I.rbm_params(N, M, 3, 0.3)
    s = I.random_configs(Ns, N, 4)
    O = oracle.jacobian(p, N, M, s)
    F = oracle.force(O, np.random.default_rng(7).normal(size=Ns))
    lam = np.sort(np.linalg.eigvalsh(oracle.qgt_dense(O)))[::-1]
    kept = lam[lam > 1e-12 * lam[0]]
    rc = float(np.sqrt(kept[-1] * kept[-2])) / lam[0]  # between the two smallest kept
    got, _ = _solve(ctx, p, N, M, s, F, "svd", 0.0, rc, "f64")
    ref = oracle.solve_svd(oracle.qgt_dense(O), F, 0.0, rc)
    assert vec_rel_err(got, ref) < 1e-8
    assert vec_rel_err(got, oracle.solve_svd(oracle.qgt_dense(O), F, 0.0, 1e-12)) > 1e-6


def test_sr_step_with_svd_matches_oracle(ctx):
    """Two SR steps of the 4 x 4 Heisenberg workload with the sample-space SVD
    solver against the oracle's step with its parameter-space SVD (the same
    truncated solve at eps = 0): samples bit-exact, update at 1e-8.  The
    parameters have sigma = 0.2, which keeps the kept spectrum within a
    factor ~1e4 (at sigma = 0.01 eigenvalues near 1e-10 of the largest are
    kept, and the oracle's own two forms then differ at 1e-3)."""
    N, M, C, ns = 16, 32, 32, 8
    ham = I.heis_square(4)
    p0 = I.rbm_params(N, M, 2, 0.2)
    s0 = oracle.chain_init(N, C, "exchange", 2, 0)
    h, _e = ham_to_device(ham)
    pd, sd = cu(p0), cu(s0)
    ch = nk.make_chains(sd)
    cfg = nk.make_cfg("exchange", "f64", "svd_samplespace", 4, ns, 0.0, 0.02, 2, svd_rcond=1e-12)
    samples = torch.empty((C * ns, N), dtype=torch.int8, device=dev())
    eloc = torch.empty(C * ns, dtype=torch.float64, device=dev())
    p, s, sweep0 = p0, s0, 0
    for it in range(2):
        nd = 4 if it == 0 else 0
        cfg.n_discard = nd
        nk.nk_sr_step(ctx, pd, N, M, h, ch, cfg, None, samples, eloc)
        ref = oracle.sr_step(p, N, M, ham, "exchange", s, sweep0, nd, ns, 2, 0, diag_shift=0.0, lr=0.02,
                             solver="svd", svd_rcond=1e-12)
        sweep0 += nd + ns
        np.testing.assert_array_equal(samples.cpu().numpy(), ref["samples"].reshape(-1, N))
        got = pd.cpu().numpy()
        assert vec_rel_err(got - p, ref["params"] - p) < 1e-8
        p, s = got, ref["state"]


def test_svd_size_limit_is_enforced(ctx):
    N, M, Ns = 100, 200, 64  # Np = 20300 > 8192 for the parameter-space form
    p = cu(I.rbm_params(N, M, 1))
    s = cu(I.random_configs(Ns, N, 1))
    F = cu(np.ones(N + M + M * N))
    d = torch.empty(N + M + M * N, dtype=torch.float64, device=dev())
    with pytest.raises(nk.NkError) as ei:
        nk.nk_sr_solve(ctx, p, N, M, s, F, d, solver="svd", diag_shift=0.0, cg_tol=0.0)
    assert ei.value.code == nk.NK_ERR_INVALID_ARG
