"""GPU parity of the symmetric RBM (RBMSymm, Sec. 5) against the oracle in
oracle/symm.py, through the C ABI.

The model is a plain RBM with alpha |G| tied hidden units, so the sampler and
the local energies are the plain kernels on the expanded parameters; what is
new on the GPU is the expansion, the permutation check, the Jacobian in the
symmetric parameters (a sum over the group per parameter) and the SR step in
those parameters.  Tolerances as for the plain RBM: 1e-10 (NK_F64) and 1e-4
(NK_MIXED local energies), solves 1e-8, samples bit-exact on the FP64 path.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import symm as osymm
from paper_2112_10526_gb300 import inputs as I
from paper_2112_10526_gb300 import nk

from gpu_util import cu, dev, ham_to_device, rel_err, vec_rel_err

pytestmark = pytest.mark.gpu

GROUPS = {
    "chain12": (12, lambda: I.translations_chain(12)),
    "square4": (16, lambda: I.translations_square(4)),
    # the paper's example group: the identity and the swap of the first and last site
    "swap4": (4, lambda: np.array([[0, 1, 2, 3], [3, 1, 2, 0]])),
    "chain37": (37, lambda: I.translations_chain(37)),
}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    with nk.Ctx() as c:
        yield c


def _perms(p):
    return cu(np.asarray(p, dtype=np.int32))


@pytest.mark.parametrize("group", list(GROUPS))
@pytest.mark.parametrize("alpha", [1, 3])
def test_expand_is_the_oracles(ctx, group, alpha):
    N, pf = GROUPS[group]
    perms = pf()
    p = np.random.default_rng(alpha).normal(size=osymm.n_params(N, alpha)) * 0.3
    M = alpha * perms.shape[0]
    out = torch.full((N + M + M * N,), np.nan, dtype=torch.float64, device=dev())
    nk.nk_symm_expand(ctx, cu(p), N, alpha, _perms(perms), out)
    np.testing.assert_array_equal(out.cpu().numpy(), osymm.expand(p, N, alpha, perms))


def test_rows_that_are_not_permutations_are_rejected(ctx):
    N, alpha = 6, 2
    p = cu(np.zeros(osymm.n_params(N, alpha)))
    out = torch.empty(N + 2 * alpha * N + 2 * alpha * N * N, dtype=torch.float64, device=dev())
    for bad in ([[0, 1, 2, 3, 4, 5], [1, 1, 2, 3, 4, 5]], [[0, 1, 2, 3, 4, 5], [0, 1, 2, 3, 4, 6]],
                [[0, 1, 2, 3, 4, 5], [-1, 1, 2, 3, 4, 5]]):
        with pytest.raises(nk.NkError) as ei:
            nk.nk_symm_expand(ctx, p, N, alpha, _perms(bad), out)
        assert ei.value.code == nk.NK_ERR_INVALID_ARG


@pytest.mark.parametrize("group", ["chain12", "square4", "swap4", "chain37"])
@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_jacobian_is_the_oracles(ctx, group, prec):
    N, pf = GROUPS[group]
    perms = pf()
    alpha = 2
    p = np.random.default_rng(5).normal(size=osymm.n_params(N, alpha)) * 0.2
    s = I.random_configs(133, N, 9)
    O = torch.empty((133, osymm.n_params(N, alpha)), dtype=torch.float64, device=dev())
    nk.nk_symm_jacobian(ctx, cu(p), N, alpha, _perms(perms), cu(s), O, precision=prec)
    ref = osymm.jacobian(p, N, alpha, perms, s)
    assert rel_err(O.cpu().numpy(), ref) < 1e-10


def test_psi_is_invariant_under_the_group(ctx):
    """ln psi of the expanded RBM (nk_rbm_logpsi) is the same on s and on every
    image of s under the group: psi transforms under the trivial irrep."""
    N, alpha = 16, 2
    perms = I.translations_square(4)
    p = np.random.default_rng(2).normal(size=osymm.n_params(N, alpha)) * 0.3
    M = alpha * perms.shape[0]
    plain = torch.empty(N + M + M * N, dtype=torch.float64, device=dev())
    nk.nk_symm_expand(ctx, cu(p), N, alpha, _perms(perms), plain)
    s = I.random_configs(7, N, 3)
    images = np.concatenate([s[:, perms[g]] for g in range(perms.shape[0])])
    out = torch.empty(images.shape[0], dtype=torch.float64, device=dev())
    nk.nk_rbm_logpsi(ctx, plain, N, M, cu(images), out)
    lp = out.cpu().numpy().reshape(perms.shape[0], 7)
    assert np.abs(lp - lp[0]).max() < 1e-12 * np.abs(lp).max()
    np.testing.assert_allclose(lp[0], osymm.logpsi(p, N, alpha, perms, s), rtol=1e-12)


STEP_CASES = [
    ("tfim-chain16", 16, lambda: I.translations_chain(16), 2, lambda: I.tfim_chain(16, 1.0, 0.8), "local", 16, 32),
    ("heis-square4", 16, lambda: I.translations_square(4), 1, lambda: I.heis_square(4), "exchange", 32, 8),
]


@pytest.mark.parametrize("name,N,pf,alpha,hf,rule,C,ns", STEP_CASES, ids=[c[0] for c in STEP_CASES])
def test_sr_step_f64_matches_oracle(ctx, name, N, pf, alpha, hf, rule, C, ns):
    """Three SR steps of the symmetric RBM on the FP64 path: samples bit-exact
    against the oracle's chains on the same Philox streams, local energies at
    1e-10, statistics, and the parameter update at 1e-8."""
    perms, ham = pf(), hf()
    p0 = np.random.default_rng(4).normal(size=osymm.n_params(N, alpha)) * 0.05
    s0 = oracle.chain_init(N, C, rule, 7, 0)
    h, _e = ham_to_device(ham)
    pd, sd, pg = cu(p0), cu(s0), _perms(perms)
    ch = nk.make_chains(sd)
    cfg = nk.make_cfg(rule, "f64", "cholesky", 8, ns, 0.01, 0.02, 7)
    stats = torch.empty(nk.SR_STATS_DOUBLES, dtype=torch.float64, device=dev())
    samples = torch.empty((C * ns, N), dtype=torch.int8, device=dev())
    eloc = torch.empty(C * ns, dtype=torch.float64, device=dev())
    p, s, sweep0 = p0, s0, 0
    for it in range(3):
        nd = 8 if it == 0 else 0
        cfg.n_discard = nd
        nk.nk_symm_sr_step(ctx, pd, N, alpha, pg, h, ch, cfg, stats, samples, eloc)
        ref = osymm.sr_step(p, N, alpha, perms, ham, rule, s, sweep0, nd, ns, 7, 0, diag_shift=0.01, lr=0.02)
        sweep0 += nd + ns
        np.testing.assert_array_equal(samples.cpu().numpy(), ref["samples"].reshape(-1, N))
        assert rel_err(eloc.cpu().numpy(), ref["eloc"]) < 1e-10
        st = nk.sr_stats_dict(stats)
        assert abs(st["energy"] - ref["stats"]["mean"]) <= 1e-10 * abs(ref["stats"]["mean"])
        got = pd.cpu().numpy()
        assert vec_rel_err(got - p, ref["params"] - p) < 1e-8
        np.testing.assert_array_equal(sd.cpu().numpy(), ref["state"])
        p, s = got, ref["state"]


@pytest.mark.parametrize("name,N,pf,alpha,hf,rule,C,ns", STEP_CASES, ids=[c[0] for c in STEP_CASES])
def test_sr_step_mixed_against_oracle_on_its_samples(ctx, name, N, pf, alpha, hf, rule, C, ns):
    """NK_MIXED: the local energies of the GPU's own samples at 1e-4 against
    the oracle, and the update equal, at 1e-8, to the oracle's dense solve of
    the same samples and local energies (the tensor-core Gram and Cholesky are
    FP64-accurate)."""
    perms, ham = pf(), hf()
    p0 = np.random.default_rng(4).normal(size=osymm.n_params(N, alpha)) * 0.05
    h, _e = ham_to_device(ham)
    pd, pg = cu(p0), _perms(perms)
    sd = torch.empty((C, N), dtype=torch.int8, device=dev())
    nk.nk_chains_init(ctx, N, C, rule, 7, 0, sd)
    ch = nk.make_chains(sd)
    cfg = nk.make_cfg(rule, "mixed", "cholesky", 8, ns, 0.01, 0.02, 7)
    samples = torch.empty((C * ns, N), dtype=torch.int8, device=dev())
    eloc = torch.empty(C * ns, dtype=torch.float64, device=dev())
    p = p0
    for it in range(3):
        cfg.n_discard = 8 if it == 0 else 0
        nk.nk_symm_sr_step(ctx, pd, N, alpha, pg, h, ch, cfg, None, samples, eloc)
        sm, e = samples.cpu().numpy(), eloc.cpu().numpy()
        assert rel_err(e, osymm.local_energy(p, N, alpha, perms, ham, sm)) < 1e-4
        O = osymm.jacobian(p, N, alpha, perms, sm)
        delta = oracle.solve_cholesky(oracle.qgt_dense(O), oracle.force(O, e), 0.01)
        got = pd.cpu().numpy()
        assert vec_rel_err((p - got) / 0.02, delta) < 1e-8
        p = got


def test_sr_step_solver_other_than_cholesky_is_refused(ctx):
    N, alpha = 8, 1
    perms = I.translations_chain(8)
    h, _e = ham_to_device(I.tfim_chain(8))
    sd = torch.empty((4, N), dtype=torch.int8, device=dev())
    nk.nk_chains_init(ctx, N, 4, "local", 1, 0, sd)
    cfg = nk.make_cfg("local", "f64", "cg", 0, 2, 0.01, 0.01, 1)
    with pytest.raises(nk.NkError) as ei:
        nk.nk_symm_sr_step(ctx, cu(np.zeros(osymm.n_params(N, alpha))), N, alpha, _perms(perms), h,
                           nk.make_chains(sd), cfg)
    assert ei.value.code == nk.NK_ERR_UNIMPLEMENTED
