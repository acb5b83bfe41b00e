"""GPU-vs-oracle parity of the MetropolisHamiltonian rule (Sec. 3.4): for a
Heisenberg-type Hamiltonian the proposal is a uniformly chosen swap across
one of the n(s) antiparallel edges, accepted with the Hastings correction
ln n(s) - ln n(s').  Chains replayed by the oracle following the GPU's
decisions must give the same samples; decisions may differ only inside the
tie band (1e-9 FP64, 1e-4 max(1, |2 dlnpsi|) mixed)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2112_10526_gb300 import inputs as I
from paper_2112_10526_gb300 import nk

from gpu_util import cu, dev, ham_to_device, rel_err, vec_rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    with nk.Ctx() as c:
        yield c


def _lnu(seed, stream, C, N, n_sweeps, sweep0):
    out = np.empty((C, n_sweeps, N))
    for c in range(C):
        for w in range(n_sweeps):
            for q in range(N):
                y = oracle.philox4x64_10(np.array([(sweep0 + w) * N + q, c, stream, 0], dtype=np.uint64),
                                         np.array([seed, 0], dtype=np.uint64))
                out[c, w, q] = np.log(((int(y[1]) >> 11) + 0.5) * 2.0 ** -53)
    return out


def _replay(ctx, p, N, M, edges, s0, sweep0, nd, ns, seed, stream, prec, K=None):
    C = s0.shape[0]
    st = cu(s0)
    samples = torch.empty((C, ns, N), dtype=torch.int8, device=dev())
    lp = torch.empty((C, ns), dtype=torch.float64, device=dev())
    nacc = torch.zeros(C, dtype=torch.int64, device=dev())
    dec = torch.empty((C, nd + ns, N), dtype=torch.uint8, device=dev())
    nk.nk_metropolis_sweep(ctx, cu(p), N, M, "hamiltonian", cu(edges), st, sweep0, nd, ns, seed, stream, samples,
                           lp, nacc, dec, precision=prec)
    K = C if K is None else K
    g_dec = dec.cpu().numpy()
    ref = oracle.metropolis(p, N, M, "hamiltonian", edges, s0[:K], sweep0, nd, ns, seed, stream,
                            forced=g_dec[:K])
    mism = ref["decisions"] != g_dec[:K]
    if prec == "f64":
        allowed = ref["margin"] < 1e-9
    else:
        lu = _lnu(seed, stream, K, N, nd + ns, sweep0)
        two_d = lu + np.where(ref["decisions"] == 1, 1, -1) * ref["margin"]
        allowed = ref["margin"] < 1e-4 * np.maximum(1.0, np.abs(two_d))
    assert not (mism & ~allowed).any(), f"{int((mism & ~allowed).sum())} decisions differ outside the tie band"
    np.testing.assert_array_equal(samples.cpu().numpy()[:K], ref["samples"])
    np.testing.assert_array_equal(st.cpu().numpy()[:K], ref["state"])
    assert rel_err(lp.cpu().numpy()[:K], ref["logpsi"]) < (1e-10 if prec == "f64" else 1e-4)
    # at S_z = 0 on a connected lattice every proposal is a move, and S_z stays 0
    assert set(np.unique(g_dec)) <= {0, 1}
    assert (st.cpu().numpy().astype(np.int64).sum(axis=1) == 0).all()
    np.testing.assert_array_equal(nacc.cpu().numpy(), (g_dec == 1).sum(axis=(1, 2)))
    return int(mism.sum())


REPLAY_CASES = [
    ("ring12", 12, 5, 16, 2, 3, 0.4, lambda: I.chain_edges(12)),
    ("sq4", 16, 32, 12, 2, 4, 0.3, lambda: I.square_edges(4)),
    ("j1j2-sq4", 16, 32, 12, 2, 4, 0.3, lambda: I.j1j2_square(4)["edges"]),
    ("sq6-ragged-M", 36, 37, 9, 1, 3, 0.2, lambda: I.square_edges(6)),
]


@pytest.mark.parametrize("name,N,M,C,nd,ns,sig,ef", REPLAY_CASES, ids=[c[0] for c in REPLAY_CASES])
@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_hamiltonian_rule_replay(ctx, name, N, M, C, nd, ns, sig, ef, prec):
    p = I.rbm_params(N, M, 5 + N, sig)
    s0 = oracle.chain_init(N, C, "hamiltonian", 41, 2)
    n = _replay(ctx, p, N, M, ef(), s0, 7, nd, ns, 41, 2, prec)
    print(f"tie-band mismatches: {n}")


def test_chain_init_hamiltonian_rule_is_sz0(ctx):
    N, C = 100, 65
    s = torch.empty((C, N), dtype=torch.int8, device=dev())
    nk.nk_chains_init(ctx, N, C, "hamiltonian", 3, 1, s)
    np.testing.assert_array_equal(s.cpu().numpy(), oracle.chain_init(N, C, "hamiltonian", 3, 1))


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_hamiltonian_rule_full_size_10x10_sampled_chains(ctx, prec):
    """The sweep configuration of the 10 x 10 Heisenberg workload (1024
    chains, 16 discarded + 8 sampled sweeps, N = 100, M = 200, sigma = 0.01)
    with the Hamiltonian rule; the first 16 chains are replayed by the
    oracle."""
    N, M, C = 100, 200, 1024
    p = I.rbm_params(N, M, 2)
    s0 = oracle.chain_init(N, C, "hamiltonian", 2, 0)
    _replay(ctx, p, N, M, I.square_edges(10), s0, 0, 16, 8, 2, 0, prec, K=16)


def _sr_compare(ctx, ham, rule, N, M, C, nd, ns, seed, solver, steps=2):
    p0 = I.rbm_params(N, M, seed, 0.1)
    s0 = oracle.chain_init(N, C, "local" if ham["kind"] == "tfim" else "hamiltonian", seed, 0)
    h, _e = ham_to_device(ham)
    pd, sd = cu(p0), cu(s0)
    ch = nk.make_chains(sd)
    cfg = nk.make_cfg(rule, "f64", solver, nd, ns, 0.01, 0.02, seed, cg_tol=1e-10, cg_maxiter=2000)
    stats = torch.empty(nk.SR_STATS_DOUBLES, dtype=torch.float64, device=dev())
    samples = torch.empty((C * ns, N), dtype=torch.int8, device=dev())
    eloc = torch.empty(C * ns, dtype=torch.float64, device=dev())
    p, s, sweep0 = p0, s0, 0
    for it in range(steps):
        cfg.n_discard = nd if it == 0 else 0
        nk.nk_sr_step(ctx, pd, N, M, h, ch, cfg, stats, samples, eloc)
        g_params = pd.cpu().numpy().copy()
        ref = oracle.sr_step(p, N, M, ham, rule, s, sweep0, cfg.n_discard, ns, seed, 0, diag_shift=0.01,
                             lr=0.02, solver="cg" if solver == "cg" else "cholesky", cg_tol=1e-10)
        sweep0 += cfg.n_discard + ns
        np.testing.assert_array_equal(samples.cpu().numpy(), ref["samples"].reshape(-1, N))
        assert rel_err(eloc.cpu().numpy(), ref["eloc"]) < 1e-10
        assert vec_rel_err(g_params - p, ref["params"] - p) < 1e-7
        p, s = g_params, ref["state"]
        np.testing.assert_array_equal(sd.cpu().numpy(), s)


@pytest.mark.parametrize("solver", ["cholesky_samplespace", "cg"])
def test_sr_step_hamiltonian_rule_heisenberg(ctx, solver):
    _sr_compare(ctx, I.heis_square(4), "hamiltonian", 16, 32, 32, 4, 8, 3, solver)


def test_sr_step_hamiltonian_rule_j1j2_and_zero_j2(ctx):
    """Both edge classes propose when J2 != 0; with J2 = 0 the second class
    connects nothing and drops out of the proposal."""
    _sr_compare(ctx, I.j1j2_square(4, 1.0, 0.5), "hamiltonian", 16, 32, 32, 4, 8, 4, "cholesky_samplespace")
    _sr_compare(ctx, I.j1j2_square(4, 1.0, 0.0), "hamiltonian", 16, 32, 32, 4, 8, 4, "cholesky_samplespace")


def test_sr_step_hamiltonian_rule_ising_is_the_local_rule(ctx):
    """The Ising model's connected configurations are the N single flips, drawn
    uniformly with the local rule's index: same chains as the oracle's local
    rule."""
    _sr_compare(ctx, I.tfim_chain(16), "hamiltonian", 16, 16, 16, 16, 64, 1, "cholesky")


def test_unknown_rule_is_rejected(ctx):
    s = torch.empty((3, 4), dtype=torch.int8, device=dev())
    with pytest.raises(nk.NkError) as ei:
        nk.nk_chains_init(ctx, 4, 3, 3, 1, 0, s)
    assert ei.value.code == nk.NK_ERR_INVALID_ARG
