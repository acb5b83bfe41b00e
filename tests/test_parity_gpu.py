"""GPU-vs-oracle parity of every hot-path entry point, called through the C ABI.

Tolerances (the FP64 path / the mixed path):
  * ln psi, E_loc per sample: 1e-10 / 1e-4 relative (relative to
    max(|ref|, rms of the batch));
  * integer and index work (chain states, samples, accept decisions): bit-exact,
    except Metropolis decisions whose margin |2 dlnpsi - ln u| is below 1e-9
    (FP64) or 1e-4 max(1, |2 dlnpsi|) (mixed), which are counted;
  * vectors (force, vjp, jvp, QGT products): 1e-10 in norm (FP64 path);
  * linear solves: 1e-8 in norm (the conditioning of S + eps I amplifies
    rounding of the right-hand side).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2112_10526_gb300 import inputs as I
from paper_2112_10526_gb300 import nk

from gpu_util import cu, dev, ham_to_device, rel_err, vec_rel_err

pytestmark = pytest.mark.gpu

LOGPSI_CASES = [(16, 16, 1000, 0.01), (100, 200, 777, 0.01), (37, 53, 129, 0.5), (400, 1600, 70, 0.01),
                (1, 1, 5, 0.3)]


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    with nk.Ctx() as c:
        yield c


@pytest.mark.parametrize("N,M,B,sig", LOGPSI_CASES)
@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_logpsi(ctx, N, M, B, sig, prec):
    p = I.rbm_params(N, M, N + M, sig)
    s = I.random_configs(B, N, 7)
    out = torch.empty(B, dtype=torch.float64, device=dev())
    nk.nk_rbm_logpsi(ctx, cu(p), N, M, cu(s), out, precision=prec)
    ref = oracle.logpsi(p, N, M, s)
    assert rel_err(out.cpu().numpy(), ref) < 1e-10


def test_logpsi_empty_batch(ctx):
    p = cu(I.rbm_params(4, 4, 1))
    out = torch.empty(0, dtype=torch.float64, device=dev())
    nk.nk_rbm_logpsi(ctx, p, 4, 4, torch.empty((0, 4), dtype=torch.int8, device=dev()), out)


@pytest.mark.parametrize("N,C,rule", [(300, 33, "local"), (100, 65, "exchange"), (16, 16, "local"),
                                      (2, 3, "exchange")])
def test_chain_init_bit_exact(ctx, N, C, rule):
    s = torch.empty((C, N), dtype=torch.int8, device=dev())
    nk.nk_chains_init(ctx, N, C, rule, 12345, 7, s)
    np.testing.assert_array_equal(s.cpu().numpy(), oracle.chain_init(N, C, rule, 12345, 7))


def _lnu(seed, stream, C, N, n_sweeps, sweep0):
    """ln u of every proposal, from the oracle's Philox (for the mixed tolerance)."""
    out = np.empty((C, n_sweeps, N))
    for c in range(C):
        for w in range(n_sweeps):
            for q in range(N):
                y = oracle.philox4x64_10(np.array([(sweep0 + w) * N + q, c, stream, 0], dtype=np.uint64),
                                         np.array([seed, 0], dtype=np.uint64))
                out[c, w, q] = np.log(((int(y[1]) >> 11) + 0.5) * 2.0 ** -53)
    return out


SWEEP_CASES = [
    ("local", 16, 16, 16, 3, 5, 0.3, None),
    ("local", 20, 40, 9, 2, 3, 0.5, None),
    ("exchange", 16, 32, 12, 2, 4, 0.3, "sq4"),
    ("exchange", 36, 72, 8, 1, 3, 0.2, "sq6"),
    ("exchange", 12, 5, 4, 0, 2, 0.4, "ring12"),
]


@pytest.mark.parametrize("rule,N,M,C,nd,ns,sig,lat", SWEEP_CASES)
@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_metropolis_replay(ctx, rule, N, M, C, nd, ns, sig, lat, prec):
    p = I.rbm_params(N, M, 3 + N, sig)
    edges = None
    if lat == "sq4":
        edges = I.square_edges(4)
    elif lat == "sq6":
        edges = I.square_edges(6)
    elif lat == "ring12":
        edges = I.chain_edges(12)
    s0 = oracle.chain_init(N, C, rule, 99, 1)
    sweep0 = 5
    st = cu(s0)
    samples = torch.empty((C, ns, N), dtype=torch.int8, device=dev())
    lp = torch.empty((C, ns), dtype=torch.float64, device=dev())
    nacc = torch.zeros(C, dtype=torch.int64, device=dev())
    dec = torch.empty((C, nd + ns, N), dtype=torch.uint8, device=dev())
    e_dev = None if edges is None else cu(edges)
    nk.nk_metropolis_sweep(ctx, cu(p), N, M, rule, e_dev, st, sweep0, nd, ns, 99, 1, samples, lp, nacc,
                           dec, precision=prec)
    g_dec = dec.cpu().numpy()
    ref = oracle.metropolis(p, N, M, rule, edges, s0, sweep0, nd, ns, 99, 1, forced=g_dec)
    mism = ref["decisions"] != g_dec
    if prec == "f64":
        allowed = ref["margin"] < 1e-9
    else:
        lu = _lnu(99, 1, C, N, nd + ns, sweep0)
        two_d = lu + np.where(ref["decisions"] == 1, 1, -1) * ref["margin"]
        allowed = ref["margin"] < 1e-4 * np.maximum(1.0, np.abs(two_d))
    assert not (mism & ~allowed).any(), f"{int((mism & ~allowed).sum())} decisions differ outside the tie band"
    # with the oracle following the GPU decisions the trajectories coincide exactly
    np.testing.assert_array_equal(samples.cpu().numpy(), ref["samples"])
    np.testing.assert_array_equal(st.cpu().numpy(), ref["state"])
    np.testing.assert_array_equal(nacc.cpu().numpy(), (g_dec == 1).sum(axis=(1, 2)))
    tol = 1e-10 if prec == "f64" else 1e-4
    assert rel_err(lp.cpu().numpy(), ref["logpsi"]) < tol
    print(f"tie-band mismatches: {int(mism.sum())} of {mism.size}")


ELOC_CASES = [
    ("tfim-chain16", 16, 16, lambda: I.tfim_chain(16, 1.0, 1.0), 1000, False, 0.01),
    ("tfim-chain16-s0.5", 16, 16, lambda: I.tfim_chain(16, 1.0, 1.0), 333, False, 0.5),
    ("heis-4x4-marshall", 16, 32, lambda: I.heis_square(4, 1.0, True), 500, True, 0.3),
    ("heis-4x4-plain", 16, 8, lambda: I.heis_square(4, 0.7, False), 200, True, 0.3),
    ("heis-10x10", 100, 200, lambda: I.heis_square(10, 1.0, True), 300, True, 0.01),
    ("tfim-20x20", 400, 1600, lambda: I.tfim_square(20, 1.0, 3.04), 40, False, 0.01),
    ("heis-24x24", 576, 4608, lambda: I.heis_square(24, 1.0, True), 6, True, 0.01),
    ("tfim-ragged", 37, 45, lambda: I.tfim_chain(37, -0.6, 0.9), 65, False, 0.4),
]


@pytest.mark.parametrize("name,N,M,hf,B,sz0,sig", ELOC_CASES, ids=[c[0] for c in ELOC_CASES])
@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_local_energy(ctx, name, N, M, hf, B, sz0, sig, prec):
    ham = hf()
    p = I.rbm_params(N, M, 17, sig)
    s = I.random_configs(B, N, 5, sz0=sz0)
    h, _e = ham_to_device(ham)
    out = torch.empty(B, dtype=torch.float64, device=dev())
    t = torch.empty((B, M), dtype=torch.float64, device=dev())
    nk.nk_local_energy(ctx, cu(p), N, M, h, cu(s), out, t, precision=prec)
    ref = oracle.local_energy(p, N, M, ham, s)
    assert rel_err(out.cpu().numpy(), ref) < (1e-10 if prec == "f64" else 1e-4)
    O = oracle.jacobian(p, N, M, s)
    assert rel_err(t.cpu().numpy(), O[:, N:N + M]) < 1e-12


@pytest.mark.parametrize("Ns,C", [(1024, 16), (8192, 1024), (777, 1), (5, 5)])
def test_stats(ctx, Ns, C):
    e = np.random.default_rng(Ns).normal(-20, 3, Ns)
    out = torch.empty(3, dtype=torch.float64, device=dev())
    nk.nk_stats(ctx, cu(e), C, out)
    ref = oracle.stats(e, n_chains=C)
    got = out.cpu().numpy()
    assert abs(got[0] - ref["mean"]) < 1e-14 * abs(ref["mean"])
    assert abs(got[1] - ref["variance"]) < 1e-12 * ref["variance"]
    assert abs(got[2] - ref["error"]) < 1e-10 * ref["error"]


JAC_CASES = [(16, 16, 1024, 0.3), (100, 200, 300, 0.01), (37, 45, 131, 0.4), (3, 2, 1, 0.5)]


@pytest.mark.parametrize("N,M,Ns,sig", JAC_CASES)
def test_jacobian_vjp_jvp_force(ctx, N, M, Ns, sig):
    p = I.rbm_params(N, M, 5, sig)
    s = I.random_configs(Ns, N, 9)
    Np = N + M + M * N
    O = oracle.jacobian(p, N, M, s)
    pd, sd = cu(p), cu(s)
    Og = torch.empty((Ns, Np), dtype=torch.float64, device=dev())
    nk.nk_jacobian(ctx, pd, N, M, sd, False, 0, Ns, Og)
    assert rel_err(Og.cpu().numpy(), O) < 1e-12
    # rows subset of the centred Jacobian
    r0, nr = Ns // 3, max(1, Ns // 2)
    nr = min(nr, Ns - r0)
    Oc = torch.empty((nr, Np), dtype=torch.float64, device=dev())
    nk.nk_jacobian(ctx, pd, N, M, sd, True, r0, nr, Oc)
    dJ = O - O.sum(axis=0) / Ns
    assert vec_rel_err(Oc.cpu().numpy(), dJ[r0:r0 + nr]) < 1e-10
    rng = np.random.default_rng(1)
    g = rng.normal(size=Ns)
    out = torch.empty(Np, dtype=torch.float64, device=dev())
    nk.nk_vjp(ctx, pd, N, M, sd, cu(g), out)
    assert vec_rel_err(out.cpu().numpy(), O.T @ g) < 1e-10
    v = rng.normal(size=Np)
    w = torch.empty(Ns, dtype=torch.float64, device=dev())
    nk.nk_jvp(ctx, pd, N, M, sd, cu(v), w)
    assert vec_rel_err(w.cpu().numpy(), O @ v) < 1e-10
    e = rng.normal(-5, 1, size=Ns)
    F = torch.empty(Np, dtype=torch.float64, device=dev())
    nk.nk_force(ctx, pd, N, M, sd, cu(e), F)
    assert vec_rel_err(F.cpu().numpy(), oracle.force(O, e)) < 1e-10


@pytest.mark.parametrize("N,M,Ns", [(16, 16, 1024), (36, 72, 500), (7, 5, 33)])
def test_qgt_matvec_both_forms(ctx, N, M, Ns):
    p = I.rbm_params(N, M, 8, 0.3)
    s = I.random_configs(Ns, N, 2)
    Np = N + M + M * N
    O = oracle.jacobian(p, N, M, s)
    v = np.random.default_rng(3).normal(size=Np)
    ref = oracle.qgt_matvec_onthefly(O, v, 0.01)
    out = torch.empty(Np, dtype=torch.float64, device=dev())
    nk.nk_qgt_matvec(ctx, cu(v), out, 0.01, params=cu(p), N=N, M=M, s=cu(s))
    assert vec_rel_err(out.cpu().numpy(), ref) < 1e-10
    dJ = torch.empty((Ns, Np), dtype=torch.float64, device=dev())
    nk.nk_jacobian(ctx, cu(p), N, M, cu(s), True, 0, Ns, dJ)
    out2 = torch.empty(Np, dtype=torch.float64, device=dev())
    nk.nk_qgt_matvec(ctx, cu(v), out2, 0.01, dJ=dJ)
    assert vec_rel_err(out2.cpu().numpy(), ref) < 1e-10


@pytest.mark.parametrize("solver", ["cholesky", "cholesky_samplespace", "cg"])
@pytest.mark.parametrize("N,M,Ns,eps", [(16, 16, 1024, 0.01), (10, 20, 100, 0.05), (6, 6, 700, 0.01),
                                        (12, 12, 130, 0.1)])
def test_sr_solve(ctx, solver, N, M, Ns, eps):
    p = I.rbm_params(N, M, 4, 0.3)
    s = I.random_configs(Ns, N, 6)
    Np = N + M + M * N
    O = oracle.jacobian(p, N, M, s)
    F = np.random.default_rng(2).normal(size=Np) * 0.1
    ref = oracle.solve_cholesky(oracle.qgt_dense(O), F, eps)
    d = torch.empty(Np, dtype=torch.float64, device=dev())
    info = nk.nk_sr_solve(ctx, cu(p), N, M, cu(s), cu(F), d, solver=solver, diag_shift=eps, cg_tol=1e-12,
                          cg_maxiter=5000)
    if solver == "cg":
        assert info["converged"] and info["residual"] <= 1e-12
    assert vec_rel_err(d.cpu().numpy(), ref) < 1e-8


def _sr_run(ctx, N, M, hamf, rule, C, nd, ns, seed, solver, eps, lr, steps, prec="f64"):
    ham = hamf()
    p0 = I.rbm_params(N, M, seed)
    s0 = oracle.chain_init(N, C, rule, seed, 0)
    h, _e = ham_to_device(ham)
    pd, sd = cu(p0), cu(s0)
    ch = nk.make_chains(sd)
    cfg = nk.make_cfg(rule, prec, solver, nd, ns, eps, lr, seed, cg_tol=1e-10, cg_maxiter=2000)
    stats = torch.empty(nk.SR_STATS_DOUBLES, dtype=torch.float64, device=dev())
    samples = torch.empty((C * ns, N), dtype=torch.int8, device=dev())
    eloc = torch.empty(C * ns, dtype=torch.float64, device=dev())
    out = []
    for it in range(steps):
        cfg.n_discard = nd if it == 0 else 0
        nk.nk_sr_step(ctx, pd, N, M, h, ch, cfg, stats, samples, eloc)
        out.append({"stats": nk.sr_stats_dict(stats), "samples": samples.cpu().numpy().copy(),
                    "eloc": eloc.cpu().numpy().copy(), "params": pd.cpu().numpy().copy(),
                    "state": sd.cpu().numpy().copy()})
    return p0, s0, ham, out


def test_sr_step_matches_oracle_config1(ctx):
    """Tutorial-size workload: periodic TFIM chain N = 16, alpha = 1, 16 chains x
    64 samples, 16 discarded sweeps, eps = lr = 0.01, dense Cholesky; the GPU
    step equals the oracle step on the same Philox streams."""
    N = M = 16
    p0, s0, ham, out = _sr_run(ctx, N, M, lambda: I.tfim_chain(16), "local", 16, 16, 64, 1, "cholesky",
                               0.01, 0.01, 3)
    p, s, sweep0 = p0, s0, 0
    for it, g in enumerate(out):
        nd = 16 if it == 0 else 0
        ref = oracle.sr_step(p, N, M, ham, "local", s, sweep0, nd, 64, 1, 0, diag_shift=0.01, lr=0.01,
                             solver="cholesky")
        sweep0 += nd + 64
        np.testing.assert_array_equal(g["samples"], ref["samples"].reshape(-1, N))
        assert rel_err(g["eloc"], ref["eloc"]) < 1e-10
        assert abs(g["stats"]["energy"] - ref["stats"]["mean"]) < 1e-10 * abs(ref["stats"]["mean"])
        assert abs(g["stats"]["error"] - ref["stats"]["error"]) < 1e-8 * ref["stats"]["error"]
        assert vec_rel_err(g["params"] - p, ref["params"] - p) < 1e-8
        p, s = ref["params"], ref["state"]
        np.testing.assert_array_equal(g["state"], s)
        # continue from the oracle's parameters so each step is compared alone
        p = g["params"]


@pytest.mark.parametrize("solver", ["cg", "cholesky_samplespace"])
def test_sr_step_heisenberg_small(ctx, solver):
    N, M = 16, 32
    p0, s0, ham, out = _sr_run(ctx, N, M, lambda: I.heis_square(4), "exchange", 32, 4, 8, 2, solver,
                               0.01, 0.02, 2)
    p, s, sweep0 = p0, s0, 0
    for it, g in enumerate(out):
        nd = 4 if it == 0 else 0
        ref = oracle.sr_step(p, N, M, ham, "exchange", s, sweep0, nd, 8, 2, 0, diag_shift=0.01, lr=0.02,
                             solver="cg" if solver == "cg" else "cholesky", cg_tol=1e-10)
        sweep0 += nd + 8
        np.testing.assert_array_equal(g["samples"], ref["samples"].reshape(-1, N))
        assert rel_err(g["eloc"], ref["eloc"]) < 1e-10
        assert vec_rel_err(g["params"] - p, ref["params"] - p) < 1e-7
        p, s = g["params"], ref["state"]


def test_invalid_arguments_are_rejected(ctx):
    p = cu(I.rbm_params(4, 4, 1))
    out = torch.empty(3, dtype=torch.float64, device=dev())
    host_s = torch.ones((3, 4), dtype=torch.int8)  # host memory
    with pytest.raises(nk.NkError) as ei:
        r = nk.make_rbm(p, 4, 4)
        code = nk.lib().nk_rbm_logpsi(ctx.handle, nk.ctypes.byref(r), 0, nk.ctypes.c_void_p(host_s.data_ptr()),
                                      3, nk.ctypes.c_void_p(out.data_ptr()), None)
        nk._check(code)
    assert ei.value.code == nk.NK_ERR_INVALID_ARG
    with pytest.raises(nk.NkError):
        nk.nk_chains_init(ctx, 5, 3, "exchange", 1, 0, torch.empty((3, 5), dtype=torch.int8, device=dev()))


def test_sr_trajectory_config1_50_iterations(ctx):
    """Tutorial workload, 50 VMC + SR iterations on the FP64 path (periodic TFIM
    chain N = 16, J = h = 1, alpha = 1, 16 chains x 64 samples, 16 discarded
    sweeps, eps = lr = 0.01, dense Cholesky): the energy trajectory equals the
    oracle's on the same Philox streams to 1e-8 relative, and every energy
    respects the variational bound E >= E0 - 4 sigma with E0 = -2/sin(pi/32)."""
    from oracle import exact
    N = M = 16
    steps = 50
    p0, s0, ham, out = _sr_run(ctx, N, M, lambda: I.tfim_chain(16), "local", 16, 16, 64, 1, "cholesky",
                               0.01, 0.01, steps)
    e0 = exact.tfim_free_fermion_e0(16)
    p, s, sweep0 = p0, s0, 0
    for it in range(steps):
        nd = 16 if it == 0 else 0
        ref = oracle.sr_step(p, N, M, ham, "local", s, sweep0, nd, 64, 1, 0, diag_shift=0.01, lr=0.01,
                             solver="cholesky")
        sweep0 += nd + 64
        g = out[it]["stats"]
        assert abs(g["energy"] - ref["stats"]["mean"]) <= 1e-8 * abs(ref["stats"]["mean"])
        assert g["energy"] >= e0 - 4 * g["error"]
        p, s = ref["params"], ref["state"]
        np.testing.assert_array_equal(out[it]["state"], s)
    # the optimisation moves down towards E0
    first = np.mean([o["stats"]["energy"] for o in out[:5]])
    last = np.mean([o["stats"]["energy"] for o in out[-5:]])
    assert last < first


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_metropolis_full_size_sampled_chains(ctx, prec):
    """The sweep configuration of the 10 x 10 Heisenberg workload (1024
    exchange chains, 16 discarded + 8 sampled sweeps, N = 100, M = 200,
    sigma = 0.01) run in full on the GPU; the first 48 chains are replayed by
    the oracle (chains are independent: the Philox counter holds the chain
    index)."""
    N, M, C, nd, ns = 100, 200, 1024, 16, 8
    p = I.rbm_params(N, M, 2)
    edges = I.square_edges(10)
    s0 = oracle.chain_init(N, C, "exchange", 2, 0)
    st = cu(s0)
    samples = torch.empty((C, ns, N), dtype=torch.int8, device=dev())
    lp = torch.empty((C, ns), dtype=torch.float64, device=dev())
    nacc = torch.zeros(C, dtype=torch.int64, device=dev())
    dec = torch.empty((C, nd + ns, N), dtype=torch.uint8, device=dev())
    nk.nk_metropolis_sweep(ctx, cu(p), N, M, "exchange", cu(edges), st, 0, nd, ns, 2, 0, samples, lp, nacc,
                           dec, precision=prec)
    K = 48
    g_dec = dec.cpu().numpy()[:K]
    ref = oracle.metropolis(p, N, M, "exchange", edges, s0[:K], 0, nd, ns, 2, 0, forced=g_dec)
    mism = ref["decisions"] != g_dec
    if prec == "f64":
        allowed = ref["margin"] < 1e-9
    else:
        lu = _lnu(2, 0, K, N, nd + ns, 0)
        two_d = lu + np.where(ref["decisions"] == 1, 1, -1) * ref["margin"]
        allowed = ref["margin"] < 1e-4 * np.maximum(1.0, np.abs(two_d))
    assert not (mism & ~allowed).any()
    np.testing.assert_array_equal(samples.cpu().numpy()[:K], ref["samples"])
    np.testing.assert_array_equal(st.cpu().numpy()[:K], ref["state"])
    assert rel_err(lp.cpu().numpy()[:K], ref["logpsi"]) < (1e-10 if prec == "f64" else 1e-4)
    # every chain keeps S_z = 0 and the accept counts match the decisions
    assert (st.cpu().numpy().astype(np.int64).sum(axis=1) == 0).all()
    np.testing.assert_array_equal(nacc.cpu().numpy(), (dec.cpu().numpy() == 1).sum(axis=(1, 2)))


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_metropolis_full_size_local_rule_sampled_chains(ctx, prec):
    """The sweep configuration of the 20 x 20 TFIM workload (16384 local-rule
    chains, N = 400, M = 1600, sigma = 0.01; one discarded and one sampled
    sweep) run in full on the GPU; the first 8 chains are replayed by the
    oracle with forced-follow."""
    N, M, C, nd, ns = 400, 1600, 16384, 1, 1
    p = I.rbm_params(N, M, 3)
    s0 = oracle.chain_init(N, C, "local", 3, 0)
    st = cu(s0)
    samples = torch.empty((C, ns, N), dtype=torch.int8, device=dev())
    lp = torch.empty((C, ns), dtype=torch.float64, device=dev())
    nacc = torch.zeros(C, dtype=torch.int64, device=dev())
    dec = torch.empty((C, nd + ns, N), dtype=torch.uint8, device=dev())
    nk.nk_metropolis_sweep(ctx, cu(p), N, M, "local", None, st, 0, nd, ns, 3, 0, samples, lp, nacc,
                           dec, precision=prec)
    K = 8
    g_dec = dec.cpu().numpy()[:K]
    ref = oracle.metropolis(p, N, M, "local", None, s0[:K], 0, nd, ns, 3, 0, forced=g_dec)
    mism = ref["decisions"] != g_dec
    if prec == "f64":
        allowed = ref["margin"] < 1e-9
    else:
        lu = _lnu(3, 0, K, N, nd + ns, 0)
        two_d = lu + np.where(ref["decisions"] == 1, 1, -1) * ref["margin"]
        allowed = ref["margin"] < 1e-4 * np.maximum(1.0, np.abs(two_d))
    assert not (mism & ~allowed).any()
    np.testing.assert_array_equal(samples.cpu().numpy()[:K], ref["samples"])
    np.testing.assert_array_equal(st.cpu().numpy()[:K], ref["state"])
    assert rel_err(lp.cpu().numpy()[:K], ref["logpsi"]) < (1e-10 if prec == "f64" else 1e-4)
    np.testing.assert_array_equal(nacc.cpu().numpy(), (dec.cpu().numpy() == 1).sum(axis=(1, 2)))


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_metropolis_full_size_24x24_sampled_chains(ctx, prec):
    """The sweep configuration of the 24 x 24 Heisenberg workload (8192
    exchange chains at S_z = 0, N = 576, M = 4608, sigma = 0.01; one
    discarded and one sampled sweep) run in full on the GPU; the first 4
    chains are replayed by the oracle with forced-follow."""
    N, M, C, nd, ns = 576, 4608, 8192, 1, 1
    p = I.rbm_params(N, M, 5)
    edges = I.square_edges(24)
    s0 = oracle.chain_init(N, C, "exchange", 5, 0)
    st = cu(s0)
    samples = torch.empty((C, ns, N), dtype=torch.int8, device=dev())
    lp = torch.empty((C, ns), dtype=torch.float64, device=dev())
    nacc = torch.zeros(C, dtype=torch.int64, device=dev())
    dec = torch.empty((C, nd + ns, N), dtype=torch.uint8, device=dev())
    nk.nk_metropolis_sweep(ctx, cu(p), N, M, "exchange", cu(edges), st, 0, nd, ns, 5, 0, samples, lp, nacc,
                           dec, precision=prec)
    K = 4
    g_dec = dec.cpu().numpy()[:K]
    ref = oracle.metropolis(p, N, M, "exchange", edges, s0[:K], 0, nd, ns, 5, 0, forced=g_dec)
    mism = ref["decisions"] != g_dec
    if prec == "f64":
        allowed = ref["margin"] < 1e-9
    else:
        lu = _lnu(5, 0, K, N, nd + ns, 0)
        two_d = lu + np.where(ref["decisions"] == 1, 1, -1) * ref["margin"]
        allowed = ref["margin"] < 1e-4 * np.maximum(1.0, np.abs(two_d))
    assert not (mism & ~allowed).any()
    np.testing.assert_array_equal(samples.cpu().numpy()[:K], ref["samples"])
    np.testing.assert_array_equal(st.cpu().numpy()[:K], ref["state"])
    assert rel_err(lp.cpu().numpy()[:K], ref["logpsi"]) < (1e-10 if prec == "f64" else 1e-4)
    assert (st.cpu().numpy().astype(np.int64).sum(axis=1) == 0).all()
    np.testing.assert_array_equal(nacc.cpu().numpy(), (dec.cpu().numpy() == 1).sum(axis=(1, 2)))


def test_sr_step_sampling_gives_the_samples_of_nk_metropolis_sweep(ctx):
    """NK_MIXED sampling inside nk_sr_step writes each sweep's theta product
    into the rows of the samples it belongs to and hands those to the local
    energies.  On the 24 x 24 sizes (2000 chains, one discarded and two
    sampled sweeps) it must give, bit for bit, the samples and chain states
    of nk_metropolis_sweep from the same start (the same Philox streams, the
    same exact theta products), and local energies equal to nk_local_energy
    on those samples."""
    N, M, C, nd, ns, seed = 576, 4608, 2000, 1, 2, 5
    ham = I.heis_square(24)
    p = cu(I.rbm_params(N, M, seed))
    s0 = oracle.chain_init(N, C, "exchange", seed, 0)
    h, edges = ham_to_device(ham)
    # the step
    sd = cu(s0)
    ch = nk.make_chains(sd)
    cfg = nk.make_cfg("exchange", "mixed", "cholesky_samplespace", nd, ns, 0.01, 0.0, seed)
    stats = torch.empty(nk.SR_STATS_DOUBLES, dtype=torch.float64, device=dev())
    samples = torch.empty((C * ns, N), dtype=torch.int8, device=dev())
    eloc = torch.empty(C * ns, dtype=torch.float64, device=dev())
    nk.nk_sr_step(ctx, p, N, M, h, ch, cfg, stats, samples, eloc)
    # the same sweeps as one launch sequence over all chains
    st2 = cu(s0)
    samples2 = torch.empty((C, ns, N), dtype=torch.int8, device=dev())
    nk.nk_metropolis_sweep(ctx, p, N, M, "exchange", edges, st2, 0, nd, ns, seed, 0, samples2, precision="mixed")
    torch.cuda.synchronize()
    np.testing.assert_array_equal(samples.cpu().numpy(), samples2.cpu().numpy().reshape(C * ns, N))
    np.testing.assert_array_equal(sd.cpu().numpy(), st2.cpu().numpy())
    e2 = torch.empty(C * ns, dtype=torch.float64, device=dev())
    nk.nk_local_energy(ctx, p, N, M, h, samples2.reshape(C * ns, N), e2, precision="mixed")
    assert rel_err(eloc.cpu().numpy(), e2.cpu().numpy()) <= 1e-12
