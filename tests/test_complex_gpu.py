"""GPU parity of the complex holomorphic RBM and of time-dependent VMC (Sec.
3.2 with complex parameters; Sec. 4.3, Eq. eq:tvmc; the Runge-Kutta steps of
Eq. eq:rk-step) against the complex oracle in oracle/holo.py, through the C
ABI.

Tolerances: ln psi, log-derivatives 1e-12 and local energies 1e-10 relative
(FP64 throughout); chains bit-exact (the same Philox streams and decisions;
both sides decide in FP64 on 2 Re dlnpsi); the slope theta_dot and the
parameters after a step 1e-8 relative in norm, on spectra with no
eigenvalue near the cutoff.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import holo
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


def cparams(N, M, seed, sigma):
    rng = np.random.default_rng(seed)
    n = N + M + M * N
    return rng.normal(0.0, sigma, n) + 1j * rng.normal(0.0, sigma, n)


def ccu(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).to(dev())


@pytest.mark.parametrize("N,M,B,sig", [(12, 12, 100, 0.3), (37, 45, 33, 0.2), (1, 1, 4, 0.5), (64, 64, 16, 0.1)])
def test_logpsi_and_jacobian(ctx, N, M, B, sig):
    p = cparams(N, M, N + M, sig)
    s = I.random_configs(B, N, 3)
    out = torch.empty(B, dtype=torch.complex128, device=dev())
    nk.nk_crbm_logpsi(ctx, ccu(p), N, M, cu(s), out)
    ref_lp = holo.logpsi(p, N, M, s)
    assert np.abs(out.cpu().numpy() - ref_lp).max() < 1e-12 * max(1.0, np.abs(ref_lp).max())
    O = torch.empty((B, N + M + M * N), dtype=torch.complex128, device=dev())
    nk.nk_crbm_jacobian(ctx, ccu(p), N, M, cu(s), O)
    ref = holo.jacobian(p, N, M, s)
    assert np.abs(O.cpu().numpy() - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())


LE_CASES = [
    ("tfim-chain10", 10, 10, lambda: I.tfim_chain(10, 1.0, 0.7), False),
    ("heis-square4", 16, 16, lambda: I.heis_square(4), True),
    ("j1j2-chain12", 12, 24, lambda: I.j1j2_chain(12, 1.0, 0.4), True),
]


@pytest.mark.parametrize("name,N,M,hf,sz0", LE_CASES, ids=[c[0] for c in LE_CASES])
def test_local_energy(ctx, name, N, M, hf, sz0):
    ham = hf()
    p = cparams(N, M, 4, 0.25)
    s = I.random_configs(40, N, 5, sz0=sz0)
    h, _e = ham_to_device(ham)
    out = torch.empty(40, dtype=torch.complex128, device=dev())
    nk.nk_crbm_local_energy(ctx, ccu(p), N, M, h, cu(s), out)
    ref = holo.local_energy(p, N, M, ham, s)
    got = out.cpu().numpy()
    scale = np.sqrt(np.mean(np.abs(ref) ** 2))
    assert np.abs(got - ref).max() < 1e-10 * scale


@pytest.mark.parametrize("rule,N,M,C,ham", [("local", 8, 8, 6, None), ("exchange", 12, 6, 5, "ring12")])
def test_metropolis_bit_exact(ctx, rule, N, M, C, ham):
    p = cparams(N, M, 6, 0.3)
    edges = I.chain_edges(N) if ham else None
    s0 = I.random_configs(C, N, 8, sz0=(rule == "exchange"))
    sd = cu(s0)
    samples = torch.empty((C, 3, N), dtype=torch.int8, device=dev())
    nk.nk_crbm_metropolis(ctx, ccu(p), N, M, rule, None if edges is None else cu(edges.astype(np.int32)), sd, 5, 2, 3,
                          17, 2, samples)
    st, ref = holo.metropolis(p, N, M, rule, edges, s0, 5, 2, 3, 17, 2)
    np.testing.assert_array_equal(samples.cpu().numpy(), ref)
    np.testing.assert_array_equal(sd.cpu().numpy(), st)


TDVP_CASES = [
    # name, N, M, hamiltonian, rule, chains, samples, real time, solver, eps, rcond, integrator
    ("real-time-svd-heun", 6, 6, lambda: I.tfim_chain(6, 1.0, 1.0), "local", 64, 8, True, "svd", 0.0, 1e-10, "heun"),
    ("imag-time-cholesky-euler", 6, 6, lambda: I.tfim_chain(6, 1.0, 0.5), "local", 64, 8, False, "cholesky", 0.01,
     0.0, "euler"),
    ("real-time-svd-exchange-euler", 8, 4, lambda: I.heis_chain(8), "exchange", 32, 8, True, "svd", 0.0, 1e-10,
     "euler"),
]


@pytest.mark.parametrize("case", TDVP_CASES, ids=[c[0] for c in TDVP_CASES])
def test_tdvp_step_matches_oracle(ctx, case):
    """One t-VMC step on the GPU against the oracle's, on the same chains and
    Philox streams: the first slope theta_dot of Eq. eq:tvmc, the chains after
    the step (bit-exact) and the new parameters."""
    name, N, M, hf, rule, C, ns, real_time, solver, eps, rcond, integ = case
    ham = hf()
    edges = np.asarray(ham["edges"]).reshape(-1, 2)
    p0 = cparams(N, M, 9, 0.2)
    s0 = I.random_configs(C, N, 10, sz0=(rule == "exchange"))
    h, _e = ham_to_device(ham)
    pd, sd = ccu(p0), cu(s0)
    ch = nk.make_chains(sd, sweeps_done=3)
    dt = 0.01
    cfg = nk.make_tdvp_cfg(rule, integ, real_time, solver, 0, ns, dt, eps, 21, 1, rcond=rcond)
    stats = torch.empty(4, dtype=torch.float64, device=dev())
    tdot = torch.empty(N + M + M * N, dtype=torch.complex128, device=dev())
    nk.nk_tdvp_step(ctx, pd, N, M, h, ch, cfg, stats, tdot)
    gamma = -1j if real_time else -1.0
    rc = rcond if solver == "svd" else None
    k1, chains1, e1 = holo.tvmc_rhs(p0, N, M, ham, rule, edges, s0, 3, 0, ns, 21, 1, gamma, eps, rc)
    assert vec_rel_err(tdot.cpu().numpy(), k1) < 1e-8
    st = stats.cpu().numpy()
    assert abs(complex(st[0], st[1]) - e1) < 1e-10 * max(1.0, abs(e1))
    if integ == "euler":
        ref_p, ref_chains = p0 + dt * k1, chains1
        assert ch.sweeps_done == 3 + ns
    else:
        ref_p, ref_chains, sweep = holo.tvmc_heun(p0, N, M, ham, rule, edges, s0, 3, ns, 21, dt, 1, gamma, eps, rc)
        assert ch.sweeps_done == sweep
    np.testing.assert_array_equal(sd.cpu().numpy(), ref_chains)
    got = pd.cpu().numpy()
    assert vec_rel_err(got - p0, ref_p - p0) < 1e-8


def test_misaligned_and_invalid_arguments_are_refused(ctx):
    N = M = 4
    p = ccu(cparams(N, M, 1, 0.1))
    s = cu(I.random_configs(3, N, 1))
    buf = torch.empty(2 * 3 + 1, dtype=torch.float64, device=dev())
    r = nk.make_crbm(p, N, M)
    code = nk.lib().nk_crbm_logpsi(ctx.handle, ctypes.byref(r), ctypes.c_void_p(s.data_ptr()), 3,
                                   ctypes.c_void_p(buf.data_ptr() + 8), None)
    assert code == nk.NK_ERR_INVALID_ARG
    h, _e = ham_to_device(I.tfim_chain(4))
    sd = cu(I.random_configs(2, N, 2))
    cfg = nk.make_tdvp_cfg("local", "euler", True, "cholesky", 0, 2, 0.01, 0.0, 1)  # Cholesky needs eps > 0
    with pytest.raises(nk.NkError) as ei:
        nk.nk_tdvp_step(ctx, p, N, M, h, nk.make_chains(sd), cfg)
    assert ei.value.code == nk.NK_ERR_INVALID_ARG
