"""Pins of the symmetric-RBM oracle (RBMSymm, Sec. 5) against facts that do
not come from its own formulas: the plain-RBM oracle in C evaluated on the
tied parameters, invariance under every group element (brute force),
central differences, the chain rule through the tied parameters, the
variational bound against the exact ground energy, and descent of the exact
energy under one SR step.  No GPU is used."""
import numpy as np
import pytest

import oracle
from oracle import exact
from oracle import symm
from paper_2112_10526_gb300 import inputs as I

CASES = [
    ("chain8-a2", 8, 2, lambda: I.translations_chain(8)),
    ("chain11-a3", 11, 3, lambda: I.translations_chain(11)),
    ("square4-a1", 16, 1, lambda: I.translations_square(4)),
]


def _params(N, alpha, seed, sigma):
    return np.random.default_rng(seed).normal(0.0, sigma, symm.n_params(N, alpha))


def test_translations_are_groups():
    for perms in (I.translations_chain(7), I.translations_square(3)):
        rows = {tuple(r) for r in perms}
        assert len(rows) == perms.shape[0]
        for g in perms:
            assert sorted(g) == list(range(perms.shape[1]))
            for h in perms:
                assert tuple(g[h]) in rows  # closed under composition


@pytest.mark.parametrize("name,N,alpha,pf", CASES, ids=[c[0] for c in CASES])
def test_logpsi_equals_the_plain_rbm_on_tied_parameters(name, N, alpha, pf):
    perms = pf()
    p = _params(N, alpha, 3, 0.4)
    s = I.random_configs(200, N, 4)
    got = symm.logpsi(p, N, alpha, perms, s)
    ref = oracle.logpsi(symm.expand(p, N, alpha, perms), N, alpha * perms.shape[0], s)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("name,N,alpha,pf", CASES, ids=[c[0] for c in CASES])
def test_logpsi_is_invariant_under_the_group(name, N, alpha, pf):
    perms = pf()
    p = _params(N, alpha, 5, 0.5)
    s = I.random_configs(20, N, 6)
    ref = symm.logpsi(p, N, alpha, perms, s)
    for g in perms:
        np.testing.assert_allclose(symm.logpsi(p, N, alpha, perms, s[:, g]), ref, rtol=1e-13, atol=1e-13)
    # a plain RBM with the same number of parameters is not invariant
    pr = I.rbm_params(N, alpha, 5, 0.5)
    lp = oracle.logpsi(pr, N, alpha, s)
    assert np.max(np.abs(oracle.logpsi(pr, N, alpha, s[:, perms[1]]) - lp)) > 1e-3


@pytest.mark.parametrize("name,N,alpha,pf", CASES[:2], ids=[c[0] for c in CASES[:2]])
def test_jacobian_central_differences(name, N, alpha, pf):
    perms = pf()
    p = _params(N, alpha, 7, 0.3)
    s = I.random_configs(5, N, 8)
    O = symm.jacobian(p, N, alpha, perms, s)
    h = 1e-6
    for k in range(p.size):
        e = np.zeros_like(p)
        e[k] = h
        fd = (symm.logpsi(p + e, N, alpha, perms, s) - symm.logpsi(p - e, N, alpha, perms, s)) / (2 * h)
        assert np.max(np.abs(fd - O[:, k])) < 1e-6 * max(1.0, np.max(np.abs(O[:, k])))


@pytest.mark.parametrize("name,N,alpha,pf", CASES, ids=[c[0] for c in CASES])
def test_jacobian_is_the_chain_rule_through_the_tied_parameters(name, N, alpha, pf):
    """d ln psi / d theta_symm = (d ln psi / d theta_rbm) T with T the linear
    tying map, using the C oracle's plain-RBM log-derivatives."""
    perms = pf()
    p = _params(N, alpha, 9, 0.3)
    s = I.random_configs(30, N, 10)
    M = alpha * perms.shape[0]
    Np = symm.n_params(N, alpha)
    T = np.stack([symm.expand(np.eye(Np)[k], N, alpha, perms) for k in range(Np)], axis=1)
    O_rbm = oracle.jacobian(symm.expand(p, N, alpha, perms), N, M, s)
    np.testing.assert_allclose(symm.jacobian(p, N, alpha, perms, s), O_rbm @ T, rtol=1e-12, atol=1e-12)


def test_variational_bound_and_local_energy_identity_tfim_chain():
    """Periodic TFIM chain N = 10 (J = h = 1): the exact energy of a symmetric
    RBM is the |psi|^2 average of its local energies and lies above the
    free-fermion ground energy; the ground state is translation invariant,
    so a trained symmetric RBM can approach it."""
    N, alpha = 10, 2
    perms = I.translations_chain(N)
    ham = I.tfim_chain(N, 1.0, 1.0)
    p = _params(N, alpha, 11, 0.3)
    pe = symm.expand(p, N, alpha, perms)
    es = exact.ExactState(pe, N, alpha * N)
    el = symm.local_energy(p, N, alpha, perms, ham, es.configs)
    e_exact = es.energy(ham)
    assert abs(np.sum(es.p * el) - e_exact) < 1e-12 * abs(e_exact)
    assert e_exact > exact.tfim_free_fermion_e0(N) - 1e-12


def test_sr_step_lowers_the_exact_energy():
    """One SR step (Sec. 4.1) in the symmetric parameters, 64 chains x 64
    samples, lowers the exact energy of the 4 x 4 Marshall-signed Heisenberg
    model at S_z = 0."""
    N, alpha = 16, 2
    perms = I.translations_square(4)
    ham = I.heis_square(4, 1.0, True)
    p = _params(N, alpha, 12, 0.1)
    M = alpha * perms.shape[0]

    def energy(q):
        return exact.ExactState(symm.expand(q, N, alpha, perms), N, M, sz0=True).energy(ham)

    s0 = oracle.chain_init(N, 64, "exchange", 13)
    r = symm.sr_step(p, N, alpha, perms, ham, "exchange", s0, 0, 8, 64, 13, diag_shift=0.01, lr=0.02)
    assert r["params"].shape == p.shape
    assert energy(r["params"]) < energy(p) - 0.1
