"""Pins of the complex holomorphic RBM and TDVP oracle (Secs. 3.2-3.5, 4.3)
against facts outside its own formulas: the RBM's hidden units summed out by
brute force, the real-parameter C oracle, the Pauli Kronecker Hamiltonian,
finite differences of the exact energy and of the normalised state (the
holomorphic gradient and the Fubini-Study metric), the Euler step as SR, and
closed-form dynamics of a product state that the ansatz follows exactly.
No GPU is used."""
import numpy as np
import pytest

import oracle
from oracle import exact
from oracle import holo as H
from paper_2112_10526_gb300 import inputs as I


def _params(N, M, seed, sigma):
    rng = np.random.default_rng(seed)
    n = H.n_params(N, M)
    return rng.normal(0.0, sigma, n) + 1j * rng.normal(0.0, sigma, n)


def test_logpsi_is_the_hidden_unit_marginal():
    N, M = 6, 4
    p = _params(N, M, 1, 0.4)
    s = I.random_configs(20, N, 2)
    np.testing.assert_allclose(np.exp(H.logpsi(p, N, M, s)), H.brute_force_marginal(p, N, M, s), rtol=1e-12)


def test_real_parameters_agree_with_the_c_oracle():
    N, M = 10, 7
    pr = I.rbm_params(N, M, 3, 0.3)
    s = I.random_configs(40, N, 4)
    ham = I.tfim_chain(N, 0.8, 1.1)
    np.testing.assert_allclose(H.logpsi(pr, N, M, s).real, oracle.logpsi(pr, N, M, s), rtol=1e-13)
    assert np.abs(H.logpsi(pr, N, M, s).imag).max() < 1e-14
    np.testing.assert_allclose(H.local_energy(pr, N, M, ham, s).real, oracle.local_energy(pr, N, M, ham, s),
                               rtol=1e-12)
    np.testing.assert_allclose(H.jacobian(pr, N, M, s).real, oracle.jacobian(pr, N, M, s), rtol=1e-13,
                               atol=1e-15)


@pytest.mark.parametrize("hf,N,sz0", [(lambda: I.tfim_chain(8, 1.0, 0.6), 8, False),
                                      (lambda: I.heis_chain(8, 1.0, False), 8, True),
                                      (lambda: I.j1j2_chain(8, 1.0, 0.5, False), 8, True)])
def test_local_energy_equals_hamiltonian_action(hf, N, sz0):
    """Complex psi: E_loc(s) = (H psi)(s) / psi(s) with H from Kronecker
    products.  Without the Marshall rotation the Heisenberg signs are carried
    by the complex parameters."""
    ham = hf()
    M = 6
    p = _params(N, M, 5, 0.3)
    v = H.exact_state(p, N, M)
    hv = exact.hamiltonian(N, ham) @ v
    s = exact.basis(N)
    if sz0:
        keep = s.astype(np.int64).sum(axis=1) == 0
        s, v, hv = s[keep], v[keep], hv[keep]
    el = H.local_energy(p, N, M, ham, s)
    np.testing.assert_allclose(el, hv / v, rtol=1e-10, atol=1e-10)


def test_holomorphic_derivatives_central_differences():
    """d ln psi / d theta along the real and the imaginary axis agree with
    O_k (Cauchy-Riemann: the map is holomorphic)."""
    N, M = 5, 3
    p = _params(N, M, 7, 0.4)
    s = I.random_configs(6, N, 8)
    O = H.jacobian(p, N, M, s)
    h = 1e-6
    for k in range(p.size):
        e = np.zeros(p.size, dtype=np.complex128)
        e[k] = h
        dr = (H.logpsi(p + e, N, M, s) - H.logpsi(p - e, N, M, s)) / (2 * h)
        di = (H.logpsi(p + 1j * e, N, M, s) - H.logpsi(p - 1j * e, N, M, s)) / (2j * h)
        np.testing.assert_allclose(dr, O[:, k], rtol=1e-6, atol=1e-8)
        np.testing.assert_allclose(di, O[:, k], rtol=1e-6, atol=1e-8)


def test_force_is_the_wirtinger_gradient_of_the_exact_energy():
    """d<H>/d theta_k^* = f~_k (Eq. eq:VMC gradient:holo), with d/d theta^* =
    (d/dx + i d/dy) / 2 taken by central differences of the exact energy."""
    N, M = 6, 4
    ham = I.tfim_chain(N, 1.0, 0.7)
    p = _params(N, M, 9, 0.3)
    f, _G, _e = H.exact_moments(p, N, M, ham)

    def energy(q):
        v = H.exact_state(q, N, M)
        return float(np.real(v.conj() @ (exact.hamiltonian(N, ham) @ v)))

    h = 1e-6
    for k in range(p.size):
        e = np.zeros(p.size, dtype=np.complex128)
        e[k] = h
        dx = (energy(p + e) - energy(p - e)) / (2 * h)
        dy = (energy(p + 1j * e) - energy(p - 1j * e)) / (2 * h)
        assert abs(0.5 * (dx + 1j * dy) - f[k]) < 1e-6 * max(1.0, abs(f[k]))


def test_qgt_is_the_fubini_study_metric():
    """G_kl = <d_k phi|d_l phi> - <d_k phi|phi><phi|d_l phi> for the normalised
    state with the component orthogonal to phi, from finite differences of
    the unnormalised state vector psi(theta) (d_k psi = O_k psi)."""
    N, M = 6, 3
    p = _params(N, M, 11, 0.3)
    _f, G, _e = H.exact_moments(p, N, M, I.tfim_chain(N))
    s = exact.basis(N)

    def psi(q):
        return np.exp(H.logpsi(q, N, M, s))

    v = psi(p)
    nrm = np.linalg.norm(v)
    h = 1e-6
    D = np.empty((v.size, p.size), dtype=np.complex128)
    for k in range(p.size):
        e = np.zeros(p.size, dtype=np.complex128)
        e[k] = h
        D[:, k] = (psi(p + e) - psi(p - e)) / (2 * h) / nrm
    phi = v / nrm
    ref = D.conj().T @ D - np.outer(D.conj().T @ phi, phi.conj() @ D)
    np.testing.assert_allclose(G, ref, rtol=1e-6, atol=1e-8)


def test_imaginary_time_euler_step_is_sr():
    """gamma = -1 with the Euler scheme is SR with learning rate dt (Sec. 4.3),
    and Heun steps in imaginary time lower the energy."""
    N, M = 6, 4
    ham = I.tfim_chain(N, 1.0, 1.0)
    p = _params(N, M, 13, 0.2)
    f, G, E0 = H.exact_moments(p, N, M, ham)
    dt, eps = 0.01, 1e-3
    step = H.euler(p, lambda q: _rhs(q, N, M, ham, -1.0, eps), dt)
    delta = np.linalg.solve(G + eps * np.eye(p.size), f)
    np.testing.assert_allclose(step, p - dt * delta, rtol=1e-10, atol=1e-12)
    q = p
    for _ in range(5):
        q = H.heun(q, lambda r: _rhs(r, N, M, ham, -1.0, eps), 0.05)
    assert H.exact_moments(q, N, M, ham)[2].real < E0.real - 1e-3


def _rhs(q, N, M, ham, gamma, eps, rcond=None):
    f, G, _e = H.exact_moments(q, N, M, ham)
    return H.theta_dot(G, f, gamma, eps, rcond)


def _product_state_exact(a0, h, t):
    """One spin under H = -h sigma^x from psi(+-1) = exp(+-a0): the amplitude
    ratio psi(-1)/psi(+1) = exp(-2 a(t)) of exp(i h t sigma^x) psi."""
    up, dn = np.exp(a0), np.exp(-a0)
    c, s = np.cos(h * t), 1j * np.sin(h * t)
    up_t, dn_t = c * up + s * dn, s * up + c * dn
    return -0.5 * np.log(dn_t / up_t)


def test_real_time_heun_follows_the_exact_product_state_dynamics():
    """With J = 0 the Ising Hamiltonian H = -h sum sigma^x moves every spin
    alone, and the product states psi(s) = exp(a.s) (W = 0, b = 0) contain the
    exact trajectory: a_i(t) has the closed form above.  Real-time TDVP (gamma
    = -i, pseudo-inverse of G) with Heun steps follows it with a second-order
    error: halving dt cuts the error about four times."""
    N, M, h, T = 4, 1, 0.9, 0.4
    ham = I.tfim_chain(N, 0.0, h)
    a0 = np.array([0.3 + 0.1j, -0.2 + 0.05j, 0.1 - 0.2j, 0.25 + 0.0j])
    p = np.concatenate([a0, np.zeros(M + M * N, dtype=np.complex128)])
    ref = _product_state_exact(a0, h, T)
    # the exact slope at t = 0
    slope = (_product_state_exact(a0, h, 1e-6) - _product_state_exact(a0, h, -1e-6)) / 2e-6
    np.testing.assert_allclose(_rhs(p, N, M, ham, -1j, 0.0, rcond=1e-10)[:N], slope, rtol=1e-7, atol=1e-9)
    err = []
    for dt in (0.02, 0.01):
        q = p
        for _ in range(int(round(T / dt))):
            q = H.heun(q, lambda r: _rhs(r, N, M, ham, -1j, 0.0, rcond=1e-10), dt)
        assert np.max(np.abs(q[N:])) < 1e-10  # the hidden part stays zero
        # a is fixed modulo i pi / 2 by psi; compare through the amplitude ratios
        err.append(np.max(np.abs(np.exp(-2 * q[:N]) - np.exp(-2 * ref))))
    assert 3.5 < err[0] / err[1] < 4.5, err
    assert err[1] < 5e-5, err


def test_real_time_energy_is_conserved_to_second_order():
    """Unitary TDVP conserves <H> in continuous time (Sec. 9.1); with Heun
    steps the drift over a fixed time falls about fourfold when dt halves."""
    N, M = 6, 3
    ham = I.tfim_chain(N, 1.0, 1.0)
    p = _params(N, M, 17, 0.2)
    E0 = H.exact_moments(p, N, M, ham)[2].real
    drift = []
    for dt in (0.02, 0.01):
        q = p
        for _ in range(int(round(0.4 / dt))):
            q = H.heun(q, lambda r: _rhs(r, N, M, ham, -1j, 0.0, rcond=1e-12), dt)
        drift.append(abs(H.exact_moments(q, N, M, ham)[2].real - E0))
    assert drift[0] / drift[1] > 3.5, drift
    assert drift[1] < 2e-3, drift


@pytest.mark.parametrize("rule", ["local", "exchange"])
def test_complex_sampler_equals_the_c_oracle_on_real_parameters(rule):
    """On real parameters the complex sampler draws the same Philox streams
    and takes the same decisions as the real-RBM C oracle: identical chains."""
    N, M = 8, 8
    pr = I.rbm_params(N, M, 3, 0.5)
    s0 = oracle.chain_init(N, 6, rule, 5, 1)
    edges = None if rule == "local" else I.chain_edges(N)
    st, sm = H.metropolis(pr, N, M, rule, edges, s0, 2, 3, 4, 5, 1)
    ref = oracle.metropolis(pr, N, M, rule, edges, s0, 2, 3, 4, 5, 1)
    np.testing.assert_array_equal(sm, ref["samples"])
    np.testing.assert_array_equal(st, ref["state"])


def test_complex_sampler_histogram_against_exact():
    """Complex parameters: the histogram of 200 chains x 300 sweeps (local
    rule, N = 8) matches |psi|^2 (TV < 0.03; i.i.d. draws of the same size
    give about 0.012), not |psi| (TV 0.33 between the two here)."""
    N, M = 8, 6
    p = _params(N, M, 21, 0.4)
    P = np.abs(H.exact_state(p, N, M)) ** 2
    s0 = oracle.chain_init(N, 200, "local", 9, 0)
    _st, sm = H.metropolis(p, N, M, "local", None, s0, 0, 10, 300, 9, 0)
    x = sm.reshape(-1, N)
    idx = ((x < 0).astype(np.int64) * (1 << (N - 1 - np.arange(N)))).sum(axis=1)
    counts = np.bincount(idx, minlength=2 ** N) / idx.size
    assert 0.5 * np.abs(counts - P).sum() < 0.03


def test_sample_moments_converge_to_the_exact_moments():
    """Force, QGT and energy as sample means (Sec. 3.3) over 2e5 i.i.d. draws
    from the exact |psi|^2 agree with the exact moments within the sampling
    error (energy within 4 sigma; force and QGT within 5 % in norm)."""
    N, M = 6, 3
    ham = I.tfim_chain(N, 1.0, 0.8)
    p = _params(N, M, 23, 0.3)
    f_ex, G_ex, e_ex = H.exact_moments(p, N, M, ham)
    P = np.abs(H.exact_state(p, N, M)) ** 2
    basis = exact.basis(N)
    idx = np.random.default_rng(4).choice(P.size, size=200000, p=P / P.sum())
    # evaluate per distinct configuration, then weight by the counts
    counts = np.bincount(idx, minlength=P.size)
    keep = counts > 0
    w = counts[keep] / idx.size
    O = H.jacobian(p, N, M, basis[keep])
    el = H.local_energy(p, N, M, ham, basis[keep])
    f_s, G_s, e_s = H._moments(O, el, w)
    sigma = np.sqrt(np.sum(w * np.abs(el - e_s) ** 2) / idx.size)
    assert abs(e_s - e_ex) < 4 * sigma
    assert np.linalg.norm(f_s - f_ex) < 0.05 * np.linalg.norm(f_ex)
    assert np.linalg.norm(G_s - G_ex) < 0.05 * np.linalg.norm(G_ex)
    # the sample-mean entry point gives the same numbers on the repeated draws
    sub = basis[idx[:2000]]
    f1, G1, e1 = H.sample_moments(p, N, M, ham, sub)
    c = np.bincount(idx[:2000], minlength=P.size)
    k = c > 0
    f2, G2, e2 = H._moments(H.jacobian(p, N, M, basis[k]), H.local_energy(p, N, M, ham, basis[k]), c[k] / 2000)
    np.testing.assert_allclose(f1, f2, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(G1, G2, rtol=1e-10, atol=1e-12)
    assert abs(e1 - e2) < 1e-10


def test_tvmc_slope_estimates_the_exact_slope():
    """The sampled equation of motion (100 chains x 100 sweeps of the complex
    sampler, eps = 0.1) estimates the exact theta_dot within its sampling
    noise (measured 14 %; a dropped conjugate or a flipped gamma gives 150-200
    %), and a Heun step of t-VMC moves the parameters by about dt theta_dot."""
    N, M = 6, 3
    ham = I.tfim_chain(N, 1.0, 0.8)
    p = _params(N, M, 29, 0.3)
    f, G, _e = H.exact_moments(p, N, M, ham)
    ex = H.theta_dot(G, f, -1j, 0.1)
    s0 = oracle.chain_init(N, 100, "local", 3, 0)
    td, st, _es = H.tvmc_rhs(p, N, M, ham, "local", None, s0, 0, 20, 100, 3, 0, -1j, 0.1)
    assert np.linalg.norm(td - ex) < 0.35 * np.linalg.norm(ex)
    assert st.shape == s0.shape
    dt = 0.01
    p1, st1, sweep = H.tvmc_heun(p, N, M, ham, "local", None, st, 120, 50, 3, dt, 0, -1j, 0.1)
    assert sweep == 220 and st1.shape == s0.shape
    assert np.linalg.norm((p1 - p) / dt - ex) < 0.5 * np.linalg.norm(ex)
