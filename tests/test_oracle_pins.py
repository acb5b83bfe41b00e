"""Pins of the FP64 CPU oracle against facts the paper and the mathematics fix.

Each test compares the oracle with something other than itself: a value the
paper prints, a published known-answer vector, a closed form, a textbook
construction (Kronecker products of Pauli matrices), brute force over tiny
inputs, finite differences, or an invariant between two different formulas
of the paper.  No GPU is used.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from oracle import exact
from paper_2112_10526_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox ----

def test_philox_known_answer_vectors():
    kat = json.load(open(os.path.join(GOLD, "philox4x64_10_kat.json")))
    for v in kat["vectors"]:
        c = np.array([int(x, 16) for x in v["counter"]], dtype=np.uint64)
        k = np.array([int(x, 16) for x in v["key"]], dtype=np.uint64)
        out = oracle.philox4x64_10(c, k)
        assert [int(x) for x in out] == [int(x, 16) for x in v["out"]]


def test_philox_matches_numpy_generator():
    # numpy.random.Philox is the same generator; it increments the counter
    # before producing a block, so its block for counter c-1 is ours for c.
    rng = np.random.default_rng(7)
    for _ in range(20):
        c = rng.integers(1, 2**63, size=4, dtype=np.uint64)
        k = rng.integers(0, 2**63, size=2, dtype=np.uint64)
        ref = np.random.Philox(key=k, counter=c - np.array([1, 0, 0, 0], dtype=np.uint64))
        assert [int(x) for x in oracle.philox4x64_10(c, k)] == [int(x) for x in ref.random_raw(4)]


# --------------------------------------------------------- Pauli algebra ----

def test_pauli_conventions_paper_operator_example():
    g = json.load(open(os.path.join(GOLD, "paper_operator_example.json")))
    op = exact.site_op(exact._SX, 0, 2) + exact.site_op(exact._SX, 1, 2)
    dense = (op @ op).toarray().real
    np.testing.assert_array_equal(dense, np.array(g["dense"]))


# ------------------------------------------------------------- ln psi -------

@pytest.mark.parametrize("N,M", [(4, 3), (5, 6), (6, 8)])
def test_logpsi_is_boltzmann_marginal(N, M):
    """The RBM amplitude is the hidden-spin marginal of a Boltzmann machine:
    psi(s) = sum_{h in {-1,1}^M} exp(a.s + b.h + h^T W s) = e^{a.s} prod_j
    2 cosh(theta_j).  Brute force over all hidden configurations pins
    ln psi up to the constant M ln 2."""
    p = I.rbm_params(N, M, 11, 0.4)
    a, b, W = oracle.unpack(p, N, M)
    s = I.random_configs(7, N, 3)
    hs = np.array(list(itertools.product([-1.0, 1.0], repeat=M)))
    for k in range(s.shape[0]):
        sk = s[k].astype(np.float64)
        z = np.exp(a @ sk + hs @ b + hs @ (W @ sk))
        ref = np.log(z.sum()) - M * np.log(2.0)
        assert abs(oracle.logpsi(p, N, M, s[k:k + 1])[0] - ref) < 1e-12 * max(1, abs(ref))


def test_logpsi_large_activation_branch_is_continuous():
    N, M = 3, 2
    for x in [19.999999, 20.0, 20.000001, 35.0, -35.0]:
        p = np.zeros(N + M + M * N)
        p[N] = x  # b_0
        lp = oracle.logpsi(p, N, M, np.ones((1, N), dtype=np.int8))[0]
        ref = abs(x) + np.log1p(np.exp(-2 * abs(x))) - np.log(2.0)
        assert abs(lp - ref) < 1e-13 * abs(ref)


# ---------------------------------------------------------- local energy ----

HAMS_SMALL = [
    ("tfim-chain8", 8, lambda: I.tfim_chain(8, 1.0, 0.7), False),
    ("tfim-chain10-J-0.5", 10, lambda: I.tfim_chain(10, -0.5, 1.3), False),
    ("heis-chain8-marshall", 8, lambda: I.heis_chain(8, 1.0, True), False),
    ("heis-chain8-plain", 8, lambda: I.heis_chain(8, 0.8, False), False),
    ("heis-4x4-marshall", 16, lambda: I.heis_square(4, 1.0, True), True),
    ("tfim-3x3-is-not-bipartite-free", 9, lambda: I.tfim_square(3, 1.0, 2.0), False),
    ("j1j2-chain8-marshall", 8, lambda: I.j1j2_chain(8, 1.0, 0.5, True), False),
    ("j1j2-chain10-plain", 10, lambda: I.j1j2_chain(10, 0.8, 0.35, False), False),
    ("j1j2-4x4-marshall", 16, lambda: I.j1j2_square(4, 1.0, 0.5, True), True),
]


@pytest.mark.parametrize("name,N,hf,sz0", HAMS_SMALL, ids=[h[0] for h in HAMS_SMALL])
def test_local_energy_equals_hamiltonian_action(name, N, hf, sz0):
    """E_loc(s) = (H psi)(s) / psi(s) for every basis state (Eq.
    eq:local-estimator), with H assembled from Pauli Kronecker products."""
    ham = hf()
    M = N if N <= 10 else 4
    p = I.rbm_params(N, M, 5, 0.35)
    es = exact.ExactState(p, N, M, sz0=sz0)
    H = exact.hamiltonian(N, ham)
    v = es.psi_full()
    hv = H @ v
    el = oracle.local_energy(p, N, M, ham, es.configs)
    ref = hv[es.index] / v[es.index]
    assert np.max(np.abs(el - ref) / np.maximum(1.0, np.abs(ref))) < 1e-11


EXPECT_CASES = HAMS_SMALL[:4] + HAMS_SMALL[6:8]


@pytest.mark.parametrize("name,N,hf,sz0", EXPECT_CASES, ids=[h[0] for h in EXPECT_CASES])
def test_exact_expectation_identity(name, N, hf, sz0):
    """<H> = sum_s p(s) E_loc(s) with p = |psi|^2/<psi|psi>  (Eq. eq:
    expectation value VMC), and the variational bound <H> >= E0."""
    ham = hf()
    p = I.rbm_params(N, N, 9, 0.3)
    es = exact.ExactState(p, N, N, sz0=sz0)
    e_dir = es.energy(ham)
    assert abs(es.eloc_mean(ham) - e_dir) < 1e-12 * max(1, abs(e_dir))
    e0, _ = exact.ground_energy(N, ham)
    assert e_dir >= e0 - 1e-10


def test_zero_variance_uniform_state():
    """a = b = W = 0 gives a uniform psi.  With J = 0 it is the sigma^x
    eigenstate of the Ising field term: E_loc = -h N for every s.  Without the
    Marshall sign it is the fully symmetric S_z = 0 state, an eigenstate of
    every sigma_i . sigma_k with eigenvalue 1: E_loc = J E for every s."""
    N, M = 10, 7
    p = np.zeros(N + M + M * N)
    s = I.random_configs(50, N, 1)
    el = oracle.local_energy(p, N, M, I.tfim_chain(N, 0.0, 1.7), s)
    np.testing.assert_allclose(el, -1.7 * N, rtol=1e-15, atol=0)
    ham = I.heis_square(4, 0.9, False)
    s = I.random_configs(50, 16, 2, sz0=True)
    el = oracle.local_energy(np.zeros(16 + 3 + 48), 16, 3, ham, s)
    np.testing.assert_allclose(el, 0.9 * ham["edges"].shape[0], rtol=1e-15, atol=0)
    # both edge classes of the J1-J2 model: E_loc = J1 E1 + J2 E2
    ham = I.j1j2_square(4, 0.9, -0.4, False)
    el = oracle.local_energy(np.zeros(16 + 3 + 48), 16, 3, ham, s)
    np.testing.assert_allclose(el, 0.9 * 32 - 0.4 * 32, rtol=1e-14, atol=0)


# ---------------------------------------------------- exact ground states ---

@pytest.mark.parametrize("N,J,h", [(8, 1.0, 1.0), (10, 1.0, 0.5), (12, 1.0, 1.0), (16, 1.0, 1.0),
                                   (10, -1.0, 2.0)])
def test_tfim_ed_matches_free_fermions(N, J, h):
    e0, _ = exact.ground_energy(N, I.tfim_chain(N, J, h))
    assert abs(e0 - exact.tfim_free_fermion_e0(N, J, h)) < 1e-10 * abs(e0)


def test_tfim_n16_closed_form_value():
    # J = h = 1: E0 = -2 / sin(pi / 2N).
    assert abs(exact.tfim_free_fermion_e0(16) - (-2.0 / np.sin(np.pi / 32))) < 1e-13


def test_heisenberg_small_closed_forms():
    """Two spins: sigma.sigma has the singlet eigenvalue -3.  Four-site ring:
    H = J (S1+S3).(S2+S4) in spin units has E0 = -2J, i.e. -8J in Pauli
    units."""
    e2, _ = exact.ground_energy(2, {"kind": "heis", "J": 1.0, "edges": np.array([[0, 1]])})
    assert abs(e2 + 3.0) < 1e-12
    e4, _ = exact.ground_energy(4, I.heis_chain(4, 1.3, False))
    assert abs(e4 + 8.0 * 1.3) < 1e-12
    e4m, _ = exact.ground_energy(4, I.heis_chain(4, 1.3, True))
    assert abs(e4m + 8.0 * 1.3) < 1e-12


@pytest.mark.parametrize("L", [8, 10, 12])
@pytest.mark.parametrize("marshall", [False, True])
def test_majumdar_ghosh_closed_form(L, marshall):
    """At J2 = J1 / 2 the periodic J1-J2 chain (Eq. eq: j1 j2 heisenberg in
    one dimension, even L) has the nearest-neighbour dimer products as exact
    ground states (Majumdar and Ghosh, J. Math. Phys. 10, 1388 (1969)), with
    E0 = -3 J1 L / 8 in spin units, i.e. -3 J1 L / 2 with Pauli matrices.
    The Marshall rotation of the nearest-neighbour sublattices leaves it
    unchanged."""
    J1 = 1.3
    e0, _ = exact.ground_energy(L, I.j1j2_chain(L, J1, J1 / 2, marshall), sz0=True)
    assert abs(e0 + 1.5 * J1 * L) < 1e-9 * L
    # away from that point the dimer energy is no longer the ground energy
    e1, _ = exact.ground_energy(L, I.j1j2_chain(L, J1, 0.2 * J1, marshall), sz0=True)
    assert e1 < -1.5 * J1 * L - 0.1


def test_marshall_rotation_makes_ground_state_positive():
    """The Marshall sign rotation leaves the spectrum unchanged and makes the
    S_z = 0 ground state of the bipartite Heisenberg lattice sign-free, which
    a real RBM (psi >= 0, Sec. 3.2 warning box) can represent."""
    ham = I.heis_square(4, 1.0, True)
    e_m, g_m = exact.ground_energy(16, ham, sz0=True)
    e_p, g_p = exact.ground_energy(16, dict(ham, marshall=False), sz0=True)
    assert abs(e_m - e_p) < 1e-9
    g = g_m[exact.sz0_mask(16)]
    g = g * np.sign(g[np.argmax(np.abs(g))])
    assert g.min() > 0
    # the un-rotated ground state has both signs
    gp = g_p[exact.sz0_mask(16)]
    assert gp.min() < 0 < gp.max()


# ---------------------------------------------------------- derivatives -----

def test_jacobian_central_differences():
    """O_k = d ln psi / d theta_k (Eq. eq:log-derivative-O) against central
    differences in FP64 with step 1e-6, relative 1e-6."""
    N, M = 6, 5
    p = I.rbm_params(N, M, 21, 0.5)
    s = I.random_configs(4, N, 4)
    O = oracle.jacobian(p, N, M, s)
    h = 1e-6
    for kk in range(p.size):
        pp, pm = p.copy(), p.copy()
        pp[kk] += h
        pm[kk] -= h
        fd = (oracle.logpsi(pp, N, M, s) - oracle.logpsi(pm, N, M, s)) / (2 * h)
        np.testing.assert_allclose(O[:, kk], fd, rtol=1e-6, atol=1e-9)


def test_jacobian_columns_central_differences_and_thread_count():
    """The column-restricted Jacobian against central differences of ln psi
    (step 1e-6, relative 1e-6) for a ragged set of columns of every block
    (a, b, W), and equal, bit for bit, to the same columns of the full rows;
    the full rows and the local energies do not depend on the number of
    OpenMP threads (each configuration is one thread's work)."""
    N, M = 7, 5
    p = I.rbm_params(N, M, 22, 0.5)
    s = I.random_configs(9, N, 5)
    cols = np.array([0, 6, N, N + 4, N + M, N + M + 3, N + M + 2 * N + 6, N + M + M * N - 1, N + 2])
    Oc = oracle.jacobian_cols(p, N, M, s, cols)
    h = 1e-6
    for c, kk in enumerate(cols):
        pp, pm = p.copy(), p.copy()
        pp[kk] += h
        pm[kk] -= h
        fd = (oracle.logpsi(pp, N, M, s) - oracle.logpsi(pm, N, M, s)) / (2 * h)
        np.testing.assert_allclose(Oc[:, c], fd, rtol=1e-6, atol=1e-9)
    np.testing.assert_array_equal(Oc, oracle.jacobian(p, N, M, s)[:, cols])
    assert oracle.jacobian_cols(p, N, M, s, []).shape == (9, 0)
    import subprocess
    import sys
    code = ("import hashlib, numpy as np, oracle; from paper_2112_10526_gb300 import inputs as I; "
            "N, M = 12, 24; p = I.rbm_params(N, M, 3, 0.3); ham = I.heis_chain(N); "
            "s0 = oracle.chain_init(N, 37, 'exchange', 3); "
            "r = oracle.metropolis(p, N, M, 'exchange', ham['edges'], s0, 0, 2, 3, 3); "
            "x = r['samples'].reshape(-1, N); "
            "e = oracle.local_energy(p, N, M, ham, x); O = oracle.jacobian(p, N, M, x); "
            "print(hashlib.sha256(b''.join(a.tobytes() for a in (r['samples'], r['decisions'], r['margin'], "
            "r['logpsi'], e, O, oracle.logpsi(p, N, M, x)))).hexdigest())")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = set()
    for threads in ("1", "5"):
        env = dict(os.environ, OMP_NUM_THREADS=threads, PYTHONPATH=root)
        outs.add(subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                                check=True, cwd=root).stdout.strip())
    assert len(outs) == 1


def test_force_is_gradient_of_exact_energy():
    """f = 2 Re Cov[O, E_loc] is the gradient of <H> (Eqs. eq:force VMC,
    eq:VMC gradient:real), checked by central differences of the exact
    energy."""
    N, M = 6, 4
    ham = I.tfim_chain(N, 1.0, 0.8)
    p = I.rbm_params(N, M, 8, 0.4)
    f = exact.ExactState(p, N, M).force(ham)
    h = 1e-5
    for kk in range(p.size):
        pp, pm = p.copy(), p.copy()
        pp[kk] += h
        pm[kk] -= h
        fd = (exact.ExactState(pp, N, M).energy(ham) - exact.ExactState(pm, N, M).energy(ham)) / (2 * h)
        assert abs(f[kk] - fd) < 1e-7 * max(1.0, abs(fd))


def test_sample_force_and_qgt_equal_exact_on_empirical_distribution():
    """The sample estimators (force: 2/N_s sum O dE; QGT: centred Gram
    dJ^T dJ / N_s, Eq. eq:qgt-compact) equal the exact covariance formulas
    (Eq. eq:qgt_est, E[O O] - E[O]E[O]) evaluated on the empirical
    distribution of the samples."""
    N, M = 6, 4
    ham = I.heis_chain(N, 1.0, True)
    p = I.rbm_params(N, M, 3, 0.4)
    s = I.random_configs(300, N, 6, sz0=True)
    O = oracle.jacobian(p, N, M, s)
    e = oracle.local_energy(p, N, M, ham, s)
    uniq, inv, cnt = np.unique(s, axis=0, return_inverse=True, return_counts=True)
    w = cnt / cnt.sum()
    Ou = oracle.jacobian(p, N, M, uniq)
    eu = oracle.local_energy(p, N, M, ham, uniq)
    mo = w @ Ou
    G = (Ou.T * w) @ Ou - np.outer(mo, mo)
    f = 2.0 * (Ou.T @ (w * (eu - w @ eu)))
    np.testing.assert_allclose(oracle.qgt_dense(O), G, atol=1e-13)
    np.testing.assert_allclose(oracle.force(O, e), f, atol=1e-12)


def test_qgt_is_fubini_study_metric():
    """d(psi_theta, psi_theta+dtheta)^2 = dtheta^T G dtheta to second order
    (Eqs. eq:fubini-study-metric and eq:qgt)."""
    N, M = 6, 4
    p = I.rbm_params(N, M, 4, 0.4)
    es = exact.ExactState(p, N, M)
    G = es.qgt()
    rng = np.random.default_rng(1)
    v0 = es.psi_full()
    for _ in range(3):
        d = rng.normal(size=p.size)
        d /= np.linalg.norm(d)
        eps = 1e-4
        # the average of +eps and -eps cancels the third-order term
        d2 = [np.arccos(min(1.0, abs(v0 @ exact.ExactState(p + sg * eps * d, N, M).psi_full()))) ** 2
              for sg in (1.0, -1.0)]
        assert abs(0.5 * sum(d2) / eps**2 - d @ G @ d) < 1e-6 * max(1e-3, d @ G @ d)


def test_qgt_onthefly_equals_dense():
    """App. B.3 (w = Jv/N_s, dw = w - <w>, J^T dw) equals App. B.2 (the
    centred Gram) applied to v, plus the diagonal shift."""
    N, M = 7, 6
    p = I.rbm_params(N, M, 2, 0.3)
    s = I.random_configs(200, N, 2)
    O = oracle.jacobian(p, N, M, s)
    v = np.random.default_rng(0).normal(size=p.size)
    np.testing.assert_allclose(oracle.qgt_matvec_onthefly(O, v, 0.01),
                               oracle.qgt_dense(O) @ v + 0.01 * v, rtol=1e-12, atol=1e-13)


# ---------------------------------------------------------------- solves ----

def test_cholesky_solve_matches_library_solve():
    N, M = 5, 5
    p = I.rbm_params(N, M, 2, 0.3)
    s = I.random_configs(64, N, 2)
    O = oracle.jacobian(p, N, M, s)
    S = oracle.qgt_dense(O)
    F = np.random.default_rng(3).normal(size=p.size)
    x = oracle.solve_cholesky(S, F, 0.01)
    ref = np.linalg.solve(S + 0.01 * np.eye(p.size), F)
    np.testing.assert_allclose(x, ref, rtol=1e-9, atol=1e-11)


def test_cg_matches_cholesky():
    N, M = 6, 6
    p = I.rbm_params(N, M, 2, 0.3)
    s = I.random_configs(128, N, 8)
    O = oracle.jacobian(p, N, M, s)
    F = np.random.default_rng(4).normal(size=p.size)
    x1 = oracle.solve_cholesky(oracle.qgt_dense(O), F, 0.05)
    x2, it, res = oracle.solve_cg(lambda v: oracle.qgt_matvec_onthefly(O, v, 0.05), F, tol=1e-12)
    assert res <= 1e-12 and it > 0
    np.testing.assert_allclose(x2, x1, rtol=1e-9, atol=1e-10)


def test_svd_solve_on_a_known_spectrum():
    """S = Q diag(2, 1e-3, 1e-20, 0) Q^T with Q orthogonal: with rcond = 1e-10
    the truncated solve keeps the first two directions, delta = Q diag(1/2,
    1e3, 0, 0) Q^T F."""
    Q, _ = np.linalg.qr(np.random.default_rng(3).normal(size=(4, 4)))
    S = Q @ np.diag([2.0, 1e-3, 1e-20, 0.0]) @ Q.T
    F = np.array([0.3, -1.2, 0.7, 2.0])
    ref = Q @ (np.array([0.5, 1e3, 0.0, 0.0]) * (Q.T @ F))
    np.testing.assert_allclose(oracle.solve_svd(S, F, 0.0, 1e-10), ref, rtol=1e-9, atol=1e-9)
    # a diagonal shift moves every singular value by eps and keeps them all
    ref_eps = Q @ ((Q.T @ F) / (np.array([2.0, 1e-3, 1e-20, 0.0]) + 0.1))
    np.testing.assert_allclose(oracle.solve_svd(S, F, 0.1, 1e-10), ref_eps, rtol=1e-12, atol=1e-12)


def test_svd_solve_equals_cholesky_when_shifted():
    N, M = 6, 6
    p = I.rbm_params(N, M, 2, 0.3)
    s = I.random_configs(128, N, 8)
    S = oracle.qgt_dense(oracle.jacobian(p, N, M, s))
    F = np.random.default_rng(4).normal(size=p.size)
    np.testing.assert_allclose(oracle.solve_svd(S, F, 0.05), oracle.solve_cholesky(S, F, 0.05),
                               rtol=1e-9, atol=1e-10)


def test_svd_solve_rank_deficient_sample_and_parameter_space():
    """N_s = 30 samples, N_p = 48 parameters: S has rank <= 29.  The truncated
    solve through the N_s x N_s Gram matrix equals the one through S; the
    result lies in the row space of the centred Jacobian and solves S delta =
    F projected on the range of S."""
    N, M, Ns = 6, 6, 30
    p = I.rbm_params(N, M, 5, 0.4)
    O = oracle.jacobian(p, N, M, I.random_configs(Ns, N, 9))
    S = oracle.qgt_dense(O)
    F = oracle.force(O, np.random.default_rng(6).normal(size=Ns))
    d1 = oracle.solve_svd(S, F, 0.0, 1e-10)
    d2 = oracle.solve_svd_samplespace(O, F, 1e-10)
    assert np.linalg.norm(d1 - d2) < 1e-8 * np.linalg.norm(d1)
    dJ = O - O.mean(axis=0)
    P = np.linalg.pinv(dJ, rcond=1e-10) @ dJ  # projector on the row space
    assert np.linalg.norm(P @ d1 - d1) < 1e-8 * np.linalg.norm(d1)
    assert np.linalg.norm(S @ d1 - P @ F) < 1e-8 * np.linalg.norm(F)


def test_sr_is_projected_imaginary_time_step():
    """SR (Eq. eq:stochastic-reconfiguration, real case) is the least-squares
    projection of the imaginary-time step (H - E) psi onto the tangent space
    spanned by the centred log-derivatives; with f = 2 Re f~ the SR solution
    is twice the projection coefficients (the gamma = -1 case of Eq. eq:tvmc).
    Checked with exact weights and a library least-squares solver."""
    N, M = 6, 3
    ham = I.tfim_chain(N, 1.0, 0.9)
    p = I.rbm_params(N, M, 6, 0.4)
    es = exact.ExactState(p, N, M)
    O = oracle.jacobian(p, N, M, es.configs)
    e = oracle.local_energy(p, N, M, ham, es.configs)
    sq = np.sqrt(es.p)
    A = (O - es.p @ O) * sq[:, None]
    rhs = (e - es.p @ e) * sq
    coef = np.linalg.lstsq(A, rhs, rcond=None)[0]
    delta = oracle.solve_cholesky(es.qgt(), es.force(ham), 0.0)
    np.testing.assert_allclose(delta, 2.0 * coef, rtol=1e-6, atol=1e-8)
    # and a small SR step lowers the exact energy
    e_new = exact.ExactState(oracle.sgd_update(p, delta, 0.01), N, M).energy(ham)
    assert e_new < es.energy(ham)


# --------------------------------------------------------------- sampler ----

def _tv(counts, p):
    return 0.5 * np.abs(counts / counts.sum() - p).sum()


def test_chain_init_rules():
    s = oracle.chain_init(300, 5, "local", seed=9, stream=2)
    assert set(np.unique(s)) <= {-1, 1}
    s2 = oracle.chain_init(300, 5, "local", seed=9, stream=2)
    np.testing.assert_array_equal(s, s2)
    # bit layout: site i <- bit (i mod 256) of block floor(i/256), word y0 lowest
    y = oracle.philox4x64_10(np.array([1, 3, 2, 1], dtype=np.uint64), np.array([9, 0], dtype=np.uint64))
    bits = [(int(y[(i % 256) // 64]) >> (i % 64)) & 1 for i in range(256, 300)]
    np.testing.assert_array_equal(s[3, 256:], np.where(np.array(bits) == 1, 1, -1))
    e = oracle.chain_init(100, 40, "exchange", seed=3)
    assert (e.sum(axis=1) == 0).all()
    assert len({tuple(r) for r in e}) == 40


def _sz0_histogram(rows, N):
    """Counts of each S_z = 0 configuration of N sites among `rows`, in the
    order of itertools.combinations of the up sites."""
    index = {c: k for k, c in enumerate(itertools.combinations(range(N), N // 2))}
    counts = np.zeros(len(index))
    for r in rows:
        counts[index[tuple(np.flatnonzero(r == 1))]] += 1
    return counts


def _chi2_pvalue(counts):
    from scipy.stats import chi2
    exp = counts.sum() / counts.size
    return float(chi2.sf(((counts - exp) ** 2 / exp).sum(), counts.size - 1))


def test_chain_init_sz0_is_uniform_over_the_sector():
    """The S_z = 0 initial states (random_state of Sec. 2.1 restricted to the
    zero-magnetisation sector) must be uniform over the C(6, 3) = 20
    configurations: a chi-square test over 40000 chains.  The same test,
    run on a shuffle with the plausible off-by-one (the swap partner drawn
    from [0, i) instead of [0, i]: Sattolo's single-cycle shuffle, which can
    never return the starting order), must reject it."""
    N, C = 6, 40000
    rows = oracle.chain_init(N, C, "exchange", seed=31, stream=5)
    assert (rows.sum(axis=1) == 0).all()
    counts = _sz0_histogram(rows, N)
    assert counts.min() > 0
    assert _chi2_pvalue(counts) > 1e-6

    def shuffled(c, partner_range):
        r = np.array([1] * (N // 2) + [-1] * (N // 2), dtype=np.int8)
        for i in range(N - 1, 0, -1):
            y = oracle.philox4x64_10(np.array([i, c, 5, 1], dtype=np.uint64), np.array([31, 0], dtype=np.uint64))
            j = (int(y[0]) >> 32) * partner_range(i) >> 32
            r[i], r[j] = r[j], r[i]
        return r

    bad = np.array([shuffled(c, lambda i: i) for c in range(4000)])
    assert _chi2_pvalue(_sz0_histogram(bad, N)) < 1e-6
    # with the inclusive range the hand-written shuffle is the oracle's own
    good = np.array([shuffled(c, lambda i: i + 1) for c in range(200)])
    np.testing.assert_array_equal(good, rows[:200])


def test_metropolis_local_tv_against_exact():
    """Histogram of single-flip Metropolis samples against exact |psi|^2 at
    N = 12 (1e6 samples, TV < 0.01).  Parameters have sigma = 0.3 so that the
    distribution is far from uniform (with sigma = 0.01 even i.i.d. sampling
    has E[TV] ~ 0.026 at 1e6 samples; i.i.d. draws give TV ~ 0.005 here).
    Larger sigma (0.5) makes |psi|^2 bimodal at this seed, and single flips
    then do not cross between the modes within the run."""
    N, M = 12, 12
    p = I.rbm_params(N, M, 12, 0.3)
    es = exact.ExactState(p, N, M)
    C, ns = 100, 10000
    s0 = oracle.chain_init(N, C, "local", seed=5)
    mc = oracle.metropolis(p, N, M, "local", None, s0, 0, 20, ns, seed=5)
    x = mc["samples"].reshape(-1, N)
    idx = ((x < 0).astype(np.int64) * (1 << (N - 1 - np.arange(N)))).sum(axis=1)
    counts = np.bincount(idx, minlength=2 ** N).astype(np.float64)
    assert _tv(counts, es.p) < 0.01


@pytest.mark.parametrize("dmax", [1, 2])
def test_metropolis_exchange_tv_and_sz(dmax):
    """Exchange rule on a 12-site ring at S_z = 0 (924 states): magnetisation
    is conserved and the histogram matches exact |psi|^2 (TV < 0.01).
    Nearest-neighbour swaps on a ring mix slowly once |psi|^2 is peaked, so
    this variant uses sigma = 0.2 and 2e6 samples (i.i.d. draws: TV ~ 0.004).
    With dmax = 2 the proposals run over the next-nearest-neighbour edges too
    (the exchange rule of the J1-J2 example of Sec. 7)."""
    N, M = 12, 12
    p = I.rbm_params(N, M, 13, 0.2)
    es = exact.ExactState(p, N, M, sz0=True)
    C, ns = 200, 10000
    edges = I.chain_edges(N) if dmax == 1 else I.j1j2_chain(N)["edges"]
    s0 = oracle.chain_init(N, C, "exchange", seed=6)
    mc = oracle.metropolis(p, N, M, "exchange", edges, s0, 0, 50, ns, seed=6)
    x = mc["samples"].reshape(-1, N)
    assert (x.astype(np.int64).sum(axis=1) == 0).all()
    full = ((x < 0).astype(np.int64) * (1 << (N - 1 - np.arange(N)))).sum(axis=1)
    pos = np.full(2 ** N, -1)
    pos[es.index] = np.arange(es.index.size)
    counts = np.bincount(pos[full], minlength=es.index.size).astype(np.float64)
    assert _tv(counts, es.p) < 0.01


@pytest.mark.parametrize("lattice", ["ring", "j1j2-ring"])
def test_metropolis_hamiltonian_rule_tv(lattice):
    """MetropolisHamiltonian rule (Sec. 3.4) on a 12-site ring at S_z = 0:
    s' is drawn uniformly from the swaps across the antiparallel edges, so
    g(s'|s) = 1/n(s) and the acceptance carries L(s, s') = ln n(s) - ln n(s').
    The histogram matches exact |psi|^2 (TV < 0.01).  Dropping the correction
    biases the chain towards configurations with many antiparallel edges
    (TV about 0.07 at these parameters).  Every proposal is a move."""
    N, M = 12, 12
    p = I.rbm_params(N, M, 13, 0.2)
    es = exact.ExactState(p, N, M, sz0=True)
    C, ns = 200, 10000
    edges = I.chain_edges(N) if lattice == "ring" else I.j1j2_chain(N)["edges"]
    s0 = oracle.chain_init(N, C, "hamiltonian", seed=7)
    mc = oracle.metropolis(p, N, M, "hamiltonian", edges, s0, 0, 50, ns, seed=7)
    assert set(np.unique(mc["decisions"])) <= {0, 1}
    x = mc["samples"].reshape(-1, N)
    assert (x.astype(np.int64).sum(axis=1) == 0).all()
    full = ((x < 0).astype(np.int64) * (1 << (N - 1 - np.arange(N)))).sum(axis=1)
    pos = np.full(2 ** N, -1)
    pos[es.index] = np.arange(es.index.size)
    counts = np.bincount(pos[full], minlength=es.index.size).astype(np.float64)
    assert _tv(counts, es.p) < 0.01


def test_metropolis_hamiltonian_rule_single_proposal_by_hand():
    """One proposal of the Hamiltonian rule against its definition, spelled out
    with numpy: the antiparallel edges of s in list order, the r-th one swapped,
    and the decision ln u < 2 (ln psi(s') - ln psi(s)) + ln n(s) - ln n(s')."""
    N, M = 8, 5
    p = I.rbm_params(N, M, 3, 0.5)
    edges = I.j1j2_chain(N)["edges"]
    s0 = np.array([[1, 1, -1, 1, -1, -1, 1, -1]], dtype=np.int8)
    # the first proposal of sweep 0: Philox block (0, chain 0, stream 3, 0)
    y = oracle.philox4x64_10(np.array([0, 0, 3, 0], dtype=np.uint64), np.array([11, 0], dtype=np.uint64))
    anti = [e for e in range(edges.shape[0]) if s0[0, edges[e, 0]] != s0[0, edges[e, 1]]]
    r = (int(y[0]) >> 32) * len(anti) >> 32
    i, k = edges[anti[r]]
    s1 = s0.copy()
    s1[0, i], s1[0, k] = s1[0, k], s1[0, i]
    n1 = sum(s1[0, a] != s1[0, b] for a, b in edges)
    lp0, lp1 = oracle.logpsi(p, N, M, s0)[0], oracle.logpsi(p, N, M, s1)[0]
    lu = np.log(((int(y[1]) >> 11) + 0.5) * 2.0 ** -53)
    expect = lu < 2 * (lp1 - lp0) + np.log(len(anti)) - np.log(n1)
    # a one-proposal run: a sweep is N proposals, so force the other N - 1
    # proposals to "reject" and read the oracle's own first decision
    forced = np.zeros((1, 1, N), dtype=np.uint8)
    forced[0, 0, 0] = 1 if expect else 0
    mc = oracle.metropolis(p, N, M, "hamiltonian", edges, s0, 0, 0, 1, seed=11, stream=3, forced=forced)
    assert mc["decisions"][0, 0, 0] == int(expect)
    assert abs(mc["margin"][0, 0, 0] - abs(2 * (lp1 - lp0) + np.log(len(anti)) - np.log(n1) - lu)) < 1e-12
    np.testing.assert_array_equal(mc["samples"][0, 0], s1[0] if expect else s0[0])


def test_metropolis_forced_follow_and_decisions():
    N, M = 10, 10
    p = I.rbm_params(N, M, 4, 0.3)
    s0 = oracle.chain_init(N, 6, "exchange", seed=1)
    ham = I.heis_chain(N)
    a = oracle.metropolis(p, N, M, "exchange", ham["edges"], s0, 3, 2, 4, seed=1)
    # replaying with its own decisions reproduces the run
    b = oracle.metropolis(p, N, M, "exchange", ham["edges"], s0, 3, 2, 4, seed=1, forced=a["decisions"])
    np.testing.assert_array_equal(a["samples"], b["samples"])
    np.testing.assert_array_equal(a["decisions"], b["decisions"])
    # non-moves are exactly the proposals whose edge spins were equal
    assert set(np.unique(a["decisions"])) <= {0, 1, 2}
    assert (a["n_accepted"] == (a["decisions"] == 1).sum(axis=(1, 2))).all()
    # ln psi of every sample is the full evaluation
    np.testing.assert_allclose(a["logpsi"].ravel(), oracle.logpsi(p, N, M, a["samples"].reshape(-1, N)),
                               rtol=0, atol=0)
    # continuing a chain equals one long run (counter-based streams)
    c1 = oracle.metropolis(p, N, M, "exchange", ham["edges"], s0, 0, 0, 3, seed=1)
    c2 = oracle.metropolis(p, N, M, "exchange", ham["edges"], c1["state"], 3, 0, 2, seed=1)
    c12 = oracle.metropolis(p, N, M, "exchange", ham["edges"], s0, 0, 0, 5, seed=1)
    np.testing.assert_array_equal(np.concatenate([c1["samples"], c2["samples"]], axis=1), c12["samples"])


def test_mc_energy_within_error_of_exact():
    """The MC estimate of <H> from the oracle's chains lies within 4 sigma of
    the exact expectation (Sec. 3.3)."""
    N, M = 10, 10
    ham = I.tfim_chain(N, 1.0, 1.0)
    p = I.rbm_params(N, M, 14, 0.3)
    e_ex = exact.ExactState(p, N, M).energy(ham)
    s0 = oracle.chain_init(N, 32, "local", seed=3)
    mc = oracle.metropolis(p, N, M, "local", None, s0, 0, 20, 200, seed=3)
    st = oracle.stats(oracle.local_energy(p, N, M, ham, mc["samples"].reshape(-1, N)), n_chains=32)
    assert abs(st["mean"] - e_ex) < 4 * st["error"]


@pytest.mark.parametrize("rho", [0.0, 0.8])
def test_stats_error_bar_is_the_spread_of_the_mean(rho):
    """The error bar estimates the standard deviation of the sample mean.
    4000 repetitions of 32 independent stationary AR(1) chains of 16 samples
    (lag-one correlation rho): the rms reported error matches the spread of
    the means across repetitions within 5 %.  For rho = 0.8 the i.i.d.
    formula sqrt(var / N_s) would be about 2.5x too small; the chain-mean
    estimate is not."""
    R, C, n = 4000, 32, 16
    rng = np.random.default_rng(8)
    x = np.empty((R, C, n))
    x[:, :, 0] = rng.normal(size=(R, C))
    for t in range(1, n):
        x[:, :, t] = rho * x[:, :, t - 1] + np.sqrt(1 - rho ** 2) * rng.normal(size=(R, C))
    means = x.reshape(R, -1).mean(axis=1)
    err = np.array([oracle.stats(x[r].ravel(), n_chains=C)["error"] for r in range(R)])
    ratio = np.sqrt(np.mean(err ** 2)) / means.std()
    assert abs(ratio - 1) < 0.05, ratio
    if rho > 0:
        naive = np.sqrt(np.mean([oracle.stats(x[r].ravel())["error"] ** 2 for r in range(R)])) / means.std()
        assert naive < 0.5, naive


def test_stats_definitions():
    e = np.array([1.0, 2.0, 3.0, 4.0, 5.0, 6.0])
    st = oracle.stats(e, n_chains=3)
    assert st["mean"] == 3.5
    assert abs(st["variance"] - 35.0 / 12.0) < 1e-15
    cm = np.array([1.5, 3.5, 5.5])
    assert abs(st["error"] - np.sqrt(cm.var() / 3)) < 1e-15
    st1 = oracle.stats(e)
    assert abs(st1["error"] - np.sqrt(35.0 / 12.0 / 6)) < 1e-15
