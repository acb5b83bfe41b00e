"""Complex holomorphic RBM and time-dependent variational Monte Carlo in
complex128, by exact enumeration of the basis (small N) or over samples.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Model (Sec. 3.2, complex parameters): ln psi(s) = a.s + sum_j ln cosh(b_j +
W_j.s) with a, b, W complex; the map theta -> psi(s) is holomorphic, so the
log-derivatives O_k = d ln psi / d theta_k (Eq. eq:log-derivative-O) are the
complex O_a = s, O_b = tanh theta, O_W = tanh theta s^T.

Expectations under p(s) = |psi(s)|^2 / sum |psi|^2 (Eq. eq: expectation
value VMC):
  force   f~_k = E[O_k^* (E_loc - E[E_loc])]        (Eq. eq:force VMC)
  QGT     G_kl = E[O_k^* O_l] - E[O_k^*] E[O_l]      (Sec. 3.5)
TDVP (Sec. 4.3, Eq. eq:tvmc): sum_l G_kl theta_dot_l = gamma f~_k, gamma = -i
(real time) or -1 (imaginary time); explicit Runge-Kutta steps (Eq.
eq:rk-step), Euler and Heun.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import core as _core
from . import exact as _exact


def n_params(N: int, M: int) -> int:
    return N + M + M * N


def unpack(params, N, M):
    p = np.asarray(params, dtype=np.complex128)
    return p[:N], p[N:N + M], p[N + M:].reshape(M, N)


def lncosh(x):
    """ln cosh x for complex x from cosh x = e^{|x|'} (1 + e^{-2|x|'}) / 2 with
    |x|' = x or -x, whichever has a non-negative real part."""
    x = np.asarray(x, dtype=np.complex128)
    y = np.where(x.real >= 0, x, -x)
    return y + np.log1p(np.exp(-2.0 * y)) - np.log(2.0)


def theta(params, N, M, s):
    _a, b, W = unpack(params, N, M)
    s = np.asarray(s, dtype=np.float64).reshape(-1, N)
    return b[None, :] + s @ W.T


def logpsi(params, N, M, s):
    a, _b, _W = unpack(params, N, M)
    s = np.asarray(s, dtype=np.float64).reshape(-1, N)
    return s @ a + lncosh(theta(params, N, M, s)).sum(axis=1)


def jacobian(params, N, M, s):
    s = np.asarray(s, dtype=np.float64).reshape(-1, N)
    t = np.tanh(theta(params, N, M, s))
    return np.concatenate([s.astype(np.complex128), t, (t[:, :, None] * s[:, None, :]).reshape(s.shape[0], -1)],
                          axis=1)


def _connected(ham, s):
    """Off-diagonal elements <s|H|s'> != 0 of one configuration: a list of
    (element, sites to flip), and the diagonal element."""
    edges = np.asarray(ham["edges"]).reshape(-1, 2)
    E1 = edges.shape[0] - int(ham.get("n_edges2", 0))
    J, J2 = float(ham["J"]), float(ham.get("J2", 0.0))
    diag = sum((J if q < E1 else J2) * s[i] * s[k] for q, (i, k) in enumerate(edges))
    out = []
    if ham["kind"] == "tfim":
        out = [(-float(ham["h"]), (i,)) for i in range(len(s))]
    else:
        for q, (i, k) in enumerate(edges):
            if s[i] != s[k]:
                el = (J if q < E1 else J2) * 2.0
                if q < E1 and ham.get("marshall", False):
                    el = -el
                out.append((el, (int(i), int(k))))
    return diag, out


def local_energy(params, N, M, ham, s):
    """E_loc(s) = sum_s' H_ss' psi(s') / psi(s) (Eq. eq:local-estimator), each
    ratio from two full evaluations of ln psi."""
    s = np.asarray(s, dtype=np.int8).reshape(-1, N)
    out = np.empty(s.shape[0], dtype=np.complex128)
    lp = logpsi(params, N, M, s)
    for k in range(s.shape[0]):
        diag, conn = _connected(ham, s[k])
        e = complex(diag)
        for el, sites in conn:
            sp = s[k].copy()
            sp[list(sites)] *= -1
            e += el * np.exp(logpsi(params, N, M, sp)[0] - lp[k])
        out[k] = e
    return out


def _moments(O, e, w):
    """Weighted force and QGT: w are probabilities summing to one."""
    Om = w @ O
    dO = O - Om
    em = w @ e
    f = dO.conj().T @ (w * (e - em))
    G = (dO.conj() * w[:, None]).T @ dO
    return f, G, em


def exact_moments(params, N, M, ham, sz0=False):
    """Force, QGT and energy under the exact |psi|^2 over all basis states."""
    s = _exact.basis(N)
    if sz0:
        s = s[s.astype(np.int64).sum(axis=1) == 0]
    lp = logpsi(params, N, M, s)
    w = np.exp(2.0 * (lp.real - lp.real.max()))
    w /= w.sum()
    return _moments(jacobian(params, N, M, s), local_energy(params, N, M, ham, s), w)


def sample_moments(params, N, M, ham, s):
    """Force, QGT and energy as sample means (Sec. 3.3)."""
    s = np.asarray(s, dtype=np.int8).reshape(-1, N)
    w = np.full(s.shape[0], 1.0 / s.shape[0])
    return _moments(jacobian(params, N, M, s), local_energy(params, N, M, ham, s), w)


def theta_dot(G, f, gamma, diag_shift=0.0, rcond=None):
    """Solve (G + eps I) theta_dot = gamma f (Eq. eq:tvmc): by a Cholesky factor
    of the Hermitian positive-definite matrix, or, with rcond set, by the
    pseudo-inverse keeping singular values above rcond times the largest."""
    A = G + diag_shift * np.eye(G.shape[0])
    rhs = gamma * f
    if rcond is not None:
        U, sig, Vh = np.linalg.svd(A)
        keep = sig > rcond * sig[0]
        return Vh[keep].conj().T @ ((U[:, keep].conj().T @ rhs) / sig[keep])
    L = np.linalg.cholesky(A)
    y = np.linalg.solve(L, rhs)
    return np.linalg.solve(L.conj().T, y)


def euler(params, rhs, dt):
    """theta(t + dt) = theta(t) + dt k1 (first-order Runge-Kutta)."""
    return params + dt * rhs(params)


def heun(params, rhs, dt):
    """Heun's second-order scheme: k1 = F(theta), k2 = F(theta + dt k1),
    theta(t + dt) = theta(t) + dt (k1 + k2) / 2 (Eq. eq:rk-step with the
    step dt inside the intermediate argument)."""
    k1 = rhs(params)
    k2 = rhs(params + dt * k1)
    return params + 0.5 * dt * (k1 + k2)


def exact_state(params, N, M, sz0=False):
    """psi over the Kronecker basis (normalised), zero outside S_z = 0 if sz0."""
    s = _exact.basis(N)
    lp = logpsi(params, N, M, s)
    v = np.exp(lp - lp.real.max())
    if sz0:
        v[s.astype(np.int64).sum(axis=1) != 0] = 0.0
    return v / np.linalg.norm(v)


def brute_force_marginal(params, N, M, s):
    """psi(s) = sum_h exp(a.s + sum_j h_j theta_j) / 2^M over h in {-1, 1}^M:
    the hidden units summed out one configuration at a time."""
    a, _b, _W = unpack(params, N, M)
    s = np.asarray(s, dtype=np.float64).reshape(-1, N)
    th = theta(params, N, M, s)
    out = np.zeros(s.shape[0], dtype=np.complex128)
    for h in itertools.product([-1.0, 1.0], repeat=M):
        out += np.exp(s @ a + th @ np.array(h))
    return out / 2 ** M


def metropolis(params, N, M, rule, edges, s, sweep0, n_discard, n_samples, seed, stream=0):
    """Metropolis-Hastings chains on |psi|^2 of the complex RBM (Sec. 3.4), on
    the Philox streams of the real-RBM oracle: proposal p of sweep w of chain
    c draws the block ((sweep0 + w) N + p, c, stream, 0) with key (seed, 0);
    the site (local) or edge (exchange) is floor(hi32(y0) n / 2^32), u =
    ((y1 >> 11) + 1/2) 2^-53, and the move is taken iff
    ln u < 2 Re[ln psi(s') - ln psi(s)] (|psi(s')/psi(s)|^2 = e^{2 Re dlnpsi}).
    An exchange proposal on an edge with equal spins is not a move.  Each
    ratio comes from two full evaluations of ln psi.  Returns the new states
    and the samples [C, n_samples, N]."""
    s = np.array(s, dtype=np.int8).reshape(-1, N)
    C = s.shape[0]
    E = 0 if edges is None else np.asarray(edges).reshape(-1, 2).shape[0]
    edges = None if edges is None else np.asarray(edges).reshape(-1, 2)
    key = np.array([seed, 0], dtype=np.uint64)
    samples = np.empty((C, n_samples, N), dtype=np.int8)
    for w in range(n_discard + n_samples):
        for p in range(N):
            q = (sweep0 + w) * N + p
            lp = logpsi(params, N, M, s)
            sp = s.copy()
            move = np.ones(C, dtype=bool)
            lu = np.empty(C)
            for c in range(C):
                y = _core.philox4x64_10(np.array([q, c, stream, 0], dtype=np.uint64), key)
                n = N if rule == "local" else E
                r = int((int(y[0]) >> 32) * n >> 32)
                lu[c] = np.log(((int(y[1]) >> 11) + 0.5) * 2.0 ** -53)
                if rule == "local":
                    sp[c, r] = -sp[c, r]
                else:
                    i, k = edges[r]
                    if s[c, i] == s[c, k]:
                        move[c] = False
                    else:
                        sp[c, i], sp[c, k] = -sp[c, i], -sp[c, k]
            take = move & (lu < 2.0 * (logpsi(params, N, M, sp) - lp).real)
            s[take] = sp[take]
        if w >= n_discard:
            samples[:, w - n_discard] = s
    return s, samples


def tvmc_rhs(params, N, M, ham, rule, edges, chains, sweep0, n_discard, n_samples, seed, stream=0,
             gamma=-1j, diag_shift=0.0, rcond=None):
    """One evaluation of the t-VMC equation of motion (Sec. 4.3): sample the
    chains, form the force and QGT as sample means, solve Eq. eq:tvmc.
    Returns (theta_dot, new chain states, sample-mean energy)."""
    state, samples = metropolis(params, N, M, rule, edges, chains, sweep0, n_discard, n_samples, seed, stream)
    f, G, e = sample_moments(params, N, M, ham, samples.reshape(-1, N))
    return theta_dot(G, f, gamma, diag_shift, rcond), state, e


def tvmc_heun(params, N, M, ham, rule, edges, chains, sweep0, n_samples, seed, dt, stream=0, gamma=-1j,
              diag_shift=0.0, rcond=None):
    """One Heun step of t-VMC: each of the two slopes is evaluated on fresh
    samples (the chains continue; the second slope draws the sweeps after the
    first).  Returns (new parameters, chain states, next sweep index)."""
    k1, chains, _e = tvmc_rhs(params, N, M, ham, rule, edges, chains, sweep0, 0, n_samples, seed, stream, gamma,
                              diag_shift, rcond)
    k2, chains, _e = tvmc_rhs(params + dt * k1, N, M, ham, rule, edges, chains, sweep0 + n_samples, 0, n_samples,
                              seed, stream, gamma, diag_shift, rcond)
    return params + 0.5 * dt * (k1 + k2), chains, sweep0 + 2 * n_samples
