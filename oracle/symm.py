"""Symmetric RBM (RBMSymm, Sec. 5 "symmetric neural quantum states") in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

A permutation group G of the sites acts on configurations.  Following the
embedding layer (Eq. eq: equivariant: embedding), feature f at group
element g is
    theta_{f,g}(s) = b_f + sum_j W_{f,j} s_{pi_g(j)},
and the wave function is the product of cosh over all features and group
elements (the RBMSymm equation of the same section),
    ln psi(s) = a sum_j s_j + sum_{f,g} ln cosh theta_{f,g}(s).
Readings: the printed equation has no biases; a hidden bias b_f per feature
and one visible bias a (the symmetric restriction of the RBM's a.s) are
kept, and both reduce to the printed form at zero.

Parameter vector: [a (1); b (alpha); W (alpha x N row-major)],
Np = 1 + alpha + alpha N.  perms: int [|G|, N], perms[g, j] = pi_g(j);
the rows must form a group.

The model equals a plain RBM with M = alpha |G| hidden units and tied
parameters (unit (f, g) has bias b_f and weight W_{f,j} on site pi_g(j),
every visible bias a), so sampling and local energies run through the RBM
oracle on the expanded parameters (`expand`); ln psi and the
log-derivatives are written out directly here.
"""
from __future__ import annotations

import numpy as np

from . import core


def n_params(N: int, alpha: int) -> int:
    return 1 + alpha + alpha * N


def unpack(params, N, alpha):
    p = np.asarray(params, dtype=np.float64)
    return p[0], p[1:1 + alpha], p[1 + alpha:].reshape(alpha, N)


def _lncosh(x):
    # ln cosh x = ln(e^x + e^-x) - ln 2
    return np.logaddexp(x, -x) - np.log(2.0)


def theta(params, N, alpha, perms, s):
    """theta_{f,g}(s) for a batch: [B, alpha, |G|]."""
    _a, b, W = unpack(params, N, alpha)
    s = np.asarray(s, dtype=np.float64).reshape(-1, N)
    sp = s[:, np.asarray(perms)]  # sp[k, g, j] = s_k[pi_g(j)]
    return b[None, :, None] + np.einsum("fj,kgj->kfg", W, sp)


def logpsi(params, N, alpha, perms, s):
    """ln psi(s) = a sum_j s_j + sum_{f,g} ln cosh theta_{f,g}(s)."""
    a, _b, _W = unpack(params, N, alpha)
    s = np.asarray(s, dtype=np.float64).reshape(-1, N)
    return a * s.sum(axis=1) + _lncosh(theta(params, N, alpha, perms, s)).sum(axis=(1, 2))


def jacobian(params, N, alpha, perms, s):
    """O_k(s) = d ln psi(s) / d theta_k (Eq. eq:log-derivative-O) for the
    symmetric RBM: O_a = sum_j s_j, O_{b_f} = sum_g tanh theta_{f,g},
    O_{W_{f,j}} = sum_g tanh theta_{f,g} s_{pi_g(j)}.  [B, Np]."""
    s = np.asarray(s, dtype=np.float64).reshape(-1, N)
    t = np.tanh(theta(params, N, alpha, perms, s))
    sp = s[:, np.asarray(perms)]
    O_W = np.einsum("kfg,kgj->kfj", t, sp).reshape(s.shape[0], -1)
    return np.concatenate([s.sum(axis=1, keepdims=True), t.sum(axis=2), O_W], axis=1)


def expand(params, N, alpha, perms):
    """Parameters of the equal plain RBM (M = alpha |G|, hidden unit index
    f |G| + g): a_i = a, b_{(f,g)} = b_f, W_{(f,g), pi_g(j)} = W_{f,j}."""
    a, b, W = unpack(params, N, alpha)
    perms = np.asarray(perms)
    G = perms.shape[0]
    We = np.zeros((alpha, G, N))
    for f in range(alpha):
        for g in range(G):
            We[f, g, perms[g]] = W[f]
    return np.concatenate([np.full(N, a), np.repeat(b, G), We.ravel()])


def local_energy(params, N, alpha, perms, ham, s):
    """E_loc (Eq. eq:local-estimator) of the symmetric RBM: the same psi as
    the expanded RBM."""
    G = np.asarray(perms).shape[0]
    return core.local_energy(expand(params, N, alpha, perms), N, alpha * G, ham, s)


def sr_step(params, N, alpha, perms, ham, rule, chains, sweep0, n_discard, n_samples, seed, stream=0,
            diag_shift=0.01, lr=0.01, solver="cholesky", cg_tol=1e-10, cg_maxiter=1000):
    """One VMC iteration with stochastic reconfiguration (Sec. 4.1) in the
    symmetric parameters: chains and local energies of the expanded RBM (the
    same psi), the Jacobian, force, QGT and update in the Np = 1 + alpha +
    alpha N symmetric parameters."""
    G = np.asarray(perms).shape[0]
    M = alpha * G
    pe = expand(params, N, alpha, perms)
    edges = np.asarray(ham["edges"]).reshape(-1, 2)
    mc = core.metropolis(pe, N, M, rule, edges, chains, sweep0, n_discard, n_samples, seed, stream)
    C = chains.shape[0]
    s = mc["samples"].reshape(-1, N)
    e = core.local_energy(pe, N, M, ham, s)
    st = core.stats(e, n_chains=C)
    O = jacobian(params, N, alpha, perms, s)
    F = core.force(O, e)
    if solver == "cholesky":
        delta = core.solve_cholesky(core.qgt_dense(O), F, diag_shift)
        iters, res = 0, 0.0
    else:
        delta, iters, res = core.solve_cg(lambda v: core.qgt_matvec_onthefly(O, v, diag_shift), F,
                                          tol=cg_tol, maxiter=cg_maxiter)
    return {"params": core.sgd_update(params, delta, lr), "state": mc["state"], "samples": mc["samples"],
            "eloc": e, "stats": st, "force": F, "delta": delta, "cg_iters": iters, "cg_residual": res}
