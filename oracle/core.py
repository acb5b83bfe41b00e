"""FP64 oracle: ctypes binding of nk_oracle.c plus numpy linear algebra.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Every function cites
the passage of the NetKet 3 paper (arXiv:2112.10526) that it restates.

Conventions shared with the product library (by specification, not by code):
  * parameters theta = [a (N); b (M); W (M x N row-major)], float64;
  * configurations int8 in {-1, +1}, row-major [batch, N];
  * Hamiltonian dict: {"kind": "tfim"|"heis", "J": float, "h": float,
    "marshall": bool, "edges": int32 [E, 2]}, optionally with "J2": float
    and "n_edges2": int, the last n_edges2 edges being the next-nearest
    neighbours of coupling J2 (Eq. eq: j1 j2 heisenberg);
  * sampler rule: "local" (single-spin flip), "exchange" (edge swap at
    fixed magnetisation) or "hamiltonian" (a uniformly chosen configuration
    connected by an off-diagonal element of a Heisenberg-type Hamiltonian on
    the given edges, with the Hastings correction).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nk_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

KIND = {"tfim": 0, "heis": 1}
RULE = {"local": 0, "exchange": 1, "hamiltonian": 2}


def build(force: bool = False) -> str:
    """Compile nk_oracle.c into liboracle.so with plain gcc (no fast-math),
    with OpenMP over independent configurations where gcc supports it (the
    thread count, OMP_NUM_THREADS, does not change any result)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P = ctypes.c_void_p
    i32, i64, u64, u32, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double
    lib.oc_logpsi.argtypes = [i32, i32, P, P, i64, P]
    lib.oc_local_energy.argtypes = [i32, i32, P, i32, f64, f64, f64, i32, i32, i32, P, P, i64, P]
    lib.oc_jacobian.argtypes = [i32, i32, P, P, i64, P]
    lib.oc_jacobian_cols.argtypes = [i32, i32, P, P, i64, i32, P, P]
    lib.oc_philox4x64_10.argtypes = [P, P, P]
    lib.oc_chain_init.argtypes = [i32, i32, i32, u64, u32, P]
    lib.oc_metropolis.argtypes = [i32, i32, P, i32, i32, P, i32, P, i64, i32, i32, u64, u32,
                                  P, P, P, P, P, P]
    for f in ("oc_logpsi", "oc_local_energy", "oc_jacobian", "oc_jacobian_cols", "oc_philox4x64_10",
              "oc_chain_init", "oc_metropolis"):
        getattr(lib, f).restype = None
    _lib = lib
    return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _cfg(s, N):
    s = np.ascontiguousarray(s, dtype=np.int8).reshape(-1, N)
    return s


def _par(params):
    return np.ascontiguousarray(params, dtype=np.float64)


def n_params(N: int, M: int) -> int:
    return N + M + M * N


def unpack(params, N, M):
    """Split theta into (a, b, W) views."""
    params = np.asarray(params, dtype=np.float64)
    return params[:N], params[N:N + M], params[N + M:].reshape(M, N)


# ---------------------------------------------------------------------------
# Per-configuration definitions (C)
# ---------------------------------------------------------------------------

def logpsi(params, N, M, s):
    """ln psi(s) = a.s + sum_j ln cosh(b_j + W_j.s)  (RBM of Sec. 3.2)."""
    lib = _load()
    s = _cfg(s, N)
    out = np.empty(s.shape[0], dtype=np.float64)
    pa = _par(params)
    lib.oc_logpsi(N, M, _p(pa), _p(s), s.shape[0], _p(out))
    return out


def local_energy(params, N, M, ham, s):
    """E_loc(s) = sum_s' H_ss' psi(s')/psi(s)  (Eq. eq:local-estimator)."""
    lib = _load()
    s = _cfg(s, N)
    out = np.empty(s.shape[0], dtype=np.float64)
    edges = np.ascontiguousarray(ham["edges"], dtype=np.int32).reshape(-1, 2)
    E2 = int(ham.get("n_edges2", 0))
    assert 0 <= E2 <= edges.shape[0]
    pa = _par(params)
    lib.oc_local_energy(N, M, _p(pa), KIND[ham["kind"]], float(ham["J"]), float(ham.get("J2", 0.0)),
                        float(ham.get("h", 0.0)), int(bool(ham.get("marshall", False))), edges.shape[0], E2,
                        _p(edges), _p(s), s.shape[0], _p(out))
    return out


def jacobian(params, N, M, s):
    """J_kl = O_l(s_k) = d ln psi(s_k)/d theta_l  (Eq. eq:log-derivative-O, App. B.1)."""
    lib = _load()
    s = _cfg(s, N)
    out = np.empty((s.shape[0], n_params(N, M)), dtype=np.float64)
    pa = _par(params)
    lib.oc_jacobian(N, M, _p(pa), _p(s), s.shape[0], _p(out))
    return out


def jacobian_cols(params, N, M, s, cols):
    """Columns `cols` of the same Jacobian, J[:, cols] (Eq.
    eq:log-derivative-O): for very large N_p, where the full rows do not fit
    in memory."""
    lib = _load()
    s = _cfg(s, N)
    cols = np.ascontiguousarray(cols, dtype=np.int64).ravel()
    assert cols.size == 0 or (cols.min() >= 0 and cols.max() < n_params(N, M))
    out = np.empty((s.shape[0], cols.size), dtype=np.float64)
    pa = _par(params)
    lib.oc_jacobian_cols(N, M, _p(pa), _p(s), s.shape[0], cols.size, _p(cols), _p(out))
    return out


def philox4x64_10(counter, key):
    """One Philox4x64-10 block (Salmon et al., SC'11)."""
    lib = _load()
    c = np.ascontiguousarray(counter, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.empty(4, dtype=np.uint64)
    lib.oc_philox4x64_10(_p(c), _p(k), _p(out))
    return out


def chain_init(N, C, rule, seed, stream=0):
    """Random initial states (random_state of Sec. 2.1); exchange rule -> S_z = 0."""
    lib = _load()
    s = np.empty((C, N), dtype=np.int8)
    lib.oc_chain_init(N, C, RULE[rule], int(seed), int(stream), _p(s))
    return s


def metropolis(params, N, M, rule, edges, s, sweep0, n_discard, n_samples, seed, stream=0,
               forced=None):
    """Metropolis-Hastings chains (Sec. 3.4).  Returns a dict with the new chain
    states, samples [C, n_samples, N], ln psi of each sample, the oracle's own
    decisions and margins per proposal, and accepted-move counts.

    `s` [C, N] is not modified; the updated states are returned."""
    lib = _load()
    s = np.array(_cfg(s, N), copy=True)
    C = s.shape[0]
    n_sweeps = n_discard + n_samples
    edges = np.ascontiguousarray(edges if edges is not None else np.zeros((0, 2)), dtype=np.int32).reshape(-1, 2)
    samples = np.empty((C, n_samples, N), dtype=np.int8)
    lp = np.empty((C, n_samples), dtype=np.float64)
    dec = np.empty((C, n_sweeps, N), dtype=np.uint8)
    margin = np.empty((C, n_sweeps, N), dtype=np.float64)
    nacc = np.empty(C, dtype=np.int64)
    f = None
    if forced is not None:
        f = np.ascontiguousarray(forced, dtype=np.uint8).reshape(C, n_sweeps, N)
    pa = _par(params)
    lib.oc_metropolis(N, M, _p(pa), RULE[rule], edges.shape[0], _p(edges), C, _p(s), int(sweep0),
                      int(n_discard), int(n_samples), int(seed), int(stream), _p(samples), _p(lp),
                      _p(f), _p(dec), _p(margin), _p(nacc))
    return {"state": s, "samples": samples, "logpsi": lp, "decisions": dec, "margin": margin,
            "n_accepted": nacc}


# ---------------------------------------------------------------------------
# Sample statistics, force, QGT, solves, update (numpy, FP64)
# ---------------------------------------------------------------------------

def stats(eloc, n_chains=None):
    """Monte Carlo mean of the local energy (Sec. 3.3, "the required classical
    expectation values are then estimated by averaging over a sequence"):
    mean = (1/N_s) sum_k E_k, variance = (1/N_s) sum_k (E_k - mean)^2.

    The error of the mean is not fixed by the paper.  Reading used here: with
    n_chains chains of >= 2 samples each (samples stored chain-major), the
    standard error sqrt(var(chain means) / n_chains); otherwise
    sqrt(variance / N_s).  Pinned statistically: over repeated independent
    runs its rms matches the spread of the mean (i.i.d. and autocorrelated
    chains)."""
    e = np.asarray(eloc, dtype=np.float64).ravel()
    ns = e.size
    mean = e.sum() / ns
    var = ((e - mean) ** 2).sum() / ns
    if n_chains and n_chains > 1 and ns // n_chains >= 2 and ns % n_chains == 0:
        cm = e.reshape(n_chains, -1).mean(axis=1)
        err = np.sqrt(((cm - cm.mean()) ** 2).sum() / n_chains / n_chains)
    else:
        err = np.sqrt(var / ns)
    return {"mean": mean, "variance": var, "error": err}


def force(O, eloc):
    """Real energy gradient f = 2 Re f~ with f~_i = E[O_i* (E_loc - E[E_loc])]
    (Eqs. eq:force VMC, eq:VMC gradient:real, eq:gradE:real)."""
    O = np.asarray(O, dtype=np.float64)
    e = np.asarray(eloc, dtype=np.float64).ravel()
    ns = e.size
    de = e - e.sum() / ns
    return 2.0 * (O.T @ de) / ns


def qgt_dense(O):
    """S = G = (1/N_s) dJ^T dJ with the centred Jacobian
    dJ_ki = J_ki - (1/N_s) sum_k J_ki  (App. B.2, Eq. eq:qgt-compact)."""
    O = np.asarray(O, dtype=np.float64)
    ns = O.shape[0]
    dJ = O - O.sum(axis=0) / ns
    return (dJ.T @ dJ) / ns


def qgt_matvec_onthefly(O, v, diag_shift=0.0):
    """QGTOnTheFly product (App. B.3): w = (1/N_s) J v;  dw = w - <w>;
    G v = J^T dw;  plus the diagonal shift eps v (Sec. 3.5)."""
    O = np.asarray(O, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    ns = O.shape[0]
    w = (O @ v) / ns
    dw = w - w.sum() / ns
    return O.T @ dw + diag_shift * v


def solve_cholesky(S, F, diag_shift):
    """(S + eps I) delta = F by a dense Cholesky factor and two triangular
    solves (Sec. 3.5 "Solving linear systems", direct solver; Eq.
    eq:stochastic-reconfiguration, real case)."""
    A = np.asarray(S, dtype=np.float64) + diag_shift * np.eye(S.shape[0])
    L = np.linalg.cholesky(A)
    y = _forward_subst(L, np.asarray(F, dtype=np.float64))
    return _backward_subst(L.T, y)


def _forward_subst(L, b):
    n = L.shape[0]
    y = np.zeros(n)
    for i in range(n):
        y[i] = (b[i] - L[i, :i] @ y[:i]) / L[i, i]
    return y


def _backward_subst(U, b):
    n = U.shape[0]
    x = np.zeros(n)
    for i in range(n - 1, -1, -1):
        x[i] = (b[i] - U[i, i + 1:] @ x[i + 1:]) / U[i, i]
    return x


def solve_cg(matvec, F, tol=1e-10, maxiter=1000):
    """Conjugate gradients on (S + eps I) delta = F with x0 = 0 (Sec. 3.5,
    iterative solver).  Stops when ||r|| <= tol ||F||.  Returns (x, iters,
    relative residual)."""
    F = np.asarray(F, dtype=np.float64)
    x = np.zeros_like(F)
    r = F.copy()
    p = r.copy()
    rr = r @ r
    fn = np.sqrt(F @ F)
    if fn == 0.0:
        return x, 0, 0.0
    it = 0
    while it < maxiter and np.sqrt(rr) > tol * fn:
        Ap = matvec(p)
        alpha = rr / (p @ Ap)
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = r @ r
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it, np.sqrt(rr) / fn


def solve_svd(S, F, diag_shift=0.0, rcond=1e-12):
    """(S + eps I) delta = F through the singular value decomposition of the
    symmetric positive semi-definite S + eps I, suppressing the singular
    values below rcond times the largest (Sec. 3.5, non-iterative solvers
    whose stability is controlled by dropping small singular values):
    delta = sum_{k: sigma_k > rcond sigma_max} v_k (u_k . F) / sigma_k."""
    A = np.asarray(S, dtype=np.float64) + diag_shift * np.eye(S.shape[0])
    U, sig, Vt = np.linalg.svd(A)
    keep = sig > rcond * sig[0] if sig.size else sig > 0
    coef = (U[:, keep].T @ np.asarray(F, dtype=np.float64)) / sig[keep]
    return Vt[keep].T @ coef


def solve_svd_samplespace(O, F, rcond=1e-12):
    """The same truncated solve (eps = 0) from the N_s x N_s Gram matrix:
    with dJ the centred Jacobian and T = dJ dJ^T / N_s = sum_k lambda_k u_k
    u_k^T, the nonzero spectrum of S = dJ^T dJ / N_s is that of T with
    singular vectors v_k = dJ^T u_k / sqrt(N_s lambda_k), so
    delta = sum_{k: lambda_k > rcond lambda_max} v_k (v_k . F) / lambda_k."""
    O = np.asarray(O, dtype=np.float64)
    ns = O.shape[0]
    dJ = O - O.sum(axis=0) / ns
    lam, U = np.linalg.eigh(dJ @ dJ.T / ns)
    order = np.argsort(lam)[::-1]
    lam, U = lam[order], U[:, order]
    keep = lam > rcond * lam[0]
    V = dJ.T @ U[:, keep] / np.sqrt(ns * lam[keep])
    return V @ ((V.T @ np.asarray(F, dtype=np.float64)) / lam[keep])


def sgd_update(params, delta, lr):
    """theta_i -> theta_i - eta delta_i  (Sec. 4.1, SGD update rule)."""
    return np.asarray(params, dtype=np.float64) - lr * np.asarray(delta, dtype=np.float64)


def sr_step(params, N, M, ham, rule, chains, sweep0, n_discard, n_samples, seed, stream=0,
            diag_shift=0.01, lr=0.01, solver="cholesky", cg_tol=1e-10, cg_maxiter=1000,
            forced=None, svd_rcond=1e-12):
    """One VMC iteration with stochastic reconfiguration (Sec. 4.1): sample,
    local energies, force, QGT solve, SGD update.  Returns the new parameters,
    new chain states and the per-step diagnostics."""
    edges = np.asarray(ham["edges"]).reshape(-1, 2)
    if rule == "hamiltonian" and ham["kind"] == "tfim":
        # the connected configurations of the Ising model are the N single
        # flips, drawn uniformly: the local rule
        rule = "local"
    elif rule == "hamiltonian" and float(ham.get("J2", 0.0)) == 0.0:
        # edges with a zero coupling connect nothing
        edges = edges[:edges.shape[0] - int(ham.get("n_edges2", 0))]
    mc = metropolis(params, N, M, rule, edges, chains, sweep0, n_discard, n_samples, seed, stream,
                    forced=forced)
    C = chains.shape[0]
    s = mc["samples"].reshape(-1, N)
    e = local_energy(params, N, M, ham, s)
    st = stats(e, n_chains=C)
    O = jacobian(params, N, M, s)
    F = force(O, e)
    if solver == "cholesky":
        delta = solve_cholesky(qgt_dense(O), F, diag_shift)
        iters, res = 0, 0.0
    elif solver == "svd":
        delta = solve_svd(qgt_dense(O), F, diag_shift, svd_rcond)
        iters, res = 0, 0.0
    else:
        delta, iters, res = solve_cg(lambda v: qgt_matvec_onthefly(O, v, diag_shift), F,
                                     tol=cg_tol, maxiter=cg_maxiter)
    new = sgd_update(params, delta, lr)
    return {"params": new, "state": mc["state"], "samples": mc["samples"], "eloc": e, "stats": st,
            "force": F, "delta": delta, "cg_iters": iters, "cg_residual": res,
            "n_accepted": mc["n_accepted"], "decisions": mc["decisions"], "margin": mc["margin"]}
