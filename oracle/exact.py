"""Exact enumeration and exact diagonalisation for small lattices.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The Hamiltonians here are assembled from Kronecker products of 2x2 Pauli
matrices (the textbook tensor-product construction of Eq.
eq:hilbert:discrete), independently of the connected-element enumeration in
nk_oracle.c, so that comparing the two pins the local estimator.

Basis order: index x in [0, 2^N) with site 0 the most significant bit; the
sigma^z eigenvalue of site i is s_i = 1 - 2 * bit_{N-1-i}(x).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import core

_SX = sp.csr_matrix(np.array([[0.0, 1.0], [1.0, 0.0]]))
_SY = sp.csr_matrix(np.array([[0.0, -1.0j], [1.0j, 0.0]]))
_SZ = sp.csr_matrix(np.array([[1.0, 0.0], [0.0, -1.0]]))
_ID = sp.identity(2, format="csr")


def basis(N):
    """All 2^N configurations as int8 [2^N, N] in the Kronecker order."""
    x = np.arange(2 ** N, dtype=np.int64)
    bits = (x[:, None] >> (N - 1 - np.arange(N))[None, :]) & 1
    return (1 - 2 * bits).astype(np.int8)


def site_op(op, i, N):
    """op acting on site i of an N-site chain of spin-1/2."""
    m = sp.identity(1, format="csr")
    for k in range(N):
        m = sp.kron(m, op if k == i else _ID, format="csr")
    return m


def two_sublattices(N, edges):
    """A two-colouring of the lattice graph (raises if it is not bipartite)."""
    col = -np.ones(N, dtype=np.int64)
    adj = [[] for _ in range(N)]
    for i, k in np.asarray(edges).reshape(-1, 2):
        adj[int(i)].append(int(k))
        adj[int(k)].append(int(i))
    for root in range(N):
        if col[root] >= 0:
            continue
        col[root] = 0
        stack = [root]
        while stack:
            u = stack.pop()
            for v in adj[u]:
                if col[v] < 0:
                    col[v] = 1 - col[u]
                    stack.append(v)
                elif col[v] == col[u]:
                    raise ValueError("lattice is not bipartite")
    return col


def hamiltonian(N, ham):
    """Sparse H (real, CSR) of the transverse-field Ising model
    H = sum_e J_e sz_i sz_k - h sum_i sx_i  (Eq. eq:tf-ising-hamiltonian) or
    the Heisenberg model H = sum_e J_e sigma_i . sigma_k  (Eq. eq: j1 j2
    heisenberg), J_e = J on the nearest-neighbour edges and J2 on the last
    ham["n_edges2"] edges (next-nearest neighbours).  With ham["marshall"],
    the Heisenberg H is conjugated by U = prod_{i in A} sz_i for the
    two-colouring A/B of the nearest-neighbour graph."""
    edges = np.asarray(ham["edges"]).reshape(-1, 2)
    E1 = edges.shape[0] - int(ham.get("n_edges2", 0))
    coupling = [float(ham["J"]) if q < E1 else float(ham.get("J2", 0.0)) for q in range(edges.shape[0])]
    dim = 2 ** N
    H = sp.csr_matrix((dim, dim), dtype=np.complex128)
    sz = [site_op(_SZ, i, N) for i in range(N)]
    if ham["kind"] == "tfim":
        h = float(ham["h"])
        for (i, k), Je in zip(edges, coupling):
            H = H + Je * (sz[i] @ sz[k])
        for i in range(N):
            H = H - h * site_op(_SX, i, N)
    else:
        sx = [site_op(_SX, i, N) for i in range(N)]
        sy = [site_op(_SY, i, N) for i in range(N)]
        for (i, k), Je in zip(edges, coupling):
            H = H + Je * (sx[i] @ sx[k] + sy[i] @ sy[k] + sz[i] @ sz[k])
        if ham.get("marshall", False):
            col = two_sublattices(N, edges[:E1])
            U = sp.identity(dim, format="csr", dtype=np.complex128)
            for i in range(N):
                if col[i] == 0:
                    U = U @ sz[i]
            H = U @ H @ U
    assert abs(H.imag).max() < 1e-12 if H.nnz else True
    return sp.csr_matrix(H.real)


def sz0_mask(N):
    """Basis states with total S_z = 0."""
    return basis(N).sum(axis=1) == 0


def ground_energy(N, ham, sz0=False):
    """Lowest eigenvalue of H (optionally restricted to S_z = 0) and its
    eigenvector in the full basis."""
    H = hamiltonian(N, ham)
    if sz0:
        m = np.flatnonzero(sz0_mask(N))
        Hs = H[m][:, m]
    else:
        m = np.arange(2 ** N)
        Hs = H
    if Hs.shape[0] <= 512:
        w, v = np.linalg.eigh(Hs.toarray())
        e0, g = w[0], v[:, 0]
    else:
        w, v = spla.eigsh(Hs, k=1, which="SA", tol=1e-14, maxiter=100000)
        e0, g = w[0], v[:, 0]
    full = np.zeros(2 ** N)
    full[m] = g
    return float(e0), full


def tfim_free_fermion_e0(N, J=1.0, h=1.0):
    """Ground energy of the periodic transverse-field Ising chain (even N) from
    its Jordan-Wigner free-fermion solution (Pfeuty, Ann. Phys. 57, 79
    (1970)): E0 = -sum_{n=0}^{N-1} sqrt(J^2 + h^2 - 2 J h cos((2n+1) pi / N))."""
    n = np.arange(N)
    k = (2 * n + 1) * np.pi / N
    return float(-np.sqrt(J * J + h * h - 2 * J * h * np.cos(k)).sum())


class ExactState:
    """The full-sum variational state of Sec. 3.1 ("ExactState"): every basis
    configuration (or every S_z = 0 configuration) weighted by |psi|^2."""

    def __init__(self, params, N, M, sz0=False):
        self.N, self.M = N, M
        self.params = np.asarray(params, dtype=np.float64)
        allc = basis(N)
        self.index = np.flatnonzero(allc.sum(axis=1) == 0) if sz0 else np.arange(2 ** N)
        self.configs = allc[self.index]
        lp = core.logpsi(self.params, N, M, self.configs)
        self.logpsi = lp
        w = np.exp(2.0 * (lp - lp.max()))
        self.p = w / w.sum()

    def psi_full(self):
        """Normalised psi as a vector over the full 2^N basis."""
        v = np.zeros(2 ** self.N)
        amp = np.exp(self.logpsi - self.logpsi.max())
        v[self.index] = amp / np.linalg.norm(amp)
        return v

    def energy(self, ham):
        """<psi|H|psi>/<psi|psi> from the Pauli-product H."""
        H = hamiltonian(self.N, ham)
        v = self.psi_full()
        return float(v @ (H @ v))

    def eloc_mean(self, ham):
        return float(self.p @ core.local_energy(self.params, self.N, self.M, ham, self.configs))

    def force(self, ham):
        """Exact f = 2 E_p[O (E_loc - E_p[E_loc])] (Eq. eq:force VMC)."""
        e = core.local_energy(self.params, self.N, self.M, ham, self.configs)
        O = core.jacobian(self.params, self.N, self.M, self.configs)
        de = e - self.p @ e
        return 2.0 * (O.T @ (self.p * de))

    def qgt(self):
        """Exact G = E_p[O O^T] - E_p[O] E_p[O]^T (Eq. eq:qgt_est)."""
        O = core.jacobian(self.params, self.N, self.M, self.configs)
        mo = self.p @ O
        return (O.T * self.p) @ O - np.outer(mo, mo)

    def sample(self, n, seed):
        """ExactSampler of Sec. 3.4: i.i.d. draws from |psi|^2 (indices into
        self.configs)."""
        rng = np.random.default_rng(seed)
        return rng.choice(self.p.size, size=n, p=self.p)
