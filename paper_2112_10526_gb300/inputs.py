"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds no arithmetic of the method: it only draws parameters and
configurations from numpy generators and lists lattice edges.  Both the CUDA
path and the CPU oracle consume what it returns.

Recipe (matching the workloads of the NetKet 3 paper, Secs. 8-10):
  * parameters a, b, W ~ N(0, sigma^2) i.i.d. from
    ``numpy.random.default_rng(seed).normal``, drawn in the order a (N),
    b (M), W (M x N row-major); sigma = 0.01 unless stated;
  * periodic chain of L sites: edges (i, i+1 mod L) for i = 0..L-1;
  * periodic L x L square lattice: site i = x L + y, edges (i, right) then
    (i, down) for every site in order, right = ((x+1) mod L) L + y,
    down = x L + (y+1) mod L  (E = 2 L^2);
  * its next-nearest neighbours (the two diagonals, Sec. 7): edges
    (i, ((x+1) mod L) L + (y+1) mod L) then (i, ((x+1) mod L) L + (y-1) mod L)
    for every site in order (2 L^2 more); on the chain (i, i+2 mod L);
  * J1-J2 models list the nearest-neighbour edges first and the
    next-nearest ones after them ("n_edges2" of them, coupling "J2");
  * symmetry groups are lists of site permutations (the lattice
    translations);
  * random configurations: i.i.d. +-1 spins, or uniformly random S_z = 0
    configurations (a random permutation of N/2 up and N/2 down spins).
"""
from __future__ import annotations

import numpy as np


def rbm_params(N: int, M: int, seed: int, sigma: float = 0.01) -> np.ndarray:
    rng = np.random.default_rng(seed)
    a = rng.normal(0.0, sigma, N)
    b = rng.normal(0.0, sigma, M)
    W = rng.normal(0.0, sigma, (M, N))
    return np.concatenate([a, b, W.ravel()]).astype(np.float64)


def symm_params(N: int, alpha: int, seed: int, sigma: float = 0.01) -> np.ndarray:
    """Symmetric-RBM parameters [a (1); b (alpha); W (alpha x N)] i.i.d.
    N(0, sigma^2), drawn in that order from default_rng(seed)."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, sigma, size=1 + alpha + alpha * N)


def chain_edges(L: int) -> np.ndarray:
    return np.array([[i, (i + 1) % L] for i in range(L)], dtype=np.int32).reshape(-1, 2)


def square_edges(L: int) -> np.ndarray:
    out = []
    for x in range(L):
        for y in range(L):
            i = x * L + y
            out.append([i, ((x + 1) % L) * L + y])
            out.append([i, x * L + (y + 1) % L])
    return np.array(out, dtype=np.int32).reshape(-1, 2)


def square_nnn_edges(L: int) -> np.ndarray:
    out = []
    for x in range(L):
        for y in range(L):
            i = x * L + y
            out.append([i, ((x + 1) % L) * L + (y + 1) % L])
            out.append([i, ((x + 1) % L) * L + (y - 1) % L])
    return np.array(out, dtype=np.int32).reshape(-1, 2)


def chain_nnn_edges(L: int) -> np.ndarray:
    return np.array([[i, (i + 2) % L] for i in range(L)], dtype=np.int32).reshape(-1, 2)


def translations_chain(L: int) -> np.ndarray:
    """Translation group of the periodic chain as site permutations:
    row g maps site j to (j + g) mod L."""
    return np.array([[(j + g) % L for j in range(L)] for g in range(L)], dtype=np.int64)


def translations_square(L: int) -> np.ndarray:
    """Translation group of the periodic L x L square lattice: row
    dx L + dy maps site x L + y to ((x + dx) mod L) L + (y + dy) mod L."""
    out = []
    for dx in range(L):
        for dy in range(L):
            out.append([((x + dx) % L) * L + (y + dy) % L for x in range(L) for y in range(L)])
    return np.array(out, dtype=np.int64)


def random_configs(B: int, N: int, seed: int, sz0: bool = False) -> np.ndarray:
    rng = np.random.default_rng(seed)
    if not sz0:
        return (2 * rng.integers(0, 2, size=(B, N)) - 1).astype(np.int8)
    base = np.array([1] * (N // 2) + [-1] * (N - N // 2), dtype=np.int8)
    return np.stack([rng.permutation(base) for _ in range(B)]).astype(np.int8)


def tfim_chain(L: int, J: float = 1.0, h: float = 1.0) -> dict:
    return {"kind": "tfim", "J": J, "h": h, "marshall": False, "edges": chain_edges(L)}


def tfim_square(L: int, J: float = 1.0, h: float = 3.04) -> dict:
    return {"kind": "tfim", "J": J, "h": h, "marshall": False, "edges": square_edges(L)}


def heis_square(L: int, J: float = 1.0, marshall: bool = True) -> dict:
    return {"kind": "heis", "J": J, "h": 0.0, "marshall": marshall, "edges": square_edges(L)}


def heis_chain(L: int, J: float = 1.0, marshall: bool = True) -> dict:
    return {"kind": "heis", "J": J, "h": 0.0, "marshall": marshall, "edges": chain_edges(L)}


def j1j2_square(L: int, J1: float = 1.0, J2: float = 0.5, marshall: bool = True) -> dict:
    e2 = square_nnn_edges(L)
    return {"kind": "heis", "J": J1, "J2": J2, "h": 0.0, "marshall": marshall,
            "edges": np.concatenate([square_edges(L), e2]), "n_edges2": int(e2.shape[0])}


def j1j2_chain(L: int, J1: float = 1.0, J2: float = 0.5, marshall: bool = True) -> dict:
    e2 = chain_nnn_edges(L)
    return {"kind": "heis", "J": J1, "J2": J2, "h": 0.0, "marshall": marshall,
            "edges": np.concatenate([chain_edges(L), e2]), "n_edges2": int(e2.shape[0])}


# The workloads (sizes from the paper's examples and benchmarks).
WORKLOADS = {
    "tfim1d_n16": dict(N=16, alpha=1, ham=lambda: tfim_chain(16, 1.0, 1.0), rule="local",
                       chains=16, per_chain=64, discard=16, seed=1, diag_shift=0.01, lr=0.01,
                       solver="cholesky"),
    "heis2d_10x10": dict(N=100, alpha=2, ham=lambda: heis_square(10, 1.0, True), rule="exchange",
                         chains=1024, per_chain=8, discard=16, seed=2, diag_shift=0.01, lr=0.01,
                         solver="cholesky_samplespace"),
    "tfim2d_20x20": dict(N=400, alpha=4, ham=lambda: tfim_square(20, 1.0, 3.04), rule="local",
                         chains=16384, per_chain=1, discard=16, seed=3, diag_shift=0.01, lr=0.01,
                         solver="cg"),
    "heis2d_24x24": dict(N=576, alpha=8, ham=lambda: heis_square(24, 1.0, True), rule="exchange",
                         chains=8192, per_chain=8, discard=16, seed=5, diag_shift=0.01, lr=0.01,
                         solver="cg"),
    # Sec. 5: the symmetric RBM (RBMSymm) on the 10 x 10 Heisenberg lattice,
    # alpha = 4 features over the 100 translations (400 tied hidden units,
    # 405 parameters), dense Cholesky in the symmetric parameters.
    "heis2d_10x10_symm": dict(N=100, alpha=4, symm="translations_square", ham=lambda: heis_square(10, 1.0, True),
                              rule="exchange", chains=1024, per_chain=8, discard=16, seed=7, diag_shift=0.01,
                              lr=0.01, solver="cholesky"),
    # Sec. 7: J1 = 1, J2 = 0.5 on the 10 x 10 square lattice, exchange moves
    # over both edge classes (d_max = 2), one sample per chain (n_chains =
    # n_samples = 1024), with the RBM of heis2d_10x10 in place of the GCNN.
    "j1j2_10x10": dict(N=100, alpha=2, ham=lambda: j1j2_square(10, 1.0, 0.5, True), rule="exchange",
                       chains=1024, per_chain=1, discard=16, seed=6, diag_shift=0.01, lr=0.02,
                       solver="cholesky_samplespace"),
}


# Sec. 9 (unitary dynamics): the quench of the periodic transverse-field
# Ising chain L = 20 to h = 1 with a complex RBM, alpha = 1, 4096 samples,
# the local rule and the Heun scheme; the truncated pseudo-inverse solves
# Eq. eq:tvmc (the default SVD-based solver of the time-evolution driver,
# eps = 0).  The paper starts from an optimised ground state; here the
# parameters are seeded: complex, real and imaginary parts N(0, sigma^2).
TDVP_WORKLOADS = {
    "tdvp_tfim1d_l20": dict(N=20, alpha=1, ham=lambda: tfim_chain(20, 1.0, 1.0), rule="local", chains=1024,
                            per_chain=4, discard=16, seed=8, sigma=0.05, dt=0.01, integrator="heun", real_time=True,
                            solver="svd", rcond=1e-12, diag_shift=0.0),
}


def complex_rbm_params(N: int, M: int, seed: int, sigma: float = 0.01) -> np.ndarray:
    """Complex RBM parameters [a (N); b (M); W (M x N)]: real parts, then
    imaginary parts, i.i.d. N(0, sigma^2) from default_rng(seed)."""
    rng = np.random.default_rng(seed)
    n = N + M + M * N
    re = rng.normal(0.0, sigma, n)
    im = rng.normal(0.0, sigma, n)
    return re + 1j * im


def serve_requests(n: int = 512, seed: int = 4) -> list:
    """Seeded serving mix (each request: local-energy expectation + one SR
    step): lattice uniform over the periodic Ising chains N in {16, 32, 64,
    128, 256} (J = h = 1) and the Marshall-signed Heisenberg squares L in
    {4, 6, 8, 12, 16}; alpha uniform in {1, 2, 4}; 1024 chains x U{1..16}
    samples; parameters seeded 40000 + r; dense Cholesky when Np <= 4096,
    else CG."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(n):
        lat = int(rng.integers(0, 10))
        alpha = int(rng.choice([1, 2, 4]))
        per_chain = int(rng.integers(1, 17))
        if lat < 5:
            N = [16, 32, 64, 128, 256][lat]
            ham, rule = tfim_chain(N, 1.0, 1.0), "local"
        else:
            L = [4, 6, 8, 12, 16][lat - 5]
            N = L * L
            ham, rule = heis_square(L, 1.0, True), "exchange"
        M = alpha * N
        Np = N + M + M * N
        out.append(dict(index=r, N=N, M=M, alpha=alpha, ham=ham, rule=rule, chains=1024, per_chain=per_chain,
                        seed=40000 + r, solver="cholesky" if Np <= 4096 else "cg"))
    return out


def poisson_arrivals(n: int, rate: float, seed: int = 4) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))
