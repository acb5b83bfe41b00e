"""Tensor-core (tcgen05) products and the NK_MIXED solves, through the C ABI.

nk_tc_gemm is compared with a plain FP64 product within the splitting bound
4 K (S + 3) 2^-8S max|a_i| max|b_j| (S slices per operand row), i.e. about
2^-50 K max|a| max|b| with 7 slices (FP64-level) and 2^-19 with 3 slices,
plus one rounding (2^-52) of the result for the accumulating modes.  The NK_MIXED SR
solves (tensor-core Cholesky, FP64-level products) must match the oracle's
dense FP64 solve within the same 1e-8 as the FP64 path.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2112_10526_gb300 import inputs as I
from paper_2112_10526_gb300 import nk

from gpu_util import cu, dev, vec_rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    with nk.Ctx() as c:
        yield c


# (rows, cols, k, mode, lower); mode 0 '=', 1 '-=', 2 '+='
GEMM_CASES = [(300, 130, 64, 0, False), (128, 64, 64, 0, False), (1, 1, 1, 0, False), (257, 65, 37, 1, False),
              (400, 400, 64, 1, True), (129, 200, 50, 2, True), (64, 300, 64, 0, False),
              # enough tiles per SM for strips of 2, 4 and 8 tiles, and more
              # than 32 tile rows (two rounds of the strip search)
              (2000, 2000, 64, 1, True), (4200, 640, 64, 2, False), (5000, 5000, 64, 1, True)]


@pytest.mark.parametrize("rows,cols,k,mode,lower", GEMM_CASES)
@pytest.mark.parametrize("slices,bits", [(7, 50), (3, 20)])
def test_tc_gemm_against_fp64(ctx, rows, cols, k, mode, lower, slices, bits):
    rng = np.random.default_rng(rows * 7 + cols)
    # rows of very different magnitudes exercise the per-row scaling
    A = rng.normal(size=(rows, k)) * np.exp2(rng.integers(-20, 20, size=(rows, 1)))
    B = rng.normal(size=(cols, k)) * np.exp2(rng.integers(-20, 20, size=(cols, 1)))
    C0 = rng.normal(size=(rows, cols))
    C = cu(C0.copy())
    nk.nk_tc_gemm(ctx, cu(A), cu(B), C, slices=slices, mode=mode, lower=lower)
    R = A @ B.T
    ref = {0: R, 1: C0 - R, 2: C0 + R}[mode]
    scale = np.abs(A) @ np.abs(B).T
    got = C.cpu().numpy()
    mask = np.tril(np.ones((rows, cols), dtype=bool)) if lower else np.ones((rows, cols), dtype=bool)
    # Splitting error: each operand row is 2^e (sum of S 8-bit slices + a
    # remainder below 2^-8S), 2^e <= 2 max|row|, and the dropped slice products
    # and remainders add up to at most (S + 3) 2^-8S per term, so
    # |err| <= 4 K (S + 3) 2^-8S max|a_i| max|b_j|; plus one rounding of the
    # result for the accumulating modes.
    amax = np.abs(A).max(axis=1)[:, None]
    bmax = np.abs(B).max(axis=1)[None, :]
    split = 4.0 * k * (slices + 3) * 2.0 ** (-8 * slices) * amax * bmax
    bound = split[mask] + 2.0 ** -52 * np.abs(ref[mask])
    assert (np.abs(got - ref)[mask] <= bound).all()
    # and, against sum |a b|, FP64-level with 7 slices
    assert (np.abs(got - ref)[mask] <= 2.0 ** -bits * scale[mask] * 64 + 2.0 ** -52 * np.abs(ref[mask])).all()
    if lower:  # entries above the diagonal are untouched
        np.testing.assert_array_equal(got[~mask], C0[~mask])


@pytest.mark.parametrize("solver", ["cholesky", "cholesky_samplespace"])
@pytest.mark.parametrize("N,M,Ns,eps", [(16, 16, 1024, 0.01), (10, 20, 100, 0.05), (6, 6, 700, 0.01),
                                        (12, 12, 130, 0.1), (36, 72, 300, 0.01)])
def test_mixed_sr_solve_matches_oracle(ctx, solver, N, M, Ns, eps):
    p = I.rbm_params(N, M, 4, 0.3)
    s = I.random_configs(Ns, N, 6)
    Np = N + M + M * N
    if solver == "cholesky" and Np > 4000:
        pytest.skip("dense parameter-space case kept small")
    O = oracle.jacobian(p, N, M, s)
    F = np.random.default_rng(2).normal(size=Np) * 0.1
    ref = oracle.solve_cholesky(oracle.qgt_dense(O), F, eps)
    d = torch.empty(Np, dtype=torch.float64, device=dev())
    nk.nk_sr_solve(ctx, cu(p), N, M, cu(s), cu(F), d, solver=solver, diag_shift=eps, precision="mixed")
    assert vec_rel_err(d.cpu().numpy(), ref) < 1e-8


@pytest.mark.parametrize("solver", ["cholesky_samplespace", "cholesky", "cg"])
def test_mixed_sr_step_against_oracle(ctx, solver):
    """One NK_MIXED step on the 4x4 Heisenberg lattice: E_loc per sample within
    1e-4 of the oracle on the GPU's own samples, and the update equal to the
    oracle's SR solution for the GPU's local energies within 1e-8 (Cholesky
    paths) or 1e-6 (CG on 4-slice tensor-core products, stopped at 1e-9)."""
    N, M, C, ns = 16, 32, 32, 8
    ham = I.heis_square(4)
    p0 = I.rbm_params(N, M, 2, 0.2)
    s0 = oracle.chain_init(N, C, "exchange", 2, 0)
    edges = cu(ham["edges"])
    h = nk.make_ham("heis", 1.0, 0.0, True, edges)
    pd, sd = cu(p0), cu(s0)
    ch = nk.make_chains(sd)
    cfg = nk.make_cfg("exchange", "mixed", solver, 4, ns, 0.01, 0.02, 2, cg_tol=1e-9, cg_maxiter=3000)
    stats = torch.empty(nk.SR_STATS_DOUBLES, dtype=torch.float64, device=dev())
    samples = torch.empty((C * ns, N), dtype=torch.int8, device=dev())
    eloc = torch.empty(C * ns, dtype=torch.float64, device=dev())
    nk.nk_sr_step(ctx, pd, N, M, h, ch, cfg, stats, samples, eloc)
    st = nk.sr_stats_dict(stats)
    assert st["solver_status"] == 0
    sm = samples.cpu().numpy()
    e = eloc.cpu().numpy()
    ref_e = oracle.local_energy(p0, N, M, ham, sm)
    assert np.max(np.abs(e - ref_e) / np.maximum(np.abs(ref_e), np.sqrt(np.mean(ref_e ** 2)))) < 1e-4
    O = oracle.jacobian(p0, N, M, sm)
    F = oracle.force(O, e)
    delta = oracle.solve_cholesky(oracle.qgt_dense(O), F, 0.01)
    got = (p0 - pd.cpu().numpy()) / 0.02
    assert vec_rel_err(got, delta) < (1e-6 if solver == "cg" else 1e-8)
    assert nk.nk_ctx_error(ctx) == 0


PROD_CASES = [(16, 16, 1024, 0.3), (100, 200, 300, 0.01), (37, 45, 131, 0.4), (400, 1600, 200, 0.01),
              (3, 2, 1, 0.5)]


@pytest.mark.parametrize("N,M,Ns,sig", PROD_CASES)
def test_mixed_jacobian_products(ctx, N, M, Ns, sig):
    """NK_MIXED J v, J^T g and the on-the-fly QGT run on the tensor cores with
    4 slices per operand row (relative error about 2^-32 of the row maximum:
    1e-8 in norm here), the force with 7 slices (1e-12)."""
    p = I.rbm_params(N, M, 5, sig)
    s = I.random_configs(Ns, N, 9)
    Np = N + M + M * N
    O = oracle.jacobian(p, N, M, s)
    pd, sd = cu(p), cu(s)
    rng = np.random.default_rng(1)
    g = rng.normal(size=Ns)
    out = torch.empty(Np, dtype=torch.float64, device=dev())
    nk.nk_vjp(ctx, pd, N, M, sd, cu(g), out, precision="mixed")
    assert vec_rel_err(out.cpu().numpy(), O.T @ g) < 1e-8
    v = rng.normal(size=Np)
    w = torch.empty(Ns, dtype=torch.float64, device=dev())
    nk.nk_jvp(ctx, pd, N, M, sd, cu(v), w, precision="mixed")
    assert vec_rel_err(w.cpu().numpy(), O @ v) < 1e-8
    e = rng.normal(-5, 1, size=Ns)
    F = torch.empty(Np, dtype=torch.float64, device=dev())
    nk.nk_force(ctx, pd, N, M, sd, cu(e), F, precision="mixed")
    assert vec_rel_err(F.cpu().numpy(), oracle.force(O, e)) < 1e-12
    q = torch.empty(Np, dtype=torch.float64, device=dev())
    nk.nk_qgt_matvec(ctx, cu(v), q, 0.01, params=pd, N=N, M=M, s=sd, precision="mixed")
    assert vec_rel_err(q.cpu().numpy(), oracle.qgt_matvec_onthefly(O, v, 0.01)) < 1e-8
    assert nk.nk_ctx_error(ctx) == 0


@pytest.mark.parametrize("N,M,Ns,eps", [(16, 16, 1024, 0.01), (36, 72, 300, 0.01), (100, 200, 512, 0.02)])
def test_mixed_cg_solve(ctx, N, M, Ns, eps):
    p = I.rbm_params(N, M, 4, 0.3)
    s = I.random_configs(Ns, N, 6)
    Np = N + M + M * N
    O = oracle.jacobian(p, N, M, s)
    F = np.random.default_rng(2).normal(size=Np) * 0.1
    ref, _, _ = oracle.solve_cg(lambda x: oracle.qgt_matvec_onthefly(O, x, eps), F, tol=1e-12, maxiter=5000)
    d = torch.empty(Np, dtype=torch.float64, device=dev())
    info = nk.nk_sr_solve(ctx, cu(p), N, M, cu(s), cu(F), d, solver="cg", diag_shift=eps, cg_tol=1e-9,
                          cg_maxiter=5000, precision="mixed")
    assert info["converged"]
    assert vec_rel_err(d.cpu().numpy(), ref) < 1e-6


def test_samplespace_solve_full_size(ctx):
    """The sample-space solve at the size the 10 x 10 Heisenberg step runs it
    (Ns = 8192, N = 100, M = 200, Np = 20300, eps = 0.01), NK_MIXED against
    NK_F64 on the GPU and both against the SR system itself, applied with the
    oracle's FP64 Jacobian: ||(S + eps I) delta - F|| / ||F||."""
    N, M, Ns, eps = 100, 200, 8192, 0.01
    p = I.rbm_params(N, M, 2, 0.05)
    s = I.random_configs(Ns, N, 12, sz0=True)
    Np = N + M + M * N
    F = np.random.default_rng(5).normal(size=Np) * 0.1
    out = {}
    for prec in ("f64", "mixed"):
        d = torch.empty(Np, dtype=torch.float64, device=dev())
        nk.nk_sr_solve(ctx, cu(p), N, M, cu(s), cu(F), d, solver="cholesky_samplespace", diag_shift=eps,
                       precision=prec)
        out[prec] = d.cpu().numpy()
    assert nk.nk_ctx_error(ctx) == 0
    O = oracle.jacobian(p, N, M, s)
    res = {k: np.linalg.norm(oracle.qgt_matvec_onthefly(O, v, eps) - F) / np.linalg.norm(F) for k, v in out.items()}
    assert res["f64"] < 1e-9, res
    assert res["mixed"] < 1e-9, res
    assert vec_rel_err(out["mixed"], out["f64"]) < 1e-8


def test_prof_trace_orders_the_bracketed_segments(ctx):
    """nk_prof_trace: every bracketed launch of an NK_MIXED sample-space solve,
    in enqueue order, with start <= end on one clock from the first start;
    the Cholesky's classes are there and the trace agrees with nk_prof_read."""
    N, M, Ns = 16, 16, 1024
    p = I.rbm_params(N, M, 4, 0.3)
    s = I.random_configs(Ns, N, 6)
    Np = N + M + M * N
    F = np.random.default_rng(2).normal(size=Np) * 0.1
    d = torch.empty(Np, dtype=torch.float64, device=dev())
    nk.nk_prof_enable(True)
    try:
        nk.nk_sr_solve(ctx, cu(p), N, M, cu(s), cu(F), d, solver="cholesky_samplespace", diag_shift=0.01,
                       precision="mixed")
        torch.cuda.synchronize()
        tr = nk.nk_prof_trace()
        per_class = {c: nk.nk_prof_read(c) for c in nk.PROF_CLASSES}
    finally:
        nk.nk_prof_enable(False)
    assert tr and tr[0][1] == 0.0
    assert all(0.0 <= t0 <= t1 for _, t0, t1 in tr)
    names = {c for c, _, _ in tr}
    assert {"gram", "chol_update", "chol_panel", "trsv"} <= names
    for c, (ms, n, _) in per_class.items():
        seg = [(t0, t1) for k, t0, t1 in tr if k == c]
        assert n == len(seg)
        assert ms == pytest.approx(sum(t1 - t0 for t0, t1 in seg), rel=1e-3, abs=1e-3)
    # a NULL count pointer and a short buffer are argument errors / truncation
    import ctypes
    assert nk.lib().nk_prof_trace(0, None, None, None, None) == -1
    assert nk.lib().nk_prof_trace(1, None, None, None, ctypes.byref(ctypes.c_int32())) == -1


def _oracle_jv(p, N, M, s, v, chunk):
    """J v from the oracle's Jacobian rows (Eq. eq:log-derivative-O), a
    chunk of samples at a time so that the rows fit in memory."""
    return np.concatenate([oracle.jacobian(p, N, M, s[k:k + chunk]) @ v for k in range(0, s.shape[0], chunk)])


def _sampled_params(rng, N, M, n_a, n_b, n_w):
    return np.concatenate([rng.choice(N, n_a, replace=False), N + rng.choice(M, n_b, replace=False),
                           N + M + rng.choice(M * N, n_w, replace=False)])


def test_mixed_jacobian_products_full_size_sampled(ctx):
    """NK_MIXED J v and J^T g at the 20 x 20 TFIM workload's full size (Ns =
    16384, N = 400, M = 1600, Np = 642 000), checked on sampled outputs the
    oracle computes: 64 entries of J v from the oracle's Jacobian rows of
    their samples, and 64 parameters of J^T g (a, b and W entries) from the
    oracle's Jacobian columns of those parameters over all samples."""
    N, M, Ns = 400, 1600, 16384
    p = I.rbm_params(N, M, 3)
    s = I.random_configs(Ns, N, 3)
    Np = N + M + M * N
    rng = np.random.default_rng(7)
    pd, sd = cu(p), cu(s)
    v = rng.normal(size=Np)
    w = torch.empty(Ns, dtype=torch.float64, device=dev())
    nk.nk_jvp(ctx, pd, N, M, sd, cu(v), w, precision="mixed")
    rows = rng.choice(Ns, 64, replace=False)
    ref_w = oracle.jacobian(p, N, M, s[rows]) @ v
    assert vec_rel_err(w.cpu().numpy()[rows], ref_w) < 1e-8
    g = rng.normal(size=Ns)
    out = torch.empty(Np, dtype=torch.float64, device=dev())
    nk.nk_vjp(ctx, pd, N, M, sd, cu(g), out, precision="mixed")
    idx = _sampled_params(rng, N, M, 8, 8, 48)
    ref = oracle.jacobian_cols(p, N, M, s, idx).T @ g
    assert vec_rel_err(out.cpu().numpy()[idx], ref) < 1e-8
    assert nk.nk_ctx_error(ctx) == 0


def test_mixed_jacobian_products_24x24_full_size_sampled(ctx):
    """NK_MIXED J v and J^T g at the 24 x 24 Heisenberg workload's full size
    (Ns = 65536, N = 576, M = 4608, Np = 2 659 392), on sampled outputs the
    oracle computes: (J v)_k for 48 samples k from the oracle's Jacobian rows,
    and (J^T g)_q for 48 parameters q (8 hidden units, with their b and four
    W entries each, and 8 visible biases) from the oracle's Jacobian columns
    over all samples."""
    N, M, Ns = 576, 4608, 65536
    p = I.rbm_params(N, M, 5)
    s = I.random_configs(Ns, N, 5, sz0=True)
    Np = N + M + M * N
    rng = np.random.default_rng(11)
    pd, sd = cu(p), cu(s)
    v = rng.normal(size=Np)
    w = torch.empty(Ns, dtype=torch.float64, device=dev())
    nk.nk_jvp(ctx, pd, N, M, sd, cu(v), w, precision="mixed")
    rows = rng.choice(Ns, 48, replace=False)
    ref_w = _oracle_jv(p, N, M, s[rows], v, 8)
    assert vec_rel_err(w.cpu().numpy()[rows], ref_w) < 1e-8
    g = rng.normal(size=Ns)
    out = torch.empty(Np, dtype=torch.float64, device=dev())
    nk.nk_vjp(ctx, pd, N, M, sd, cu(g), out, precision="mixed")
    units = rng.choice(M, 8, replace=False)
    idx = [int(i) for i in rng.choice(N, 8, replace=False)] + [N + int(j) for j in units]
    idx += [N + M + int(j) * N + int(i) for j in units for i in rng.choice(N, 4, replace=False)]
    ref = oracle.jacobian_cols(p, N, M, s, idx).T @ g
    assert vec_rel_err(out.cpu().numpy()[idx], ref) < 1e-8
    assert nk.nk_ctx_error(ctx) == 0


@pytest.mark.parametrize("tol,bound", [(1e-9, 1e-8), (1e-6, 5e-6)])
def test_mixed_cg_solve_full_size_sampled_residual(ctx, tol, bound):
    """The NK_MIXED CG solve of (S + eps I) delta = F at the 20 x 20 TFIM
    workload's full size (Ns = 16384, Np = 642 000, on-the-fly QGT), checked
    by the residual on 64 sampled components, with the QGT product of App.
    B.3 taken through the oracle's Jacobian: w = J delta over all samples from
    its rows, Delta w centred, then (S delta)_q = (1/Ns) sum_k O_kq Delta w_k
    from its columns of the sampled q, at the two CG tolerances of the tests
    and of the bench (the 4-slice products carry about 2^-32)."""
    N, M, Ns, eps = 400, 1600, 16384, 0.01
    p = I.rbm_params(N, M, 3)
    s = I.random_configs(Ns, N, 3)
    Np = N + M + M * N
    rng = np.random.default_rng(13)
    F = rng.normal(size=Np) * 0.1
    d = torch.empty(Np, dtype=torch.float64, device=dev())
    info = nk.nk_sr_solve(ctx, cu(p), N, M, cu(s), cu(F), d, solver="cg", diag_shift=eps, cg_tol=tol,
                          cg_maxiter=3000, precision="mixed")
    assert info["converged"]
    delta = d.cpu().numpy()
    w = _oracle_jv(p, N, M, s, delta, 256)
    dw = w - w.mean()
    idx = _sampled_params(rng, N, M, 8, 8, 48)
    r = oracle.jacobian_cols(p, N, M, s, idx).T @ dw / Ns + eps * delta[idx] - F[idx]
    assert np.abs(r).max() <= bound * np.linalg.norm(F)
