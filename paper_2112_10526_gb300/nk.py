"""Thin ctypes binding of libnk.so (include/nk.h): argument marshalling only.

Every function here has the name of the C entry point it calls and takes
torch CUDA tensors for the device arrays; all arithmetic runs in the CUDA
library.  There is no fallback: if libnk.so is missing or fails to load,
``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnk.so")

NK_OK = 0
NK_ERR_INVALID_ARG = -1
NK_ERR_CUDA = -2
NK_ERR_OOM = -3
NK_ERR_TIMEOUT = -4
NK_ERR_NOT_CONVERGED = -5
NK_ERR_UNIMPLEMENTED = -6

NK_F64, NK_MIXED = 0, 1
NK_RULE_LOCAL, NK_RULE_EXCHANGE, NK_RULE_HAMILTONIAN = 0, 1, 2
NK_TFIM, NK_HEIS = 0, 1
NK_SOLVER_CHOLESKY, NK_SOLVER_CHOLESKY_SAMPLESPACE, NK_SOLVER_CG = 0, 1, 2
NK_SOLVER_SVD, NK_SOLVER_SVD_SAMPLESPACE = 3, 4
NK_QGT_ONTHEFLY, NK_QGT_JACOBIAN = 0, 1

PRECISION = {"f64": NK_F64, "mixed": NK_MIXED}
RULE = {"local": NK_RULE_LOCAL, "exchange": NK_RULE_EXCHANGE, "hamiltonian": NK_RULE_HAMILTONIAN}
KIND = {"tfim": NK_TFIM, "heis": NK_HEIS}
SOLVER = {"cholesky": NK_SOLVER_CHOLESKY, "cholesky_samplespace": NK_SOLVER_CHOLESKY_SAMPLESPACE,
          "cg": NK_SOLVER_CG, "svd": NK_SOLVER_SVD, "svd_samplespace": NK_SOLVER_SVD_SAMPLESPACE}


class NkError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libnk error {code}: {msg}")
        self.code = code


class nk_rbm(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("M", ctypes.c_int32), ("params", ctypes.c_void_p)]


class nk_ham(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("J", ctypes.c_double), ("h", ctypes.c_double),
                ("marshall", ctypes.c_int32), ("n_edges", ctypes.c_int32), ("edges", ctypes.c_void_p),
                ("J2", ctypes.c_double), ("n_edges2", ctypes.c_int32)]


class nk_qgt(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("rbm", ctypes.POINTER(nk_rbm)), ("precision", ctypes.c_int32),
                ("s", ctypes.c_void_p), ("dJ", ctypes.c_void_p), ("Ns", ctypes.c_int64),
                ("Np", ctypes.c_int32)]


class nk_rbm_symm(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("alpha", ctypes.c_int32), ("n_group", ctypes.c_int32),
                ("perms", ctypes.c_void_p), ("params", ctypes.c_void_p)]


class nk_crbm(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("M", ctypes.c_int32), ("params", ctypes.c_void_p)]


class nk_tdvp_cfg(ctypes.Structure):
    _fields_ = [("rule", ctypes.c_int32), ("integrator", ctypes.c_int32), ("real_time", ctypes.c_int32),
                ("solver", ctypes.c_int32), ("n_discard", ctypes.c_int32), ("n_samples", ctypes.c_int32),
                ("dt", ctypes.c_double), ("diag_shift", ctypes.c_double), ("rcond", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("stream_id", ctypes.c_uint32)]


NK_TDVP_EULER, NK_TDVP_HEUN = 1, 2
TDVP_STATS_FIELDS = ["energy_re", "energy_im", "variance", "error"]


class nk_chains(ctypes.Structure):
    _fields_ = [("C", ctypes.c_int32), ("s", ctypes.c_void_p), ("sweeps_done", ctypes.c_int64),
                ("n_accepted", ctypes.c_void_p)]


class nk_sr_cfg(ctypes.Structure):
    _fields_ = [("rule", ctypes.c_int32), ("precision", ctypes.c_int32), ("solver", ctypes.c_int32),
                ("n_discard", ctypes.c_int32), ("n_samples", ctypes.c_int32),
                ("cg_maxiter", ctypes.c_int32), ("diag_shift", ctypes.c_double), ("lr", ctypes.c_double),
                ("cg_tol", ctypes.c_double), ("seed", ctypes.c_uint64), ("stream_id", ctypes.c_uint32),
                ("svd_rcond", ctypes.c_double)]


NK_REQ_EXPECT, NK_REQ_SR_STEP = 0, 1


class nk_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("N", ctypes.c_int32), ("M", ctypes.c_int32),
                ("params", ctypes.c_void_p), ("ham_kind", ctypes.c_int32), ("J", ctypes.c_double),
                ("h", ctypes.c_double), ("marshall", ctypes.c_int32), ("n_edges", ctypes.c_int32),
                ("edges", ctypes.c_void_p), ("n_chains", ctypes.c_int32), ("cfg", nk_sr_cfg),
                ("J2", ctypes.c_double), ("n_edges2", ctypes.c_int32)]


class nk_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("slot", ctypes.c_int32), ("energy", ctypes.c_double),
                ("variance", ctypes.c_double), ("error", ctypes.c_double), ("acceptance", ctypes.c_double),
                ("cg_iters", ctypes.c_double), ("solver_status", ctypes.c_double), ("queue_ms", ctypes.c_double),
                ("run_ms", ctypes.c_double), ("latency_ms", ctypes.c_double), ("device_bytes", ctypes.c_size_t),
                ("message", ctypes.c_char * 128)]


class nk_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("inflight", ctypes.c_int64), ("queued", ctypes.c_int64), ("hbm_in_use", ctypes.c_size_t),
                ("hbm_budget", ctypes.c_size_t), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double)]


SR_STATS_FIELDS = ["energy", "variance", "error", "acceptance", "cg_iters", "cg_residual", "f_norm",
                   "delta_norm", "solver_status"]
SR_STATS_DOUBLES = len(SR_STATS_FIELDS)

_lib = None


def lib():
    """Load libnk.so (raises if it is missing: there is no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing; build it with "
                           "`python -m paper_2112_10526_gb300.build`")
    L = ctypes.CDLL(LIB_PATH)
    P, i32, i64, u64, u32, f64 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                  ctypes.c_uint32, ctypes.c_double)
    sig = {
        "nk_ctx_create": [i32, ctypes.POINTER(P)],
        "nk_ctx_destroy": [P],
        "nk_rbm_logpsi": [P, ctypes.POINTER(nk_rbm), i32, P, i64, P, P],
        "nk_chains_init": [P, i32, i32, i32, u64, u32, P, P],
        "nk_metropolis_sweep": [P, ctypes.POINTER(nk_rbm), i32, i32, i32, P, i32, P, i64, i32, i32, u64,
                                u32, P, P, P, P, P],
        "nk_local_energy": [P, ctypes.POINTER(nk_rbm), i32, ctypes.POINTER(nk_ham), P, i64, P, P, P],
        "nk_local_energy_noalloc": [ctypes.POINTER(nk_rbm), i32, ctypes.POINTER(nk_ham), P, i64, P, P, P],
        "nk_stats": [P, P, i64, i32, P, P],
        "nk_jacobian": [P, ctypes.POINTER(nk_rbm), i32, P, i64, i32, i64, i64, P, P],
        "nk_vjp": [P, ctypes.POINTER(nk_rbm), i32, P, i64, P, P, P],
        "nk_jvp": [P, ctypes.POINTER(nk_rbm), i32, P, i64, P, P, P],
        "nk_force": [P, ctypes.POINTER(nk_rbm), i32, P, i64, P, P, P],
        "nk_qgt_matvec": [P, ctypes.POINTER(nk_qgt), f64, P, P, P],
        "nk_ctx_error": [P, ctypes.POINTER(ctypes.c_int32), P],
        "nk_server_create": [i32, ctypes.c_size_t, i32, ctypes.POINTER(P)],
        "nk_server_submit": [P, ctypes.POINTER(nk_request), P, ctypes.POINTER(ctypes.c_uint64)],
        "nk_server_poll": [P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(nk_result)],
        "nk_server_wait": [P, ctypes.c_uint64, ctypes.POINTER(nk_result)],
        "nk_server_stats_get": [P, ctypes.POINTER(nk_server_stats)],
        "nk_server_destroy": [P],
        "nk_tc_gemm": [P, i64, i64, i32, P, i64, P, i64, i32, i32, i32, P, i64, P],
        "nk_sr_solve": [P, ctypes.POINTER(nk_rbm), i32, P, i64, P, i32, f64, f64, i32, P,
                        ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double), P],
        "nk_sr_step": [P, ctypes.POINTER(nk_rbm), ctypes.POINTER(nk_ham), ctypes.POINTER(nk_chains),
                       ctypes.POINTER(nk_sr_cfg), P, P, P, P],
        "nk_symm_expand": [P, ctypes.POINTER(nk_rbm_symm), P, P],
        "nk_crbm_logpsi": [P, ctypes.POINTER(nk_crbm), P, i64, P, P],
        "nk_crbm_metropolis": [P, ctypes.POINTER(nk_crbm), i32, i32, P, i32, P, i64, i32, i32, u64, u32, P, P, P],
        "nk_crbm_local_energy": [P, ctypes.POINTER(nk_crbm), ctypes.POINTER(nk_ham), P, i64, P, P],
        "nk_crbm_jacobian": [P, ctypes.POINTER(nk_crbm), P, i64, P, P],
        "nk_tdvp_step": [P, ctypes.POINTER(nk_crbm), ctypes.POINTER(nk_ham), ctypes.POINTER(nk_chains),
                         ctypes.POINTER(nk_tdvp_cfg), P, P, P],
        "nk_symm_jacobian": [P, ctypes.POINTER(nk_rbm_symm), i32, P, i64, P, P],
        "nk_symm_sr_step": [P, ctypes.POINTER(nk_rbm_symm), ctypes.POINTER(nk_ham), ctypes.POINTER(nk_chains),
                            ctypes.POINTER(nk_sr_cfg), P, P, P, P],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int32
    L.nk_last_error.argtypes = []
    L.nk_last_error.restype = ctypes.c_char_p
    L.nk_version.argtypes = []
    L.nk_version.restype = ctypes.c_int32
    L.nk_prof_enable.argtypes = [i32]
    L.nk_prof_enable.restype = ctypes.c_int32
    L.nk_prof_read.argtypes = [i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                               ctypes.POINTER(ctypes.c_double)]
    L.nk_prof_read.restype = ctypes.c_int32
    L.nk_prof_read_executed.argtypes = [i32, ctypes.POINTER(ctypes.c_double)]
    L.nk_prof_read_executed.restype = ctypes.c_int32
    L.nk_prof_trace.argtypes = [i32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)]
    L.nk_prof_trace.restype = ctypes.c_int32
    L.nk_launch_count.argtypes = []
    L.nk_launch_count.restype = ctypes.c_int64
    L.nk_request_bytes.argtypes = [ctypes.POINTER(nk_request)]
    L.nk_request_bytes.restype = ctypes.c_size_t
    _lib = L
    return L


def _check(code, allow=()):
    if code != NK_OK and code not in allow:
        raise NkError(code, lib().nk_last_error().decode())
    return code


def _ptr(t):
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _prec(p):
    return PRECISION[p] if isinstance(p, str) else int(p)


class Ctx:
    """Owns one nk_ctx (device workspace); close() or use as a context manager."""

    def __init__(self, device=None):
        dev = torch.cuda.current_device() if device is None else int(device)
        h = ctypes.c_void_p()
        _check(lib().nk_ctx_create(dev, ctypes.byref(h)))
        self.handle = h
        self.device = dev

    def close(self):
        if self.handle:
            lib().nk_ctx_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_rbm(params, N, M):
    assert params.dtype == torch.float64 and params.is_cuda and params.numel() == N + M + M * N
    return nk_rbm(N, M, params.data_ptr())


def make_ham(kind, J, h, marshall, edges, J2=0.0, n_edges2=0):
    """edges: device int32 [E, 2], the last n_edges2 of them next-nearest
    neighbours with coupling J2."""
    assert edges.dtype == torch.int32 and edges.is_cuda
    e = edges.reshape(-1, 2)
    return nk_ham(KIND[kind] if isinstance(kind, str) else int(kind), float(J), float(h), int(bool(marshall)),
                  int(e.shape[0]), e.data_ptr(), float(J2), int(n_edges2))


# ------------------------------------------------------------ entry points --

def nk_rbm_logpsi(ctx, params, N, M, s, out, precision="f64", stream=None):
    r = make_rbm(params, N, M)
    _check(lib().nk_rbm_logpsi(ctx.handle, ctypes.byref(r), _prec(precision), _ptr(s), s.shape[0],
                               _ptr(out), _stream(stream)))
    return out


def nk_chains_init(ctx, N, C, rule, seed, stream_id, s_out, stream=None):
    _check(lib().nk_chains_init(ctx.handle, N, C, RULE[rule] if isinstance(rule, str) else rule, seed,
                                stream_id, _ptr(s_out), _stream(stream)))
    return s_out


def nk_metropolis_sweep(ctx, params, N, M, rule, edges, s, sweep0, n_discard, n_samples, seed,
                        stream_id, samples_out, logpsi_out=None, n_accepted=None, decisions_out=None,
                        precision="f64", stream=None):
    r = make_rbm(params, N, M)
    ne = 0 if edges is None else int(edges.reshape(-1, 2).shape[0])
    _check(lib().nk_metropolis_sweep(ctx.handle, ctypes.byref(r), _prec(precision),
                                     RULE[rule] if isinstance(rule, str) else rule, ne, _ptr(edges),
                                     s.shape[0], _ptr(s), sweep0, n_discard, n_samples, seed, stream_id,
                                     _ptr(samples_out), _ptr(logpsi_out), _ptr(n_accepted),
                                     _ptr(decisions_out), _stream(stream)))
    return samples_out


def nk_local_energy(ctx, params, N, M, ham, s, eloc_out, t_out=None, precision="f64", stream=None):
    r = make_rbm(params, N, M)
    _check(lib().nk_local_energy(ctx.handle, ctypes.byref(r), _prec(precision), ctypes.byref(ham),
                                 _ptr(s), s.shape[0], _ptr(eloc_out), _ptr(t_out), _stream(stream)))
    return eloc_out


def nk_local_energy_noalloc(params, N, M, ham, s, eloc_out, t_out=None, precision="f64", stream=None):
    """nk_local_energy without a context or any device allocation (fixed
    library scratch; see include/nk.h)."""
    r = make_rbm(params, N, M)
    _check(lib().nk_local_energy_noalloc(ctypes.byref(r), _prec(precision), ctypes.byref(ham), _ptr(s),
                                         s.shape[0], _ptr(eloc_out), _ptr(t_out), _stream(stream)))
    return eloc_out


def nk_stats(ctx, eloc, n_chains, out, stream=None):
    _check(lib().nk_stats(ctx.handle, _ptr(eloc), eloc.numel(), n_chains, _ptr(out), _stream(stream)))
    return out


def nk_jacobian(ctx, params, N, M, s, centered, row0, rows, O_out, precision="f64", stream=None):
    r = make_rbm(params, N, M)
    _check(lib().nk_jacobian(ctx.handle, ctypes.byref(r), _prec(precision), _ptr(s), s.shape[0],
                             int(bool(centered)), row0, rows, _ptr(O_out), _stream(stream)))
    return O_out


def nk_vjp(ctx, params, N, M, s, g, out, precision="f64", stream=None):
    r = make_rbm(params, N, M)
    _check(lib().nk_vjp(ctx.handle, ctypes.byref(r), _prec(precision), _ptr(s), s.shape[0], _ptr(g),
                        _ptr(out), _stream(stream)))
    return out


def nk_jvp(ctx, params, N, M, s, v, out, precision="f64", stream=None):
    r = make_rbm(params, N, M)
    _check(lib().nk_jvp(ctx.handle, ctypes.byref(r), _prec(precision), _ptr(s), s.shape[0], _ptr(v),
                        _ptr(out), _stream(stream)))
    return out


def nk_force(ctx, params, N, M, s, eloc, F_out, precision="f64", stream=None):
    r = make_rbm(params, N, M)
    _check(lib().nk_force(ctx.handle, ctypes.byref(r), _prec(precision), _ptr(s), s.shape[0],
                          _ptr(eloc), _ptr(F_out), _stream(stream)))
    return F_out


def nk_qgt_matvec(ctx, v, out, diag_shift, params=None, N=None, M=None, s=None, dJ=None,
                  precision="f64", stream=None):
    """On-the-fly QGT when `s` is given, stored centred Jacobian when `dJ` is."""
    if dJ is not None:
        q = nk_qgt(NK_QGT_JACOBIAN, None, 0, None, dJ.data_ptr(), dJ.shape[0], dJ.shape[1])
        _check(lib().nk_qgt_matvec(ctx.handle, ctypes.byref(q), float(diag_shift), _ptr(v), _ptr(out),
                                   _stream(stream)))
        return out
    r = make_rbm(params, N, M)
    q = nk_qgt(NK_QGT_ONTHEFLY, ctypes.pointer(r), _prec(precision), s.data_ptr(), None, s.shape[0], 0)
    _check(lib().nk_qgt_matvec(ctx.handle, ctypes.byref(q), float(diag_shift), _ptr(v), _ptr(out),
                               _stream(stream)))
    return out


def nk_ctx_error(ctx, stream=None):
    """Sticky tensor-core time-out code of the context (0 = none); resets it."""
    code = ctypes.c_int32()
    _check(lib().nk_ctx_error(ctx.handle, ctypes.byref(code), _stream(stream)))
    return int(code.value)


def nk_tc_gemm(ctx, A, B, C, slices=7, mode=0, lower=False, stream=None):
    """C (mode 0 '=', 1 '-=', 2 '+=') A @ B.T on the tensor cores, FP64-accurate at 7 slices."""
    rows, k = A.shape
    cols = B.shape[0]
    _check(lib().nk_tc_gemm(ctx.handle, rows, cols, k, _ptr(A), A.stride(0), _ptr(B), B.stride(0), slices, mode,
                            int(bool(lower)), _ptr(C), C.stride(0), _stream(stream)))
    return C


def nk_sr_solve(ctx, params, N, M, s, F, delta_out, solver="cg", diag_shift=0.01, cg_tol=1e-10,
                cg_maxiter=1000, precision="f64", stream=None):
    r = make_rbm(params, N, M)
    info = (ctypes.c_int32 * 2)()
    res = ctypes.c_double()
    code = lib().nk_sr_solve(ctx.handle, ctypes.byref(r), _prec(precision), _ptr(s), s.shape[0], _ptr(F),
                             SOLVER[solver] if isinstance(solver, str) else solver, float(diag_shift),
                             float(cg_tol), int(cg_maxiter), _ptr(delta_out), info, ctypes.byref(res),
                             _stream(stream))
    _check(code, allow=(NK_ERR_NOT_CONVERGED,))
    return {"iters": int(info[0]), "converged": bool(info[1]), "residual": res.value, "code": code}


def nk_sr_step(ctx, params, N, M, ham, chains, cfg, stats_out=None, samples_out=None, eloc_out=None,
               stream=None):
    """`chains` is an nk_chains structure (its sweeps_done advances); `cfg` an nk_sr_cfg."""
    r = make_rbm(params, N, M)
    code = lib().nk_sr_step(ctx.handle, ctypes.byref(r), ctypes.byref(ham), ctypes.byref(chains),
                            ctypes.byref(cfg), _ptr(stats_out), _ptr(samples_out), _ptr(eloc_out),
                            _stream(stream))
    _check(code, allow=(NK_ERR_NOT_CONVERGED,))
    return code


def make_symm(params, N, alpha, perms):
    """nk_rbm_symm over device tensors: params float64 [1 + alpha + alpha N],
    perms int32 [|G|, N]."""
    assert perms.dtype == torch.int32 and perms.is_contiguous() and perms.shape[1] == N
    assert params.dtype == torch.float64 and params.numel() == 1 + alpha + alpha * N
    return nk_rbm_symm(N, alpha, perms.shape[0], perms.data_ptr(), params.data_ptr())


def nk_symm_expand(ctx, params, N, alpha, perms, plain_out, stream=None):
    m = make_symm(params, N, alpha, perms)
    _check(lib().nk_symm_expand(ctx.handle, ctypes.byref(m), _ptr(plain_out), _stream(stream)))
    return plain_out


def nk_symm_jacobian(ctx, params, N, alpha, perms, s, O_out, precision="f64", stream=None):
    m = make_symm(params, N, alpha, perms)
    _check(lib().nk_symm_jacobian(ctx.handle, ctypes.byref(m), _prec(precision), _ptr(s), s.shape[0], _ptr(O_out),
                                  _stream(stream)))
    return O_out


def nk_symm_sr_step(ctx, params, N, alpha, perms, ham, chains, cfg, stats_out=None, samples_out=None,
                    eloc_out=None, stream=None):
    """One SR step of the symmetric RBM; params (device float64) updated in place."""
    m = make_symm(params, N, alpha, perms)
    _check(lib().nk_symm_sr_step(ctx.handle, ctypes.byref(m), ctypes.byref(ham), ctypes.byref(chains),
                                 ctypes.byref(cfg), _ptr(stats_out), _ptr(samples_out), _ptr(eloc_out),
                                 _stream(stream)))


def make_crbm(params, N, M):
    """nk_crbm over a device complex128 tensor [N + M + M N]."""
    assert params.dtype == torch.complex128 and params.is_cuda and params.numel() == N + M + M * N
    return nk_crbm(N, M, params.data_ptr())


def nk_crbm_logpsi(ctx, params, N, M, s, out, stream=None):
    r = make_crbm(params, N, M)
    _check(lib().nk_crbm_logpsi(ctx.handle, ctypes.byref(r), _ptr(s), s.shape[0], _ptr(out), _stream(stream)))
    return out


def nk_crbm_metropolis(ctx, params, N, M, rule, edges, s, sweep0, n_discard, n_samples, seed, stream_id, samples_out,
                       n_accepted=None, stream=None):
    r = make_crbm(params, N, M)
    ne = 0 if edges is None else edges.shape[0]
    _check(lib().nk_crbm_metropolis(ctx.handle, ctypes.byref(r), RULE[rule] if isinstance(rule, str) else rule, ne,
                                    _ptr(edges), s.shape[0], _ptr(s), int(sweep0), int(n_discard), int(n_samples),
                                    int(seed), int(stream_id), _ptr(samples_out), _ptr(n_accepted), _stream(stream)))
    return samples_out


def nk_crbm_local_energy(ctx, params, N, M, ham, s, out, stream=None):
    r = make_crbm(params, N, M)
    _check(lib().nk_crbm_local_energy(ctx.handle, ctypes.byref(r), ctypes.byref(ham), _ptr(s), s.shape[0], _ptr(out),
                                      _stream(stream)))
    return out


def nk_crbm_jacobian(ctx, params, N, M, s, O_out, stream=None):
    r = make_crbm(params, N, M)
    _check(lib().nk_crbm_jacobian(ctx.handle, ctypes.byref(r), _ptr(s), s.shape[0], _ptr(O_out), _stream(stream)))
    return O_out


def make_tdvp_cfg(rule, integrator, real_time, solver, n_discard, n_samples, dt, diag_shift, seed, stream_id=0,
                  rcond=0.0):
    return nk_tdvp_cfg(RULE[rule] if isinstance(rule, str) else rule,
                       {"euler": NK_TDVP_EULER, "heun": NK_TDVP_HEUN}.get(integrator, integrator), int(bool(real_time)),
                       SOLVER[solver] if isinstance(solver, str) else solver, int(n_discard), int(n_samples),
                       float(dt), float(diag_shift), float(rcond), int(seed), int(stream_id))


def nk_tdvp_step(ctx, params, N, M, ham, chains, cfg, stats_out=None, theta_dot_out=None, stream=None):
    """One t-VMC step of the complex RBM; params (device complex128) updated in place."""
    r = make_crbm(params, N, M)
    _check(lib().nk_tdvp_step(ctx.handle, ctypes.byref(r), ctypes.byref(ham), ctypes.byref(chains), ctypes.byref(cfg),
                              _ptr(stats_out), _ptr(theta_dot_out), _stream(stream)))


def sr_stats_dict(t):
    """Read an nk_sr_stats device buffer (float64 [8]) into a dict."""
    v = t.detach().cpu().tolist()
    return dict(zip(SR_STATS_FIELDS, v))


def make_cfg(rule, precision, solver, n_discard, n_samples, diag_shift, lr, seed, stream_id=0,
             cg_tol=1e-10, cg_maxiter=1000, svd_rcond=0.0):
    return nk_sr_cfg(RULE[rule] if isinstance(rule, str) else rule, _prec(precision),
                     SOLVER[solver] if isinstance(solver, str) else solver, int(n_discard), int(n_samples),
                     int(cg_maxiter), float(diag_shift), float(lr), float(cg_tol), int(seed), int(stream_id),
                     float(svd_rcond))


def make_chains(s, sweeps_done=0, n_accepted=None):
    return nk_chains(int(s.shape[0]), s.data_ptr(), int(sweeps_done),
                     None if n_accepted is None else n_accepted.data_ptr())


PROF_CLASSES = {"sweep": 0, "eloc": 1, "gram": 2, "chol_update": 3, "chol_panel": 4, "trsv": 5,
                "jvp_vjp": 6}


def nk_prof_enable(on=True):
    _check(lib().nk_prof_enable(int(bool(on))))


def nk_prof_read(cls):
    """(milliseconds, launches, algorithmic work) of a tracked kernel class
    since nk_prof_enable."""
    ms, n, w = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
    c = PROF_CLASSES[cls] if isinstance(cls, str) else int(cls)
    _check(lib().nk_prof_read(c, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(w)))
    return ms.value, n.value, w.value


def nk_prof_read_executed(cls):
    """Work the hardware executed for the same launches (BF16 slice-product
    flops of the tensor-core paths)."""
    x = ctypes.c_double()
    c = PROF_CLASSES[cls] if isinstance(cls, str) else int(cls)
    _check(lib().nk_prof_read_executed(c, ctypes.byref(x)))
    return x.value


def nk_prof_trace():
    """[(class name, start ms, end ms)] of the bracketed launches since
    nk_prof_enable, in enqueue order, on one clock across streams."""
    n = ctypes.c_int32()
    _check(lib().nk_prof_trace(0, None, None, None, ctypes.byref(n)))
    m = n.value
    cls = (ctypes.c_int32 * max(m, 1))()
    t0 = (ctypes.c_double * max(m, 1))()
    t1 = (ctypes.c_double * max(m, 1))()
    _check(lib().nk_prof_trace(m, cls, t0, t1, ctypes.byref(n)))
    names = {v: k for k, v in PROF_CLASSES.items()}
    return [(names.get(cls[i], str(cls[i])), t0[i], t1[i]) for i in range(min(m, n.value))]


def nk_launch_count():
    return int(lib().nk_launch_count())


# ------------------------------------------------------------------ serving --

def make_request(kind, N, M, params, ham, n_chains, cfg):
    """An nk_request for host arrays: params float64 [Np], ham dict with int32
    edges [E, 2] (numpy).  The arrays must stay alive until submission."""
    import numpy as np
    p = np.ascontiguousarray(params, dtype=np.float64)
    e = np.ascontiguousarray(ham["edges"], dtype=np.int32).reshape(-1, 2)
    req = nk_request(NK_REQ_SR_STEP if kind in ("sr_step", NK_REQ_SR_STEP) else NK_REQ_EXPECT, int(N), int(M),
                     p.ctypes.data, KIND[ham["kind"]], float(ham["J"]), float(ham.get("h", 0.0)),
                     int(bool(ham.get("marshall", False))), int(e.shape[0]), e.ctypes.data, int(n_chains), cfg,
                     float(ham.get("J2", 0.0)), int(ham.get("n_edges2", 0)))
    req._keep = (p, e)
    return req


def nk_request_bytes(req):
    return int(lib().nk_request_bytes(ctypes.byref(req)))


def nk_server_create(device, hbm_budget, slots):
    h = ctypes.c_void_p()
    _check(lib().nk_server_create(int(device), int(hbm_budget), int(slots), ctypes.byref(h)))
    return h


def nk_server_submit(srv, req, params_out=None):
    rid = ctypes.c_uint64()
    out = None if params_out is None else params_out.ctypes.data_as(ctypes.c_void_p)
    _check(lib().nk_server_submit(srv, ctypes.byref(req), out, ctypes.byref(rid)))
    return int(rid.value)


def _result_dict(r):
    d = {f: getattr(r, f) for f, _ in nk_result._fields_}
    d["message"] = d["message"].decode(errors="replace")
    return d


def nk_server_poll(srv, rid):
    done = ctypes.c_int32()
    r = nk_result()
    _check(lib().nk_server_poll(srv, ctypes.c_uint64(rid), ctypes.byref(done), ctypes.byref(r)))
    return _result_dict(r) if done.value else None


def nk_server_wait(srv, rid):
    r = nk_result()
    _check(lib().nk_server_wait(srv, ctypes.c_uint64(rid), ctypes.byref(r)))
    return _result_dict(r)


def nk_server_stats_get(srv):
    st = nk_server_stats()
    _check(lib().nk_server_stats_get(srv, ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in nk_server_stats._fields_}


def nk_server_destroy(srv):
    _check(lib().nk_server_destroy(srv))


class Server:
    """Thin owner of an nk_server handle."""

    def __init__(self, device=0, hbm_budget=32 << 30, slots=8):
        self.handle = nk_server_create(device, hbm_budget, slots)

    def submit(self, req, params_out=None):
        return nk_server_submit(self.handle, req, params_out)

    def wait(self, rid):
        return nk_server_wait(self.handle, rid)

    def poll(self, rid):
        return nk_server_poll(self.handle, rid)

    def stats(self):
        return nk_server_stats_get(self.handle)

    def close(self):
        if self.handle:
            nk_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
