"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point include/nk.h declares, and fails cleanly without a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nk.h")


def declared_symbols():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(nk_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libnk():
    from paper_2112_10526_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_hot_path_calls():
    syms = declared_symbols()
    for name in ["nk_rbm_logpsi", "nk_metropolis_sweep", "nk_local_energy", "nk_jacobian",
                 "nk_qgt_matvec", "nk_sr_step", "nk_vjp", "nk_jvp", "nk_force", "nk_stats",
                 "nk_sr_solve", "nk_chains_init", "nk_ctx_create", "nk_ctx_destroy",
                 "nk_last_error", "nk_version"]:
        assert name in syms


def test_library_exports_every_declared_symbol(libnk):
    missing = [s for s in declared_symbols() if not hasattr(libnk, s)]
    assert not missing, missing


def test_version_and_error_string(libnk):
    libnk.nk_version.restype = ctypes.c_int32
    assert libnk.nk_version() >= 100
    libnk.nk_last_error.restype = ctypes.c_char_p
    assert isinstance(libnk.nk_last_error(), bytes)


def test_binding_names_match_the_abi():
    from paper_2112_10526_gb300 import nk
    for name in declared_symbols():
        if name in ("nk_ctx_create", "nk_ctx_destroy", "nk_last_error", "nk_version"):
            continue
        assert hasattr(nk, name), name


def test_null_arguments_rejected_without_touching_a_device(libnk):
    # A NULL context is rejected before any CUDA call.
    f = libnk.nk_rbm_logpsi
    f.restype = ctypes.c_int32
    assert f(None, None, 0, None, 0, None, None) == -1
    g = libnk.nk_sr_step
    g.restype = ctypes.c_int32
    assert g(None, None, None, None, None, None, None, None, None) == -1
    out = ctypes.c_void_p(1)
    c = libnk.nk_ctx_create
    c.restype = ctypes.c_int32
    code = c(0, ctypes.byref(out))
    if code != 0:  # no GPU here: a clean error, no handle
        assert code in (-1, -2) and not out.value
    else:
        libnk.nk_ctx_destroy(out)


def test_request_bytes_plan_only_without_gpu(libnk):
    """The admission estimate is a plan-only pass: it needs no GPU, grows
    with the sample count and counts the Ns x Ns factor of the sample-space
    solve."""
    from paper_2112_10526_gb300 import inputs as I
    from paper_2112_10526_gb300 import nk

    def req(ns, solver):
        N, M = 100, 200
        cfg = nk.make_cfg("exchange", "mixed", solver, 0, ns, 0.01, 0.01, 1)
        return nk.make_request("sr_step", N, M, I.rbm_params(N, M, 1), I.heis_square(10), 1024, cfg)

    a = nk.nk_request_bytes(req(1, "cg"))
    b = nk.nk_request_bytes(req(8, "cg"))
    c = nk.nk_request_bytes(req(8, "cholesky_samplespace"))
    if a == 0:
        pytest.skip("no CUDA driver to create the planning context")
    assert b > a > 0
    assert c >= b + 8192 * 8192 * 8


@pytest.mark.parametrize("kind", ["expect", "sr_step"])
def test_request_bytes_hamiltonian_rule_plans_like_its_effective_rule(libnk, kind):
    """NK_RULE_HAMILTONIAN is the local rule for the Ising model and an
    edge-swap rule for the Heisenberg model.  The plan-only pass (no GPU)
    accepts it for both request kinds; an SR step of the Ising model then
    carves no edge tables, so it plans exactly the bytes of the local rule."""
    from paper_2112_10526_gb300 import inputs as I
    from paper_2112_10526_gb300 import nk

    def req(rule, ham, N):
        M = 2 * N
        cfg = nk.make_cfg(rule, "mixed", "cg", 0, 4, 0.01, 0.01, 1)
        return nk.make_request(kind, N, M, I.rbm_params(N, M, 1), ham, 256, cfg)

    tfim, heis = I.tfim_square(8), I.heis_square(8)  # E = 2N: edge tables differ in size from site tables
    b_loc = nk.nk_request_bytes(req("local", tfim, 64))
    if b_loc == 0:
        pytest.skip("no CUDA driver to create the planning context")
    assert nk.nk_request_bytes(req("hamiltonian", tfim, 64)) == b_loc
    assert nk.nk_request_bytes(req("hamiltonian", heis, 64)) == nk.nk_request_bytes(req("exchange", heis, 64)) > 0


def test_request_bytes_plans_a_j1j2_request(libnk):
    """A serving request carries the second edge class (J2, n_edges2) of the
    J1-J2 model; the plan-only pass sizes it with both classes."""
    from paper_2112_10526_gb300 import inputs as I
    from paper_2112_10526_gb300 import nk

    N, M = 100, 200
    cfg = nk.make_cfg("exchange", "mixed", "cholesky_samplespace", 0, 1, 0.01, 0.02, 6)
    ham = I.j1j2_square(10)
    r = nk.make_request("sr_step", N, M, I.rbm_params(N, M, 6), ham, 1024, cfg)
    assert (r.J2, r.n_edges2, r.n_edges) == (0.5, 200, 400)
    b = nk.nk_request_bytes(r)
    if b == 0:
        pytest.skip("no CUDA driver to create the planning context")
    r1 = nk.make_request("sr_step", N, M, I.rbm_params(N, M, 6), I.heis_square(10), 1024, cfg)
    assert b > nk.nk_request_bytes(r1) > 0  # twice the edge tables


def test_library_leaves_no_internal_symbol_undefined():
    """A shared library links even when one of its own functions is missing;
    every nk:: symbol the library uses must be defined in it."""
    import shutil
    import subprocess
    from paper_2112_10526_gb300 import build
    if shutil.which("nm") is None:
        pytest.skip("no nm")
    lib = build.build()
    out = subprocess.run(["nm", "-D", "--undefined-only", lib], capture_output=True, text=True, check=True).stdout
    missing = [ln.split()[-1] for ln in out.splitlines() if "_ZN2nk" in ln or " nk_" in ln]
    assert not missing, missing
