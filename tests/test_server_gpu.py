"""The serving loop (nk_server_*): each request's result is the same alone and
in a concurrent mix; admission under a tight HBM budget queues requests
instead of failing them; a request that can never fit fails cleanly."""
import numpy as np
import pytest
import torch

from paper_2112_10526_gb300 import inputs as I
from paper_2112_10526_gb300 import nk

pytestmark = pytest.mark.gpu


def _requests():
    reqs = []
    specs = [("tfim", 16, 1, 1024, "local"), ("heis", 16, 2, 1024, "exchange"), ("tfim", 32, 2, 2048, "local"),
             ("heis", 36, 1, 1024, "exchange"), ("tfim", 64, 1, 1024, "local"), ("heis", 64, 2, 2048, "exchange"),
             ("tfim", 16, 4, 3072, "local"), ("heis", 16, 1, 1024, "exchange")]
    for r, (kind, N, alpha, ns, rule) in enumerate(specs):
        M = alpha * N
        if kind == "tfim":
            ham = I.tfim_chain(N, 1.0, 1.0)
        else:
            L = int(round(N ** 0.5))
            ham = I.heis_square(L, 1.0, True)
        p = I.rbm_params(N, M, 40000 + r)
        Np = N + M + M * N
        solver = "cholesky" if Np <= 4096 else "cg"
        prec = "mixed" if r % 2 else "f64"
        cfg = nk.make_cfg(rule, prec, solver, 8, ns // 1024, 0.01, 0.01, 40000 + r, stream_id=r, cg_tol=1e-8,
                          cg_maxiter=2000)
        reqs.append((nk.make_request("sr_step", N, M, p, ham, 1024, cfg), Np))
    return reqs


def _run(slots, budget, reqs):
    outs = []
    with nk.Server(torch.cuda.current_device(), budget, slots) as srv:
        ids = []
        for req, Np in reqs:
            po = np.empty(Np)
            ids.append((srv.submit(req, po), po))
        for rid, po in ids:
            outs.append((srv.wait(rid), po))
        st = srv.stats()
    return outs, st


@pytest.fixture(scope="module")
def alone():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    reqs = _requests()
    return [_run(1, 64 << 30, [rq])[0][0] for rq in reqs]


def test_results_identical_alone_and_in_mix(alone):
    mixed, st = _run(8, 64 << 30, _requests())
    assert st["completed"] == len(mixed) and st["failed"] == 0
    for (ra, pa), (rm, pm) in zip(alone, mixed):
        assert ra["status"] == 0 and rm["status"] == 0
        assert ra["energy"] == rm["energy"] and ra["error"] == rm["error"]
        np.testing.assert_array_equal(pa, pm)
    assert len({r["slot"] for r, _ in mixed}) > 1  # ran concurrently on several slots


def test_admission_under_tight_budget(alone):
    reqs = _requests()
    biggest = max(nk.nk_request_bytes(r) for r, _ in reqs)
    outs, st = _run(8, int(biggest * 1.6), reqs)
    assert st["failed"] == 0 and st["completed"] == len(reqs)
    for (ra, pa), (rm, pm) in zip(alone, outs):
        assert ra["energy"] == rm["energy"]
        np.testing.assert_array_equal(pa, pm)
    assert max(r["queue_ms"] for r, _ in outs) > 0.0
    assert st["p99_ms"] >= st["p50_ms"] > 0.0


def test_request_that_can_never_fit_fails_cleanly():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    reqs = _requests()
    outs, st = _run(2, 1 << 20, reqs[:2])  # 1 MiB budget
    assert st["failed"] == 2
    assert all(r["status"] == nk.NK_ERR_OOM for r, _ in outs)


def _serve_mix(n):
    out = []
    for sp in I.serve_requests(n, seed=4):
        cfg = nk.make_cfg(sp["rule"], "mixed", sp["solver"], 8, sp["per_chain"], 0.01, 0.01, sp["seed"],
                          stream_id=sp["index"], cg_tol=1e-8, cg_maxiter=200)
        p = I.rbm_params(sp["N"], sp["M"], sp["seed"])
        out.append((nk.make_request("sr_step", sp["N"], sp["M"], p, sp["ham"], sp["chains"], cfg),
                    sp["N"] + sp["M"] + sp["M"] * sp["N"]))
    return out


def test_heterogeneous_mix_concurrent_launches():
    """Slots launch the same kernels with different shared-memory sizes at
    the same time; every request must still succeed and match its solo run."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    reqs = _serve_mix(64)
    mixed, st = _run(8, 64 << 30, reqs)
    bad = [(k, r["status"], r["message"]) for k, (r, _) in enumerate(mixed) if r["status"] != 0]
    assert not bad and st["failed"] == 0
    for k in range(0, 64, 9):
        (ra, pa), = _run(1, 64 << 30, [reqs[k]])[0]
        assert ra["energy"] == mixed[k][0]["energy"]
        np.testing.assert_array_equal(pa, mixed[k][1])
