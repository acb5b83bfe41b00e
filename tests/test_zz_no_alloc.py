"""The no-allocation local-energy entry point (nk_local_energy_noalloc).

It serves callers that cannot let a library allocate device memory: their
HBM belongs to another allocator, or they cannot pay for cudaMalloc's
device-wide synchronisation.  Its tables live in a fixed array compiled into
the library, so its results must equal those of nk_local_energy, which keeps
the same tables in a context workspace.  This file is collected last so that
a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

from paper_2112_10526_gb300 import inputs as I
from paper_2112_10526_gb300 import nk

from gpu_util import cu, dev, ham_to_device, rel_err

pytestmark = pytest.mark.gpu

CASES = [
    ("tfim-chain16-f64", 16, 16, lambda: I.tfim_chain(16), False, 1000, "f64", 1e-10),
    ("heis-10x10-f64", 100, 200, lambda: I.heis_square(10), True, 513, "f64", 1e-10),
    ("heis-4x4-mixed", 16, 32, lambda: I.heis_square(4, 0.8, False), True, 77, "mixed", 1e-4),
    ("tfim-ragged-mixed", 37, 45, lambda: I.tfim_chain(37, -0.6, 0.9), False, 65, "mixed", 1e-4),
]


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    with nk.Ctx() as c:
        yield c


@pytest.mark.parametrize("name,N,M,hf,sz0,B,prec,tol", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_workspace_entry_point_twice(ctx, name, N, M, hf, sz0, B, prec, tol):
    ham = hf()
    p = cu(I.rbm_params(N, M, 23, 0.3))
    s = cu(I.random_configs(B, N, 11, sz0=sz0))
    h, _edges = ham_to_device(ham)
    ref = torch.empty(B, dtype=torch.float64, device=dev())
    tref = torch.empty((B, M), dtype=torch.float64, device=dev())
    nk.nk_local_energy(ctx, p, N, M, h, s, ref, tref, precision=prec)
    for _ in range(2):  # the second call reuses the scratch left by the first
        out = torch.full((B,), np.nan, dtype=torch.float64, device=dev())
        t = torch.full((B, M), np.nan, dtype=torch.float64, device=dev())
        nk.nk_local_energy_noalloc(p, N, M, h, s, out, t, precision=prec)
        torch.cuda.synchronize()
        assert rel_err(out.cpu().numpy(), ref.cpu().numpy()) <= tol
        assert rel_err(t.cpu().numpy(), tref.cpu().numpy()) <= 1e-12


def test_noalloc_rejects_sizes_beyond_its_scratch():
    N, M = 400, 1600  # TFIM tables need ~15 MB > the fixed 8 MiB
    ham = I.tfim_square(20)
    p = cu(I.rbm_params(N, M, 3))
    s = cu(I.random_configs(4, N, 1))
    h, _edges = ham_to_device(ham)
    out = torch.empty(4, dtype=torch.float64, device=dev())
    with pytest.raises(nk.NkError) as ei:
        nk.nk_local_energy_noalloc(p, N, M, h, s, out)
    assert ei.value.code == nk.NK_ERR_INVALID_ARG
    assert "scratch" in str(ei.value)
