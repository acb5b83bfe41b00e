"""The no-allocation local-energy entry point (nk_local_energy_noalloc).

It serves callers that cannot let a library allocate device memory: their
HBM belongs to another allocator, or they cannot pay for cudaMalloc's
device-wide synchronisation.  Its tables live in a fixed array compiled into
the library.  In FP64 it runs the kernels of nk_local_energy on the same
tables, so its results must be bit-identical to that entry point's.  In the
mixed precision it rebuilds the hidden activations per sample in FP64
instead of taking the tensor-core product, so it must agree within the mixed
tolerance (1e-4 relative per sample), with nk_local_energy and with the
oracle.  This file is collected last so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2112_10526_gb300 import inputs as I
from paper_2112_10526_gb300 import nk

from gpu_util import cu, dev, ham_to_device, rel_err

pytestmark = pytest.mark.gpu

CASES = [
    ("tfim-chain16-f64", 16, 16, lambda: I.tfim_chain(16), False, 1000, "f64"),
    ("heis-10x10-f64", 100, 200, lambda: I.heis_square(10), True, 513, "f64"),
    ("heis-4x4-mixed", 16, 32, lambda: I.heis_square(4, 0.8, False), True, 77, "mixed"),
    ("tfim-ragged-mixed", 37, 45, lambda: I.tfim_chain(37, -0.6, 0.9), False, 65, "mixed"),
    # M >= 1024: the local-energy kernel's hidden-unit mapping with theta
    # rebuilt per sample (tables 16 x 1024 fit the fixed array)
    ("heis-4x4-wide-mixed", 16, 1024, lambda: I.heis_square(4), True, 96, "mixed"),
    ("tfim-chain16-wide-mixed", 16, 1040, lambda: I.tfim_chain(16, 1.0, 0.7), False, 40, "mixed"),
]
MIXED_TOL = 1e-4


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    with nk.Ctx() as c:
        yield c


@pytest.mark.parametrize("name,N,M,hf,sz0,B,prec", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_workspace_entry_point_twice(ctx, name, N, M, hf, sz0, B, prec):
    ham = hf()
    p_host = I.rbm_params(N, M, 23, 0.3)
    s_host = I.random_configs(B, N, 11, sz0=sz0)
    p, s = cu(p_host), cu(s_host)
    h, _edges = ham_to_device(ham)
    ref = torch.empty(B, dtype=torch.float64, device=dev())
    tref = torch.empty((B, M), dtype=torch.float64, device=dev())
    nk.nk_local_energy(ctx, p, N, M, h, s, ref, tref, precision=prec)
    torch.cuda.synchronize()
    ref_h, tref_h = ref.cpu().numpy(), tref.cpu().numpy()
    eo = oracle.local_energy(p_host, N, M, ham, s_host) if prec == "mixed" else None
    for _ in range(2):  # the second call reuses the scratch left by the first
        out = torch.full((B,), np.nan, dtype=torch.float64, device=dev())
        t = torch.full((B, M), np.nan, dtype=torch.float64, device=dev())
        nk.nk_local_energy_noalloc(p, N, M, h, s, out, t, precision=prec)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        if prec == "f64":
            np.testing.assert_array_equal(got, ref_h)
            np.testing.assert_array_equal(t.cpu().numpy(), tref_h)
        else:
            assert rel_err(got, ref_h) <= MIXED_TOL
            assert rel_err(got, eo) <= MIXED_TOL
            assert rel_err(t.cpu().numpy(), tref_h) <= 1e-12


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


def test_noalloc_rejects_memory_the_current_device_cannot_use():
    """Host memory, pinned or pageable, is refused before any launch (and so
    would another GPU's memory be: the check compares the pointer's device
    with the current one)."""
    N, M = 16, 16
    ham = I.tfim_chain(16)
    p = cu(I.rbm_params(N, M, 3))
    h, _edges = ham_to_device(ham)
    out = torch.empty(4, dtype=torch.float64, device=dev())
    for s in (torch.from_numpy(I.random_configs(4, N, 1)),
              torch.from_numpy(I.random_configs(4, N, 1)).pin_memory()):
        with pytest.raises(nk.NkError) as ei:
            nk.nk_local_energy_noalloc(p, N, M, h, s, out)
        assert ei.value.code == nk.NK_ERR_INVALID_ARG
        assert "current device" in str(ei.value)
    if torch.cuda.device_count() > 1:
        other = (torch.cuda.current_device() + 1) % torch.cuda.device_count()
        s = torch.from_numpy(I.random_configs(4, N, 1)).to(torch.device("cuda", other))
        with pytest.raises(nk.NkError) as ei:
            nk.nk_local_energy_noalloc(p, N, M, h, s, out)
        assert ei.value.code == nk.NK_ERR_INVALID_ARG
