"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import torch

from paper_2112_10526_gb300 import nk


def dev():
    return torch.device("cuda", torch.cuda.current_device())


def cu(x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(dev())


def ham_to_device(ham):
    edges = cu(np.asarray(ham["edges"], dtype=np.int32).reshape(-1, 2))
    return nk.make_ham(ham["kind"], ham["J"], ham.get("h", 0.0), ham.get("marshall", False), edges,
                       ham.get("J2", 0.0), ham.get("n_edges2", 0)), edges


def rel_err(got, ref, floor=None):
    """max |got - ref| / max(|ref|, floor) with floor = rms(ref) by default."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if floor is None:
        floor = float(np.sqrt(np.mean(ref ** 2))) if ref.size else 1.0
        floor = max(floor, 1e-300)
    return float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), floor))) if ref.size else 0.0


def vec_rel_err(got, ref):
    """||got - ref|| / ||ref|| (real or complex vectors)."""
    cplx = np.iscomplexobj(got) or np.iscomplexobj(ref)
    got = np.asarray(got, dtype=np.complex128 if cplx else np.float64).ravel()
    ref = np.asarray(ref, dtype=np.complex128 if cplx else np.float64).ravel()
    n = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / (n if n > 0 else 1.0))
