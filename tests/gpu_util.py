"""Helpers shared by the GPU parity tests: device transfer and error norms."""

import numpy as np
import pytest


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def dev(torch, a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    """||a - b|| / ||b||."""
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


def emax(a, b):
    """Element-wise: max |a - b| / max |b| (one wrong element shows at any size)."""
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def round_storage(x, prec):
    """Round every real component as the library stores it: double -> float -> half/bf16."""
    import torch as _t
    if prec == "fp64":
        return np.array(x)
    f = np.asarray(x).astype(np.complex64)
    if prec == "fp32":
        return f.astype(np.complex128)
    re = _t.from_numpy(np.ascontiguousarray(f.real))
    im = _t.from_numpy(np.ascontiguousarray(f.imag))
    dt = _t.float16 if prec == "fp16" else _t.bfloat16
    re = re.to(dt).to(_t.float64).numpy()
    im = im.to(dt).to(_t.float64).numpy()
    return re + 1j * im
