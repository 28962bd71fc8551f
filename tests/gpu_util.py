"""Helpers for the GPU parity tests (test infrastructure)."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def colrel(a, b):
    """Per-column relative error of blocks (..., n): max over columns of ||a-b|| / ||b||."""
    a = np.asarray(a).reshape(-1, a.shape[-1])
    b = np.asarray(b).reshape(-1, b.shape[-1])
    return float(np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)))


def make_ctx(dims, mass, U, bc_t=-1):
    torch = need_gpu()
    from paper_1808_01829_gb300.api import RhmcContext

    ctx = RhmcContext(dims, mass, bc_t=bc_t, device=0)
    ctx.set_gauge(torch.from_numpy(np.ascontiguousarray(U)).cuda())
    return ctx


def to_gpu(a):
    torch = need_gpu()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()
