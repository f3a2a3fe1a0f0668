"""Shared helpers of the GPU parity tests (test code; no solver arithmetic)."""
import os
import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_BUILT = False


def lib():
    global _BUILT
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not _BUILT:
        import __graft_entry__
        __graft_entry__.build()
        _BUILT = True
    import paper_1810_01609_gb300 as m
    return m


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def to_host(t):
    return t.cpu().numpy()


def parity_of(dims):
    X, Y, Z, T = dims
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    return (x + y + z + t) % 2
