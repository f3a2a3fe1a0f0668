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


# Relative 2-norm tolerances of applies (whole output or sampled sites), and per-5D-site
# bounds: max over sites of |got - ref|_site / rms_site(ref).  Rounding to 16 bits gives
# a max-site / rms error ratio of 2.3 (F16 + norm) and 2.5 (BF16) times the relative
# 2-norm error over 2M Gaussian sites, so the 16-bit site bounds are 2.5x the 2-norm
# tolerance; FP64 / FP32 errors sit far below theirs.  A wrong tile, column or boundary
# term gives O(1) at the sites it touches.  16-bit fixed point (I16): half a unit of
# 1/32767 of the site norm on every stored input, link and output (1.5e-5 each) and FP32
# arithmetic give a few 1e-5; 1e-4 leaves 3x, and the site bound is 2.5x that.
# Emulated FP64 (f64e: float pairs, compensated sums): inputs and links split with a
# relative error below 2^-46 (1.4e-14), each product exact up to its cross terms (2^-48),
# each output real a sum of 8 direction terms whose error parts are added in float (a few
# 2^-48 of the terms): ~1e-14 relative; the FP64 bar 1e-13 leaves several times that.
TOL = {"f64": 1e-13, "f32": 1e-6, "f16": 2e-3, "bf16": 8e-3, "i16": 1e-4, "f64e": 1e-13}
SITE_TOL = {"f64": 1e-13, "f32": 1e-6, "f16": 5e-3, "bf16": 2e-2, "i16": 2.5e-4, "f64e": 1e-13}


def site_rel(got, ref, keep=None):
    """max over 5D sites of |got - ref| / rms over sites of |ref|; a site is every index
    but the trailing (spin, colour) axes.  keep: boolean mask broadcast against the site
    axes (e.g. a [t, z, y, x] parity mask) selecting the sites compared."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    d = np.sqrt(np.sum(np.abs(got - ref) ** 2, axis=(-2, -1)))
    r = np.sum(np.abs(ref) ** 2, axis=(-2, -1))
    if keep is not None:
        k = np.broadcast_to(keep, d.shape)
        d, r = d[k], r[k]
    return float(d.max() / np.sqrt(r.mean()))


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def to_host(t):
    return t.cpu().numpy()


def parity_of(dims):
    X, Y, Z, T = dims
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    return (x + y + z + t) % 2
