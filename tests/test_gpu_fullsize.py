"""Parity at the full lattice sizes of the benchmark workloads, in the launch
configuration bench.py times, on sampled outputs the oracle computes site by site
(oracle.sample), plus whole-lattice properties (FP64 true residual) for solves.

Sizes: 16^3x32 Ls=12 (the benchmark workload), 24^3x64 Ls=10, 32^3x64 Ls=12 with 12
right-hand sides (the batched propagator launch).  Tolerances as in test_gpu_apply
(relative 2-norm over the sampled sites)."""
import numpy as np
import pytest

import inputs
from oracle import dirac, sample
from oracle.dirac import MobiusParams
from gpu_common import lib, rel, to_dev, to_host, parity_of, torch

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f32": 1e-6, "f16": 2e-3, "bf16": 8e-3}
_LINKS = {}


def _links(dims, eps, seed):
    key = (dims, eps, seed)
    if key not in _LINKS:
        _LINKS.clear()
        _LINKS[key] = inputs.gauge_links(dims, eps, seed)
    return _LINKS[key]


def _sites(dims, n, parity, seed):
    rng = np.random.default_rng(seed)
    X, Y, Z, T = dims
    out = []
    while len(out) < n:
        c = (rng.integers(X), rng.integers(Y), rng.integers(Z), rng.integers(T))
        if parity is None or sum(c) % 2 == parity:
            out.append(c)
    # include lattice corners (boundary wrap, t = 0 and t = T-1)
    for c in [(0, 0, 0, 0), (X - 1, Y - 1, Z - 1, T - 1), (1, 0, 0, T - 1), (0, 1, Z - 1, 0)]:
        if parity is None or sum(c) % 2 == parity:
            out.append(c)
    return np.array(out, dtype=np.int64)


def _apply(m, ctx, op, prec, psi_dev, nrhs):
    nb = ctx.field_bytes(prec, nrhs)
    fin = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    fout = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    m.mdwf_pack(ctx.h, psi_dev, fin, m.PRECS[prec], nrhs)
    m.mdwf_apply(ctx.h, m.OP[op], m.PRECS[prec], fin, fout, nrhs)
    out = torch.empty_like(psi_dev)
    m.mdwf_unpack(ctx.h, fout, out, m.PRECS[prec], nrhs)
    del fin, fout
    return out


def _check_ops(m, ctx, Ub, p, dims, psi_dev, nrhs, precs, seed):
    odd = _sites(dims, 24, 1, seed)
    anyp = _sites(dims, 24, None, seed + 1)
    src = inputs.DeviceSites(psi_dev)
    for prec in precs:
        for op in ("HOP_OE_M5INV", "MPC", "FULL_D"):
            got = inputs.DeviceSites(_apply(m, ctx, op, prec, psi_dev, nrhs))
            for r in range(nrhs):
                fr = _RHS(src, r)
                if op == "HOP_OE_M5INV":
                    ref = sample._s(p, "A5inv", sample.hop_at(Ub, fr, odd, dims))
                    sites = odd
                elif op == "MPC":
                    ref = sample.mpc_at(Ub, fr, odd, p, dims)
                    sites = odd
                else:
                    ref = sample.mobius_at(Ub, fr, anyp, p, dims)
                    sites = anyp
                g = _RHS(got, r)[..., sites[:, 3], sites[:, 2], sites[:, 1], sites[:, 0], :, :]
                err = rel(g, ref)
                assert err <= TOL[prec], (op, prec, r, err)


class _RHS:
    """field[r] view for DeviceSites."""

    def __init__(self, f, r):
        self.f, self.r = f, r

    def __getitem__(self, idx):
        full = self.f[idx]
        return full[self.r]


def test_fullsize_16x32_ls12_applies():
    m = lib()
    dims, Ls, mf, eps, seed = (16, 16, 16, 32), 12, 0.02, 0.4, 2
    U = _links(dims, eps, seed)
    ctx = m.Context(dims, Ls, mf=mf)
    ctx.load_gauge(U)
    p = MobiusParams(Ls=Ls, mf=mf)
    Ub = dirac.boundary_links(U, -1.0)
    psi = inputs.gaussian_spinor5d_device(dims, Ls, seed + 100, nrhs=1)
    _check_ops(m, ctx, Ub, p, dims, psi, 1, ("f64", "f32", "f16", "bf16"), 5)


def test_fullsize_16x32_ls12_solves_point_source():
    m = lib()
    dims, Ls, mf, eps, seed = (16, 16, 16, 32), 12, 0.02, 0.4, 2
    U = _links(dims, eps, seed)
    ctx = m.Context(dims, Ls, mf=mf)
    ctx.load_gauge(U)
    p = MobiusParams(Ls=Ls, mf=mf)
    Ub = dirac.boundary_links(U, -1.0)
    b4 = torch.from_numpy(inputs.point_source4d(dims, 0, 0)).cuda().reshape((1,) + ctx.shape4d())
    eta = ctx.make_source_4d(b4, nrhs=1)[0]
    bnorm = float(torch.linalg.vector_norm(eta))
    sites = np.concatenate([_sites(dims, 24, None, 9), np.array([[0, 0, 0, 0], [1, 0, 0, 0], [0, 0, 0, 1]])])
    for sloppy in ("f64", "f16"):
        x, info = ctx.solve(eta, tol=1e-10, sloppy=sloppy)
        assert info.status == 0 and info.true_residual <= 1e-10, (sloppy, info.true_residual)
        assert info.full_residual <= 1e-9
        # oracle residual b - D x at sampled sites (including the source and its neighbours)
        xs, bs = inputs.DeviceSites(x), inputs.DeviceSites(eta)
        res = sample.gather(bs, sites) - sample.mobius_at(Ub, xs, sites, p, dims)
        assert np.linalg.norm(res) <= 1e-9 * bnorm, (sloppy, np.linalg.norm(res) / bnorm)


def test_fullsize_24x64_ls10_f16_applies():
    m = lib()
    dims, Ls, mf, eps, seed = (24, 24, 24, 64), 10, 0.01, 0.5, 3
    U = _links(dims, eps, seed)
    ctx = m.Context(dims, Ls, mf=mf)
    ctx.load_gauge(U)
    p = MobiusParams(Ls=Ls, mf=mf)
    Ub = dirac.boundary_links(U, -1.0)
    psi = inputs.gaussian_spinor5d_device(dims, Ls, seed + 100, nrhs=1)
    _check_ops(m, ctx, Ub, p, dims, psi, 1, ("f16", "bf16"), 6)


def test_fullsize_32x64_ls12_12rhs_applies():
    m = lib()
    dims, Ls, mf, eps, seed = (32, 32, 32, 64), 12, 0.01, 0.5, 4
    U = _links(dims, eps, seed)
    ctx = m.Context(dims, Ls, mf=mf)
    ctx.load_gauge(U)
    p = MobiusParams(Ls=Ls, mf=mf)
    Ub = dirac.boundary_links(U, -1.0)
    psi = inputs.gaussian_spinor5d_device(dims, Ls, seed + 100, nrhs=12)
    _check_ops(m, ctx, Ub, p, dims, psi, 12, ("f16",), 7)
