"""Parity at the full lattice sizes of the benchmark workloads, in the launch
configuration bench.py times (the autotuner on, as in bench.py).

* 16^3x32, Ls=12: the WHOLE output of HOP_OE_M5INV, MPC, MPC_DAG and FULL_D at all four
  precisions against the full-lattice FP64 oracle (oracle.dirac), checked as a relative
  2-norm and per 5D site (gpu_common.site_rel).
* 24^3x64, Ls=10 and 32^3x64, Ls=12 with 12 right-hand sides: sampled outputs the oracle
  computes site by site (oracle.sample) at >= 2000 4D sites (all s and right-hand sides):
  random sites, the first and last site of many tiles of every tile size the autotuner
  picked for the launching kernels, every site of the last tile, lattice corners.
* Solves at 16^3x32: FP64 true residual and the oracle's b - D x at sampled sites.
"""

import numpy as np
import pytest

import inputs
from oracle import dirac, sample
from oracle.dirac import MobiusParams
from gpu_common import lib, rel, site_rel, to_dev, to_host, parity_of, torch, TOL, SITE_TOL

pytestmark = pytest.mark.gpu

_LINKS = {}


def _links(dims, eps, seed):
    key = (dims, eps, seed)
    if key not in _LINKS:
        _LINKS.clear()
        _LINKS[key] = inputs.gauge_links(dims, eps, seed)
    return _LINKS[key]


def _apply(m, ctx, op, prec, psi_dev, nrhs):
    nb = ctx.field_bytes(prec, nrhs)
    fin = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    fout = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    m.mdwf_pack(ctx.h, psi_dev, fin, m.PRECS[prec], nrhs)
    m.mdwf_apply(ctx.h, m.OP[op], m.PRECS[prec], fin, fout, nrhs)
    out = torch.zeros_like(psi_dev)
    m.mdwf_unpack(ctx.h, fout, out, m.PRECS[prec], nrhs)
    del fin, fout
    return out


def _cb_to_coords(dims, x_cb, parity):
    """Checkerboard index within a parity half -> (x, y, z, t), the library's site order
    ((t Z + z) Y + y) X/2 + x/2 (the documented internal layout)."""
    X, Y, Z, T = dims
    Xh = X // 2
    xh = x_cb % Xh
    rest = x_cb // Xh
    y = rest % Y
    rest //= Y
    z = rest % Z
    t = rest // Z
    x = 2 * xh + ((parity + y + z + t) & 1)
    return np.stack([x, y, z, t], axis=1).astype(np.int64)


def _tuned_tiles(ctx, tag="hop"):
    """Sites-per-CTA values the autotuner chose for this lattice's hop kernels."""
    out = set()
    for key, ns, _ in ctx.tune_entries():
        if key.startswith(tag + "|") or key.startswith(tag + "dag|"):
            out.add(ns & 0xFFFF)
    return sorted(out) or [1]


def _sites(dims, parity, tiles, seed, n_random=2000, n_tiles=500):
    """>= 2000 sites of one parity (None: both): random ones, the first and last site of
    n_tiles random tiles of every tile size, the whole last tile, lattice corners."""
    X, Y, Z, T = dims
    vh = X * Y * Z * T // 2
    rng = np.random.default_rng(seed)
    pars = [0, 1] if parity is None else [parity]
    out = []
    for par in pars:
        out.append(_cb_to_coords(dims, rng.integers(0, vh, n_random // len(pars)), par))
        for ns in tiles:
            nb = (vh + ns - 1) // ns
            b = rng.integers(0, nb, n_tiles // len(pars))
            first = b * ns
            last = np.minimum(first + ns - 1, vh - 1)
            out.append(_cb_to_coords(dims, np.concatenate([first, last]), par))
            out.append(_cb_to_coords(dims, np.arange((nb - 1) * ns, vh), par))
    corners = np.array([(0, 0, 0, 0), (X - 1, Y - 1, Z - 1, T - 1), (1, 0, 0, T - 1), (0, 1, Z - 1, 0)])
    if parity is not None:
        corners = corners[corners.sum(1) % 2 == parity]
    out.append(corners)
    s = np.unique(np.concatenate(out), axis=0)
    return s


def _sampled_check(m, ctx, Ub, p, dims, psi_dev, nrhs, precs, seed):
    src = inputs.DeviceSites(psi_dev)
    for prec in precs:
        for op in ("HOP_OE_M5INV", "MPC", "MPC_DAG", "FULL_D"):
            got_dev = _apply(m, ctx, op, prec, psi_dev, nrhs)
            tiles = _tuned_tiles(ctx)
            if op == "FULL_D":
                sites = _sites(dims, None, tiles, seed)
                ref = sample.mobius_at(Ub, src, sites, p, dims)
            else:
                sites = _sites(dims, 1, tiles, seed)
                if op == "HOP_OE_M5INV":
                    ref = sample._s(p, "A5inv", sample.hop_at(Ub, src, sites, dims))
                elif op == "MPC":
                    ref = sample.mpc_at(Ub, src, sites, p, dims)
                else:
                    ref = sample.mpc_dag_at(Ub, src, sites, p, dims)
            assert len(sites) >= 2000
            got = sample.gather(inputs.DeviceSites(got_dev), sites)
            del got_dev
            err = rel(got, ref)
            assert err <= TOL[prec], (op, prec, err)
            serr = site_rel(got, ref)
            assert serr <= SITE_TOL[prec], (op, prec, "per site", serr)


def test_wholelattice_16x32_ls12_per_site():
    """Every 5D site of the 16^3x32x12 outputs against the full-lattice oracle."""
    m = lib()
    dims, Ls, mf, eps, seed = (16, 16, 16, 32), 12, 0.02, 0.4, 2
    U = _links(dims, eps, seed)
    ctx = m.Context(dims, Ls, mf=mf)
    ctx.load_gauge(U)
    p = MobiusParams(Ls=Ls, mf=mf)
    Ub = dirac.boundary_links(U, -1.0)
    par = parity_of(dims)
    psi = inputs.gaussian_spinor5d(dims, Ls, seed + 100)
    psi_dev = to_dev(psi)
    refs = {
        "HOP_OE_M5INV": (dirac.on_parity(dirac.s_op(p, "A5inv", dirac.hop(Ub, dirac.on_parity(psi, par, 0))),
                                         par, 1), par == 1),
        "MPC": (dirac.mpc(Ub, dirac.on_parity(psi, par, 1), p), par == 1),
        "MPC_DAG": (dirac.mpc_dag(Ub, dirac.on_parity(psi, par, 1), p), par == 1),
        "FULL_D": (dirac.mobius(Ub, psi, p), None),
    }
    for prec in ("f64", "f32", "f16", "bf16"):
        for op, (ref, keep) in refs.items():
            got = to_host(_apply(m, ctx, op, prec, psi_dev, 1))
            if keep is not None:
                assert not np.any(got[..., ~keep, :, :]), (op, prec, "other parity written")
            err = rel(got, ref)
            assert err <= TOL[prec], (op, prec, err)
            serr = site_rel(got, ref, keep)
            assert serr <= SITE_TOL[prec], (op, prec, "per site", serr)


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
    rng = np.random.default_rng(9)
    sites = np.concatenate([np.stack([rng.integers(0, d, 24) for d in dims], 1),
                            np.array([[0, 0, 0, 0], [1, 0, 0, 0], [0, 0, 0, 1]])])
    for sloppy in ("f64", "f16"):
        x, info = ctx.solve(eta, tol=1e-10, sloppy=sloppy, full_residual=True)
        assert info.status == 0 and info.true_residual <= 1e-10, (sloppy, info.true_residual)
        assert info.full_residual <= 1e-9
        # oracle residual b - D x at sampled sites (including the source and its neighbours)
        xs, bs = inputs.DeviceSites(x), inputs.DeviceSites(eta)
        res = sample.gather(bs, sites) - sample.mobius_at(Ub, xs, sites, p, dims)
        assert np.linalg.norm(res) <= 1e-9 * bnorm, (sloppy, np.linalg.norm(res) / bnorm)


def test_fullsize_24x64_ls10_sampled():
    m = lib()
    dims, Ls, mf, eps, seed = (24, 24, 24, 64), 10, 0.01, 0.5, 3
    U = _links(dims, eps, seed)
    ctx = m.Context(dims, Ls, mf=mf)
    ctx.load_gauge(U)
    p = MobiusParams(Ls=Ls, mf=mf)
    Ub = dirac.boundary_links(U, -1.0)
    psi = inputs.gaussian_spinor5d_device(dims, Ls, seed + 100, nrhs=1)[0]
    _sampled_check(m, ctx, Ub, p, dims, psi, 1, ("f16", "bf16", "f32"), 6)


def test_fullsize_32x64_ls12_12rhs_sampled():
    m = lib()
    dims, Ls, mf, eps, seed = (32, 32, 32, 64), 12, 0.01, 0.5, 4
    U = _links(dims, eps, seed)
    ctx = m.Context(dims, Ls, mf=mf)
    ctx.load_gauge(U)
    p = MobiusParams(Ls=Ls, mf=mf)
    Ub = dirac.boundary_links(U, -1.0)
    psi = inputs.gaussian_spinor5d_device(dims, Ls, seed + 100, nrhs=12)
    _sampled_check(m, ctx, Ub, p, dims, psi, 12, ("f16",), 7)
