"""GPU parity of the operator kernels (C ABI mdwf_apply / mdwf_pack / mdwf_unpack) against
the FP64 oracle on the same seeded inputs.  Tolerances: relative 2-norm difference of the
whole output, FP64 1e-13, FP32 1e-6, F16 (+norm) 2e-3, BF16 8e-3 (8 significant bits:
unit roundoff 2^-9 on input and output, plus the 16-bit projection and link rounding),
emulated FP64 (FP64 storage, double-float hops) 1e-13."""
import numpy as np
import pytest

import inputs
from oracle import dirac, storage
from oracle.dirac import MobiusParams
from gpu_common import lib, rel, site_rel, to_dev, to_host, parity_of, torch, TOL, SITE_TOL

pytestmark = pytest.mark.gpu

# (dims, Ls, nrhs): several tiles, ragged last tile for ns >= 16 (Vh = 72 = 8 * 9)
CASES = [((4, 4, 4, 4), 8, 1), ((6, 2, 2, 6), 6, 1), ((4, 4, 4, 4), 5, 3)]


def _setup(dims, Ls, nrhs, mf=0.05, seed=1, eps=0.3, recon=18):
    m = lib()
    U = inputs.gauge_links(dims, eps, seed)
    ctx = m.Context(dims, Ls, mf=mf, recon=recon)
    ctx.load_gauge(U)
    psi = inputs.gaussian_spinor5d(dims, Ls, seed + 100, nrhs=nrhs)
    p = MobiusParams(Ls=Ls, mf=mf)
    return m, ctx, U, dirac.boundary_links(U, -1.0), psi, p


def _gpu_apply(m, ctx, op, prec, psi, nrhs):
    nb = ctx.field_bytes(prec, nrhs)
    fin = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    fout = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    d = to_dev(psi)
    m.mdwf_pack(ctx.h, d, fin, m.PRECS[prec], nrhs)
    m.mdwf_apply(ctx.h, m.OP[op], m.PRECS[prec], fin, fout, nrhs)
    out = torch.zeros_like(d)
    m.mdwf_unpack(ctx.h, fout, out, m.PRECS[prec], nrhs)
    torch.cuda.synchronize()
    return to_host(out)


def _oracle(op, Ub, psi, p, par):
    e = lambda f: dirac.on_parity(f, par, 0)
    o = lambda f: dirac.on_parity(f, par, 1)
    if op == "HOP_EO":
        return e(dirac.hop(Ub, o(psi)))
    if op == "HOP_OE":
        return o(dirac.hop(Ub, e(psi)))
    if op == "HOP_EO_DAG":
        return e(dirac.hop(Ub, o(psi), dagger=True))
    if op == "HOP_OE_DAG":
        return o(dirac.hop(Ub, e(psi), dagger=True))
    if op in ("D5", "M5", "M5INV"):
        return dirac.s_op(p, {"D5": "D5", "M5": "A5", "M5INV": "A5inv"}[op], psi)
    if op in ("D5_DAG", "M5_DAG", "M5INV_DAG"):
        return dirac.s_op(p, {"D5_DAG": "D5", "M5_DAG": "A5", "M5INV_DAG": "A5inv"}[op], psi, dagger=True)
    if op == "HOP_EO_M5INV":
        return e(dirac.s_op(p, "A5inv", dirac.hop(Ub, o(psi))))
    if op == "HOP_OE_M5INV":
        return o(dirac.s_op(p, "A5inv", dirac.hop(Ub, e(psi))))
    if op == "MPC":
        return dirac.mpc(Ub, o(psi), p)
    if op == "MPC_DAG":
        return dirac.mpc_dag(Ub, o(psi), p)
    if op == "MDAGM":
        return dirac.mpc_dag(Ub, dirac.mpc(Ub, o(psi), p), p)
    if op == "MPC_SYM":
        return dirac.mpc_sym(Ub, o(psi), p)
    if op == "MPC_SYM_DAG":
        return dirac.mpc_sym_dag(Ub, o(psi), p)
    if op == "FULL_D":
        return dirac.mobius(Ub, psi, p)
    if op == "FULL_D_DAG":
        return dirac.mobius(Ub, psi, p, dagger=True)
    raise ValueError(op)


def _mask(op, par, shape):
    """Which parity halves an op writes (the rest of `out` stays zero)."""
    if op in ("HOP_EO", "HOP_EO_DAG", "HOP_EO_M5INV"):
        keep = par == 0
    elif op in ("HOP_OE", "HOP_OE_DAG", "HOP_OE_M5INV", "MPC", "MPC_DAG", "MDAGM", "MPC_SYM", "MPC_SYM_DAG"):
        keep = par == 1
    else:
        return None
    return keep


ALL_OPS = ["HOP_EO", "HOP_OE", "HOP_EO_DAG", "HOP_OE_DAG", "D5", "D5_DAG", "M5", "M5_DAG", "M5INV",
           "M5INV_DAG", "HOP_EO_M5INV", "HOP_OE_M5INV", "MPC", "MPC_DAG", "MDAGM", "FULL_D", "FULL_D_DAG",
           "MPC_SYM", "MPC_SYM_DAG"]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16", "i16", "f64e"])
def test_apply_parity(case, prec, monkeypatch):
    dims, Ls, nrhs = case
    if dims == (6, 2, 2, 6):
        monkeypatch.setenv("MDWF_FORCE_NS", "16")
    m, ctx, U, Ub, psi, p = _setup(dims, Ls, nrhs)
    par = parity_of(dims)
    for op in ALL_OPS:
        got = _gpu_apply(m, ctx, op, prec, psi, nrhs)
        ref = np.stack([_oracle(op, Ub, psi[r], p, par) for r in range(nrhs)])
        keep = _mask(op, par, ref.shape)
        if keep is not None:
            # untouched half stays zero
            other = np.broadcast_to((~keep)[None, None, ..., None, None], got.shape)
            assert not np.any(got[other]), op
        err = rel(got, ref)
        assert err <= TOL[prec], (op, prec, err)
        serr = site_rel(got, ref, keep)
        assert serr <= SITE_TOL[prec], (op, prec, "per site", serr)


TC_CASES = CASES + [((4, 4, 4, 8), 12, 12), ((4, 2, 2, 4), 10, 2)]


@pytest.mark.parametrize("prec", ["f16", "bf16"])
@pytest.mark.parametrize("force_ns", [None, "1", "16"])
def test_tensor_core_hop_matches_oracle(prec, force_ns, monkeypatch):
    """The tcgen05 hop kernel (MDWF_TC=1) on every hop-based op: several tiles, a ragged
    last tile (16 sites per CTA on a 72-site half lattice), Ls 5..12, up to 12 RHS
    (144 accumulator columns per site, several 16-column TMEM loads)."""
    monkeypatch.setenv("MDWF_TC", "1")
    if force_ns:
        monkeypatch.setenv("MDWF_FORCE_NS", force_ns)
    for case in TC_CASES:
        dims, Ls, nrhs = case
        if force_ns == "16" and nrhs * Ls > 16:
            continue          # 16 sites of more than 16 columns exceed the tensor-memory budget
        m, ctx, U, Ub, psi, p = _setup(dims, Ls, nrhs)
        par = parity_of(dims)
        for op in ["HOP_EO", "HOP_OE_DAG", "HOP_OE_M5INV", "MPC", "MPC_DAG", "MDAGM", "FULL_D", "FULL_D_DAG",
                   "MPC_SYM", "MPC_SYM_DAG"]:
            got = _gpu_apply(m, ctx, op, prec, psi, nrhs)
            ref = np.stack([_oracle(op, Ub, psi[r], p, par) for r in range(nrhs)])
            keep = _mask(op, par, ref.shape)
            assert rel(got, ref) <= TOL[prec], (op, prec, case)
            assert site_rel(got, ref, keep) <= SITE_TOL[prec], (op, prec, case, "per site")


PAIR_BIT = 1 << 18   # tuner value flag of the paired-column hop kernel
PAIR_CASES = [((4, 4, 4, 4), 8, 1), ((6, 2, 2, 6), 6, 1), ((4, 4, 4, 8), 12, 12), ((4, 2, 2, 4), 10, 2)]
PAIR_OPS = ["HOP_EO", "HOP_OE_DAG", "HOP_OE_M5INV", "MPC", "MPC_DAG", "MDAGM", "FULL_D", "FULL_D_DAG",
            "MPC_SYM", "MPC_SYM_DAG"]


BULK_BIT = 1 << 19   # tuner value flag of the bulk-staged hop kernel


@pytest.mark.parametrize("variant,prec", [("pair", "f32"), ("pair", "f16"), ("pair", "bf16"), ("pair", "i16"),
                                          ("bulk", "f16"), ("bulk", "bf16"), ("bulk", "i16")])
@pytest.mark.parametrize("ns", [1, 3, 16])
def test_variant_hop_matches_oracle_and_single_column(variant, prec, ns, monkeypatch):
    """The paired-column hop kernel (two columns per thread on packed FP32 pairs) and the
    bulk-staged one (neighbour rows copied into shared memory by bulk asynchronous copies)
    on every hop-based op: parity with the oracle, and bit-identical to the single-column
    kernel with the same sites per CTA (same roundings in the same order).  Cases: several
    tiles, ragged last tiles (3 and 16 sites per CTA on 72- and 32-site half lattices),
    1..12 RHS."""
    monkeypatch.setenv("MDWF_TC", "0")
    flag = PAIR_BIT if variant == "pair" else BULK_BIT
    for dims, Ls, nrhs in PAIR_CASES:
        if ns * nrhs * Ls > 256:
            continue      # more threads than a CTA of the single-column kernel takes
        m, ctx, U, Ub, psi, p = _setup(dims, Ls, nrhs)
        par = parity_of(dims)
        for op in PAIR_OPS:
            monkeypatch.setenv("MDWF_FORCE_NS", str(ns))
            single = _gpu_apply(m, ctx, op, prec, psi, nrhs)
            monkeypatch.setenv("MDWF_FORCE_NS", str(flag | ns))
            got = _gpu_apply(m, ctx, op, prec, psi, nrhs)
            ref = np.stack([_oracle(op, Ub, psi[r], p, par) for r in range(nrhs)])
            keep = _mask(op, par, ref.shape)
            assert rel(got, ref) <= TOL[prec], (op, prec, dims, Ls, nrhs)
            assert site_rel(got, ref, keep) <= SITE_TOL[prec], (op, prec, dims, Ls, nrhs, "per site")
            assert np.array_equal(got, single), (op, prec, dims, Ls, nrhs, float(np.abs(got - single).max()))


def test_paired_hop_chosen_by_tuner_only_for_even_columns(monkeypatch):
    """nrhs * Ls odd: the paired kernel is no candidate, a forced pair value falls back to
    the tuner, and the result is still right."""
    monkeypatch.setenv("MDWF_TC", "0")
    monkeypatch.setenv("MDWF_FORCE_NS", str(PAIR_BIT | 4))
    dims, Ls, nrhs = (4, 4, 4, 4), 5, 3
    m, ctx, U, Ub, psi, p = _setup(dims, Ls, nrhs)
    par = parity_of(dims)
    got = _gpu_apply(m, ctx, "MPC", "f16", psi, nrhs)
    ref = np.stack([_oracle("MPC", Ub, psi[r], p, par) for r in range(nrhs)])
    assert rel(got, ref) <= TOL["f16"]
    assert not any((v >> 18) & 1 for _, v, _ in ctx.tune_entries())


@pytest.mark.parametrize("prec", ["f16", "bf16"])
def test_tensor_core_hop_recon12(prec, monkeypatch):
    """12-real links (third row rebuilt in the tensor-core kernel's link-matrix build,
    with the time-boundary sign) against the 18-real result."""
    monkeypatch.setenv("MDWF_TC", "1")
    dims, Ls = (4, 4, 4, 4), 6
    outs = []
    for recon in (18, 12):
        m, ctx, U, Ub, psi, p = _setup(dims, Ls, 1, recon=recon)
        outs.append(_gpu_apply(m, ctx, "MPC", prec, psi, 1))
    par = parity_of(dims)
    ref = _oracle("MPC", Ub, psi[0], p, par)
    assert rel(outs[1][0], ref) <= TOL[prec] and rel(outs[0][0], ref) <= TOL[prec]


def test_recon12_matches_recon18():
    m = lib()
    dims, Ls = (4, 4, 4, 4), 6
    for prec in ("f64", "f32", "f16"):
        outs = []
        for recon in (18, 12):
            m_, ctx, U, Ub, psi, p = _setup(dims, Ls, 1, recon=recon)
            outs.append(_gpu_apply(m, ctx, "FULL_D", prec, psi, 1))
        assert rel(outs[1], outs[0]) <= {"f64": 1e-14, "f32": 1e-6, "f16": 2e-3}[prec]


def _internal_half_f16(raw, ctx, nrhs, parity):
    """Decode the documented internal F16 layout of one parity half into
    (halves [vh, nrhs, Ls, 24] in [colour][spin][re,im] order, norms [vh, nrhs, Ls])."""
    X, Y, Z, T = ctx.dims
    vh = X * Y * Z * T // 2
    Ls = ctx.Ls
    W = nrhs * Ls
    dbytes = vh * 3 * W * 16
    data = raw[parity * dbytes:(parity + 1) * dbytes].view(np.float16).reshape(vh, 3, nrhs, Ls, 8)
    h = np.transpose(data, (0, 2, 3, 1, 4)).reshape(vh, nrhs, Ls, 24)
    nb = vh * W * 4
    norms = raw[2 * dbytes + parity * nb: 2 * dbytes + (parity + 1) * nb].view(np.float32).reshape(vh, nrhs, Ls)
    return h, norms


def test_pack_f16_bit_exact_and_roundtrip():
    m = lib()
    dims, Ls, nrhs = (4, 4, 2, 4), 4, 2
    ctx = m.Context(dims, Ls)
    psi = inputs.gaussian_spinor5d(dims, Ls, 7, nrhs=nrhs)
    psi[0, 1, 0, 0, 0, 0] = 0.0        # an all-zero 5D site
    psi[1, 2, 1] *= 1e-30              # tiny magnitudes
    d = to_dev(psi)
    nb = ctx.field_bytes("f16", nrhs)
    buf = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    m.mdwf_pack(ctx.h, d, buf, m.PRECS["f16"], nrhs)
    raw = buf.cpu().numpy()
    X, Y, Z, T = dims
    par = parity_of(dims)
    for parity in (0, 1):
        h, n = _internal_half_f16(raw, ctx, nrhs, parity)
        # site order of the half: x_cb = full index // 2 over sites of this parity
        t, z, y, x = np.nonzero(par == parity)
        order = np.argsort(((t * Z + z) * Y + y) * X + x)
        t, z, y, x = t[order], z[order], y[order], x[order]
        sites = psi[:, :, t, z, y, x]                 # [nrhs, Ls, vh, spin, colour]
        reals = np.stack([sites.real, sites.imag], -1)  # [..., spin, colour, 2]
        reals = np.transpose(reals, (2, 0, 1, 4, 3, 5)).reshape(len(t), nrhs, Ls, 24)
        eh, en = storage.quantize_f16(reals)
        assert np.array_equal(n, en)
        assert np.array_equal(h.view(np.uint16), eh.view(np.uint16))
    # FP64 round trip is bit-exact
    nb64 = ctx.field_bytes("f64", nrhs)
    b64 = torch.zeros(nb64, dtype=torch.uint8, device="cuda")
    m.mdwf_pack(ctx.h, d, b64, 0, nrhs)
    back = torch.zeros_like(d)
    m.mdwf_unpack(ctx.h, b64, back, 0, nrhs)
    assert np.array_equal(to_host(back), psi)
    # BF16 values are the nearest-even 8-bit roundings
    nbb = ctx.field_bytes("bf16", nrhs)
    bb = torch.zeros(nbb, dtype=torch.uint8, device="cuda")
    m.mdwf_pack(ctx.h, d, bb, 3, nrhs)
    m.mdwf_unpack(ctx.h, bb, back, 3, nrhs)
    got = to_host(back)
    assert np.array_equal(got.real, storage.round_bf16(psi.real))
    assert np.array_equal(got.imag, storage.round_bf16(psi.imag))


def test_pack_i16_bit_exact_and_roundtrip():
    """16-bit fixed point: the stored int16 and norms are the oracle's quantisation, and
    unpacking gives the oracle's q * (norm / 32767) exactly."""
    m = lib()
    dims, Ls, nrhs = (4, 4, 2, 4), 4, 2
    ctx = m.Context(dims, Ls)
    psi = inputs.gaussian_spinor5d(dims, Ls, 8, nrhs=nrhs)
    psi[0, 1, 0, 0, 0, 0] = 0.0        # an all-zero 5D site
    psi[1, 2, 1] *= 1e-30              # tiny magnitudes
    d = to_dev(psi)
    buf = torch.zeros(ctx.field_bytes("i16", nrhs), dtype=torch.uint8, device="cuda")
    m.mdwf_pack(ctx.h, d, buf, m.PRECS["i16"], nrhs)
    raw = buf.cpu().numpy()
    X, Y, Z, T = dims
    par = parity_of(dims)
    for parity in (0, 1):
        h, n = _internal_half_f16(raw, ctx, nrhs, parity)   # same 16-bit layout
        t, z, y, x = np.nonzero(par == parity)
        order = np.argsort(((t * Z + z) * Y + y) * X + x)
        t, z, y, x = t[order], z[order], y[order], x[order]
        sites = psi[:, :, t, z, y, x]
        reals = np.stack([sites.real, sites.imag], -1)
        reals = np.transpose(reals, (2, 0, 1, 4, 3, 5)).reshape(len(t), nrhs, Ls, 24)
        eq, en = storage.quantize_i16(reals)
        assert np.array_equal(n, en)
        assert np.array_equal(h.view(np.int16), eq)
    back = torch.zeros_like(d)
    m.mdwf_unpack(ctx.h, buf, back, m.PRECS["i16"], nrhs)
    got = to_host(back)
    for parity in (0, 1):
        h, n = _internal_half_f16(raw, ctx, nrhs, parity)
        t, z, y, x = np.nonzero(par == parity)
        order = np.argsort(((t * Z + z) * Y + y) * X + x)
        t, z, y, x = t[order], z[order], y[order], x[order]
        ev = storage.dequantize_i16(h.view(np.int16), n).reshape(len(t), nrhs, Ls, 3, 4, 2)
        ev = np.transpose(ev, (1, 2, 0, 4, 3, 5))           # [nrhs, Ls, vh, spin, colour, 2]
        g = got[:, :, t, z, y, x]
        assert np.array_equal(g.real, ev[..., 0]) and np.array_equal(g.imag, ev[..., 1])
