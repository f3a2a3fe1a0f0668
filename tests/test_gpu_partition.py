"""T-partitioned operator on one GPU: the lattice split into 2 and 4 partitions in t,
each a context driven by its own host thread and stream, faces exchanged in-process by
the library; every operator's output is bit-identical to the undecomposed context's
(same kernels, same reals at every site), for all storage precisions and for the
single-column, the paired-column and the tcgen05 hop kernels."""
import numpy as np
import pytest

import inputs
from gpu_common import lib, to_dev, torch

pytestmark = pytest.mark.gpu

OPS = ["HOP_EO", "HOP_OE_DAG", "HOP_OE_M5INV", "MPC", "MPC_DAG", "MDAGM", "MPC_SYM", "FULL_D", "FULL_D_DAG"]


def _whole(m, ctx, op, prec, psi, nrhs):
    nb = ctx.field_bytes(prec, nrhs)
    fin = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    fout = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    m.mdwf_pack(ctx.h, psi, fin, m.PRECS[prec], nrhs)
    m.mdwf_apply(ctx.h, m.OP[op], m.PRECS[prec], fin, fout, nrhs)
    out = torch.zeros_like(psi)
    m.mdwf_unpack(ctx.h, fout, out, m.PRECS[prec], nrhs)
    torch.cuda.synchronize()
    return out


PAIR_BIT = 1 << 18   # tuner value flag of the paired-column hop kernel


@pytest.mark.parametrize("tc", ["0", "1", "pair"])
@pytest.mark.parametrize("nparts,recon", [(2, 18), (4, 18), (2, 12)])
def test_partitioned_operators_bit_identical(nparts, recon, tc, monkeypatch):
    """tc "pair": the partitions run the paired-column kernel, the undecomposed context the
    single-column one (4 sites per CTA each)."""
    monkeypatch.setenv("MDWF_TC", "0" if tc == "pair" else tc)
    monkeypatch.setenv("MDWF_TUNE", "0")
    m = lib()
    from paper_1810_01609_gb300.partition import PartitionedLattice
    dims, Ls, mf, nrhs = (4, 4, 2, 16), 6, 0.05, 2
    U = inputs.gauge_links(dims, 0.4, 21)
    whole = m.Context(dims, Ls, mf=mf, recon=recon)
    whole.load_gauge(U)
    part = PartitionedLattice(dims, Ls, nparts, mf=mf, recon=recon)
    part.load_gauge(U)
    psi = to_dev(inputs.gaussian_spinor5d(dims, Ls, 22, nrhs=nrhs))
    precs = {"1": ("f16", "bf16"), "0": ("f64", "f32", "f16", "bf16", "i16"), "pair": ("f32", "f16", "bf16", "i16")}[tc]
    for prec in precs:
        for op in OPS:
            if tc == "pair":
                monkeypatch.setenv("MDWF_FORCE_NS", "4")
            ref = _whole(m, whole, op, prec, psi, nrhs)
            if tc == "pair":
                monkeypatch.setenv("MDWF_FORCE_NS", str(PAIR_BIT | 4))
            got = part.apply(op, prec, psi, nrhs)
            assert torch.equal(got, ref), (op, prec, nparts, float((got - ref).abs().max()))


def test_partitioned_context_rejects_solve():
    m = lib()
    ctx = m.Context((4, 4, 4, 4), 4, t_ranks=2, t_rank=0)
    from paper_1810_01609_gb300.partition import split_links
    ctx.load_gauge(split_links(inputs.gauge_links((4, 4, 4, 8), 0.3, 3), 2)[0])
    b = torch.zeros((4, 4, 4, 4, 4, 4, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(m.MdwfError) as e:
        ctx.solve(b)
    assert e.value.code == m.MDWF_ERR_STATE
