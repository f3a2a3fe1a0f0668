"""The allocation-free nucleon contraction (mdwf_contract_nucleon_noalloc) gives what the
regular entry point gives, on two calls in a row, through the C ABI.

It exists for callers that cannot allocate device memory (graph capture, pool-owned
device memory, pre-planned memory budgets); its scratch is a fixed array in the library.
This file is collected last so that a stop-at-first-failure run has run everything else.
"""
import numpy as np
import pytest

from gpu_common import lib, rel, to_dev, to_host, torch

pytestmark = pytest.mark.gpu


def _props(ctx, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((12,) + ctx.shape4d() + (2,)).view(np.complex128)[..., 0] for _ in range(3)]


def test_noalloc_matches_regular_twice():
    m = lib()
    ctx = m.Context((4, 4, 2, 8), 4)
    T = ctx.dims[3]
    for call, seed in enumerate((21, 22)):
        props = [to_dev(p) for p in _props(ctx, seed)]
        ref = torch.empty(T, dtype=torch.complex128, device="cuda")
        m.mdwf_contract_nucleon(ctx.h, *props, ref)
        got = torch.full((T,), np.nan, dtype=torch.complex128, device="cuda")
        m.mdwf_contract_nucleon_noalloc(ctx.h, *props, got)
        torch.cuda.synchronize()
        assert rel(to_host(got), to_host(ref)) <= 1e-13, call


def test_noalloc_rejects_oversized_lattice():
    m = lib()
    ctx = m.Context((64, 64, 64, 4), 4)   # 1048576 sites > 524288
    small = torch.zeros(16, dtype=torch.complex128, device="cuda")
    with pytest.raises(m.MdwfError) as e:
        m.mdwf_contract_nucleon_noalloc(ctx.h, small, small, small, small)
    assert e.value.code == m.MDWF_ERR_ARG
    assert "at most 524288" in str(e.value)


def test_noalloc_captured_in_graph_and_allocates_nothing():
    """The use it exists for: after one warm call, the call is captured in a CUDA graph
    on a side stream and replayed with new propagator contents; and a warm call leaves the
    device's free memory unchanged."""
    m = lib()
    ctx = m.Context((4, 4, 2, 8), 4)
    T = ctx.dims[3]
    props = [to_dev(p) for p in _props(ctx, 31)]
    got = torch.zeros(T, dtype=torch.complex128, device="cuda")
    ref = torch.empty(T, dtype=torch.complex128, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        m.mdwf_contract_nucleon_noalloc(ctx.h, *props, got, stream=s)   # warm call (set-up)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    with torch.cuda.stream(s):
        m.mdwf_contract_nucleon_noalloc(ctx.h, *props, got, stream=s)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        m.mdwf_contract_nucleon_noalloc(ctx.h, *props, got, stream=s)
    for seed in (32, 33):
        for dst, src in zip(props, _props(ctx, seed)):
            dst.copy_(to_dev(src))
        got.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        m.mdwf_contract_nucleon(ctx.h, *props, ref)
        torch.cuda.synchronize()
        assert rel(to_host(got), to_host(ref)) <= 1e-13, seed
