"""Runtime behaviour on the GPU: the autotuner (cache file written and re-read, a
corrupted cache ignored, tuned results equal to untuned ones thanks to backup/restore of
in-place outputs), run-to-run bitwise determinism of the FP64-accumulated reductions, and
host-detected failures (NaN source -> breakdown status) that fault no GPU."""
import json
import os
import numpy as np
import pytest

import inputs
from gpu_common import lib, rel, to_dev, to_host, torch

pytestmark = pytest.mark.gpu


def _ctx(m, dims=(4, 4, 4, 8), Ls=6, mf=0.05, seed=2):
    ctx = m.Context(dims, Ls, mf=mf)
    ctx.load_gauge(inputs.gauge_links(dims, 0.3, seed))
    return ctx


def test_tuner_cache_roundtrip_and_equivalence(tmp_path, monkeypatch):
    m = lib()
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("MDWF_TUNE_CACHE", str(cache))
    monkeypatch.setenv("MDWF_TUNE", "1")
    ctx = _ctx(m)
    b = to_dev(inputs.gaussian_spinor5d(ctx.dims, ctx.Ls, 3))
    x1, i1 = ctx.solve(b, sloppy="f16", tol=1e-10)
    entries = ctx.tune_entries()
    assert len(entries) >= 5 and all(ns >= 1 and ms > 0 for _, ns, ms in entries)
    data = json.loads(cache.read_text())
    assert set(data) == {k for k, _, _ in entries}
    # a second context reads the cache and reproduces the solve bit for bit
    ctx2 = _ctx(m)
    assert {k for k, _, _ in ctx2.tune_entries()} == set(data)
    x2, i2 = ctx2.solve(b, sloppy="f16", tol=1e-10)
    assert i2.iterations == i1.iterations
    assert torch.equal(x1, x2)
    # untuned (tuning off, defaults) gives the same answer to solver accuracy
    monkeypatch.setenv("MDWF_TUNE", "0")
    monkeypatch.delenv("MDWF_TUNE_CACHE")
    ctx3 = _ctx(m)
    x3, i3 = ctx3.solve(b, sloppy="f16", tol=1e-10)
    assert rel(to_host(x3), to_host(x1)) < 1e-8


def test_corrupted_tune_cache_is_ignored(tmp_path, monkeypatch):
    m = lib()
    cache = tmp_path / "bad.json"
    cache.write_text('{\n  "hop|4x4x4x8|Ls6|n1|p2|garbage": {"ns": "x", "ms": 1},\n  "junk\n  {"ns": 9999}\n}')
    monkeypatch.setenv("MDWF_TUNE_CACHE", str(cache))
    ctx = _ctx(m)
    assert ctx.tune_entries() == []
    b = to_dev(inputs.gaussian_spinor5d(ctx.dims, ctx.Ls, 3))
    x, info = ctx.solve(b, sloppy="f64", tol=1e-10)
    assert info.true_residual <= 1e-10


def test_reductions_bitwise_deterministic(monkeypatch):
    m = lib()
    monkeypatch.setenv("MDWF_TUNE", "0")
    ctx = _ctx(m)
    b = to_dev(inputs.gaussian_spinor5d(ctx.dims, ctx.Ls, 4))
    outs = [ctx.solve(b, sloppy=s, tol=1e-10) for s in ("f64", "f64", "f16", "f16")]
    assert torch.equal(outs[0][0], outs[1][0]) and outs[0][1].iterations == outs[1][1].iterations
    assert torch.equal(outs[2][0], outs[3][0]) and outs[2][1].iterations == outs[3][1].iterations


def test_nan_source_reports_breakdown():
    """A NaN poked into a host source buffer before upload is detected on the host from
    the device-resident CG scalars; nothing faults."""
    m = lib()
    ctx = _ctx(m)
    b = inputs.gaussian_spinor5d(ctx.dims, ctx.Ls, 5)
    b[2, 1, 1, 1, 1, 0, 0] = np.nan
    with pytest.raises(m.MdwfError) as e:
        ctx.solve(b, sloppy="f16", tol=1e-10)
    assert e.value.code == m.MDWF_ERR_BREAKDOWN
    # the context stays usable
    b[2, 1, 1, 1, 1, 0, 0] = 0.0
    x, info = ctx.solve(b, sloppy="f16", tol=1e-10)
    assert info.true_residual <= 1e-10


def test_graph_and_eager_iterations_agree():
    m = lib()
    ctx = _ctx(m)
    b = to_dev(inputs.gaussian_spinor5d(ctx.dims, ctx.Ls, 6))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        xg, ig = ctx.solve(b, sloppy="f16", tol=1e-10, use_graph=True, stream=s)
        xe, ie = ctx.solve(b, sloppy="f16", tol=1e-10, use_graph=False, stream=s)
    torch.cuda.synchronize()
    assert ig.iterations == ie.iterations
    assert torch.equal(xg, xe)
    assert ctx.launch_count() > 0 and ctx.algorithmic_bytes() > 0


def test_graph_survives_reduction_buffer_growth():
    """A captured CG graph holds the reduction-partials buffer's address.  A 12-RHS solve
    in between needs a larger buffer; the graph replayed afterwards must not write into the
    freed one: the third solve (graph) equals an eager solve bit for bit."""
    m = lib()
    ctx = _ctx(m, dims=(4, 4, 4, 8), Ls=4)
    b1 = to_dev(inputs.gaussian_spinor5d(ctx.dims, ctx.Ls, 11))
    b12 = to_dev(inputs.gaussian_spinor5d(ctx.dims, ctx.Ls, 12, nrhs=12))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        x0, i0 = ctx.solve(b1, sloppy="f16", tol=1e-10, use_graph=True, stream=s)
        xm, im = ctx.solve_multi(b12, sloppy="f16", tol=1e-10, use_graph=True, stream=s)
        xg, ig = ctx.solve(b1, sloppy="f16", tol=1e-10, use_graph=True, stream=s)
        xe, ie = ctx.solve(b1, sloppy="f16", tol=1e-10, use_graph=False, stream=s)
    torch.cuda.synchronize()
    assert all(i.true_residual <= 1e-10 for i in im)
    assert ig.true_residual <= 1e-10 and ig.iterations == ie.iterations
    assert torch.equal(xg, xe) and torch.equal(x0, xe)
