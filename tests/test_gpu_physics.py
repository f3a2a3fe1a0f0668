"""GPU parity of the propagator pieces around the solve: 4D source injection
D(1) P (b at s=0), projection q = P_- y_0 + P_+ y_{Ls-1}, the Feynman-Hellmann source
gamma_3 gamma_5 q and the nucleon two-point contraction, against the oracle."""
import numpy as np
import pytest

import inputs
from oracle import dirac, solve, hadron
from oracle.dirac import MobiusParams
from gpu_common import lib, rel, to_dev, to_host, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("emulation", [True, False])
def test_source_projection_fh(emulation):
    """emulation: the injection's FP64 hops in emulated FP64 (the default) or native."""
    m = lib()
    dims, Ls, mf = (4, 4, 2, 6), 6, 0.05
    U = inputs.gauge_links(dims, 0.3, 9)
    Ub = dirac.boundary_links(U, -1.0)
    p = MobiusParams(Ls=Ls, mf=mf)
    ctx = m.Context(dims, Ls, mf=mf, f64_emulation=emulation)
    ctx.load_gauge(U)
    rng = np.random.default_rng(3)
    b4 = rng.standard_normal((2,) + ctx.shape4d() + (2,)).view(np.complex128)[..., 0]
    eta = to_host(ctx.make_source_4d(to_dev(b4), nrhs=2))
    for r in range(2):
        assert rel(eta[r], hadron.inject_source(Ub, b4[r], p)) <= 1e-13
    y = inputs.gaussian_spinor5d(dims, Ls, 4, nrhs=2)
    q = to_host(ctx.project_4d(to_dev(y), nrhs=2))
    for r in range(2):
        assert np.array_equal(q[r], hadron.project_4d(y[r]))
    f = to_host(ctx.fh_source(to_dev(q), nrhs=2))
    for r in range(2):
        assert rel(f[r], hadron.fh_source(q[r])) <= 1e-15


def test_propagator_call_matches_chain(monkeypatch):
    """mdwf_propagator (injection, batched solve and projection chained on the device, one
    C-ABI call) gives bit for bit the columns of the three separate calls, on the host and
    on the device path, and the oracle's propagator to the solve's accuracy."""
    monkeypatch.setenv("MDWF_TC", "0")
    m = lib()
    dims, Ls, mf = (4, 4, 2, 6), 6, 0.05
    U = inputs.gauge_links(dims, 0.3, 9)
    Ub = dirac.boundary_links(U, -1.0)
    p = MobiusParams(Ls=Ls, mf=mf)
    ctx = m.Context(dims, Ls, mf=mf)
    ctx.load_gauge(U)
    b4 = np.stack([inputs.point_source4d(dims, 0, 0), inputs.point_source4d(dims, 3, 2)])
    eta = ctx.make_source_4d(to_dev(b4), nrhs=2)
    y, infos_c = ctx.solve_multi(eta, tol=1e-10, sloppy="f16")
    q_chain = to_host(ctx.project_4d(y, nrhs=2))
    q_dev, infos = ctx.propagator(to_dev(b4), nrhs=2, tol=1e-10, sloppy="f16")
    q_host, infos_h = ctx.propagator(b4, nrhs=2, tol=1e-10, sloppy="f16")
    assert all(i.status == 0 and i.true_residual <= 1e-10 for i in infos + infos_h)
    assert [i.iterations for i in infos] == [i.iterations for i in infos_c]
    assert np.array_equal(to_host(q_dev), q_chain)
    assert np.array_equal(q_host, q_chain)
    for r in range(2):
        yo, _, _ = solve.solve_eo(Ub, hadron.inject_source(Ub, b4[r], p), p, tol=1e-12)
        assert rel(q_host[r], hadron.project_4d(yo)) <= 1e-8


def _cols_to_oracle(S):
    """[12][t,z,y,x,spin,colour] columns -> oracle layout [t,z,y,x,spin,colour,spin',colour']."""
    T, Z, Y, X = S.shape[1:5]
    return np.transpose(S.reshape(4, 3, T, Z, Y, X, 4, 3), (2, 3, 4, 5, 6, 7, 0, 1))


def test_nucleon_contraction_random_propagators():
    m = lib()
    dims = (2, 2, 2, 4)
    ctx = m.Context(dims, 4)
    rng = np.random.default_rng(11)
    props = [rng.standard_normal((12,) + ctx.shape4d() + (2,)).view(np.complex128)[..., 0] for _ in range(3)]
    got = to_host(ctx.contract_nucleon(*[to_dev(s) for s in props]))
    ref = hadron.nucleon_2pt(*[_cols_to_oracle(s) for s in props])
    assert rel(got, ref) <= 1e-13
    # host buffers give the same numbers
    got_h = ctx.contract_nucleon(*props)
    assert np.array_equal(got_h, got)


def test_point_propagator_fh_chain():
    """12 point-source columns through inject -> solve_multi -> project, the FH sequential
    solve, and the contraction, vs the oracle chain."""
    m = lib()
    dims, Ls, mf = (2, 2, 2, 4), 4, 0.1
    U = inputs.gauge_links(dims, 0.3, 3)
    Ub = dirac.boundary_links(U, -1.0)
    p = MobiusParams(Ls=Ls, mf=mf)
    ctx = m.Context(dims, Ls, mf=mf)
    ctx.load_gauge(U)
    b4 = np.stack([inputs.point_source4d(dims, k // 3, k % 3) for k in range(12)])
    eta = ctx.make_source_4d(to_dev(b4), nrhs=12)
    y, infos = ctx.solve_multi(eta, tol=1e-11, sloppy="f16")
    S = ctx.project_4d(y, nrhs=12)
    yf, infos_f = ctx.solve_multi(ctx.make_source_4d(ctx.fh_source(S, nrhs=12), nrhs=12), tol=1e-11, sloppy="f16")
    SF = ctx.project_4d(yf, nrhs=12)
    S_h, SF_h = to_host(S), to_host(SF)
    # oracle chain
    So = np.zeros_like(S_h)
    SFo = np.zeros_like(S_h)
    for k in range(12):
        yo, _, _ = solve.solve_eo(Ub, hadron.inject_source(Ub, b4[k], p), p, tol=1e-12)
        So[k] = hadron.project_4d(yo)
        yfo, _, _ = solve.solve_eo(Ub, hadron.inject_source(Ub, hadron.fh_source(So[k]), p), p, tol=1e-12)
        SFo[k] = hadron.project_4d(yfo)
    assert rel(S_h, So) <= 1e-8
    assert rel(SF_h, SFo) <= 1e-8
    C = to_host(ctx.contract_nucleon(S, S, S))
    Co = hadron.nucleon_2pt(*[_cols_to_oracle(So)] * 3)
    assert rel(C, Co) <= 1e-8
    CF = to_host(ctx.contract_nucleon(SF, S, S)) + to_host(ctx.contract_nucleon(S, S, SF))
    CFo = hadron.nucleon_2pt(_cols_to_oracle(SFo), _cols_to_oracle(So), _cols_to_oracle(So)) + \
        hadron.nucleon_2pt(_cols_to_oracle(So), _cols_to_oracle(So), _cols_to_oracle(SFo))
    assert rel(CF, CFo) <= 1e-8
    # the effective-coupling estimator of the product against the oracle's on the oracle's
    # correlators (bit-level), and on the GPU correlators within their parity bound
    assert np.max(np.abs(m.mdwf_fh_effective_coupling(Co, CFo) - hadron.fh_effective_coupling(Co, CFo))) <= \
        1e-13 * np.max(np.abs(hadron.fh_effective_coupling(Co, CFo)))
    g, go = m.mdwf_fh_effective_coupling(C, CF), hadron.fh_effective_coupling(Co, CFo)
    assert np.max(np.abs(g - go)) <= 1e-6 * max(1.0, np.max(np.abs(go)))


def test_gauge_errors():
    m = lib()
    dims = (4, 4, 4, 4)
    ctx = m.Context(dims, 4)
    U = inputs.gauge_links(dims, 0.2, 1)
    U[1, 2, 3, 0, 2] *= 1.01   # not unitary
    with pytest.raises(m.MdwfError) as e:
        ctx.load_gauge(U)
    assert e.value.code == m.MDWF_ERR_NOT_SU3
    nb = ctx.field_bytes("f64")
    a = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    b = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    with pytest.raises(m.MdwfError) as e:
        m.mdwf_apply(ctx.h, m.OP["MPC"], 0, a, b, 1)
    assert e.value.code == m.MDWF_ERR_STATE
