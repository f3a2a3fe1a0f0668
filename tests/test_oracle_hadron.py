"""Pins of oracle.hadron: Feynman-Hellmann propagator vs dense S (sum Gamma) S, nucleon
trace formula vs a brute-force Wick sum over Grassmann pairings, gauge invariance."""
import itertools
import numpy as np

import inputs
from oracle import dirac, hadron, solve
from oracle.dirac import MobiusParams
from oracle.gamma import GAMMA, GAMMA5, CHARGE_C, ID4
from _dense import dense, crandn
from test_oracle_wilson import gauge_transform, random_gauge


def _prop_point(Ub, p, dims, tol=1e-12):
    """Full 4D propagator S[t,z,y,x,s,c,s',c'] from the origin through the oracle route."""
    X, Y, Z, T = dims
    S = np.zeros((T, Z, Y, X, 4, 3, 4, 3), dtype=np.complex128)
    for sp in range(4):
        for co in range(3):
            b4 = inputs.point_source4d(dims, sp, co)
            y, _, _ = solve.solve_eo(Ub, hadron.inject_source(Ub, b4, p), p, tol=tol)
            S[..., sp, co] = hadron.project_4d(y)
    return S


def test_fh_propagator_matches_dense():
    dims = (2, 2, 2, 4)
    X, Y, Z, T = dims
    p = MobiusParams(Ls=4, mf=0.1)
    Ub = dirac.boundary_links(inputs.gauge_links(dims, 0.3, 3), p.t_bc)
    sh4 = (T, Z, Y, X, 4, 3)
    sh5 = (p.Ls,) + sh4
    n4 = int(np.prod(sh4))
    Dm = dense(lambda v: dirac.mobius(Ub, v, p), sh5)
    D1 = dense(lambda v: dirac.mobius(Ub, v, p, mf=1.0), sh5)
    W = np.stack([hadron.embed_wall(np.eye(n4)[i].reshape(sh4), p.Ls).ravel()
                  for i in range(n4)], axis=1)
    Ysol = np.linalg.solve(Dm, D1 @ W)
    S = np.stack([hadron.project_4d(Ysol[:, i].reshape(sh5)).ravel() for i in range(n4)], 1)
    Gam = np.kron(np.eye(X * Y * Z * T), np.kron(GAMMA[2] @ GAMMA5, np.eye(3)))
    SFH = S @ Gam @ S
    for sp, co in ((0, 0), (3, 2)):
        b4 = inputs.point_source4d(dims, sp, co)
        y, _, _ = solve.solve_eo(Ub, hadron.inject_source(Ub, b4, p), p, tol=1e-13)
        q = hadron.project_4d(y)
        yf, _, _ = solve.solve_eo(Ub, hadron.inject_source(Ub, hadron.fh_source(q), p), p,
                                  tol=1e-13)
        qf = hadron.project_4d(yf)
        col = b4.ravel().argmax()
        assert np.linalg.norm(q.ravel() - S[:, col]) < 1e-10 * np.linalg.norm(S[:, col])
        assert np.linalg.norm(qf.ravel() - SFH[:, col]) < 1e-9 * np.linalg.norm(SFH[:, col])


def _pair_sign(seq, pairs):
    """Sign of the permutation that brings each (quark, antiquark) pair of positions
    next to each other as q qbar q qbar ... (Grassmann reordering)."""
    order = [i for pr in pairs for i in pr]
    sign = 1
    o = list(order)
    for i in range(len(o)):
        for j in range(i + 1, len(o)):
            if o[i] > o[j]:
                sign = -sign
    return sign


def test_nucleon_contraction_brute_force_wick():
    rng = np.random.default_rng(8)
    T = 2
    Sdim = (T, 1, 1, 1, 4, 3, 4, 3)
    U1, Dd, U2 = crandn(rng, Sdim), crandn(rng, Sdim), crandn(rng, Sdim)
    got = hadron.nucleon_2pt(U1, Dd, U2)
    G1 = CHARGE_C @ GAMMA5
    G1b = GAMMA[3] @ np.conj(G1.T) @ GAMMA[3]
    P = 0.5 * (ID4 + GAMMA[3])
    eps = hadron._EPS
    # field string: u_{a al} d_{b be} u_{c g} ubar_{c' g'} dbar_{b' be'} ubar_{a' al'}
    # positions     0          1        2        3            4            5
    pairings = [((0, 5), (1, 4), (2, 3)), ((0, 3), (1, 4), (2, 5))]
    signs = [_pair_sign(None, pr) for pr in pairings]
    nz = lambda M: [(i, j) for i in range(4) for j in range(4) if M[i, j] != 0]
    for t in range(T):
        S1, Sd, S2 = U1[t, 0, 0, 0], Dd[t, 0, 0, 0], U2[t, 0, 0, 0]
        tot = 0.0
        for (a, b, c) in itertools.permutations(range(3)):
            for (ap, bp, cp) in itertools.permutations(range(3)):
                e = eps[a, b, c] * eps[ap, bp, cp]
                for (al, be) in nz(G1):
                    for (bep, alp) in nz(G1b):
                        w = e * G1[al, be] * G1b[bep, alp]
                        for g in range(4):
                            for gp in range(4):
                                if P[gp, g] == 0:
                                    continue
                                # index tuples (spin, colour) of the six fields
                                q = {0: (al, a), 1: (be, b), 2: (g, c),
                                     3: (gp, cp), 4: (bep, bp), 5: (alp, ap)}
                                for pr, sg in zip(pairings, signs):
                                    val = sg
                                    for (i, j) in pr:
                                        # u line from sink field 0 -> U1, field 2 -> U2
                                        Sm = {0: S1, 1: Sd, 2: S2}[i]
                                        val *= Sm[q[i][0], q[i][1], q[j][0], q[j][1]]
                                    tot += P[gp, g] * w * val
        assert abs(got[t] - tot) < 1e-11 * max(1.0, abs(tot)), (t, got[t], tot)


def test_nucleon_gauge_invariance():
    dims = (2, 2, 2, 4)
    X, Y, Z, T = dims
    p = MobiusParams(Ls=4, mf=0.2)
    U = inputs.gauge_links(dims, 0.5, 41)
    Om = random_gauge(dims, 42)
    Ub = dirac.boundary_links(U, p.t_bc)
    # gauge transform with Om(0) = 1 so the point source is unchanged
    Om[0, 0, 0, 0] = np.eye(3)
    Ubg = dirac.boundary_links(gauge_transform(U, Om), p.t_bc)
    S = _prop_point(Ub, p, dims)
    Sg = _prop_point(Ubg, p, dims)
    C = hadron.nucleon_2pt(S, S, S)
    Cg = hadron.nucleon_2pt(Sg, Sg, Sg)
    assert np.abs(C - Cg).max() < 1e-10 * np.abs(C).max()
    # the propagator transforms as Om(x) S(x) Om(0)^+
    rotS = np.einsum("tzyxab,tzyxibjc->tzyxiajc", Om, S)
    assert np.abs(Sg - rotS).max() < 1e-9 * np.abs(S).max()


def test_fh_effective_coupling_closed_form():
    """C(t) = A e^{-Mt}(1 + a e^{-Dt}) e^{i phi}, C_FH(t) = C(t) (c0 + g t): the ratio is
    linear in t, so g_eff(t) = g at every t, whatever the phase and excited state."""
    from oracle import hadron
    T = 16
    t = np.arange(T)
    C = 0.7 * np.exp(-0.45 * t) * (1 + 0.3 * np.exp(-0.6 * t)) * np.exp(0.37j)
    CF = C * (1.9 + 1.27 * t)
    g = hadron.fh_effective_coupling(C, CF)
    assert g.shape == (T - 1,)
    assert np.max(np.abs(g - 1.27)) < 1e-12
    # an excited-state term in the FH correlator decays out of the slope
    CF2 = C * (1.9 + 1.27 * t + 0.5 * np.exp(-1.1 * t))
    g2 = hadron.fh_effective_coupling(C, CF2)
    d = 0.5 * (np.exp(-1.1 * (t[:-1] + 1)) - np.exp(-1.1 * t[:-1]))
    assert np.max(np.abs(g2 - (1.27 + d))) < 1e-12
