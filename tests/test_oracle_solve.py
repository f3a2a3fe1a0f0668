"""Pins of the oracle's solvers: even-odd CGNR vs dense LU (brute force), vs the
unpreconditioned CGNR route, vs the momentum-space free-field propagator, and gauge
covariance of the solution."""
import numpy as np
import pytest

import inputs
from oracle import dirac, solve
from oracle.dirac import MobiusParams
from oracle.gamma import GAMMA, ID4, P_MINUS, P_PLUS
from _dense import dense, crandn
from test_oracle_wilson import gauge_transform, random_gauge


@pytest.mark.parametrize("dims,Ls,mf", [((2, 2, 2, 4), 4, 0.05), ((4, 2, 2, 2), 6, 0.01)])
def test_eo_solve_matches_dense_lu(dims, Ls, mf):
    rng = np.random.default_rng(5)
    X, Y, Z, T = dims
    p = MobiusParams(Ls=Ls, mf=mf)
    Ub = dirac.boundary_links(inputs.gauge_links(dims, 0.4, 2), p.t_bc)
    sh = (Ls, T, Z, Y, X, 4, 3)
    D = dense(lambda v: dirac.mobius(Ub, v, p), sh)
    b = crandn(rng, sh)
    xd = np.linalg.solve(D, b.ravel()).reshape(sh)
    x, it, res = solve.solve_eo(Ub, b, p, tol=1e-12)
    assert res <= 1e-12
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-10
    assert solve.residual_full(Ub, b, x, p) < 1e-10
    xf, itf, resf = solve.solve_full(Ub, b, p, tol=1e-12)
    assert np.linalg.norm(xf - xd) / np.linalg.norm(xd) < 1e-9


def test_free_field_momentum_space_propagator():
    """Unit links: D(p) = W(p) (b5 + c5 B) + 1 - B per momentum, with
    B = Bm (x) P_- + Bp (x) P_+ on (s, spin); x(x) = (1/V) sum_p e^{ipx} D(p)^-1 u."""
    dims = (4, 4, 4, 4)
    X, Y, Z, T = dims
    p = MobiusParams(Ls=8, mf=0.05)
    U = np.broadcast_to(np.eye(3), (T, Z, Y, X, 4, 3, 3)).astype(np.complex128)
    Ub = dirac.boundary_links(U, p.t_bc)
    rng = np.random.default_rng(6)
    u = crandn(rng, (p.Ls, 4, 3))
    b = np.zeros((p.Ls, T, Z, Y, X, 4, 3), dtype=np.complex128)
    b[:, 0, 0, 0, 0] = u
    x, it, res = solve.solve_eo(Ub, b, p, tol=1e-12)
    # momentum space, written from the plane-wave eigenvalues
    Bm = np.diag(np.ones(p.Ls - 1), 1); Bm[-1, 0] = -p.mf
    Bp = np.diag(np.ones(p.Ls - 1), -1); Bp[0, -1] = -p.mf
    Bfull = np.kron(Bm, P_MINUS) + np.kron(Bp, P_PLUS)
    I5 = np.eye(4 * p.Ls)
    xm = np.zeros_like(b)
    t, z, y, xx = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X),
                              indexing="ij")
    for nt in range(T):
        for nz in range(Z):
            for ny in range(Y):
                for nx in range(X):
                    pm = 2 * np.pi * np.array([nx / X, ny / Y, nz / Z, (nt + 0.5) / T])
                    W = sum(1j * GAMMA[m] * np.sin(pm[m]) for m in range(4)) \
                        + (np.sum(1 - np.cos(pm)) - p.M5) * ID4
                    Dp = np.kron(np.eye(p.Ls), W) @ (p.b5 * I5 + p.c5 * Bfull) + I5 - Bfull
                    sol = np.linalg.solve(Dp, u.reshape(4 * p.Ls, 3)).reshape(p.Ls, 4, 3)
                    ph = np.exp(1j * (pm[0] * xx + pm[1] * y + pm[2] * z + pm[3] * t))
                    xm += ph[None, ..., None, None] * sol[:, None, None, None, None]
    xm /= X * Y * Z * T
    assert np.linalg.norm(x - xm) / np.linalg.norm(xm) < 1e-10


def test_solution_gauge_covariance():
    rng = np.random.default_rng(7)
    dims = (4, 2, 2, 4)
    X, Y, Z, T = dims
    p = MobiusParams(Ls=4, mf=0.1)
    U = inputs.gauge_links(dims, 0.5, 31)
    Om = random_gauge(dims, 32)
    rot = lambda f: np.swapaxes(Om @ np.swapaxes(f, -1, -2), -1, -2)
    b = crandn(rng, (p.Ls, T, Z, Y, X, 4, 3))
    x, _, _ = solve.solve_eo(dirac.boundary_links(U, p.t_bc), b, p, tol=1e-12)
    xg, _, _ = solve.solve_eo(dirac.boundary_links(gauge_transform(U, Om), p.t_bc), rot(b),
                              p, tol=1e-12)
    assert np.linalg.norm(xg - rot(x)) / np.linalg.norm(x) < 1e-9


def test_symmetric_form_matches_dense_schur_complement():
    """M_sym and its adjoint against the Schur complement built densely from the
    definition: D~ = D D5^-1 (dense D, dense D5 on the whole 5D space), split into
    parity blocks, M = 1 - D~_oo^-1 D~_oe D~_ee^-1 D~_eo on the odd sites."""
    dims, Ls, mf = (2, 2, 2, 4), 4, 0.05
    X, Y, Z, T = dims
    p = MobiusParams(Ls=Ls, mf=mf)
    Ub = dirac.boundary_links(inputs.gauge_links(dims, 0.4, 12), p.t_bc)
    sh = (Ls, T, Z, Y, X, 4, 3)
    D = dense(lambda v: dirac.mobius(Ub, v, p), sh)
    D5 = dense(lambda v: dirac.s_op(p, "D5", v), sh)
    Dt = D @ np.linalg.inv(D5)
    par = np.broadcast_to(dirac.parity_mask(dims)[None, ..., None, None], sh).ravel()
    o, e = np.nonzero(par == 1)[0], np.nonzero(par == 0)[0]
    blk = lambda a, b: Dt[np.ix_(a, b)]
    Msym = np.eye(len(o)) - np.linalg.solve(blk(o, o), blk(o, e) @ np.linalg.solve(blk(e, e), blk(e, o)))

    def on_odd(fn, v):
        f = np.zeros(np.prod(sh), complex)
        f[o] = v
        return fn(f.reshape(sh)).ravel()[o]

    rng = np.random.default_rng(13)
    v = crandn(rng, len(o))
    got = on_odd(lambda f: dirac.mpc_sym(Ub, f, p), v)
    assert np.linalg.norm(got - Msym @ v) / np.linalg.norm(Msym @ v) < 1e-12
    gotd = on_odd(lambda f: dirac.mpc_sym_dag(Ub, f, p), v)
    assert np.linalg.norm(gotd - Msym.conj().T @ v) / np.linalg.norm(gotd) < 1e-12


def test_symmetric_form_solve_matches_dense_lu():
    dims, Ls, mf = (2, 2, 2, 4), 4, 0.05
    X, Y, Z, T = dims
    p = MobiusParams(Ls=Ls, mf=mf)
    Ub = dirac.boundary_links(inputs.gauge_links(dims, 0.4, 14), p.t_bc)
    sh = (Ls, T, Z, Y, X, 4, 3)
    D = dense(lambda v: dirac.mobius(Ub, v, p), sh)
    b = crandn(np.random.default_rng(15), sh)
    xd = np.linalg.solve(D, b.ravel()).reshape(sh)
    x, it, res = solve.solve_eo_sym(Ub, b, p, tol=1e-12)
    assert res <= 1e-12
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-10
