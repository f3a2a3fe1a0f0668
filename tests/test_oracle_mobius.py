"""Pins of the oracle's 5D Moebius operator and its even-odd pieces:
overlap closed form of the 4D effective operator, Gamma5 R5 hermiticity of
D_-^-1 D, adjoints, A5^-1 closed form, M_pc^+ M_pc positivity, gauge covariance."""
import numpy as np
import pytest

import inputs
from oracle import dirac, hadron
from oracle.dirac import MobiusParams
from oracle.gamma import GAMMA5
from _dense import dense, crandn
from test_oracle_wilson import gauge_transform, random_gauge


def _setup(dims, Ls, mf, eps=0.3, seed=1, b5=1.5, c5=0.5):
    p = MobiusParams(Ls=Ls, b5=b5, c5=c5, M5=1.3, mf=mf)
    Ub = dirac.boundary_links(inputs.gauge_links(dims, eps, seed), p.t_bc)
    return p, Ub


@pytest.mark.parametrize("Ls,b5,c5", [(4, 1.5, 0.5), (6, 1.0, 0.0), (5, 2.0, 1.0)])
def test_overlap_closed_form(Ls, b5, c5):
    """[P^-1 D(m)^-1 D(1) P]_00 = D_ov^-1 with D_ov = (1+m)/2 + (1-m)/2 g5 eps_Ls(H_M),
    H_M = g5 (b+c) D_W (2 + (b-c) D_W)^-1, eps_Ls(h) = tanh(Ls artanh h)."""
    dims = (2, 2, 2, 4)
    X, Y, Z, T = dims
    p, Ub = _setup(dims, Ls, 0.07, b5=b5, c5=c5)
    sh4 = (T, Z, Y, X, 4, 3)
    sh5 = (Ls,) + sh4
    n4 = int(np.prod(sh4))
    DW = dense(lambda v: dirac.wilson(Ub, v, p.M5), sh4)
    Dm = dense(lambda v: dirac.mobius(Ub, v, p), sh5)
    D1 = dense(lambda v: dirac.mobius(Ub, v, p, mf=1.0), sh5)
    W = np.zeros((Dm.shape[0], n4), dtype=np.complex128)
    for i in range(n4):
        e = np.zeros(n4, dtype=np.complex128)
        e[i] = 1.0
        W[:, i] = hadron.embed_wall(e.reshape(sh4), Ls).ravel()
    Ysol = np.linalg.solve(Dm, D1 @ W)
    Deff_inv = np.stack([hadron.project_4d(Ysol[:, i].reshape(sh5)).ravel()
                         for i in range(n4)], axis=1)
    V = X * Y * Z * T
    G5 = np.kron(np.eye(V), np.kron(GAMMA5, np.eye(3)))
    I = np.eye(n4)
    HM = G5 @ ((b5 + c5) * DW) @ np.linalg.inv(2 * I + (b5 - c5) * DW)
    assert np.abs(HM - HM.conj().T).max() < 1e-13
    w, v = np.linalg.eigh(0.5 * (HM + HM.conj().T))
    eps = ((1 + w) ** Ls - (1 - w) ** Ls) / ((1 + w) ** Ls + (1 - w) ** Ls)
    Dov = (1 + p.mf) / 2 * I + (1 - p.mf) / 2 * G5 @ ((v * eps) @ v.conj().T)
    assert np.abs(np.linalg.inv(Dov) - Deff_inv).max() < 1e-12


def test_gamma5_r5_hermiticity():
    """D_-^-1 D is Gamma5 R5 hermitian, D_- = c5 D_W - 1 per slice, R5: s -> Ls-1-s."""
    dims = (2, 2, 2, 4)
    X, Y, Z, T = dims
    p, Ub = _setup(dims, 4, 0.1)
    sh4 = (T, Z, Y, X, 4, 3)
    n4 = int(np.prod(sh4))
    DW = dense(lambda v: dirac.wilson(Ub, v, p.M5), sh4)
    Dm = dense(lambda v: dirac.mobius(Ub, v, p), (p.Ls,) + sh4)
    I = np.eye(n4)
    A = np.linalg.solve(np.kron(np.eye(p.Ls), p.c5 * DW - I), Dm)
    G5 = np.kron(np.eye(p.Ls), np.kron(np.eye(X * Y * Z * T), np.kron(GAMMA5, np.eye(3))))
    R5 = np.kron(np.fliplr(np.eye(p.Ls)), I)
    assert np.abs(G5 @ R5 @ A @ R5 @ G5 - A.conj().T).max() < 1e-12


def test_adjoints():
    rng = np.random.default_rng(3)
    dims = (4, 4, 2, 4)
    X, Y, Z, T = dims
    p, Ub = _setup(dims, 6, 0.05, eps=0.5)
    sh = (p.Ls, T, Z, Y, X, 4, 3)
    x, y = crandn(rng, sh), crandn(rng, sh)
    a = np.vdot(y, dirac.mobius(Ub, x, p))
    b = np.vdot(dirac.mobius(Ub, y, p, dagger=True), x)
    assert abs(a - b) < 1e-12 * abs(a)
    par = dirac.parity_mask(dims)
    xo, yo = dirac.on_parity(x, par, 1), dirac.on_parity(y, par, 1)
    a = np.vdot(yo, dirac.mpc(Ub, xo, p))
    b = np.vdot(dirac.mpc_dag(Ub, yo, p), xo)
    assert abs(a - b) < 1e-12 * abs(a)
    # M_pc^+ M_pc is hermitian positive
    n = np.vdot(xo, dirac.mpc_dag(Ub, dirac.mpc(Ub, xo, p), p))
    assert abs(n.imag) < 1e-12 * abs(n) and n.real > 0
    assert np.isclose(n.real, np.vdot(dirac.mpc(Ub, xo, p), dirac.mpc(Ub, xo, p)).real,
                      rtol=1e-12)


def test_mpc_positivity_lanczos_free():
    """Smallest eigenvalue of M_pc^+ M_pc on a tiny lattice is positive (dense)."""
    dims = (2, 2, 2, 4)
    X, Y, Z, T = dims
    p, Ub = _setup(dims, 4, 0.02, eps=0.6)
    par = dirac.parity_mask(dims)
    sh = (p.Ls, T, Z, Y, X, 4, 3)
    M = dense(lambda v: dirac.mpc(Ub, dirac.on_parity(v, par, 1), p), sh)
    odd = np.broadcast_to((par == 1)[None, ..., None, None], sh).ravel()
    Mo = M[np.ix_(odd, odd)]
    ev = np.linalg.eigvalsh(Mo.conj().T @ Mo)
    assert ev.min() > 1e-6


@pytest.mark.parametrize("Ls,mf", [(8, 0.05), (12, 0.01), (10, 0.3)])
def test_a5inv_closed_form(Ls, mf):
    """(alpha + beta S)^-1 = sum_{k<Ls} rho^k S^k / (alpha (1 + m rho^Ls)), rho = -beta/alpha,
    for each chirality block S of B (S^Ls = -m)."""
    p = MobiusParams(Ls=Ls, mf=mf)
    Bm, Bp = dirac.b_matrices(Ls, mf)
    inv_m, inv_p = dirac.s_matrices(p, "A5inv")
    rho = -p.beta / p.alpha
    for S, inv in ((Bm, inv_m), (Bp, inv_p)):
        assert np.allclose(np.linalg.matrix_power(S, Ls), -mf * np.eye(Ls), atol=1e-15)
        cf = sum(rho ** k * np.linalg.matrix_power(S, k) for k in range(Ls))
        cf = cf / (p.alpha * (1 + mf * rho ** Ls))
        assert np.abs(cf - inv).max() < 1e-15


def test_gauge_covariance_5d():
    rng = np.random.default_rng(4)
    dims = (4, 2, 2, 4)
    X, Y, Z, T = dims
    p = MobiusParams(Ls=4, mf=0.1)
    U = inputs.gauge_links(dims, 0.6, 21)
    Om = random_gauge(dims, 22)
    psi = crandn(rng, (p.Ls, T, Z, Y, X, 4, 3))
    rot = lambda f: np.swapaxes(Om @ np.swapaxes(f, -1, -2), -1, -2)
    Ub = dirac.boundary_links(U, p.t_bc)
    Ubg = dirac.boundary_links(gauge_transform(U, Om), p.t_bc)
    assert np.allclose(dirac.mobius(Ubg, rot(psi), p), rot(dirac.mobius(Ub, psi, p)),
                       atol=1e-12)
    par = dirac.parity_mask(dims)
    po = dirac.on_parity(psi, par, 1)
    assert np.allclose(dirac.mpc(Ubg, rot(po), p), rot(dirac.mpc(Ub, po, p)), atol=1e-12)
