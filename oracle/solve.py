"""CG on the normal equations (CGNR) and the even-odd solve (oracle; test
infrastructure only).

The paper (Sec. "Current State of the Art") uses conjugate gradient on the normal
equations with red-black preconditioning for the Moebius domain-wall operator.  The
iteration below is textbook CGNR written in the order of its definition:

  x = 0, r = p = A^+ b, gamma = |r|^2
  loop:  q = A p;  alpha = gamma / |q|^2;  x += alpha p;  r -= alpha A^+ q
         gamma' = |r|^2;  p = r + (gamma'/gamma) p;  gamma = gamma'

Stopping reading (the paper only says "relative residual"): stop when the TRUE
relative residual |b - A x| / |b| <= tol.  It is recomputed when the iterated normal
residual |r| first falls below tol * |A^+ b|, and every 50 iterations after that.
"""
import numpy as np

from . import dirac


def _nrm(v):
    return float(np.sqrt(np.vdot(v, v).real))


def cgnr(A, Adag, b, tol=1e-10, maxiter=100000, check_every=50):
    """Returns (x, iterations, true relative residual)."""
    x = np.zeros_like(b)
    r = Adag(b)
    p = r.copy()
    gamma = np.vdot(r, r).real
    bnorm = _nrm(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    normal_stop = tol * np.sqrt(gamma)
    checking = False
    last = 0
    true = np.inf
    for k in range(1, maxiter + 1):
        q = A(p)
        alpha = gamma / np.vdot(q, q).real
        x = x + alpha * p
        r = r - alpha * Adag(q)
        gamma_new = np.vdot(r, r).real
        if np.sqrt(gamma_new) <= normal_stop and (not checking or k - last >= check_every):
            checking, last = True, k
            true = _nrm(b - A(x)) / bnorm
            if true <= tol:
                return x, k, true
        p = r + (gamma_new / gamma) * p
        gamma = gamma_new
    return x, maxiter, true


def solve_eo(Ub, b, p, tol=1e-10, maxiter=100000):
    """Full 5D solution of D x = b by CGNR on the odd-site Schur complement M_pc.
    Returns (x, iterations, true preconditioned residual)."""
    dims = (b.shape[-3], b.shape[-4], b.shape[-5], b.shape[-6])
    par = dirac.parity_mask(dims)
    bt = dirac.prepare_source(Ub, b, p, par)
    A = lambda v: dirac.mpc(Ub, v, p)
    Ad = lambda v: dirac.mpc_dag(Ub, v, p)
    xo, it, res = cgnr(A, Ad, bt, tol, maxiter)
    return dirac.reconstruct(Ub, b, xo, p, par), it, res


def solve_eo_sym(Ub, b, p, tol=1e-10, maxiter=100000):
    """The same solution through the symmetric form: CGNR on M_sym y = D5 b~_o, then
    x_o = D5^-1 y.  Returns (x, iterations, true relative residual of that system)."""
    dims = (b.shape[-3], b.shape[-4], b.shape[-5], b.shape[-6])
    par = dirac.parity_mask(dims)
    rhs = dirac.s_op(p, "D5", dirac.prepare_source(Ub, b, p, par))
    A = lambda v: dirac.mpc_sym(Ub, v, p)
    Ad = lambda v: dirac.mpc_sym_dag(Ub, v, p)
    y, it, res = cgnr(A, Ad, rhs, tol, maxiter)
    return dirac.reconstruct(Ub, b, dirac.s_op(p, "D5inv", y), p, par), it, res


def solve_full(Ub, b, p, tol=1e-10, maxiter=100000, mf=None):
    """Unpreconditioned route: CGNR on the full 5D operator D (independent check of the
    even-odd machinery)."""
    A = lambda v: dirac.mobius(Ub, v, p, mf=mf)
    Ad = lambda v: dirac.mobius(Ub, v, p, mf=mf, dagger=True)
    return cgnr(A, Ad, b, tol, maxiter)


def residual_full(Ub, b, x, p):
    """|b - D x| / |b| of the full 5D system."""
    return _nrm(b - dirac.mobius(Ub, x, p)) / _nrm(b)
