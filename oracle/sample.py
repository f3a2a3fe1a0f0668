"""Site-sampled evaluation of the operators of ``oracle.dirac`` for lattices too large
for a full oracle pass (oracle; test infrastructure only).

Every function evaluates the SAME definitions as ``oracle.dirac`` at a list of 4D
sites (all s and right-hand sides), gathering only the neighbours it needs.  Sites are
integer arrays [n, 4] of (x, y, z, t).  5D fields are [.., s, t, z, y, x, spin, colour].
"""
import numpy as np

from .gamma import GAMMA, ID4
from . import dirac

_MU_VEC = np.eye(4, dtype=np.int64)


def _wrap(c, dims):
    return np.mod(c, np.asarray(dims, dtype=np.int64))


def gather(field, sites):
    """field[..., s, t, z, y, x, :, :] at sites -> [..., s, n, 4, 3]."""
    x, y, z, t = sites[:, 0], sites[:, 1], sites[:, 2], sites[:, 3]
    return field[..., t, z, y, x, :, :]


def gather_links(Ub, sites, mu):
    x, y, z, t = sites[:, 0], sites[:, 1], sites[:, 2], sites[:, 3]
    return Ub[t, z, y, x, mu]  # [n, 3, 3]


def local_hop(Ub, sites, nbr_fn, dims, dagger=False):
    """(H v)(x) at the given sites where v at any site list is nbr_fn(sites) -> [..., s, n, 4, 3]."""
    sig = -1.0 if dagger else 1.0
    out = 0.0
    for mu in range(4):
        fw = _wrap(sites + _MU_VEC[mu], dims)
        bw = _wrap(sites - _MU_VEC[mu], dims)
        Uf = gather_links(Ub, sites, mu)           # U_mu(x)
        Ubk = gather_links(Ub, bw, mu)             # U_mu(x - mu)
        vf = nbr_fn(fw) @ np.swapaxes(Uf, -1, -2)
        vb = nbr_fn(bw) @ np.conj(Ubk)
        out = out + (ID4 - sig * GAMMA[mu]) @ vf + (ID4 + sig * GAMMA[mu]) @ vb
    return out


def _s(p, which, v, dagger=False):
    # v: [..., s, n, 4, 3] -> put into the [.., s, t,z,y,x, 4, 3] shape s_op expects
    w = v[..., :, None, None, None, :, :, :]
    return dirac.s_op(p, which, w, dagger)[..., :, 0, 0, 0, :, :, :]


def hop_at(Ub, psi, sites, dims, dagger=False):
    return local_hop(Ub, sites, lambda c: gather(psi, c), dims, dagger)


def mpc_at(Ub, psi_o, sites, p, dims):
    """M_pc psi_o at odd sites."""
    inner = lambda c: _s(p, "D5", _s(p, "A5inv", local_hop(
        Ub, c, lambda c2: _s(p, "D5", gather(psi_o, c2)), dims)))
    return gather(psi_o, sites) - 0.25 * _s(p, "A5inv", local_hop(Ub, sites, inner, dims))


def mpc_dag_at(Ub, psi_o, sites, p, dims):
    """M_pc^dagger psi_o at odd sites."""
    inner = lambda c: _s(p, "A5inv", _s(p, "D5", local_hop(
        Ub, c, lambda c2: _s(p, "A5inv", gather(psi_o, c2), True), dims, True), True), True)
    return gather(psi_o, sites) - 0.25 * _s(p, "D5", local_hop(Ub, sites, inner, dims, True), True)


def mobius_at(Ub, psi, sites, p, dims, mf=None):
    """Full 5D D psi at the given sites."""
    if mf is not None:
        p = dirac.MobiusParams(p.Ls, p.b5, p.c5, p.M5, mf, p.t_bc)
    d5 = lambda c: _s(p, "D5", gather(psi, c))
    w = (4.0 - p.M5) * d5(sites) - 0.5 * local_hop(Ub, sites, d5, dims)
    v = gather(psi, sites)
    return w + v - _s(p, "B", v)
