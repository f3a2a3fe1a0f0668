"""The site-sampled evaluators of oracle.sample agree with the full-lattice oracle
(which is itself pinned by the physics tests)."""
import numpy as np

import inputs
from oracle import dirac, sample
from oracle.dirac import MobiusParams
from _dense import crandn


def test_sampled_operators_match_full():
    rng = np.random.default_rng(9)
    dims = (4, 4, 2, 4)
    X, Y, Z, T = dims
    p = MobiusParams(Ls=6, mf=0.03)
    Ub = dirac.boundary_links(inputs.gauge_links(dims, 0.5, 4), p.t_bc)
    psi = crandn(rng, (p.Ls, T, Z, Y, X, 4, 3))
    par = dirac.parity_mask(dims)
    po = dirac.on_parity(psi, par, 1)
    allsites = np.array([(x, y, z, t) for t in range(T) for z in range(Z)
                         for y in range(Y) for x in range(X)])
    odd = allsites[(allsites.sum(1) % 2) == 1][::3]
    full = dirac.hop(Ub, psi)
    assert np.allclose(sample.hop_at(Ub, psi, allsites[::5], dims), sample.gather(full, allsites[::5]), atol=1e-12)
    full = dirac.hop(Ub, psi, dagger=True)
    assert np.allclose(sample.hop_at(Ub, psi, odd, dims, True), sample.gather(full, odd), atol=1e-12)
    assert np.allclose(sample.mpc_at(Ub, po, odd, p, dims), sample.gather(dirac.mpc(Ub, po, p), odd), atol=1e-12)
    assert np.allclose(sample.mpc_dag_at(Ub, po, odd, p, dims),
                       sample.gather(dirac.mpc_dag(Ub, po, p), odd), atol=1e-12)
    assert np.allclose(sample.mobius_at(Ub, psi, allsites[::7], p, dims),
                       sample.gather(dirac.mobius(Ub, psi, p), allsites[::7]), atol=1e-12)
    assert np.allclose(sample.mobius_at(Ub, psi, allsites[::7], p, dims, mf=1.0),
                       sample.gather(dirac.mobius(Ub, psi, p, mf=1.0), allsites[::7]), atol=1e-12)
