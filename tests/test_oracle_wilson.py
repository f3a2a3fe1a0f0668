"""Pins of the oracle's 4D Wilson pieces: free-field plane waves (momentum-space
formula), gamma5-hermiticity, adjointness of H, gauge covariance."""
import numpy as np
import pytest

import inputs
from oracle import dirac
from oracle.gamma import GAMMA, GAMMA5, ID4
from _dense import crandn


def _plane_wave(dims, n, u):
    X, Y, Z, T = dims
    pm = np.array([2 * np.pi * n[0] / X, 2 * np.pi * n[1] / Y, 2 * np.pi * n[2] / Z,
                   2 * np.pi * (n[3] + 0.5) / T])
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X),
                             indexing="ij")
    ph = np.exp(1j * (pm[0] * x + pm[1] * y + pm[2] * z + pm[3] * t))
    return pm, ph[..., None, None] * u


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (4, 4, 4, 8)])
def test_free_field_plane_waves(dims):
    # D_W(p) = i sum_mu gamma_mu sin p_mu + sum_mu (1 - cos p_mu) - M5, antiperiodic p_t
    rng = np.random.default_rng(0)
    X, Y, Z, T = dims
    U = np.broadcast_to(np.eye(3), (T, Z, Y, X, 4, 3, 3)).astype(np.complex128)
    Ub = dirac.boundary_links(U, -1.0)
    M5 = 1.3
    for _ in range(6):
        n = rng.integers(0, 4, size=4)
        u = crandn(rng, (4, 3))
        pm, psi = _plane_wave(dims, n, u)
        W = sum(1j * GAMMA[m] * np.sin(pm[m]) for m in range(4)) \
            + (np.sum(1 - np.cos(pm)) - M5) * ID4
        expect = np.einsum("ij,...jc->...ic", W, psi)
        assert np.allclose(dirac.wilson(Ub, psi, M5), expect, atol=1e-12)


def test_gamma5_hermiticity_and_hop_adjoint():
    rng = np.random.default_rng(1)
    dims = (4, 4, 4, 4)
    Ub = dirac.boundary_links(inputs.gauge_links(dims, 0.5, 11), -1.0)
    x = crandn(rng, (4, 4, 4, 4, 4, 3))
    y = crandn(rng, (4, 4, 4, 4, 4, 3))
    lhs = np.vdot(y, dirac.hop(Ub, x))
    rhs = np.vdot(dirac.hop(Ub, y, dagger=True), x)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)
    # H^dagger = gamma5 H gamma5 ; D_W^dagger = gamma5 D_W gamma5
    assert np.allclose(dirac.hop(Ub, x, dagger=True),
                       dirac.gamma5(dirac.hop(Ub, dirac.gamma5(x))), atol=1e-12)
    lhs = np.vdot(y, dirac.wilson(Ub, x, 1.3))
    rhs = np.vdot(dirac.gamma5(dirac.wilson(Ub, dirac.gamma5(y), 1.3)), x)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def gauge_transform(U, Om):
    """U^Om_mu(x) = Om(x) U_mu(x) Om(x+mu)^dagger"""
    out = np.empty_like(U)
    axes = {0: 3, 1: 2, 2: 1, 3: 0}
    for mu in range(4):
        Om_f = np.roll(Om, -1, axis=axes[mu])
        out[:, :, :, :, mu] = Om @ U[:, :, :, :, mu] @ np.conj(np.swapaxes(Om_f, -1, -2))
    return out


def random_gauge(dims, seed):
    X, Y, Z, T = dims
    rng = np.random.Generator(np.random.Philox(seed))
    return inputs.random_su3(X * Y * Z * T, 2.0, rng).reshape(T, Z, Y, X, 3, 3)


def test_gauge_covariance_wilson():
    rng = np.random.default_rng(2)
    dims = (4, 2, 4, 4)
    U = inputs.gauge_links(dims, 0.7, 5)
    Om = random_gauge(dims, 9)
    psi = crandn(rng, (4, 4, 2, 4, 4, 3))
    Ub = dirac.boundary_links(U, -1.0)
    Ubg = dirac.boundary_links(gauge_transform(U, Om), -1.0)
    lhs = dirac.hop(Ubg, np.swapaxes(Om @ np.swapaxes(psi, -1, -2), -1, -2))
    rhs = np.swapaxes(Om @ np.swapaxes(dirac.hop(Ub, psi), -1, -2), -1, -2)
    assert np.allclose(lhs, rhs, atol=1e-12)
