"""The seeded input generators shared by the oracle, the parity tests and the benchmark:
links are SU(3) and reproducible per seed, sources have the documented structure."""
import numpy as np

import inputs


def test_gauge_links_are_su3_and_seeded():
    dims = (4, 4, 2, 6)
    U = inputs.gauge_links(dims, 0.5, 11)
    assert U.shape == (6, 2, 4, 4, 4, 3, 3) and U.dtype == np.complex128
    M = U.reshape(-1, 3, 3)
    eye = np.eye(3)
    assert np.abs(np.conj(np.swapaxes(M, -1, -2)) @ M - eye).max() < 1e-14
    assert np.abs(np.linalg.det(M) - 1.0).max() < 1e-14
    assert np.array_equal(U, inputs.gauge_links(dims, 0.5, 11))
    assert not np.allclose(U, inputs.gauge_links(dims, 0.5, 12))
    # the roughness parameter: eps = 0 gives unit links, small eps links near unity
    assert np.abs(inputs.gauge_links(dims, 0.0, 11).reshape(-1, 3, 3) - eye).max() < 1e-15
    d_small = np.abs(inputs.gauge_links(dims, 0.05, 11).reshape(-1, 3, 3) - eye).max()
    d_big = np.abs(M - eye).max()
    assert d_small < 0.5 and d_small < d_big


def test_gaussian_spinor_moments_and_layout():
    dims, Ls = (4, 4, 4, 8), 6
    psi = inputs.gaussian_spinor5d(dims, Ls, 3)
    assert psi.shape == (Ls, 8, 4, 4, 4, 4, 3)
    assert np.array_equal(psi, inputs.gaussian_spinor5d(dims, Ls, 3))
    re, im = psi.real.ravel(), psi.imag.ravel()
    n = re.size
    for part in (re, im):
        assert abs(part.mean()) < 5 / np.sqrt(n)
        assert abs(part.var() - 1.0) < 10 * np.sqrt(2.0 / n)
    batch = inputs.gaussian_spinor5d(dims, Ls, 3, nrhs=2)
    assert batch.shape == (2,) + psi.shape


def test_point_and_z2_sources():
    dims = (4, 4, 4, 8)
    b = inputs.point_source4d(dims, 2, 1, site=(1, 2, 3, 4))
    assert b.shape == (8, 4, 4, 4, 4, 3)
    assert b[4, 3, 2, 1, 2, 1] == 1.0 and np.count_nonzero(b) == 1
    z = inputs.z2_source4d(dims, 5)
    assert z.shape == (8, 4, 4, 4, 4, 3)
    assert np.all(z.imag == 0) and set(np.unique(z.real)) == {-1.0, 1.0}
    assert np.array_equal(z, inputs.z2_source4d(dims, 5))
