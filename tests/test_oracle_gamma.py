"""Pins of oracle.gamma: Clifford algebra, hermiticity, gamma5 product, C relation."""
import numpy as np

from oracle.gamma import GAMMA, GAMMA5, CHARGE_C, P_MINUS, P_PLUS, ID4


def test_clifford():
    for m in range(4):
        for n in range(4):
            ac = GAMMA[m] @ GAMMA[n] + GAMMA[n] @ GAMMA[m]
            assert np.allclose(ac, 2.0 * (m == n) * ID4, atol=0)


def test_hermitian():
    for m in range(4):
        assert np.array_equal(GAMMA[m], np.conj(GAMMA[m].T))


def test_gamma5_is_product_and_chiral():
    g = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
    assert np.allclose(g, GAMMA5, atol=0)
    assert np.array_equal(np.diag(GAMMA5).real, [-1, -1, 1, 1])
    for m in range(4):
        assert np.allclose(GAMMA5 @ GAMMA[m], -GAMMA[m] @ GAMMA5, atol=0)
    assert np.allclose(P_MINUS + P_PLUS, ID4) and np.allclose(P_MINUS @ P_PLUS, 0)


def test_charge_conjugation():
    Ci = np.linalg.inv(CHARGE_C)
    for m in range(4):
        assert np.allclose(CHARGE_C @ GAMMA[m] @ Ci, -GAMMA[m].T, atol=1e-15)
    assert np.allclose(CHARGE_C @ GAMMA5 @ Ci, GAMMA5.T, atol=1e-15)
