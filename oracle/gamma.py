"""Gamma matrices in the chiral basis (oracle; test infrastructure only).

Reading (the paper names no basis, Sec. "Current State of the Art"):
  gamma_k = [[0, i sigma_k], [-i sigma_k, 0]]  for k = 1, 2, 3  (x, y, z)
  gamma_4 = [[0, 1], [1, 0]]                                    (t)
  gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(-1, -1, +1, +1)
  P_-     = (1 - gamma_5)/2 = diag(1, 1, 0, 0)   (upper spins)
  P_+     = (1 + gamma_5)/2 = diag(0, 0, 1, 1)   (lower spins)
  C       = gamma_2 gamma_4                      (charge conjugation)
Pinned in tests/test_oracle_gamma.py by the Clifford algebra, hermiticity,
gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 and C gamma_mu C^-1 = -gamma_mu^T.
"""
import numpy as np

_s1 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_s2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_s3 = np.array([[1, 0], [0, -1]], dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)
_Z2 = np.zeros((2, 2), dtype=np.complex128)


def _offdiag(x):
    """[[0, x], [x^dagger, 0]]"""
    return np.block([[_Z2, x], [np.conj(x.T), _Z2]])


# mu = 0, 1, 2, 3  <->  x, y, z, t
GAMMA = np.stack([_offdiag(1j * _s1), _offdiag(1j * _s2), _offdiag(1j * _s3),
                  _offdiag(_I2)])
GAMMA5 = np.diag([-1.0, -1.0, 1.0, 1.0]).astype(np.complex128)
ID4 = np.eye(4, dtype=np.complex128)
P_MINUS = 0.5 * (ID4 - GAMMA5)
P_PLUS = 0.5 * (ID4 + GAMMA5)
CHARGE_C = GAMMA[1] @ GAMMA[3]
