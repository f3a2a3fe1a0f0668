"""Dense-matrix helpers for the oracle pins on tiny lattices."""
import numpy as np


def dense(fn, shape):
    n = int(np.prod(shape))
    M = np.zeros((n, n), dtype=np.complex128)
    for i in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[i] = 1.0
        M[:, i] = fn(e.reshape(shape)).ravel()
    return M


def crandn(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
