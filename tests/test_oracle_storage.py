"""Pins of oracle.storage against hand-derived IEEE round-to-nearest-even cases
(tests/golden/storage_cases.txt) and the per-site norm reading."""
import os
import numpy as np

from oracle import storage

GOLD = os.path.join(os.path.dirname(__file__), "golden", "storage_cases.txt")


def _cases(kind):
    out = []
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        if f[0] == kind:
            out.append(f[1:])
    return out


def test_f16_rounding_cases():
    for v, e in _cases("f16"):
        v, e = eval(v), eval(e)
        # norm = 2: a value 2v (v <= 1) stores round(v); a value v (v > 1, normal
        # range) stores round(v/2) = e/2 since scaling by 2 is exact in binary
        site = np.zeros(24)
        site[0] = 2.0
        site[5] = 2.0 * v if abs(v) <= 1 else v
        expect = e if abs(v) <= 1 else e / 2
        h, n = storage.quantize_f16(site)
        assert n == np.float32(2.0)
        assert float(h[5]) == expect, (v, float(h[5]), expect)


def test_f16_norm_and_zero_site():
    site = np.array([0.5, -3.0, 1.5] + [0.0] * 21)
    h, n = storage.quantize_f16(site)
    assert n == np.float32(3.0)
    assert list(h[:3].astype(float)) == [0.5 / 3.0 == 0.5 / 3.0 and float(np.float16(0.5 / 3.0)),
                                         -1.0, 0.5]
    h0, n0 = storage.quantize_f16(np.zeros(24))
    assert n0 == 0.0 and not np.any(h0)
    back = storage.dequantize_f16(h, n)
    assert np.max(np.abs(back - site)) <= 3.0 * 2.0 ** -12


def test_bf16_rounding_cases():
    for v, e, bits in _cases("bf16"):
        v, e = eval(v), eval(e)
        assert storage.round_bf16(np.array([v]))[0] == e, (v, e)
        assert int(storage.bf16_bits(np.array([v]))[0]) == int(bits, 16)
