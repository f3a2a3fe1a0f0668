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


def test_i16_rounding_cases():
    """norm = 2 (site[0]); the value 2 v stores RNE(32767 v)."""
    for v, e in _cases("i16"):
        v, e = eval(v), int(e)
        site = np.zeros(24)
        site[0] = 2.0
        site[7] = 2.0 * v
        q, n = storage.quantize_i16(site)
        assert n == np.float32(2.0) and q[0] == 32767
        assert int(q[7]) == e, (v, int(q[7]), e)


def test_i16_norm_zero_site_and_roundtrip_bound():
    rng = np.random.default_rng(4)
    v = rng.standard_normal((1000, 24))
    v[3] = 0.0
    q, n = storage.quantize_i16(v)
    assert n[3] == 0.0 and not np.any(q[3])
    assert np.all(np.abs(q).max(axis=-1)[n > 0] == 32767)     # the largest real maps to +-32767
    back = storage.dequantize_i16(q, n)
    # half a unit of 1/32767 of the norm (plus the float32 rounding of the norm)
    bound = n.astype(np.float64)[:, None] * (0.5 / 32767 + 2.0 ** -23)
    assert np.all(np.abs(back - v) <= bound)
