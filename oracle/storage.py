"""Low-precision storage formats of spinor fields (oracle; test infrastructure only).

The paper (Sec. "Current State of the Art") runs the inner CG on "16-bit precision
fixed-point storage" with single-precision arithmetic.  Reading used here (the paper
gives no format): a 5D site's 24 reals are stored as IEEE half precision after division
by a per-site scale, norm = float32(max |component|) over the 24 reals, each half being
the round-to-nearest-even of (v / norm) computed in FP64; an all-zero site stores
norm 0 and zeros.  BF16 storage keeps no norm and rounds each FP64 value to nearest
even at 8 significant bits.  FP32 storage is the nearest-even float32.  16-bit fixed
point (the paper's "16-bit fixed-point" storage, read literally): the same per-site norm,
each real stored as the int16 nearest (ties to even) to 32767 v / norm, computed in FP64
as a product then a quotient; the value it stands for is q * (norm / 32767).
Pinned by hand-derived cases in tests/golden/storage_cases.txt.
"""
import numpy as np


def quantize_f16(site_reals):
    """site_reals: float64 [..., 24].  Returns (halves float16 [..., 24], norm float32 [...])."""
    v = np.asarray(site_reals, dtype=np.float64)
    norm = np.max(np.abs(v), axis=-1).astype(np.float32)
    n64 = norm.astype(np.float64)[..., None]
    safe = np.where(n64 > 0, n64, 1.0)
    h = np.where(n64 > 0, v / safe, 0.0).astype(np.float16)
    return h, norm


def dequantize_f16(h, norm):
    return h.astype(np.float64) * norm.astype(np.float64)[..., None]


def round_bf16(v):
    """Nearest-even rounding of FP64 values to 8 significant bits (bfloat16 values,
    normal range), returned as float64."""
    v = np.asarray(v, dtype=np.float64)
    m, e = np.frexp(v)                 # v = m * 2^e, |m| in [0.5, 1)
    return np.ldexp(np.rint(m * 256.0), e - 8)


def bf16_bits(v):
    """uint16 bit patterns of round_bf16(v)."""
    f = round_bf16(v).astype(np.float32)
    return (f.view(np.uint32) >> 16).astype(np.uint16)


def quantize_i16(site_reals):
    """site_reals: float64 [..., 24].  Returns (int16 [..., 24], norm float32 [...])."""
    v = np.asarray(site_reals, dtype=np.float64)
    norm = np.max(np.abs(v), axis=-1).astype(np.float32)
    n64 = norm.astype(np.float64)[..., None]
    safe = np.where(n64 > 0, n64, 1.0)
    q = np.where(n64 > 0, np.rint((32767.0 * v) / safe), 0.0).astype(np.int16)
    return q, norm


def dequantize_i16(q, norm):
    return q.astype(np.float64) * (norm.astype(np.float64) / 32767.0)[..., None]
