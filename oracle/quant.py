"""Quantisation reference -- TEST INFRASTRUCTURE (oracle side).

Only the test suite may import this module; the product path never does.

* The symmetric scheme of the thesis's section on quantisation (Eqs. of
  x = S x_q and x_q = clip(round(x / S), -alpha_q, alpha_q)): the scale maps
  the interval bound alpha onto the largest code, S = alpha / q_max.
* FP8-E4M3 (the FP8 format of the precision paths), written from the format's
  definition: 1 sign bit, 4 exponent bits with bias 7, 3 mantissa bits;
  exponent field 0 holds the subnormals m * 2^-9; the code with all exponent
  and mantissa bits set is NaN; there are no infinities, so the largest finite
  magnitude is 1.75 * 2^8 = 448. Encoding rounds to the nearest representable
  value, ties to the code with an even mantissa, and saturates at +-448
  ("satfinite"). The encoder is a brute-force nearest search over the decode
  table, so it shares no arithmetic with a bit-twiddling encoder.

Pinned by tests/test_oracle_pins.py: the thesis's worked example S = 10.8/127,
the closed-form values of landmark codes, the round trip of all finite codes,
tie and saturation cases.
"""
from __future__ import annotations

import numpy as np

E4M3_MAX = 448.0


def symmetric_scale(alpha: float, q_max: int) -> float:
    """S such that alpha maps to the largest code q_max."""
    return alpha / q_max


def quantize(x, scale: float, alpha_q: int):
    """x_q = clip(round(x / S), -alpha_q, alpha_q), round half to even."""
    return np.clip(np.rint(np.asarray(x, np.float64) / scale), -alpha_q, alpha_q)


def dequantize(xq, scale: float):
    return np.asarray(xq, np.float64) * scale


def e4m3_decode(code: int) -> float:
    """Value of one E4M3 code (NaN for 0x7F / 0xFF)."""
    code = int(code) & 0xFF
    sign = -1.0 if code & 0x80 else 1.0
    e = (code >> 3) & 0xF
    m = code & 0x7
    if e == 0xF and m == 0x7:
        return float("nan")
    if e == 0:
        return sign * m * 2.0 ** -9
    return sign * (1.0 + m / 8.0) * 2.0 ** (e - 7)


_CODES = np.array([c for c in range(256) if not np.isnan(e4m3_decode(c))], np.int64)
_VALUES = np.array([e4m3_decode(c) for c in _CODES], np.float64)


def e4m3_encode(x: float) -> int:
    """Nearest finite E4M3 code to x (ties: even mantissa), saturating at
    +-448; NaN -> 0x7F. Zero keeps its sign."""
    x = float(x)
    if np.isnan(x):
        return 0x7F
    neg = np.signbit(x)
    a = abs(x)
    if a >= E4M3_MAX:
        return (0x80 if neg else 0x00) | 0x7E
    pos = _CODES[(_CODES & 0x80) == 0]
    vals = _VALUES[(_CODES & 0x80) == 0]
    d = np.abs(vals - a)
    best = np.flatnonzero(d == d.min())
    if best.size > 1:  # a tie between two neighbours: the even mantissa wins
        best = [b for b in best if (pos[b] & 1) == 0]
    code = int(pos[best[0]])
    return (0x80 if neg else 0x00) | code


def e4m3_encode_array(x) -> np.ndarray:
    return np.array([e4m3_encode(v) for v in np.asarray(x, np.float64).ravel()], np.uint8)
