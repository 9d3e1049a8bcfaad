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

* INT8 post-training quantisation of the embedding MLP (the thesis's INT8
  embedding, Sec. on MLP quantisation): every layer's input quantised with a
  static per-tensor scale S_a = alpha / 127 (alpha from calibration), the
  weights with a per-output-channel scale S_w = max |W_row| / 127, codes
  clip(round(v / S), -127, 127), exact integer dot products, then
  y = S_a S_w acc + b, ReLU between layers, the last layer's y the
  embedding. The quantisation decisions, the combined scale and y are
  float32 (the precision the kernel takes them in); the sums are exact.

Pinned by tests/test_oracle_pins.py: the thesis's worked example S = 10.8/127,
the closed-form values of landmark codes, the round trip of all finite codes,
tie and saturation cases; the INT8 layer on exactly representable inputs,
where it must equal the float product.
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


QMAX = 127


def int8_weight_scales(W) -> np.ndarray:
    """Per-output-channel weight scales S_w = max |W_row| / 127 (1 for a zero
    row), float32 like the kernel's."""
    W = np.asarray(W, np.float32)
    a = np.abs(W).max(axis=1)
    return np.where(a > 0, a / np.float32(QMAX), np.float32(1.0)).astype(np.float32)


def int8_codes(v, inv_scale) -> np.ndarray:
    """clip(round(v * (127 / alpha)), -127, 127), the product and the rounding
    (half to even) in float32."""
    q = np.rint(np.asarray(v, np.float32) * np.float32(inv_scale))
    return np.clip(q, -QMAX, QMAX).astype(np.int64)


def int8_layer(x_codes, alpha: float, W, b):
    """One quantised Linear: input codes of scale alpha / 127, weights
    quantised per output channel; returns y = s acc + b with the combined
    scale s = (alpha / 127) S_w formed in float32 and y rounded once to
    float32 (a fused multiply-add, as the kernel evaluates it)."""
    W = np.asarray(W, np.float32)
    sw = int8_weight_scales(W)
    Wq = np.clip(np.rint(W / sw[:, None]), -QMAX, QMAX).astype(np.int64)
    acc = np.asarray(x_codes, np.int64) @ Wq.T
    s = np.float32(np.float32(alpha) / np.float32(QMAX)) * sw
    y = acc.astype(np.float64) * s.astype(np.float64)[None, :] + np.asarray(b, np.float32).astype(np.float64)
    return y.astype(np.float32)


def int8_embed(layers, alphas, feats):
    """The INT8 embedding of feats [n][3] (float32 features): `layers` =
    [(W, b)], `alphas` = the calibrated range of each layer's input."""
    x = np.asarray(feats, np.float32)
    for l, (W, b) in enumerate(layers):
        inv = np.float32(QMAX) / np.float32(alphas[l])
        y = int8_layer(int8_codes(x, inv), alphas[l], W, b)
        if l + 1 < len(layers):
            y = np.maximum(y, 0.0)
        x = y
    return x


def embed_amax(layers, feats):
    """Max calibration: the largest |input| of every layer of the float64
    embedding over `feats`."""
    x = np.asarray(feats, np.float64)
    out = []
    for l, (W, b) in enumerate(layers):
        out.append(float(np.abs(x).max()) if x.size else 0.0)
        x = x @ np.asarray(W, np.float64).T + np.asarray(b, np.float64)
        if l + 1 < len(layers):
            x = np.maximum(x, 0.0)
    return out
