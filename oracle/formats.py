"""Feature storage formats, written from their definitions -- oracle side.

Test infrastructure only (see ``oracle/__init__``).  These functions say what
a stored feature value means, so the oracle can score exactly the values the
GPU reads, and give the expected output of the library's packing kernel.
Nothing here is shared with the CUDA library.

Formats (non-negative feature values only, as counts are):

* u8 + overflow list -- the byte plane holds min(v, 255); every v > 255 adds a
  list entry (column, v - 255) to its row, columns ascending.  Exact for any
  count below 255 + 65535.
* BF16 -- 1 sign, 8 exponent (bias 127), 7 stored significand bits; rounding
  is to nearest, ties to an even significand.  Exact for integers <= 256.
* FP8 E4M3 (the "fn" variant: no infinities, one NaN code 0x7F/0xFF) --
  1 sign, 4 exponent (bias 7), 3 significand bits; exponent field 0 is
  subnormal (m/8 * 2**-6); largest finite value 448.  Exact for integers
  <= 16.  Each row carries a power-of-two scale 2**e with
  e = max(0, ceil(log2(max_row / 448))), stored as an int8; the stored byte is
  the nearest E4M3 value (ties to even significand) of v / 2**e.
"""
from __future__ import annotations

import numpy as np

U8_MAX = 255


# ----------------------------------------------------------------------------
# u8 + overflow list
# ----------------------------------------------------------------------------
def pack_u8_overflow(V):
    """u16/u32 counts (n x F) -> (plane u8, row_ptr int64[n+1], col u16, add u16)."""
    V = np.asarray(V)
    if V.ndim != 2:
        raise ValueError("expected a matrix")
    if (V < 0).any() or (V > U8_MAX + 65535).any():
        raise ValueError("value outside the u8+overflow range")
    V = V.astype(np.int64)
    plane = np.minimum(V, U8_MAX).astype(np.uint8)
    rows, cols = np.nonzero(V > U8_MAX)          # row-major order: cols ascending
    add = (V[rows, cols] - U8_MAX).astype(np.uint16)
    row_ptr = np.zeros(V.shape[0] + 1, np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return plane, row_ptr, cols.astype(np.uint16), add


def unpack_u8_overflow(plane, row_ptr, col, add):
    V = plane.astype(np.float64)
    for i in range(plane.shape[0]):
        for k in range(int(row_ptr[i]), int(row_ptr[i + 1])):
            V[i, int(col[k])] += float(add[k])
    return V


# ----------------------------------------------------------------------------
# BF16
# ----------------------------------------------------------------------------
def bf16_round(v):
    """Nearest BF16 value of each non-negative v (ties to even significand)."""
    v = np.asarray(v, dtype=np.float64)
    out = np.zeros_like(v)
    nz = v > 0
    e = np.floor(np.log2(v[nz]))
    # guard log2 rounding at exact powers of two
    e = np.where(2.0 ** e > v[nz], e - 1, e)
    e = np.where(2.0 ** (e + 1) <= v[nz], e + 1, e)
    spacing = 2.0 ** (e - 7)
    q = v[nz] / spacing                      # in [128, 256)
    fl = np.floor(q)
    frac = q - fl
    up = (frac > 0.5) | ((frac == 0.5) & (fl % 2 == 1))
    out[nz] = (fl + up) * spacing
    return out


def bf16_bits(v):
    """Bit patterns (uint16) of bf16_round(v) for non-negative v."""
    r = bf16_round(v).astype(np.float32)
    return (r.view(np.uint32) >> 16).astype(np.uint16)


def bf16_decode(bits):
    bits = np.asarray(bits, dtype=np.uint16).astype(np.uint32)
    sign = np.where(bits >> 15, -1.0, 1.0)
    ex = (bits >> 7) & 0xFF
    man = (bits & 0x7F).astype(np.float64)
    val = np.where(ex == 0, man / 128.0 * 2.0 ** -126,
                   (1.0 + man / 128.0) * 2.0 ** (ex.astype(np.float64) - 127))
    val = np.where(ex == 0xFF, np.where(man == 0, np.inf, np.nan), val)
    return sign * val


# ----------------------------------------------------------------------------
# FP8 E4M3 with a per-row power-of-two scale
# ----------------------------------------------------------------------------
def e4m3_decode(bits):
    bits = np.asarray(bits, dtype=np.uint8).astype(np.int64)
    sign = np.where(bits >> 7, -1.0, 1.0)
    ex = (bits >> 3) & 0xF
    man = (bits & 0x7).astype(np.float64)
    val = np.where(ex == 0, man / 8.0 * 2.0 ** -6,
                   (1.0 + man / 8.0) * 2.0 ** (ex.astype(np.float64) - 7))
    val = np.where((ex == 0xF) & (man == 0x7), np.nan, val)
    return sign * val


_E4M3_CODES = np.arange(0x7F, dtype=np.uint8)          # 0x00..0x7E: finite, >= 0
_E4M3_VALUES = e4m3_decode(_E4M3_CODES)                # ascending
E4M3_MAX = float(_E4M3_VALUES[-1])                     # 448


def e4m3_encode(v):
    """Nearest finite non-negative E4M3 code of v in [0, 448] (ties to even)."""
    v = np.asarray(v, dtype=np.float64)
    if (v < 0).any() or (v > E4M3_MAX).any():
        raise ValueError("value outside [0, 448]")
    hi = np.searchsorted(_E4M3_VALUES, v, side="left")  # first value >= v
    hi = np.minimum(hi, len(_E4M3_VALUES) - 1)
    lo = np.maximum(hi - 1, 0)
    dv_hi = _E4M3_VALUES[hi] - v
    dv_lo = v - _E4M3_VALUES[lo]
    pick_hi = (dv_hi < dv_lo) | ((dv_hi == dv_lo) & (_E4M3_CODES[hi] % 2 == 0))
    exact = _E4M3_VALUES[hi] == v
    code = np.where(exact | pick_hi, _E4M3_CODES[hi], _E4M3_CODES[lo])
    return code.astype(np.uint8)


def e4m3_row_exponent(V):
    """Smallest e >= 0 with max_row <= 448 * 2**e, per row (int8)."""
    V = np.asarray(V, dtype=np.float64)
    m = V.max(axis=1) if V.shape[1] else np.zeros(V.shape[0])
    e = np.zeros(V.shape[0], np.int64)
    while True:
        need = m > E4M3_MAX * 2.0 ** e
        if not need.any():
            break
        e = e + need
    return e.astype(np.int8)


def pack_e4m3(V):
    """(codes u8 n x F, row exponent int8 n) for non-negative V."""
    V = np.asarray(V, dtype=np.float64)
    e = e4m3_row_exponent(V)
    scaled = V / (2.0 ** e.astype(np.float64))[:, None]
    return e4m3_encode(scaled), e


def unpack_e4m3(codes, row_exp):
    return e4m3_decode(codes) * (2.0 ** np.asarray(row_exp, np.float64))[:, None]
