"""Storage rounding for the mixed-precision path, from the format definitions.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The precision variant keeps the method's arithmetic in FP32/FP64 and changes
only how kernel tables and visibilities are stored: as bfloat16 or IEEE
binary16 (float16) pairs.  This module rounds FP64 values to those formats
(round to nearest, ties to even, with gradual underflow and overflow to
infinity) so that the FP64 oracle can be run on exactly the values the
16-bit storage holds:

* bfloat16: 8 significant bits, exponent range of binary32 (smallest normal
  2^-126, largest finite (2 - 2^-7) 2^127);
* float16: 11 significant bits, smallest normal 2^-14, largest finite 65504.

Float16 tables are stored scaled by 2^e (e from ``f16_exp2``) so that the
largest entry, the w = 0, o = 0 centre tap of the table (Section 1.7.1: the
integrand there is the non-negative taper product with no phase), lies in
[2^14, 2^15); the oracle applies the same scale, rounds, and scales back.

Pins (tests/test_oracle_precision.py): float16 rounding against numpy's own
binary16 conversion, bfloat16 rounding of binary32 inputs against the
integer round-half-even on the binary32 bit pattern, hand-checked ties,
subnormals and overflow.
"""
from __future__ import annotations

import numpy as np

BF16 = (8, -126, float.fromhex("0x1.fep127"))      # (significant bits, min normal exponent, max)
F16 = (11, -14, 65504.0)
_FORMATS = {"bf16": BF16, "f16": F16}


def round_format(x, fmt) -> np.ndarray:
    """Round FP64 values to a binary format (p bits, min normal 2^emin, max),
    nearest with ties to even; returns FP64 holding the rounded values."""
    p, emin, vmax = fmt
    x = np.asarray(x, dtype=np.float64)
    ax = np.abs(x)
    _, e = np.frexp(ax)                    # ax = m 2^e, m in [0.5, 1)
    # unit in the last place: 2^(e - p) for normals, 2^(emin - p + 1) below 2^emin
    q = np.maximum(e - p, emin - p + 1)
    r = np.rint(np.ldexp(ax, -q))          # power-of-two scaling is exact; rint ties to even
    y = np.ldexp(r, q)
    y = np.where(y > vmax, np.inf, y)
    return np.copysign(y, x)


def round_bf16(x) -> np.ndarray:
    return round_format(x, BF16)


def round_f16(x) -> np.ndarray:
    return round_format(x, F16)


def f16_exp2(peak: float) -> int:
    """Scale exponent e with peak * 2^e in [2^14, 2^15)."""
    _, e = np.frexp(float(peak))
    return int(15 - e)


def quantise(z, kind: str, exp2: int = 0) -> np.ndarray:
    """Complex values as the 16-bit storage of ``kind`` holds them (re and im
    rounded separately after scaling by 2^exp2), scaled back: complex128."""
    z = np.asarray(z, dtype=np.complex128)
    if kind == "c64":
        return z.astype(np.complex64).astype(np.complex128)
    fmt = _FORMATS[kind]
    re = np.ldexp(round_format(np.ldexp(z.real, exp2), fmt), -exp2)
    im = np.ldexp(round_format(np.ldexp(z.imag, exp2), fmt), -exp2)
    return re + 1j * im


def bits16(x, kind: str) -> np.ndarray:
    """Bit patterns (uint16) of values already representable in ``kind``."""
    x = np.asarray(x, dtype=np.float64)
    if kind == "f16":
        return x.astype(np.float16).view(np.uint16)
    # a bfloat16 is the upper half of the binary32 with the same value
    return (x.astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)


def table_exp2(tables, kind: str) -> int:
    """Storage exponent of a plan's 16-bit tables (0 except for float16)."""
    if kind != "f16":
        return 0
    t0 = tables.planes[0]
    b2, h = t0.shape[0] // 2, t0.shape[2] // 2
    return f16_exp2(float(np.real(t0[b2, b2, h, h])))


class QuantisedTables:
    """A KernelTables look-alike whose planes hold the stored values of a
    16-bit table (rounded after scaling by 2^exp2, scaled back)."""

    def __init__(self, tables, kind: str):
        self.kind = kind
        self.exp2 = table_exp2(tables, kind)
        self.prm = tables.prm
        self.beta = tables.beta
        self.w = tables.w
        self.support = tables.support
        self.scale = tables.scale
        self.planes = [quantise(t, kind, self.exp2) for t in tables.planes]

    def flat(self):
        offs = np.zeros(len(self.planes) + 1, dtype=np.int64)
        for p, tab in enumerate(self.planes):
            offs[p + 1] = offs[p] + tab.size
        return np.concatenate([t.ravel() for t in self.planes]), offs
