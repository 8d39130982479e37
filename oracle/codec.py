"""Storage rounding of the 16-bit state forms, written from the IEEE 754 formats
(test infrastructure: only the tests may import it; it shares no code with the CUDA path).

The paper stores f in FP32 and says nothing about reduced precision; the library adds two
storage forms in which a value f of block id b is kept as a 16-bit code q = f / s_b,
rounded to nearest with ties to even, and read back as q * s_b.  s_b is the smallest
power of two that is >= the largest |f| of block id b (at least 2^-126, at most 2^127,
1 when that maximum is 0).  Scaling by a power of two is exact in binary floating point,
so the only error is the rounding of f / s_b to the code format:

* bfloat16: 1 sign bit, 8 exponent bits (the FP32 range), 7 fraction bits;
* float16 (IEEE binary16): 5 exponent bits, 10 fraction bits, subnormals down to 2^-24.
"""
from __future__ import annotations

import numpy as np

BF16, F16 = 1, 2  # storage codes of the library's vl_storage


def pow2_at_least(m) -> np.ndarray:
    """Smallest power of two >= m (elementwise, m >= 0), clamped to [2^-126, 2^127];
    1 where m == 0.  Uses frexp: m = f 2^e with f in [0.5, 1), so m is a power of two
    exactly when f == 0.5."""
    m = np.asarray(m, dtype=np.float64)
    f, e = np.frexp(m)
    p = np.where(f == 0.5, m, np.ldexp(1.0, e))
    p = np.clip(p, 2.0 ** -126, 2.0 ** 127)
    return np.where(m > 0, p, 1.0)


def round_bf16(x) -> np.ndarray:
    """float32 -> nearest bfloat16 (ties to even), returned as float32.  A bfloat16 is
    the upper 16 bits of a float32: add half of the dropped range, plus one when the kept
    part is odd (the tie goes to the even neighbour), then clear the dropped 16 bits.
    Finite inputs only (the state holds no inf or NaN)."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    keep_odd = (u >> 16) & 1
    r = ((u + 0x7FFF + keep_odd) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def round_f16(x) -> np.ndarray:
    """float32 -> nearest IEEE binary16 (ties to even, gradual underflow), as float32."""
    return np.asarray(x, dtype=np.float32).astype(np.float16).astype(np.float32)


def block_scales(ids, vals, nb: int) -> np.ndarray:
    """s_b for every block id from per-block values (vals: nblocks x 64, float32)."""
    vals = np.asarray(vals, dtype=np.float32).reshape(-1, 64)
    m = np.zeros(nb, dtype=np.float32)
    if len(vals):
        np.maximum.at(m, np.asarray(ids, dtype=np.int64), np.abs(vals).max(axis=1))
    return pow2_at_least(m).astype(np.float32)


def encode_decode(ids, vals, nb: int, storage: int, scales=None) -> np.ndarray:
    """The float32 values a 16-bit state holds after storing vals (nblocks x 64 float32):
    q = round(f * (1/s_b)), returned as q * s_b."""
    vals = np.asarray(vals, dtype=np.float32).reshape(-1, 64)
    s = block_scales(ids, vals, nb) if scales is None else np.asarray(scales, dtype=np.float32)
    sb = s[np.asarray(ids, dtype=np.int64)][:, None]
    q = vals * (np.float32(1.0) / sb)  # exact: 1/s_b is a power of two
    q = round_bf16(q) if storage == BF16 else round_f16(q)
    return (q * sb).astype(np.float32)


def unit_roundoff(storage: int) -> float:
    """Largest relative rounding error of a normal code: 2^-8 (bfloat16), 2^-11 (float16)."""
    return 2.0 ** -8 if storage == BF16 else 2.0 ** -11


def subnormal_floor(storage: int) -> float:
    """Largest absolute error of a code below the normal range, relative to s_b: half the
    smallest subnormal of float16 (2^-25); bfloat16 codes of the state never get there."""
    return 2.0 ** -25 if storage == F16 else 0.0
