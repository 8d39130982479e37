"""Storage rounding of the 16-bit state forms, written from the IEEE 754 formats
(test infrastructure: only the tests may import it; it shares no code with the CUDA path).

The paper stores f in FP32 and says nothing about reduced precision; the library adds two
storage forms with a scale per stored chunk: the 64 values of a 4x4x4 velocity block are
four chunks of 16 (one vz plane of the block each, values 16 q .. 16 q + 15 of the block),
and a value f of chunk c is kept as a 16-bit code q = f / s_c, rounded to nearest with
ties to even, and read back as q * s_c.  s_c is the smallest power of two that is >= the
largest |f| of the chunk, clamped to [2^-126, 2^126] (so 2^-126 when the chunk is all
zero): both s_c and 1 / s_c are then normal binary32 numbers.  Scaling by a power of two
is exact in binary floating point, so the only error is the rounding of f / s_c to the
code format, and every code lies in [-1, 1] (values above 2^126 aside):

* bfloat16: 1 sign bit, 8 exponent bits (the FP32 range), 7 fraction bits;
* float16 (IEEE binary16): 5 exponent bits, 10 fraction bits, subnormals down to 2^-24.
"""
from __future__ import annotations

import numpy as np

BF16, F16 = 1, 2  # storage codes of the library's vl_storage


def pow2_at_least(m) -> np.ndarray:
    """Smallest power of two >= m (elementwise, m >= 0), clamped to [2^-126, 2^126]
    (2^-126 where m == 0).  Uses frexp: m = f 2^e with f in [0.5, 1), so m is a power of
    two exactly when f == 0.5."""
    m = np.asarray(m, dtype=np.float64)
    f, e = np.frexp(m)
    p = np.where(f == 0.5, m, np.ldexp(1.0, e))
    return np.clip(np.where(m > 0, p, 0.0), 2.0 ** -126, 2.0 ** 126)


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


def chunk_scales(vals) -> np.ndarray:
    """s_c of every chunk (nblocks x 4, float32) from per-block values (nblocks x 64)."""
    vals = np.asarray(vals, dtype=np.float32).reshape(-1, 4, 16)
    return pow2_at_least(np.abs(vals).max(axis=2) if len(vals) else np.zeros((0, 4))).astype(np.float32)


def encode_decode(vals, storage: int) -> np.ndarray:
    """The float32 values a 16-bit state holds after storing vals (nblocks x 64 float32):
    q = round(f * (1/s_c)), returned as q * s_c."""
    vals = np.asarray(vals, dtype=np.float32).reshape(-1, 64)
    s = np.repeat(chunk_scales(vals), 16, axis=1)
    q = vals * (np.float32(1.0) / s)  # exact: 1/s_c is a power of two
    q = round_bf16(q) if storage == BF16 else round_f16(q)
    return (q * s).astype(np.float32)


def unit_roundoff(storage: int) -> float:
    """Largest relative rounding error of a normal code: 2^-8 (bfloat16), 2^-11 (float16)."""
    return 2.0 ** -8 if storage == BF16 else 2.0 ** -11


def subnormal_floor(storage: int) -> float:
    """Largest absolute error of a code below the normal range, relative to s_c: half the
    smallest subnormal of float16 (2^-25); bfloat16 codes of the state never get there."""
    return 2.0 ** -25 if storage == F16 else 0.0
