"""Pins of the 16-bit storage rounding (oracle/codec.py) to the IEEE formats: hand-worked
ties and boundaries of bfloat16 and binary16, and the power-of-two scale rule."""
import numpy as np
import pytest

from oracle import codec


def f32(x):
    return np.asarray(x, dtype=np.float32)


@pytest.mark.parametrize("x, want", [
    (1.0, 1.0),
    (1.0 + 2.0 ** -8, 1.0),                          # tie between 1 and 1+2^-7: even (1)
    (1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -6),          # tie between odd and even: even
    (1.0 + 2.0 ** -8 + 2.0 ** -20, 1.0 + 2.0 ** -7),  # just above the tie: up
    (1.0 + 2.0 ** -8 - 2.0 ** -20, 1.0),              # just below: down
    (-(1.0 + 3 * 2.0 ** -8), -(1.0 + 2.0 ** -6)),     # sign-symmetric
    (3.0, 3.0),                                      # exactly representable
    (0.1, 0.10009765625),                            # 0x3DCCCCCD -> 0x3DCD
    (2.0 ** -130, 2.0 ** -130),                      # float32 subnormal with a short fraction
])
def test_bfloat16_rounding(x, want):
    assert codec.round_bf16(f32([x]))[0] == np.float32(want)


@pytest.mark.parametrize("x, want", [
    (1.0 + 2.0 ** -11, 1.0),                  # tie: even
    (1.0 + 3 * 2.0 ** -11, 1.0 + 2.0 ** -9),  # tie between odd and even: even
    (2.0 ** -24, 2.0 ** -24),                 # smallest subnormal
    (2.0 ** -25, 0.0),                        # half of it: tie to even (0)
    (3 * 2.0 ** -26, 2.0 ** -24),             # 0.75 of it: up
    (65504.0, 65504.0),                       # largest finite
    (2.0 ** -14, 2.0 ** -14),                 # smallest normal
])
def test_float16_rounding(x, want):
    assert codec.round_f16(f32([x]))[0] == np.float32(want)


@pytest.mark.parametrize("m, want", [
    (3.0, 4.0), (4.0, 4.0), (4.000001, 8.0), (0.75, 1.0), (0.0, 1.0),
    (1e-40, 2.0 ** -126), (2.0 ** -126, 2.0 ** -126), (1e39, 2.0 ** 127),
])
def test_power_of_two_scale(m, want):
    assert codec.pow2_at_least(m) == want


def test_scale_is_per_block_id_maximum():
    ids = np.array([2, 0, 2], dtype=np.uint16)
    vals = np.zeros((3, 64), dtype=np.float32)
    vals[0, 5] = 3.0
    vals[1, 0] = -0.3
    vals[2, 63] = -5.0
    s = codec.block_scales(ids, vals, nb=4)
    np.testing.assert_array_equal(s, [0.5, 1.0, 8.0, 1.0])


@pytest.mark.parametrize("storage", [codec.BF16, codec.F16])
def test_encode_decode_error_bound_and_idempotence(storage):
    rng = np.random.default_rng(5)
    nb = 8
    ids = rng.integers(0, nb, 400).astype(np.uint16)
    # per block id magnitudes spanning many decades, values within a block spanning 2^-9
    mag = 10.0 ** rng.uniform(-30, 3, nb)
    vals = (mag[ids][:, None] * rng.uniform(2.0 ** -9, 1.0, (400, 64))).astype(np.float32)
    out = codec.encode_decode(ids, vals, nb, storage)
    s = codec.block_scales(ids, vals, nb)[ids][:, None]
    err = np.abs(out.astype(np.float64) - vals)
    bound = codec.unit_roundoff(storage) * np.abs(vals) + codec.subnormal_floor(storage) * s
    assert np.all(err <= bound * (1 + 1e-12))
    # stored values are fixed points of storing (same scales): a restart changes nothing
    np.testing.assert_array_equal(codec.encode_decode(ids, out, nb, storage), out)


def test_bfloat16_codes_equal_unscaled_rounding():
    """With power-of-two scales the bfloat16 form is plain bfloat16 rounding of f."""
    rng = np.random.default_rng(6)
    ids = rng.integers(0, 4, 50).astype(np.uint16)
    vals = (10.0 ** rng.uniform(-20, 2, (50, 64))).astype(np.float32)
    np.testing.assert_array_equal(codec.encode_decode(ids, vals, 4, codec.BF16), codec.round_bf16(vals))
