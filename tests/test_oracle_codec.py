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
    (3.0, 4.0), (4.0, 4.0), (4.000001, 8.0), (0.75, 1.0), (0.0, 2.0 ** -126),
    (1e-40, 2.0 ** -126), (2.0 ** -126, 2.0 ** -126), (2.0 ** 126, 2.0 ** 126), (1e38, 2.0 ** 126),
])
def test_power_of_two_scale(m, want):
    assert codec.pow2_at_least(m) == want


def test_scale_is_per_chunk_maximum():
    """Four chunks of 16 values per block (values 16 q .. 16 q + 15), each with its own
    scale: the smallest power of two >= its largest magnitude, 2^-126 for an all-zero
    chunk."""
    vals = np.zeros((2, 64), dtype=np.float32)
    vals[0, 5] = 3.0       # chunk 0 of block 0
    vals[0, 16] = -0.3     # chunk 1
    vals[0, 47] = 0.25     # chunk 2 (a power of two is its own scale)
    vals[1, 63] = -5.0     # chunk 3 of block 1
    z = 2.0 ** -126
    np.testing.assert_array_equal(codec.chunk_scales(vals), [[4.0, 0.5, 0.25, z], [z, z, z, 8.0]])


@pytest.mark.parametrize("storage", [codec.BF16, codec.F16])
def test_encode_decode_error_bound_and_idempotence(storage):
    rng = np.random.default_rng(5)
    # per block magnitudes spanning many decades, values within a chunk spanning 2^-9
    mag = 10.0 ** rng.uniform(-30, 3, (400, 4, 1))
    vals = (mag * rng.uniform(2.0 ** -9, 1.0, (400, 4, 16))).astype(np.float32).reshape(400, 64)
    out = codec.encode_decode(vals, storage)
    s = np.repeat(codec.chunk_scales(vals), 16, axis=1)
    err = np.abs(out.astype(np.float64) - vals)
    bound = codec.unit_roundoff(storage) * np.abs(vals) + codec.subnormal_floor(storage) * s
    assert np.all(err <= bound * (1 + 1e-12))
    # stored values are fixed points of storing: a restart changes nothing
    np.testing.assert_array_equal(codec.encode_decode(out, storage), out)


def test_float16_chunks_keep_small_values_that_one_scale_per_id_would_lose():
    """Two chunks of one block id, 10^-12 apart in magnitude: each keeps 11 significant
    bits under its own scale, where a single scale for both would flush the small one."""
    vals = np.zeros((2, 64), dtype=np.float32)
    vals[0, :16] = 1.0 + np.arange(16) / 64.0
    vals[1, :16] = 1e-12 * (1.0 + np.arange(16) / 64.0)
    out = codec.encode_decode(vals, codec.F16)
    rel = np.abs(out[:, :16] - vals[:, :16]) / vals[:, :16]
    assert rel.max() <= 2.0 ** -11
    assert codec.round_f16(vals[1, :16] / np.float32(2.0))[0] == 0.0  # one scale (2) for both: lost


def test_bfloat16_codes_equal_unscaled_rounding():
    """With power-of-two scales the bfloat16 form is plain bfloat16 rounding of f."""
    rng = np.random.default_rng(6)
    vals = (10.0 ** rng.uniform(-20, 2, (50, 64))).astype(np.float32)
    np.testing.assert_array_equal(codec.encode_decode(vals, codec.BF16), codec.round_bf16(vals))


def test_shock_window_needs_scales_finer_than_one_per_block_id():
    """The premise of the GPU's float16 shock-window tests: across the shock front (24 x 4
    x 4 cells at x = 52 of the shock workload, threshold 1e-15 of the peak) one scale per
    block id would put about 0.5% of the values below float16's normal range (relative
    error up to 1e-2), while one scale per chunk keeps every value normal (relative error
    within 2^-11)."""
    from paper_2504_21450_gb300 import inputs
    cfg = inputs.CONFIGS["shock"]
    init = inputs.generate(cfg, origin=(52, 0, 0), size=(24, 4, 4), thr=1e-15 * inputs.peak_f(cfg))
    v = np.abs(init.vals.astype(np.float64))
    ids = init.ids.astype(np.int64)
    s_id = np.zeros(ids.max() + 1)
    np.maximum.at(s_id, ids, v.max(axis=1))
    s_id = codec.pow2_at_least(s_id)[ids][:, None]
    s_chunk = np.repeat(codec.chunk_scales(init.vals), 16, axis=1)
    nz = v > 0
    assert np.mean((v < 2.0 ** -14 * s_id)[nz]) > 1e-3
    assert not np.any((v < 2.0 ** -14 * s_chunk)[nz])
    rel = np.abs(codec.encode_decode(init.vals, codec.F16) - v)[nz] / v[nz]
    assert rel.max() <= 2.0 ** -11
