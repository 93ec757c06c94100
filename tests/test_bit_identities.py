"""Exact binary32 identities the FP32 kernel uses instead of int<->float
conversion instructions (checked here in IEEE binary32 with numpy)."""
import numpy as np


def f32_from_bits(b):
    return np.asarray(b, dtype=np.uint32).view(np.float32)


def test_uniform_from_mantissa_bits_is_exact():
    # U(w) = (w>>9 + 1/2) 2^-23  ==  float(1.m) - (1 - 2^-24), for all 2^23 values
    k = np.arange(1 << 23, dtype=np.uint32)
    got = f32_from_bits(np.uint32(0x3F800000) | k) - np.float32(0.99999994)
    want = (k.astype(np.float64) + 0.5) * 2.0**-23
    assert np.float32(0.99999994) == np.float32(1.0 - 2.0**-24)
    assert np.array_equal(got.astype(np.float64), want)


def test_small_integer_from_mantissa_bits_is_exact():
    u = np.arange(0, 1 << 23, 7, dtype=np.uint32)
    got = f32_from_bits(np.uint32(0x4B000000) | u) - np.float32(8388608.0)
    assert np.array_equal(got.astype(np.int64), u.astype(np.int64))


def test_floor_by_round_down_add():
    # round-down(f + 1.5*2^23) = floor(f) + 1.5*2^23 for f in [0, 2^22]; the
    # binary32 spacing there is 1, and the exact sum is formed in binary64
    rng = np.random.default_rng(0)
    f = np.concatenate([rng.uniform(0, 200, 100000), np.arange(0, 200, 0.25),
                        [0.0, 1.0 - 2**-24, 63.0, 62.99999]]).astype(np.float32)
    exact = f.astype(np.float64) + 12582912.0
    rd = np.floor(exact)  # spacing 1 at this magnitude: round-down = floor
    bits = rd.astype(np.float32).view(np.uint32).astype(np.int64) - 0x4B400000
    assert np.array_equal(bits, np.floor(f.astype(np.float64)).astype(np.int64))
