"""Pins for the reduced-precision rounding helpers (oracle/lowprec.py):
numpy's own IEEE casts, and hand-worked bf16 / e4m3 values."""
import numpy as np

from oracle import lowprec as lp


def test_fp16_and_fp32_match_numpy_casts():
    x = np.random.default_rng(0).standard_normal(1000) * np.logspace(-9, 4, 1000)
    np.testing.assert_array_equal(lp.to_fp32(x), x.astype(np.float32).astype(np.float64))
    np.testing.assert_array_equal(lp.to_fp16(x), x.astype(np.float32).astype(np.float16).astype(np.float64))


def test_bf16_hand_values():
    # 8 significant bits: spacing 2^-7 in [1, 2); ties to even
    assert lp.to_bf16(1.0 + 2.0 ** -8) == 1.0                      # tie -> even (1.0)
    assert lp.to_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2 * 2.0 ** -7  # tie -> even (1 + 2^-6)
    assert lp.to_bf16(1.0 + 2.0 ** -8 + 2.0 ** -12) == 1.0 + 2.0 ** -7
    # rounded from the float32 value, as the GPU's conversion is: 2^-30 is
    # lost in float32, leaving the tie 1 + 2^-8, which goes to even (1.0)
    assert lp.to_bf16(1.0 + 2.0 ** -8 + 2.0 ** -30) == 1.0
    assert lp.to_fp16(1.0 + 2.0 ** -11 + 2.0 ** -30) == 1.0       # same for fp16 (tie 1 + 2^-11)
    assert lp.to_bf16(-3.0) == -3.0
    assert lp.to_bf16(2.0 ** -130) > 0                              # subnormal range kept
    x = np.random.default_rng(1).standard_normal(1000)
    assert np.max(np.abs(lp.to_bf16(x) - x) / np.abs(x)) <= 2.0 ** -8


def test_e4m3_hand_values():
    assert lp.to_e4m3(448.0) == 448.0
    assert lp.to_e4m3(1e6) == 448.0                # saturating
    assert lp.to_e4m3(-500.0) == -448.0
    assert lp.to_e4m3(2.0 ** -9) == 2.0 ** -9      # smallest subnormal
    assert lp.to_e4m3(2.0 ** -11) == 0.0           # below half the smallest subnormal
    assert lp.to_e4m3(1.0625) == 1.0               # tie between 1.0 and 1.125 -> even
    assert lp.to_e4m3(1.1875) == 1.25              # tie between 1.125 and 1.25 -> even
    assert lp.to_e4m3(0.3) == 0.3125               # spacing 2^-5 in [0.25, 0.5)
    assert lp.to_e4m3(15.5) == 16.0
    vals = lp.to_e4m3(np.linspace(-448, 448, 20001))
    assert len(np.unique(np.abs(vals))) <= 127


def test_mxfp8_hand_values():
    """Block of 4 with amax 3.0 = 1.5 * 2^1: scale 2^(1 - 8) = 2^-7, elements
    x * 128 rounded to E4M3 (spacing 32 in [256, 512), 16 in [128, 256)), so
    3.0 -> 384 exactly, 1.3 -> 166.4 -> 160 (x 2^-7 = 1.25), 0.01 -> 1.28 ->
    1.25 (spacing 2^-3 in [1, 2)), -2.9 -> -371.2 -> -384 (-3.0).  Second
    block, amax 3.75 = 1.875 * 2^1, same scale: 3.75 -> 480 saturates to 448
    (3.5), which only the block maximum's binade [256, 512) produces (a
    scale one binade larger would give 240, exact); 0.5 -> 64, -1 -> -128,
    0 -> 0."""
    x = np.array([3.0, 1.3, 0.01, -2.9, 3.75, 0.5, -1.0, 0.0])
    np.testing.assert_array_equal(lp.to_mxfp8(x, block=4), [3.0, 1.25, 1.25 / 128, -3.0, 3.5, 0.5, -1.0, 0.0])


def test_mxfp8_blocks_are_independent_and_zero_blocks_stay_zero():
    """Each block is scaled by its own maximum: a block of tiny values keeps
    E4M3's relative precision (2^-4 for normal elements) instead of flushing
    to zero as one shared scale would, except that scaled values in (448,
    512) saturate to 448 (the MX scale puts the maximum in [256, 512)); an
    all-zero block stays zero; a ragged last block is padded; the axis
    argument selects the blocks."""
    rng = np.random.default_rng(2)
    big = rng.uniform(-1e3, 1e3, 32)
    tiny = rng.uniform(-1e-6, 1e-6, 32)
    x = np.concatenate([big, tiny, np.zeros(32), rng.standard_normal(5)])
    y = lp.to_mxfp8(x)
    for blk in (big, tiny):
        amax = np.abs(blk).max()
        scale = 2.0 ** (np.frexp(amax)[1] - 1 - 8)
        yb = lp.to_mxfp8(blk)
        sat = np.abs(blk) / scale > 448.0
        normal = (np.abs(blk) >= amax / 2 ** 6) & ~sat   # E4M3 normals after the block scale
        assert np.all(np.abs(yb - blk)[normal] <= 2.0 ** -4 * np.abs(blk)[normal])
        np.testing.assert_array_equal(np.abs(yb[sat]), 448.0 * scale)
    np.testing.assert_array_equal(y[:32], lp.to_mxfp8(big))
    np.testing.assert_array_equal(y[32:64], lp.to_mxfp8(tiny))
    assert np.all(y[64:96] == 0)
    M = rng.standard_normal((3, 64))
    np.testing.assert_array_equal(lp.to_mxfp8(M.T, axis=0), lp.to_mxfp8(M, axis=1).T)
