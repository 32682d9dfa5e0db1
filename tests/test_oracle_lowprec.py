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
