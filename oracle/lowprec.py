"""Rounding to reduced-precision formats, for checks of reduced-precision
kernels against FP64 arithmetic on the same rounded values (the idea of
Section 4: round to the target format at chosen points, compute in higher
precision).  All functions take and return float64 arrays; rounding is
round-to-nearest-even from the float32 value, as a float32 -> narrow
conversion on the GPU does.
"""
from __future__ import annotations

import numpy as np


def to_fp32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def to_bf16(x):
    """float64 -> float32 (RNE) -> bfloat16 (RNE), returned as float64."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


def to_fp16(x):
    """float64 -> float32 (RNE) -> IEEE binary16 (RNE, with subnormals)."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    return f.astype(np.float16).astype(np.float64)


E4M3_MAX = 448.0


def to_e4m3(x):
    """float64 -> float32 -> FP8 E4M3 (bias 7, 3 mantissa bits, subnormal
    quantum 2^-9, no infinities), round-to-nearest-even, saturating at +-448."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)
    a = np.abs(f)
    m, e = np.frexp(a)                      # a = m 2^e, m in [0.5, 1)
    ex = np.maximum(e - 1, -6)              # floor(log2 a), clamped to the subnormal range
    q = np.ldexp(1.0, ex - 3)               # spacing of representable values
    y = np.rint(a / q) * q
    y = np.minimum(y, E4M3_MAX)
    y = np.where(a == 0, 0.0, y)
    return np.sign(f) * y


def to_mxfp8(x, axis: int = -1, block: int = 32):
    """Block-scaled FP8 (the MX format: E4M3 elements with one power-of-two
    scale per `block` consecutive elements along `axis`, the contraction
    axis of a product).  The scale is 2^(floor(log2 amax) - 8), 8 being
    E4M3's largest normal exponent, so each block's largest element lands in
    [256, 512) before the (saturating) E4M3 rounding; an all-zero block stays
    zero.  Returns the represented values (scale x element) as float64."""
    a = np.moveaxis(np.asarray(x, dtype=np.float64), axis, -1)
    n = a.shape[-1]
    pad = (-n) % block
    b = np.concatenate([a, np.zeros(a.shape[:-1] + (pad,))], axis=-1) if pad else a
    b = b.reshape(b.shape[:-1] + (-1, block))
    amax = np.abs(b).max(axis=-1, keepdims=True)
    _, e = np.frexp(np.where(amax > 0, amax, 1.0))  # amax = m 2^e, m in [0.5, 1)
    scale = np.ldexp(1.0, (e - 1) - 8)
    y = to_e4m3(b / scale) * scale
    y = np.where(amax > 0, y, 0.0).reshape(b.shape[:-2] + (-1,))[..., :n]
    return np.moveaxis(y, -1, axis)


ROUND = {"f64": lambda x: np.asarray(x, dtype=np.float64), "f32": to_fp32,
         "bf16": to_bf16, "f16": to_fp16, "e4m3": to_e4m3}
