"""Observed data for a synthetic problem (Section 5): b = A x_true + e with the
noise scaled so that ||e||_2 / ||A x_true||_2 equals the noise level.
The noise direction g (standard normal) is drawn by the input generator."""
from __future__ import annotations

import numpy as np

from .kron import KronOperator, apply_A


def observe(op: KronOperator, X_true: np.ndarray, g: np.ndarray, noise_level: float):
    """Returns (B, ||e||)."""
    Bt = apply_A(op, X_true)
    e = noise_level * np.linalg.norm(Bt) * g / np.linalg.norm(g)
    return Bt + e, float(np.linalg.norm(e))
