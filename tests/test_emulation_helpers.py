"""The reduced-precision emulations that several GPU parity tests compare
against (tests/gpu_common.py) are pinned to the FP64 oracle on the CPU: with
every rounding replaced by the identity they reduce to the oracle's operator
and preconditioner solve (so they compute the same mathematics, and the
E4M3 emulation's power-of-two scales cancel exactly), and with rounding they
stay within the format's error."""
import numpy as np
import pytest

from gpu_common import emulate_apply_A_bf16, emulate_minv, rel
from oracle import kpsvd as okp, kron, lowprec as lp
from paper_2311_15393_gb300 import synth


@pytest.fixture(scope="module")
def problem():
    n_r, n_c = 48, 40
    P = synth.gaussian_psf(n_r, n_c, 24, 20, 2.0, 1.3, 0.5)
    op = kron.kron_operator(P, (24, 20), "reflexive", rank=3)
    kp = okp.kp_svd(op, "projected")
    rng = np.random.default_rng(4)
    return op, kp, rng.standard_normal((n_r, n_c)), rng.standard_normal((n_r, n_c))


@pytest.fixture
def exact(monkeypatch):
    ident = lambda x: np.asarray(x, dtype=np.float64)  # noqa: E731
    for name in ("to_fp32", "to_bf16", "to_fp16", "to_e4m3"):
        monkeypatch.setattr(lp, name, ident)
    for key in list(lp.ROUND):
        monkeypatch.setitem(lp.ROUND, key, ident)


def test_emulations_without_rounding_are_the_oracle(problem, exact):
    op, kp, X, R = problem
    lam = 0.02
    np.testing.assert_allclose(emulate_apply_A_bf16(op, X), kron.apply_A(op, X), rtol=0,
                               atol=1e-13 * np.abs(kron.apply_A(op, X)).max())
    Z64 = okp.precond_apply(kp, okp.precond_scale(kp.Sigma, lam), R)
    for fmt in ("f16", "bf16", "e4m3"):
        np.testing.assert_allclose(emulate_minv(kp, kp.Sigma, R, lam, fmt), Z64, rtol=0,
                                   atol=1e-11 * np.abs(Z64).max())


def test_emulations_with_rounding_stay_within_the_format_error(problem):
    """bf16 operator: two GEMMs with bf16 operands, relative error a few
    2^-9; FP16 / BF16 (hi + lo factors) preconditioner within 5e-3 of FP64 for
    a broadband residual; E4M3 within sqrt(8) 2^-4 / sqrt(3) (eight roundings)."""
    op, kp, X, R = problem
    lam = 0.02
    e_op = rel(emulate_apply_A_bf16(op, X), kron.apply_A(op, X))
    assert 1e-5 < e_op < 4 * 2.0 ** -9
    Z64 = okp.precond_apply(kp, okp.precond_scale(kp.Sigma, lam), R)
    for fmt, bound in (("f16", 5e-3), ("bf16", 5e-3), ("e4m3", np.sqrt(8.0) * 2.0 ** -4 / np.sqrt(3.0))):
        e = rel(emulate_minv(kp, kp.Sigma, R, lam, fmt), Z64)
        assert 0 < e < bound, (fmt, e)
