"""Full-size parity: the 1024 x 1024 workload (rank-4 BF16 tensor-core
operator, FP16 preconditioner, FP32 vectors, FPCG to relative residual 1e-7)
in the configuration the benchmark times, against the FP64 oracle's x_lambda
and GCV lambda.  The oracle solves the same system in FP64 on the host
(KP-SVD preconditioned CG to 1e-9, far below the 1e-4 compared), so this runs for a minute or two."""
import numpy as np
import pytest

from gpu_common import OracleProblem, lib, rel, setup_ctx, torch
from oracle import lam as olam, pcg as opcg

pytestmark = pytest.mark.gpu

TOL = 1e-7


@pytest.fixture(scope="module")
def kpsvd():
    return lib()


@pytest.fixture(scope="module")
def problems():
    return [OracleProblem("deblur1024_mixed", noise_idx=i) for i in (0, 1)]


@pytest.mark.parametrize("noise_idx", [0, 1])
def test_fullsize_lambda_and_solution_match_oracle(kpsvd, problems, noise_idx):
    pr = problems[noise_idx]
    lam_o = olam.choose_lambda(pr.kp, pr.B, "gcv")
    x_star = opcg.tik_exact(pr.op, pr.kp, pr.B, lam_o, tol=1e-9)
    _, io = opcg.tik_pcg(pr.op, pr.kp, pr.B, lam_o, TOL, 500, True)   # FP64-preconditioned FPCG
    with setup_ctx(kpsvd, pr, "bf16", "f16", "f32") as ctx:
        b = kpsvd.to_device(pr.B, torch.float32)
        lam_g = ctx.choose_lambda(b, "gcv")
        assert abs(lam_g / lam_o - 1.0) < 1e-4
        # the oracle's lambda on both sides, as the parity run prescribes
        x = torch.zeros_like(b)
        info = ctx.tik_pcg(b, lam_o, TOL, 500, True, x)
        assert info.status == kpsvd.KP_OK
        X = kpsvd.from_device(x, pr.P.n_r, pr.P.n_c)
        err = rel(X, x_star)
        print(f"1024^2 noise {pr.P.noise_levels[noise_idx]}: lambda gpu {lam_g:.10g} oracle {lam_o:.10g}, "
              f"iterations {info.iters} ({info.replacements} replacements; oracle FP64 FPCG {io.iters}), "
              f"rel. error {err:.2e}")
        assert err < 1e-4
        assert info.iters <= io.iters + 3
        # sampled entries recomputed one by one from the oracle's solution
        rng = np.random.default_rng(7)
        idx = rng.integers(0, X.size, 64)
        np.testing.assert_allclose(X.reshape(-1)[idx], x_star.reshape(-1)[idx],
                                   rtol=0, atol=1e-3 * np.abs(x_star).max())


def test_fullsize_e4m3_preconditioner(kpsvd, problems):
    """The 1024^2 workload at 0.5% noise with the FP8 (E4M3) preconditioner
    (each apply ~7% off FP64, a property of the 3-bit mantissa): FPCG still
    converges towards x_lambda, but slowly, and stops as stagnated (the true
    residual no longer halves over three replacements) near 2.8e-7 after
    ~445 iterations, against 110 for FP16; its error against the oracle's
    x_lambda there, 2.6e-4 when measured, is above the metric's 1e-4.  The
    test pins that behaviour: a normal stop (converged or stagnated) with the
    error within 1e-3; the FP16 preconditioner is the one that meets 1e-4."""
    pr = problems[0]
    lam_o = olam.choose_lambda(pr.kp, pr.B, "gcv")
    x_star = opcg.tik_exact(pr.op, pr.kp, pr.B, lam_o, tol=1e-9)
    with setup_ctx(kpsvd, pr, "bf16", "e4m3", "f32") as ctx:
        b = kpsvd.to_device(pr.B, torch.float32)
        x = torch.zeros_like(b)
        info = ctx.tik_pcg(b, lam_o, TOL, 500, True, x, check=False)
        err = rel(kpsvd.from_device(x, pr.P.n_r, pr.P.n_c), x_star)
        print(f"1024^2 E4M3 preconditioner: status {info.status}, {info.iters} iterations, "
              f"{info.replacements} replacements, rel_res {info.rel_res:.2e}, rel. error vs x_lambda {err:.2e}")
    assert info.status in (kpsvd.KP_OK, kpsvd.KP_ENOCONV)
    assert err < 1e-3
