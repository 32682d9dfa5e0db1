"""The half-precision setup (option setup_half; the paper's future work,
Section 3 after eq. PreconSolve): the products that form the factor SVDs'
V_c, V_r and the KP spectrum take bf16 inputs with FP32 accumulation on the
tensor cores.  The spectrum then agrees with the oracle's to bf16 level,
and flexible PCG with the resulting preconditioner still reaches the
oracle's x_lambda to the metric's 1e-4, in about the iterations of the
FP32 setup."""
import numpy as np
import pytest

from gpu_common import OracleProblem, lib, rel, torch
from oracle import lam as olam, pcg as opcg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kpsvd():
    return lib()


@pytest.mark.parametrize("name,n", [("deblur256_fp32", 256), ("deblur1024_mixed", 512)])
def test_half_setup_solve(kpsvd, name, n):
    pr = OracleProblem(name, n=n)
    P = pr.P
    lam = olam.choose_lambda(pr.kp, pr.B, "gcv")
    x_star = opcg.tik_exact(pr.op, pr.kp, pr.B, lam, tol=1e-10)
    res = {}
    for half in (0, 1):
        with kpsvd.KpContext(0) as ctx:
            ctx.kp_set_option("setup_half", half)
            ctx.kp_setup(kpsvd.to_device(P.psf), n, n, P.center, P.bc, P.op_rank, "bf16", "f16", "f32", "projected")
            sig = ctx.kp_get_spectrum()
            b = kpsvd.to_device(pr.B, torch.float32)
            x = torch.zeros_like(b)
            info = ctx.tik_pcg(b, lam, 1e-7, 500, True, x)
            res[half] = (info, rel(kpsvd.from_device(x, n, n), x_star),
                         np.abs(sig - pr.kp.Sigma).max() / np.abs(pr.kp.Sigma).max())
    (i0, e0, s0), (i1, e1, s1) = res[0], res[1]
    print(f"{name} {n}^2: spectrum error (max / max|Sigma|) fp32 setup {s0:.2e}, half setup {s1:.2e}; "
          f"iterations {i0.iters} / {i1.iters}; error vs x_lambda {e0:.2e} / {e1:.2e}")
    assert s1 < 2.0 ** -7
    assert i1.status == kpsvd.KP_OK
    assert e1 < 1e-4
    assert i1.iters <= i0.iters + 3
