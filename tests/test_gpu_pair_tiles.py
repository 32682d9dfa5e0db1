"""GPU parity of the CTA-pair tensor-core GEMM (256 x 256 tiles over two SMs,
tcgen05 cta_group::2) against the one-CTA GEMM and the oracle.

The operator's four GEMMs run on CTA pairs when their 256 x 256 tiles fill
most SM pairs (option tc_pair 0); tc_pair 2 forces pairs wherever the shape
allows and tc_pair 1 turns them off.  Both forms compute the same bf16
products with FP32 accumulation, so on a spike image (exact first-GEMM
outputs) they agree with the emulation to the derived bound, and on dense
inputs with each other within the bound of the FP32 accumulation."""
import numpy as np
import pytest

from gpu_common import OracleProblem, check_bf16_operator, lib, rel, setup_ctx, torch
from oracle import kron, lam as olam, pcg as opcg
from paper_2311_15393_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kpsvd():
    return lib()


def _ctx(kpsvd, pr, pair):
    ctx = kpsvd.KpContext(0)
    ctx.kp_set_option("tc_pair", pair)
    P = pr.P
    ctx.kp_setup(kpsvd.to_device(P.psf), P.n_r, P.n_c, P.center, P.bc, P.op_rank, "bf16", "f16", "f32", "projected")
    torch.cuda.synchronize()
    return ctx


@pytest.mark.parametrize("shape", [(512, 512), (768, 512), (512, 1024)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_pair_tiles_operator(kpsvd, shape):
    """A, A^T against the emulation (spike and dense images) with pairs forced,
    K p against the one-CTA GEMMs, and the accurate operator (kp_forward,
    six bf16 products per GEMM) against the oracle's b."""
    n_r, n_c = shape
    pr = OracleProblem("deblur1024_mixed", n=max(n_r, n_c), shape=shape, rank=4)
    with _ctx(kpsvd, pr, 2) as c2, _ctx(kpsvd, pr, 1) as c1:
        check_bf16_operator(kpsvd, c2, pr, n_r, n_c)
        X = synth.random_matrix(n_r, n_c, 5)
        x = kpsvd.to_device(X, torch.float32)
        q2, q1 = torch.empty_like(x), torch.empty_like(x)
        c2.kp_apply_K(x, q2, 0.02)
        c1.kp_apply_K(x, q1, 0.02)
        d = rel(kpsvd.from_device(q2, n_r, n_c), kpsvd.from_device(q1, n_r, n_c))
        print(f"{shape}: K p, CTA pairs vs one CTA {d:.2e}")
        assert d < 2e-3
        xt = kpsvd.to_device(pr.P.x_true, torch.float32)
        g = kpsvd.to_device(pr.P.noise_dirs[0], torch.float32)
        b = torch.empty_like(xt)
        c2.kp_forward(xt, g, pr.P.noise_levels[0], b)
        assert rel(kpsvd.from_device(b, n_r, n_c), pr.B) < 2e-6


def test_pair_tiles_solve(kpsvd):
    """512 x 512, pairs forced: GCV lambda and FPCG to 1e-7 reach the oracle's
    x_lambda to 1e-4 within +3 iterations of the oracle's FP64 FPCG."""
    pr = OracleProblem("deblur1024_mixed", n=512, rank=4)
    lam = olam.choose_lambda(pr.kp, pr.B, "gcv")
    x_star = opcg.tik_exact(pr.op, pr.kp, pr.B, lam, tol=1e-10)
    _, io = opcg.tik_pcg(pr.op, pr.kp, pr.B, lam, 1e-7, 500, True)
    with _ctx(kpsvd, pr, 2) as ctx:
        b = kpsvd.to_device(pr.B, torch.float32)
        x = torch.zeros_like(b)
        info = ctx.tik_pcg(b, lam, 1e-7, 500, True, x)
        err = rel(kpsvd.from_device(x, 512, 512), x_star)
        print(f"512^2 pairs: {info.iters} iterations (oracle {io.iters}), rel. error {err:.2e}")
    assert info.status == kpsvd.KP_OK
    assert err < 1e-4
    assert info.iters <= io.iters + 3
