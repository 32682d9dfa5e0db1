"""GPU parity of the tensor-core path at sizes that end in partial tiles.

The tensor-core GEMMs use 128-row tiles, 64- to 256-column tiles and k-blocks
of 64 elements; the other GPU tests use 64 x 64 (one partial tile) and
multiples of 128.  Here every dimension spans several tiles and ends in a
ragged tail: 208 = 128 + 80 rows and 3 k-blocks + 16, 144 = 128 + 16 rows and
2 k-blocks + 16; (144, 256) runs the operator's per-term (batched) GEMMs with
a ragged output width.  Loads beyond the edges are zero-filled by TMA and the
epilogue stores only in-range rows and columns, so the results must match
the oracle exactly as at the tile-aligned sizes."""
import numpy as np
import pytest

from gpu_common import GpuKpsvd, OracleProblem, check_bf16_operator, emulate_minv, lib, rel, setup_ctx, torch
from oracle import kpsvd as okp, kron, lam as olam, pcg as opcg
from paper_2311_15393_gb300 import synth

pytestmark = pytest.mark.gpu

SHAPES = [(208, 208), (144, 208), (144, 256)]


@pytest.fixture(scope="module")
def kpsvd():
    return lib()


def _problem(shape, psf=None):
    return OracleProblem("deblur256_fp32", n=256, shape=shape, rank=3, psf=psf)


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{s[0]}x{s[1]}")
def test_operator_with_tile_tails(kpsvd, shape):
    """Inner BF16 operator A and A^T against the emulation (check_bf16_operator);
    the accurate operator (kp_forward) against the oracle's b, which also
    checks the GPU's terms against the oracle's."""
    n_r, n_c = shape
    pr = _problem(shape)
    with setup_ctx(kpsvd, pr, "bf16", "f16", "f32") as ctx:
        check_bf16_operator(kpsvd, ctx, pr, n_r, n_c)
        xt = kpsvd.to_device(pr.P.x_true, torch.float32)
        g = kpsvd.to_device(pr.P.noise_dirs[0], torch.float32)
        b = torch.empty_like(xt)
        ctx.kp_forward(xt, g, pr.P.noise_levels[0], b)
        assert rel(kpsvd.from_device(b, n_r, n_c), pr.B) < 2e-6


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{s[0]}x{s[1]}")
def test_fp16_preconditioner_with_tile_tails(kpsvd, shape):
    """FP16 KP-SVD solve against its emulation on the GPU's own factors and
    spectrum (so both sides round the same V) and against FP64 (a narrow PSF
    keeps the factor singular values far above rounding level)."""
    n_r, n_c = shape
    psf = synth.gaussian_psf(n_r, n_c, n_r // 2, n_c // 2, 0.8, 0.6, 0.3)
    pr = _problem(shape, psf=psf)
    assert min(pr.kp.sc.min(), pr.kp.sr.min()) > 1e-3 * max(pr.kp.sc[0], pr.kp.sr[0])
    lam = 0.02
    with setup_ctx(kpsvd, pr, "f32", "f16", "f32") as ctx:
        R = synth.random_matrix(n_r, n_c, 5)
        r = kpsvd.to_device(R, torch.float32)
        z = torch.empty_like(r)
        ctx.kp_apply_Minv(r, z, lam)
        Z = kpsvd.from_device(z, n_r, n_c)
        gk = GpuKpsvd(ctx)
        assert rel(Z, emulate_minv(gk, gk.Sigma, R, lam, "f16")) < 0.5 * 2.0 ** -11
        assert rel(Z, okp.precond_apply(pr.kp, okp.precond_scale(pr.kp.Sigma, lam), R)) < 5e-3


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{s[0]}x{s[1]}")
def test_solve_with_tile_tails(kpsvd, shape):
    """GCV lambda and the BF16 / FP16 / FP32 FPCG solve against the oracle:
    lambda by the oracle's GCV value (FP32 setup), x within 1e-4 of x_lambda."""
    n_r, n_c = shape
    pr = _problem(shape)
    bh = olam.spectral_coeffs(pr.kp, pr.B)
    lam_o = olam.choose_lambda(pr.kp, pr.B, "gcv")
    with setup_ctx(kpsvd, pr, "bf16", "f16", "f32") as ctx:
        b = kpsvd.to_device(pr.B, torch.float32)
        lam = ctx.choose_lambda(b, "gcv")
        x = torch.zeros_like(b)
        info = ctx.tik_pcg(b, lam_o, 1e-7, 500, True, x)
        X = kpsvd.from_device(x, n_r, n_c)
    assert olam.gcv(pr.kp.Sigma, bh, lam) <= olam.gcv(pr.kp.Sigma, bh, lam_o) * (1.0 + 1e-5)
    assert info.status == kpsvd.KP_OK
    x_star = opcg.tik_exact(pr.op, pr.kp, pr.B, lam_o, tol=1e-10)
    cond = (np.max(np.abs(pr.kp.Sigma)) ** 2 + lam_o ** 2) / lam_o ** 2
    assert rel(X, x_star) < (1e-4 if cond <= 1e4 else cond * 1e-7)
