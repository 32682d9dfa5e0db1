"""GPU parity of kp_setup, the operator hooks and the preconditioner solve
against the FP64 oracle (all calls through the C ABI)."""
import numpy as np
import pytest

from gpu_common import GpuKpsvd, OracleProblem, check_bf16_operator, emulate_minv, lib, rel, setup_ctx, torch, vt
from oracle import kpsvd as okp, kron
from paper_2311_15393_gb300 import synth

pytestmark = pytest.mark.gpu

CASES = [
    # (workload, n, shape, bc, rank)
    ("deblur64_fp64", None, None, "zero", 0),          # full 64 x 64 workload, full rank
    ("deblur256_fp32", 64, None, "reflexive", 3),
    ("deblur256_fp32", 64, (48, 40), "reflexive", 4),  # rectangular, off-centre sizes
    ("deblur64_fp64", 64, (40, 56), "zero", 5),
]


@pytest.fixture(scope="module")
def kpsvd():
    return lib()


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{c[1]}-{c[2]}-{c[3]}-r{c[4]}")
def test_setup_fp64_matches_oracle(kpsvd, case):
    name, n, shape, bc, rank = case
    pr = OracleProblem(name, n=n, shape=shape, bc=bc, rank=rank)
    with setup_ctx(kpsvd, pr, "f64", "f64", "f64") as ctx:
        s, U, V = ctx.kp_get_terms()
        r = pr.op.rank
        assert ctx.kp_get_rank() == r
        keep = pr.op.s > 1e-9 * pr.op.s[0]
        np.testing.assert_allclose(s[keep], pr.op.s[keep], rtol=1e-10)
        for m in range(min(3, r)):
            np.testing.assert_allclose(np.outer(U[:, m], V[:, m]), np.outer(pr.op.u[:, m], pr.op.v[:, m]),
                                       rtol=0, atol=1e-11 * np.abs(pr.P.psf).max())
        svd = ctx.kp_get_kpsvd()
        np.testing.assert_allclose(svd["sr"], pr.kp.sr, rtol=0, atol=1e-12 * pr.kp.sr[0])
        np.testing.assert_allclose(svd["sc"], pr.kp.sc, rtol=0, atol=1e-12 * pr.kp.sc[0])
        Sg = ctx.kp_get_spectrum()
        np.testing.assert_allclose(Sg, pr.kp.Sigma, rtol=0, atol=1e-11 * np.abs(pr.kp.Sigma).max())
        # factor SVDs reconstruct the factors
        A1 = pr.op.Ar[0]
        np.testing.assert_allclose(svd["Ur"] @ np.diag(svd["sr"]) @ svd["Vr"].T, A1, rtol=0, atol=1e-12)


@pytest.mark.parametrize("case", CASES[1:], ids=lambda c: f"{c[0]}-{c[2]}-{c[3]}-r{c[4]}")
def test_setup_fp32_products_match_oracle(kpsvd, case):
    """FP32 vectors: the O(n^3) products of the setup run in FP32 (rotations in
    FP64); the KP-SVD then agrees with the oracle to FP32 level, and with the
    all-FP64 setup ("setup_fp64" option) likewise."""
    name, n, shape, bc, rank = case
    pr = OracleProblem(name, n=n, shape=shape, bc=bc, rank=rank)
    out = {}
    for fp64 in (0, 1):
        ctx = kpsvd.KpContext(0)
        ctx.kp_set_option("setup_fp64", fp64)
        P = pr.P
        ctx.kp_setup(kpsvd.to_device(P.psf), P.n_r, P.n_c, P.center, P.bc, P.op_rank, "f32", "f32", "f32")
        out[fp64] = (ctx.kp_get_kpsvd(), ctx.kp_get_spectrum())
        ctx.close()
    svd, Sg = out[0]
    u32 = 2.0 ** -23
    n_max = max(pr.P.n_r, pr.P.n_c)
    np.testing.assert_allclose(svd["sr"], pr.kp.sr, rtol=0, atol=8 * n_max * u32 * pr.kp.sr[0])
    np.testing.assert_allclose(svd["sc"], pr.kp.sc, rtol=0, atol=8 * n_max * u32 * pr.kp.sc[0])
    smax = np.abs(pr.kp.Sigma).max()
    np.testing.assert_allclose(Sg, pr.kp.Sigma, rtol=0, atol=8 * n_max * u32 * smax)
    np.testing.assert_allclose(Sg, out[1][1], rtol=0, atol=8 * n_max * u32 * smax)
    for side in ("r", "c"):
        A1 = pr.op.Ar[0] if side == "r" else pr.op.Ac[0]
        U, S, V = svd["U" + side], svd["s" + side], svd["V" + side]
        np.testing.assert_allclose(U @ np.diag(S) @ V.T, A1, rtol=0, atol=8 * n_max * u32 * S[0])
        np.testing.assert_allclose(U.T @ U, np.eye(U.shape[0]), rtol=0, atol=1e-4)
        np.testing.assert_allclose(V.T @ V, np.eye(V.shape[0]), rtol=0, atol=1e-4)


@pytest.mark.parametrize("shape", [(200, 140), (12, 7)])
def test_block_jacobi_matches_oracle_and_round_form(kpsvd, shape):
    """The FP32 factor SVDs of eq. AKronSVD with the Jacobi sweeps in the
    register block form (default: blocks of 4 columns, a full sweep over two
    blocks per launch) with the second run (U from F^T) started from the
    first run's V (default), and in the one-pair-per-thread-block form
    started from the transform.  One-sided
    Jacobi in FP32 stops when no pair's inner product is above the noise
    floor m u ||A||_F (u = 2^-24 rounding, 2^-23 in the floor), so every
    singular value is fixed to a few times that floor, whatever the rotation
    order: both forms agree with the oracle, and with each other, to
    4 m 2^-23 ||A||_F, and return orthonormal U, V.  Singular vectors are
    unique (up to sign) only for isolated singular values: within a cluster
    of near-equal ones only the subspace is, and U (from a second run, or V
    with signs for a symmetric factor) may be rotated there against V.  So
    G = U^T A V must equal diag(sigma) to the same level wherever
    |sigma_i - sigma_j| exceeds 10 times it (i = j: sigma_i isolated).
    140 columns are 35 blocks (one padding block), 200 are 50; a 7-column
    factor is two blocks, one partly padding."""
    pr = OracleProblem("deblur256_fp32", shape=shape, bc="zero", rank=3)
    P = pr.P
    out = {}
    for blk in (1, 0):  # block form with the warm second run (defaults), and the former form
        ctx = kpsvd.KpContext(0)
        ctx.kp_set_option("jacobi_block", blk)
        ctx.kp_set_option("jacobi_warm_u", blk)
        ctx.kp_setup(kpsvd.to_device(P.psf), P.n_r, P.n_c, P.center, P.bc, P.op_rank, "f32", "f32", "f32")
        out[blk] = (ctx.kp_get_kpsvd(), ctx.kp_get_spectrum())
        ctx.close()
    for side in ("r", "c"):
        A1 = pr.op.Ar[0] if side == "r" else pr.op.Ac[0]
        m = A1.shape[0]
        bound = 4 * m * 2.0 ** -23 * np.linalg.norm(A1)
        s_o = pr.kp.sr if side == "r" else pr.kp.sc
        for blk in (1, 0):
            svd = out[blk][0]
            U, S, V = svd["U" + side], svd["s" + side], svd["V" + side]
            print(f"{shape} side {side} block {blk}: max |sigma - oracle| {np.abs(S - s_o).max():.2e} "
                  f"(bound {bound:.2e})")
            np.testing.assert_allclose(S, s_o, rtol=0, atol=bound)
            G = U.T @ A1 @ V - np.diag(S)
            gap = np.abs(S[:, None] - S[None, :])
            np.fill_diagonal(gap, np.inf)
            apart = gap > 10 * bound
            apart[np.diag_indices(m)] = gap.min(axis=1) > 10 * bound
            assert np.abs(G[apart]).max() <= bound, np.abs(G[apart]).max()
            np.testing.assert_allclose(U.T @ U, np.eye(m), rtol=0, atol=1e-4)
            np.testing.assert_allclose(V.T @ V, np.eye(m), rtol=0, atol=1e-4)
        np.testing.assert_allclose(out[1][0]["s" + side], out[0][0]["s" + side], rtol=0, atol=bound)


@pytest.mark.parametrize("vec", ["f64", "f32"])
@pytest.mark.parametrize("case", CASES[1:3], ids=lambda c: f"{c[2]}-{c[3]}")
def test_apply_A_and_K(kpsvd, case, vec):
    name, n, shape, bc, rank = case
    pr = OracleProblem(name, n=n, shape=shape, bc=bc, rank=rank)
    tol = 1e-12 if vec == "f64" else 2e-6
    with setup_ctx(kpsvd, pr, vec, vec, vec) as ctx:
        X = synth.random_matrix(pr.P.n_r, pr.P.n_c, 7)
        x = kpsvd.to_device(X, vt(vec))
        y = torch.empty_like(x)
        ctx.kp_apply_A(x, y, False)
        assert rel(kpsvd.from_device(y, pr.P.n_r, pr.P.n_c), kron.apply_A(pr.op, X)) < tol
        ctx.kp_apply_A(x, y, True)
        assert rel(kpsvd.from_device(y, pr.P.n_r, pr.P.n_c), kron.apply_AT(pr.op, X)) < tol
        ctx.kp_apply_K(x, y, 0.03)
        assert rel(kpsvd.from_device(y, pr.P.n_r, pr.P.n_c), kron.apply_K(pr.op, X, 0.03)) < tol


@pytest.mark.parametrize("vec", ["f64", "f32"])
def test_apply_Minv_simt(kpsvd, vec):
    pr = OracleProblem("deblur256_fp32", n=64, rank=3)
    lam = 0.02
    with setup_ctx(kpsvd, pr, vec, vec, vec) as ctx:
        R = synth.random_matrix(64, 64, 3)
        r = kpsvd.to_device(R, vt(vec))
        z = torch.empty_like(r)
        ctx.kp_apply_Minv(r, z, lam)
        Zref = okp.precond_apply(pr.kp, okp.precond_scale(pr.kp.Sigma, lam), R)
        assert rel(kpsvd.from_device(z, 64, 64), Zref) < (1e-11 if vec == "f64" else 1e-5)


def test_forward_matches_oracle(kpsvd):
    pr = OracleProblem("deblur256_fp32", n=64, rank=3)
    with setup_ctx(kpsvd, pr, "f64", "f64", "f64") as ctx:
        x = kpsvd.to_device(pr.P.x_true)
        g = kpsvd.to_device(pr.P.noise_dirs[0])
        b = torch.empty_like(x)
        en = ctx.kp_forward(x, g, pr.P.noise_levels[0], b)
        assert rel(kpsvd.from_device(b, 64, 64), pr.B) < 1e-12
        assert abs(en - pr.enorm) < 1e-12 * pr.enorm


# ------------------------------------------------------------ tensor-core paths
@pytest.mark.parametrize("n", [64, 256])
def test_tensor_core_operator_bf16(kpsvd, n):
    """Inner BF16 operator (one bf16 slice), A and A^T: equal to the bf16
    emulation of the GPU's own factors within the bound derived from FP32
    accumulation (exact-intermediate spike image and a dense random image),
    and to FP64 within bf16 rounding."""
    pr = OracleProblem("deblur256_fp32", n=n, rank=3)
    with setup_ctx(kpsvd, pr, "bf16", "f16", "f32") as ctx:
        check_bf16_operator(kpsvd, ctx, pr, n, n)


@pytest.mark.parametrize("n", [64, 256])
def test_tensor_core_accurate_operator(kpsvd, n):
    """The six-product bf16 split (used for A^T b, true residuals and
    kp_forward) is FP32-accurate."""
    pr = OracleProblem("deblur256_fp32", n=n, rank=3)
    with setup_ctx(kpsvd, pr, "bf16", "f16", "f32") as ctx:
        x = kpsvd.to_device(pr.P.x_true, torch.float32)
        g = kpsvd.to_device(pr.P.noise_dirs[0], torch.float32)
        b = torch.empty_like(x)
        ctx.kp_forward(x, g, pr.P.noise_levels[0], b)
        assert rel(kpsvd.from_device(b, n, n), pr.B) < 2e-6


@pytest.mark.parametrize("fmt", ["f16", "bf16", "e4m3"])
@pytest.mark.parametrize("n", [64, 256])
def test_tensor_core_preconditioner_vs_emulation(kpsvd, fmt, n):
    """Reduced-precision KP-SVD solve equals its emulation (same rounded
    factors, same rounding points).  A narrow PSF keeps every factor singular
    value well above rounding level, so V is unique up to column signs on
    both sides and both round the same numbers."""
    c = (n // 2, n // 2)
    psf = synth.gaussian_psf(n, n, c[0], c[1], 0.8, 0.6, 0.3)
    pr = OracleProblem("deblur256_fp32", n=n, psf=psf, rank=3)
    assert min(pr.kp.sc.min(), pr.kp.sr.min()) > 1e-3 * pr.kp.sc[0]
    lam = 0.02
    with setup_ctx(kpsvd, pr, "f32", fmt, "f32") as ctx:
        R = synth.random_matrix(n, n, 5)
        r = kpsvd.to_device(R, torch.float32)
        z = torch.empty_like(r)
        ctx.kp_apply_Minv(r, z, lam)
        Z = kpsvd.from_device(z, n, n)
        # the only differences are FP32 accumulation order flipping a rounding
        # at the same points: bounded by half a unit of the narrow format
        u = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8, "e4m3": 2.0 ** -4}[fmt]
        gk = GpuKpsvd(ctx)
        assert rel(Z, emulate_minv(gk, gk.Sigma, R, lam, fmt)) < 0.5 * u


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
@pytest.mark.parametrize("n", [64, 256])
def test_tensor_core_preconditioner_vs_fp64(kpsvd, fmt, n):
    """Single preconditioner apply against FP64: within 5e-3 for a broadband
    residual (for smooth residuals the 1 / lam^2 amplification of the input
    rounding dominates; the solver tests cover that regime)."""
    pr = OracleProblem("deblur256_fp32", n=n, rank=3)
    lam = 0.02
    with setup_ctx(kpsvd, pr, "f32", fmt, "f32") as ctx:
        R = synth.random_matrix(n, n, 5)
        r = kpsvd.to_device(R, torch.float32)
        z = torch.empty_like(r)
        ctx.kp_apply_Minv(r, z, lam)
        Z = kpsvd.from_device(z, n, n)
        Z64 = okp.precond_apply(pr.kp, okp.precond_scale(pr.kp.Sigma, lam), R)
        assert rel(Z, Z64) < 5e-3


@pytest.mark.parametrize("n", [64, 256])
def test_e4m3_preconditioner_vs_fp64(kpsvd, n):
    """FP8 (E4M3) single apply against FP64.  The four GEMMs round eight
    operands (R, T1, W, T3 and the two factors twice) to E4M3, unit roundoff
    u = 2^-4; eight independent roundings give a relative error of about
    sqrt(8) u / sqrt(3) ~ 0.1 (the FP64 emulation of the same rounding points
    gives 0.073 here), above the 3e-2 a single FP8 rounding would allow."""
    pr = OracleProblem("deblur256_fp32", n=n, rank=3)
    lam = 0.02
    with setup_ctx(kpsvd, pr, "f32", "e4m3", "f32") as ctx:
        R = synth.random_matrix(n, n, 5)
        r = kpsvd.to_device(R, torch.float32)
        z = torch.empty_like(r)
        ctx.kp_apply_Minv(r, z, lam)
        Z = kpsvd.from_device(z, n, n)
        Z64 = okp.precond_apply(pr.kp, okp.precond_scale(pr.kp.Sigma, lam), R)
        err = rel(Z, Z64)
        assert err < np.sqrt(8.0) * 2.0 ** -4 / np.sqrt(3.0)
        assert abs(err - rel(emulate_minv(pr.kp, pr.kp.Sigma, R, lam, "e4m3"), Z64)) < 0.01
