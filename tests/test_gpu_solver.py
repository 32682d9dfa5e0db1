"""GPU parity of tik_pcg (PCG / flexible PCG) and choose_lambda against the
FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from gpu_common import OracleProblem, lib, rel, setup_ctx, torch, vt
from oracle import forward, kpsvd as okp, kron, lam as olam, pcg as opcg
from paper_2311_15393_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kpsvd():
    return lib()


def run(kpsvd, ctx, pr, lam, tol, maxit, flexible, vec, x0=None, hist=0):
    b = kpsvd.to_device(pr.B, vt(vec))
    x = torch.zeros_like(b) if x0 is None else kpsvd.to_device(x0, vt(vec))
    info = ctx.tik_pcg(b, lam, tol, maxit, flexible, x, warm_start=x0 is not None, hist_len=hist, check=False)
    return kpsvd.from_device(x, pr.P.n_r, pr.P.n_c), info


@pytest.mark.parametrize("flexible", [False, True])
def test_fp64_iterates_match_oracle(kpsvd, flexible):
    """64 x 64 FP64 workload (full-rank zero-BC operator, lambda = 0.01): the
    iterates after k steps equal the oracle's."""
    pr = OracleProblem("deblur64_fp64")
    lam = pr.P.lam
    with setup_ctx(kpsvd, pr, "f64", "f64", "f64") as ctx:
        for k in [1, 5, 20, 50]:
            x, info = run(kpsvd, ctx, pr, lam, 0.0, k, flexible, "f64", hist=k + 1)
            xo, io = opcg.tik_pcg(pr.op, pr.kp, pr.B, lam, 0.0, k, flexible)
            assert info.iters == k
            assert rel(x, xo) < 1e-9, k
            np.testing.assert_allclose(info.res_hist, io.res_hist, rtol=1e-7)


@pytest.mark.parametrize("flexible", [False, True])
def test_fp64_iterates_with_separate_preconditioner_lambda(kpsvd, flexible):
    """64 x 64 FP64 workload with the preconditioner built for lambda_M = 3
    lambda (option pc_lambda_ratio; Section 5.3): the iterates after k steps
    equal the oracle's with lam_pc = 3 lambda."""
    pr = OracleProblem("deblur64_fp64")
    lam = pr.P.lam
    with setup_ctx(kpsvd, pr, "f64", "f64", "f64") as ctx:
        ctx.kp_set_option("pc_lambda_ratio", 3.0)
        for k in [1, 5, 20]:
            x, info = run(kpsvd, ctx, pr, lam, 0.0, k, flexible, "f64")
            xo, _ = opcg.tik_pcg(pr.op, pr.kp, pr.B, lam, 0.0, k, flexible, lam_pc=3 * lam)
            assert info.iters == k
            assert rel(x, xo) < 1e-9, k


def test_separate_preconditioner_lambda_reaches_oracle_solution(kpsvd):
    """256 x 256, BF16 operator, FP16 preconditioner built for lambda_M = 2
    lambda: FPCG still reaches the oracle's x_lambda to 1e-4."""
    pr = OracleProblem("deblur256_fp32")
    lam = olam.choose_lambda(pr.kp, pr.B, "gcv")
    x_star = opcg.tik_exact(pr.op, pr.kp, pr.B, lam)
    with setup_ctx(kpsvd, pr, "bf16", "f16", "f32") as ctx:
        ctx.kp_set_option("pc_lambda_ratio", 2.0)
        x, info = run(kpsvd, ctx, pr, lam, 1e-7, 500, True, "f32")
        print(f"lambda_M = 2 lambda: {info.iters} iterations")
        assert info.status == kpsvd.KP_OK
        assert rel(x, x_star) < 1e-4


def test_fp64_workload_stops_by_rule(kpsvd):
    """50 iterations or relative residual 1e-8, whichever comes first."""
    pr = OracleProblem("deblur64_fp64")
    with setup_ctx(kpsvd, pr, "f64", "f64", "f64") as ctx:
        x, info = run(kpsvd, ctx, pr, pr.P.lam, 1e-8, 50, False, "f64")
        xo, io = opcg.tik_pcg(pr.op, pr.kp, pr.B, pr.P.lam, 1e-8, 50, False)
        assert info.iters == io.iters
        assert (info.status == kpsvd.KP_OK) == io.converged
        assert rel(x, xo) < 1e-9


def test_separable_zero_bc_converges_in_one_iteration(kpsvd):
    n = 32
    psf = synth.separable_psf(n, n, 16, 16, 2.5, 1.5)
    pr = OracleProblem("deblur64_fp64", n=n, psf=psf, center=(16, 16), bc="zero", rank=1)
    lam = 0.02
    x_star = opcg.tik_exact_dense(pr.op, pr.B, lam)
    with setup_ctx(kpsvd, pr, "f64", "f64", "f64") as ctx:
        x, info = run(kpsvd, ctx, pr, lam, 1e-10, 10, False, "f64")
        assert info.iters == 1
        assert rel(x, x_star) < 1e-10


U32 = 2.0 ** -24


@pytest.mark.parametrize("lam", [0.3, 0.15, 0.03])
def test_fp32_path_fixed_iterations(kpsvd, lam):
    """256 x 256 workload, all-FP32 path (FP32 operator, preconditioner and
    vectors; reliable updates off): x after 10 iterations vs the FP64
    oracle's.  Two FP32 effects bound the difference: GEMM accumulation over
    K = r n terms (~ sqrt(K) u) and the rounding of r, whose white part M^-1
    amplifies by up to 1 / lam^2; bound 8 u (sqrt(r n) + 1 / lam^2)
    (1.9e-5 at lam = 0.3, 3.4e-5 at 0.15, 5.5e-4 at 0.03).  Where the
    1 / lam^2 amplification is moderate (lam >= 0.15) the difference also
    meets the stated 1e-5 of the all-FP32 path at a fixed iteration count
    (numpy's FP32 BLAS gives 1.5e-6 / 5.7e-6 / 1.3e-4 at the three lambdas)."""
    pr = OracleProblem("deblur256_fp32")
    with setup_ctx(kpsvd, pr, "f32", "f32", "f32") as ctx:
        ctx.kp_set_option("reliable_delta", 0.0)
        x, info = run(kpsvd, ctx, pr, lam, 0.0, 10, True, "f32")
        xo, _ = opcg.tik_pcg(pr.op, pr.kp, pr.B, lam, 0.0, 10, True)
        err = rel(x, xo)
        bound = 8 * U32 * (np.sqrt(pr.op.rank * pr.P.n_c) + 1.0 / lam ** 2)
        print(f"lambda {lam}: all-FP32 x_10 vs FP64 oracle {err:.3e} (bound {bound:.2e})")
        assert err < bound
        if lam >= 0.15:
            assert err < 1e-5


@pytest.mark.parametrize("flexible", [False, True])
def test_fp32_path_converges_to_oracle_solution(kpsvd, flexible):
    """FP32 operator and preconditioner with reliable residual updates reach
    x_lambda (GCV lambda) to 1e-4 within +3 iterations of the FP64 oracle."""
    pr = OracleProblem("deblur256_fp32")
    lam = olam.choose_lambda(pr.kp, pr.B, "gcv")
    x_star = opcg.tik_exact(pr.op, pr.kp, pr.B, lam)
    _, io = opcg.tik_pcg(pr.op, pr.kp, pr.B, lam, 1e-7, 500, flexible)
    with setup_ctx(kpsvd, pr, "f32", "f32", "f32") as ctx:
        x, info = run(kpsvd, ctx, pr, lam, 1e-7, 500, flexible, "f32")
        assert info.status == kpsvd.KP_OK
        assert rel(x, x_star) < 1e-4
        assert info.iters <= io.iters + 3


@pytest.mark.parametrize("op", ["bf16", "bf16x3"])
@pytest.mark.parametrize("pc", ["f16", "bf16"])
@pytest.mark.parametrize("fold", [0, 1])
def test_reduced_precision_fpcg_reaches_oracle_solution(kpsvd, op, pc, fold):
    """256 x 256: BF16 tensor-core operator with reliable residual updates and a
    half-precision preconditioner reaches the oracle's x_lambda to 1e-4 with
    an iteration count within +3 of the oracle's FP64 FPCG (Section 5.2:
    same final error, about the same iterations), with the quantisation of r
    as a separate pass and folded into the x / r update."""
    pr = OracleProblem("deblur256_fp32")
    lam = olam.choose_lambda(pr.kp, pr.B, "gcv")
    tol = 1e-7
    x_star = opcg.tik_exact(pr.op, pr.kp, pr.B, lam)
    _, io = opcg.tik_pcg(pr.op, pr.kp, pr.B, lam, tol, 500, True)
    with setup_ctx(kpsvd, pr, op, pc, "f32") as ctx:
        ctx.kp_set_option("cg_fuse", fold)
        x, info = run(kpsvd, ctx, pr, lam, tol, 500, True, "f32")
        print(f"{op}/{pc} fold {fold}: {info.iters} iterations, {info.replacements} replacements "
              f"(oracle FP64 {io.iters}), rel. error {rel(x, x_star):.2e}")
        assert info.status == kpsvd.KP_OK
        assert rel(x, x_star) < 1e-4
        assert info.iters <= io.iters + 3


def test_folded_quantisation_matches_separate_pass(kpsvd):
    """256 x 256, BF16 operator and FP16 preconditioner: with the narrow copy of
    r written by the x / r update (scale from the bound max|r| + |alpha|
    max|q|) the solve takes the iterations of the separate quantisation pass
    (scale from the exact max|r|) to within 2 and reaches the same x_lambda.
    (A fixed-iteration comparison with the oracle is not meaningful here: the
    BF16 inner operator alone moves x_k by up to cond(K) times its rounding.)"""
    pr = OracleProblem("deblur256_fp32")
    lam = olam.choose_lambda(pr.kp, pr.B, "gcv")
    x_star = opcg.tik_exact(pr.op, pr.kp, pr.B, lam)
    res = {}
    with setup_ctx(kpsvd, pr, "bf16", "f16", "f32") as ctx:
        for fold in (0, 1):
            ctx.kp_set_option("cg_fuse", fold)
            x, info = run(kpsvd, ctx, pr, lam, 1e-7, 500, True, "f32")
            assert info.status == kpsvd.KP_OK
            res[fold] = (x, info.iters)
    print(f"iterations: separate {res[0][1]}, folded {res[1][1]}; between the solutions {rel(res[1][0], res[0][0]):.2e}")
    assert abs(res[1][1] - res[0][1]) <= 2
    assert rel(res[1][0], x_star) < 1e-4
    assert rel(res[1][0], res[0][0]) < 5e-5


def test_solve_ignores_stale_device_memory(kpsvd):
    """Device memory a new context receives may hold old data (here NaN bit
    patterns of a freed buffer): no kernel of setup or solve reads a buffer
    before writing it (the first p = z does not read the old p)."""
    junk = torch.full((256 * 1024 * 1024,), float("nan"), dtype=torch.float32, device="cuda:0")
    del junk
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    pr = OracleProblem("deblur256_fp32", n=128, rank=3)
    lam = olam.choose_lambda(pr.kp, pr.B, "gcv")
    x_star = opcg.tik_exact(pr.op, pr.kp, pr.B, lam)
    for op, pc in (("bf16", "f16"), ("f32", "f32")):
        with setup_ctx(kpsvd, pr, op, pc, "f32") as ctx:
            x, info = run(kpsvd, ctx, pr, lam, 1e-7, 500, True, "f32")
            assert info.status == kpsvd.KP_OK
            assert rel(x, x_star) < 1e-4


def test_ill_conditioned_problem_raises_inner_operator(kpsvd):
    """256 x 256, zero BC, wide PSF (sigma = 3.4 x 8), 0.14% noise: at the GCV
    lambda cond(A^T A + lambda^2 I) ~ 1e5, where the BF16 inner operator's
    rounding stalls FPCG.  With op_auto_cond = 1e4 the solve switches its
    inner operator to BF16X3, converges to 1e-7, and x is within the
    forward-error bound cond(K) tol of the oracle's x_lambda."""
    P = synth.make_problem("deblur256_fp32", n=256)
    psf = synth.gaussian_psf(256, 256, 128, 128, 3.4, 8.0, 0.17)
    pr = OracleProblem("deblur256_fp32", n=256, psf=psf, bc="zero", rank=4)
    pr.B, _ = forward.observe(pr.op, pr.P.x_true, pr.P.noise_dirs[0], 0.0014)
    lam = olam.choose_lambda(pr.kp, pr.B, "gcv")
    cond = (np.max(np.abs(pr.kp.Sigma)) ** 2 + lam ** 2) / lam ** 2
    assert cond > 1e4
    x_star = opcg.tik_exact(pr.op, pr.kp, pr.B, lam, tol=1e-10)
    with setup_ctx(kpsvd, pr, "bf16", "f16", "f32") as ctx:
        ctx.kp_set_option("op_auto_cond", 1e4)
        x, info = run(kpsvd, ctx, pr, lam, 1e-7, 500, True, "f32")
        print(f"cond(K) {cond:.2e}: {info.iters} iterations, {info.replacements} replacements, "
              f"rel. error {rel(x, x_star):.2e}")
        assert info.status == kpsvd.KP_OK
        assert rel(x, x_star) < cond * 1e-7


def test_stagnation_below_attainable_accuracy(kpsvd):
    """FP32 vectors cannot reach a 1e-12 normal-equations residual: the solve
    stops with KP_ENOCONV once three residual replacements in a row fail to
    halve the true residual, long before maxit, with x at the oracle's
    x_lambda to the usual accuracy."""
    pr = OracleProblem("deblur256_fp32", n=128, rank=3)
    lam = olam.choose_lambda(pr.kp, pr.B, "gcv")
    x_star = opcg.tik_exact(pr.op, pr.kp, pr.B, lam)
    with setup_ctx(kpsvd, pr, "bf16", "f16", "f32") as ctx:
        x, info = run(kpsvd, ctx, pr, lam, 1e-12, 2000, True, "f32")
        print(f"stagnation: {info.iters} iterations, {info.replacements} replacements, rel_res {info.rel_res:.2e}")
        assert info.status == kpsvd.KP_ENOCONV
        assert info.iters < 400
        assert 1e-12 < info.rel_res < 1e-6
        assert rel(x, x_star) < 1e-4


def test_e4m3_fpcg_reaches_oracle_solution(kpsvd):
    """256 x 256: FPCG with the FP8 (E4M3) preconditioner, whose every apply
    is ~7% off the FP64 one, still reaches the oracle's x_lambda to 1e-4
    (flexible PCG treats the inexact preconditioner as variable); it needs
    more iterations than FP16."""
    pr = OracleProblem("deblur256_fp32")
    lam = olam.choose_lambda(pr.kp, pr.B, "gcv")
    tol = 1e-7
    x_star = opcg.tik_exact(pr.op, pr.kp, pr.B, lam)
    _, io = opcg.tik_pcg(pr.op, pr.kp, pr.B, lam, tol, 500, True)
    with setup_ctx(kpsvd, pr, "bf16", "e4m3", "f32") as ctx:
        x, info = run(kpsvd, ctx, pr, lam, tol, 500, True, "f32")
        print(f"e4m3 FPCG iterations {info.iters} (oracle FP64 {io.iters})")
        assert info.status == kpsvd.KP_OK
        assert rel(x, x_star) < 1e-4
        assert info.iters <= 3 * io.iters


def test_edge_cases(kpsvd):
    pr = OracleProblem("deblur256_fp32", n=64, rank=2)
    with setup_ctx(kpsvd, pr, "f64", "f64", "f64") as ctx:
        b = torch.zeros(64 * 64, dtype=torch.float64, device="cuda")
        x = torch.ones_like(b)
        info = ctx.tik_pcg(b, 0.1, 1e-8, 10, False, x)
        assert info.iters == 0 and float(x.abs().max()) == 0.0
        x, info = run(kpsvd, ctx, pr, 0.01, 1e-14, 3, False, "f64")
        assert info.status == kpsvd.KP_ENOCONV and info.iters == 3
        # warm start from the converged solution stops at once
        x_star = opcg.tik_exact_dense(pr.op, pr.B, 0.05)
        x, info = run(kpsvd, ctx, pr, 0.05, 1e-9, 10, False, "f64", x0=x_star)
        assert info.iters <= 1 and rel(x, x_star) < 1e-9
        with pytest.raises(kpsvd.KpError):
            ctx.tik_pcg(b, -1.0, 1e-6, 10, False, torch.zeros_like(b))
        with pytest.raises(kpsvd.KpError):
            ctx.kp_setup(kpsvd.to_device(pr.P.psf), 64, 64, (64, 0), "zero", 1)
    ctx = kpsvd.KpContext(0)
    with pytest.raises(kpsvd.KpError) as e:
        ctx.tik_pcg(b, 0.1, 1e-6, 10, False, torch.zeros_like(b))
    assert e.value.status == kpsvd.KP_ESTATE
    ctx.close()


@pytest.mark.parametrize("vec", ["f64", "f32"])
@pytest.mark.parametrize("method", ["gcv", "wgcv", "discrepancy", "opt"])
def test_choose_lambda_matches_oracle(kpsvd, method, vec):
    pr = OracleProblem("deblur256_fp32", n=128, rank=3)
    param = {"gcv": 0.0, "wgcv": 3.0, "discrepancy": 1.01 * pr.enorm, "opt": 0.0}[method]
    lo = olam.choose_lambda(pr.kp, pr.B, method, param, X_true=pr.P.x_true)
    with setup_ctx(kpsvd, pr, vec, vec, vec) as ctx:
        b = kpsvd.to_device(pr.B, vt(vec))
        xt = kpsvd.to_device(pr.P.x_true, vt(vec)) if method == "opt" else None
        lg = ctx.choose_lambda(b, method, param, xt)
    tol = 1e-9 if (method == "discrepancy" and vec == "f64") else (1e-6 if vec == "f64" else 1e-4)
    assert abs(np.log(lg) - np.log(lo)) < tol, (lg, lo)


def test_discrepancy_without_root(kpsvd):
    pr = OracleProblem("deblur256_fp32", n=64, rank=2)
    with setup_ctx(kpsvd, pr, "f64", "f64", "f64") as ctx:
        b = kpsvd.to_device(pr.B)
        with pytest.raises(kpsvd.KpError) as e:
            ctx.choose_lambda(b, "discrepancy", 2.0 * np.linalg.norm(pr.B))
        assert e.value.status == kpsvd.KP_ENOROOT


@pytest.mark.parametrize("op,pc,flexible", [("f32", "f32", False), ("f32", "f32", True), ("bf16", "f16", True)])
def test_discrepancy_lambda_solve_reaches_oracle_solution(kpsvd, op, pc, flexible):
    """256 x 256 with lambda by the discrepancy principle (eps = 1.01 times the
    generator's noise norm, the workload's second parameter choice): the
    GPU's lambda equals the oracle's root, and PCG / FPCG reach the oracle's
    x_lambda to 1e-4 within +3 iterations of the oracle's FP64 run."""
    pr = OracleProblem("deblur256_fp32")
    eps = 1.01 * pr.enorm
    lam = olam.choose_lambda(pr.kp, pr.B, "discrepancy", eps)
    x_star = opcg.tik_exact(pr.op, pr.kp, pr.B, lam)
    _, io = opcg.tik_pcg(pr.op, pr.kp, pr.B, lam, 1e-7, 500, flexible)
    with setup_ctx(kpsvd, pr, op, pc, "f32") as ctx:
        lg = ctx.choose_lambda(kpsvd.to_device(pr.B, torch.float32), "discrepancy", eps)
        x, info = run(kpsvd, ctx, pr, lam, 1e-7, 500, flexible, "f32")
    assert abs(np.log(lg / lam)) < 1e-4
    assert info.status == kpsvd.KP_OK
    assert rel(x, x_star) < 1e-4
    assert info.iters <= io.iters + 3


@pytest.mark.parametrize("pc", ["f16", "bf16"])
def test_fp32_operator_with_half_precision_preconditioner(kpsvd, pc):
    """The 256 x 256 configuration as stated: rank-3 operator in FP32 (SIMT),
    KP-SVD preconditioner in FP16 or BF16 on the tensor cores with FP32
    accumulation; FPCG with the GCV lambda reaches the oracle's x_lambda to
    1e-4 within +3 iterations of the oracle's FP64 FPCG."""
    pr = OracleProblem("deblur256_fp32")
    lam = olam.choose_lambda(pr.kp, pr.B, "gcv")
    x_star = opcg.tik_exact(pr.op, pr.kp, pr.B, lam)
    _, io = opcg.tik_pcg(pr.op, pr.kp, pr.B, lam, 1e-7, 500, True)
    with setup_ctx(kpsvd, pr, "f32", pc, "f32") as ctx:
        x, info = run(kpsvd, ctx, pr, lam, 1e-7, 500, True, "f32")
    assert info.status == kpsvd.KP_OK
    assert rel(x, x_star) < 1e-4
    assert info.iters <= io.iters + 3


@pytest.mark.parametrize("vec", ["f64", "f32"])
def test_non_finite_data_is_reported(kpsvd, vec):
    """A NaN in b is a status, not a result: tik_pcg returns KP_ENUMERIC
    (A^T b is not finite) and choose_lambda returns KP_ENUMERIC for GCV and
    the discrepancy principle instead of a lambda; the context then solves
    finite data as before."""
    pr = OracleProblem("deblur256_fp32", n=64, rank=2)
    op = "f64" if vec == "f64" else "bf16"
    pc = "f64" if vec == "f64" else "f16"
    with setup_ctx(kpsvd, pr, op, pc, vec) as ctx:
        Bn = pr.B.copy()
        Bn[3, 5] = np.nan
        b = kpsvd.to_device(Bn, vt(vec))
        x = torch.zeros_like(b)
        info = ctx.tik_pcg(b, 0.05, 1e-6, 50, True, x, check=False)
        assert info.status == kpsvd.KP_ENUMERIC
        for method, param in (("gcv", 0.0), ("discrepancy", 1.01 * pr.enorm)):
            with pytest.raises(kpsvd.KpError) as e:
                ctx.choose_lambda(b, method, param)
            assert e.value.status == kpsvd.KP_ENUMERIC
        x, info = run(kpsvd, ctx, pr, 0.05, 1e-7, 300, True, vec)
        assert info.status == kpsvd.KP_OK
        assert rel(x, opcg.tik_exact(pr.op, pr.kp, pr.B, 0.05)) < 1e-4


def test_non_finite_or_zero_psf_is_rejected(kpsvd):
    """kp_setup checks the PSF before factoring it: a NaN gives KP_ENUMERIC,
    an all-zero PSF KP_EINVAL, and a solve on the context then reports that
    no problem is set up (KP_ESTATE); the same context then takes a valid
    PSF, whose KP spectrum matches the oracle to FP32 level."""
    pr = OracleProblem("deblur256_fp32", n=64, rank=2)
    P = pr.P
    args = (P.n_r, P.n_c, P.center, P.bc, P.op_rank, "f32", "f32", "f32")
    with kpsvd.KpContext(0) as ctx:
        bad = P.psf.copy()
        bad[10, 20] = np.nan
        with pytest.raises(kpsvd.KpError) as e:
            ctx.kp_setup(kpsvd.to_device(bad), *args)
        assert e.value.status == kpsvd.KP_ENUMERIC
        with pytest.raises(kpsvd.KpError) as e:
            ctx.kp_setup(kpsvd.to_device(np.zeros_like(P.psf)), *args)
        assert e.value.status == kpsvd.KP_EINVAL
        b = kpsvd.to_device(pr.B, torch.float32)
        info = ctx.tik_pcg(b, 0.05, 1e-6, 10, True, torch.zeros_like(b), check=False)
        assert info.status == kpsvd.KP_ESTATE
        ctx.kp_setup(kpsvd.to_device(P.psf), *args)
        smax = np.abs(pr.kp.Sigma).max()
        np.testing.assert_allclose(ctx.kp_get_spectrum(), pr.kp.Sigma, rtol=0, atol=8 * 64 * 2.0 ** -23 * smax)
