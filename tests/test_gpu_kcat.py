"""GPU parity of the K-concatenated tensor-core GEMM (tc_gemm_kcat_kernel) that
computes the inner operator's second and fourth GEMMs as ONE product over all
Kronecker terms (eq. KronSumDecomp: sum_k A_c^(k) X A_r^(k)^T with the terms
summed in the tensor-memory accumulator, 128 x 64 tiles), the fourth also
reducing p^T q and max |q| in its epilogue for the alpha step.

Option tc_kcat 1 uses it where its tiles fill most SMs (1024^2), 2 wherever
the shape allows, 0 (default: measured faster at 1024^2) never (per-term
products and a separate term sum); tc_kcat_cluster 4 groups the CTAs in
clusters of four along N that share their A tiles by TMA multicast (n_r a
multiple of 256).  The operator
is checked against the emulation on the GPU's own terms (spike and dense
images, A and A^T), the K application against the per-term form, and the
solve, whose alpha step takes p^T q from the GEMM epilogue, against the
oracle's x_lambda and iteration count."""
import pytest

from gpu_common import OracleProblem, check_bf16_operator, lib, rel, torch
from oracle import lam as olam, pcg as opcg
from paper_2311_15393_gb300 import synth

pytestmark = pytest.mark.gpu

# (n_r, n_c, CTAs per cluster): n_r is the GEMMs' N, n_c their M; ragged
# tails 208 = 128 + 80 and 144 = 128 + 16 (with clusters of four N stays a
# multiple of 256: whole clusters of 64-wide tiles)
CASES = [(256, 256, 1), (208, 144, 1), (256, 256, 4), (512, 208, 4), (256, 144, 4)]


@pytest.fixture(scope="module")
def kpsvd():
    return lib()


def _ctx(kpsvd, P, kcat, cluster=1):
    ctx = kpsvd.KpContext(0)
    ctx.kp_set_option("tc_kcat", kcat)
    ctx.kp_set_option("tc_kcat_cluster", cluster)
    ctx.kp_setup(kpsvd.to_device(P.psf), P.n_r, P.n_c, P.center, P.bc, P.op_rank, "bf16", "f16", "f32", "projected")
    torch.cuda.synchronize()
    return ctx


def _kapply_launches(ctx):
    """Kernels launched per K application (kp_time_parts)."""
    _, launches = ctx.kp_time_parts(0.02, 2)
    return launches[0]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}-cl{c[2]}")
def test_kcat_operator(kpsvd, case):
    """tc_kcat 2: A, A^T against the emulation on the GPU's own terms (the
    bound of check_bf16_operator), K p against the per-term form (tc_kcat 0);
    four launches per K application (no term sums)."""
    n_r, n_c, cl = case
    pr = OracleProblem("deblur256_fp32", n=max(n_r, n_c), shape=(n_r, n_c), rank=3)
    with _ctx(kpsvd, pr.P, 2, cl) as ck, _ctx(kpsvd, pr.P, 0) as c0:
        check_bf16_operator(kpsvd, ck, pr, n_r, n_c)
        X = synth.random_matrix(n_r, n_c, 7)
        x = kpsvd.to_device(X, torch.float32)
        qk, q0 = torch.empty_like(x), torch.empty_like(x)
        ck.kp_apply_K(x, qk, 0.02)
        c0.kp_apply_K(x, q0, 0.02)
        d = rel(kpsvd.from_device(qk, n_r, n_c), kpsvd.from_device(q0, n_r, n_c))
        lk, l0 = _kapply_launches(ck), _kapply_launches(c0)
        print(f"{case}: K p, K-concatenated vs per-term {d:.2e}; launches per K application {lk} vs {l0}")
        assert d < 2e-3
        assert lk == 4


@pytest.mark.parametrize("case", [(256, 256, 1), (208, 144, 1), (512, 208, 4)], ids=lambda c: f"{c[0]}x{c[1]}-cl{c[2]}")
def test_kcat_solve(kpsvd, case):
    """tc_kcat 2: GCV lambda and the BF16 / FP16 / FP32 FPCG solve (alpha from
    the fused p^T q) reach the oracle's x_lambda to 1e-4 within +3 iterations
    of the oracle's FP64 FPCG, and match the per-term form's solve."""
    n_r, n_c, cl = case
    pr = OracleProblem("deblur256_fp32", n=max(n_r, n_c), shape=(n_r, n_c), rank=3)
    lam = olam.choose_lambda(pr.kp, pr.B, "gcv")
    x_star = opcg.tik_exact(pr.op, pr.kp, pr.B, lam, tol=1e-10)
    _, io = opcg.tik_pcg(pr.op, pr.kp, pr.B, lam, 1e-7, 500, True)
    res = {}
    for kc in (2, 0):
        with _ctx(kpsvd, pr.P, kc, cl) as ctx:
            b = kpsvd.to_device(pr.B, torch.float32)
            x = torch.zeros_like(b)
            info = ctx.tik_pcg(b, lam, 1e-7, 500, True, x)
            res[kc] = (info, kpsvd.from_device(x, n_r, n_c))
    (ik, xk), (i0, x0) = res[2], res[0]
    err = rel(xk, x_star)
    print(f"{case}: K-concatenated {ik.iters} iterations, per-term {i0.iters}, oracle {io.iters}; "
          f"rel. error {err:.2e}, vs per-term {rel(xk, x0):.2e}")
    assert ik.status == kpsvd.KP_OK
    assert err < 1e-4
    assert ik.iters <= io.iters + 3
    assert abs(ik.iters - i0.iters) <= 3
    assert rel(xk, x0) < 1e-4


@pytest.mark.parametrize("cl", [1, 4])
def test_kcat_size_rule_at_1024(kpsvd, cl):
    """1024^2 (the benchmark size), tc_kcat 1: the K-concatenated form is the
    one used (four launches per K application), K p agrees with the per-term
    form, and both noise levels' solves match the per-term form's iterations
    and iterates."""
    P = synth.make_problem("deblur1024_mixed")
    f32 = torch.float32
    with _ctx(kpsvd, P, 1, cl) as ck, _ctx(kpsvd, P, 0) as c0:
        assert _kapply_launches(ck) == 4
        assert _kapply_launches(c0) == 6
        X = synth.random_matrix(P.n_r, P.n_c, 9)
        x = kpsvd.to_device(X, f32)
        qk, q0 = torch.empty_like(x), torch.empty_like(x)
        ck.kp_apply_K(x, qk, 0.02)
        c0.kp_apply_K(x, q0, 0.02)
        d = rel(kpsvd.from_device(qk, P.n_r, P.n_c), kpsvd.from_device(q0, P.n_r, P.n_c))
        print(f"1024^2 clusters of {cl}: K p, K-concatenated vs per-term {d:.2e}")
        assert d < 2e-3
        xt = kpsvd.to_device(P.x_true, f32)
        for g, nl in zip(P.noise_dirs, P.noise_levels):
            b = torch.empty_like(xt)
            c0.kp_forward(xt, kpsvd.to_device(g, f32), nl, b)
            lam = c0.choose_lambda(b, "gcv")
            xs, its = [], []
            for ctx in (ck, c0):
                xx = torch.zeros_like(b)
                info = ctx.tik_pcg(b, lam, 1e-7, 500, True, xx)
                assert info.status == kpsvd.KP_OK
                xs.append(kpsvd.from_device(xx, P.n_r, P.n_c))
                its.append(info.iters)
            dx = rel(xs[0], xs[1])
            print(f"noise {nl}: iterations K-concatenated {its[0]}, per-term {its[1]}; iterates differ by {dx:.2e}")
            assert abs(its[0] - its[1]) <= 3
            assert dx < 2e-4
