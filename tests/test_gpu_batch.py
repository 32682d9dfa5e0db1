"""GPU parity of kp_solve_batch (independent problems of uneven sizes, each
with its own PSF, boundary condition, noise level and GCV lambda; BF16
operator, FP16 preconditioner, FP32 vectors) against the FP64 oracle, and
against the same problems solved one at a time, in the grouped form (one
launch per iteration step over all problems, workers = 0) and with host
threads (workers > 0)."""
import numpy as np
import pytest

from gpu_common import lib, rel, torch
from oracle import forward, kpsvd as okp, kron, lam as olam, pcg as opcg
from paper_2311_15393_gb300 import synth

pytestmark = pytest.mark.gpu

SIZES = [(128, 128), (128, 256), (256, 128), (256, 256)]
TOL = 1e-7


@pytest.fixture(scope="module")
def kpsvd():
    return lib()


@pytest.fixture(scope="module")
def problems():
    """Six problems drawn by the batched workload's generator at small sizes,
    at the generator's own noise levels (0.1% to 5%), with the oracle's
    observed data b (its own FP64 operator)."""
    out = []
    for P in synth.make_batch(6, sizes=SIZES, seed=77):
        op = kron.kron_operator(P.psf, P.center, P.bc, P.op_rank)
        kp = okp.kp_svd(op, "projected")
        B, _ = forward.observe(op, P.x_true, P.noise_dirs[0], P.noise_levels[0])
        out.append(dict(P=P, op=op, kp=kp, B=B))
    return out


def device_problems(kpsvd, problems):
    dev = []
    for pr in problems:
        P = pr["P"]
        b = kpsvd.to_device(pr["B"], torch.float32)
        dev.append(dict(psf=kpsvd.to_device(P.psf), b=b, x=torch.zeros_like(b), n_r=P.n_r, n_c=P.n_c,
                        center=P.center, bc=P.bc, op_rank=P.op_rank))
    return dev


@pytest.mark.parametrize("workers", [0, 3])
def test_batch_matches_oracle(kpsvd, problems, workers):
    """Every problem: the GCV lambda minimises the oracle's GCV function (its
    value there within 1e-5 of the oracle's minimum: the minimum can be so
    flat that the FP32 spectrum moves the argmin by ~1% while the value stays
    put), and x is within 1e-4 of the oracle's x_lambda at that lambda (the
    metric's bar) where cond(K) = (sigma_max^2 + lambda^2) / lambda^2 <= 1e4,
    else within the forward-error bound cond(K) tol of the residual stopping
    rule.  A problem may stop as stagnated (KP_ENOCONV: the true residual no
    longer halves at FP32 accuracy) only where cond(K) > 1e4; such a problem
    is not a solve at the metric's bar and is reported, not counted."""
    dev = device_problems(kpsvd, problems)
    st, ms, res = kpsvd.kp_solve_batch(dev, tol=TOL, workers=workers, check=False)
    assert st in (kpsvd.KP_OK, kpsvd.KP_ENOCONV), kpsvd._lib.kp_last_error().decode()
    if workers == 0:  # every problem that iterated did so in the grouped loop
        n_grouped, passes, _, shape = kpsvd.kp_batch_grouped(0)
        print(f"launches per iteration / grouped launches per pass: {shape}")
        print(f"grouped loop: {n_grouped} problems, {passes} passes")
        assert n_grouped == sum(info.iters > 0 for _, info in res), kpsvd._lib.kp_last_error().decode()
        assert passes >= 1
    for pr, d, (lam, info) in zip(problems, dev, res):
        P = pr["P"]
        lam_o = olam.choose_lambda(pr["kp"], pr["B"], "gcv")
        x_star = opcg.tik_exact(pr["op"], pr["kp"], pr["B"], lam, tol=1e-10)
        X = kpsvd.from_device(d["x"], P.n_r, P.n_c)
        print(f"{P.n_r}x{P.n_c} {P.bc} nl {P.noise_levels[0]:.4f}: lambda {lam:.6g} (oracle {lam_o:.6g}), "
              f"{info.iters} iterations, rel. error {rel(X, x_star):.2e}, cond(K) "
              f"{(np.max(np.abs(pr['kp'].Sigma)) ** 2 + lam ** 2) / lam ** 2:.1e}")
        cond = (np.max(np.abs(pr["kp"].Sigma)) ** 2 + lam ** 2) / lam ** 2
        assert info.status == kpsvd.KP_OK or (info.status == kpsvd.KP_ENOCONV and cond > 1e4)
        bh = olam.spectral_coeffs(pr["kp"], pr["B"])
        g_gpu, g_o = olam.gcv(pr["kp"].Sigma, bh, lam), olam.gcv(pr["kp"].Sigma, bh, lam_o)
        assert g_gpu <= g_o * (1.0 + 1e-5)
        assert abs(np.log(lam / lam_o)) < 0.1
        assert rel(X, x_star) < (1e-4 if cond <= 1e4 else cond * TOL)


@pytest.mark.parametrize("workers", [0, 4])
def test_batch_equals_single_solves(kpsvd, problems, workers):
    """The batch computes for each problem what kp_setup + choose_lambda +
    tik_pcg compute for it alone on one context.  With host threads the
    results are identical.  Grouped, the setup and lambda are identical and
    the iterations run the same kernel bodies, but with one-CTA tiles and no
    K split in the GEMMs and another block count in the reductions, so their
    sums are rounded in another order: the same status, at most 3 more or
    fewer iterations, and x within the forward-error bound of the stopping
    rule (10 cond(K) tol) of the single solve's."""
    dev = device_problems(kpsvd, problems)
    st, _, res = kpsvd.kp_solve_batch(dev, tol=TOL, workers=workers, check=False)
    for pr, d, (lam, info) in zip(problems, dev, res):
        P = pr["P"]
        with kpsvd.KpContext(0) as ctx:
            ctx.kp_set_option("op_auto_cond", 1e4)  # what the batch sets for a BF16 operator
            ctx.kp_setup(d["psf"], P.n_r, P.n_c, P.center, P.bc, P.op_rank, "bf16", "f16", "f32", "projected")
            lam1 = ctx.choose_lambda(d["b"], "gcv")
            x1 = torch.zeros_like(d["b"])
            info1 = ctx.tik_pcg(d["b"], lam1, TOL, 500, True, x1, check=False)
            if info1.status in (kpsvd.KP_ENOCONV, kpsvd.KP_EBREAKDOWN, kpsvd.KP_ENUMERIC):
                # the batch's rule: a stalled BF16 inner operator is solved again with BF16X3
                ctx.kp_set_option("op_auto_cond", 1.0)
                x1.zero_()
                info1 = ctx.tik_pcg(d["b"], lam1, TOL, 500, True, x1, check=False)
        assert lam1 == lam
        assert info1.status == info.status
        d_x = rel(kpsvd.from_device(d["x"], P.n_r, P.n_c), kpsvd.from_device(x1, P.n_r, P.n_c))
        if workers > 0:
            assert info1.iters == info.iters
            assert d_x < 1e-12
        else:
            cond = (np.max(np.abs(pr["kp"].Sigma)) ** 2 + lam ** 2) / lam ** 2
            print(f"{P.n_r}x{P.n_c}: iterations grouped {info.iters} alone {info1.iters}, x differs by {d_x:.2e}")
            assert abs(info1.iters - info.iters) <= 3
            assert d_x < 10 * cond * TOL


@pytest.mark.parametrize("workers", [0, 2])
def test_batch_fixed_lambda_and_failing_problem(kpsvd, problems, workers):
    """A problem with lambda > 0 keeps it; a problem the tensor-core setup
    rejects (size not a multiple of 16) fails alone: its status is returned,
    the others are solved."""
    dev = device_problems(kpsvd, problems[:2])
    dev[0]["lam"] = 0.05
    P = problems[0]["P"]
    bad_b = torch.zeros(100 * 100, dtype=torch.float32, device="cuda:0")
    bad = dict(psf=kpsvd.to_device(synth.gaussian_psf(100, 100, 50, 50, 2.0, 2.0, 0.0)), b=bad_b,
               x=torch.zeros_like(bad_b), n_r=100, n_c=100, center=(50, 50), bc="zero", op_rank=2)
    st, _, res = kpsvd.kp_solve_batch(dev + [bad], tol=TOL, workers=workers, check=False)
    assert st != kpsvd.KP_OK
    assert res[2][1].status == st
    assert res[0][0] == 0.05 and res[0][1].status == kpsvd.KP_OK
    assert res[1][1].status == kpsvd.KP_OK
    x_star = opcg.tik_exact(problems[0]["op"], problems[0]["kp"], problems[0]["B"], 0.05, tol=1e-10)
    assert rel(kpsvd.from_device(dev[0]["x"], P.n_r, P.n_c), x_star) < 1e-4


def test_grouped_batch_edge_cases(kpsvd, problems):
    """Grouped form: a problem whose b is zero stops before the loop (x = 0,
    no iterations) while the others iterate in the grouped loop; a batch whose
    operator has no fused iteration (FP32 SIMT operator) cannot be grouped, so
    every problem runs alone, and each is still solved to the oracle's x_lambda."""
    dev = device_problems(kpsvd, problems[:3])
    dev[1]["b"].zero_()
    dev[1]["x"].fill_(1.0)
    dev[1]["lam"] = 0.05  # (no lambda criterion has a minimum for b = 0)
    st, _, res = kpsvd.kp_solve_batch(dev, tol=TOL, workers=0, check=False)
    assert res[1][1].status == kpsvd.KP_OK and res[1][1].iters == 0
    assert torch.count_nonzero(dev[1]["x"]).item() == 0
    n_grouped, passes, _, _ = kpsvd.kp_batch_grouped(0)
    assert n_grouped == sum(info.iters > 0 for _, info in res) == 2
    for k in (0, 2):
        pr, d, (lam, info) = problems[k], dev[k], res[k]
        P = pr["P"]
        x_star = opcg.tik_exact(pr["op"], pr["kp"], pr["B"], lam, tol=1e-10)
        cond = (np.max(np.abs(pr["kp"].Sigma)) ** 2 + lam ** 2) / lam ** 2
        assert rel(kpsvd.from_device(d["x"], P.n_r, P.n_c), x_star) < (1e-4 if cond <= 1e4 else cond * TOL)

    dev = device_problems(kpsvd, problems[:2])
    st, _, res = kpsvd.kp_solve_batch(dev, op_prec="f32", pc_prec="f32", tol=TOL, workers=0, check=False)
    assert st == kpsvd.KP_OK, kpsvd._lib.kp_last_error().decode()
    assert kpsvd.kp_batch_grouped(0)[0] == 0
    for pr, d, (lam, info) in zip(problems[:2], dev, res):
        P = pr["P"]
        x_star = opcg.tik_exact(pr["op"], pr["kp"], pr["B"], lam, tol=1e-10)
        cond = (np.max(np.abs(pr["kp"].Sigma)) ** 2 + lam ** 2) / lam ** 2
        assert info.status == kpsvd.KP_OK
        assert rel(kpsvd.from_device(d["x"], P.n_r, P.n_c), x_star) < (1e-4 if cond <= 1e4 else cond * TOL)
