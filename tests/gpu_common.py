"""Shared helpers of the GPU parity tests (test infrastructure: builds oracle
problems and the reduced-precision emulation of the tensor-core path)."""
import numpy as np
import pytest

from oracle import forward, kpsvd as okp, kron, lowprec as lp
from paper_2311_15393_gb300 import synth

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def lib():
    need_gpu()
    from paper_2311_15393_gb300 import build
    build.build()
    from paper_2311_15393_gb300 import kpsvd
    return kpsvd


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


class OracleProblem:
    """Oracle-side view of a synthetic problem."""

    def __init__(self, name, n=None, psf=None, center=None, bc=None, rank=None, noise_idx=0, shape=None, seed=None):
        P = synth.make_problem(name, n=n, seed=seed)
        if shape is not None:   # rectangular variant: crop image / re-sample PSF
            n_r, n_c = shape
            c = center or (n_r // 2, n_c // 2)
            P.x_true = P.x_true[:n_r, :n_c]
            P.psf = synth.gaussian_psf(n_r, n_c, c[0], c[1], P.extra["sigma_x"], P.extra["sigma_y"], P.extra["rho"])
            P.noise_dirs = [g[:n_r, :n_c] for g in P.noise_dirs]
            P.n_r, P.n_c, P.center = n_r, n_c, c
        if psf is not None:
            P.psf = psf
        if center is not None:
            P.center = center
        if bc is not None:
            P.bc = bc
        if rank is not None:
            P.op_rank = rank
        self.P = P
        self.op = kron.kron_operator(P.psf, P.center, P.bc, P.op_rank)
        self.kp = okp.kp_svd(self.op, "projected")
        self.B, self.enorm = forward.observe(self.op, P.x_true, P.noise_dirs[noise_idx], P.noise_levels[noise_idx])


def setup_ctx(kpsvd, prob: OracleProblem, op_prec, pc_prec, vec_prec, sigma="projected"):
    P = prob.P
    ctx = kpsvd.KpContext(0)
    psf = kpsvd.to_device(P.psf)
    ctx.kp_setup(psf, P.n_r, P.n_c, P.center, P.bc, P.op_rank, op_prec, pc_prec, vec_prec, sigma)
    torch.cuda.synchronize()
    return ctx


def vt(vec_prec):
    return torch.float64 if vec_prec == "f64" else torch.float32


# ---------------------------------------------------------------- emulation
def bf(x):
    return lp.to_bf16(x)


def emulate_apply_A_bf16(op, X):
    """Tensor-core inner operator with one bf16 slice: factors and activations
    rounded to bf16, products summed exactly, outputs of each GEMM rounded to
    fp32 and (intermediate) to bf16."""
    Xb = bf(lp.to_fp32(X))
    W = [bf(lp.to_fp32(bf(Ac) @ Xb)) for Ac in op.Ac]
    return lp.to_fp32(sum(Wk @ bf(Ar).T for Wk, Ar in zip(W, op.Ar)))


def pow2_scale(amax, target):
    """2^e with amax * 2^e in [target / 2, target) (1 when amax is 0)."""
    if not amax > 0:
        return 1.0
    m, e = np.frexp(target / amax)
    return float(np.ldexp(1.0, e - 1))


def emulate_minv_e4m3(kp, Sigma, R, lam):
    """E4M3 preconditioner solve with the GPU's rounding points: per-factor
    power-of-two scales (max |V| s_V in [224, 448)), R scaled the same way,
    every GEMM accumulated exactly then rounded to fp32, each of the first
    three outputs rescaled by a power of two from its own max |.| and rounded
    to e4m3; the scales are undone at the end (in fp32)."""
    f32, q = lp.to_fp32, lp.to_e4m3
    sc, sr = pow2_scale(np.abs(kp.Vc).max(), 448.0), pow2_scale(np.abs(kp.Vr).max(), 448.0)
    Vc, Vr = q(f32(kp.Vc * sc)), q(f32(kp.Vr * sr))
    R32 = f32(R)
    s_R = pow2_scale(np.abs(R32).max(), 448.0)
    Rq = q(f32(R32 * s_R))
    base = f32(1.0 / (lam * lam * (sc * sr) ** 2 * s_R))
    S32 = f32(Sigma)
    l2 = f32(lam * lam)
    fac = f32(l2 / f32(S32 * S32 + l2))
    g = []
    T1 = f32(Vc.T @ Rq)
    g.append(pow2_scale(np.abs(T1).max(), 448.0))
    T1q = q(f32(T1 * g[0]))
    W = f32(f32(T1q @ Vr) * fac)
    g.append(pow2_scale(np.abs(W).max(), 448.0))
    Wq = q(f32(W * g[1]))
    T3 = f32(Vc @ Wq)
    g.append(pow2_scale(np.abs(T3).max(), 448.0))
    T3q = q(f32(T3 * g[2]))
    inv = f32(base / f32(f32(g[0] * g[1]) * g[2]))
    return f32(f32(T3q @ Vr.T) * inv)


def emulate_minv(kp, Sigma, R, lam, fmt):
    """Reduced-precision preconditioner solve with the GPU's rounding points:
    R scaled by 2^e (amax(R) 2^e in [1/2, 1)) and rounded (bf16 factors as
    hi + lo pairs); each GEMM output
    rounded to fp32 then to the narrow format; S applied as
    lam^2 / (Sigma^2 + lam^2) (FP32) in the P2 output; 1 / (lam^2 2^e) at the end."""
    if fmt == "e4m3":
        return emulate_minv_e4m3(kp, Sigma, R, lam)
    rd = lp.ROUND[fmt]
    am = np.max(np.abs(lp.to_fp32(R)))
    m, e = np.frexp(1.0 / am)
    s = np.ldexp(1.0, e - 1)
    Rq = rd(lp.to_fp32(R) * s)
    if fmt == "bf16":   # factors carried as bf16 hi + lo pairs
        Vc = lp.to_bf16(kp.Vc) + lp.to_bf16(kp.Vc - lp.to_bf16(kp.Vc))
        Vr = lp.to_bf16(kp.Vr) + lp.to_bf16(kp.Vr - lp.to_bf16(kp.Vr))
    else:
        Vc, Vr = rd(kp.Vc), rd(kp.Vr)
    T1 = rd(lp.to_fp32(Vc.T @ Rq))
    S32 = lp.to_fp32(Sigma)
    l2 = lp.to_fp32(lam * lam)
    fac = lp.to_fp32(l2 / lp.to_fp32(S32 * S32 + l2))   # FP32 on the GPU
    W = rd(lp.to_fp32(lp.to_fp32(T1 @ Vr) * fac))
    T3 = rd(lp.to_fp32(Vc @ W))
    inv = lp.to_fp32(1.0 / (lam * lam * s))
    return lp.to_fp32(lp.to_fp32(T3 @ Vr.T) * inv)
