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


def gpu_operator(ctx, prob: OracleProblem):
    """Operator built from the context's own Kronecker terms (kp_get_terms)
    by the oracle's factor construction (eq. KronSumDecomp).  A
    reduced-precision emulation fed with it rounds exactly the factor values
    the GPU rounds, so comparing against it checks the GEMMs alone; how the
    GPU's setup arrived at its terms is checked against the oracle apart."""
    s, U, V = ctx.kp_get_terms()
    P = prob.P
    c_r, c_c = P.center
    Ac = [kron.blur_factor(U[:, m], c_r, P.bc) for m in range(U.shape[1])]
    Ar = [kron.blur_factor(V[:, m], c_c, P.bc) for m in range(V.shape[1])]
    return kron.KronOperator(Ac=Ac, Ar=Ar, s=s, u=U, v=V, bc=P.bc)


class GpuKpsvd:
    """The context's own KP-SVD factors and spectrum (getters), in the shape
    the emulations read (Vc, Vr, Sigma)."""

    def __init__(self, ctx):
        f = ctx.kp_get_kpsvd()
        self.Vc, self.Vr, self.sc, self.sr = f["Vc"], f["Vr"], f["sc"], f["sr"]
        self.Uc, self.Ur = f["Uc"], f["Ur"]
        self.Sigma = ctx.kp_get_spectrum()


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


def emulate_apply_AT_bf16(op, Y):
    """A^T Y on the tensor-core inner operator, with the rounding points of
    emulate_apply_A_bf16 (G3 output rounded to bf16, G4 accumulated)."""
    Yb = bf(lp.to_fp32(Y))
    W = [bf(lp.to_fp32(bf(Ac).T @ Yb)) for Ac in op.Ac]
    return lp.to_fp32(sum(Wk @ bf(Ar) for Wk, Ar in zip(W, op.Ar)))


U32 = 2.0 ** -24


def bf16_operator_bound(op, X, transpose=False):
    """Bound on |GPU - emulation| / |emulation| for the inner BF16 operator
    applied to X, derived from the arithmetic.  The two sides round the same
    bf16 operands and products of bf16 values are exact in FP32; they differ
    only by FP32 accumulation.  A sum of m nonzero products accumulated in
    FP32 in any order (rounded or truncated) is within 2 (m - 1) u32 sum |.|
    of the exact sum.  (1) Where that interval around an exact first-GEMM
    output straddles a bf16 rounding boundary, the GPU's bf16 intermediate W
    may be one bf16 step off the emulation's (D); (2) the second GEMM's FP32
    sum adds its own accumulation error.  Returns
    (|| sum_k D_k |B_k| || + || 2 (m - 1) u32 sum_k |W_k| |B_k| ||) / ||Y||,
    with B_k the second factor as the second GEMM reads it."""
    Xb = bf(lp.to_fp32(X))
    first = [bf(Ac).T if transpose else bf(Ac) for Ac in op.Ac]
    second = [bf(Ar) if transpose else bf(Ar).T for Ar in op.Ar]
    nz = lambda A: (A != 0).astype(np.float64)  # noqa: E731
    Y = 0.0
    flips = 0.0
    acc = 0.0
    cnt2 = 0.0
    for F, G in zip(first, second):
        S = F @ Xb
        m1 = nz(F) @ nz(Xb)
        E = 2.0 * np.maximum(m1 - 1.0, 0.0) * U32 * (np.abs(F) @ np.abs(Xb))
        W = bf(lp.to_fp32(S))
        D = np.maximum(np.abs(bf(lp.to_fp32(S + E)) - W), np.abs(bf(lp.to_fp32(S - E)) - W))
        Y = Y + W @ G
        flips = flips + D @ np.abs(G)
        acc = acc + np.abs(W) @ np.abs(G)
        cnt2 = cnt2 + nz(W) @ nz(G)
    acc_err = 2.0 * np.maximum(cnt2 - 1.0, 0.0) * U32 * acc
    return (np.linalg.norm(flips) + np.linalg.norm(acc_err)) / np.linalg.norm(Y)


def spike_image(n_r, n_c, seed=0):
    """Sparse test image for the tensor-core operator: one entry per used
    column (so every element of the first GEMM's output is a single product,
    exact in FP32 and in bf16), at rows and columns that reach the first,
    the interior and the ragged last tiles of both dimensions (128-row and
    64-element blocks), with values +-2^e, e in {-1, 0, 1}."""
    rng = np.random.default_rng(seed)
    cols = sorted({c for c in (0, 1, 31, 63, 64, 100, 127, 128, 191, 192, 255, n_c - 17, n_c - 2, n_c - 1)
                   if 0 <= c < n_c})
    rows = [0, 15, 63, 64, 127, 128, 150, n_r - 33, n_r - 16, n_r - 1]
    X = np.zeros((n_r, n_c))
    for m, c in enumerate(cols):
        r = rows[m % len(rows)] % n_r
        X[r, c] = rng.choice([-1.0, 1.0]) * 2.0 ** int(rng.integers(-1, 2))
    return X


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


def check_bf16_operator(kpsvd, ctx, pr, n_r, n_c):
    """Inner BF16 operator A and A^T against their emulation on the GPU's own
    terms (both sides round the same factor values):
    - on a spike image every product of the first GEMM stands alone, so both
      sides form the same bf16 intermediate and differ only by the second
      GEMM's FP32 sum of a few dozen exact products: agreement to the
      derived bound (~1e-5, typically ~1e-7 measured), which any misplaced,
      dropped or stale row, column or k-block of a ragged tile would exceed
      by orders of magnitude;
    - on a dense random image, within the bound derived from the FP32
      accumulation (bf16_operator_bound), and within bf16 rounding of FP64."""
    gop = gpu_operator(ctx, pr)
    for name, X in (("spike", spike_image(n_r, n_c, 3)), ("random", synth.random_matrix(n_r, n_c, 11))):
        x = kpsvd.to_device(X, torch.float32)
        y = torch.empty_like(x)
        for tr in (False, True):
            ctx.kp_apply_A(x, y, tr)
            Y = kpsvd.from_device(y, n_r, n_c)
            emu = emulate_apply_AT_bf16(gop, X) if tr else emulate_apply_A_bf16(gop, X)
            e_emu = rel(Y, emu)
            bound = bf16_operator_bound(gop, X, tr)
            print(f"{(n_r, n_c)} {name} {'A^T' if tr else 'A'}: vs emulation {e_emu:.3e} (bound {bound:.2e})")
            assert e_emu <= bound
            if name == "spike":   # exact intermediates: only the second sum's rounding remains
                assert bound < 1e-4
            ref = kron.apply_AT(pr.op, X) if tr else kron.apply_A(pr.op, X)
            assert rel(Y, ref) < 2e-2
