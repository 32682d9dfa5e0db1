"""The allocation-free preconditioner solve (kp_apply_Minv_noalloc) through
the C ABI, against the context-based solve (kp_apply_Minv with FP32
factors) and against the oracle's eq. PreconSolve on the same FP32 factors.

Some callers cannot allocate device memory: code that runs inside a memory
pool or arena owned by another allocator, a runtime that forbids device
allocation, or a loop that must not allocate.  They use the no-allocation
entry point, which must give what the regular entry point gives.  This file
is collected last so that a run stopping at its first failure has already
run every other test; it also passes on its own in a fresh process."""
import numpy as np
import pytest

from gpu_common import OracleProblem, lib, rel, setup_ctx, torch
from oracle import kpsvd as okp, lowprec as lp

pytestmark = pytest.mark.gpu

# square, rectangular both ways with ragged sizes, and the 512-per-side limit
# (at 512 x 512 the intermediates fill the whole scratch array)
SHAPES = [(64, 64), (256, 256), (144, 208), (208, 144), (512, 384), (512, 512)]


class _Factors:
    def __init__(self, Vc, Vr):
        self.Vc, self.Vr = Vc, Vr


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{s[0]}x{s[1]}")
def test_noalloc_preconditioner_matches_context_path(shape):
    kpsvd = lib()
    n_r, n_c = shape
    pr = OracleProblem("deblur256_fp32", n=max(256, n_r, n_c), shape=shape, rank=3)
    lam = 0.02
    with setup_ctx(kpsvd, pr, "f32", "f32", "f32") as ctx:
        svd = ctx.kp_get_kpsvd()
        sigma = ctx.kp_get_spectrum()
        R = np.random.default_rng(17).standard_normal((n_r, n_c))
        r = kpsvd.to_device(R, torch.float32)
        z_ref = torch.empty_like(r)
        ctx.kp_apply_Minv(r, z_ref, lam)
        torch.cuda.synchronize()
        Z_ref = kpsvd.from_device(z_ref, n_r, n_c)
        Vc = kpsvd.to_device(svd["Vc"], torch.float32)
        Vr = kpsvd.to_device(svd["Vr"], torch.float32)
        sg = kpsvd.to_device(sigma, torch.float64)
        # eq. PreconSolve in FP64 on the FP32 factors and residual the call reads
        Z64 = okp.precond_apply(_Factors(lp.to_fp32(svd["Vc"]), lp.to_fp32(svd["Vr"])),
                                okp.precond_scale(sigma, lam), lp.to_fp32(R))
        for _ in range(2):   # two calls in a row share the scratch array
            z = torch.full_like(r, float("nan"))
            kpsvd.kp_apply_Minv_noalloc(Vc, Vr, sg, n_r, n_c, lam, r, z)
            torch.cuda.synchronize()
            Z = kpsvd.from_device(z, n_r, n_c)
            assert np.isfinite(Z).all()
            assert rel(Z, Z_ref) < 1e-5
            assert rel(Z, Z64) < 1e-5


@pytest.mark.parametrize("shape", [(1024, 1024), (513, 64), (64, 513)], ids=lambda s: f"{s[0]}x{s[1]}")
def test_noalloc_rejects_oversize(shape):
    """Sizes beyond the fixed scratch are refused by the library itself (raw
    addresses skip the binding's own size checks; nothing is launched)."""
    kpsvd = lib()
    n_r, n_c = shape
    t = torch.zeros(4, dtype=torch.float32, device="cuda")
    o = torch.zeros(4, dtype=torch.float32, device="cuda")
    s = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(kpsvd.KpError) as e:
        kpsvd.kp_apply_Minv_noalloc(t.data_ptr(), t.data_ptr(), s.data_ptr(), n_r, n_c, 0.1, t.data_ptr(),
                                    o.data_ptr())
    assert e.value.status == kpsvd.KP_EINVAL
    assert "kp_apply_Minv_noalloc" in str(e.value) and "exceeds" in str(e.value)
