"""The allocation-free preconditioner solve (kp_apply_Minv_noalloc) against
the context-based one (kp_apply_Minv with FP32 factors), through the C ABI.

Callers that cannot allocate device memory use the no-allocation entry
point; it must give what the regular entry point gives.  This file is
collected last so that a run stopping at its first failure has already run
every other test; it also passes on its own in a fresh process."""
import numpy as np
import pytest

from gpu_common import OracleProblem, lib, rel, setup_ctx, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [64, 256])
def test_noalloc_preconditioner_matches_context_path(n):
    kpsvd = lib()
    pr = OracleProblem("deblur256_fp32", n=n, rank=3)
    lam = 0.02
    with setup_ctx(kpsvd, pr, "f32", "f32", "f32") as ctx:
        svd = ctx.kp_get_kpsvd()
        sigma = ctx.kp_get_spectrum()
        R = np.random.default_rng(17).standard_normal((n, n))
        r = kpsvd.to_device(R, torch.float32)
        z_ref = torch.empty_like(r)
        ctx.kp_apply_Minv(r, z_ref, lam)
        torch.cuda.synchronize()
        Vc = kpsvd.to_device(svd["Vc"], torch.float32)
        Vr = kpsvd.to_device(svd["Vr"], torch.float32)
        sg = kpsvd.to_device(sigma, torch.float64)
        for _ in range(2):   # two calls in a row share the scratch array
            z = torch.full_like(r, float("nan"))
            kpsvd.kp_apply_Minv_noalloc(Vc, Vr, sg, n, n, lam, r, z)
            torch.cuda.synchronize()
            assert rel(z.cpu().numpy(), z_ref.cpu().numpy()) < 1e-5


def test_noalloc_rejects_oversize():
    kpsvd = lib()
    t = torch.zeros(4, dtype=torch.float32, device="cuda")
    s = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(kpsvd.KpError) as e:
        kpsvd.kp_apply_Minv_noalloc(t, t, s, 1024, 1024, 0.1, t, t.clone())
    assert e.value.status == kpsvd.KP_EINVAL
