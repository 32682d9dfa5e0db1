"""Failure detection without a GPU fault: an injected allocation failure
(KPSVD_FAULT=alloc:N) is reported as KP_ENOMEM and leaves the context
usable; a bounded device wait that nothing releases gives up as KP_ETIMEOUT
and the context then solves as before."""
import numpy as np
import pytest

from gpu_common import OracleProblem, lib, rel, torch
from oracle import pcg as opcg

pytestmark = pytest.mark.gpu


def _setup(kpsvd, ctx, pr):
    P = pr.P
    ctx.kp_setup(kpsvd.to_device(P.psf), P.n_r, P.n_c, P.center, P.bc, P.op_rank, "bf16", "f16", "f32", "projected")


def _solve(kpsvd, ctx, pr, lam):
    b = kpsvd.to_device(pr.B, torch.float32)
    x = torch.zeros_like(b)
    info = ctx.tik_pcg(b, lam, 1e-7, 500, True, x)
    return info, kpsvd.from_device(x, pr.P.n_r, pr.P.n_c)


def test_injected_allocation_failure(monkeypatch):
    kpsvd = lib()
    pr = OracleProblem("deblur256_fp32", n=128, rank=3)
    lam = 0.05
    x_star = opcg.tik_exact(pr.op, pr.kp, pr.B, lam)
    with kpsvd.KpContext(0) as ctx:
        for n in (1, 7, 40):   # early, middle and late allocations of a setup
            monkeypatch.setenv("KPSVD_FAULT", f"alloc:{n}")
            with pytest.raises(kpsvd.KpError) as e:
                _setup(kpsvd, ctx, pr)
            assert e.value.status == kpsvd.KP_ENOMEM and "injected" in str(e.value)
            b = kpsvd.to_device(pr.B, torch.float32)
            info = ctx.tik_pcg(b, lam, 1e-7, 10, True, torch.zeros_like(b), check=False)
            assert info.status == kpsvd.KP_ESTATE   # no problem set up after the failure
        monkeypatch.delenv("KPSVD_FAULT")
        _setup(kpsvd, ctx, pr)
        info, X = _solve(kpsvd, ctx, pr, lam)
    assert info.status == kpsvd.KP_OK and rel(X, x_star) < 1e-4


def test_bounded_wait_gives_up_and_context_stays_usable():
    kpsvd = lib()
    pr = OracleProblem("deblur256_fp32", n=128, rank=3)
    lam = 0.05
    x_star = opcg.tik_exact(pr.op, pr.kp, pr.B, lam)
    with kpsvd.KpContext(0) as ctx:
        _setup(kpsvd, ctx, pr)
        import time
        t0 = time.perf_counter()
        st = ctx.kp_test_bounded_wait(50.0)
        dt = time.perf_counter() - t0
        assert st == kpsvd.KP_ETIMEOUT
        assert 0.04 < dt < 5.0
        info, X = _solve(kpsvd, ctx, pr, lam)
    assert info.status == kpsvd.KP_OK and rel(X, x_star) < 1e-4
