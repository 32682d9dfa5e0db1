"""The tile autotuner (option tc_autotune, cache file KPSVD_TUNE_CACHE): the
tuned GEMMs compute what the built-in tile rule computes, the choices are
written to the cache file once per shape and read back by a new context,
and a solve with them reaches the oracle's x_lambda."""
import os

import numpy as np
import pytest

from gpu_common import OracleProblem, lib, rel, torch
from oracle import lam as olam, pcg as opcg
from paper_2311_15393_gb300 import synth

pytestmark = pytest.mark.gpu


def _ctx(kpsvd, pr, tune):
    ctx = kpsvd.KpContext(0)
    ctx.kp_set_option("tc_autotune", tune)
    P = pr.P
    ctx.kp_setup(kpsvd.to_device(P.psf), P.n_r, P.n_c, P.center, P.bc, P.op_rank, "bf16", "f16", "f32", "projected")
    torch.cuda.synchronize()
    return ctx


def test_autotuned_tiles(tmp_path, monkeypatch):
    kpsvd = lib()
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("KPSVD_TUNE_CACHE", str(cache))
    n = 512
    pr = OracleProblem("deblur1024_mixed", n=n)
    X = synth.random_matrix(n, n, 3)
    with _ctx(kpsvd, pr, 0) as c0, _ctx(kpsvd, pr, 1) as c1:
        x = kpsvd.to_device(X, torch.float32)
        q0, q1, z0, z1 = (torch.empty_like(x) for _ in range(4))
        c0.kp_apply_K(x, q0, 0.02)
        c1.kp_apply_K(x, q1, 0.02)
        c0.kp_apply_Minv(x, z0, 0.02)
        c1.kp_apply_Minv(x, z1, 0.02)
        d_k = rel(kpsvd.from_device(q1, n, n), kpsvd.from_device(q0, n, n))
        d_m = rel(kpsvd.from_device(z1, n, n), kpsvd.from_device(z0, n, n))
        print(f"tuned vs built-in tiles: K p {d_k:.2e}, M^-1 r {d_m:.2e}")
        # the same bf16 / fp16 products summed in FP32; only a K split may
        # change the order of the sums
        assert d_k < 1e-6 and d_m < 1e-3
    lines = cache.read_text().splitlines()
    assert len(lines) >= 4 and all(len(l.split()) == 13 for l in lines)
    lam = olam.choose_lambda(pr.kp, pr.B, "gcv")
    x_star = opcg.tik_exact(pr.op, pr.kp, pr.B, lam, tol=1e-10)
    with _ctx(kpsvd, pr, 1) as c2:   # served from the cache: no new lines
        b = kpsvd.to_device(pr.B, torch.float32)
        xs = torch.zeros_like(b)
        info = c2.tik_pcg(b, lam, 1e-7, 500, True, xs)
        err = rel(kpsvd.from_device(xs, n, n), x_star)
    assert len(cache.read_text().splitlines()) == len(lines)
    assert info.status == kpsvd.KP_OK and err < 1e-4
