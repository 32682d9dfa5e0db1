"""GPU parity of the learned-lambda pieces against the FP64 oracle
(oracle/mlp.py): spectral features, the MLP forward pass, its gradients and
the Adam step, through the C ABI."""
import numpy as np
import pytest

from gpu_common import OracleProblem, lib, setup_ctx, torch
from oracle import lam as olam, lowprec as lp, mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kpsvd():
    return lib()


def test_features_match_oracle(kpsvd):
    """FP64 setup (Sigma exact to rounding, so no component changes bin): the
    256 features equal the oracle's from its own Sigma and b_hat."""
    pr = OracleProblem("deblur256_fp32", n=128, rank=3)
    f_o = omlp.features(pr.kp.Sigma, olam.spectral_coeffs(pr.kp, pr.B))
    with setup_ctx(kpsvd, pr, "f64", "f64", "f64") as ctx:
        b = kpsvd.to_device(pr.B, torch.float64)
        f = torch.empty(omlp.N_FEAT, dtype=torch.float32, device="cuda:0")
        ctx.kp_lambda_features(b, f)
        f = f.cpu().double().numpy()
    np.testing.assert_allclose(f, f_o, rtol=0, atol=2e-6 * np.abs(f_o).max())


def _net(width, depth, seed):
    """Oracle net with FP32-representable parameters, and its GPU parameter vector."""
    rng = np.random.default_rng(seed)
    net = omlp.init(width, depth, rng, mean=rng.standard_normal(omlp.N_FEAT),
                    inv_std=rng.uniform(0.5, 2.0, omlp.N_FEAT))
    for c in net.c:
        c[:] = rng.standard_normal(c.shape) * 0.1
    net.mean, net.inv_std = lp.to_fp32(net.mean), lp.to_fp32(net.inv_std)
    net.W = [lp.to_fp32(w) for w in net.W]
    net.c = [lp.to_fp32(c) for c in net.c]
    vec = [net.mean, net.inv_std] + [a.ravel() for l in range(len(net.W)) for a in (net.W[l], net.c[l])]
    return net, np.concatenate(vec).astype(np.float32), rng


def _dev(a):
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda:0")


@pytest.mark.parametrize("width,depth,batch", [(64, 2, 37), (256, 3, 256)])
def test_forward_and_gradients_match_oracle(kpsvd, width, depth, batch):
    """Forward and backward with bf16 weights, FP32 activations and
    accumulation, against the oracle in FP64 on the same bf16 weights: FP32
    sums over <= 256 terms, relative ~1e-5 of the largest entry."""
    net, vec, rng = _net(width, depth, 11)
    X = lp.to_fp32(rng.standard_normal((batch, omlp.N_FEAT)))
    y = lp.to_fp32(rng.standard_normal(batch))
    with kpsvd.Mlp(width, depth, 512) as m:
        assert m.param_count == vec.size
        m.set_params(vec)
        np.testing.assert_array_equal(m.get_params(), vec)
        out = torch.empty(batch, dtype=torch.float32, device="cuda:0")
        m.forward(_dev(X), out)
        pred_o, _, _ = omlp.forward(net, X)
        np.testing.assert_allclose(out.cpu().double().numpy(), pred_o, rtol=0, atol=1e-5 * np.abs(pred_o).max())
        g, loss = m.gradients(_dev(X), _dev(y))
    assert loss == pytest.approx(omlp.loss(net, X, y), rel=1e-5)
    gW, gc = omlp.gradients(net, X, y)
    k = 2 * omlp.N_FEAT
    assert np.all(g[:k] == 0)
    for l in range(depth + 1):
        for ref in (gW[l], gc[l]):
            n = ref.size
            np.testing.assert_allclose(g[k:k + n], ref.ravel(), rtol=0, atol=2e-5 * np.abs(ref).max() + 1e-12)
            k += n
    assert k == g.size


def test_adam_step_matches_oracle(kpsvd):
    """One train step = the oracle's gradients followed by its Adam update
    (bias-corrected first step: w - lr g / (|g| + eps)); entries whose
    gradient is too small for its sign to be certain in FP32 may differ by at
    most the step size."""
    net, vec, rng = _net(64, 2, 12)
    X = lp.to_fp32(rng.standard_normal((50, omlp.N_FEAT)))
    y = lp.to_fp32(rng.standard_normal(50))
    lr = 1e-3
    with kpsvd.Mlp(64, 2, 64) as m:
        m.set_params(vec)
        m.train_step(_dev(X), _dev(y), lr)
        got = m.get_params().astype(np.float64)
    gW, gc = omlp.gradients(net, X, y)
    omlp.adam_step(net, gW, gc, lr)
    k = 2 * omlp.N_FEAT
    for l in range(3):
        for new, g in ((net.W[l], gW[l]), (net.c[l], gc[l])):
            n = new.size
            d = np.abs(got[k:k + n] - new.ravel())
            sure = np.abs(g.ravel()) > 1e-5 * max(np.abs(g).max(), 1e-30)
            assert d[sure].max(initial=0.0) < 1e-6
            assert d.max(initial=0.0) <= 2 * lr + 1e-7
            k += n


def test_training_reduces_the_loss(kpsvd):
    """A few hundred Adam steps on a smooth synthetic target (a fixed random
    projection of the features) cut the loss by more than 10x."""
    rng = np.random.default_rng(13)
    _, vec, _ = _net(128, 2, 14)
    vec[:omlp.N_FEAT] = 0.0
    vec[omlp.N_FEAT:2 * omlp.N_FEAT] = 1.0
    X = rng.standard_normal((1024, omlp.N_FEAT)).astype(np.float32)
    w = rng.standard_normal(omlp.N_FEAT) / np.sqrt(omlp.N_FEAT)
    y = np.tanh(X @ w).astype(np.float32)
    Xd, yd = _dev(X), _dev(y)
    with kpsvd.Mlp(128, 2, 256) as m:
        m.set_params(vec)
        first = None
        for step in range(400):
            i = (step % 4) * 256
            loss = m.train_step(Xd[i:i + 256], yd[i:i + 256], 1e-3)
            first = loss if first is None else first
        _, last = m.gradients(Xd[:256], yd[:256])
    assert last < first / 10


def _problem_data(kpsvd, ctx, P, feat):
    """Set up one generated problem; its observed b (the context's own
    operator), noise norm and spectral features."""
    ctx.kp_setup(kpsvd.to_device(P.psf), P.n_r, P.n_c, P.center, P.bc, P.op_rank, "bf16", "f16", "f32", "projected")
    xt = kpsvd.to_device(P.x_true, torch.float32)
    b = torch.empty_like(xt)
    enorm = ctx.kp_forward(xt, kpsvd.to_device(P.noise_dirs[0], torch.float32), P.noise_levels[0], b)
    ctx.kp_lambda_features(b, feat)
    return b, enorm, feat.cpu().numpy().astype(np.float64)


def test_learned_lambda_gains_over_gcv(kpsvd):
    """What the trained network gains over closed-form GCV: an MLP trained
    (hand-written tcgen05 forward / backward kernels and Adam) on 2,048
    generated 256^2 problems labelled by the discrepancy principle, then on
    64 new problems lambda from the MLP against GCV's: FPCG (tol 1e-7) takes
    at least 20% fewer iterations on average, and the median relative
    reconstruction error against x_true is within 10% of GCV's."""
    from paper_2311_15393_gb300 import synth
    feat = torch.empty(omlp.N_FEAT, dtype=torch.float32, device="cuda:0")
    seed = synth.SEED_BASE + 4
    Xtr, ytr = [], []
    with kpsvd.KpContext(0) as ctx:
        for P in synth.make_batch(2048, sizes=[(256, 256)], seed=seed):
            b, enorm, f = _problem_data(kpsvd, ctx, P, feat)
            Xtr.append(f)
            ytr.append(np.log10(ctx.choose_lambda(b, "discrepancy", 1.01 * enorm)))
        Xtr, ytr = np.array(Xtr), np.array(ytr)
        mean, std = Xtr.mean(axis=0), np.maximum(Xtr.std(axis=0), 1e-3)
        rng = np.random.default_rng(seed)
        width, depth, bs = 256, 3, 256
        sizes = [omlp.N_FEAT] + [width] * depth + [1]
        vec = [mean, 1.0 / std]
        for l in range(depth + 1):
            vec += [rng.standard_normal((sizes[l + 1], sizes[l])).ravel() * np.sqrt(2.0 / sizes[l]),
                    np.zeros(sizes[l + 1])]
        vec = np.concatenate(vec).astype(np.float32)
        Xd, yd = _dev(Xtr), _dev(ytr)
        rows = []
        with kpsvd.Mlp(width, depth, bs) as m:
            m.set_params(vec)
            for ep in range(40):
                perm = torch.tensor(rng.permutation(len(ytr)), device="cuda:0")
                Xs, ys = Xd[perm], yd[perm]
                for i in range(0, len(ytr) - bs + 1, bs):
                    m.train_step(Xs[i:i + bs], ys[i:i + bs], 1e-3)
            out = torch.empty(1, dtype=torch.float32, device="cuda:0")
            for P in synth.make_batch(64, sizes=[(256, 256)], seed=seed + 500):
                b, enorm, f = _problem_data(kpsvd, ctx, P, feat)
                m.forward(feat.view(1, omlp.N_FEAT), out)
                lams = {"mlp": float(10.0 ** out.item()), "gcv": ctx.choose_lambda(b, "gcv")}
                r = {}
                for name, lam in lams.items():
                    x = torch.zeros_like(b)
                    info = ctx.tik_pcg(b, lam, 1e-7, 500, True, x, check=False)
                    X = kpsvd.from_device(x, P.n_r, P.n_c)
                    r[name] = (info.iters, np.linalg.norm(X - P.x_true) / np.linalg.norm(P.x_true))
                rows.append(r)
    it = {k: float(np.mean([r[k][0] for r in rows])) for k in ("mlp", "gcv")}
    err = {k: float(np.median([r[k][1] for r in rows])) for k in ("mlp", "gcv")}
    print(f"learned lambda vs GCV on 64 new problems: mean iterations {it['mlp']:.1f} vs {it['gcv']:.1f}, "
          f"median error {err['mlp']:.4f} vs {err['gcv']:.4f}")
    assert it["mlp"] <= 0.8 * it["gcv"]
    assert err["mlp"] <= 1.10 * err["gcv"]
