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
