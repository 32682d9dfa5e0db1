"""Pins for the learned-lambda oracle (oracle/mlp.py): GELU against the
normal CDF, the backward pass against central finite differences of the
loss, the first two Adam steps against their closed forms, and the spectral
features against a hand-built spectrum."""
import numpy as np
import pytest
from scipy.stats import norm

from oracle import mlp


def test_gelu_is_x_times_normal_cdf():
    x = np.linspace(-6, 6, 241)
    np.testing.assert_allclose(mlp.gelu(x), x * norm.cdf(x), rtol=1e-14, atol=1e-300)
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_grad(x), (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h), rtol=1e-7, atol=1e-9)


def test_forward_pass_by_hand():
    """One hidden unit, fed by feature 0 alone: x_0 = 3, mean 1, inv_std 0.5
    normalise to 1; the unit's pre-activation is 1 (weight 1, bias 0), GELU(1)
    = Phi(1) = 0.8413447461 (standard normal table); the output layer gives
    2 Phi(1) + 0.5.  Every other feature equals its mean.  The output weight
    is stored as 2 + 2^-7, a tie between the bf16 neighbours 2 and 2 + 2^-6
    that rounds to even (2): the forward pass uses bf16-rounded weights."""
    rng = np.random.default_rng(6)
    x = rng.standard_normal(mlp.N_FEAT)
    mean = x.copy()
    inv_std = rng.uniform(0.5, 2.0, mlp.N_FEAT)
    x[0], mean[0], inv_std[0] = 3.0, 1.0, 0.5
    net = mlp.init(1, 1, rng, mean=mean, inv_std=inv_std)
    net.W[0][:] = 0.0
    net.W[0][0, 0] = 1.0
    net.W[1][:] = 2.0 + 2.0 ** -7
    net.c[1][:] = 0.5
    pred, _, _ = mlp.forward(net, x[None, :])
    assert pred[0] == pytest.approx(2.0 * 0.8413447461 + 0.5, abs=2e-10)
    assert mlp.loss(net, x[None, :], [pred[0] + 0.25]) == pytest.approx(0.0625, rel=1e-14)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(3)
    net = mlp.init(8, 2, rng, mean=rng.standard_normal(mlp.N_FEAT), inv_std=rng.uniform(0.5, 2, mlp.N_FEAT))
    for c in net.c:
        c[:] = rng.standard_normal(c.shape) * 0.1
    X = rng.standard_normal((5, mlp.N_FEAT))
    y = rng.standard_normal(5)
    gW, gc = mlp.gradients(net, X, y, bf16=False)
    h = 1e-6
    for l in range(len(net.W)):
        for arr, g in ((net.W[l], gW[l]), (net.c[l], gc[l])):
            flat = arr.reshape(-1)
            idx = rng.choice(flat.size, size=min(12, flat.size), replace=False)
            for k in idx:
                old = flat[k]
                flat[k] = old + h
                lp_ = mlp.loss(net, X, y, bf16=False)
                flat[k] = old - h
                lm_ = mlp.loss(net, X, y, bf16=False)
                flat[k] = old
                assert abs((lp_ - lm_) / (2 * h) - g.reshape(-1)[k]) <= 1e-6 * max(1.0, abs(g.reshape(-1)[k]))


def test_adam_first_two_steps_closed_form():
    rng = np.random.default_rng(4)
    net = mlp.init(4, 1, rng)
    w0 = [p.copy() for p in net.params()]
    g1 = [rng.standard_normal(p.shape) for p in w0]
    g2 = [rng.standard_normal(p.shape) for p in w0]
    lr, eps = 1e-3, 1e-8
    split = lambda g: ([g[0], g[2]], [g[1], g[3]])  # noqa: E731  (W, c) per layer
    mlp.adam_step(net, *split(g1), lr)
    for p, p0, a in zip(net.params(), w0, g1):  # m_hat = g, v_hat = g^2
        np.testing.assert_allclose(p, p0 - lr * a / (np.abs(a) + eps), rtol=0, atol=1e-15)
    w1 = [p.copy() for p in net.params()]
    mlp.adam_step(net, *split(g2), lr)
    for p, p1, a, b in zip(net.params(), w1, g1, g2):
        mh = (0.9 * 0.1 * a + 0.1 * b) / (1 - 0.9 ** 2)
        vh = (0.999 * 0.001 * a * a + 0.001 * b * b) / (1 - 0.999 ** 2)
        np.testing.assert_allclose(p, p1 - lr * mh / (np.sqrt(vh) + eps), rtol=0, atol=1e-15)


def test_features_of_a_hand_built_spectrum():
    """s2 = (1, 1, 0.5, 1e-3, 1e-20, 0): bins 0, 0, 2 (0.301 * 127/16 = 2.39),
    23 (3 * 127/16 = 23.8); 1e-20 and 0 are below the 16-decade floor."""
    sig = np.sqrt(np.array([1.0, 1.0, 0.5, 1e-3, 1e-20, 0.0]))
    bh = np.array([2.0, 1.0, 3.0, 0.5, 7.0, 9.0])
    f = mlp.features(sig, bh)
    n, tiny = 6, 1e-30
    exp = {0: np.log10((4.0 + 1.0 + tiny) / 3), 2: np.log10((9.0 + tiny) / 2), 23: np.log10((0.25 + tiny) / 2)}
    for j in range(mlp.NB):
        e = exp.get(j, np.log10(tiny / 1.0))
        assert f[j] == pytest.approx(e, rel=1e-12, abs=1e-12), j
        c = {0: 2, 2: 1, 23: 1}.get(j, 0)
        assert f[mlp.NB + j] == pytest.approx(np.log10((c + 1.0) / n), rel=1e-12), j
    # the deepest bins holding >= n / 8 = 0.75 components: bin 23 alone
    assert f[254] == pytest.approx(np.log10(0.25 + tiny), rel=1e-12)
    assert f[255] == pytest.approx(0.0, abs=1e-15)


def test_features_are_permutation_invariant_and_shift_with_scale():
    rng = np.random.default_rng(5)
    sig = np.exp(-rng.uniform(0, 12, 400))
    bh = rng.standard_normal(400)
    f = mlp.features(sig, bh)
    perm = rng.permutation(400)
    np.testing.assert_allclose(mlp.features(sig[perm], bh[perm]), f, rtol=1e-13, atol=1e-13)
    g = mlp.features(sig, 10.0 * bh)
    occupied = f[mlp.NB:2 * mlp.NB] > np.log10(1.0 / 400) + 1e-9
    np.testing.assert_allclose(g[:mlp.NB][occupied], f[:mlp.NB][occupied] + 2.0, atol=1e-12)
    assert g[254] == pytest.approx(f[254] + 2.0, abs=1e-12)
    # scaling Sigma by 10 scales s2 by 100: bins and counts (relative to
    # s2max) stay, f[255] = log10(s2max) moves by 2
    h = mlp.features(10.0 * sig, bh)
    np.testing.assert_array_equal(h[mlp.NB:2 * mlp.NB], f[mlp.NB:2 * mlp.NB])
    np.testing.assert_allclose(h[:mlp.NB][occupied], f[:mlp.NB][occupied], atol=1e-12)
    assert h[255] == pytest.approx(f[255] + 2.0, abs=1e-12)
