"""FP64 oracle of the learned-lambda regressor (scope-table NEXT 2; not in the
paper, which only asks for a systematic choice of the regularisation
parameter, Section 5): spectral features of a problem, and a multilayer
perceptron with GELU activations mapping them to log10(lambda), with its
backward pass and the Adam update.

Test infrastructure only: the product path never imports this module.

Features (N_FEAT = 256) of a problem with KP spectrum Sigma and coefficients
b_hat = vec(U_c^T B U_r) (eq. GCVTikSVD's notation), with s2 = Sigma^2 and
s2max = max s2:
  * bins: component i belongs to bin j = floor(-log10(s2_i / s2max) * NB / DEC)
    for s2_i > s2max 10^-DEC (NB = 127 bins over DEC = 16 decades); smaller
    ones (and zeros) to no bin;
  * f[j]       = log10((sum_{i in bin j} b_hat_i^2 + TINY s2max) / (count_j + 1)), j < NB
  * f[NB + j]  = log10((count_j + 1) / N)
  * f[254]     = log10 of the mean b_hat^2 over the deepest bins holding at
                 least N / 8 components together (a noise-level estimate:
                 an orthogonal transform keeps white noise white, and where
                 Sigma is tiny b_hat is mostly noise)
  * f[255]     = log10(s2max)
Model: x -> (x - mean) * inv_std -> [Linear(256, W) -> GELU] x depth ->
Linear(W, 1); the Linear weights are used rounded to bf16 (the GPU keeps FP32
masters for the optimiser and bf16 copies for the products), biases in full
precision.  GELU(x) = x Phi(x) = x erfc(-x / sqrt 2) / 2.  Loss: mean
squared error of log10(lambda).  Adam (Kingma and Ba 2015) with bias
correction.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy.special import erfc

from . import lowprec as lp

N_FEAT = 256
NB = 127
DEC = 16.0
TINY = 1e-30


def features(Sigma: np.ndarray, Bhat: np.ndarray) -> np.ndarray:
    """The 256 features of one problem (module docstring)."""
    s2 = np.asarray(Sigma, dtype=np.float64).ravel() ** 2
    b2 = np.asarray(Bhat, dtype=np.float64).ravel() ** 2
    n = s2.size
    s2max = s2.max()
    f = np.zeros(N_FEAT)
    cnt = np.zeros(NB)
    sb = np.zeros(NB)
    for i in range(n):  # plain loop: the definition, element by element
        if s2[i] > s2max * 10.0 ** (-DEC):
            j = int(np.floor(-np.log10(s2[i] / s2max) * NB / DEC))
            j = min(j, NB - 1)
            cnt[j] += 1
            sb[j] += b2[i]
    for j in range(NB):
        f[j] = np.log10((sb[j] + TINY * s2max) / (cnt[j] + 1.0))
        f[NB + j] = np.log10((cnt[j] + 1.0) / n)
    acc_c, acc_b = 0.0, 0.0
    for j in range(NB - 1, -1, -1):
        acc_c += cnt[j]
        acc_b += sb[j]
        if acc_c >= n / 8.0:
            break
    f[2 * NB] = np.log10((acc_b + TINY * s2max) / max(acc_c, 1.0))
    f[2 * NB + 1] = np.log10(s2max)
    return f


def _phi(x):  # normal CDF, erfc form (no cancellation in the lower tail)
    return 0.5 * erfc(-x / np.sqrt(2.0))


def gelu(x):
    return x * _phi(x)


def gelu_grad(x):
    return _phi(x) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


@dataclass
class MLP:
    """Weights W[l] (out x in), biases c[l]; the last layer has out = 1."""
    W: list
    c: list
    mean: np.ndarray
    inv_std: np.ndarray
    # Adam moments, one per parameter array (W then c per layer)
    m: list = field(default_factory=list)
    v: list = field(default_factory=list)
    t: int = 0

    def params(self):
        return [a for l in range(len(self.W)) for a in (self.W[l], self.c[l])]


def init(width: int, depth: int, rng: np.random.Generator, mean=None, inv_std=None) -> MLP:
    """He-style normal initialisation (std sqrt(2 / fan_in)), zero biases."""
    sizes = [N_FEAT] + [width] * depth + [1]
    W = [rng.standard_normal((sizes[l + 1], sizes[l])) * np.sqrt(2.0 / sizes[l]) for l in range(len(sizes) - 1)]
    c = [np.zeros(sizes[l + 1]) for l in range(len(sizes) - 1)]
    mean = np.zeros(N_FEAT) if mean is None else np.asarray(mean, dtype=np.float64)
    inv_std = np.ones(N_FEAT) if inv_std is None else np.asarray(inv_std, dtype=np.float64)
    return MLP(W, c, mean, inv_std)


def _w(W, bf16: bool):
    return lp.to_bf16(W) if bf16 else W


def forward(net: MLP, X: np.ndarray, bf16: bool = True):
    """X (batch x 256) -> predictions (batch), with the layer inputs and the
    pre-activations for the backward pass.  Weights rounded to bf16 (bf16 =
    False uses them exactly, for derivative checks)."""
    a = (np.asarray(X, dtype=np.float64) - net.mean) * net.inv_std
    acts, pres = [a], []
    L = len(net.W)
    for l in range(L):
        z = a @ _w(net.W[l], bf16).T + net.c[l]
        pres.append(z)
        a = gelu(z) if l < L - 1 else z
        acts.append(a)
    return a[:, 0], acts, pres


def loss(net: MLP, X, y, bf16: bool = True):
    pred, _, _ = forward(net, X, bf16)
    return np.mean((pred - np.asarray(y, dtype=np.float64)) ** 2)


def gradients(net: MLP, X, y, bf16: bool = True):
    """d loss / d (W, c) per layer (with respect to the bf16-rounded weights,
    used as the masters' gradients)."""
    pred, acts, pres = forward(net, X, bf16)
    B = pred.size
    L = len(net.W)
    g = (2.0 / B) * (pred - np.asarray(y, dtype=np.float64))[:, None]  # d loss / d z_last
    gW, gc = [None] * L, [None] * L
    for l in range(L - 1, -1, -1):
        gW[l] = g.T @ acts[l]
        gc[l] = g.sum(axis=0)
        if l > 0:
            g = (g @ _w(net.W[l], bf16)) * gelu_grad(pres[l - 1])
    return gW, gc


def adam_step(net: MLP, gW, gc, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update of every weight and bias (in place)."""
    if not net.m:
        net.m = [np.zeros_like(p) for p in net.params()]
        net.v = [np.zeros_like(p) for p in net.params()]
    net.t += 1
    grads = [a for l in range(len(net.W)) for a in (gW[l], gc[l])]
    params = net.params()
    for k, (p, gk) in enumerate(zip(params, grads)):
        net.m[k] = b1 * net.m[k] + (1.0 - b1) * gk
        net.v[k] = b2 * net.v[k] + (1.0 - b2) * gk * gk
        mh = net.m[k] / (1.0 - b1 ** net.t)
        vh = net.v[k] / (1.0 - b2 ** net.t)
        p -= lr * mh / (np.sqrt(vh) + eps)
