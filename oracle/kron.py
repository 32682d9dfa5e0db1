"""PSF -> Kronecker-sum blurring operator (oracle, FP64).

The blur of an n_r x n_c image X by a PSF P with 0-based centre (c_r, c_c) is
    B[i, j] = sum_{k, l} P[c_r + i - k, c_c + j - l] X_ext[k, l],
where X_ext extends X by zeros (zero boundary conditions) or by half-sample
symmetric reflection (reflexive boundary conditions).  Writing the PSF as a
sum of outer products P = sum_m u_m v_m^T makes the blur
    B = sum_m A_c^(m) X A_r^(m)^T,  i.e.  A = sum_m A_r^(m) (x) A_c^(m)
(Section 3: (C (x) D) vec(Y) = vec(D Y C^T); eq. KronSumDecomp, Section 5),
with A_c^(m) = F(u_m) (n_r x n_r, acts on columns) and A_r^(m) = F(v_m)
(n_c x n_c, acts on rows):
    zero BC       F(u) = T(u),          T(u)[i, j] = u[c + i - j]
    reflexive BC  F(u) = T(u) + H(u),   H(u)[i, j] = u[c + i + j + 1] + u[c + i + j + 1 - 2n]
(out-of-range indices contribute 0).

The terms come from the SVD of the weighted PSF D_c P D_r, D = diag(sqrt(w)),
w[k] = n - |k - c| (the number of times PSF row / column k appears in the
Toeplitz factor), so the first term is the Frobenius-optimal Kronecker
product (Section 5, the argmin below eq. KronSumDecomp); at full rank the sum
is exact for any weighting.  Sign convention: each u_m is flipped so that its
largest-magnitude entry is positive (v_m flips with it).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def kron_weights(n: int, c: int) -> np.ndarray:
    """w[k] = n - |k - c|: occurrences of PSF offset k - c in an n x n Toeplitz factor."""
    k = np.arange(n)
    return (n - np.abs(k - c)).astype(np.float64)


def psf_kron_terms(psf: np.ndarray, center, rank: int, weighted: bool = True):
    """Leading ``rank`` terms (u_m, v_m) of the PSF's weighted SVD.

    Returns (s, Uk, Vk): s the weighted singular values, Uk (n_r x r) the
    column-direction vectors u_m, Vk (n_c x r) the row-direction vectors v_m,
    with P ~= sum_m u_m v_m^T (exact at full rank)."""
    n_r, n_c = psf.shape
    c_r, c_c = center
    r = min(n_r, n_c) if rank in (0, None) else int(rank)
    if weighted:
        dc = np.sqrt(kron_weights(n_r, c_r))
        dr = np.sqrt(kron_weights(n_c, c_c))
    else:
        dc = np.ones(n_r)
        dr = np.ones(n_c)
    W = dc[:, None] * psf * dr[None, :]
    Ut, s, Vt = np.linalg.svd(W)
    Uk = np.empty((n_r, r))
    Vk = np.empty((n_c, r))
    for m in range(r):
        u = np.sqrt(s[m]) * Ut[:, m] / dc
        v = np.sqrt(s[m]) * Vt[m, :] / dr
        if u[np.argmax(np.abs(u))] < 0:
            u, v = -u, -v
        Uk[:, m] = u
        Vk[:, m] = v
    return s[:r], Uk, Vk


def _take(u: np.ndarray, k: np.ndarray) -> np.ndarray:
    """u[k] where 0 <= k < n, else 0."""
    n = u.shape[0]
    ok = (k >= 0) & (k < n)
    return np.where(ok, u[np.clip(k, 0, n - 1)], 0.0)


def toeplitz_factor(u: np.ndarray, c: int) -> np.ndarray:
    """T(u)[i, j] = u[c + i - j], zero outside 0 <= c + i - j < n."""
    n = u.shape[0]
    i, j = np.indices((n, n))
    return _take(u, c + i - j)


def hankel_factor(u: np.ndarray, c: int) -> np.ndarray:
    """H(u)[i, j] = u[c + i + j + 1] + u[c + i + j + 1 - 2n] (each term zero when
    its index is out of range): the reflections of the half-sample symmetric
    extension across the two image borders."""
    n = u.shape[0]
    i, j = np.indices((n, n))
    return _take(u, c + i + j + 1) + _take(u, c + i + j + 1 - 2 * n)


def blur_factor(u: np.ndarray, c: int, bc: str) -> np.ndarray:
    if bc == "zero":
        return toeplitz_factor(u, c)
    if bc == "reflexive":
        return toeplitz_factor(u, c) + hankel_factor(u, c)
    raise ValueError(f"unknown boundary condition {bc!r}")


@dataclass
class KronOperator:
    """A = sum_k A_r[k] (x) A_c[k] acting on n_r x n_c images."""
    Ac: list
    Ar: list
    s: np.ndarray
    u: np.ndarray
    v: np.ndarray
    bc: str

    @property
    def rank(self):
        return len(self.Ac)

    @property
    def shape(self):
        return self.Ac[0].shape[0], self.Ar[0].shape[0]


def kron_operator(psf: np.ndarray, center, bc: str, rank: int = 0,
                  weighted: bool = True) -> KronOperator:
    """Kronecker-sum operator of the blur (eq. KronSumDecomp)."""
    c_r, c_c = center
    s, Uk, Vk = psf_kron_terms(psf, center, rank, weighted)
    Ac = [blur_factor(Uk[:, m], c_r, bc) for m in range(Uk.shape[1])]
    Ar = [blur_factor(Vk[:, m], c_c, bc) for m in range(Vk.shape[1])]
    return KronOperator(Ac=Ac, Ar=Ar, s=s, u=Uk, v=Vk, bc=bc)


def apply_A(op: KronOperator, X: np.ndarray) -> np.ndarray:
    """A vec(X) = vec(sum_k A_c^(k) X A_r^(k)^T)."""
    out = np.zeros(X.shape)
    for Ac, Ar in zip(op.Ac, op.Ar):
        out += Ac @ X @ Ar.T
    return out


def apply_AT(op: KronOperator, Y: np.ndarray) -> np.ndarray:
    """A^T vec(Y) = vec(sum_k A_c^(k)^T Y A_r^(k))."""
    out = np.zeros(Y.shape)
    for Ac, Ar in zip(op.Ac, op.Ar):
        out += Ac.T @ Y @ Ar
    return out


def apply_K(op: KronOperator, X: np.ndarray, lam: float) -> np.ndarray:
    """(A^T A + lam^2 I) vec(X), the Tikhonov normal-equations matrix (eq. tik:normal2)."""
    return apply_AT(op, apply_A(op, X)) + lam * lam * X


def dense_A(op: KronOperator) -> np.ndarray:
    """Explicit N x N matrix sum_k A_r^(k) (x) A_c^(k) (small sizes only)."""
    n_r, n_c = op.shape
    A = np.zeros((n_r * n_c, n_r * n_c))
    for Ac, Ar in zip(op.Ac, op.Ar):
        A += np.kron(Ar, Ac)
    return A


def vec(X: np.ndarray) -> np.ndarray:
    """Column stacking (Section 3)."""
    return np.asarray(X).reshape(-1, order="F")


def unvec(x: np.ndarray, n_r: int, n_c: int) -> np.ndarray:
    return np.asarray(x).reshape((n_r, n_c), order="F")
