"""Pins for the oracle's Kronecker-sum operator (oracle/kron.py).

Each check compares against something other than the oracle's own formulas:
the Kronecker identity through np.kron (Section 3), a brute-force 2-D
convolution of unit images with np.pad boundary extension, the Van Loan -
Pitsianis rank-1 optimum of the rearranged dense matrix (Section 5, argmin
below eq. KronSumDecomp), and the exact rank one of a separable PSF
(Table 1, Gauss row: one Kronecker term).
"""
import json
import os

import numpy as np
import pytest

from oracle import kron
from paper_2311_15393_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def direct_blur(X, P, center, bc):
    """B[i, j] = sum_{a,b} P[a, b] X_ext[i - (a - c_r), j - (b - c_c)] by brute force."""
    n_r, n_c = X.shape
    c_r, c_c = center
    mode = {"zero": "constant", "reflexive": "symmetric"}[bc]
    Xp = np.pad(X, ((n_r, n_r), (n_c, n_c)), mode=mode)
    B = np.zeros_like(X)
    for a in range(n_r):
        for b in range(n_c):
            s, t = a - c_r, b - c_c
            B += P[a, b] * Xp[n_r - s:2 * n_r - s, n_c - t:2 * n_c - t]
    return B


def dense_blur_matrix(P, center, bc):
    n_r, n_c = P.shape
    N = n_r * n_c
    A = np.zeros((N, N))
    for col in range(N):
        E = np.zeros(N)
        E[col] = 1.0
        A[:, col] = kron.vec(direct_blur(kron.unvec(E, n_r, n_c), P, center, bc))
    return A


def test_kronecker_identity_8x8():
    """(C (x) D) vec(Y) = vec(D Y C^T) on explicit 8 x 8 factors (Section 3)."""
    rng = np.random.default_rng(0)
    Ac = [rng.standard_normal((8, 8)) for _ in range(2)]
    Ar = [rng.standard_normal((8, 8)) for _ in range(2)]
    op = kron.KronOperator(Ac=Ac, Ar=Ar, s=None, u=None, v=None, bc="zero")
    X = rng.standard_normal((8, 8))
    dense = sum(np.kron(r, c) for r, c in zip(Ar, Ac))
    np.testing.assert_allclose(kron.vec(kron.apply_A(op, X)), dense @ kron.vec(X), rtol=0, atol=1e-12)
    np.testing.assert_allclose(kron.vec(kron.apply_AT(op, X)), dense.T @ kron.vec(X), rtol=0, atol=1e-12)
    # vec is column stacking
    assert np.array_equal(kron.vec(np.array([[1, 2], [3, 4]])), np.array([1, 3, 2, 4]))


@pytest.mark.parametrize("bc", ["zero", "reflexive"])
@pytest.mark.parametrize("n_r,n_c,center", [(8, 8, (4, 4)), (12, 10, (5, 3)), (16, 16, (8, 8))])
def test_full_rank_sum_equals_direct_convolution(bc, n_r, n_c, center):
    """At full rank the Kronecker sum equals the blur itself, for both BCs and
    off-centre / rectangular grids."""
    P = synth.gaussian_psf(n_r, n_c, center[0], center[1], 2.0, 1.3, 0.55)
    op = kron.kron_operator(P, center, bc, rank=0)
    A_direct = dense_blur_matrix(P, center, bc)
    A_kron = kron.dense_A(op)
    assert np.max(np.abs(A_kron - A_direct)) <= 1e-14 * np.max(np.abs(A_direct)) * 16


@pytest.mark.parametrize("bc", ["zero", "reflexive"])
def test_truncation_error_decreases(bc):
    P = synth.gaussian_psf(12, 12, 6, 6, 2.0, 1.5, 0.6)
    A_direct = dense_blur_matrix(P, (6, 6), bc)
    errs = []
    for r in range(1, 7):
        op = kron.kron_operator(P, (6, 6), bc, rank=r)
        errs.append(np.linalg.norm(kron.dense_A(op) - A_direct))
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:]))


def test_weighted_first_term_is_van_loan_pitsianis_optimum():
    """Zero BC: the weighted first term attains min ||A - A_r (x) A_c||_F over
    all Kronecker products, computed by the SVD of the rearranged dense A."""
    n = 8
    P = synth.gaussian_psf(n, n, 4, 4, 1.8, 1.1, 0.6)
    A = dense_blur_matrix(P, (4, 4), "zero")
    # rearrangement: row (j, l) = vec of block (j, l)
    R = np.empty((n * n, n * n))
    for j in range(n):
        for l in range(n):
            R[j * n + l] = A[j * n:(j + 1) * n, l * n:(l + 1) * n].reshape(-1, order="F")
    s = np.linalg.svd(R, compute_uv=False)
    best = np.sqrt(np.sum(s[1:] ** 2))
    op = kron.kron_operator(P, (4, 4), "zero", rank=1)
    ours = np.linalg.norm(A - kron.dense_A(op))
    assert abs(ours - best) <= 1e-10 * np.linalg.norm(A)
    # the unweighted truncation is no better (and in general worse)
    op_u = kron.kron_operator(P, (4, 4), "zero", rank=1, weighted=False)
    assert np.linalg.norm(A - kron.dense_A(op_u)) >= best - 1e-12


def test_separable_psf_is_one_kronecker_term():
    """Table 1 (Gauss row): a separable Gaussian blur is exactly one term."""
    with open(os.path.join(GOLDEN, "paper_claims.json")) as f:
        claims = json.load(f)
    assert claims["table1_gauss_terms"]["value"] == 1
    P = synth.separable_psf(32, 32, 16, 16, 3.0, 1.5)
    s, U, V = kron.psf_kron_terms(P, (16, 16), rank=0)
    assert s[1] / s[0] < 1e-14
    op1 = kron.kron_operator(P, (16, 16), "zero", rank=1)
    opf = kron.kron_operator(P, (16, 16), "zero", rank=0)
    X = synth.phantom(32, 32, 5, np.random.default_rng(3))
    np.testing.assert_allclose(kron.apply_A(op1, X), kron.apply_A(opf, X), rtol=0, atol=1e-13)


def test_sign_convention_and_exact_sum():
    """Each u_m has a positive largest entry; the full sum of outer products is the PSF."""
    P = synth.gaussian_psf(16, 16, 8, 8, 2.0, 1.0, 0.5)
    s, U, V = kron.psf_kron_terms(P, (8, 8), rank=0)
    for m in range(U.shape[1]):
        assert U[np.argmax(np.abs(U[:, m])), m] > 0
    np.testing.assert_allclose(U @ V.T, P, rtol=0, atol=1e-15)
