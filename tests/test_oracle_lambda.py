"""Pins for the oracle's closed-form parameter choice (oracle/lam.py).

The closed forms over the KP spectrum (eqs. GCVTikSVD, wGCVTikSVD,
DSCTikSVD, OptTikSVD) are checked against their matrix definitions
(eqs. GCVTik, wGCVTik, DSCTik, OptTik) evaluated with dense matrices on a
separable blur, where the KP-SVD is the exact SVD of A; the minimisers are
checked against an exhaustive 10^4-point grid.
"""
import numpy as np
import pytest

from oracle import forward, kpsvd, kron, lam
from paper_2311_15393_gb300 import synth


def separable_problem():
    """12 x 12 separable blur (reflexive BC), 2% noise: the KP-SVD is the exact SVD of A."""
    n = 12
    P = synth.separable_psf(n, n, 6, 6, 1.6, 1.1)
    rng = np.random.default_rng(11)
    X = synth.phantom(n, n, 4, rng)
    op = kron.kron_operator(P, (6, 6), "reflexive", rank=1)
    kp = kpsvd.kp_svd(op, "projected")
    B, enorm = forward.observe(op, X, synth.noise_direction(n, n, rng), 0.02)
    A = kron.dense_A(op)
    return op, kp, A, B, X, enorm


@pytest.fixture(scope="module")
def separable():
    return separable_problem()


def _influence(A, l):
    """A A_lam^+ with A_lam^+ = (A^T A + lam^2 I)^-1 A^T (Section 2.2)."""
    return A @ np.linalg.solve(A.T @ A + l * l * np.eye(A.shape[1]), A.T)


@pytest.mark.parametrize("l", [1e-3, 1e-2, 0.1, 0.5])
def test_gcv_closed_form_matches_trace_definition(separable, l):
    op, kp, A, B, X, _ = separable
    b = kron.vec(B)
    N = b.size
    I_AA = np.eye(N) - _influence(A, l)
    G_def = N * np.linalg.norm(I_AA @ b) ** 2 / np.trace(I_AA) ** 2
    Bh = lam.spectral_coeffs(kp, B)
    assert abs(lam.gcv(kp.Sigma, Bh, l) - G_def) <= 1e-9 * G_def


@pytest.mark.parametrize("omega", [0.5, 1.0, 3.0])
@pytest.mark.parametrize("l", [1e-2, 0.1, 0.5])
def test_wgcv_closed_form_matches_trace_definition(separable, omega, l):
    op, kp, A, B, X, _ = separable
    b = kron.vec(B)
    N = b.size
    H = _influence(A, l)
    G_def = N * np.linalg.norm(b - H @ b) ** 2 / np.trace(np.eye(N) - omega * H) ** 2
    Bh = lam.spectral_coeffs(kp, B)
    assert abs(lam.wgcv(kp.Sigma, Bh, l, omega) - G_def) <= 1e-8 * G_def
    if omega == 1.0:
        assert abs(lam.gcv(kp.Sigma, Bh, l) - G_def) <= 1e-9 * G_def


@pytest.mark.parametrize("l", [1e-3, 3e-2, 0.3])
def test_discrepancy_and_opt_match_residual_definitions(separable, l):
    op, kp, A, B, X, enorm = separable
    b, x = kron.vec(B), kron.vec(X)
    x_l = np.linalg.solve(A.T @ A + l * l * np.eye(A.shape[1]), A.T @ b)
    eps = 1.01 * enorm
    D_def = np.linalg.norm(A @ x_l - b) ** 2 - eps ** 2
    Bh = lam.spectral_coeffs(kp, B)
    assert abs(lam.discrepancy(kp.Sigma, Bh, l, eps) - D_def) <= 1e-10 * np.linalg.norm(b) ** 2
    O_def = np.linalg.norm(x_l - x) ** 2
    Xh = lam.solution_coeffs(kp, X)
    assert abs(lam.opt_error(kp.Sigma, Bh, Xh, l) - O_def) <= 1e-9 * O_def


@pytest.mark.parametrize("method", ["gcv", "wgcv", "opt"])
def test_minimisers_match_exhaustive_grid(separable, method):
    op, kp, A, B, X, _ = separable
    param = 3.0 if method == "wgcv" else 0.0
    l_star = lam.choose_lambda(kp, B, method, param, X_true=X)
    Bh = lam.spectral_coeffs(kp, B)
    Xh = lam.solution_coeffs(kp, X)
    lo, hi = lam.lambda_bounds(kp.Sigma)
    if method == "wgcv":
        lo = lam.wgcv_lower_limit(kp.Sigma, param, lo, hi)
    f = {"gcv": lambda l: lam.gcv(kp.Sigma, Bh, l),
         "wgcv": lambda l: lam.wgcv(kp.Sigma, Bh, l, param),
         "opt": lambda l: lam.opt_error(kp.Sigma, Bh, Xh, l)}[method]
    grid = np.exp(np.linspace(np.log(lo), np.log(hi), 10_000))
    vals = np.array([f(g) for g in grid])
    assert f(l_star) <= vals.min() * (1 + 1e-12)
    assert abs(np.log(l_star) - np.log(grid[np.argmin(vals)])) <= 2 * np.log(hi / lo) / 10_000


def test_lambda_search_bounds_by_hand():
    """The search runs between the smallest nonzero |sigma| and the largest
    (Section 2.2), the lower end floored at 1e-10 sigma_max; PROJECTED
    spectra may hold negative entries, which count by magnitude."""
    assert lam.lambda_bounds(np.array([[0.5, 0.01], [-1.0, 0.0]])) == (0.01, 1.0)
    assert lam.lambda_bounds(np.array([1e-12, 0.0, 1e-3, 2.0])) == (2e-10, 2.0)


def test_discrepancy_root_and_no_root(separable):
    op, kp, A, B, X, enorm = separable
    eps = 1.01 * enorm
    l = lam.choose_lambda(kp, B, "discrepancy", eps)
    Bh = lam.spectral_coeffs(kp, B)
    assert abs(lam.discrepancy(kp.Sigma, Bh, l, eps)) <= 1e-10 * eps * eps
    assert lam.choose_lambda(kp, B, "discrepancy", 1.01 * np.linalg.norm(B)) is None


def test_wgcv_spurious_minimum_is_excluded(separable):
    """For omega > 1 the unrestricted G_w falls to 0 as lam -> 0; the search
    keeps to the range where trace(I - omega A A^+) > 0."""
    op, kp, A, B, X, _ = separable
    Bh = lam.spectral_coeffs(kp, B)
    lo, hi = lam.lambda_bounds(kp.Sigma)
    assert lam.wgcv_trace(kp.Sigma, lo, 3.0) < 0
    l0 = lam.wgcv_lower_limit(kp.Sigma, 3.0, lo, hi)
    assert lam.wgcv_trace(kp.Sigma, l0 * 1.0001, 3.0) > 0
    assert lam.choose_lambda(kp, B, "wgcv", 3.0) > l0


def test_discrepancy_lambda_increases_with_eta(separable):
    """eq. DSCTikSVD's residual norm increases with lambda, so the root for
    eps = eta ||e|| increases with the safety factor eta (the eta sweeps of
    Section 5.1), and at each root the residual norm equals eps."""
    op, kp, A, B, X, enorm = separable
    b = kron.vec(B)
    lams = [lam.choose_lambda(kp, B, "discrepancy", eta * enorm) for eta in (0.9, 1.0, 1.01, 1.1, 1.5)]
    assert all(a < c for a, c in zip(lams, lams[1:]))
    for eta, l in zip((0.9, 1.0, 1.01, 1.1, 1.5), lams):
        x = np.linalg.solve(A.T @ A + l * l * np.eye(A.shape[1]), A.T @ b)
        assert np.linalg.norm(A @ x - b) == pytest.approx(eta * enorm, rel=1e-8)


def test_wgcv_with_omega_one_is_gcv(separable):
    """wGCV's denominator N - omega tr(A A_lam^+) is GCV's at omega = 1 (eqs.
    wGCVTik, GCVTik), so both choose the same lambda."""
    op, kp, A, B, X, _ = separable
    assert lam.choose_lambda(kp, B, "wgcv", 1.0) == pytest.approx(lam.choose_lambda(kp, B, "gcv"), rel=1e-8)
