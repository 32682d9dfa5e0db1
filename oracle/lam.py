"""Regularisation-parameter choice in closed form over the KP spectrum (oracle).

With A ~= U Sigma V^T (here the KP-SVD), b_hat = U^T b = vec(U_c^T B U_r),
x_hat = V^T x_true = vec(V_c^T X_true V_r), and d_i = sigma_i^2 + lam^2:
  O(lam)   = sum (sigma_i b_hat_i / d_i - x_hat_i)^2                  (eq. OptTikSVD)
  G(lam)   = N sum (b_hat_i / d_i)^2 / (sum 1 / d_i)^2                (eq. GCVTikSVD)
  G_w(lam) = N sum (lam^2 b_hat_i / d_i)^2
             / (sum ((1 - w) sigma_i^2 + lam^2) / d_i)^2              (eq. wGCVTikSVD)
  D(lam)   = sum (lam^2 b_hat_i / d_i)^2 - eps^2                      (eq. DSCTikSVD)
Minimisers are searched on lam in [sigma_lo, sigma_max] (the paper bounds the
search by the smallest and largest singular values, Section 2.2), with
sigma_lo = max(min |Sigma| > 0, 1e-10 * max |Sigma|): a 400-point grid in
log lam, then a bounded scalar minimisation in log lam over the two grid cells
around the best grid point (ties go to the larger lam).  For wGCV with
omega > 1 the search starts above the root of trace(I - omega A A_lam^+),
where G_w is finite and meaningful (below it the trace is negative and G_w
falls to a spurious minimum at lam -> 0).  The discrepancy
equation D(lam) = 0 (D increases with lam) is solved by bracketing in log lam
and Brent's root finder (the paper uses an unbounded root finder); it has no
root when eps >= ||b_hat||, or when D stays positive down to 1e-16 sigma_max.
"""
from __future__ import annotations

import numpy as np

from .kpsvd import KPSVD

N_GRID = 400


def spectral_coeffs(kp: KPSVD, B: np.ndarray) -> np.ndarray:
    """b_hat as an n_r x n_c array: U_c^T B U_r = unvec((U_r (x) U_c)^T vec(B))."""
    return kp.Uc.T @ B @ kp.Ur


def solution_coeffs(kp: KPSVD, X: np.ndarray) -> np.ndarray:
    """x_hat = V_c^T X V_r."""
    return kp.Vc.T @ X @ kp.Vr


def gcv(Sigma, Bhat, lam):
    d = Sigma * Sigma + lam * lam
    return Sigma.size * np.sum((Bhat / d) ** 2) / np.sum(1.0 / d) ** 2


def wgcv(Sigma, Bhat, lam, omega):
    s2 = Sigma * Sigma
    d = s2 + lam * lam
    num = Sigma.size * np.sum((lam * lam * Bhat / d) ** 2)
    den = np.sum(((1.0 - omega) * s2 + lam * lam) / d) ** 2
    return num / den


def discrepancy(Sigma, Bhat, lam, eps):
    d = Sigma * Sigma + lam * lam
    return np.sum((lam * lam * Bhat / d) ** 2) - eps * eps


def opt_error(Sigma, Bhat, Xhat, lam):
    d = Sigma * Sigma + lam * lam
    return np.sum((Sigma * Bhat / d - Xhat) ** 2)


def wgcv_trace(Sigma, lam, omega):
    """trace(I - omega A A_lam^+) = sum ((1 - omega) sigma^2 + lam^2) / (sigma^2 + lam^2)."""
    s2 = Sigma * Sigma
    return np.sum(((1.0 - omega) * s2 + lam * lam) / (s2 + lam * lam))


def wgcv_lower_limit(Sigma, omega, lo, hi):
    """For omega > 1 the weighted trace is negative at small lam (it tends to
    N (1 - omega)) while the numerator tends to 0, so G_w has a spurious
    minimum at lam -> 0.  The search keeps to lam where the trace is
    positive: returns the root of the trace in [lo, hi] (bisection in
    log lam), or lo when the trace is already positive there."""
    if omega <= 1.0 or wgcv_trace(Sigma, lo, omega) > 0:
        return lo
    a, b = np.log(lo), np.log(hi)
    if wgcv_trace(Sigma, hi, omega) <= 0:
        return hi
    for _ in range(200):
        m = 0.5 * (a + b)
        if wgcv_trace(Sigma, np.exp(m), omega) > 0:
            b = m
        else:
            a = m
    return float(np.exp(b))


def lambda_bounds(Sigma):
    a = np.abs(Sigma)
    smax = float(a.max())
    pos = a[a > 0]
    smin = float(pos.min()) if pos.size else smax
    return max(smin, 1e-10 * smax), smax


def minimize_log(f, lo: float, hi: float, n_grid: int = N_GRID):
    """Global grid in log lam, then bounded Brent in the best cell."""
    from scipy.optimize import minimize_scalar
    t = np.linspace(np.log(lo), np.log(hi), n_grid)
    vals = np.array([f(np.exp(tt)) for tt in t])
    k = n_grid - 1 - int(np.argmin(vals[::-1]))      # ties -> larger lam
    a, b = t[max(k - 1, 0)], t[min(k + 1, n_grid - 1)]
    res = minimize_scalar(lambda tt: f(np.exp(tt)), bounds=(a, b), method="bounded",
                          options={"xatol": 1e-12, "maxiter": 500})
    if res.fun <= vals[k]:
        return float(np.exp(res.x))
    return float(np.exp(t[k]))


def root_discrepancy(Sigma, Bhat, eps: float):
    """lam with D(lam) = 0, or None when no root exists.  The bracket starts
    at [sigma_lo, sigma_max] and widens by decades (down to 1e-16 sigma_max,
    up until D > 0) before Brent's method runs in log lam."""
    from scipy.optimize import brentq
    lo, hi = lambda_bounds(Sigma)
    if np.sum(Bhat * Bhat) <= eps * eps:
        return None
    D = lambda tt: discrepancy(Sigma, Bhat, np.exp(tt), eps)  # noqa: E731
    tl, th = np.log(lo), np.log(hi)
    t_floor = np.log(1e-16 * hi)
    while D(tl) > 0:
        tl -= np.log(10.0)
        if tl < t_floor:
            return None
    for _ in range(64):
        if D(th) > 0:
            break
        th += np.log(10.0)
    else:
        return None
    return float(np.exp(brentq(D, tl, th, xtol=1e-15, rtol=4 * np.finfo(float).eps, maxiter=500)))


def choose_lambda(kp: KPSVD, B: np.ndarray, method: str, param: float = 0.0,
                  X_true: np.ndarray | None = None):
    """method in {"gcv", "wgcv", "discrepancy", "opt"}; param = omega (wgcv) or
    eps = eta * ||e|| (discrepancy)."""
    Sigma = kp.Sigma
    Bhat = spectral_coeffs(kp, B)
    lo, hi = lambda_bounds(Sigma)
    if method == "gcv":
        return minimize_log(lambda l: gcv(Sigma, Bhat, l), lo, hi)
    if method == "wgcv":
        lo = max(lo, wgcv_lower_limit(Sigma, param, lo, hi))
        return minimize_log(lambda l: wgcv(Sigma, Bhat, l, param), lo, hi)
    if method == "opt":
        Xhat = solution_coeffs(kp, X_true)
        return minimize_log(lambda l: opt_error(Sigma, Bhat, Xhat, l), lo, hi)
    if method == "discrepancy":
        return root_discrepancy(Sigma, Bhat, param)
    raise ValueError(method)
