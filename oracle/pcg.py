"""Preconditioned CG and flexible PCG on the Tikhonov normal equations
(A^T A + lam^2 I) x = A^T b (eq. tik:normal2), oracle in FP64.

Iteration (x_0 = 0 unless a warm start is given, r_0 = A^T b - K x_0,
z_0 = M^-1 r_0, p_0 = z_0), each step one application of K = A^T A + lam^2 I:
    q = K p;  alpha = z^T r / p^T q;  x += alpha p;  r_new = r - alpha q
    stop when ||r_new|| / ||A^T b|| <= tol or the iteration count reaches maxit
    z_new = M^-1 r_new
    beta = z_new^T r_new / z^T r                (PCG, Fletcher-Reeves form)
    beta = z_new^T (r_new - r) / z^T r          (flexible PCG, Polak-Ribiere form;
                                                 Section 3, last paragraph)
    p = z_new + beta p
The residual is the recurred residual of the normal equations.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import kron, kpsvd


@dataclass
class PCGInfo:
    iters: int = 0
    converged: bool = False
    res_hist: list = field(default_factory=list)   # ||r_k|| / ||A^T b||, k = 0..iters


def pcg(apply_K, apply_Minv, rhs: np.ndarray, tol: float, maxit: int,
        flexible: bool = False, x0: np.ndarray | None = None, callback=None):
    """Generic PCG / FPCG on arrays of any shape (inner products over all entries)."""
    x = np.zeros_like(rhs) if x0 is None else x0.copy()
    r = rhs - apply_K(x) if x0 is not None else rhs.copy()
    rhs_norm = np.linalg.norm(rhs)
    info = PCGInfo()
    info.res_hist.append(np.linalg.norm(r) / rhs_norm if rhs_norm > 0 else 0.0)
    if rhs_norm == 0.0:
        info.converged = True
        return x, info
    z = apply_Minv(r)
    p = z.copy()
    zr = np.vdot(z, r)
    for it in range(1, maxit + 1):
        q = apply_K(p)
        alpha = zr / np.vdot(p, q)
        x = x + alpha * p
        r_new = r - alpha * q
        rel = np.linalg.norm(r_new) / rhs_norm
        info.res_hist.append(rel)
        info.iters = it
        if callback is not None:
            callback(it, x)
        if rel <= tol:
            info.converged = True
            break
        if it == maxit:
            break
        z_new = apply_Minv(r_new)
        zr_new = np.vdot(z_new, r_new)
        if flexible:
            beta = np.vdot(z_new, r_new - r) / zr
        else:
            beta = zr_new / zr
        p = z_new + beta * p
        r, z, zr = r_new, z_new, zr_new
    return x, info


def tik_pcg(op: kron.KronOperator, kp: kpsvd.KPSVD | None, B: np.ndarray, lam: float,
            tol: float, maxit: int, flexible: bool = False, X0=None, callback=None, lam_pc: float | None = None):
    """KP-SVD preconditioned (F)PCG for the deblurring problem; kp=None gives plain CG.
    lam_pc: the preconditioner's lambda (default: the system's, eq. PreconSystem;
    Section 5.3 suggests a larger one against the early error jump)."""
    rhs = kron.apply_AT(op, B)
    if kp is not None:
        S = kpsvd.precond_scale(kp.Sigma, lam if lam_pc is None else lam_pc)
        minv = lambda R: kpsvd.precond_apply(kp, S, R)  # noqa: E731
    else:
        minv = lambda R: R.copy()  # noqa: E731
    return pcg(lambda X: kron.apply_K(op, X, lam), minv, rhs, tol, maxit, flexible,
               x0=X0, callback=callback)


def tik_exact_dense(op: kron.KronOperator, B: np.ndarray, lam: float) -> np.ndarray:
    """x_lam = (A^T A + lam^2 I)^-1 A^T b by a dense Cholesky solve (small N)."""
    import scipy.linalg as sla
    n_r, n_c = op.shape
    A = kron.dense_A(op)
    K = A.T @ A + lam * lam * np.eye(A.shape[1])
    rhs = A.T @ kron.vec(B)
    c = sla.cho_factor(K, lower=True)
    return kron.unvec(sla.cho_solve(c, rhs), n_r, n_c)


def tik_exact(op: kron.KronOperator, kp: kpsvd.KPSVD, B: np.ndarray, lam: float,
              tol: float = 1e-13, maxit: int = 2000) -> np.ndarray:
    """x_lam: dense Cholesky when N <= 4096, otherwise FP64 PCG to ``tol``."""
    n_r, n_c = op.shape
    if n_r * n_c <= 4096:
        return tik_exact_dense(op, B, lam)
    x, info = tik_pcg(op, kp, B, lam, tol, maxit, flexible=False)
    if not info.converged:
        raise RuntimeError("oracle PCG did not reach the reference tolerance")
    return x


def multiterm_minv(op: kron.KronOperator, kp: kpsvd.KPSVD, lam: float, k: int, inner_iters: int,
                   inner_tol: float = 0.0):
    """Preconditioner from the first k Kronecker terms of A (scope-table NEXT 3;
    Section 5.3 finds the one-term preconditioner of no use for some blurs with
    many terms): z ~ (M_k^T M_k + lam^2 I)^-1 r with M_k = sum_{j<k} A_r^(j) (x)
    A_c^(j).  For k > 1 no single KP-SVD diagonalises M_k^T M_k, so z comes from
    `inner_iters` PCG steps on it, preconditioned by the one-term KP-SVD solve
    (eq. PreconSolve), from z = 0.  The result varies with r (an inexact inner
    solve), hence flexible PCG outside."""
    opk = kron.KronOperator(Ac=op.Ac[:k], Ar=op.Ar[:k], s=op.s[:k], u=op.u[:, :k], v=op.v[:, :k], bc=op.bc)
    S = kpsvd.precond_scale(kp.Sigma, lam)

    def minv(R):
        z, _ = pcg(lambda X: kron.apply_K(opk, X, lam), lambda Q: kpsvd.precond_apply(kp, S, Q), R,
                   inner_tol, inner_iters, flexible=False)
        return z

    return minv


def tik_fpcg_multiterm(op: kron.KronOperator, kp: kpsvd.KPSVD, B: np.ndarray, lam: float, k: int,
                       inner_iters: int, tol: float, maxit: int, inner_tol: float = 0.0, callback=None):
    """Flexible PCG on the Tikhonov normal equations with multiterm_minv."""
    rhs = kron.apply_AT(op, B)
    return pcg(lambda X: kron.apply_K(op, X, lam), multiterm_minv(op, kp, lam, k, inner_iters, inner_tol), rhs, tol,
               maxit, flexible=True, callback=callback)
