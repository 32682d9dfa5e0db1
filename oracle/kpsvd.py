"""KP-SVD of the first Kronecker term and the preconditioner solve (oracle, FP64).

eq. AKronSVD (Section 3):  A ~= A_r (x) A_c = (U_r (x) U_c)(Sigma_r (x) Sigma_c)(V_r (x) V_c)^T
with A_r = A_r^(1) = U_r Sigma_r V_r^T and A_c = A_c^(1) = U_c Sigma_c V_c^T.
The KP spectrum, stored as an n_r x n_c array (vec order i + n_r j), is
  PRODUCT    Sigma[i, j] = sigma_c[i] * sigma_r[j]                    (eq. AKronSVD)
  PROJECTED  Sigma = diag((U_r (x) U_c)^T A (V_r (x) V_c))
             = sum_k diag(U_c^T A_c^(k) V_c)[i] * diag(U_r^T A_r^(k) V_r)[j]
             (the diagonal of the full operator in the KP basis; equal to
             PRODUCT when A has one term).
eq. PreconSystem (Section 2.3): M = V (Sigma^T Sigma + lam^2 I) V^T, z = V D^-1 V^T r.
eq. PreconSolve (Section 3):   Z = V_c (S .* (V_c^T R V_r)) V_r^T, vec(S) = diag(D^-1).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .kron import KronOperator


@dataclass
class KPSVD:
    Ur: np.ndarray
    sr: np.ndarray
    Vr: np.ndarray
    Uc: np.ndarray
    sc: np.ndarray
    Vc: np.ndarray
    Sigma: np.ndarray   # n_r x n_c KP spectrum


def kp_svd(op: KronOperator, sigma_mode: str = "projected") -> KPSVD:
    """Factor SVDs of the first Kronecker term and the KP spectrum."""
    Ur, sr, Vrt = np.linalg.svd(op.Ar[0])
    Uc, sc, Vct = np.linalg.svd(op.Ac[0])
    Vr, Vc = Vrt.T, Vct.T
    if sigma_mode == "product":
        Sigma = np.outer(sc, sr)
    elif sigma_mode == "projected":
        Sigma = np.zeros((sc.shape[0], sr.shape[0]))
        for Ac, Ar in zip(op.Ac, op.Ar):
            dc = np.diag(Uc.T @ Ac @ Vc)
            dr = np.diag(Ur.T @ Ar @ Vr)
            Sigma += np.outer(dc, dr)
    else:
        raise ValueError(sigma_mode)
    return KPSVD(Ur=Ur, sr=sr, Vr=Vr, Uc=Uc, sc=sc, Vc=Vc, Sigma=Sigma)


def precond_scale(Sigma: np.ndarray, lam: float) -> np.ndarray:
    """S = 1 / (Sigma^2 + lam^2), i.e. vec(S) = diag(D^-1) (eq. PreconSolve)."""
    return 1.0 / (Sigma * Sigma + lam * lam)


def precond_apply(kp: KPSVD, S: np.ndarray, R: np.ndarray) -> np.ndarray:
    """Z = V_c (S .* (V_c^T R V_r)) V_r^T (eq. PreconSolve)."""
    return kp.Vc @ (S * (kp.Vc.T @ R @ kp.Vr)) @ kp.Vr.T


def dense_M(kp: KPSVD, lam: float) -> np.ndarray:
    """Explicit M = (V_r (x) V_c) diag(vec(Sigma)^2 + lam^2) (V_r (x) V_c)^T (small sizes)."""
    V = np.kron(kp.Vr, kp.Vc)
    d = kp.Sigma.reshape(-1, order="F") ** 2 + lam * lam
    return V @ np.diag(d) @ V.T
