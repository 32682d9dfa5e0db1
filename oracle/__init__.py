"""FP64 CPU oracle for KP-SVD preconditioned Tikhonov deblurring
(Chen, Ji, Nagy, "Half-Precision Kronecker Product SVD Preconditioner for
Structured Inverse Problems", arXiv 2311.15393).

TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously correct NumPy/SciPy code in
float64, written from the paper's definitions.  Only the test-suite, the
smoke check and the CPU-baseline leg of the benchmark may import it; the CUDA
library shares no code with it and never calls it.

Modules
  kron      PSF -> Kronecker-sum operator A = sum_k A_r^(k) (x) A_c^(k)
            (Section 3 Kronecker identities; eq. KronSumDecomp, Section 5)
  kpsvd     KP-SVD of the first term and the preconditioner solve
            (eqs. AKronSVD, PreconSystem, PreconSolve)
  pcg       PCG / flexible PCG on the Tikhonov normal equations
            (eq. tik:normal2; Section 3 last paragraph; Section 5.2)
  lam       closed-form parameter choice over the KP spectrum
            (eqs. OptTikSVD, GCVTikSVD, wGCVTikSVD, DSCTikSVD)
  forward   observed data b = A x_true + e at a given noise level (Section 5)
  lowprec   rounding to bf16 / fp16 / e4m3 / fp32 and block-scaled FP8 for
            reduced-precision checks (Section 4 uses the same
            rounding-simulation idea)
  mlp       spectral features and the GELU MLP of the learned lambda, with
            its backward pass and Adam (not in the paper, which asks for a
            systematic parameter choice, Section 5)

Parity status: every function is pinned by a `-m "not gpu"` test against
closed forms, brute force, identities or hand-worked values
(tests/test_oracle_*.py); the rounding helpers in ``lowprec`` are pinned
against numpy's own float16/float32 casts and hand-worked values.
tests/test_oracle_planted_mistakes.py plants plausible mistakes in copies of
these modules and checks that a pin fails for each.
"""
from . import kron, kpsvd, pcg, lam, forward, lowprec, mlp  # noqa: F401
