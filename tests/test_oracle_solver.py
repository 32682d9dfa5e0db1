"""Pins for the oracle's KP-SVD, preconditioner and PCG / FPCG
(oracle/kpsvd.py, oracle/pcg.py, oracle/forward.py).

References used instead of the oracle's own formulas: dense np.kron
matrices and np.linalg.solve / svd; the closed form that a separable PSF
with zero BC makes the preconditioner exact so PCG stops after one iteration
with alpha = 1; a dense Cholesky solve at 16 x 16; the SVD filter-factor
formula (eq. TikSV); CG orthogonality invariants.
"""
import numpy as np
import pytest

from oracle import forward, kpsvd, kron, pcg
from paper_2311_15393_gb300 import synth


def _problem(n=16, bc="reflexive", rank=3, rho=0.6, seed=5):
    P = synth.gaussian_psf(n, n, n // 2, n // 2, 2.0, 1.2, rho)
    rng = np.random.default_rng(seed)
    X = synth.phantom(n, n, 4, rng)
    op = kron.kron_operator(P, (n // 2, n // 2), bc, rank)
    B, _ = forward.observe(op, X, synth.noise_direction(n, n, rng), 0.01)
    return op, X, B


def test_kp_svd_of_separable_psf_matches_dense_svd():
    """Separable PSF: sorted Sigma_r (x) Sigma_c equals the singular values of dense A."""
    P = synth.separable_psf(12, 12, 6, 6, 2.0, 1.0)
    op = kron.kron_operator(P, (6, 6), "zero", rank=1)
    kp = kpsvd.kp_svd(op, "product")
    s_dense = np.linalg.svd(kron.dense_A(op), compute_uv=False)
    np.testing.assert_allclose(np.sort(kp.Sigma.ravel())[::-1], s_dense, rtol=0, atol=1e-13)


@pytest.mark.parametrize("bc", ["zero", "reflexive"])
def test_projected_sigma_is_diag_in_kp_basis(bc):
    """PROJECTED Sigma = diag((U_r (x) U_c)^T A (V_r (x) V_c)) with every matrix dense."""
    op, _, _ = _problem(n=8, bc=bc, rank=3)
    kp = kpsvd.kp_svd(op, "projected")
    U = np.kron(kp.Ur, kp.Uc)
    V = np.kron(kp.Vr, kp.Vc)
    d = np.diag(U.T @ kron.dense_A(op) @ V)
    np.testing.assert_allclose(kron.vec(kp.Sigma), d, rtol=0, atol=1e-13)
    kp1 = kpsvd.kp_svd(kron.KronOperator(op.Ac[:1], op.Ar[:1], None, None, None, bc), "projected")
    np.testing.assert_allclose(kp1.Sigma, np.outer(kp.sc, kp.sr), rtol=0, atol=1e-13)


def test_preconditioner_solve_matches_dense_solve():
    """eq. PreconSolve vs a dense solve with M = A1^T A1 + lam^2 I, A1 = A_r^(1) (x) A_c^(1)."""
    op, _, _ = _problem(n=16, bc="reflexive", rank=2)
    kp = kpsvd.kp_svd(op, "product")
    lam = 0.03
    A1 = np.kron(op.Ar[0], op.Ac[0])
    M = A1.T @ A1 + lam * lam * np.eye(A1.shape[0])
    R = np.random.default_rng(1).standard_normal((16, 16))
    Z = kpsvd.precond_apply(kp, kpsvd.precond_scale(kp.Sigma, lam), R)
    z_ref = np.linalg.solve(M, kron.vec(R))
    assert np.linalg.norm(kron.vec(Z) - z_ref) <= 1e-10 * np.linalg.norm(z_ref)
    # eq. PreconSystem's explicit M is the same matrix for the PRODUCT spectrum
    np.testing.assert_allclose(kpsvd.dense_M(kp, lam), M, rtol=0, atol=1e-12 * np.abs(M).max())


def test_separable_zero_bc_pcg_converges_in_one_iteration():
    """Separable PSF + zero BC => M = K exactly, alpha = 1, x_1 = x_lam (closed form)."""
    n = 16
    P = synth.separable_psf(n, n, 8, 8, 2.5, 1.5)
    rng = np.random.default_rng(2)
    X = synth.phantom(n, n, 4, rng)
    op = kron.kron_operator(P, (8, 8), "zero", rank=1)
    kp = kpsvd.kp_svd(op, "projected")
    B, _ = forward.observe(op, X, synth.noise_direction(n, n, rng), 0.01)
    lam = 0.02
    x_star = pcg.tik_exact_dense(op, B, lam)
    x1, info = pcg.tik_pcg(op, kp, B, lam, tol=0.0, maxit=1)
    assert np.linalg.norm(x1 - x_star) <= 1e-9 * np.linalg.norm(x_star)
    # alpha = z0^T r0 / p0^T K p0 = 1
    rhs = kron.apply_AT(op, B)
    z0 = kpsvd.precond_apply(kp, kpsvd.precond_scale(kp.Sigma, lam), rhs)
    alpha = np.vdot(z0, rhs) / np.vdot(z0, kron.apply_K(op, z0, lam))
    assert abs(alpha - 1.0) < 1e-10


@pytest.mark.parametrize("bc", ["zero", "reflexive"])
@pytest.mark.parametrize("flexible", [False, True])
def test_pcg_converges_to_dense_cholesky(bc, flexible):
    """Converged (F)PCG equals a dense Cholesky solve at 16 x 16."""
    op, _, B = _problem(n=16, bc=bc, rank=3)
    kp = kpsvd.kp_svd(op, "projected")
    lam = 0.05
    x_star = pcg.tik_exact_dense(op, B, lam)
    x, info = pcg.tik_pcg(op, kp, B, lam, tol=1e-14, maxit=300, flexible=flexible)
    assert np.linalg.norm(x - x_star) <= 1e-11 * np.linalg.norm(x_star)


def test_filter_factor_solution_equals_cholesky():
    """eq. TikSV with the explicit dense SVD of A equals the normal-equations solve."""
    op, _, B = _problem(n=12, bc="zero", rank=4)
    lam = 0.04
    A = kron.dense_A(op)
    U, s, Vt = np.linalg.svd(A)
    phi = s ** 2 / (s ** 2 + lam ** 2)
    x_svd = Vt.T @ (phi * (U.T @ kron.vec(B)) / s)
    np.testing.assert_allclose(x_svd, kron.vec(pcg.tik_exact_dense(op, B, lam)), rtol=0, atol=1e-10)


def test_pcg_invariants():
    """r_k^T z_j = 0 (j < k), p_k^T K p_j = 0 (j < k), recurred residual = true
    residual, K-norm error decreasing."""
    op, _, B = _problem(n=16, bc="reflexive", rank=3)
    kp = kpsvd.kp_svd(op, "projected")
    lam = 0.05
    S = kpsvd.precond_scale(kp.Sigma, lam)
    K = lambda X: kron.apply_K(op, X, lam)  # noqa: E731
    Minv = lambda R: kpsvd.precond_apply(kp, S, R)  # noqa: E731
    rhs = kron.apply_AT(op, B)
    xs = [np.zeros_like(rhs)]
    x, info = pcg.pcg(K, Minv, rhs, 0.0, 8, callback=lambda it, xk: xs.append(xk.copy()))
    x_star = pcg.tik_exact_dense(op, B, lam)
    rs = [rhs - K(xk) for xk in xs]
    zs = [Minv(r) for r in rs]
    ps = [xs[k + 1] - xs[k] for k in range(len(xs) - 1)]       # alpha_k p_k
    for k in range(1, len(rs)):
        for j in range(k):
            assert abs(np.vdot(rs[k], zs[j])) <= 1e-8 * np.linalg.norm(rs[j]) * np.linalg.norm(zs[j])
    for k in range(1, len(ps)):
        for j in range(k):
            assert abs(np.vdot(ps[k], K(ps[j]))) <= 1e-8 * np.linalg.norm(ps[k]) * np.linalg.norm(K(ps[j]))
    for k, rel in enumerate(info.res_hist):
        assert abs(np.linalg.norm(rs[k]) / np.linalg.norm(rhs) - rel) <= 1e-9
    errs = [np.vdot(xk - x_star, K(xk - x_star)) for xk in xs]
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:]))


def test_fpcg_equals_pcg_with_constant_preconditioner():
    """With an exact (FP64, constant) preconditioner Polak-Ribiere = Fletcher-Reeves."""
    op, _, B = _problem(n=16, bc="reflexive", rank=3)
    kp = kpsvd.kp_svd(op, "projected")
    lam = 0.03
    x1, i1 = pcg.tik_pcg(op, kp, B, lam, 0.0, 12, flexible=False)
    x2, i2 = pcg.tik_pcg(op, kp, B, lam, 0.0, 12, flexible=True)
    assert np.linalg.norm(x1 - x2) <= 1e-10 * np.linalg.norm(x1)


def _directions_and_residuals(op, B, lam, minv, flexible, iters):
    rhs = kron.apply_AT(op, B)
    K = lambda X: kron.apply_K(op, X, lam)  # noqa: E731
    xs = [np.zeros_like(rhs)]
    pcg.pcg(K, minv, rhs, 0.0, iters, flexible, callback=lambda it, xk: xs.append(xk.copy()))
    ps = [xs[k + 1] - xs[k] for k in range(len(xs) - 1)]       # alpha_k p_k
    rs = [rhs - K(xk) for xk in xs]
    return ps, rs, K


def test_fpcg_local_conjugacy_with_a_varying_preconditioner():
    """Flexible PCG (Polak-Ribiere beta, Section 3's last paragraph) keeps
    p_{k+1}^T K p_k = 0 and p_k^T r_{k+1} = 0 for ANY sequence of
    preconditioners: with alpha_k = z_k^T r_k / p_k^T K p_k and r_{k+1} - r_k
    = -alpha_k K p_k, beta_k = -z_{k+1}^T K p_k / p_k^T K p_k.  Here every
    application uses another lambda_M; the Fletcher-Reeves beta loses the
    property under the same preconditioners."""
    op, _, B = _problem(n=16, bc="reflexive", rank=3)
    kp = kpsvd.kp_svd(op, "projected")
    lam = 0.05
    calls = []

    def minv(R):
        calls.append(None)
        lam_m = lam * (1.0 + 0.8 * np.sin(1.7 * len(calls)))
        return kpsvd.precond_apply(kp, kpsvd.precond_scale(kp.Sigma, lam_m), R)

    def worst(flexible):
        calls.clear()
        ps, rs, K = _directions_and_residuals(op, B, lam, minv, flexible, 8)
        conj = max(abs(np.vdot(ps[k + 1], K(ps[k]))) / (np.linalg.norm(ps[k + 1]) * np.linalg.norm(K(ps[k])))
                   for k in range(len(ps) - 1))
        orth = max(abs(np.vdot(ps[k], rs[k + 1])) / (np.linalg.norm(ps[k]) * np.linalg.norm(rs[k + 1]))
                   for k in range(len(ps)))
        return conj, orth

    conj, orth = worst(True)
    assert conj <= 1e-9 and orth <= 1e-9
    conj_fr, _ = worst(False)
    assert conj_fr > 1e-4


def test_unpreconditioned_cg_is_slower():
    """The preconditioner pays (Section 5.2 break-even m_P < 8/9 m_N) on a blur it
    approximates well."""
    op, _, B = _problem(n=16, bc="zero", rank=2, rho=0.3)
    kp = kpsvd.kp_svd(op, "projected")
    _, ip = pcg.tik_pcg(op, kp, B, 0.01, 1e-8, 500)
    _, iN = pcg.tik_pcg(op, None, B, 0.01, 1e-8, 500)
    assert ip.iters < (8.0 / 9.0) * iN.iters


def test_warm_start_and_zero_rhs():
    op, _, B = _problem(n=8, bc="zero", rank=2)
    kp = kpsvd.kp_svd(op, "projected")
    x_star = pcg.tik_exact_dense(op, B, 0.05)
    x, info = pcg.tik_pcg(op, kp, B, 0.05, 1e-12, 100, X0=x_star)
    assert info.iters <= 1 and np.linalg.norm(x - x_star) <= 1e-10 * np.linalg.norm(x_star)
    x0, info0 = pcg.tik_pcg(op, kp, np.zeros_like(B), 0.05, 1e-8, 10)
    assert info0.iters == 0 and not np.any(x0)


def test_noise_level_is_exact():
    """Section 5: noise level = ||e|| / ||b_true||."""
    op, X, _ = _problem(n=16, bc="zero", rank=2)
    g = synth.noise_direction(16, 16, np.random.default_rng(9))
    B, enorm = forward.observe(op, X, g, 0.05)
    Bt = kron.apply_A(op, X)
    assert abs(np.linalg.norm(B - Bt) / np.linalg.norm(Bt) - 0.05) < 1e-14
    assert abs(enorm - np.linalg.norm(B - Bt)) < 1e-12


def test_preconditioner_lambda_changes_the_path_not_the_solution():
    """A preconditioner built with lambda_M != lambda (Section 5.3's remedy
    for the early error jump) is still SPD, so (F)PCG converges to the same
    x_lambda (dense Cholesky); lambda_M = lambda gives the default iterates
    exactly, and a different lambda_M gives different iterates."""
    op, _, B = _problem(n=16, bc="reflexive", rank=3)
    kp = kpsvd.kp_svd(op, "projected")
    lam = 0.05
    K = kron.dense_A(op).T @ kron.dense_A(op) + lam * lam * np.eye(256)
    x_chol = np.linalg.solve(K, kron.vec(kron.apply_AT(op, B)))
    for flexible in (False, True):
        x3, info = pcg.tik_pcg(op, kp, B, lam, 1e-13, 500, flexible, lam_pc=3 * lam)
        assert info.converged
        assert np.linalg.norm(kron.vec(x3) - x_chol) <= 1e-10 * np.linalg.norm(x_chol)
        xa, _ = pcg.tik_pcg(op, kp, B, lam, 0.0, 3, flexible)
        xb, _ = pcg.tik_pcg(op, kp, B, lam, 0.0, 3, flexible, lam_pc=lam)
        xc, _ = pcg.tik_pcg(op, kp, B, lam, 0.0, 3, flexible, lam_pc=3 * lam)
        assert np.array_equal(xa, xb)
        assert np.linalg.norm(xc - xa) > 1e-6 * np.linalg.norm(xa)


def test_multiterm_preconditioner_with_all_terms_is_exact():
    """With k = all terms and the inner solve run to convergence the
    preconditioner is K^-1 itself: flexible PCG stops after one iteration at
    x_lambda (alpha = 1, x_1 = K^-1 A^T b)."""
    op, _, B = _problem(n=16, bc="reflexive", rank=3)
    kp = kpsvd.kp_svd(op, "projected")
    lam = 0.05
    x_chol = pcg.tik_exact_dense(op, B, lam)
    x, info = pcg.tik_fpcg_multiterm(op, kp, B, lam, k=3, inner_iters=300, tol=1e-10, maxit=5, inner_tol=1e-15)
    assert info.iters == 1
    assert np.linalg.norm(x - x_chol) <= 1e-10 * np.linalg.norm(x_chol)


def test_multiterm_preconditioner_with_one_term_is_the_kp_svd_solve():
    """k = 1 with the PRODUCT spectrum: M_1^T M_1 + lam^2 I is diagonalised
    exactly by V_r (x) V_c with eigenvalues sigma_c^2 sigma_r^2 + lam^2 (eq.
    AKronSVD), so one inner step already returns eq. PreconSolve's z."""
    op, _, B = _problem(n=16, bc="reflexive", rank=3)
    kp = kpsvd.kp_svd(op, "product")
    lam = 0.05
    R = np.random.default_rng(7).standard_normal((16, 16))
    z1 = pcg.multiterm_minv(op, kp, lam, k=1, inner_iters=1)(R)
    z_kp = kpsvd.precond_apply(kp, kpsvd.precond_scale(kp.Sigma, lam), R)
    np.testing.assert_allclose(z1, z_kp, rtol=0, atol=1e-12 * np.abs(z_kp).max())


@pytest.mark.parametrize("k", [2, 3])
def test_multiterm_fpcg_converges_to_the_tikhonov_solution(k):
    """Two inner steps with k terms: the preconditioner varies with r, and
    flexible PCG still converges to the dense Cholesky x_lambda."""
    op, _, B = _problem(n=16, bc="zero", rank=3)
    kp = kpsvd.kp_svd(op, "projected")
    lam = 0.05
    x_chol = pcg.tik_exact_dense(op, B, lam)
    x, info = pcg.tik_fpcg_multiterm(op, kp, B, lam, k=k, inner_iters=2, tol=1e-13, maxit=300)
    assert info.converged
    assert np.linalg.norm(x - x_chol) <= 1e-10 * np.linalg.norm(x_chol)


def test_multiterm_outer_iteration_is_flexible():
    """The inner solve makes the preconditioner vary with r, and the outer
    iteration keeps flexible PCG's local conjugacy p_{k+1}^T K p_k = 0 (which
    the Fletcher-Reeves beta loses under a varying preconditioner)."""
    op, _, B = _problem(n=16, bc="reflexive", rank=3)
    kp = kpsvd.kp_svd(op, "projected")
    lam = 0.05
    K = lambda X: kron.apply_K(op, X, lam)  # noqa: E731
    xs = [np.zeros_like(B)]
    pcg.tik_fpcg_multiterm(op, kp, B, lam, k=2, inner_iters=2, tol=0.0, maxit=6,
                           callback=lambda it, xk: xs.append(xk.copy()))
    ps = [xs[j + 1] - xs[j] for j in range(len(xs) - 1)]
    for j in range(len(ps) - 1):
        c = abs(np.vdot(ps[j + 1], K(ps[j]))) / (np.linalg.norm(ps[j + 1]) * np.linalg.norm(K(ps[j])))
        assert c <= 1e-9, j


def test_exact_solution_above_the_dense_size_uses_pcg_to_the_filter_factor_solution():
    """N = 72^2 > 4096 takes the FP64 PCG branch; a separable blur makes the
    KP-SVD the exact SVD of A, so x_lam = V_c ((Sigma .* B_hat) ./ (Sigma^2 +
    lam^2)) V_r^T with B_hat = U_c^T B U_r (eq. TikSV, filter factors)."""
    n = 72
    P = synth.separable_psf(n, n, n // 2, n // 2, 2.5, 1.5)
    rng = np.random.default_rng(8)
    X = synth.phantom(n, n, 8, rng)
    op = kron.kron_operator(P, (n // 2, n // 2), "reflexive", rank=1)
    kp = kpsvd.kp_svd(op, "product")
    B, _ = forward.observe(op, X, synth.noise_direction(n, n, rng), 0.01)
    lam = 0.02
    Ur, sr, Vrt = np.linalg.svd(op.Ar[0])
    Uc, sc, Vct = np.linalg.svd(op.Ac[0])
    Sig = np.outer(sc, sr)
    x_ff = Vct.T @ (Sig * (Uc.T @ B @ Ur) / (Sig ** 2 + lam ** 2)) @ Vrt
    x = pcg.tik_exact(op, kp, B, lam)
    assert np.linalg.norm(x - x_ff) <= 1e-11 * np.linalg.norm(x_ff)
    # a non-separable blur (the preconditioner no longer exact): the normal
    # equations hold to the branch's tolerance
    P2 = synth.gaussian_psf(n, n, n // 2, n // 2, 2.5, 1.5, 0.6)
    op2 = kron.kron_operator(P2, (n // 2, n // 2), "reflexive", rank=2)
    x2 = pcg.tik_exact(op2, kpsvd.kp_svd(op2, "projected"), B, lam)
    rhs = kron.apply_AT(op2, B)
    assert np.linalg.norm(kron.apply_K(op2, x2, lam) - rhs) <= 1e-12 * np.linalg.norm(rhs)


@pytest.mark.parametrize("bc", ["zero", "reflexive"])
def test_projected_and_product_spectra_coincide_for_one_term(bc):
    """With one Kronecker term A = A_r (x) A_c, diag((U_r (x) U_c)^T A (V_r (x) V_c))
    is sigma_c,i sigma_r,j, eq. AKronSVD's product spectrum; with more terms
    they differ."""
    op1, _, _ = _problem(n=12, bc=bc, rank=1)
    np.testing.assert_allclose(kpsvd.kp_svd(op1, "projected").Sigma, kpsvd.kp_svd(op1, "product").Sigma,
                               rtol=0, atol=1e-13)
    op3, _, _ = _problem(n=12, bc=bc, rank=3)
    assert np.abs(kpsvd.kp_svd(op3, "projected").Sigma - kpsvd.kp_svd(op3, "product").Sigma).max() > 1e-6


@pytest.mark.parametrize("bc", ["zero", "reflexive"])
def test_delta_psf_is_the_identity(bc):
    """Degenerate blur: a PSF that is 1 at its centre and 0 elsewhere gives
    A = I for either boundary condition (one Kronecker term), a KP spectrum
    of ones, and x_lambda = b / (1 + lambda^2) (eq. TikSV with every singular
    value 1), which PCG reaches in one iteration."""
    n_r, n_c, c = 12, 10, (5, 4)
    P = np.zeros((n_r, n_c))
    P[c] = 1.0
    op = kron.kron_operator(P, c, bc, rank=0)
    np.testing.assert_allclose(kron.dense_A(op), np.eye(n_r * n_c), rtol=0, atol=1e-14)
    kp = kpsvd.kp_svd(op, "projected")
    np.testing.assert_allclose(np.abs(kp.Sigma), 1.0, rtol=0, atol=1e-14)
    B = np.random.default_rng(3).standard_normal((n_r, n_c))
    lam = 0.3
    x, info = pcg.tik_pcg(op, kp, B, lam, 1e-14, 5)
    assert info.iters == 1
    np.testing.assert_allclose(x, B / (1.0 + lam * lam), rtol=0, atol=1e-14)
