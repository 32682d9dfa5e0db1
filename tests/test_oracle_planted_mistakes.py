"""Planted mistakes: each case plants one plausible error (a dropped term, a
wrong sign, index or exponent, a transposed or swapped operand) in a copy of
one oracle module's source, on the CPU, and checks that the named pin of the
oracle suite fails against it.  The pins are the suite's own test functions,
called unchanged; the real modules are restored after each case (pytest's
monkeypatch), and the source must hold the planted snippet exactly once, so
a case cannot silently stop planting anything when the oracle changes.
A change that leaves every result the same (a redundant check, a branch
choice between two ways of computing x_lambda) plants nothing and has no
case.
"""
import importlib
import inspect
import types
import warnings

import pytest

import test_oracle_kron as TK
import test_oracle_lambda as TL
import test_oracle_lowprec as TP
import test_oracle_mlp as TM
import test_oracle_solver as TS


def plant(monkeypatch, modname, old, new):
    """Replace every function of oracle.<modname> by its counterpart compiled
    from the source with `old` replaced by `new`."""
    real = importlib.import_module(f"oracle.{modname}")
    src = inspect.getsource(real)
    assert src.count(old) == 1, f"{old!r} must occur exactly once in oracle/{modname}.py"
    mod = types.ModuleType(real.__name__)
    mod.__package__ = "oracle"
    exec(compile(src.replace(old, new), real.__file__, "exec"), mod.__dict__)
    for name, obj in vars(mod).items():
        if inspect.isfunction(obj) and obj.__module__ == real.__name__:
            monkeypatch.setattr(real, name, obj)


def _sep():
    return TL.separable_problem()


# (case, module, planted snippet, replacement, the pin that must fail)
CASES = [
    # Kronecker-sum operator (oracle/kron.py)
    ("Toeplitz index transposed", "kron",
     "return _take(u, c + i - j)", "return _take(u, c + j - i)",
     lambda: TK.test_full_rank_sum_equals_direct_convolution("zero", 12, 10, (5, 3))),
    ("Hankel reflection off by one", "kron",
     "_take(u, c + i + j + 1) + _take", "_take(u, c + i + j) + _take",
     lambda: TK.test_full_rank_sum_equals_direct_convolution("reflexive", 8, 8, (4, 4))),
    ("Hankel second reflection dropped", "kron",
     "return _take(u, c + i + j + 1) + _take(u, c + i + j + 1 - 2 * n)", "return _take(u, c + i + j + 1)",
     lambda: TK.test_full_rank_sum_equals_direct_convolution("reflexive", 8, 8, (4, 4))),
    ("reflexive factor without its Hankel part", "kron",
     "return toeplitz_factor(u, c) + hankel_factor(u, c)", "return toeplitz_factor(u, c)",
     lambda: TK.test_full_rank_sum_equals_direct_convolution("reflexive", 16, 16, (8, 8))),
    ("weights used without the square root", "kron",
     "dc = np.sqrt(kron_weights(n_r, c_r))", "dc = kron_weights(n_r, c_r)",
     TK.test_weighted_first_term_is_van_loan_pitsianis_optimum),
    ("weights lose the absolute value", "kron",
     "return (n - np.abs(k - c)).astype(np.float64)", "return (n - (k - c)).astype(np.float64)",
     TK.test_weighted_first_term_is_van_loan_pitsianis_optimum),
    ("column vector not unweighted", "kron",
     "u = np.sqrt(s[m]) * Ut[:, m] / dc", "u = np.sqrt(s[m]) * Ut[:, m]",
     lambda: TK.test_full_rank_sum_equals_direct_convolution("zero", 8, 8, (4, 4))),
    ("sign flip applied to u only", "kron",
     "u, v = -u, -v", "u, v = -u, v",
     TK.test_sign_convention_and_exact_sum),
    ("A applies A_r untransposed", "kron",
     "out += Ac @ X @ Ar.T", "out += Ac @ X @ Ar",
     TK.test_kronecker_identity_8x8),
    ("A^T applies A_c untransposed", "kron",
     "out += Ac.T @ Y @ Ar", "out += Ac @ Y @ Ar",
     TK.test_kronecker_identity_8x8),
    ("K adds lambda instead of lambda^2", "kron",
     "+ lam * lam * X", "+ lam * X",
     lambda: TS.test_pcg_converges_to_dense_cholesky("reflexive", False)),
    ("dense A with the Kronecker factors swapped", "kron",
     "A += np.kron(Ar, Ac)", "A += np.kron(Ac, Ar)",
     lambda: TK.test_full_rank_sum_equals_direct_convolution("zero", 12, 10, (5, 3))),
    ("requested rank ignored", "kron",
     "r = min(n_r, n_c) if rank in (0, None) else int(rank)", "r = min(n_r, n_c)",
     lambda: TK.test_truncation_error_decreases("zero")),
    ("vec stacks rows", "kron",
     'return np.asarray(X).reshape(-1, order="F")', 'return np.asarray(X).reshape(-1, order="C")',
     TK.test_kronecker_identity_8x8),
    # KP-SVD and preconditioner (oracle/kpsvd.py)
    ("V taken untransposed from the SVD", "kpsvd",
     "Vr, Vc = Vrt.T, Vct.T", "Vr, Vc = Vrt, Vct",
     TS.test_preconditioner_solve_matches_dense_solve),
    ("preconditioner in the U basis", "kpsvd",
     "return kp.Vc @ (S * (kp.Vc.T @ R @ kp.Vr)) @ kp.Vr.T",
     "return kp.Uc @ (S * (kp.Uc.T @ R @ kp.Ur)) @ kp.Ur.T",
     TS.test_preconditioner_solve_matches_dense_solve),
    ("preconditioner bases transposed", "kpsvd",
     "return kp.Vc @ (S * (kp.Vc.T @ R @ kp.Vr)) @ kp.Vr.T",
     "return kp.Vc.T @ (S * (kp.Vc @ R @ kp.Vr.T)) @ kp.Vr",
     TS.test_preconditioner_solve_matches_dense_solve),
    ("S with Sigma not squared", "kpsvd",
     "return 1.0 / (Sigma * Sigma + lam * lam)", "return 1.0 / (Sigma + lam * lam)",
     TS.test_preconditioner_solve_matches_dense_solve),
    ("PRODUCT spectrum transposed", "kpsvd",
     "Sigma = np.outer(sc, sr)", "Sigma = np.outer(sr, sc)",
     TS.test_preconditioner_solve_matches_dense_solve),
    ("PROJECTED spectrum keeps one term", "kpsvd",
     "Sigma += np.outer(dc, dr)", "Sigma = np.outer(dc, dr)",
     lambda: TS.test_projected_sigma_is_diag_in_kp_basis("zero")),
    ("PROJECTED spectrum with V on both sides", "kpsvd",
     "dc = np.diag(Uc.T @ Ac @ Vc)", "dc = np.diag(Vc.T @ Ac @ Vc)",
     lambda: TS.test_projected_sigma_is_diag_in_kp_basis("reflexive")),
    ("PROJECTED spectrum with the row bases swapped", "kpsvd",
     "dr = np.diag(Ur.T @ Ar @ Vr)", "dr = np.diag(Vr.T @ Ar @ Ur)",
     lambda: TS.test_projected_sigma_is_diag_in_kp_basis("reflexive")),
    ("explicit M with the Kronecker factors swapped", "kpsvd",
     "V = np.kron(kp.Vr, kp.Vc)", "V = np.kron(kp.Vc, kp.Vr)",
     TS.test_preconditioner_solve_matches_dense_solve),
    # PCG / FPCG (oracle/pcg.py)
    ("alpha from p^T p", "pcg",
     "alpha = zr / np.vdot(p, q)", "alpha = zr / np.vdot(p, p)",
     lambda: TS.test_pcg_converges_to_dense_cholesky("reflexive", False)),
    ("residual update with the wrong sign", "pcg",
     "r_new = r - alpha * q", "r_new = r + alpha * q",
     lambda: TS.test_pcg_converges_to_dense_cholesky("zero", False)),
    ("Polak-Ribiere beta with r_new + r", "pcg",
     "beta = np.vdot(z_new, r_new - r) / zr", "beta = np.vdot(z_new, r_new + r) / zr",
     TS.test_fpcg_local_conjugacy_with_a_varying_preconditioner),
    ("flexible PCG falls back to Fletcher-Reeves", "pcg",
     "if flexible:", "if False:",
     TS.test_fpcg_local_conjugacy_with_a_varying_preconditioner),
    ("Fletcher-Reeves beta over r^T r", "pcg",
     "beta = zr_new / zr", "beta = zr_new / np.vdot(r, r)",
     TS.test_pcg_invariants),
    ("new direction built from the old z", "pcg",
     "p = z_new + beta * p", "p = z + beta * p",
     TS.test_pcg_invariants),
    ("first direction not preconditioned", "pcg",
     "z = apply_Minv(r)\n    p = z.copy()", "z = r.copy()\n    p = z.copy()",
     TS.test_separable_zero_bc_pcg_converges_in_one_iteration),
    ("warm start residual without K x_0", "pcg",
     "r = rhs - apply_K(x) if x0 is not None else rhs.copy()", "r = rhs.copy()",
     TS.test_warm_start_and_zero_rhs),
    ("preconditioner lambda ignored", "pcg",
     "S = kpsvd.precond_scale(kp.Sigma, lam if lam_pc is None else lam_pc)",
     "S = kpsvd.precond_scale(kp.Sigma, lam)",
     TS.test_preconditioner_lambda_changes_the_path_not_the_solution),
    ("dense solve with A A^T", "pcg",
     "K = A.T @ A + lam * lam * np.eye(A.shape[1])", "K = A @ A.T + lam * lam * np.eye(A.shape[1])",
     TS.test_filter_factor_solution_equals_cholesky),
    ("dense solve with b for A^T b", "pcg",
     "rhs = A.T @ kron.vec(B)", "rhs = kron.vec(B)",
     TS.test_filter_factor_solution_equals_cholesky),
    ("multiterm preconditioner keeps one term", "pcg",
     "Ac=op.Ac[:k], Ar=op.Ar[:k]", "Ac=op.Ac[:1], Ar=op.Ar[:1]",
     TS.test_multiterm_preconditioner_with_all_terms_is_exact),
    ("multiterm outer iteration not flexible", "pcg",
     "maxit, flexible=True, callback=callback)", "maxit, flexible=False, callback=callback)",
     TS.test_multiterm_outer_iteration_is_flexible),
    ("multiterm inner solve on the full operator", "pcg",
     "pcg(lambda X: kron.apply_K(opk, X, lam)", "pcg(lambda X: kron.apply_K(op, X, lam)",
     TS.test_multiterm_preconditioner_with_one_term_is_the_kp_svd_solve),
    ("exact solution's PCG stopped early", "pcg",
     "tol: float = 1e-13, maxit: int = 2000", "tol: float = 1e-6, maxit: int = 2000",
     TS.test_exact_solution_above_the_dense_size_uses_pcg_to_the_filter_factor_solution),
    # observed data (oracle/forward.py)
    ("noise scaled by the image instead of the blurred image", "forward",
     "e = noise_level * np.linalg.norm(Bt)", "e = noise_level * np.linalg.norm(X_true)",
     TS.test_noise_level_is_exact),
    ("noise direction not normalised", "forward",
     "* g / np.linalg.norm(g)", "* g",
     TS.test_noise_level_is_exact),
    # closed-form parameter choice (oracle/lam.py)
    ("GCV without the factor N", "lam",
     "return Sigma.size * np.sum((Bhat / d) ** 2) / np.sum(1.0 / d) ** 2",
     "return np.sum((Bhat / d) ** 2) / np.sum(1.0 / d) ** 2",
     lambda: TL.test_gcv_closed_form_matches_trace_definition(_sep(), 0.1)),
    ("GCV denominator not squared", "lam",
     "/ np.sum(1.0 / d) ** 2", "/ np.sum(1.0 / d)",
     lambda: TL.test_gcv_closed_form_matches_trace_definition(_sep(), 0.1)),
    ("GCV residual filter 1/d not squared", "lam",
     "np.sum((Bhat / d) ** 2)", "np.sum(Bhat * Bhat / d)",
     lambda: TL.test_gcv_closed_form_matches_trace_definition(_sep(), 0.1)),
    ("wGCV weight with the wrong sign", "lam",
     "den = np.sum(((1.0 - omega) * s2", "den = np.sum(((1.0 + omega) * s2",
     lambda: TL.test_wgcv_closed_form_matches_trace_definition(_sep(), 3.0, 0.1)),
    ("discrepancy filter lambda instead of lambda^2", "lam",
     "return np.sum((lam * lam * Bhat / d) ** 2) - eps * eps", "return np.sum((lam * Bhat / d) ** 2) - eps * eps",
     lambda: TL.test_discrepancy_and_opt_match_residual_definitions(_sep(), 3e-2)),
    ("discrepancy with eps not squared", "lam",
     ") ** 2) - eps * eps", ") ** 2) - eps",
     lambda: TL.test_discrepancy_and_opt_match_residual_definitions(_sep(), 3e-2)),
    ("optimal-error filter without sigma", "lam",
     "return np.sum((Sigma * Bhat / d - Xhat) ** 2)", "return np.sum((Bhat / d - Xhat) ** 2)",
     lambda: TL.test_discrepancy_and_opt_match_residual_definitions(_sep(), 3e-2)),
    ("b_hat with the row and column bases swapped", "lam",
     "return kp.Uc.T @ B @ kp.Ur", "return kp.Ur.T @ B @ kp.Uc",
     lambda: TL.test_gcv_closed_form_matches_trace_definition(_sep(), 0.1)),
    ("x_hat in the U basis", "lam",
     "return kp.Vc.T @ X @ kp.Vr", "return kp.Uc.T @ X @ kp.Ur",
     lambda: TL.test_discrepancy_and_opt_match_residual_definitions(_sep(), 3e-2)),
    ("search bounds without the 1e-10 floor", "lam",
     "return max(smin, 1e-10 * smax), smax", "return smin, smax",
     TL.test_lambda_search_bounds_by_hand),
    ("search bounds floored at 1e-8", "lam",
     "return max(smin, 1e-10 * smax), smax", "return max(smin, 1e-8 * smax), smax",
     TL.test_lambda_search_bounds_by_hand),
    ("grid search keeps the largest value", "lam",
     "int(np.argmin(vals[::-1]))", "int(np.argmax(vals[::-1]))",
     lambda: TL.test_minimisers_match_exhaustive_grid(_sep(), "gcv")),
    ("wGCV search not kept above the trace root", "lam",
     "lo = max(lo, wgcv_lower_limit(Sigma, param, lo, hi))", "lo = lo",
     lambda: TL.test_wgcv_spurious_minimum_is_excluded(_sep())),
    ("wGCV trace root not found", "lam",
     "    return float(np.exp(b))", "    return lo",
     lambda: TL.test_wgcv_spurious_minimum_is_excluded(_sep())),
    ("discrepancy returns the bracket's end", "lam",
     "return float(np.exp(brentq(D, tl, th, xtol=1e-15, rtol=4 * np.finfo(float).eps, maxiter=500)))",
     "return float(np.exp(th))",
     lambda: TL.test_discrepancy_root_and_no_root(_sep())),
    # rounding helpers (oracle/lowprec.py)
    ("bf16 by truncation", "lowprec",
     "u = ((u + 0x7FFF + lsb) & 0xFFFF0000)", "u = (u & 0xFFFF0000)",
     TP.test_bf16_hand_values),
    ("bf16 ties away from zero", "lowprec",
     "u = ((u + 0x7FFF + lsb) & 0xFFFF0000)", "u = ((u + 0x8000) & 0xFFFF0000)",
     TP.test_bf16_hand_values),
    ("fp16 rounded from float64 directly", "lowprec",
     "return f.astype(np.float16).astype(np.float64)",
     "return np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)",
     TP.test_bf16_hand_values),
    ("e4m3 ties away from zero", "lowprec",
     "y = np.rint(a / q) * q", "y = np.floor(a / q + 0.5) * q",
     TP.test_e4m3_hand_values),
    ("e4m3 with four mantissa bits", "lowprec",
     "q = np.ldexp(1.0, ex - 3)", "q = np.ldexp(1.0, ex - 4)",
     TP.test_e4m3_hand_values),
    ("e4m3 without subnormal clamp", "lowprec",
     "ex = np.maximum(e - 1, -6)", "ex = e - 1",
     TP.test_e4m3_hand_values),
    ("e4m3 not saturating", "lowprec",
     "y = np.minimum(y, E4M3_MAX)", "y = y",
     TP.test_e4m3_hand_values),
    ("MX scale one binade too high", "lowprec",
     "scale = np.ldexp(1.0, (e - 1) - 8)", "scale = np.ldexp(1.0, (e - 1) - 7)",
     TP.test_mxfp8_hand_values),
    # learned-lambda regressor (oracle/mlp.py)
    ("feature bins rounded up", "mlp",
     "j = int(np.floor(-np.log10(s2[i] / s2max) * NB / DEC))", "j = int(np.ceil(-np.log10(s2[i] / s2max) * NB / DEC))",
     TM.test_features_of_a_hand_built_spectrum),
    ("feature count without the +1", "mlp",
     "f[j] = np.log10((sb[j] + TINY * s2max) / (cnt[j] + 1.0))", "f[j] = np.log10((sb[j] + TINY * s2max) / max(cnt[j], 1.0))",
     TM.test_features_of_a_hand_built_spectrum),
    ("16-decade floor not applied", "mlp",
     "if s2[i] > s2max * 10.0 ** (-DEC):", "if s2[i] > 0:",
     TM.test_features_of_a_hand_built_spectrum),
    ("noise estimate from the shallowest bins", "mlp",
     "for j in range(NB - 1, -1, -1):", "for j in range(NB):",
     TM.test_features_of_a_hand_built_spectrum),
    ("count feature over n + 1", "mlp",
     "f[NB + j] = np.log10((cnt[j] + 1.0) / n)", "f[NB + j] = np.log10((cnt[j] + 1.0) / (n + 1.0))",
     TM.test_features_of_a_hand_built_spectrum),
    ("noise estimate over the deepest quarter", "mlp",
     "if acc_c >= n / 8.0:", "if acc_c >= n / 4.0:",
     TM.test_features_of_a_hand_built_spectrum),
    ("largest-spectrum feature from sigma, not sigma^2", "mlp",
     "f[2 * NB + 1] = np.log10(s2max)", "f[2 * NB + 1] = np.log10(np.sqrt(s2max))",
     TM.test_features_are_permutation_invariant_and_shift_with_scale),
    ("GELU by its tanh approximation (Hendrycks and Gimpel)", "mlp",
     "return x * _phi(x)\n", "return 0.5 * x * (1.0 + np.tanh(np.sqrt(2.0 / np.pi) * (x + 0.044715 * x ** 3)))\n",
     TM.test_gelu_is_x_times_normal_cdf),
    ("GELU derivative without the density term", "mlp",
     "return _phi(x) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)", "return _phi(x)",
     TM.test_gelu_is_x_times_normal_cdf),
    ("input normalisation adds the mean", "mlp",
     "- net.mean) * net.inv_std", "+ net.mean) * net.inv_std",
     TM.test_forward_pass_by_hand),
    ("GELU on the output layer", "mlp",
     "a = gelu(z) if l < L - 1 else z", "a = gelu(z)",
     TM.test_forward_pass_by_hand),
    ("hidden layer without its bias", "mlp",
     "z = a @ _w(net.W[l], bf16).T + net.c[l]", "z = a @ _w(net.W[l], bf16).T",
     TM.test_forward_pass_by_hand),
    ("weights used unrounded", "mlp",
     "return lp.to_bf16(W) if bf16 else W", "return W",
     TM.test_forward_pass_by_hand),
    ("backward pass skips the activation derivative", "mlp",
     "g = (g @ _w(net.W[l], bf16)) * gelu_grad(pres[l - 1])", "g = g @ _w(net.W[l], bf16)",
     TM.test_gradients_match_finite_differences),
    ("bias gradient averaged over the batch", "mlp",
     "gc[l] = g.sum(axis=0)", "gc[l] = g.mean(axis=0)",
     TM.test_gradients_match_finite_differences),
    ("loss summed instead of averaged", "mlp",
     "return np.mean((pred - np.asarray(y, dtype=np.float64)) ** 2)",
     "return np.sum((pred - np.asarray(y, dtype=np.float64)) ** 2)",
     TM.test_gradients_match_finite_differences),
    ("Adam without bias correction", "mlp",
     "mh = net.m[k] / (1.0 - b1 ** net.t)", "mh = net.m[k]",
     TM.test_adam_first_two_steps_closed_form),
    ("Adam first moment with the second moment's decay", "mlp",
     "net.m[k] = b1 * net.m[k] + (1.0 - b1) * gk", "net.m[k] = b2 * net.m[k] + (1.0 - b2) * gk",
     TM.test_adam_first_two_steps_closed_form),
    ("Adam epsilon inside the square root", "mlp",
     "p -= lr * mh / (np.sqrt(vh) + eps)", "p -= lr * mh / np.sqrt(vh + eps)",
     TM.test_adam_first_two_steps_closed_form),
    ("Adam second moment not squared", "mlp",
     "(1.0 - b2) * gk * gk", "(1.0 - b2) * abs(gk)",
     TM.test_adam_first_two_steps_closed_form),
]


@pytest.mark.parametrize("case,module,old,new,pin", CASES, ids=[c[0] for c in CASES])
def test_pin_catches_planted_mistake(monkeypatch, case, module, old, new, pin):
    plant(monkeypatch, module, old, new)
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")      # a planted mistake may overflow or divide by zero
        with pytest.raises(AssertionError):
            pin()


def test_pins_pass_on_the_real_oracle():
    """The same pins, unplanted, pass (the control for every case above)."""
    for _, _, _, _, pin in CASES:
        pin()
