/*
 * kpsvd.h - C ABI of the GB300 (sm_103a) library for Kronecker-product SVD
 * preconditioned Tikhonov deblurring.
 *
 * Problem (arXiv 2311.15393, Section 1 eqs. invp, lsp:Tik, tik:normal1):
 * given blurred, noisy data b = A x_true + eps of an n_r x n_c image, the PSF
 * that defines A, and a regularisation parameter lambda, solve the Tikhonov
 * normal equations (A^T A + lambda^2 I) x = A^T b by preconditioned CG or
 * flexible PCG (Section 2.3; Section 3 last paragraph), with the
 * preconditioner M = V (Sigma^T Sigma + lambda^2 I) V^T of the Kronecker
 * product SVD of the blur (eqs. AKronSVD, PreconSystem, PreconSolve), and
 * choose lambda in closed form over the KP spectrum (Section 2.2).
 *
 * Conventions shared by every entry point
 *  - Images are column-major n_r x n_c arrays (vec = column stacking,
 *    Section 3): element (i, j) at offset i + n_r * j.
 *  - Pointers documented "device" are device memory of the context's GPU,
 *    at least 16-byte aligned, owned by the caller, and must stay valid until
 *    the call's work on the context's stream has finished.  Pointers
 *    documented "host" are ordinary host memory.
 *  - The element type of image arguments is the context's vector precision
 *    (KP_F64 -> double, KP_F32 -> float) set by kp_setup.
 *  - All work is issued on the stream given to kp_create.  Calls that return
 *    scalars to the host (choose_lambda, tik_pcg info, kp_forward noise norm,
 *    getters) synchronise that stream before returning; kp_apply_* are
 *    asynchronous.
 *  - No call aborts or throws.  Each returns a kp_status; on failure a
 *    message is kept per thread and read with kp_last_error().  A CUDA error
 *    leaves the context usable only if the error is not sticky.
 *  - A context is not thread safe; use one context per host thread.
 */
#ifndef KPSVD_H
#define KPSVD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kp_ctx kp_ctx; /* opaque; owns all factor and workspace device memory */

typedef enum {
  KP_OK = 0,
  KP_EINVAL = 1,      /* bad argument (shape, pointer, enum, combination) */
  KP_ENOMEM = 2,      /* device or host allocation failed */
  KP_ECUDA = 3,       /* CUDA runtime / driver error */
  KP_ENOTSUP = 4,     /* valid but unsupported combination or device */
  KP_ENOCONV = 5,     /* maxit reached before tol, or the true residual stagnated
                         above tol; x holds the last iterate */
  KP_EBREAKDOWN = 6,  /* p^T K p <= 0 or z^T r <= 0 in (F)PCG */
  KP_ENUMERIC = 7,    /* NaN / Inf met in a reduction */
  KP_ENOROOT = 8,     /* discrepancy equation has no root */
  KP_ETIMEOUT = 9,    /* a bounded device-side wait gave up */
  KP_ESTATE = 10      /* call out of order (e.g. solve before kp_setup) */
} kp_status;

typedef enum { KP_BC_ZERO = 0, KP_BC_REFLEXIVE = 1 } kp_bc;

/* Arithmetic of a part of the path.
 *   KP_F64   FP64 SIMT kernels
 *   KP_F32   FP32 SIMT kernels
 *   KP_BF16  tcgen05 BF16 x BF16 -> FP32 (operator: one product per GEMM,
 *            with reliable residual updates through an FP32-accurate
 *            six-product split; preconditioner: bf16 activations, factors
 *            V_c, V_r carried as bf16 hi + lo pairs)
 *   KP_BF16X3 tcgen05, operands split into bf16 hi + lo, three products
 *   KP_F16   tcgen05 FP16 x FP16 -> FP32 (preconditioner)
 *   KP_E4M3  tcgen05 FP8 E4M3 x E4M3 -> FP32 with power-of-two per-tensor
 *            scales (preconditioner) */
typedef enum { KP_F64 = 0, KP_F32 = 1, KP_BF16 = 2, KP_BF16X3 = 3, KP_F16 = 4, KP_E4M3 = 5 } kp_prec;

/* KP spectrum used by the preconditioner and by choose_lambda:
 *   PRODUCT    Sigma = Sigma_r (x) Sigma_c (eq. AKronSVD)
 *   PROJECTED  Sigma = diag((U_r (x) U_c)^T A (V_r (x) V_c)), the diagonal of
 *              the full Kronecker-sum operator in the KP basis (equal to
 *              PRODUCT when A has one term). */
typedef enum { KP_SIGMA_PRODUCT = 0, KP_SIGMA_PROJECTED = 1 } kp_sigma;

typedef enum {
  KP_LAMBDA_GCV = 0,          /* eq. GCVTikSVD */
  KP_LAMBDA_WGCV = 1,         /* eq. wGCVTikSVD, param = omega */
  KP_LAMBDA_DISCREPANCY = 2,  /* eq. DSCTikSVD, param = eps = eta ||e||_2 (absolute) */
  KP_LAMBDA_OPT = 3           /* eq. OptTikSVD, needs x_true */
} kp_lambda_method;

typedef struct {
  int iters;             /* (F)PCG iterations done (one K application each) */
  int replacements;      /* reliable residual updates done */
  double rel_res;        /* ||r|| / ||A^T b|| of the residual the solver ended with */
  kp_status status;      /* same as the return value of tik_pcg */
  double ms_solve;       /* device time of the solve (CUDA events) */
  double ms_setup;       /* device time of the context's last kp_setup (CUDA events) */
  double* res_hist;      /* optional caller-owned host buffer of res_hist_len doubles: */
  int res_hist_len;      /*   ||r_k|| / ||A^T b|| for k = 0 .. min(iters, len - 1) */
} kp_solve_info;

/* Create a context on CUDA device `device`, issuing work on `cuda_stream`
 * (a cudaStream_t).  NULL means the legacy default stream: the work then
 * runs on a private stream of the context that is ordered after the
 * default stream's earlier work at each call and before its later work. */
kp_status kp_create(kp_ctx** out, int device, void* cuda_stream);

/* Release every device allocation of the context.  NULL is allowed. */
void kp_destroy(kp_ctx* ctx);

/* Build the operator and the preconditioner from the PSF (Sections 3 and 5).
 *   psf      device, double, column-major n_r x n_c, PSF with 0-based
 *            centre (center_r, center_c) (the entry weighting the pixel itself)
 *   bc       boundary condition of the blur
 *   op_rank  number of Kronecker terms of A (eq. KronSumDecomp), from the
 *            SVD of the weighted PSF D_c P D_r (Frobenius-optimal first term);
 *            0 = full rank min(n_r, n_c)
 *   pc_rank  Kronecker terms behind the preconditioner, 1 .. op_rank.  1: the
 *            KP-SVD preconditioner M = V (Sigma^2 + lambda^2 I) V^T of the
 *            first term (eqs. PreconSystem, PreconSolve).  k > 1 (Section
 *            5.3 finds the one-term M weak for blurs with many terms):
 *            z ~ (M_k^T M_k + lambda^2 I)^-1 r, M_k the first k terms of A,
 *            by "pc_inner_iters" (default 2) PCG steps on that system from
 *            z = 0, preconditioned by the one-term KP-SVD solve; it varies
 *            with r, so use it with flexible = 1 in tik_pcg
 *   op_prec  KP_F64 | KP_F32 | KP_BF16 | KP_BF16X3
 *   pc_prec  KP_F64 | KP_F32 | KP_BF16 | KP_F16 | KP_E4M3 (rank-1 KP-SVD preconditioner)
 *   vec_prec KP_F64 | KP_F32: element type of images and of the PCG vectors
 *   sigma    KP spectrum definition
 * Supported combinations: (F64, F64, F64); (F32, F32|BF16|F16|E4M3, F32);
 * (BF16|BF16X3, F32|BF16|F16|E4M3, F32).  Tensor-core precisions need
 * n_r and n_c multiples of 16.  The factor SVDs (one-sided Jacobi), the PSF
 * terms, Sigma and the spectral quantities are computed on the device: in
 * FP64 for FP64 vectors; for FP32 vectors the O(n^3) products, the Jacobi
 * rotations and the PSF subspace iteration run in FP32 (norms, sorting and
 * the stored Sigma stay FP64; option "setup_fp64" restores FP64).  May be
 * called again on the same context to replace the problem.  Errors:
 * KP_EINVAL for a NULL or unaligned psf, n_r or n_c < 2, a centre outside the
 * grid, op_rank outside [0, min(n_r, n_c)], pc_rank outside [1, op_rank], an
 * unknown bc or sigma, or an
 * unsupported precision combination; KP_ENOTSUP when tensor-core precisions
 * meet a device other than sm_103 or sizes not multiples of 16.  These
 * checks run first and leave the context's previous problem in place.  A
 * failure after them leaves the context without a problem, and later calls
 * other than kp_setup return KP_ESTATE: KP_ENUMERIC for a PSF holding a NaN
 * or Inf, KP_EINVAL for an all-zero PSF, KP_ENOMEM, KP_ECUDA.
 * Synchronises. */
kp_status kp_setup(kp_ctx* ctx, const double* psf, int n_r, int n_c, int center_r, int center_c,
                   kp_bc bc, int op_rank, int pc_rank, kp_prec op_prec, kp_prec pc_prec, kp_prec vec_prec,
                   kp_sigma sigma);

/* Observed data (eq. invp, Section 5 noise level): b = A x + e with
 * e = noise_level * ||A x||_2 * g / ||g||_2, A applied in FP64-accurate
 * arithmetic of the context's vector type.
 *   x, g    device, vec type, n_r x n_c (g: caller's noise direction)
 *   b       device, vec type, n_r x n_c, written
 *   noise_norm  host, nullable: ||e||_2 */
kp_status kp_forward(kp_ctx* ctx, const void* x, const void* g, double noise_level, void* b,
                     double* noise_norm);

/* Solve (A^T A + lambda^2 I) x = A^T b (eq. tik:normal2) by PCG (flexible =
 * 0, Fletcher-Reeves beta) or flexible PCG (flexible = 1, Polak-Ribiere beta,
 * Section 3 last paragraph), preconditioned by the KP-SVD (eq. PreconSolve)
 * with the same lambda (times option "pc_lambda_ratio", default 1).  Stops
 * when ||r|| <= tol ||A^T b||; after maxit iterations it returns KP_ENOCONV
 * with x = last iterate, and likewise when three residual replacements in a
 * row fail to halve the true residual (the attainable accuracy of the
 * reduced-precision operator and FP32 vectors lies above tol).  Other
 * errors: KP_EBREAKDOWN (p^T K p <= 0 or z^T r <= 0), KP_ENUMERIC (NaN / Inf),
 * KP_ETIMEOUT (a bounded device wait gave up), KP_ESTATE before kp_setup,
 * KP_EINVAL for lambda <= 0 or not finite, tol < 0, maxit < 1, or b, x NULL
 * or not 16-byte aligned.
 *   b        device, vec type, n_r x n_c
 *   x        device, vec type, n_r x n_c; input when warm_start != 0, output
 *   info     host, nullable
 * With an operator below FP64 the residual is replaced by the true residual
 * A^T (b - A x) - lambda^2 x, computed with an FP32-accurate operator,
 * whenever ||r|| has fallen by the reliable-update factor since the last
 * replacement, after 50 iterations without one, and always before
 * convergence is declared. */
kp_status tik_pcg(kp_ctx* ctx, const void* b, double lambda, double tol, int maxit, int flexible,
                  void* x, int warm_start, kp_solve_info* info);

/* Choose lambda in closed form over the KP spectrum (Section 2.2; eqs.
 * GCVTikSVD, wGCVTikSVD, DSCTikSVD, OptTikSVD):
 * b_hat = vec(U_c^T B U_r), x_hat = vec(V_c^T X_true V_r).
 * GCV / wGCV / OPT: minimum on lambda in [max(min|Sigma|>0, 1e-10 max|Sigma|),
 * max|Sigma|] by a 400-point grid in log lambda (one launch), the best point
 * re-checked in FP64, then refined in the two adjacent cells in FP64: GCV and
 * wGCV by safeguarded Newton on log G in log lambda from the vertex of the
 * parabola through the best point and its neighbours, OPT by golden-section
 * search (ties -> larger lambda; for wGCV with omega > 1 the range starts at
 * the root of trace(I - omega A A^+)).  DISCREPANCY: root of D(lambda)
 * (increasing) bracketed by decades in log lambda (down to 1e-16 max|Sigma|)
 * and refined by safeguarded Newton; KP_ENOROOT when no root exists (eps >=
 * ||b||, or D > 0 down to 1e-16 max|Sigma|).  KP_ENUMERIC when b (or x_true
 * for OPT) holds a NaN or Inf.  KP_EINVAL for NULL b or lambda_out, an unknown
 * method, omega <= 0, eps <= 0, or a missing x_true for OPT; KP_ESTATE before
 * kp_setup.
 *   b        device, vec type
 *   x_true   device, vec type, only for KP_LAMBDA_OPT (else NULL)
 *   lambda_out host */
kp_status choose_lambda(kp_ctx* ctx, const void* b, kp_lambda_method method, double param,
                        const void* x_true, double* lambda_out);

/* Operator hooks (asynchronous).  y = A x (transpose = 0) or y = A^T x
 * (transpose = 1) with the context's operator precision; kp_apply_K gives
 * y = (A^T A + lambda^2 I) x.  x, y: device, vec type, n_r x n_c, distinct. */
kp_status kp_apply_A(kp_ctx* ctx, const void* x, void* y, int transpose);
kp_status kp_apply_K(kp_ctx* ctx, const void* x, void* y, double lambda);

/* Preconditioner solve z = M^-1 r = V_c (S .* (V_c^T R V_r)) V_r^T with
 * S = 1 / (Sigma^2 + lambda^2) (eq. PreconSolve), in the context's
 * preconditioner precision.  r, z: device, vec type, distinct. */
kp_status kp_apply_Minv(kp_ctx* ctx, const void* r, void* z, double lambda);

/* Preconditioner solve that allocates nothing, for callers that cannot call
 * cudaMalloc: code running where the allocator is off limits (a memory
 * pool or arena owned by someone else, an embedding runtime that forbids
 * device allocation, a real-time loop that must not allocate).  It needs no
 * context: the caller passes every input and output, and the intermediates
 * go to a fixed 5 MiB scratch array inside the library (held by every GPU
 * that loads the library until the process exits).  The paper has no
 * counterpart; the arithmetic is that of kp_apply_Minv with FP32
 * preconditioner factors:
 *   z = V_c (S .* (V_c^T R V_r)) V_r^T,  S = 1 / (Sigma^2 + lambda^2).
 *   Vc       device, float, column-major n_r x n_r (right singular vectors of A_c^(1))
 *   Vr       device, float, column-major n_c x n_c (right singular vectors of A_r^(1))
 *   sigma    device, double, column-major n_r x n_c KP spectrum
 *   r, z     device, float, column-major n_r x n_c, distinct
 *   cuda_stream  cudaStream_t the work is issued on (asynchronous); it must
 *            belong to the current device (KP_EINVAL otherwise), since the
 *            scratch address is looked up for the current device
 * Limits: n_r, n_c <= 512 (KP_EINVAL beyond).  The first call on a device
 * looks up the scratch address on that device (make it before any stream
 * capture).  All calls share the scratch array and it keeps the last call's
 * contents: calls that overlap on the GPU (two streams at once) race. */
kp_status kp_apply_Minv_noalloc(const float* Vc, const float* Vr, const double* sigma, int n_r, int n_c,
                                double lambda, const float* r, float* z, void* cuda_stream);

/* Getters (synchronise; host buffers).
 *   kp_get_spectrum  sigma: n_r * n_c doubles, column-major KP spectrum
 *   kp_get_terms     s: op_rank doubles (weighted PSF singular values),
 *                    u: n_r * op_rank, v: n_c * op_rank (column m = term m;
 *                    u_m's largest-magnitude entry is positive); any may be NULL
 *   kp_get_kpsvd     sr (n_c), Vr (n_c x n_c col-major), sc (n_r), Vc (n_r x n_r),
 *                    Ur, Uc likewise; any may be NULL; singular values descending
 *   kp_get_rank      op_rank in use */
kp_status kp_get_spectrum(kp_ctx* ctx, double* sigma);
kp_status kp_get_terms(kp_ctx* ctx, double* s, double* u, double* v);
kp_status kp_get_kpsvd(kp_ctx* ctx, double* sr, double* Ur, double* Vr, double* sc, double* Uc,
                       double* Vc);
kp_status kp_get_rank(kp_ctx* ctx, int* op_rank);

/* Tuning knobs (name = value); unknown names return KP_EINVAL.
 *   "reliable_delta"  factor by which ||r|| must fall before a reliable
 *                     residual update (default 0.1 for F32 / BF16 / BF16X3
 *                     operators, 0 = off for the F64 operator)
 *   "check_every"     iterations between host convergence checks (default 2)
 *   "pc_lambda_ratio" > 0 (default 1): the preconditioner of tik_pcg uses
 *                     lambda_M = ratio * lambda (eq. PreconSystem has the
 *                     system's lambda; Section 5.3 suggests a larger one
 *                     against the error jump of the first iterations); the
 *                     solution is the same x_lambda
 *   "op_auto_cond"    > 0 (default 0 = off): with a BF16 operator, each tik_pcg
 *                     uses the BF16X3 inner operator (three bf16 pairs) when
 *                     cond(A^T A + lambda^2 I) ~ (max Sigma^2 + lambda^2) /
 *                     lambda^2 exceeds this value, else BF16 (kp_solve_batch
 *                     sets 1e4 for BF16 batches, and solves a problem again
 *                     with BF16X3 if its BF16 solve stalls or breaks down)
 *   "cg_fuse"         1 (default): with a BF16 / BF16X3 operator, an F16 / BF16
 *                     preconditioner and FP32 vectors, the x / r update also
 *                     writes the preconditioner's narrow input, scaled by a
 *                     power of two from the bound max|r| + |alpha| max|q|
 *                     (no separate quantisation pass); 0: separate pass
 *                     scaled from the exact max|r|
 *   "jacobi_tol"      one-sided Jacobi rotation threshold (default 1e-15)
 *   "jacobi_max_sweeps" (default 40)
 *   "jacobi_block"    1 (default): the FP32 Jacobi sweeps (FP32-vector setup)
 *                     in block form, each launch running a full sweep over
 *                     two blocks of 4 columns held in registers (n / 4
 *                     launches per sweep instead of n - 1) where m, n <= 1024;
 *                     0: one launch per round of column pairs
 *   "jacobi_warm_u"   1 (default): for a factor that is not symmetric, the
 *                     second Jacobi run (U, from F^T) starts from the first
 *                     run's V instead of the DCT / DST transform; 0: from the
 *                     transform
 *   "splitk"          > 0: fixed split-K factor of the square tensor-core
 *                     GEMMs (default 0 = chosen per shape)
 *   "tc_bn"           64, 128 or 256: fixed tensor-core tile width (default 0 =
 *                     chosen per shape)
 *   "tc_ctas_per_sm"  1 or 2: fixed CTAs per SM for 128-wide tiles (default 0)
 *   "tc_kblocks_per_stage" 1, 2 or 4 (4: 64-wide tiles only): k-blocks per
 *                     shared-memory ring stage (default 0 = 4 for 64-wide
 *                     tiles, 1 with two CTAs per SM, else 2)
 *   "tc_autotune"     nonzero: at kp_setup each tensor-core GEMM shape's tile
 *                     configuration (tile width, CTAs per SM, k-blocks per
 *                     stage, CTA pairs) is chosen by timing the candidates
 *                     (CUDA events, a scratch output); the choices are kept per
 *                     process and, when the environment variable
 *                     KPSVD_TUNE_CACHE names a file, read from and appended
 *                     to it (one line per shape); default 0: the built-in rule
 *   "tc_pair"         0 (default): BF16 GEMMs whose 256 x 256 tiles fill most
 *                     SM pairs run on CTA pairs (tcgen05 cta_group::2, one
 *                     256 x 256 tile per pair of SMs); 1: never; 2: wherever
 *                     the shape allows (N >= 256, per-term blocks of 256 rows)
 *   "tc_kcat"         0 (default): the second and fourth GEMM of the inner
 *                     operator as per-term products and a separate term sum
 *                     (measured faster at 1024^2); 1: where 128 x 64 tiles of
 *                     the sum over terms fill most SMs, as ONE product over
 *                     all terms (the terms summed in the tensor-memory
 *                     accumulator: no per-term outputs, no term sum), the
 *                     fourth GEMM's epilogue also reducing p^T q and max |q|;
 *                     2: the same wherever the shape allows (any size; n_r a
 *                     multiple of 256 with clusters of four)
 *   "tc_kcat_cluster" 1 (default) or 4: CTAs per cluster of those products;
 *                     4: neighbouring tiles share their A tiles by TMA
 *                     multicast
 *                     The tile options take effect at the next kp_setup.
 *   "device_loop"     1 (default): tik_pcg runs its whole iteration as one CUDA
 *                     graph with a device-side while loop (the residual
 *                     replacement in a nested conditional), no host round
 *                     trip until the solve stops; 0: blocks of check_every
 *                     iterations launched and checked by the host (also the
 *                     fallback when the device loop cannot be built)
 *   "pdl"             0: launch the iteration's kernels without programmatic
 *                     dependent launch (default 1: each kernel's launch and
 *                     prologue overlap the tail of the previous one)
 *   "pc_inner_iters"  1 .. 64 (default 2): inner PCG steps of a preconditioner
 *                     with pc_rank > 1
 *   "setup_fp64"      nonzero: keep the O(n^3) products of kp_setup and of
 *                     choose_lambda's spectral coefficients, the Jacobi
 *                     rotations and the PSF subspace iteration in FP64 also
 *                     for FP32 vectors.  By default they run in FP32 when
 *                     vec_prec is KP_F32 (Gram convergence test at FP32
 *                     tolerance), which moves the chosen lambda by ~2.5e-7
 *                     relative at 1024^2; FP64 vectors always use FP64.
 *                     Takes effect at the next kp_setup.
 *   "setup_half"      nonzero: with the FP32 setup on the tensor cores (FP32
 *                     vectors, n_r and n_c multiples of 16, "setup_fp64"
 *                     off), the products that form V_r, V_c and Sigma (the
 *                     DCT / DST transform of each factor before its Jacobi
 *                     SVD, the projected spectrum) take bf16 inputs with FP32
 *                     accumulation instead of the FP32-level three-slice
 *                     split (Section 3, after eq. PreconSolve: the
 *                     preconditioner computed, not only stored, in half
 *                     precision); the Jacobi rotations stay FP32.  Default 0.
 *                     Takes effect at the next kp_setup. */
kp_status kp_set_option(kp_ctx* ctx, const char* name, double value);

/* ---- Batched independent problems of uneven sizes ------------------------
 * Many deblurring problems, each with its own PSF, size, boundary condition,
 * b and lambda (given, or chosen per problem), solved with one set of
 * precisions and solver settings.  Not part of the paper; the batched
 * configuration of the project's workloads.  Each problem computes what
 * kp_setup, choose_lambda and tik_pcg compute for it alone.
 * Grouped form (workers <= 0, the default): one host thread; setup and
 * lambda of each problem in a cooperative fiber on the calling thread (a
 * fiber that waits for the GPU yields to the others, so the setups overlap on
 * the GPU), then the (F)PCG iterations of all problems together: every launch of the iteration (a tensor-core GEMM, a vector
 * update, a reduction) is ONE launch over all problems (GEMMs: a persistent
 * kernel over the (problem, tile) units of all problems, each problem's
 * tensor maps in a device table; vector kernels: one grid row per problem),
 * inside one CUDA graph whose device-side while loop runs until every
 * problem has stopped; a stopped problem's part of each launch does no
 * work.  Reductions may then sum their partials in another order than
 * alone (rounding-level differences).  The library keeps one context per
 * problem slot for the next call on the device (kp_batch_release frees
 * them); concurrent calls on one device are serialised.  Problems whose
 * iteration cannot run grouped (an operator or preconditioner without the
 * fused iteration) run alone after the group.
 * workers > 0: `workers` host threads each own one context (and stream) and
 * take the problems largest first.
 *   psf, b, x   device pointers as for kp_setup / tik_pcg (x: written)
 *   lambda      in: > 0 a fixed lambda; <= 0 chosen by `method` with
 *               lambda_param (choose_lambda's param); out: the lambda used
 *   info        out: the problem's solve summary (info.status = its status)
 * The caller owns every pointer; all must stay valid until the call returns. */
typedef struct {
  const double* psf;
  int n_r, n_c, center_r, center_c;
  kp_bc bc;
  int op_rank;
  const void* b;
  void* x;
  double lambda;
  double lambda_param;
  kp_solve_info info;
} kp_problem;

typedef struct {
  kp_prec op_prec, pc_prec, vec_prec;
  kp_sigma sigma;
  kp_lambda_method method; /* used for problems with lambda <= 0 */
  double tol;
  int maxit;
  int flexible;
  int workers;  /* <= 0: grouped form (one host thread); > 0: that many host threads */
  int autotune; /* grouped form, tile shapes of the grouped GEMMs: 0 = one shape for every
                   problem (128 wide; each step is then one launch), 1 = each GEMM shape's
                   chosen by timing (the tc_autotune option; cache file KPSVD_TUNE_CACHE),
                   2 = each GEMM shape's by the size rule of single solves */
} kp_batch_opts;

/* Solve probs[0..nprob) (device `device`).  Returns KP_OK when every problem
 * returned KP_OK, else the status of the first failing problem (its message
 * in kp_last_error); KP_EINVAL for NULL arguments or nprob < 0.  ms_total
 * (host, nullable): wall time of the whole batch in milliseconds. */
kp_status kp_solve_batch(int device, kp_problem* probs, int nprob, const kp_batch_opts* opts, double* ms_total);

/* Free the contexts and device table that the grouped form keeps for `device`. */
void kp_batch_release(int device);

/* How many problems the last grouped kp_solve_batch call on `device` ran in
 * its grouped loop (0 when none did); passes (nullable): that loop's passes;
 * ms (nullable, 3 doubles): host wall time of the steps before the loop
 * (setups, lambdas, starts), of recording and building the loop, and of
 * running it; shape (nullable, 6 ints): for the first epoch, the launches of
 * one problem's iteration outside the residual replacement and the grouped
 * launches they became, then the same inside the replacement; then 1 if the
 * setups ran as fibers, and how many times their waits yielded. */
int kp_batch_grouped(int device, int* passes, double* ms, int* shape);

/* ---- Learned lambda (not in the paper; Section 5 asks for a systematic
 * parameter choice) ----------------------------------------------------------
 * Spectral features of b for the context's problem: with s2 = Sigma^2 and
 * s2max = max s2, component i falls in bin j = floor(-log10(s2_i / s2max)
 * 127 / 16) when s2_i > s2max 1e-16; features[j] = log10((sum over bin j of
 * b_hat^2 + 1e-30 s2max) / (count_j + 1)), features[127 + j] =
 * log10((count_j + 1) / N) (j < 127), features[254] = log10 of the mean
 * b_hat^2 over the deepest bins that together hold >= N / 8 components (a
 * noise estimate), features[255] = log10(s2max); b_hat = vec(U_c^T B U_r).
 *   b         device, vec type;  features  device, 256 floats (written)
 * Asynchronous, except when it is the first of kp_lambda_features and
 * choose_lambda after a kp_setup: that call synchronises once to read the
 * spectrum's extremes; b is not checked (a NaN
 * or Inf in b gives non-finite features, where choose_lambda would return
 * KP_ENUMERIC). */
kp_status kp_lambda_features(kp_ctx* ctx, const void* b, float* features);

/* Multilayer perceptron features -> log10(lambda): x -> (x - mean) inv_std
 * -> [Linear(256, width) -> GELU] x depth -> Linear(width, 1); FP32 master
 * weights with bf16 copies used in the products, FP32 biases, activations
 * and accumulation; GELU(z) = z Phi(z); loss = mean squared error; Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).  The parameter vector
 * (host, kp_mlp_param_count floats) is mean (256), inv_std (256), then per
 * layer W (out x in, row-major) and the bias (out).  X: device, batch x 256
 * row-major; y, labels: device, batch floats.  Work runs on cuda_stream
 * (NULL: a private stream); set/get_params and the loss output synchronise. */
typedef struct kp_mlp kp_mlp;
kp_status kp_mlp_create(kp_mlp** out, int device, void* cuda_stream, int width, int depth, int max_batch);
void kp_mlp_destroy(kp_mlp* mlp);
long long kp_mlp_param_count(const kp_mlp* mlp);
kp_status kp_mlp_set_params(kp_mlp* mlp, const float* params); /* also resets the Adam state */
kp_status kp_mlp_get_params(kp_mlp* mlp, float* params);
kp_status kp_mlp_forward(kp_mlp* mlp, const float* X, int batch, float* y);
/* gradients (host, param_count floats; zero for mean / inv_std) and loss (host, nullable) */
kp_status kp_mlp_gradients(kp_mlp* mlp, const float* X, const float* labels, int batch, float* grads, double* loss);
kp_status kp_mlp_train_step(kp_mlp* mlp, const float* X, const float* labels, int batch, float lr, double* loss);

/* Timing of the parts of one (F)PCG iteration (a benchmark hook): each part
 * is launched `reps` times on the context's stream between CUDA events, on
 * the context's own solver vectors (r = p = the last A^T b; the caller's
 * data is not touched), and its average device time per launch goes to
 * ms[k] (host, 4 doubles); launches (host, nullable, 4 long longs) receives
 * the kernels per part:
 *   [0] the K application q = (A^T A + lambda^2 I) p as the iteration runs it
 *   [1] the preconditioner solve z = M^-1 r (eq. PreconSolve)
 *   [2] the vector phase: x / r update with ||r||^2, z^T r (and z^T r_old),
 *       beta, p = z + beta p
 *   [3] one residual replacement A^T (b - A x) - lambda^2 x with the
 *       accurate operator, and its norm
 * Synchronises.  KP_ESTATE before kp_setup; KP_EINVAL for reps < 1, lambda
 * <= 0 or ms NULL.  Meaningful after a tik_pcg on the context. */
kp_status kp_time_parts(kp_ctx* ctx, double lambda, int reps, double* ms, long long* launches);

/* Test hook for the bounded device-side waits: one kernel waits on a barrier
 * that nothing releases, bounded by limit_ms (0 < limit_ms <= 10000) of
 * device time, and gives up as every bounded wait of the library does: it
 * sets the timeout bit of the status word, and the call returns KP_ETIMEOUT.
 * The status word is cleared again, and the context stays usable.
 * Synchronises.  KP_EINVAL for a NULL context or a limit out of range.
 *
 * Fault injection (environment): KPSVD_FAULT=alloc:N makes the N-th device
 * allocation of the library after the variable was set (or changed) fail
 * with KP_ENOMEM, as a failing cudaMalloc would. */
kp_status kp_test_bounded_wait(kp_ctx* ctx, double limit_ms);

/* Number of this library's kernel launches issued on the context since the
 * last reset (reset = 1 clears it after reading). */
long long kp_launch_count(kp_ctx* ctx, int reset);

const char* kp_status_str(kp_status s);
const char* kp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* KPSVD_H */
