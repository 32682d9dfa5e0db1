// Operator and preconditioner applications on device images (kp_ops.cu).
#pragma once
#include "kp_internal.h"

enum OpMode : int { OP_INNER = 0, OP_ACCURATE = 1 };

// workspaces + tensor-core plans for the current problem
kp_status ops_prepare(kp_ctx* ctx);

// y = A x (transpose = 0) or A^T x, vec-type images
kp_status op_apply(kp_ctx* ctx, const void* x, void* y, int transpose, int mode);

// q = (A^T A + lam2 I) p in the inner operator precision.  For tensor-core
// operators `p_slices_ready` says the bf16 slices of p are already in
// ctx->w_img2 (written by the p update); otherwise they are made here.
// With pq_out, p^T q may be computed on the way (and pq_post run on it);
// *pq_done says whether it was (else the caller computes it).  With qmax,
// max |q| goes to pq_out[1] as well (only when *pq_done).
struct PostOp;
// `terms` > 0: the operator of the first `terms` Kronecker terms only (the
// multi-term preconditioner's inner system); 0: all of them.
kp_status op_apply_K(kp_ctx* ctx, const void* p, void* q, double lam2, bool p_slices_ready, const int* flags,
                     double* pq_out = nullptr, const PostOp* pq_post = nullptr, bool* pq_done = nullptr,
                     bool qmax = false, int terms = 0);

// r = A^T (b - A x) - lam2 x with the accurate operator
kp_status op_true_residual(kp_ctx* ctx, const void* b, const void* x, void* r, double lam2, const int* flags);

// z = M^-1 r (pc_rank 1: the KP-SVD solve of eq. PreconSolve; pc_rank > 1:
// pc_inner_iters PCG steps on the first pc_rank terms, see kp_ops.cu).
// `stat` points to device [||r||^2, amax(r)] when known (else
// computed here); `inv_slot` is a device float used for the output scale.
// narrow_ready (F16 / BF16 preconditioners): ctx->pc_in and the inverse
// scale slot already hold the narrow copy of r (written by the x / r update).
kp_status pc_apply(kp_ctx* ctx, const void* r, void* z, double lam2, const double* stat, const int* flags,
                   bool narrow_ready = false);

// the preconditioner's narrow input made from r, as pc_apply makes it when
// it is not made by the x / r update (F16 / BF16 one-term preconditioners)
kp_status pc_prepare_input(kp_ctx* ctx, const void* r, double lam2, const double* stat, const int* flags);

// number of bf16 slices the inner operator wants for p (0 for SIMT operators)
int op_inner_slices(kp_ctx* ctx);

// switch a tensor-core operator's inner precision between BF16 (one factor x
// activation pair) and BF16X3 (three pairs of the same bf16 slices); the
// plans of each variant are built once per setup
kp_status ops_set_inner(kp_ctx* ctx, kp_prec p);

// ---- folded quantisation (tensor-core operator with batched term sums,
// F16 / BF16 preconditioner, FP32 vectors): the K application's term sum
// also gives max |q|, and the x / r update writes the preconditioner's
// narrow input with a scale bounded from max |r_old| + |alpha| max |q|
bool cg_fusable(kp_ctx* ctx);
// the inverse-scale slot of the narrow preconditioner input
float* cg_inv_slot(kp_ctx* ctx);
