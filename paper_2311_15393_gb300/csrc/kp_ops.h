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
// *pq_done says whether it was (else the caller computes it).
struct PostOp;
kp_status op_apply_K(kp_ctx* ctx, const void* p, void* q, double lam2, bool p_slices_ready, const int* flags,
                     double* pq_out = nullptr, const PostOp* pq_post = nullptr, bool* pq_done = nullptr);

// r = A^T (b - A x) - lam2 x with the accurate operator
kp_status op_true_residual(kp_ctx* ctx, const void* b, const void* x, void* r, double lam2, const int* flags);

// z = M^-1 r.  `stat` points to device [||r||^2, amax(r)] when known (else
// computed here); `inv_slot` is a device float used for the output scale.
kp_status pc_apply(kp_ctx* ctx, const void* r, void* z, double lam2, const double* stat, const int* flags);

// number of bf16 slices the inner operator wants for p (0 for SIMT operators)
int op_inner_slices(kp_ctx* ctx);
