// tik_pcg: preconditioned CG / flexible PCG on (A^T A + lam^2 I) x = A^T b
// (eq. tik:normal2), KP-SVD preconditioner with the same lambda
// (eq. PreconSystem), Fletcher-Reeves beta (PCG) or Polak-Ribiere beta
// (flexible PCG; Section 3, last paragraph).
//
// All scalars (alpha, beta, inner products, norms) are FP64 values in device
// memory; the host never waits inside an iteration.  Iterations run in
// blocks of `check_every`, captured once per solve as a CUDA graph.  Each
// kernel returns at once while the device pause flag is set; the flag is
// raised on convergence of the recurred residual, when a reliable residual
// update is due, at maxit, or on breakdown / NaN.  The host reads the flags
// after each block and acts (replace the residual, stop).
//
// Reliable updates: with a reduced-precision operator the recurred residual
// drifts from the true one, by about the operator's rounding error times
// cond(A^T A + lam^2 I).  Whenever ||r|| has fallen by `reliable_delta`
// since the last replacement, and before convergence is declared, r is
// replaced by A^T (b - A x) - lam^2 x computed with the FP32-accurate
// operator; the search direction is kept.
#include <algorithm>
#include <cmath>
#include <vector>

#include "kp_group.cuh"
#include "kp_internal.h"
#include "kp_ops.h"
#include "kp_vec.cuh"


namespace {
// after a reliable update: record ||r_true|| in the history and either
// resume (clear the pause), stop as converged (the true residual meets the
// tolerance: F_REASON = R_CONV | R_TRUE), or stop as stagnated (R_STAGNATE:
// three replacements in a row that did not halve the true residual, i.e.
// the attainable accuracy of the FP32 vectors and the accurate operator is
// reached above the tolerance)
constexpr int R_TRUE = 32;
constexpr int R_STAGNATE = 64;
constexpr int STAG_REPLACEMENTS = 3;
__global__ void k_after_replace(double* s, int* f, double* hist, int hist_cap) {
  const double rr = s[S_RR];
  const int it = f[F_ITER];
  if (it < hist_cap) hist[it] = sqrt(rr / s[S_RR0]);
  const double prev = s[S_RTPREV];
  f[F_STAG] = (prev > 0.0 && rr > 0.25 * prev) ? f[F_STAG] + 1 : 0;
  f[F_SINCE] = 0;
  s[S_RTPREV] = rr;
  if (rr <= s[S_TOL2]) {
    f[F_REASON] = R_CONV | R_TRUE;
    f[F_PAUSE] = 1;
  } else if (f[F_STAG] >= STAG_REPLACEMENTS) {
    f[F_REASON] = R_STAGNATE;
    f[F_PAUSE] = 1;
  } else {
    f[F_REASON] = 0;
    f[F_PAUSE] = 0;
  }
}
}  // namespace

// ---------------------------------------------------------------- device-side loop
// The iteration as a CUDA graph while loop, with the residual replacement in
// a nested if: per iteration half_a, whose x / r update ends (in the last
// block of its reduction) by deciding whether a replacement is due (the
// reliable-update rule, or a convergence / maxit stop with a reduced-
// precision operator) and whether the loop goes on; then, if due, the
// replacement and k_loop_after_replace (which decides the loop); then half_b
// (whose kernels skip when a stop is flagged).  The host launches the graph
// once and reads the flags after it.
// after a replacement: k_after_replace's rule, a maxit stop stays a stop
// (batched loop: `flags` is the problem's skip word, F_NOTDUE, and the
// decision goes to F_BLOOP for the loop's own condition kernel)
__device__ __forceinline__ void k_loop_after_replace_body(double* s, int* f, double* hist, int hist_cap,
                                                          cudaGraphConditionalHandle h_loop, const int* flags,
                                                          int batch) {
  KP_PDL_WAIT();
  KP_PDL_TRIGGER();
  if (flags && *(volatile const int*)flags) return;
  const double rr = s[S_RR];
  const int it = f[F_ITER];
  if (it < hist_cap) hist[it] = sqrt(rr / s[S_RR0]);
  const double prev = s[S_RTPREV];
  f[F_STAG] = (prev > 0.0 && rr > 0.25 * prev) ? f[F_STAG] + 1 : 0;
  f[F_SINCE] = 0;
  f[F_REPL] += 1;
  s[S_RTPREV] = rr;
  if (rr <= s[S_TOL2]) {
    f[F_REASON] = R_CONV | R_TRUE;
    f[F_PAUSE] = 1;
  } else if (f[F_STAG] >= STAG_REPLACEMENTS && !(f[F_SAVED] & R_MAXIT)) {
    f[F_REASON] = R_STAGNATE;
    f[F_PAUSE] = 1;
  } else if (f[F_SAVED] & R_MAXIT) {
    f[F_REASON] = R_MAXIT;
    f[F_PAUSE] = 1;
  } else {
    f[F_REASON] = 0;
    f[F_PAUSE] = 0;
  }
  const unsigned int go = (f[F_PAUSE] || f[F_GUARD] > f[F_MAXIT] + 8) ? 0u : 1u;
  if (batch) {
    f[F_BLOOP] = (int)go;
    if (!go) f[F_PAUSE] = 1;
  } else {
    cudaGraphSetConditional(h_loop, go);
  }
}
__global__ void k_loop_after_replace(double* s, int* f, double* hist, int hist_cap, cudaGraphConditionalHandle h_loop,
                                     const int* flags, int batch) {
  k_loop_after_replace_body(s, f, hist, hist_cap, h_loop, flags, batch);
}
KP_BODY(AfterReplace, k_loop_after_replace_body);

// dst = src (one scalar), unless flagged
__device__ __forceinline__ void k_copy_scalar_body(double* dst, const double* src, const int* flags) {
  KP_PDL_WAIT();
  KP_PDL_TRIGGER();
  if (flags && *(volatile const int*)flags) return;
  if (threadIdx.x == 0) *dst = *src;
}
__global__ void k_copy_scalar(double* dst, const double* src, const int* flags) { k_copy_scalar_body(dst, src, flags); }
KP_BODY(CopyScalar, k_copy_scalar_body);

struct SolveBufs {
  void *r, *r_old, *p, *q, *z, *rhs;
};

static SolveBufs bufs(kp_ctx* ctx) {
  SolveBufs b;
  b.r = ctx->vbuf[0];
  b.r_old = ctx->vbuf[1];
  b.p = ctx->vbuf[2];
  b.q = ctx->vbuf[3];
  b.z = ctx->vbuf[4];
  b.rhs = ctx->vbuf[5];
  return b;
}

// conditions of the loop graph, set by the x / r update's last block
struct LoopConds {
  cudaGraphConditionalHandle h_rep = 0, h_loop = 0;
  int mode = 1;  // PostOp::cond: 1 device loop, 2 batched loop
};

// first half of an iteration: q = K p, alpha, x/r update, convergence flags
static kp_status half_a(kp_ctx* ctx, const SolveBufs& B, void* x, double lam2, const LoopConds* lc) {
  const long long N = (long long)ctx->n_r * ctx->n_c;
  const bool f64 = ctx->vec_prec == KP_F64;
  const int* fl = ctx->dflags;
  double* s = ctx->dscal;
  PostOp pa;  // alpha = zr / p^T K p, by the last block of the dot product
  pa.kind = POST_ALPHA;
  pa.s = s;
  pa.f = ctx->dflags;
  PostOp pc = pa;  // iteration count, history and stopping flags, after the update
  pc.kind = POST_CHECK;
  pc.hist = ctx->hist;
  pc.hist_cap = ctx->hist_cap;
  if (lc) {
    pc.cond = lc->mode;
    pc.h_rep = lc->h_rep;
    pc.h_loop = lc->h_loop;
  }
  bool fused = false;
  KP_TRY(op_apply_K(ctx, B.p, B.q, lam2, op_inner_slices(ctx) > 0, fl, s + S_PQ, &pa, &fused));
  if (!fused) KP_TRY(dot2_dev(ctx, B.p, B.q, nullptr, N, f64, s + S_PQ, fl, pa));
  KP_TRY(update_xr_dev(ctx, x, B.r, B.r_old, B.p, B.q, N, f64, s + S_ALPHA, s + S_RR, fl, pc));
  KP_CUDA(cudaGetLastError());
  return KP_OK;
}

// second half: z = M^-1 r, beta, p = z + beta p (+ bf16 slices of p)
// (narrow_ready: the narrow copy of r for the preconditioner is already made)
static kp_status half_b(kp_ctx* ctx, const SolveBufs& B, double lam2_pc, bool narrow_ready) {
  const long long N = (long long)ctx->n_r * ctx->n_c;
  const bool f64 = ctx->vec_prec == KP_F64;
  const int* fl = ctx->dflags;
  double* s = ctx->dscal;
  KP_TRY(pc_apply(ctx, B.r, B.z, lam2_pc, s + S_RR, fl, narrow_ready));
  PostOp pb;  // beta and zr, by the last block of the dot products
  pb.kind = POST_BETA;
  pb.s = s;
  pb.f = ctx->dflags;
  KP_TRY(dot2_dev(ctx, B.z, B.r, B.r_old, N, f64, s + S_ZRNEW, fl, pb));
  const int sl = op_inner_slices(ctx);
  KP_TRY(p_update_dev(ctx, B.p, B.z, N, f64, s + S_BETA, sl ? (__nv_bfloat16*)ctx->w_img2 : nullptr, sl, N, fl));
  return KP_OK;
}

// The first half with the quantisation of r folded into the x / r update
// (cg_fusable): the K application's term sum also gives max |q|, so the
// update writes the preconditioner's narrow input with a scale bounded from
// max |r_old| + |alpha| max |q| >= max |r_new|, known before the update.
static kp_status half_a_folded(kp_ctx* ctx, const SolveBufs& B, void* x, double lam2, double lam2_pc,
                               const LoopConds* lc) {
  const long long N = (long long)ctx->n_r * ctx->n_c;
  const int* fl = ctx->dflags;
  double* s = ctx->dscal;
  PostOp pa;
  pa.kind = POST_ALPHA;
  pa.s = s;
  pa.f = ctx->dflags;
  PostOp pc = pa;
  pc.kind = POST_CHECK;
  pc.hist = ctx->hist;
  pc.hist_cap = ctx->hist_cap;
  if (lc) {
    pc.cond = lc->mode;
    pc.h_rep = lc->h_rep;
    pc.h_loop = lc->h_loop;
  }
  bool fused = false;
  KP_TRY(op_apply_K(ctx, B.p, B.q, lam2, true, fl, s + S_QPQ, &pa, &fused, true));
  if (!fused) {
    kp_set_error("tik_pcg: folded iteration without a fused term sum");
    return KP_ENOTSUP;
  }
  const int nt = ctx->pc_prec == KP_BF16 ? NT_BF16 : NT_F16;
  KP_TRY(update_xr_q_dev(ctx, x, B.r, B.r_old, B.p, B.q, N, s + S_ALPHA, s + S_RR, s + S_QMAX, nt, lam2_pc, ctx->pc_in,
                         cg_inv_slot(ctx), fl, pc));
  return KP_OK;
}

struct HostFlags {
  int pause, reason, iter, maxit, flex;
};

static kp_status read_flags(kp_ctx* ctx, HostFlags* h, double* hs) {
  KP_CUDA(cudaMemcpyAsync(h, ctx->dflags, sizeof(HostFlags), cudaMemcpyDeviceToHost, ctx->stream));
  if (hs) KP_CUDA(cudaMemcpyAsync(hs, ctx->dscal, 12 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  KP_CUDA(kp_wait(ctx, ctx->stream));
  return KP_OK;
}

static kp_status set_scalar(kp_ctx* ctx, int slot, double v) {
  KP_CUDA(cudaMemcpyAsync(ctx->dscal + slot, &v, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  KP_CUDA(kp_wait(ctx, ctx->stream));  // v is a host stack value
  return KP_OK;
}

// replace r by the true residual; returns its ||r||^2 via the RR / RMAX slots
// (`flags`: skip word of a batched loop's replacement, else null)
static kp_status replace_residual(kp_ctx* ctx, const SolveBufs& B, const void* b, const void* x, double lam2,
                                  const int* flags = nullptr) {
  const long long N = (long long)ctx->n_r * ctx->n_c;
  KP_TRY(op_true_residual(ctx, b, x, B.r, lam2, flags));
  KP_TRY(norm_amax_dev(ctx, B.r, N, ctx->vec_prec == KP_F64, ctx->dscal + S_RR, flags));
  if (flags) {
    KP_CUDA(kp_launch_g<CopyScalar>(ctx, k_copy_scalar, dim3(1), dim3(32), 0, ctx->dscal + S_RMAX,
                                    (const double*)ctx->dscal + S_RR, flags));
    KP_LAUNCHED(ctx);
  } else {
    KP_CUDA(cudaMemcpyAsync(ctx->dscal + S_RMAX, ctx->dscal + S_RR, sizeof(double), cudaMemcpyDeviceToDevice,
                            ctx->stream));
  }
  return KP_OK;
}

// ---- the device-side loop graph (see k_loop_after_replace)
struct LoopGraph {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long launches_body = 0, launches_replace = 0;
  ~LoopGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (g) cudaGraphDestroy(g);
  }
};

struct LoopConds;
static kp_status half_a(kp_ctx* ctx, const SolveBufs& B, void* x, double lam2, const LoopConds* lc);
static kp_status half_b(kp_ctx* ctx, const SolveBufs& B, double lam2_pc, bool narrow_ready);
static kp_status half_a_folded(kp_ctx* ctx, const SolveBufs& B, void* x, double lam2, double lam2_pc,
                               const LoopConds* lc);

static kp_status build_loop_graph(kp_ctx* ctx, const SolveBufs& B, const void* b, void* x, double lam2, double lam2_pc,
                                  bool reliable, bool folded, LoopGraph* L) {
  cudaStream_t st = ctx->stream;
  if (!ctx->aux_stream) KP_CUDA(cudaStreamCreateWithFlags(&ctx->aux_stream, cudaStreamNonBlocking));
  KP_CUDA(cudaGraphCreate(&L->g, 0));
  cudaGraphConditionalHandle h_loop, h_rep;
  KP_CUDA(cudaGraphConditionalHandleCreate(&h_loop, L->g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams wp = {};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = h_loop;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wnode;
  KP_CUDA(cudaGraphAddNode(&wnode, L->g, nullptr, nullptr, 0, &wp));
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  KP_CUDA(cudaGraphConditionalHandleCreate(&h_rep, body, 0, 0));
  const long long l0 = ctx->launches;
  KP_CUDA(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  LoopConds lc;
  lc.h_rep = h_rep;
  lc.h_loop = h_loop;
  (void)reliable;  // the update's last block reads it from the tolerance slots
  kp_status cs = folded ? half_a_folded(ctx, B, x, lam2, lam2_pc, &lc) : half_a(ctx, B, x, lam2, &lc);
  cudaGraph_t ibody = nullptr;
  bool aux_capturing = false;
  if (cs == KP_OK) {
    cudaStreamCaptureStatus cst;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* ed = nullptr;
    size_t nd = 0;
    cudaGraphNodeParams ip = {};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = h_rep;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t inode;
    cudaError_t e = cudaStreamGetCaptureInfo(st, &cst, nullptr, &cg, &deps, &ed, &nd);
    if (e == cudaSuccess) e = cudaGraphAddNode(&inode, cg, deps, ed, nd, &ip);
    if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(st, &inode, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess) {
      ibody = ip.conditional.phGraph_out[0];
      e = cudaStreamBeginCaptureToGraph(ctx->aux_stream, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    }
    if (e != cudaSuccess) {
      kp_set_error("tik_pcg: loop graph: %s", cudaGetErrorString(e));
      cs = KP_ECUDA;
    } else {
      aux_capturing = true;
      // the replacement (and the preconditioner input from the new r) in the if body
      const long long l1 = ctx->launches;
      ctx->stream = ctx->aux_stream;
      cs = replace_residual(ctx, B, b, x, lam2);
      if (cs == KP_OK) {
        k_loop_after_replace<<<1, 1, 0, ctx->stream>>>(ctx->dscal, ctx->dflags, ctx->hist, ctx->hist_cap, h_loop,
                                                       nullptr, 0);
        KP_LAUNCHED(ctx);
        if (folded) cs = pc_prepare_input(ctx, B.r, lam2_pc, ctx->dscal + S_RR, nullptr);
      }
      ctx->stream = st;
      L->launches_replace = ctx->launches - l1;
      cudaGraph_t tmp = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(ctx->aux_stream, &tmp);
      aux_capturing = false;
      if (cs == KP_OK && e2 != cudaSuccess) {
        kp_set_error("tik_pcg: loop graph (replacement): %s", cudaGetErrorString(e2));
        cs = KP_ECUDA;
      }
    }
  }
  if (cs == KP_OK) cs = half_b(ctx, B, lam2_pc, folded);
  if (aux_capturing) {
    cudaGraph_t tmp = nullptr;
    cudaStreamEndCapture(ctx->aux_stream, &tmp);
  }
  cudaGraph_t tmp = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(st, &tmp);
  L->launches_body = ctx->launches - l0 - L->launches_replace;
  ctx->launches = l0;
  if (cs != KP_OK) return cs;
  if (ee != cudaSuccess) {
    kp_set_error("tik_pcg: loop graph capture: %s", cudaGetErrorString(ee));
    return KP_ECUDA;
  }
  KP_CUDA(cudaGraphInstantiate(&L->exec, L->g, 0));
  return KP_OK;
}

// With op_auto_cond > 0 and a BF16 operator: the inner operator of this solve
// is BF16X3 when cond(A^T A + lam^2 I) ~ (max Sigma^2 + lam^2) / lam^2
// exceeds op_auto_cond (the BF16 inner operator's rounding, ~2^-8, then
// stalls or breaks the recurrences; BF16X3's is ~2^-16), else BF16.
static kp_status choose_inner(kp_ctx* ctx, double lam2) {
  if (!(ctx->op_auto_cond > 0) || ctx->op_prec_setup != KP_BF16) return KP_OK;
  if (ctx->sigma_max < 0) {
    double h[2];
    KP_TRY(norm_amax_dev(ctx, ctx->Sigma64, (long long)ctx->n_r * ctx->n_c, true, ctx->dscal + S_RR));
    KP_CUDA(cudaMemcpyAsync(h, ctx->dscal + S_RR, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    KP_CUDA(kp_wait(ctx, ctx->stream));
    ctx->sigma_max = h[1];
  }
  const double cond = (ctx->sigma_max * ctx->sigma_max + lam2) / lam2;
  return ops_set_inner(ctx, cond > ctx->op_auto_cond ? KP_BF16X3 : KP_BF16);
}

// One solve's state between its steps: the steps before the loop
// (solve_begin), the loop (on the device, on the host, or as part of a
// batched loop), and the results (solve_finish).
struct SolveRun {
  const void* b = nullptr;
  void* x = nullptr;
  SolveBufs B;
  double lam2 = 0.0, lam2_pc = 0.0, rr0 = 0.0, final_rr = 0.0;
  bool f64 = false, reliable = false, folded = false;
  int maxit = 0, iters = 0, repl = 0;
  kp_status result = KP_OK;
  bool need_loop = false;  // the iterations are still to run
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};

// Everything before the iterations: flags, A^T b and its norm, x0 / r0 (or
// the true residual of a warm start), and z0 = M^-1 r0, p0 = z0 when the
// start does not already meet the tolerance (then R->need_loop).
static kp_status solve_begin(kp_ctx* ctx, const void* b, double lambda, double tol, int maxit, int flexible, void* x,
                             int warm_start, SolveRun* R) {
  const long long N = (long long)ctx->n_r * ctx->n_c;
  KP_TRY(choose_inner(ctx, lambda * lambda));
  const bool f64 = ctx->vec_prec == KP_F64;
  const double lam2 = lambda * lambda;
  // the preconditioner's lambda (eq. PreconSystem uses the system's; a larger
  // one is the remedy Section 5.3 suggests for the early error jump)
  const double lam2_pc = lam2 * ctx->pc_lambda_ratio * ctx->pc_lambda_ratio;
  const SolveBufs B = bufs(ctx);
  cudaStream_t st = ctx->stream;
  // default: reliable updates for every operator below FP64
  double delta = ctx->reliable_delta >= 0 ? ctx->reliable_delta : (ctx->op_prec == KP_F64 ? 0.0 : 0.1);
  const bool reliable = delta > 0.0;
  R->b = b;
  R->x = x;
  R->B = B;
  R->lam2 = lam2;
  R->lam2_pc = lam2_pc;
  R->f64 = f64;
  R->reliable = reliable;
  R->folded = cg_fusable(ctx);
  R->maxit = maxit;
  R->need_loop = false;
  R->result = KP_OK;

  KP_CUDA(cudaEventCreate(&R->e0));
  KP_CUDA(cudaEventCreate(&R->e1));
  KP_CUDA(cudaEventRecord(R->e0, st));
  KP_CUDA(cudaMemsetAsync(ctx->dflags, 0, 64, st));
  KP_CUDA(cudaMemsetAsync(ctx->dev_status, 0, sizeof(int), st));
  {
    int hf[5] = {0, 0, 0, maxit, flexible ? 1 : 0};
    KP_CUDA(cudaMemcpyAsync(ctx->dflags, hf, sizeof(hf), cudaMemcpyHostToDevice, st));
    KP_CUDA(kp_wait(ctx, st));
  }
  // rhs = A^T b (accurate operator) and its norm
  KP_TRY(op_apply(ctx, b, B.rhs, 1, OP_ACCURATE));
  KP_TRY(dot2_dev(ctx, B.rhs, B.rhs, nullptr, N, f64, ctx->dscal + S_RR0, nullptr));
  HostFlags hf;
  double hs[12];
  KP_TRY(read_flags(ctx, &hf, hs));
  const double rr0 = hs[S_RR0];
  R->rr0 = rr0;
  if (!(rr0 > 0.0) || !std::isfinite(rr0)) {
    if (!std::isfinite(rr0)) {
      kp_set_error("tik_pcg: A^T b is not finite");
      R->result = KP_ENUMERIC;
    } else {
      KP_CUDA(cudaMemsetAsync(x, 0, N * (f64 ? 8 : 4), st));
    }
    return KP_OK;
  }
  KP_TRY(set_scalar(ctx, S_TOL2, tol * tol * rr0));
  KP_TRY(set_scalar(ctx, S_DELTA2, reliable ? delta * delta : 0.0));
  if (warm_start) {
    KP_TRY(replace_residual(ctx, B, b, x, lam2));
  } else {
    KP_CUDA(cudaMemsetAsync(x, 0, N * (f64 ? 8 : 4), st));
    KP_TRY(copy_vec(ctx, B.rhs, B.r, N, f64));
    KP_TRY(norm_amax_dev(ctx, B.r, N, f64, ctx->dscal + S_RR));
    KP_CUDA(cudaMemcpyAsync(ctx->dscal + S_RMAX, ctx->dscal + S_RR, 8, cudaMemcpyDeviceToDevice, st));
  }
  KP_CUDA(cudaMemcpyAsync(ctx->dscal + S_RTPREV, ctx->dscal + S_RR, 8, cudaMemcpyDeviceToDevice, st));
  KP_TRY(read_flags(ctx, &hf, hs));
  double h0 = std::sqrt(hs[S_RR] / rr0);
  KP_CUDA(cudaMemcpyAsync(ctx->hist, &h0, sizeof(double), cudaMemcpyHostToDevice, st));
  R->final_rr = hs[S_RR];
  if (hs[S_RR] <= tol * tol * rr0) return KP_OK;  // converged at the start
  // z0 = M^-1 r0, zr, p0 = z0
  KP_TRY(pc_apply(ctx, B.r, B.z, lam2_pc, ctx->dscal + S_RR, nullptr));
  KP_TRY(dot2_dev(ctx, B.z, B.r, nullptr, N, f64, ctx->dscal + S_ZR, nullptr));
  const int sl = op_inner_slices(ctx);
  KP_TRY(p_update_dev(ctx, B.p, B.z, N, f64, nullptr, sl ? (__nv_bfloat16*)ctx->w_img2 : nullptr, sl, N, nullptr));
  KP_CUDA(kp_wait(ctx, st));  // h0 is a host stack value
  R->need_loop = true;
  return KP_OK;
}

// the solve's status from the flags of a device-side (or batched) loop
static void loop_result(SolveRun* R, const int* fl) {
  const int reason = fl[F_REASON];
  const int iters = R->iters;
  const double rel = std::sqrt(R->final_rr / R->rr0);
  if (reason & R_NUMERIC) {
    kp_set_error("tik_pcg: NaN / Inf at iteration %d", iters);
    R->result = KP_ENUMERIC;
  } else if (reason & R_BREAKDOWN) {
    kp_set_error("tik_pcg: breakdown (p^T K p <= 0 or z^T r <= 0) at iteration %d", iters);
    R->result = KP_EBREAKDOWN;
  } else if (reason & R_TRUE) {
    R->result = KP_OK;
  } else if (reason & R_STAGNATE) {
    R->result = KP_ENOCONV;
    kp_set_error("tik_pcg: stagnated at ||r||/||A^T b|| = %.3e (iteration %d): the tolerance is below the "
                 "attainable accuracy of this precision", rel, iters);
  } else if (reason & R_MAXIT) {
    R->result = KP_ENOCONV;
    kp_set_error("tik_pcg: maxit %d reached, ||r||/||A^T b|| = %.3e", R->maxit, rel);
  } else if (reason & R_CONV) {
    R->result = KP_OK;
  } else {
    R->result = KP_ENOCONV;
    kp_set_error("tik_pcg: the device loop ended without a stop reason (iteration %d)", iters);
  }
}

// after the loop: timing, the device status word, the info record
static kp_status solve_finish(kp_ctx* ctx, SolveRun* R, kp_solve_info* info) {
  KP_CUDA(cudaEventRecord(R->e1, ctx->stream));
  KP_CUDA(cudaEventSynchronize(R->e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, R->e0, R->e1);
  cudaEventDestroy(R->e0);
  cudaEventDestroy(R->e1);
  R->e0 = R->e1 = nullptr;
  kp_status result = R->result;
  kp_status dst = read_status(ctx);
  if (dst != KP_OK) result = dst;
  if (info) {
    info->iters = R->iters;
    info->replacements = R->repl;
    info->rel_res = R->rr0 > 0 ? std::sqrt(R->final_rr / R->rr0) : 0.0;
    info->status = result;
    info->ms_solve = ms;
    info->ms_setup = ctx->last_setup_ms;
    if (info->res_hist && info->res_hist_len > 0) {
      int n = std::min(info->res_hist_len, std::min(R->iters + 1, ctx->hist_cap));
      KP_CUDA(cudaMemcpy(info->res_hist, ctx->hist, sizeof(double) * n, cudaMemcpyDeviceToHost));
    }
  }
  return result;
}

static kp_status tik_pcg_impl(kp_ctx* ctx, const void* b, double lambda, double tol, int maxit, int flexible, void* x,
                              int warm_start, kp_solve_info* info) {
  SolveRun R;
  {
    const kp_status bs = solve_begin(ctx, b, lambda, tol, maxit, flexible, x, warm_start, &R);
    if (bs != KP_OK) {
      if (R.e0) cudaEventDestroy(R.e0);
      if (R.e1) cudaEventDestroy(R.e1);
      return bs;
    }
  }
  const long long N = (long long)ctx->n_r * ctx->n_c;
  const bool f64 = R.f64;
  const double lam2 = R.lam2, lam2_pc = R.lam2_pc;
  const bool reliable = R.reliable, folded = R.folded;
  const SolveBufs B = R.B;
  cudaStream_t st = ctx->stream;
  const double rr0 = R.rr0;
  kp_status result = R.result;
  int iters = 0, repl = 0;
  double final_rr = R.final_rr;
  HostFlags hf;
  double hs[12];
  (void)N;
  (void)f64;
  if (R.need_loop) {
    {
      bool done_device = false;
      if (ctx->device_loop) {
        // the whole loop on the device (one graph launch); on any failure
        // to build it, the host-driven loop below
        LoopGraph L;
        const kp_status bs = build_loop_graph(ctx, B, b, x, lam2, lam2_pc, reliable, folded, &L);
        if (bs == KP_OK) {
          KP_CUDA(cudaGraphLaunch(L.exec, st));
          int fl[16];
          KP_CUDA(cudaMemcpyAsync(fl, ctx->dflags, sizeof(fl), cudaMemcpyDeviceToHost, st));
          KP_CUDA(cudaMemcpyAsync(hs, ctx->dscal, 12 * sizeof(double), cudaMemcpyDeviceToHost, st));
          KP_CUDA(cudaStreamSynchronize(st));
          iters = fl[F_ITER];
          repl = fl[F_REPL];
          final_rr = hs[S_RR];
          ctx->launches += (long long)fl[F_GUARD] * L.launches_body + (long long)repl * L.launches_replace;
          R.iters = iters;
          R.final_rr = final_rr;
          loop_result(&R, fl);
          result = R.result;
          done_device = true;
        } else {
          cudaGetLastError();  // a capture error is not sticky; use the host loop
        }
      }
      if (!done_device) {
      // capture one block of iterations
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      const int blk = std::max(1, ctx->check_every);
      long long l0 = ctx->launches;
      KP_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      kp_status cs = KP_OK;
      for (int i = 0; i < blk && cs == KP_OK; ++i) {
        cs = folded ? half_a_folded(ctx, B, x, lam2, lam2_pc, nullptr) : half_a(ctx, B, x, lam2, nullptr);
        if (cs == KP_OK) cs = half_b(ctx, B, lam2_pc, folded);
      }
      cudaError_t ce = cudaStreamEndCapture(st, &graph);
      const long long per_block = ctx->launches - l0;
      ctx->launches = l0;
      if (cs != KP_OK) return cs;
      if (ce != cudaSuccess) {
        kp_set_error("tik_pcg: graph capture failed: %s", cudaGetErrorString(ce));
        return KP_ECUDA;
      }
      KP_CUDA(cudaGraphInstantiate(&exec, graph, 0));
      // Blocks are launched one ahead: while block k runs, block k + 1 is
      // queued, and the host inspects block k's flags (copied to pinned
      // memory behind it) without leaving the GPU idle.  If block k paused,
      // block k + 1 runs as no-ops (every kernel sees the pause flag).
      struct Mirror {
        HostFlags f;
        int pad[3];
        double s[12];
      };
      if (!ctx->hmirror) KP_CUDA(cudaHostAlloc(&ctx->hmirror, 2 * sizeof(Mirror), cudaHostAllocDefault));
      for (auto& e : ctx->ev_blk)
        if (!e) KP_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      Mirror* mir = static_cast<Mirror*>(ctx->hmirror);
      auto launch_block = [&](int slot) -> kp_status {
        KP_CUDA(cudaGraphLaunch(exec, st));
        ctx->launches += per_block;
        KP_CUDA(cudaMemcpyAsync(&mir[slot].f, ctx->dflags, sizeof(HostFlags), cudaMemcpyDeviceToHost, st));
        KP_CUDA(cudaMemcpyAsync(mir[slot].s, ctx->dscal, 12 * sizeof(double), cudaMemcpyDeviceToHost, st));
        KP_CUDA(cudaEventRecord(ctx->ev_blk[slot], st));
        return KP_OK;
      };
      int cur = 0;
      KP_TRY(launch_block(cur));
      bool done = false;
      while (!done) {
        KP_TRY(launch_block(cur ^ 1));
        KP_CUDA(cudaEventSynchronize(ctx->ev_blk[cur]));
        hf = mir[cur].f;
        std::copy(mir[cur].s, mir[cur].s + 12, hs);
        if (!hf.pause) {
          cur ^= 1;
          continue;
        }
        KP_CUDA(cudaStreamSynchronize(st));  // drain the no-op block behind it
        iters = hf.iter;
        final_rr = hs[S_RR];
        if (hf.reason & R_NUMERIC) {
          kp_set_error("tik_pcg: NaN / Inf at iteration %d", iters);
          result = KP_ENUMERIC;
          break;
        }
        if (hf.reason & R_BREAKDOWN) {
          kp_set_error("tik_pcg: breakdown (p^T K p <= 0 or z^T r <= 0) at iteration %d", iters);
          result = KP_EBREAKDOWN;
          break;
        }
        if (hf.reason & R_TRUE) {  // converged on a true residual computed without a host check
          result = KP_OK;
          break;
        }
        if (hf.reason & R_STAGNATE) {
          result = KP_ENOCONV;
          kp_set_error("tik_pcg: stagnated at ||r||/||A^T b|| = %.3e (iteration %d): the tolerance is below the "
                       "attainable accuracy of this precision", std::sqrt(final_rr / rr0), iters);
          break;
        }
        if (hf.reason == R_REPLACE) {
          // reliable update in the middle of the run: replace, check and
          // resume on the device, with no host round trip
          KP_TRY(replace_residual(ctx, B, b, x, lam2));
          ++repl;
          k_after_replace<<<1, 1, 0, st>>>(ctx->dscal, ctx->dflags, ctx->hist, ctx->hist_cap);
          KP_LAUNCHED(ctx);
          KP_TRY(half_b(ctx, B, lam2_pc, false));
          cur = 0;
          KP_TRY(launch_block(cur));
          continue;
        }
        bool need_replace = reliable && (hf.reason & (R_CONV | R_REPLACE | R_MAXIT));
        if (need_replace) {
          const int reason = hf.reason;
          KP_TRY(replace_residual(ctx, B, b, x, lam2));
          ++repl;
          k_after_replace<<<1, 1, 0, st>>>(ctx->dscal, ctx->dflags, ctx->hist, ctx->hist_cap);
          KP_LAUNCHED(ctx);
          KP_TRY(read_flags(ctx, &hf, hs));
          final_rr = hs[S_RR];
          if (hf.reason & R_TRUE) {
            result = KP_OK;
            break;
          }
          if ((hf.reason & R_STAGNATE) && !(reason & R_MAXIT)) {
            result = KP_ENOCONV;
            kp_set_error("tik_pcg: stagnated at ||r||/||A^T b|| = %.3e (iteration %d): the tolerance is below the "
                         "attainable accuracy of this precision", std::sqrt(final_rr / rr0), iters);
            break;
          }
          hf.reason = reason;
        } else if (hf.reason & R_CONV) {
          result = KP_OK;
          break;
        }
        if (hf.reason & R_MAXIT) {
          result = KP_ENOCONV;
          kp_set_error("tik_pcg: maxit %d reached, ||r||/||A^T b|| = %.3e", maxit, std::sqrt(final_rr / rr0));
          break;
        }
        // resume: clear the pause, finish the interrupted iteration, continue
        int zero2[2] = {0, 0};
        KP_CUDA(cudaMemcpyAsync(ctx->dflags, zero2, sizeof(zero2), cudaMemcpyHostToDevice, st));
        KP_TRY(half_b(ctx, B, lam2_pc, false));
        KP_CUDA(cudaStreamSynchronize(st));
        cur = 0;
        KP_TRY(launch_block(cur));
      }
      cudaGraphExecDestroy(exec);
      cudaGraphDestroy(graph);
      }  // host loop
    }
  }
  R.iters = iters;
  R.repl = repl;
  R.final_rr = final_rr;
  R.result = result;
  return solve_finish(ctx, &R, info);
}

extern "C" kp_status tik_pcg(kp_ctx* ctx, const void* b, double lambda, double tol, int maxit, int flexible, void* x,
                             int warm_start, kp_solve_info* info) {
  KP_TRY(kp_check_ready(ctx));
  if (!b || !x || ((uintptr_t)b & 15) || ((uintptr_t)x & 15)) {
    kp_set_error("tik_pcg: b and x must be non-NULL, 16-byte aligned device pointers");
    return KP_EINVAL;
  }
  if (!(lambda > 0.0) || !std::isfinite(lambda) || !(tol >= 0.0) || maxit < 1) {
    kp_set_error("tik_pcg: need lambda > 0, tol >= 0, maxit >= 1");
    return KP_EINVAL;
  }
  KP_TRY(kp_enter(ctx));
  kp_status s = tik_pcg_impl(ctx, b, lambda, tol, maxit, flexible, x, warm_start, info);
  kp_status l = kp_leave(ctx);
  return s != KP_OK ? s : l;
}

// ---------------------------------------------------------------- batched solves
// One problem's solve around an iteration loop that runs grouped with other
// problems' (kp_batch.cu): the steps before the loop, the loop's body
// recorded in three segments (first half; the residual replacement, skipped
// by the problems for which none is due; second half), the decision flags,
// and the results after the loop.
struct BatchRun {
  SolveRun R;
  bool looped = false;
};

kp_status batch_begin(kp_ctx* ctx, const void* b, double lambda, double tol, int maxit, int flexible, void* x,
                      BatchRun** out) {
  *out = nullptr;
  auto* br = new BatchRun();
  const kp_status s = solve_begin(ctx, b, lambda, tol, maxit, flexible, x, 0, &br->R);
  if (s != KP_OK) {
    if (br->R.e0) cudaEventDestroy(br->R.e0);
    if (br->R.e1) cudaEventDestroy(br->R.e1);
    delete br;
    return s;
  }
  *out = br;
  return KP_OK;
}

// the loop is still to run, and its body has the form the grouped loop runs
// (the folded iteration of a tensor-core operator)
bool batch_groupable(const BatchRun* br) { return br->R.need_loop && br->R.folded && br->R.reliable; }
bool batch_needs_loop(const BatchRun* br) { return br->R.need_loop; }

kp_status batch_record(kp_ctx* ctx, BatchRun* br, KpRecorder* seg_a, KpRecorder* seg_r, KpRecorder* seg_b) {
  const SolveRun& R = br->R;
  LoopConds lc;
  lc.mode = 2;
  const int* nd = ctx->dflags + F_NOTDUE;
  kp_status s;
  ctx->rec = seg_a;
  s = half_a_folded(ctx, R.B, R.x, R.lam2, R.lam2_pc, &lc);
  ctx->rec = seg_r;
  if (s == KP_OK) s = replace_residual(ctx, R.B, R.b, R.x, R.lam2, nd);
  if (s == KP_OK) {
    const cudaError_t e = kp_launch_g<AfterReplace>(ctx, k_loop_after_replace, dim3(1), dim3(1), 0, ctx->dscal,
                                                    ctx->dflags, ctx->hist, ctx->hist_cap,
                                                    (cudaGraphConditionalHandle)0, nd, 1);
    if (e != cudaSuccess) {
      kp_set_error("batched solve: %s", cudaGetErrorString(e));
      s = KP_ECUDA;
    }
  }
  if (s == KP_OK) s = pc_prepare_input(ctx, R.B.r, R.lam2_pc, ctx->dscal + S_RR, nd);
  ctx->rec = seg_b;
  if (s == KP_OK) s = half_b(ctx, R.B, R.lam2_pc, true);
  ctx->rec = nullptr;
  return s;
}

// before the grouped loop: no replacement due, the loop goes on
kp_status batch_arm(kp_ctx* ctx, BatchRun* br) {
  const int v[2] = {1, 1};
  static_assert(F_BLOOP == F_NOTDUE + 1, "adjacent flag slots");
  KP_CUDA(cudaMemcpyAsync(ctx->dflags + F_NOTDUE, v, sizeof(v), cudaMemcpyHostToDevice, ctx->stream));
  KP_CUDA(cudaStreamSynchronize(ctx->stream));  // v is a host stack value
  br->looped = true;
  return KP_OK;
}

// after the grouped loop (or without one): status and info; frees br
kp_status batch_finish(kp_ctx* ctx, BatchRun* br, kp_solve_info* info) {
  SolveRun& R = br->R;
  if (br->looped) {
    int fl[16];
    double hs[12];
    KP_CUDA(cudaMemcpyAsync(fl, ctx->dflags, sizeof(fl), cudaMemcpyDeviceToHost, ctx->stream));
    KP_CUDA(cudaMemcpyAsync(hs, ctx->dscal, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
    KP_CUDA(cudaStreamSynchronize(ctx->stream));
    R.iters = fl[F_ITER];
    R.repl = fl[F_REPL];
    R.final_rr = hs[S_RR];
    loop_result(&R, fl);
  }
  const kp_status s = solve_finish(ctx, &R, info);
  delete br;
  return s;
}

void batch_discard(BatchRun* br) {
  if (!br) return;
  if (br->R.e0) cudaEventDestroy(br->R.e0);
  if (br->R.e1) cudaEventDestroy(br->R.e1);
  delete br;
}

// ---------------------------------------------------------------- operator hooks
extern "C" kp_status kp_apply_A(kp_ctx* ctx, const void* x, void* y, int transpose) {
  KP_TRY(kp_check_ready(ctx));
  if (!x || !y || x == y) {
    kp_set_error("kp_apply_A: x and y must be distinct device pointers");
    return KP_EINVAL;
  }
  KP_TRY(kp_enter(ctx));
  KP_TRY(op_apply(ctx, x, y, transpose ? 1 : 0, OP_INNER));
  return kp_leave(ctx);
}

extern "C" kp_status kp_apply_K(kp_ctx* ctx, const void* x, void* y, double lambda) {
  KP_TRY(kp_check_ready(ctx));
  if (!x || !y || x == y) {
    kp_set_error("kp_apply_K: x and y must be distinct device pointers");
    return KP_EINVAL;
  }
  KP_TRY(kp_enter(ctx));
  KP_TRY(op_apply_K(ctx, x, y, lambda * lambda, false, nullptr));
  return kp_leave(ctx);
}

extern "C" kp_status kp_apply_Minv(kp_ctx* ctx, const void* r, void* z, double lambda) {
  KP_TRY(kp_check_ready(ctx));
  if (!r || !z || r == z || !(lambda > 0.0)) {
    kp_set_error("kp_apply_Minv: need distinct device pointers and lambda > 0");
    return KP_EINVAL;
  }
  KP_TRY(kp_enter(ctx));
  KP_TRY(pc_apply(ctx, r, z, lambda * lambda, nullptr, nullptr));
  return kp_leave(ctx);
}

// observed data b = A x + nl ||A x|| g / ||g|| (accurate operator)
extern "C" kp_status kp_forward(kp_ctx* ctx, const void* x, const void* g, double noise_level, void* b,
                                double* noise_norm) {
  KP_TRY(kp_check_ready(ctx));
  if (!x || !g || !b || !(noise_level >= 0.0)) {
    kp_set_error("kp_forward: bad arguments");
    return KP_EINVAL;
  }
  KP_TRY(kp_enter(ctx));
  const long long N = (long long)ctx->n_r * ctx->n_c;
  const bool f64 = ctx->vec_prec == KP_F64;
  KP_TRY(op_apply(ctx, x, b, 0, OP_ACCURATE));
  KP_TRY(dot2_dev(ctx, b, b, nullptr, N, f64, ctx->dscal + 20, nullptr));
  KP_TRY(dot2_dev(ctx, g, g, nullptr, N, f64, ctx->dscal + 21, nullptr));
  double h[2];
  KP_CUDA(cudaMemcpyAsync(h, ctx->dscal + 20, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  KP_CUDA(cudaStreamSynchronize(ctx->stream));
  const double scale = h[1] > 0 ? noise_level * std::sqrt(h[0]) / std::sqrt(h[1]) : 0.0;
  KP_TRY(axpby_dev(ctx, g, b, N, f64, scale, 1.0));
  if (noise_norm) *noise_norm = scale * std::sqrt(h[1]);
  return kp_leave(ctx);
}

// ---------------------------------------------------------------- per-part timing
// The parts of one (F)PCG iteration launched `reps` times each on the
// context's stream between CUDA events, on the context's own solver vectors
// (the caller's data is not touched): [0] the K application as the iteration
// runs it (bf16 slices of p ready, p^T q and alpha fused where the iteration
// fuses them), [1] the preconditioner solve (narrow input made by the x / r
// update where the iteration folds it), [2] the vector phase (x / r update,
// z^T r / beta, p update), [3] one residual replacement (true residual with
// the accurate operator, its norm).  No pause flag is passed, so every kernel
// does its full work whatever the scalars hold.
extern "C" kp_status kp_time_parts(kp_ctx* ctx, double lambda, int reps, double* ms, long long* launches) {
  KP_TRY(kp_check_ready(ctx));
  if (!ms || reps < 1 || !(lambda > 0.0)) {
    kp_set_error("kp_time_parts: need ms (4 doubles), reps >= 1 and lambda > 0");
    return KP_EINVAL;
  }
  KP_TRY(kp_enter(ctx));
  const long long N = (long long)ctx->n_r * ctx->n_c;
  const bool f64 = ctx->vec_prec == KP_F64;
  const size_t vs = f64 ? 8 : 4;
  const double lam2 = lambda * lambda;
  const SolveBufs B = bufs(ctx);
  void* x = ctx->tmp_img;
  cudaStream_t st = ctx->stream;
  // contents: r = p = the last right-hand side A^T b, the other vectors zero
  for (void* v : {B.r_old, B.q, B.z, x}) KP_CUDA(cudaMemsetAsync(v, 0, vs * N, st));
  KP_TRY(copy_vec(ctx, B.rhs, B.r, N, f64));
  KP_TRY(copy_vec(ctx, B.rhs, B.p, N, f64));
  if (op_inner_slices(ctx) > 0)
    KP_TRY(split_bf16(ctx, B.p, false, N, ctx->w_img2, op_inner_slices(ctx), N));
  KP_TRY(norm_amax_dev(ctx, B.r, N, f64, ctx->dscal + S_RR));
  const bool folded = cg_fusable(ctx);
  double* s = ctx->dscal;
  PostOp pa;
  pa.kind = POST_ALPHA;
  pa.s = s;
  pa.f = ctx->dflags;
  PostOp pc = pa;
  pc.kind = POST_CHECK;
  pc.hist = ctx->hist;
  pc.hist_cap = ctx->hist_cap;
  PostOp pb = pa;
  pb.kind = POST_BETA;
  const int sl = op_inner_slices(ctx);
  const int nt = ctx->pc_prec == KP_BF16 ? NT_BF16 : NT_F16;
  auto part = [&](int k) -> kp_status {
    if (k == 0) {
      bool fused = false;
      return op_apply_K(ctx, B.p, B.q, lam2, sl > 0, nullptr, s + (folded ? S_QPQ : S_PQ), &pa, &fused, folded);
    }
    if (k == 1) return pc_apply(ctx, B.r, B.z, lam2, s + S_RR, nullptr, folded);
    if (k == 2) {
      if (folded)
        KP_TRY(update_xr_q_dev(ctx, x, B.r, B.r_old, B.p, B.q, N, s + S_ALPHA, s + S_RR, s + S_QMAX, nt, lam2,
                               ctx->pc_in, cg_inv_slot(ctx), nullptr, pc));
      else
        KP_TRY(update_xr_dev(ctx, x, B.r, B.r_old, B.p, B.q, N, f64, s + S_ALPHA, s + S_RR, nullptr, pc));
      KP_TRY(dot2_dev(ctx, B.z, B.r, B.r_old, N, f64, s + S_ZRNEW, nullptr, pb));
      return p_update_dev(ctx, B.p, B.z, N, f64, s + S_BETA, sl ? (__nv_bfloat16*)ctx->w_img2 : nullptr, sl, N,
                          nullptr);
    }
    KP_TRY(op_true_residual(ctx, B.rhs, x, B.r, lam2, nullptr));
    return norm_amax_dev(ctx, B.r, N, f64, s + S_RR);
  };
  cudaEvent_t e0, e1;
  KP_CUDA(cudaEventCreate(&e0));
  KP_CUDA(cudaEventCreate(&e1));
  kp_status res = KP_OK;
  for (int k = 0; k < 4 && res == KP_OK; ++k) {
    for (int w = 0; w < 2 && res == KP_OK; ++w) res = part(k);
    if (res != KP_OK) break;
    const long long l0 = ctx->launches;
    cudaEventRecord(e0, st);
    for (int i = 0; i < reps && res == KP_OK; ++i) res = part(k);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      kp_set_error("kp_time_parts: %s", cudaGetErrorString(cudaGetLastError()));
      res = KP_ECUDA;
      break;
    }
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    ms[k] = t / reps;
    if (launches) launches[k] = (ctx->launches - l0) / reps;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  KP_TRY(res);
  KP_TRY(read_status(ctx));
  return kp_leave(ctx);
}
