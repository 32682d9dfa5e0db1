// Operator and preconditioner applications.
//
// Layout: images are column-major n_r x n_c (vec order, Section 3).  The
// Kronecker sum A vec(X) = vec(sum_k A_c^(k) X A_r^(k)^T) (eq. KronSumDecomp)
// runs as two GEMMs whose operands are all K-major:
//   G1  W = [A_c^(1); ...; A_c^(r)] X           M = r n_r, N = n_c, K = n_r
//       (output row-major W_k[i', j], stacked over k)
//   G2  Z^T = sum_k A_r^(k) W_k^T                M = n_c, N = n_r, K = n_c per term
//       (output row-major [l][i'] = column-major Z)
// and A^T vec(Y) = vec(sum_k A_c^(k)^T Y A_r^(k)) is G3 / G4 with the
// transposed factors.  The preconditioner solve Z = V_c (S .* (V_c^T R V_r)) V_r^T
// (eq. PreconSolve) is P1..P4 with the same alternation, S applied in the
// P2 epilogue as lam^2 / (Sigma^2 + lam^2) and 1 / lam^2 folded into P4.
// A BF16 preconditioner keeps V_c, V_r as bf16 hi + lo slices (two products
// per GEMM); FP16 keeps them as single fp16 values.
//
// Tensor-core operators split activations and factors into bf16 slices.
// The inner (per-iteration) operator uses the slice pairs {(0,0)} (KP_BF16)
// or {(0,0),(0,1),(1,0)} (KP_BF16X3); the accurate operator used for true
// residuals uses {(0,0),(0,1),(1,0),(0,2),(1,1),(2,0)}, whose dropped terms are
// below 2^-24 relative (FP32 level).
#include <algorithm>

#include "kp_group.cuh"
#include "kp_ops.h"
#include "kp_vec.cuh"

namespace {
struct OpsState {
  TcGemmPlan* G[2][4] = {{nullptr}};  // [mode][gemm]
  TcGemmPlan* Gin[2][4] = {{nullptr}};  // inner-operator plans per variant: [0] BF16 pair, [1] BF16X3 pairs
  TcGemmPlan* Gk[4] = {nullptr};      // inner operator of the first pc_rank terms (multi-term preconditioner)
  bool batched = false;               // G2 / G4 write per-term outputs, summed by k_term_reduce
  TcGemmPlan* P[4] = {nullptr};
  float* inv_slot = nullptr;          // device scale for P4
  float* e4m3_slots = nullptr;        // E4M3: [0] 1/(lam^2 s_R s_V^2), [1..3] stage scales g
  unsigned int* amax8 = nullptr;      // E4M3: per-stage max |T| of the FP32 GEMM outputs
  double* stat = nullptr;             // device [rr, amax] scratch
};
}  // namespace

static OpsState* ops(kp_ctx* ctx) { return reinterpret_cast<OpsState*>(ctx->ops_state); }

// plans made in this scope are for grouped launches when the context is a
// batched solve's (tc_group)
struct GroupedPlans {
  kp_ctx* c;
  bool old;
  explicit GroupedPlans(kp_ctx* ctx) : c(ctx), old(ctx->tc_grouping) { c->tc_grouping = c->tc_group; }
  ~GroupedPlans() { c->tc_grouping = old; }
};

void ops_state_free(kp_ctx* ctx) {
  delete ops(ctx);
  ctx->ops_state = nullptr;
}

static bool op_is_tc(kp_ctx* ctx) { return ctx->op_prec == KP_BF16 || ctx->op_prec == KP_BF16X3; }
static bool pc_is_tc(kp_ctx* ctx) {
  return ctx->pc_prec == KP_BF16 || ctx->pc_prec == KP_F16 || ctx->pc_prec == KP_E4M3;
}
static bool vec64(kp_ctx* ctx) { return ctx->vec_prec == KP_F64; }

int op_inner_slices(kp_ctx* ctx) {
  if (!op_is_tc(ctx)) return 0;
  return ctx->op_prec == KP_BF16X3 ? 2 : 1;
}

static void pairs_for(kp_ctx* ctx, int mode, GemmDesc& g) {
  static const int acc_a[6] = {0, 0, 1, 0, 1, 2}, acc_b[6] = {0, 1, 0, 2, 1, 0};
  static const int x3_a[3] = {0, 0, 1}, x3_b[3] = {0, 1, 0};
  if (mode == OP_ACCURATE) {
    g.npairs = 6;
    for (int i = 0; i < 6; ++i) {
      g.sa[i] = acc_a[i];
      g.sb[i] = acc_b[i];
    }
  } else if (ctx->op_prec == KP_BF16X3) {
    g.npairs = 3;
    for (int i = 0; i < 3; ++i) {
      g.sa[i] = x3_a[i];
      g.sb[i] = x3_b[i];
    }
  } else {
    g.npairs = 1;
    g.sa[0] = g.sb[0] = 0;
  }
}

// split-K factor for the square GEMMs: 0 lets the GEMM plan pick enough
// (tile, split) units to fill the GPU
static int square_splits(kp_ctx* ctx) { return ctx->splitk_override > 0 ? ctx->splitk_override : 0; }

// GEMM descriptors of the operator: which = 0..3 (G1..G4), over the first
// `terms` Kronecker terms (the full operator: terms = rank; the factor
// blocks stay laid out for all rank terms)
static GemmDesc op_desc(kp_ctx* ctx, int which, int mode, const void* bptr, int terms = 0) {
  const int n_r = ctx->n_r, n_c = ctx->n_c, r = ctx->rank;
  const int t = terms > 0 ? terms : r;
  const long long N = (long long)n_r * n_c;
  GemmDesc g;
  pairs_for(ctx, mode, g);
  const int slices = op_is_tc(ctx) ? 3 : 1;
  if (which == 0 || which == 2) {  // G1 / G3: stacked factors x image
    g.M = t * n_r;
    g.N = n_c;
    g.K = n_r;
    g.nkron = 1;
    g.A.ptr = which == 0 ? ctx->opAc : ctx->opAcT;
    g.A.rows = t * n_r;
    g.A.K = n_r;
    g.A.ld = n_r;
    g.A.tstride = (long long)r * n_r * n_r;
    g.A.nterm_idx = slices;
    g.a_terms = 1;
    g.B.ptr = bptr;
    g.B.rows = n_c;
    g.B.K = n_r;
    g.B.ld = n_r;
    g.B.tstride = N;
    g.B.nterm_idx = slices;
    g.b_terms = 1;
  } else {  // G2 / G4: sum over terms of factor x stacked intermediate
    g.M = n_c;
    g.N = n_r;
    g.K = n_c;
    g.nkron = t;
    g.A.ptr = which == 1 ? ctx->opAr : ctx->opArT;
    g.A.rows = n_c;
    g.A.K = n_c;
    g.A.ld = n_c;
    g.A.tstride = (long long)n_c * n_c;
    g.A.nterm_idx = slices * r;
    g.a_terms = r;
    g.B.ptr = ctx->w_stack;
    g.B.rows = n_r;
    g.B.K = n_c;
    g.B.ld = n_c;
    g.B.tstride = N;
    g.B.nterm_idx = slices * r;
    g.b_terms = r;
  }
  return g;
}

static GemmDesc pc_desc(kp_ctx* ctx, int which) {
  const int n_r = ctx->n_r, n_c = ctx->n_c;
  GemmDesc g;
  g.npairs = 1;
  g.nkron = 1;
  if (which == 0 || which == 2) {  // P1: V_c^T R ; P3: V_c W
    g.M = n_r;
    g.N = n_c;
    g.K = n_r;
    g.A.ptr = which == 0 ? ctx->pcVcT : ctx->pcVc;
    g.A.rows = n_r;
    g.A.ld = n_r;
    g.B.ptr = which == 0 ? ctx->pc_in : ctx->pc_t2;
    g.B.rows = n_c;
    g.B.ld = n_r;
  } else {  // P2: V_r^T T1^T ; P4: V_r T3^T
    g.M = n_c;
    g.N = n_r;
    g.K = n_c;
    g.A.ptr = which == 1 ? ctx->pcVrT : ctx->pcVr;
    g.A.rows = n_c;
    g.A.ld = n_c;
    g.B.ptr = which == 1 ? ctx->pc_t1 : ctx->pc_t3;
    g.B.rows = n_r;
    g.B.ld = n_c;
  }
  g.A.K = g.K;
  g.B.K = g.K;
  g.A.tstride = (long long)g.A.rows * g.A.ld;
  g.B.tstride = (long long)g.B.rows * g.B.ld;
  g.A.nterm_idx = 1;
  g.B.nterm_idx = 1;
  if (ctx->pc_prec == KP_BF16) {  // factor slices hi, lo times the single activation slice
    g.npairs = 2;
    g.sa[0] = 0;
    g.sa[1] = 1;
    g.sb[0] = g.sb[1] = 0;
    g.A.nterm_idx = 2;
  }
  return g;
}

// Sum of the per-term outputs of a batched G2 / G4 with the fused epilogue of
// the image-shaped product: out = alpha sum_k Z_k + beta aux, as FP32 or as
// bf16 slices (hi, lo, ...).  Z holds `terms` blocks of nel FP32 values; the
// terms are added in order.
// With dot non-null (FP32 output), also dot = sum out * aux (p^T q of the
// iteration) by the deterministic tree of the vector kernels, and the scalar
// step po by its last block.
// With qmax also max |out| into out[1].
struct TermDot {
  double* out = nullptr;
  double* partials = nullptr;
  unsigned int* counter = nullptr;
  PostOp po;
  int qmax = 0;
};

// the term sum's dot (and max) reduction: one double-float sum, or a sum
// and a max
__device__ __forceinline__ void term_dot_finish(float (&dh)[2], float (&dl)[2], const TermDot& td) {
  if (td.qmax) {
    kpv::reduce_finish_df<2>(dh, dl, true, td.partials, td.counter, td.out, 2, td.po);
  } else {
    float h1[1] = {dh[0]}, l1[1] = {dl[0]};
    kpv::reduce_finish_df<1>(h1, l1, false, td.partials, td.counter, td.out, 1, td.po);
  }
}

__device__ __forceinline__ void k_term_reduce_body(const float* __restrict__ Z, int terms, long long nel, float alpha,
                                                   float beta, const float* __restrict__ aux, int slices_mode,
                                                   void* __restrict__ out, int slices, long long sstride, int vec,
                                                   TermDot td, const int* flags) {
  KP_PDL_WAIT();
  KP_PDL_TRIGGER();
  if (flags && *(volatile const int*)flags) return;
  float dh[2] = {0.f, 0.f}, dl[2] = {0.f, 0.f};  // p^T q as a double-float pair; max |q| in dh[1]
  if (!vec) {  // out / aux not 16-byte aligned: one element at a time
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nel; i += (long long)gridDim.x * blockDim.x) {
      float a = Z[i];
      for (int k = 1; k < terms; ++k) a += Z[k * nel + i];
      float v = alpha * a;
      if (aux) v = fmaf(beta, aux[i], v);
      if (!slices_mode) {
        ((float*)out)[i] = v;
        if (td.out) {
          kpv::df_add_prod(dh[0], dl[0], v, aux[i]);
          dh[1] = fmaxf(dh[1], fabsf(v));
        }
      } else {
        for (int sl = 0; sl < slices; ++sl) {
          const __nv_bfloat16 h = __float2bfloat16_rn(v);
          ((__nv_bfloat16*)out)[sl * sstride + i] = h;
          v -= __bfloat162float(h);
        }
      }
    }
    if (td.out) term_dot_finish(dh, dl, td);
    return;
  }
  const long long n4 = nel >> 2;
  const float4* Z4 = reinterpret_cast<const float4*>(Z);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
    float4 a = Z4[i];
    for (int k = 1; k < terms; ++k) {
      const float4 t = Z4[k * n4 + i];
      a.x += t.x;
      a.y += t.y;
      a.z += t.z;
      a.w += t.w;
    }
    float v[4] = {alpha * a.x, alpha * a.y, alpha * a.z, alpha * a.w};
    if (aux) {
      const float4 t = reinterpret_cast<const float4*>(aux)[i];
      v[0] = fmaf(beta, t.x, v[0]);
      v[1] = fmaf(beta, t.y, v[1]);
      v[2] = fmaf(beta, t.z, v[2]);
      v[3] = fmaf(beta, t.w, v[3]);
    }
    if (!slices_mode) {
      reinterpret_cast<float4*>(out)[i] = make_float4(v[0], v[1], v[2], v[3]);
      if (td.out) {
        const float4 t = reinterpret_cast<const float4*>(aux)[i];
        kpv::df_add_prod(dh[0], dl[0], v[0], t.x);
        kpv::df_add_prod(dh[0], dl[0], v[1], t.y);
        kpv::df_add_prod(dh[0], dl[0], v[2], t.z);
        kpv::df_add_prod(dh[0], dl[0], v[3], t.w);
        dh[1] = fmaxf(dh[1], fmaxf(fmaxf(fabsf(v[0]), fabsf(v[1])), fmaxf(fabsf(v[2]), fabsf(v[3]))));
      }
    } else {
      __nv_bfloat16* o = (__nv_bfloat16*)out + 4 * i;
      for (int sl = 0; sl < slices; ++sl) {
        __nv_bfloat162 h0 = __floats2bfloat162_rn(v[0], v[1]);
        __nv_bfloat162 h1 = __floats2bfloat162_rn(v[2], v[3]);
        uint2 pk;
        pk.x = *reinterpret_cast<uint32_t*>(&h0);
        pk.y = *reinterpret_cast<uint32_t*>(&h1);
        *reinterpret_cast<uint2*>(o + sl * sstride) = pk;
        v[0] -= __bfloat162float(h0.x);
        v[1] -= __bfloat162float(h0.y);
        v[2] -= __bfloat162float(h1.x);
        v[3] -= __bfloat162float(h1.y);
      }
    }
  }
  if (td.out) term_dot_finish(dh, dl, td);
}
__global__ void __launch_bounds__(VEC_THREADS)
    k_term_reduce(const float* __restrict__ Z, int terms, long long nel, float alpha, float beta,
                  const float* __restrict__ aux, int slices_mode, void* __restrict__ out, int slices, long long sstride,
                  int vec, TermDot td, const int* flags) {
  k_term_reduce_body(Z, terms, nel, alpha, beta, aux, slices_mode, out, slices, sstride, vec, td, flags);
}
KP_BODY(TermReduce, k_term_reduce_body);

// tensor-core plan of GEMM w of the operator in `mode` for the current pairs
static kp_status op_plan(kp_ctx* ctx, OpsState* os, int mode, int w, TcGemmPlan** out, int terms = 0) {
  const void* bptr = w == 0 ? (mode == OP_INNER ? ctx->w_img2 : ctx->w_img3) : (w == 2 ? ctx->w_img : nullptr);
  const int t = terms > 0 ? terms : ctx->rank;
  GemmDesc g = op_desc(ctx, w, mode, bptr, t);
  if ((w == 1 || w == 3) && mode == OP_INNER && ctx->tc_kcat && ctx->splitk_override == 0) {
    // the sum over terms as one product (terms summed in the accumulator, no
    // per-term outputs, no term sum), where its tiles fit
    GemmDesc gk = g;
    gk.kcat = ctx->tc_kcat_cluster;
    TcGemmPlan* pl = nullptr;
    KP_TRY(tc_plan_create(ctx, gk, TC_BF16, 1, &pl));
    if (tc_plan_is_kcat(pl)) {
      *out = pl;
      return KP_OK;
    }
    tc_plan_release(ctx, pl);
  }
  int splits = (w == 1 || w == 3) ? square_splits(ctx) : 1;
  if ((w == 1 || w == 3) && os->batched) {
    g.batch_rows = ctx->n_c;
    g.M = t * ctx->n_c;
    splits = 1;
  }
  return tc_plan_create(ctx, g, TC_BF16, splits, out);
}

kp_status ops_set_inner(kp_ctx* ctx, kp_prec p) {
  if (!op_is_tc(ctx) || (p != KP_BF16 && p != KP_BF16X3)) {
    kp_set_error("ops_set_inner: needs a tensor-core operator and BF16 / BF16X3");
    return KP_ENOTSUP;
  }
  if (ctx->op_prec == p) return KP_OK;
  GroupedPlans gp(ctx);
  OpsState* os = ops(ctx);
  const int v = p == KP_BF16X3 ? 1 : 0;
  const kp_prec old = ctx->op_prec;
  ctx->op_prec = p;  // the pairs and slice counts follow it
  for (int w = 0; w < 4; ++w) {
    if (!os->Gin[v][w]) {
      const kp_status st = op_plan(ctx, os, OP_INNER, w, &os->Gin[v][w]);
      if (st != KP_OK) {
        ctx->op_prec = old;
        return st;
      }
    }
    os->G[OP_INNER][w] = os->Gin[v][w];
  }
  return KP_OK;
}

kp_status ops_prepare(kp_ctx* ctx) {
  const int n_r = ctx->n_r, n_c = ctx->n_c, r = ctx->rank;
  const long long N = (long long)n_r * n_c;
  const size_t vs = vec64(ctx) ? 8 : 4;
  ops_state_free(ctx);
  GroupedPlans gp(ctx);
  OpsState* os = new OpsState();
  ctx->ops_state = os;
  KP_TRY(kp_alloc(ctx, (void**)&os->inv_slot, 16));
  KP_TRY(kp_alloc(ctx, (void**)&os->e4m3_slots, 16));
  KP_TRY(kp_alloc(ctx, (void**)&os->amax8, 16));
  KP_CUDA(cudaMemsetAsync(os->amax8, 0, 16, ctx->stream));
  KP_TRY(kp_alloc(ctx, (void**)&os->stat, 4 * sizeof(double)));
  // solver vectors and scratch images
  for (int i = 0; i < 8; ++i) KP_TRY(kp_alloc(ctx, &ctx->vbuf[i], vs * N));
  KP_TRY(kp_alloc(ctx, &ctx->tmp_img, vs * N));
  KP_TRY(kp_alloc(ctx, &ctx->tmp_img2, vs * N));
  ctx->hist_cap = 1 << 16;
  KP_TRY(kp_alloc(ctx, (void**)&ctx->hist, sizeof(double) * ctx->hist_cap));
  // operator workspaces
  if (op_is_tc(ctx)) {
    const size_t b = sizeof(__nv_bfloat16);
    KP_TRY(kp_alloc(ctx, &ctx->w_stack, b * 3 * r * N));
    KP_TRY(kp_alloc(ctx, &ctx->w_img, b * 3 * N));
    KP_TRY(kp_alloc(ctx, &ctx->w_img2, b * 3 * N));
    KP_TRY(kp_alloc(ctx, &ctx->w_img3, b * 3 * N));
  } else {
    KP_TRY(kp_alloc(ctx, &ctx->w_stack, vs * r * N));
    KP_TRY(kp_alloc(ctx, &ctx->w_img, vs * N));
  }
  // preconditioner workspaces
  {
    const size_t es = pc_is_tc(ctx) ? (ctx->pc_prec == KP_E4M3 ? 1 : 2) : vs;
    KP_TRY(kp_alloc(ctx, &ctx->pc_in, es * N));
    KP_TRY(kp_alloc(ctx, &ctx->pc_t1, es * N));
    KP_TRY(kp_alloc(ctx, &ctx->pc_t2, es * N));
    KP_TRY(kp_alloc(ctx, &ctx->pc_t3, es * N));
    KP_TRY(kp_alloc(ctx, (void**)&ctx->pc_f32, sizeof(float) * N));
  }
  // split-K workspace: up to 8 partial images
  const long long nmax = std::max(n_r, n_c);
  ctx->w_split_elems = 8 * nmax * nmax;
  KP_TRY(kp_alloc(ctx, (void**)&ctx->w_split, sizeof(float) * ctx->w_split_elems));
  // partial tiles of SIMT GEMMs split over blocks (small problems on the FP64
  // / FP32 operator or preconditioner): up to 4 x the stacked intermediate
  if ((!op_is_tc(ctx) || !pc_is_tc(ctx)) && (long long)((n_c + 63) / 64) * ((n_r + 63) / 64) < ctx->sm_count) {
    ctx->simt_ws_bytes = vs * 4 * (size_t)std::max(r, 1) * (size_t)N;
    KP_TRY(kp_alloc(ctx, &ctx->simt_ws, ctx->simt_ws_bytes));
  }

  if (op_is_tc(ctx)) {
    // G2 / G4 as one GEMM over the stacked per-term products (4x the tiles
    // of the term sum, no K split) when the per-term outputs fit the split
    // workspace; k_term_reduce adds them with the fused epilogue
    os->batched = r >= 2 && n_c % 128 == 0 && n_r % 4 == 0 && (long long)r * N <= ctx->w_split_elems &&
                  ctx->splitk_override == 0;
    for (int mode = 0; mode < 2; ++mode)
      for (int w = 0; w < 4; ++w) KP_TRY(op_plan(ctx, os, mode, w, &os->G[mode][w]));
    for (int w = 0; w < 4; ++w) os->Gin[ctx->op_prec == KP_BF16X3 ? 1 : 0][w] = os->G[OP_INNER][w];
    if (ctx->pc_rank > 1 && ctx->pc_rank < r)
      for (int w = 0; w < 4; ++w) KP_TRY(op_plan(ctx, os, OP_INNER, w, &os->Gk[w], ctx->pc_rank));
  }
  if (ctx->pc_rank > 1)  // inner solve of the multi-term preconditioner: r, r_old, p, q, z
    for (int i = 0; i < 5; ++i) KP_TRY(kp_alloc(ctx, &ctx->pc_inner[i], vs * N));
  if (pc_is_tc(ctx)) {
    const int kind = ctx->pc_prec == KP_BF16 ? TC_BF16 : (ctx->pc_prec == KP_F16 ? TC_F16 : TC_E4M3);
    for (int w = 0; w < 4; ++w) {
      GemmDesc g = pc_desc(ctx, w);
      KP_TRY(tc_plan_create(ctx, g, kind, kind == TC_E4M3 ? 1 : square_splits(ctx), &os->P[w]));
    }
  }
  return KP_OK;
}

// ------------------------------------------------------------- operator
template <typename T>
static kp_status simt_op(kp_ctx* ctx, int which, const void* bptr, EpiParams e, const int* flags, int terms) {
  GemmDesc g = op_desc(ctx, which, OP_INNER, bptr, terms);
  g.npairs = 1;
  g.sa[0] = g.sb[0] = 0;
  e.mode = EPI_T;
  g.epi = e;
  g.flags = flags;
  return simt_gemm<T>(ctx, g);
}

static kp_status run_op(kp_ctx* ctx, int which, int mode, const void* bptr, const EpiParams& e, const int* flags,
                        const TermDot* td = nullptr, bool* dot_done = nullptr, int terms = 0) {
  if (dot_done) *dot_done = false;
  const int nterm = terms > 0 ? terms : ctx->rank;
  if (op_is_tc(ctx)) {
    OpsState* os = ops(ctx);
    TcGemmPlan* pl = (nterm < ctx->rank && mode == OP_INNER) ? os->Gk[which] : os->G[mode][which];
    if (!pl) {
      kp_set_error("operator: no plan for %d terms", nterm);
      return KP_ESTATE;
    }
    tc_plan_set_runtime(pl, nullptr, flags);
    if (tc_plan_is_kcat(pl)) {  // the terms summed in the accumulator; the dot in the epilogue
      if (td && e.mode == EPI_F32 && e.aux) {
        if (dot_done) *dot_done = true;
        return tc_plan_run_dot(ctx, pl, e, td->out, td->partials, td->counter, td->po, td->qmax);
      }
      return tc_plan_run(ctx, pl, &e);
    }
    if (!(os->batched && (which == 1 || which == 3))) return tc_plan_run(ctx, pl, &e);
    // per-term FP32 outputs into the split workspace, then the term sum
    EpiParams ez;
    ez.mode = EPI_F32;
    ez.out = ctx->w_split;
    ez.ldd = ctx->n_r;
    KP_TRY(tc_plan_run(ctx, pl, &ez));
    const long long nel = (long long)ctx->n_r * ctx->n_c;
    const int g = std::max(1, std::min((int)((nel / 4 + VEC_THREADS - 1) / VEC_THREADS), ctx->sm_count * 8));
    const int vec = ((((uintptr_t)e.out | (uintptr_t)e.aux) & 15) == 0 && (e.slice_stride % 4) == 0) ? 1 : 0;
    TermDot t;
    if (td && e.mode == EPI_F32 && e.aux) {
      t = *td;
      if (dot_done) *dot_done = true;
    }
    KP_CUDA(kp_launch_g<TermReduce>(ctx, k_term_reduce, dim3(g), dim3(VEC_THREADS), 0, (const float*)ctx->w_split, nterm, nel,
                      (float)e.alpha, (float)e.beta, (const float*)e.aux, e.mode == EPI_SLICES ? 1 : 0, e.out,
                      e.slices, e.slice_stride, vec, t, flags));
    KP_LAUNCHED(ctx);
    return KP_OK;
  }
  if (vec64(ctx)) return simt_op<double>(ctx, which, bptr, e, flags, nterm);
  return simt_op<float>(ctx, which, bptr, e, flags, nterm);
}

// epilogue writing the stacked intermediate (G1 / G3 output)
static EpiParams epi_stack(kp_ctx* ctx, int mode) {
  EpiParams e;
  e.out = ctx->w_stack;
  e.ldd = ctx->n_c;
  if (op_is_tc(ctx)) {
    e.mode = EPI_SLICES;
    e.slices = mode == OP_ACCURATE ? 3 : op_inner_slices(ctx);
    e.slice_stride = (long long)ctx->rank * ctx->n_r * ctx->n_c;
  } else {
    e.mode = EPI_T;
  }
  return e;
}
// epilogue writing an image-shaped output (G2 / G4): out = alpha acc + beta aux
static EpiParams epi_img(kp_ctx* ctx, int mode, void* out, bool as_slices, double alpha, double beta,
                         const void* aux) {
  EpiParams e;
  e.out = out;
  e.ldd = ctx->n_r;
  e.alpha = alpha;
  e.beta = beta;
  e.aux = aux;
  e.ld_aux = ctx->n_r;
  if (op_is_tc(ctx)) {
    if (as_slices) {
      e.mode = EPI_SLICES;
      e.slices = mode == OP_ACCURATE ? 3 : op_inner_slices(ctx);
      e.slice_stride = (long long)ctx->n_r * ctx->n_c;
    } else {
      e.mode = EPI_F32;
    }
  } else {
    e.mode = EPI_T;
  }
  return e;
}

// B operand of G1 for image x: tensor cores need bf16 slices in w_img2 / w_img3
static kp_status stage_input(kp_ctx* ctx, const void* x, int mode, const void** bptr, const int* flags = nullptr) {
  if (!op_is_tc(ctx)) {
    *bptr = x;
    return KP_OK;
  }
  void* dst = mode == OP_INNER ? ctx->w_img2 : ctx->w_img3;
  const int slices = mode == OP_ACCURATE ? 3 : op_inner_slices(ctx);
  KP_TRY(split_bf16(ctx, x, false, (long long)ctx->n_r * ctx->n_c, dst, slices, (long long)ctx->n_r * ctx->n_c, flags));
  *bptr = dst;
  return KP_OK;
}

kp_status op_apply(kp_ctx* ctx, const void* x, void* y, int transpose, int mode) {
  const void* bx;
  KP_TRY(stage_input(ctx, x, mode, &bx));
  const int g_first = transpose ? 2 : 0;
  if (transpose && op_is_tc(ctx)) {
    // G3 reads its image operand from w_img (slices)
    const int slices = mode == OP_ACCURATE ? 3 : op_inner_slices(ctx);
    KP_TRY(split_bf16(ctx, x, false, (long long)ctx->n_r * ctx->n_c, ctx->w_img, slices,
                      (long long)ctx->n_r * ctx->n_c));
    bx = ctx->w_img;
  }
  KP_TRY(run_op(ctx, g_first, mode, bx, epi_stack(ctx, mode), nullptr));
  KP_TRY(run_op(ctx, g_first + 1, mode, nullptr, epi_img(ctx, mode, y, false, 1.0, 0.0, nullptr), nullptr));
  return KP_OK;
}

kp_status op_apply_K(kp_ctx* ctx, const void* p, void* q, double lam2, bool p_slices_ready, const int* flags,
                     double* pq_out, const PostOp* pq_post, bool* pq_done, bool qmax, int terms) {
  if (pq_done) *pq_done = false;
  const void* bx = p;
  if (op_is_tc(ctx)) {
    if (!p_slices_ready) KP_TRY(stage_input(ctx, p, OP_INNER, &bx));
    bx = ctx->w_img2;
  }
  const bool tc = op_is_tc(ctx);
  KP_TRY(run_op(ctx, 0, OP_INNER, bx, epi_stack(ctx, OP_INNER), flags, nullptr, nullptr, terms));
  KP_TRY(run_op(ctx, 1, OP_INNER, nullptr, epi_img(ctx, OP_INNER, ctx->w_img, tc, 1.0, 0.0, nullptr), flags, nullptr,
                nullptr, terms));
  KP_TRY(run_op(ctx, 2, OP_INNER, ctx->w_img, epi_stack(ctx, OP_INNER), flags, nullptr, nullptr, terms));
  if (pq_out) {  // p^T q (and the alpha step) fused into the term sum when G4 is batched
    TermDot td;
    td.out = pq_out;
    td.partials = ctx->red_part;
    td.counter = ctx->red_count;
    if (pq_post) td.po = *pq_post;
    td.qmax = qmax ? 1 : 0;
    KP_TRY(run_op(ctx, 3, OP_INNER, nullptr, epi_img(ctx, OP_INNER, q, false, 1.0, lam2, p), flags, &td, pq_done,
                  terms));
    return KP_OK;
  }
  KP_TRY(run_op(ctx, 3, OP_INNER, nullptr, epi_img(ctx, OP_INNER, q, false, 1.0, lam2, p), flags, nullptr, nullptr,
                terms));
  return KP_OK;
}

kp_status op_true_residual(kp_ctx* ctx, const void* b, const void* x, void* r, double lam2, const int* flags) {
  const void* bx;
  const int mode = OP_ACCURATE;
  if (op_is_tc(ctx)) {
    KP_TRY(stage_input(ctx, x, mode, &bx, flags));
  } else {
    bx = x;
  }
  const bool tc = op_is_tc(ctx);
  KP_TRY(run_op(ctx, 0, mode, bx, epi_stack(ctx, mode), flags));
  // data-space residual b - A x
  KP_TRY(run_op(ctx, 1, mode, nullptr, epi_img(ctx, mode, ctx->w_img, tc, -1.0, 1.0, b), flags));
  KP_TRY(run_op(ctx, 2, mode, ctx->w_img, epi_stack(ctx, mode), flags));
  KP_TRY(run_op(ctx, 3, mode, nullptr, epi_img(ctx, mode, r, false, 1.0, -lam2, x), flags));
  return KP_OK;
}

// ------------------------------------------------------------- preconditioner
template <typename T>
static kp_status simt_pc(kp_ctx* ctx, const void* r, void* z, double lam2, const int* flags) {
  for (int w = 0; w < 4; ++w) {
    GemmDesc g = pc_desc(ctx, w);
    if (w == 0) g.B.ptr = r;
    if (w == 2) g.B.ptr = ctx->pc_t2;
    g.flags = flags;
    g.epi.mode = EPI_T;
    g.epi.ldd = g.N;
    g.epi.out = w == 0 ? ctx->pc_t1 : (w == 1 ? ctx->pc_t2 : (w == 2 ? ctx->pc_t3 : z));
    if (w == 1) {
      g.epi.sigma64 = ctx->Sigma64;
      g.epi.lam2 = lam2;
    }
    if (w == 3) g.epi.alpha = 1.0 / lam2;
    KP_TRY(simt_gemm<T>(ctx, g));
  }
  return KP_OK;
}

static kp_status pc_apply_kp(kp_ctx* ctx, const void* r, void* z, double lam2, const double* stat, const int* flags,
                             bool narrow_ready);

// Multi-term preconditioner (pc_rank = k > 1): z ~ (M_k^T M_k + lam2 I)^-1 r,
// M_k the first k Kronecker terms of A, from `pc_inner_iters` PCG steps on
// that system from z = 0, each preconditioned by the one-term KP-SVD solve
// (eq. PreconSolve) and with the Fletcher-Reeves beta.  All scalars live in a
// block of device slots of their own; the kernels follow the outer pause
// flag.  The result changes with r, so the outer iteration is flexible PCG.
static kp_status pc_apply_multiterm(kp_ctx* ctx, const void* r, void* z, double lam2, const double* stat,
                                    const int* flags) {
  const long long N = (long long)ctx->n_r * ctx->n_c;
  const bool f64 = vec64(ctx);
  const size_t vs = f64 ? 8 : 4;
  void *ir = ctx->pc_inner[0], *ir_old = ctx->pc_inner[1], *ip = ctx->pc_inner[2], *iq = ctx->pc_inner[3],
       *iz = ctx->pc_inner[4];
  double* s = ctx->dscal + S_INNER;
  int* f = ctx->dflags + F_INNER;
  const int k = ctx->pc_rank;
  const int m = std::max(1, ctx->pc_inner_iters);
  const int sl = op_inner_slices(ctx);
  PostOp pa;  // alpha of the inner iteration
  pa.kind = POST_ALPHA;
  pa.s = s;
  pa.f = f;
  PostOp pb = pa;  // Fletcher-Reeves beta (the inner flags keep F_FLEX = 0)
  pb.kind = POST_BETA;
  KP_CUDA(cudaMemsetAsync(z, 0, vs * N, ctx->stream));
  KP_CUDA(cudaMemsetAsync(f, 0, 8 * sizeof(int), ctx->stream));
  KP_TRY(copy_vec(ctx, r, ir, N, f64));
  KP_TRY(pc_apply_kp(ctx, ir, iz, lam2, stat, flags, false));
  KP_TRY(dot2_dev(ctx, iz, ir, nullptr, N, f64, s + S_ZR, flags));
  KP_TRY(p_update_dev(ctx, ip, iz, N, f64, nullptr, sl ? (__nv_bfloat16*)ctx->w_img2 : nullptr, sl, N, flags));
  for (int it = 1; it <= m; ++it) {
    bool fused = false;
    KP_TRY(op_apply_K(ctx, ip, iq, lam2, sl > 0, flags, s + S_PQ, &pa, &fused, false, k));
    if (!fused) KP_TRY(dot2_dev(ctx, ip, iq, nullptr, N, f64, s + S_PQ, flags, pa));
    KP_TRY(update_xr_dev(ctx, z, ir, ir_old, ip, iq, N, f64, s + S_ALPHA, s + S_RR, flags));
    if (it == m) break;
    KP_TRY(pc_apply_kp(ctx, ir, iz, lam2, s + S_RR, flags, false));
    KP_TRY(dot2_dev(ctx, iz, ir, ir_old, N, f64, s + S_ZRNEW, flags, pb));
    KP_TRY(p_update_dev(ctx, ip, iz, N, f64, s + S_BETA, sl ? (__nv_bfloat16*)ctx->w_img2 : nullptr, sl, N, flags));
  }
  return KP_OK;
}

kp_status pc_apply(kp_ctx* ctx, const void* r, void* z, double lam2, const double* stat, const int* flags,
                   bool narrow_ready) {
  if (ctx->pc_rank > 1) return pc_apply_multiterm(ctx, r, z, lam2, stat, flags);
  return pc_apply_kp(ctx, r, z, lam2, stat, flags, narrow_ready);
}

static kp_status pc_apply_kp(kp_ctx* ctx, const void* r, void* z, double lam2, const double* stat, const int* flags,
                             bool narrow_ready) {
  if (!pc_is_tc(ctx)) {
    if (vec64(ctx)) return simt_pc<double>(ctx, r, z, lam2, flags);
    return simt_pc<float>(ctx, r, z, lam2, flags);
  }
  OpsState* os = ops(ctx);
  const long long N = (long long)ctx->n_r * ctx->n_c;
  if (!stat) {
    KP_TRY(norm_amax_dev(ctx, r, N, false, os->stat));
    stat = os->stat;
  }
  const int nt = ctx->pc_prec == KP_BF16 ? NT_BF16 : (ctx->pc_prec == KP_F16 ? NT_F16 : NT_E4M3);
  if (nt == NT_E4M3) {
    // FP8: E4M3 holds only [2^-9, 448], so every stage is rescaled: the GEMMs
    // write FP32 with their max |.| (fused in the epilogue), k_quant8 scales
    // by a power of two g into [224, 448) and rounds; the factors' scales
    // s_V, the residual's s_R and the g's are undone in the last GEMM
    const double fscale = (double)ctx->pc_vscale_c * ctx->pc_vscale_r;
    KP_TRY(quantize_dev(ctx, r, N, false, stat, nt, lam2 * fscale * fscale, ctx->pc_in, os->e4m3_slots, flags,
                        os->amax8, 3));
    for (int w = 0; w < 3; ++w) {
      EpiParams e;
      e.mode = EPI_F32;
      e.out = ctx->pc_f32;
      e.ldd = w == 0 || w == 2 ? ctx->n_c : ctx->n_r;
      e.amax_bits = os->amax8 + w;
      if (w == 1) {
        e.sigma32 = ctx->Sigma32;
        e.lam2 = lam2;
      }
      tc_plan_set_runtime(os->P[w], nullptr, flags);
      KP_TRY(tc_plan_run(ctx, os->P[w], &e));
      void* dst = w == 0 ? ctx->pc_t1 : (w == 1 ? ctx->pc_t2 : ctx->pc_t3);
      KP_TRY(quant8_dev(ctx, ctx->pc_f32, N, os->amax8 + w, os->e4m3_slots + 1, w, os->e4m3_slots, os->inv_slot, dst,
                        flags));
    }
    EpiParams e;
    e.mode = EPI_F32;
    e.out = z;
    e.ldd = ctx->n_r;
    tc_plan_set_runtime(os->P[3], os->inv_slot, flags);
    return tc_plan_run(ctx, os->P[3], &e);
  }
  if (!narrow_ready) KP_TRY(quantize_dev(ctx, r, N, false, stat, nt, lam2, ctx->pc_in, os->inv_slot, flags));
  for (int w = 0; w < 4; ++w) {
    EpiParams e;
    e.ldd = w == 0 || w == 2 ? ctx->n_c : ctx->n_r;
    e.narrow = nt;
    if (w < 3) {
      e.mode = EPI_NARROW;
      e.out = w == 0 ? ctx->pc_t1 : (w == 1 ? ctx->pc_t2 : ctx->pc_t3);
      if (w == 1) {
        e.sigma32 = ctx->Sigma32;
        e.lam2 = lam2;
      }
      tc_plan_set_runtime(os->P[w], nullptr, flags);
    } else {
      e.mode = EPI_F32;
      e.out = z;
      tc_plan_set_runtime(os->P[w], os->inv_slot, flags);
    }
    KP_TRY(tc_plan_run(ctx, os->P[w], &e));
  }
  return KP_OK;
}

// the preconditioner's narrow input made from r (F16 / BF16 tensor-core
// preconditioners; nothing to do otherwise), as pc_apply makes it when the
// x / r update has not: after a residual replacement inside the device loop
kp_status pc_prepare_input(kp_ctx* ctx, const void* r, double lam2, const double* stat, const int* flags) {
  if (!pc_is_tc(ctx) || ctx->pc_prec == KP_E4M3 || ctx->pc_rank > 1) return KP_OK;
  const int nt = ctx->pc_prec == KP_BF16 ? NT_BF16 : NT_F16;
  return quantize_dev(ctx, r, (long long)ctx->n_r * ctx->n_c, false, stat, nt, lam2, ctx->pc_in, ops(ctx)->inv_slot,
                      flags);
}

// ------------------------------------------------------------- folded quantisation
bool cg_fusable(kp_ctx* ctx) {
  if (!ctx->cg_fuse || !op_is_tc(ctx) || !pc_is_tc(ctx) || ctx->vec_prec != KP_F32 || ctx->pc_rank > 1) return false;
  if (ctx->pc_prec != KP_F16 && ctx->pc_prec != KP_BF16) return false;
  return ops(ctx)->batched;
}

float* cg_inv_slot(kp_ctx* ctx) { return ops(ctx)->inv_slot; }
