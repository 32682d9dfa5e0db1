// choose_lambda: regularisation parameter in closed form over the KP spectrum
// (Section 2.2; the paper evaluates these with the Kronecker product
// approximate SVD, Section 5.1).
//
// b_hat = vec(U_c^T B U_r), x_hat = vec(V_c^T X_true V_r) (FP64 GEMMs), and
// with phi_i = lam^2 / (sigma_i^2 + lam^2) in (0, 1]:
//   GCV  (eq. GCVTikSVD)    G(lam)   = N sum (phi b_hat)^2 / (sum phi)^2
//   wGCV (eq. wGCVTikSVD)   G_w(lam) = N sum (phi b_hat)^2 / (sum ((1-w) sigma^2 + lam^2) / d)^2
//   disc (eq. DSCTikSVD)    D(lam)   = sum (phi b_hat)^2 - eps^2
//   opt  (eq. OptTikSVD)    O(lam)   = sum (sigma b_hat / d - x_hat)^2
// (the lam^4 factors of GCV cancel, so the phi form equals eq. GCVTikSVD and
// keeps every term bounded).  Minimisation: the 400 log-spaced grid values
// are evaluated in one launch (FP32 terms, FP64 block sums), the best grid
// point is re-checked in FP64 with its neighbours, then refined in the two
// adjacent cells in FP64: GCV / wGCV by Newton on log G in t = log lam with
// analytic derivatives of the sums (one pass gives all six), bisection as
// safeguard; the optimal-error lambda by golden-section search.  The
// discrepancy root is bracketed by decades in log lam and refined by the
// same safeguarded Newton (D' > 0).
#include <algorithm>
#include <cmath>
#include <vector>

#include "kp_internal.h"
#include "kp_vec.cuh"

namespace {

constexpr int NGRID = 400;
constexpr int GPB = 16;  // grid values per block
constexpr int LT = 256;
constexpr size_t LAM_FEAT_BYTES = 127 * (sizeof(unsigned long long) + sizeof(double));  // feature bins

enum LMethod { LM_GCV = 0, LM_WGCV = 1, LM_DISC = 2, LM_OPT = 3, LM_TRACE = 4 };

struct LamData {
  const double* s2;   // sigma^2
  const double* sg;   // sigma
  const double* bh;   // b_hat
  const double* xh;   // x_hat (opt)
  const float* s2f;
  const float* sgf;
  const float* bhf;
  const float* xhf;
  long long n;
  double omega;
  int method;
};

// 1 / x in FP64 from an FP32 reciprocal and two Newton steps (FP64 division
// is a long instruction sequence on this part); x > 0
__device__ __forceinline__ double drcp(double x) {
  if (!(x > 1e-30 && x < 1e30)) return 1.0 / x;
  double r = (double)__frcp_rn((float)x);
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}
__device__ __forceinline__ float drcp(float x) { return __frcp_rn(x); }

// per-element contributions (s1, s2) of the sums for one lambda
template <typename T>
__device__ __forceinline__ void terms(int method, T s2, T sg, T bh, T xh, T lam2, T omega, T& a, T& b) {
  const T rd = drcp(s2 + lam2);
  const T phi = lam2 * rd;
  switch (method) {
    case LM_OPT: {
      const T e = sg * bh * rd - xh;
      a = e * e;
      b = T(0);
      break;
    }
    case LM_TRACE:
      a = T(0);
      b = ((T(1) - omega) * s2 + lam2) * rd;
      break;
    default: {  // GCV / wGCV / discrepancy share the residual sum
      const T pb = phi * bh;
      a = pb * pb;
      b = ((T(1) - omega) * s2 + lam2) * rd;
      break;
    }
  }
}
// FP32 form for the grid scan: one reciprocal per term (the grid only
// brackets the minimum; the FP64 forms above decide it)
__device__ __forceinline__ void terms_grid(int method, float s2, float sg, float bh, float xh, float lam2, float omega,
                                           float& a, float& b) {
  const float rd = __frcp_rn(s2 + lam2);
  if (method == LM_OPT) {
    const float e = sg * bh * rd - xh;
    a = e * e;
    b = 0.f;
  } else if (method == LM_TRACE) {
    a = 0.f;
    b = fmaf(1.f - omega, s2, lam2) * rd;
  } else {
    const float pb = lam2 * rd * bh;
    a = pb * pb;
    b = fmaf(1.f - omega, s2, lam2) * rd;
  }
}

__device__ __forceinline__ double lwarp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// grid scan: blockIdx.y = group of GPB lambdas, blockIdx.x = element chunk
__global__ void __launch_bounds__(LT) k_lam_grid(LamData d, const double* __restrict__ lam2s, int ng,
                                                 double* __restrict__ part) {
  const int g0 = blockIdx.y * GPB;
  float l2[GPB];
  float acc_a[GPB], acc_b[GPB];
#pragma unroll
  for (int q = 0; q < GPB; ++q) {
    l2[q] = (g0 + q < ng) ? (float)lam2s[g0 + q] : 1.f;
    acc_a[q] = 0.f;
    acc_b[q] = 0.f;
  }
  const float om = (float)d.omega;
  const bool opt = d.method == LM_OPT;
  for (long long i = blockIdx.x * (long long)LT + threadIdx.x; i < d.n; i += (long long)gridDim.x * LT) {
    const float s2 = d.s2f[i], bh = d.bhf[i];
    const float sg = opt ? d.sgf[i] : 0.f, xh = opt ? d.xhf[i] : 0.f;
#pragma unroll
    for (int q = 0; q < GPB; ++q) {
      float a, b;
      terms_grid(d.method, s2, sg, bh, xh, l2[q], om, a, b);
      acc_a[q] += a;
      acc_b[q] += b;
    }
  }
  // warp sums in FP32 (the grid only brackets the minimum), block sums in FP64
  __shared__ double sh[LT / 32][GPB][2];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < GPB; ++q) {
    float a = acc_a[q], b = acc_b[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
      sh[wid][q][0] = (double)a;
      sh[wid][q][1] = (double)b;
    }
  }
  __syncthreads();
  if (threadIdx.x < GPB * 2) {
    const int q = threadIdx.x >> 1, w = threadIdx.x & 1;
    double t = 0.0;
    for (int k = 0; k < LT / 32; ++k) t += sh[k][q][w];
    if (g0 + q < ng) part[((long long)(g0 + q) * gridDim.x + blockIdx.x) * 2 + w] = t;
  }
}

__global__ void k_lam_grid_finish(const double* __restrict__ part, int nchunks, int ng, double* __restrict__ out) {
  const int g = blockIdx.x;
  if (g >= ng) return;
  double a = 0, b = 0;
  for (int c = threadIdx.x; c < nchunks; c += blockDim.x) {
    a += part[((long long)g * nchunks + c) * 2];
    b += part[((long long)g * nchunks + c) * 2 + 1];
  }
  __shared__ double sa[256], sb[256];
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sa[threadIdx.x] += sa[threadIdx.x + o];
      sb[threadIdx.x] += sb[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[2 * g] = sa[0];
    out[2 * g + 1] = sb[0];
  }
}

// FP64 evaluation of (s1, s2) for a few lambdas (one per blockIdx.y)
__global__ void __launch_bounds__(LT) k_lam_eval64(LamData d, const double* __restrict__ lam2s,
                                                   double* __restrict__ part) {
  const double l2 = lam2s[blockIdx.y];
  double a = 0, b = 0;
  for (long long i = blockIdx.x * (long long)LT + threadIdx.x; i < d.n; i += (long long)gridDim.x * LT) {
    double ta, tb;
    terms<double>(d.method, d.s2[i], d.sg[i], d.bh[i], d.xh ? d.xh[i] : 0.0, l2, d.omega, ta, tb);
    a += ta;
    b += tb;
  }
  __shared__ double sh[LT / 32][2];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  a = lwarp_sum(a);
  b = lwarp_sum(b);
  if (lane == 0) {
    sh[wid][0] = a;
    sh[wid][1] = b;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double t = 0;
    for (int k = 0; k < LT / 32; ++k) t += sh[k][threadIdx.x];
    part[((long long)blockIdx.y * gridDim.x + blockIdx.x) * 2 + threadIdx.x] = t;
  }
}

// FP64 sums and their first two derivatives in t = log(lam) at one lambda,
// for the residual family (phi = lam^2 / d, psi = sigma^2 / d = 1 - phi):
//   s1 = sum phi^2 b^2          s1' = sum 4 phi^2 psi b^2     s1'' = sum 8 phi^2 psi (2 - 3 phi) b^2
//   s2 = sum (1 - w + w phi)    s2' = w sum 2 phi psi         s2'' = w sum 4 phi psi (1 - 2 phi)
__global__ void __launch_bounds__(LT) k_lam_deriv64(LamData d, double lam2, double* __restrict__ part) {
  double acc[6] = {0, 0, 0, 0, 0, 0};
  const double w = d.omega;
  for (long long i = blockIdx.x * (long long)LT + threadIdx.x; i < d.n; i += (long long)gridDim.x * LT) {
    const double s2 = d.s2[i], b = d.bh[i];
    const double rd = drcp(s2 + lam2);
    const double phi = lam2 * rd, psi = s2 * rd, b2 = b * b;
    const double pp = phi * psi;
    acc[0] = fma(phi * phi, b2, acc[0]);
    acc[1] += 1.0 - w + w * phi;
    acc[2] = fma(4.0 * phi * pp, b2, acc[2]);
    acc[3] += 2.0 * w * pp;
    acc[4] = fma(8.0 * phi * pp * (2.0 - 3.0 * phi), b2, acc[4]);
    acc[5] += 4.0 * w * pp * (1.0 - 2.0 * phi);
  }
  __shared__ double sh[LT / 32][6];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const double v = lwarp_sum(acc[k]);
    if (lane == 0) sh[wid][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double t = 0;
    for (int q = 0; q < LT / 32; ++q) t += sh[q][threadIdx.x];
    part[(long long)blockIdx.x * 6 + threadIdx.x] = t;
  }
}

__global__ void k_sum6_finish(const double* __restrict__ part, int nchunks, double* __restrict__ out) {
  __shared__ double sh[6][256];
  for (int k = 0; k < 6; ++k) {
    double a = 0;
    for (int c = threadIdx.x; c < nchunks; c += blockDim.x) a += part[(long long)c * 6 + k];
    sh[k][threadIdx.x] = a;
  }
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int k = 0; k < 6; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 6) out[threadIdx.x] = sh[threadIdx.x][0];
}

// spectrum-only arrays (once per kp_setup)
__global__ void k_prep_sigma(const double* __restrict__ Sigma, long long n, double* __restrict__ s2,
                             float* __restrict__ s2f, float* __restrict__ sgf) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double s = Sigma[i];
    s2[i] = s * s;
    s2f[i] = (float)(s * s);
    sgf[i] = (float)s;
  }
}
// coefficient arrays (every call)
__global__ void k_prep_coeffs(const double* __restrict__ bh, const double* __restrict__ xh, long long n,
                              float* __restrict__ bhf, float* __restrict__ xhf) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    bhf[i] = (float)bh[i];
    if (xh) xhf[i] = (float)xh[i];
  }
}

template <typename T>
__global__ void k_to_f64(const T* __restrict__ x, long long n, double* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

// per-block max |S| and min |S| over |S| > 0 (part[2 b], part[2 b + 1]);
// then one block combines the partials
__global__ void k_absmax_min_part(const double* __restrict__ S, long long n, double* __restrict__ part) {
  double mx = 0.0, mn = INFINITY;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double a = fabs(S[i]);
    mx = fmax(mx, a);
    if (a > 0) mn = fmin(mn, a);
  }
  __shared__ double smx[256], smn[256];
  smx[threadIdx.x] = mx;
  smn[threadIdx.x] = mn;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      smx[threadIdx.x] = fmax(smx[threadIdx.x], smx[threadIdx.x + o]);
      smn[threadIdx.x] = fmin(smn[threadIdx.x], smn[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = smx[0];
    part[2 * blockIdx.x + 1] = smn[0];
  }
}
__global__ void k_absmax_min_finish(const double* __restrict__ part, int nb, double* __restrict__ out) {
  double mx = 0.0, mn = INFINITY;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    mx = fmax(mx, part[2 * i]);
    mn = fmin(mn, part[2 * i + 1]);
  }
  __shared__ double smx[256], smn[256];
  smx[threadIdx.x] = mx;
  smn[threadIdx.x] = mn;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      smx[threadIdx.x] = fmax(smx[threadIdx.x], smx[threadIdx.x + o]);
      smn[threadIdx.x] = fmin(smn[threadIdx.x], smn[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = smx[0];
    out[1] = smn[0];
  }
}

}  // namespace

struct LamCtx {
  kp_ctx* ctx;
  LamData d;
  double* lam2_dev;
  double* part;
  double* sums;
  int chunks;
};

// FP64 sums (s1, s2) at the given lambdas (host), up to 16 at once
static kp_status eval64(LamCtx& L, const double* lams, int k, double* s1, double* s2) {
  kp_ctx* ctx = L.ctx;
  double l2[16];
  for (int i = 0; i < k; ++i) l2[i] = lams[i] * lams[i];
  KP_CUDA(cudaMemcpyAsync(L.lam2_dev, l2, sizeof(double) * k, cudaMemcpyHostToDevice, ctx->stream));
  dim3 grid(L.chunks, k);
  k_lam_eval64<<<grid, LT, 0, ctx->stream>>>(L.d, L.lam2_dev, L.part);
  KP_LAUNCHED(ctx);
  k_lam_grid_finish<<<k, 256, 0, ctx->stream>>>(L.part, L.chunks, k, L.sums);
  KP_LAUNCHED(ctx);
  double h[32];
  KP_CUDA(cudaMemcpyAsync(h, L.sums, sizeof(double) * 2 * k, cudaMemcpyDeviceToHost, ctx->stream));
  KP_CUDA(kp_wait(ctx, ctx->stream));
  for (int i = 0; i < k; ++i) {
    s1[i] = h[2 * i];
    s2[i] = h[2 * i + 1];
  }
  return KP_OK;
}

// s[0..5] = (s1, s2, s1', s2', s1'', s2'') at lam
static kp_status deriv64(LamCtx& L, double lam, double* s6) {
  kp_ctx* ctx = L.ctx;
  k_lam_deriv64<<<L.chunks, LT, 0, ctx->stream>>>(L.d, lam * lam, L.part);
  KP_LAUNCHED(ctx);
  k_sum6_finish<<<1, 256, 0, ctx->stream>>>(L.part, L.chunks, L.sums);
  KP_LAUNCHED(ctx);
  KP_CUDA(cudaMemcpyAsync(s6, L.sums, sizeof(double) * 6, cudaMemcpyDeviceToHost, ctx->stream));
  KP_CUDA(kp_wait(ctx, ctx->stream));
  return KP_OK;
}

static double objective(int method, double s1, double s2, double N, double eps) {
  switch (method) {
    case LM_GCV:
    case LM_WGCV: return N * s1 / (s2 * s2);
    case LM_DISC: return s1 - eps * eps;
    case LM_OPT: return s1;
    default: return s2;
  }
}

static kp_status f64_at(LamCtx& L, int method, double lam, double N, double eps, double* f) {
  double s1, s2;
  KP_TRY(eval64(L, &lam, 1, &s1, &s2));
  *f = objective(method, s1, s2, N, eps);
  return KP_OK;
}

// With coeffs_only non-null: stop after b_hat = vec(U_c^T B U_r) and the
// spectrum's bounds, returning the device pointer to b_hat (FP64, N values,
// valid until the next call on the context) instead of choosing lambda.
static kp_status choose_lambda_impl(kp_ctx* ctx, const void* b, kp_lambda_method method, double param,
                                    const void* x_true, double* lambda_out, const double** coeffs_only = nullptr,
                                    void** feat_ws_out = nullptr) {
  const int n_r = ctx->n_r, n_c = ctx->n_c;
  const long long N = (long long)n_r * n_c;
  cudaStream_t st = ctx->stream;
  const bool f64 = ctx->vec_prec == KP_F64;
  const int gr = std::max(1, std::min((int)((N + 255) / 256), ctx->sm_count * 8));
  // scratch: allocated at the first call after a kp_setup, kept with the problem
  if (!ctx->lam_ws) {
    const int chunks_max = std::max(1, std::min((int)((N + LT - 1) / LT), ctx->sm_count * 2));
    auto r256 = [](size_t b) { return (b + 255) & ~(size_t)255; };  // as `take` below rounds
    const size_t bytes = 5 * r256(sizeof(double) * (size_t)N) + 4 * r256(sizeof(float) * (size_t)N) +
                         r256(sizeof(double) * NGRID) + r256(sizeof(double) * 2 * (size_t)chunks_max * NGRID) +
                         r256(sizeof(double) * 2 * NGRID) + r256(sizeof(double) * 2) + r256(LAM_FEAT_BYTES);
    KP_TRY(kp_alloc(ctx, &ctx->lam_ws, bytes));
  }
  char* wp = (char*)ctx->lam_ws;
  auto take = [&](size_t bytes) {
    void* q = wp;
    wp += (bytes + 255) & ~(size_t)255;
    return q;
  };
  double* B64 = (double*)take(sizeof(double) * N);
  double* T = (double*)take(sizeof(double) * N);
  double* bh = (double*)take(sizeof(double) * N);
  double* s2 = (double*)take(sizeof(double) * N);
  double* xh = (double*)take(sizeof(double) * N);
  float* s2f = (float*)take(sizeof(float) * N);
  float* sgf = (float*)take(sizeof(float) * N);
  float* bhf = (float*)take(sizeof(float) * N);
  float* xhf = (float*)take(sizeof(float) * N);
  double* lam2_dev = (double*)take(sizeof(double) * NGRID);
  const int chunks = std::max(1, std::min((int)((N + LT - 1) / LT), ctx->sm_count * 2));
  double* part = (double*)take(sizeof(double) * 2 * (size_t)chunks * NGRID);
  double* sums = (double*)take(sizeof(double) * 2 * NGRID);
  double* ext = (double*)take(sizeof(double) * 2);
  void* feat_ws = take(LAM_FEAT_BYTES);  // bins of kp_lambda_features
  if (method != KP_LAMBDA_OPT) {
    xh = nullptr;
    xhf = nullptr;
  }

  // coefficients in the KP basis: Y^ = U_c^T Y U_r (or V for x_true); in
  // FP32 from FP32 images when the setup kept FP32 copies of the bases
  auto kp_coeffs32 = [&](const float* img, const float* Lc, const float* Rr, double* out) -> kp_status {
    float* T32 = (float*)T;  // T holds N doubles: room for two FP32 images
    float* O32 = T32 + N;
    if (ctx->setup_tc) {
      // tensor cores, inputs as three bf16 slices (FP32-level products); the
      // bases' slices and the plans are made once per setup
      kp_ctx::LamTc& lt = ctx->lam_tc[Lc == ctx->Uc32 ? 0 : 1];
      if (!ctx->lam_img16) {
        KP_TRY(kp_alloc(ctx, &ctx->lam_img16, sizeof(__nv_bfloat16) * 3 * N));
        KP_TRY(kp_alloc(ctx, &ctx->lam_t16, sizeof(__nv_bfloat16) * 3 * N));
        KP_TRY(kp_alloc(ctx, (void**)&ctx->lam_t32, sizeof(float) * N));
        KP_TRY(kp_alloc(ctx, (void**)&ctx->lam_o32, sizeof(float) * N));
      }
      if (!lt.p1) {
        KP_TRY(kp_alloc(ctx, &lt.L16, sizeof(__nv_bfloat16) * 3 * (size_t)n_r * n_r));
        KP_TRY(kp_alloc(ctx, &lt.R16, sizeof(__nv_bfloat16) * 3 * (size_t)n_c * n_c));
        KP_TRY(tc_operand_slices(ctx, Lc, false, (long long)n_r * n_r, 3, lt.L16));
        KP_TRY(tc_operand_slices(ctx, Rr, false, (long long)n_c * n_c, 3, lt.R16));
        // T[i'][j] = sum_i Lc[i, i'] Y[i, j]; out[l][i'] = sum_j Rr[j, l] T[i'][j]
        KP_TRY(tc_product_plan(ctx, lt.L16, n_r, ctx->lam_img16, n_c, n_r, 3, ctx->lam_t32, &lt.p1));
        KP_TRY(tc_product_plan(ctx, lt.R16, n_c, ctx->lam_t16, n_r, n_c, 3, ctx->lam_o32, &lt.p2));
      }
      KP_TRY(tc_operand_slices(ctx, img, false, N, 3, ctx->lam_img16));
      KP_TRY(tc_plan_run(ctx, lt.p1, nullptr));
      KP_TRY(tc_operand_slices(ctx, ctx->lam_t32, false, N, 3, ctx->lam_t16));
      KP_TRY(tc_plan_run(ctx, lt.p2, nullptr));
      k_to_f64<float><<<gr, 256, 0, st>>>(ctx->lam_o32, N, out);
      KP_LAUNCHED(ctx);
      return KP_OK;
    }
    GemmDesc g1;
    g1.M = n_r;
    g1.N = n_c;
    g1.K = n_r;
    g1.A.ptr = Lc;
    g1.A.ld = n_r;
    g1.B.ptr = img;
    g1.B.ld = n_r;
    g1.epi.mode = EPI_T;
    g1.epi.out = T32;
    g1.epi.ldd = n_c;
    KP_TRY(simt_gemm<float>(ctx, g1));
    GemmDesc g2;
    g2.M = n_c;
    g2.N = n_r;
    g2.K = n_c;
    g2.A.ptr = Rr;
    g2.A.ld = n_c;
    g2.B.ptr = T32;
    g2.B.ld = n_c;
    g2.epi.mode = EPI_T;
    g2.epi.out = O32;
    g2.epi.ldd = n_r;
    KP_TRY(simt_gemm<float>(ctx, g2));
    k_to_f64<float><<<gr, 256, 0, st>>>(O32, N, out);
    KP_LAUNCHED(ctx);
    return KP_OK;
  };
  auto kp_coeffs = [&](const void* img, const double* Lc, const double* Rr, double* out) -> kp_status {
    if (!f64 && ctx->Uc32) {
      const bool u = Lc == ctx->Uc;
      return kp_coeffs32((const float*)img, u ? ctx->Uc32 : ctx->Vc32, u ? ctx->Ur32 : ctx->Vr32, out);
    }
    const double* src;
    if (f64) {
      src = (const double*)img;
    } else {
      k_to_f64<float><<<gr, 256, 0, st>>>((const float*)img, N, B64);
      KP_LAUNCHED(ctx);
      src = B64;
    }
    GemmDesc g1;  // T[i'][j] = sum_i Lc[i, i'] Y[i, j]
    g1.M = n_r;
    g1.N = n_c;
    g1.K = n_r;
    g1.A.ptr = Lc;
    g1.A.ld = n_r;
    g1.B.ptr = src;
    g1.B.ld = n_r;
    g1.epi.mode = EPI_T;
    g1.epi.out = T;
    g1.epi.ldd = n_c;
    KP_TRY(simt_gemm<double>(ctx, g1));
    GemmDesc g2;  // out[l][i'] = sum_j Rr[j, l] T[i'][j]  (column-major result)
    g2.M = n_c;
    g2.N = n_r;
    g2.K = n_c;
    g2.A.ptr = Rr;
    g2.A.ld = n_c;
    g2.B.ptr = T;
    g2.B.ld = n_c;
    g2.epi.mode = EPI_T;
    g2.epi.out = out;
    g2.epi.ldd = n_r;
    return simt_gemm<double>(ctx, g2);
  };
  if (!ctx->lam_sigma_ready) {  // spectrum-only arrays and bounds, once per setup
    k_prep_sigma<<<gr, 256, 0, st>>>(ctx->Sigma64, N, s2, s2f, sgf);
    KP_LAUNCHED(ctx);
    const int nb = std::max(1, std::min((int)((N + 255) / 256), ctx->sm_count * 4));
    k_absmax_min_part<<<nb, 256, 0, st>>>(ctx->Sigma64, N, part);
    k_absmax_min_finish<<<1, 256, 0, st>>>(part, nb, ext);
    ctx->launches += 2;
    KP_CUDA(cudaMemcpyAsync(ctx->lam_sigma_ext, ext, sizeof(double) * 2, cudaMemcpyDeviceToHost, st));
  }
  KP_TRY(kp_coeffs(b, ctx->Uc, ctx->Ur, bh));
  if (method == KP_LAMBDA_OPT) KP_TRY(kp_coeffs(x_true, ctx->Vc, ctx->Vr, xh));
  k_prep_coeffs<<<gr, 256, 0, st>>>(bh, xh, N, bhf, xhf);
  KP_LAUNCHED(ctx);
  if (!ctx->lam_sigma_ready) {
    KP_CUDA(kp_wait(ctx, st));
    ctx->lam_sigma_ready = true;
  }
  if (coeffs_only) {
    *coeffs_only = bh;
    if (feat_ws_out) *feat_ws_out = feat_ws;
    return KP_OK;
  }
  const double* he = ctx->lam_sigma_ext;
  const double smax = he[0];
  const double smin = std::isfinite(he[1]) ? he[1] : smax;
  if (!(smax > 0)) {
    kp_set_error("choose_lambda: KP spectrum is zero");
    return KP_ENUMERIC;
  }
  double lo = std::max(smin, 1e-10 * smax), hi = smax;

  LamCtx L;
  L.ctx = ctx;
  L.d.s2 = s2;
  L.d.sg = ctx->Sigma64;
  L.d.bh = bh;
  L.d.xh = xh;
  L.d.s2f = s2f;
  L.d.sgf = sgf;
  L.d.bhf = bhf;
  L.d.xhf = xhf;
  L.d.n = N;
  L.d.omega = 1.0;
  L.lam2_dev = lam2_dev;
  L.part = part;
  L.sums = sums;
  L.chunks = chunks;
  const double Nd = (double)N;

  int lm = LM_GCV;
  double eps = 0.0;
  switch (method) {
    case KP_LAMBDA_GCV: lm = LM_GCV; break;
    case KP_LAMBDA_WGCV: lm = LM_WGCV; L.d.omega = param; break;
    case KP_LAMBDA_DISCREPANCY: lm = LM_DISC; eps = param; break;
    case KP_LAMBDA_OPT: lm = LM_OPT; break;
  }
  L.d.method = lm == LM_WGCV ? LM_GCV : lm;  // wGCV shares the GCV sums with omega != 1

  if (lm == LM_DISC) {
    // D increases with lambda; D(inf) = ||b_hat||^2 - eps^2
    double bb;
    {
      double s1, s2v, big = 1e30 * smax;
      KP_TRY(eval64(L, &big, 1, &s1, &s2v));
      bb = s1;
    }
    if (!std::isfinite(bb)) {
      kp_set_error("choose_lambda: the KP coefficients of b are not finite");
      return KP_ENUMERIC;
    }
    if (!(bb > eps * eps)) {
      kp_set_error("choose_lambda: discrepancy has no root (eps >= ||b_hat||)");
      return KP_ENOROOT;
    }
    double tl = std::log(lo), th = std::log(hi), fl, fh;
    const double tfloor = std::log(1e-16 * hi);
    KP_TRY(f64_at(L, lm, lo, Nd, eps, &fl));
    while (fl > 0) {
      tl -= std::log(10.0);
      if (tl < tfloor) {
        kp_set_error("choose_lambda: discrepancy has no root above 1e-16 sigma_max");
        return KP_ENOROOT;
      }
      KP_TRY(f64_at(L, lm, std::exp(tl), Nd, eps, &fl));
    }
    KP_TRY(f64_at(L, lm, hi, Nd, eps, &fh));
    int guard = 0;
    while (fh < 0 && guard++ < 64) {
      th += std::log(10.0);
      KP_TRY(f64_at(L, lm, std::exp(th), Nd, eps, &fh));
    }
    if (fh < 0) {
      kp_set_error("choose_lambda: discrepancy bracket failed");
      return KP_ENOROOT;
    }
    // safeguarded Newton in t = log lambda (D' = s1' > 0), bisection when a
    // step leaves the bracket
    double t = 0.5 * (tl + th);
    for (int it = 0; it < 200; ++it) {
      double s6[6];
      KP_TRY(deriv64(L, std::exp(t), s6));
      const double D = s6[0] - eps * eps, Dp = s6[2];
      if (D == 0.0) break;
      if (D < 0) tl = t; else th = t;
      double tn = (Dp > 0) ? t - D / Dp : 0.5 * (tl + th);
      if (!(tn > tl && tn < th)) tn = 0.5 * (tl + th);
      const bool done = std::fabs(tn - t) <= 1e-14 * std::max(1.0, std::fabs(t)) || th - tl <= 1e-15 * std::max(1.0, std::fabs(t));
      t = tn;
      if (done) break;
    }
    *lambda_out = std::exp(t);
    return KP_OK;
  }

  if (lm == LM_WGCV && param > 1.0) {
    // start the search where trace(I - omega A A^+) > 0 (bisection in log lam)
    L.d.method = LM_TRACE;
    double tr;
    KP_TRY(f64_at(L, LM_TRACE, lo, Nd, 0.0, &tr));
    if (!(tr > 0)) {
      double trh;
      KP_TRY(f64_at(L, LM_TRACE, hi, Nd, 0.0, &trh));
      if (!(trh > 0)) {
        lo = hi;
      } else {
        double a = std::log(lo), bnd = std::log(hi);
        for (int it = 0; it < 200 && bnd - a > 1e-15 * std::max(1.0, std::fabs(a)); ++it) {
          double m = 0.5 * (a + bnd), tm;
          KP_TRY(f64_at(L, LM_TRACE, std::exp(m), Nd, 0.0, &tm));
          if (tm > 0)
            bnd = m;
          else
            a = m;
        }
        lo = std::exp(bnd);
      }
    }
    L.d.method = LM_GCV;
  }

  // ---- grid scan (all grid values in one launch)
  std::vector<double> tg(NGRID), l2(NGRID);
  const double tlo = std::log(lo), thi = std::log(hi);
  for (int g = 0; g < NGRID; ++g) {
    tg[g] = NGRID > 1 ? tlo + (thi - tlo) * g / (NGRID - 1) : tlo;
    double l = std::exp(tg[g]);
    l2[g] = l * l;
  }
  KP_CUDA(cudaMemcpyAsync(lam2_dev, l2.data(), sizeof(double) * NGRID, cudaMemcpyHostToDevice, st));
  {
    dim3 grid(chunks, (NGRID + GPB - 1) / GPB);
    k_lam_grid<<<grid, LT, 0, st>>>(L.d, lam2_dev, NGRID, part);
    KP_LAUNCHED(ctx);
    k_lam_grid_finish<<<NGRID, 256, 0, st>>>(part, chunks, NGRID, sums);
    KP_LAUNCHED(ctx);
  }
  std::vector<double> hsum(2 * NGRID);
  KP_CUDA(cudaMemcpyAsync(hsum.data(), sums, sizeof(double) * 2 * NGRID, cudaMemcpyDeviceToHost, st));
  KP_CUDA(kp_wait(ctx, st));
  // every grid sum is bounded for finite data (phi in [0, 1], d >= lam^2 > 0):
  // a NaN or Inf comes from b (or x_true) and would leave no minimum to find
  for (int g = 0; g < 2 * NGRID; ++g) {
    if (!std::isfinite(hsum[g])) {
      kp_set_error("choose_lambda: the KP coefficients of %s are not finite", lm == LM_OPT ? "b or x_true" : "b");
      return KP_ENUMERIC;
    }
  }
  int best = 0;
  double bv = INFINITY;
  for (int g = 0; g < NGRID; ++g) {
    double f = objective(lm, hsum[2 * g], hsum[2 * g + 1], Nd, eps);
    if (f <= bv) {  // ties -> larger lambda
      bv = f;
      best = g;
    }
  }
  // FP64 re-check of the best grid point and its neighbours
  double t_start;
  {
    int g0 = std::max(0, best - 2), g1 = std::min(NGRID - 1, best + 2);
    double lams[5], s1v[5], s2v[5], fv[5];
    int k = g1 - g0 + 1;
    for (int i = 0; i < k; ++i) lams[i] = std::exp(tg[g0 + i]);
    KP_TRY(eval64(L, lams, k, s1v, s2v));
    bv = INFINITY;
    for (int i = 0; i < k; ++i) {
      fv[i] = objective(lm, s1v[i], s2v[i], Nd, eps);
      if (fv[i] <= bv) {
        bv = fv[i];
        best = g0 + i;
      }
    }
    // start of the refinement: the vertex of the parabola through the best
    // point and its two neighbours (in t = log lambda, on log f), when it is
    // a minimum inside their span; else the best grid point
    t_start = tg[best];
    const int ib = best - g0;
    if (ib > 0 && ib < k - 1 && fv[ib - 1] > 0 && fv[ib] > 0 && fv[ib + 1] > 0) {
      const double fl = std::log(fv[ib - 1]), f0 = std::log(fv[ib]), fr = std::log(fv[ib + 1]);
      const double h = tg[best + 1] - tg[best];
      const double curv = fl - 2.0 * f0 + fr;
      if (curv > 0 && h > 0) {
        const double tv = tg[best] + 0.5 * h * (fl - fr) / curv;
        if (tv > tg[best - 1] && tv < tg[best + 1]) t_start = tv;
      }
    }
  }
  double a = tg[std::max(best - 1, 0)], c = tg[std::min(best + 1, NGRID - 1)];
  if (lm == LM_GCV || lm == LM_WGCV) {
    // safeguarded Newton on g(t) = log s1 - 2 log s2 (= log G - log N) in
    // t = log lambda over [t_{best-1}, t_{best+1}], from the parabola's vertex
    double t = t_start;
    for (int it = 0; it < 60; ++it) {
      double s6[6];
      KP_TRY(deriv64(L, std::exp(t), s6));
      if (!(s6[1] > 0.0) || !(s6[0] > 0.0)) {  // below the wGCV lower limit: move right
        a = t;
        t = 0.5 * (a + c);
        continue;
      }
      const double r1 = s6[2] / s6[0], r2 = s6[3] / s6[1];
      const double gp = r1 - 2.0 * r2;
      const double gpp = s6[4] / s6[0] - r1 * r1 - 2.0 * (s6[5] / s6[1] - r2 * r2);
      if (gp > 0) c = t; else a = t;
      double tn = (gpp > 0) ? t - gp / gpp : 0.5 * (a + c);
      if (!(tn > a && tn < c)) tn = 0.5 * (a + c);
      const bool done = std::fabs(tn - t) <= 1e-12 * std::max(1.0, std::fabs(t)) || c - a <= 1e-12 * std::max(1.0, std::fabs(t));
      t = tn;
      if (done || gp == 0.0) break;
    }
    double ft;
    KP_TRY(f64_at(L, lm, std::exp(t), Nd, eps, &ft));
    *lambda_out = std::exp(ft <= bv ? t : tg[best]);
    return KP_OK;
  }
  // optimal-error lambda: golden-section search in log lambda over the cell pair
  const double gr_ = 0.5 * (std::sqrt(5.0) - 1.0);
  double x1 = c - gr_ * (c - a), x2 = a + gr_ * (c - a), f1, f2;
  KP_TRY(f64_at(L, lm, std::exp(x1), Nd, eps, &f1));
  KP_TRY(f64_at(L, lm, std::exp(x2), Nd, eps, &f2));
  for (int it = 0; it < 200 && (c - a) > 1e-12; ++it) {
    if (f1 < f2) {
      c = x2;
      x2 = x1;
      f2 = f1;
      x1 = c - gr_ * (c - a);
      KP_TRY(f64_at(L, lm, std::exp(x1), Nd, eps, &f1));
    } else {
      a = x1;
      x1 = x2;
      f1 = f2;
      x2 = a + gr_ * (c - a);
      KP_TRY(f64_at(L, lm, std::exp(x2), Nd, eps, &f2));
    }
  }
  double tbest = f1 < f2 ? x1 : x2, fbest = std::min(f1, f2);
  if (!(fbest <= bv)) tbest = tg[best];
  *lambda_out = std::exp(tbest);
  return KP_OK;
}

extern "C" kp_status choose_lambda(kp_ctx* ctx, const void* b, kp_lambda_method method, double param,
                                   const void* x_true, double* lambda_out) {
  KP_TRY(kp_check_ready(ctx));
  if (!b || !lambda_out) {
    kp_set_error("choose_lambda: NULL argument");
    return KP_EINVAL;
  }
  if (method < KP_LAMBDA_GCV || method > KP_LAMBDA_OPT) {
    kp_set_error("choose_lambda: unknown method %d", (int)method);
    return KP_EINVAL;
  }
  if (method == KP_LAMBDA_OPT && !x_true) {
    kp_set_error("choose_lambda: KP_LAMBDA_OPT needs x_true");
    return KP_EINVAL;
  }
  if (method == KP_LAMBDA_DISCREPANCY && !(param > 0.0)) {
    kp_set_error("choose_lambda: discrepancy needs eps > 0");
    return KP_EINVAL;
  }
  if (method == KP_LAMBDA_WGCV && !(param > 0.0)) {
    kp_set_error("choose_lambda: wGCV needs omega > 0");
    return KP_EINVAL;
  }
  KP_TRY(kp_enter(ctx));
  kp_status s = choose_lambda_impl(ctx, b, method, param, x_true, lambda_out);
  kp_status l = kp_leave(ctx);
  return s != KP_OK ? s : l;
}

// ---------------------------------------------------------------- spectral features
// Features of a problem for the learned lambda (not in the paper; its
// Section 5 asks for a systematic parameter choice): with s2 = Sigma^2 and
// s2max = max s2, component i goes to bin j = floor(-log10(s2_i / s2max)
// NB / DEC) when s2_i > s2max 10^-DEC (NB = 127 bins over DEC = 16 decades);
// f[j] = log10((sum_bin b_hat^2 + TINY s2max) / (count_j + 1)),
// f[NB + j] = log10((count_j + 1) / N), f[254] = log10 of the mean b_hat^2
// over the deepest bins that together hold >= N / 8 components (a noise
// estimate), f[255] = log10(s2max).
namespace {
constexpr int FT_NB = 127;
constexpr double FT_DEC = 16.0, FT_TINY = 1e-30;

__global__ void k_feat_bins(const double* __restrict__ sig, const double* __restrict__ bh, long long n, double s2max,
                            unsigned long long* __restrict__ cnt, double* __restrict__ sb) {
  __shared__ unsigned int c_sh[FT_NB];
  __shared__ double b_sh[FT_NB];
  for (int j = threadIdx.x; j < FT_NB; j += blockDim.x) {
    c_sh[j] = 0u;
    b_sh[j] = 0.0;
  }
  __syncthreads();
  const double floor_ = s2max * pow(10.0, -FT_DEC);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double s2 = sig[i] * sig[i];
    if (s2 > floor_) {
      int j = (int)floor(-log10(s2 / s2max) * FT_NB / FT_DEC);
      j = min(max(j, 0), FT_NB - 1);
      atomicAdd(&c_sh[j], 1u);
      atomicAdd(&b_sh[j], bh[i] * bh[i]);
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < FT_NB; j += blockDim.x) {
    if (c_sh[j]) {
      atomicAdd(&cnt[j], (unsigned long long)c_sh[j]);
      atomicAdd(&sb[j], b_sh[j]);
    }
  }
}

__global__ void k_feat_finish(const unsigned long long* __restrict__ cnt, const double* __restrict__ sb, long long n,
                              double s2max, float* __restrict__ f) {
  const int j = threadIdx.x;
  if (j < FT_NB) {
    f[j] = (float)log10((sb[j] + FT_TINY * s2max) / ((double)cnt[j] + 1.0));
    f[FT_NB + j] = (float)log10(((double)cnt[j] + 1.0) / (double)n);
  }
  if (j == 0) {
    double ac = 0.0, ab = 0.0;
    for (int q = FT_NB - 1; q >= 0; --q) {
      ac += (double)cnt[q];
      ab += sb[q];
      if (ac >= (double)n / 8.0) break;
    }
    f[2 * FT_NB] = (float)log10((ab + FT_TINY * s2max) / fmax(ac, 1.0));
    f[2 * FT_NB + 1] = (float)log10(s2max);
  }
}
}  // namespace

extern "C" kp_status kp_lambda_features(kp_ctx* ctx, const void* b, float* features) {
  KP_TRY(kp_check_ready(ctx));
  if (!b || !features) {
    kp_set_error("kp_lambda_features: NULL argument");
    return KP_EINVAL;
  }
  KP_TRY(kp_enter(ctx));
  const double* bh = nullptr;
  void* w = nullptr;
  double dummy = 0.0;
  kp_status s = choose_lambda_impl(ctx, b, KP_LAMBDA_GCV, 0.0, nullptr, &dummy, &bh, &w);
  if (s == KP_OK) {
    cudaStream_t st = ctx->stream;
    const long long N = (long long)ctx->n_r * ctx->n_c;
    const double smax = ctx->lam_sigma_ext[0];
    const double s2max = smax * smax;
    {
      unsigned long long* cnt = (unsigned long long*)w;
      double* sb = (double*)(cnt + FT_NB);
      cudaMemsetAsync(w, 0, FT_NB * (sizeof(unsigned long long) + sizeof(double)), st);
      const int g = std::max(1, std::min((int)((N + 255) / 256), ctx->sm_count * 4));
      k_feat_bins<<<g, 256, 0, st>>>(ctx->Sigma64, bh, N, s2max, cnt, sb);
      k_feat_finish<<<1, 128, 0, st>>>(cnt, sb, N, s2max, features);
      ctx->launches += 2;
      if (cudaGetLastError() != cudaSuccess) {
        kp_set_error("kp_lambda_features: launch failed");
        s = KP_ECUDA;
      }
    }
  }
  kp_status l = kp_leave(ctx);
  return s != KP_OK ? s : l;
}

