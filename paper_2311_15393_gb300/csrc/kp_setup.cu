// kp_setup: PSF -> Kronecker-sum operator and KP-SVD preconditioner, on the GPU.
//
//  1. weighted PSF W = D_c P D_r, D = diag(sqrt(w)), w[k] = n - |k - c|: the
//     number of times PSF row / column k occurs in a Toeplitz factor, so that
//     the leading SVD term is the Frobenius-optimal Kronecker product
//     (Section 5, the argmin below eq. KronSumDecomp);
//  2. SVD of W in FP64: subspace iteration for the leading `rank` terms when
//     rank <= min(n_r, n_c) / 4, else the full one-sided Jacobi SVD; terms
//     u_m = sqrt(s_m) D_c^-1 u~_m, v_m = sqrt(s_m) D_r^-1 v~_m, m < rank, with the
//     largest-magnitude entry of u_m made positive;
//  3. factors A_c^(m) = F(u_m), A_r^(m) = F(v_m) with F(u) = T(u) (zero BC) or
//     T(u) + H(u) (reflexive BC), T(u)[i,j] = u[c+i-j],
//     H(u)[i,j] = u[c+i+j+1] + u[c+i+j+1-2n] (eq. KronSumDecomp);
//  4. SVDs of A_r^(1), A_c^(1) (eq. AKronSVD) by one-sided Jacobi (FP64),
//     preconditioned by the DCT-II / DST-I (see kp_jacobi.cu);
//  5. KP spectrum Sigma = sigma_c sigma_r^T (PRODUCT) or
//     sum_k diag(U_c^T A_c^(k) V_c) diag(U_r^T A_r^(k) V_r)^T (PROJECTED);
//  6. copies of the factors in the operator precision (FP64, FP32 or bf16
//     slices) in the four GEMM layouts, of V_c, V_r in the preconditioner
//     precision, and the tensor-core GEMM plans.
#include <algorithm>
#include <cmath>

#include "kp_internal.h"
#include "kp_ops.h"
#include "kp_vec.cuh"

namespace {

__global__ void k_weight_psf(const double* __restrict__ P, int n_r, int n_c, int c_r, int c_c, double* __restrict__ W) {
  long long tot = (long long)n_r * n_c;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % n_r), j = (int)(t / n_r);
    double wc = (double)(n_r - abs(i - c_r)), wr = (double)(n_c - abs(j - c_c));
    W[t] = sqrt(wc) * P[t] * sqrt(wr);
  }
}

__global__ void k_transpose64(const double* __restrict__ A, int rows, int cols, double* __restrict__ B) {
  // A col-major rows x cols -> B col-major cols x rows
  long long tot = (long long)rows * cols;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % rows), j = (int)(t / rows);
    B[j + (long long)cols * i] = A[t];
  }
}

// term m: u = sqrt(s) Uw[:, m] / sqrt(w_c), v = sqrt(s) Vw[:, m] / sqrt(w_r); sign so
// that u's largest-|.| entry (first on ties) is positive.  One block per term.
__global__ void k_terms(const double* __restrict__ Uw, const double* __restrict__ sw, const double* __restrict__ Vw,
                        int n_r, int n_c, int c_r, int c_c, double* __restrict__ u, double* __restrict__ v,
                        double* __restrict__ s_out) {
  const int m = blockIdx.x;
  const double s = sw[m];
  const double rs = sqrt(fmax(s, 0.0));
  __shared__ double bv[256];
  __shared__ int bi[256];
  double best = -1.0;
  int besti = 0x7fffffff;
  for (int i = threadIdx.x; i < n_r; i += blockDim.x) {
    double val = rs * Uw[(long long)m * n_r + i] / sqrt((double)(n_r - abs(i - c_r)));
    u[(long long)m * n_r + i] = val;
    double a = fabs(val);
    if (a > best || (a == best && i < besti)) {
      best = a;
      besti = i;
    }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = besti;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      double a = bv[threadIdx.x + o];
      int ai = bi[threadIdx.x + o];
      if (a > bv[threadIdx.x] || (a == bv[threadIdx.x] && ai < bi[threadIdx.x])) {
        bv[threadIdx.x] = a;
        bi[threadIdx.x] = ai;
      }
    }
    __syncthreads();
  }
  const double sign = u[(long long)m * n_r + bi[0]] < 0 ? -1.0 : 1.0;
  __syncthreads();
  for (int i = threadIdx.x; i < n_r; i += blockDim.x) u[(long long)m * n_r + i] *= sign;
  for (int j = threadIdx.x; j < n_c; j += blockDim.x)
    v[(long long)m * n_c + j] = sign * rs * Vw[(long long)m * n_c + j] / sqrt((double)(n_c - abs(j - c_c)));
  if (threadIdx.x == 0) s_out[m] = s;
}

__device__ __forceinline__ double take(const double* u, int n, int k) { return (k >= 0 && k < n) ? u[k] : 0.0; }

// F[k][i][j] row-major, F = T(u_k) (+ H(u_k) for reflexive BC)
__global__ void k_build_factor(const double* __restrict__ u, int n, int c, int rank, int reflexive,
                               double* __restrict__ F) {
  long long tot = (long long)rank * n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    int j = (int)(t % n);
    int i = (int)((t / n) % n);
    int k = (int)(t / ((long long)n * n));
    const double* uk = u + (long long)k * n;
    double val = take(uk, n, c + i - j);
    if (reflexive) val += take(uk, n, c + i + j + 1) + take(uk, n, c + i + j + 1 - 2 * n);
    F[t] = val;
  }
}

// out[k][a][b] = in[k][b][a] (square n x n blocks), with conversion
template <typename O>
__global__ void k_transpose_blocks(const double* __restrict__ in, int n, int blocks, O* __restrict__ out) {
  long long tot = (long long)blocks * n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    int b = (int)(t % n);
    int a = (int)((t / n) % n);
    long long k = t / ((long long)n * n);
    out[t] = (O)in[k * n * n + (long long)b * n + a];
  }
}

template <typename O>
__global__ void k_cast(const double* __restrict__ in, long long n, O* __restrict__ out, double scale) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    out[t] = (O)(in[t] * scale);
}

// bf16 slices of FP64 data, optionally transposed per square block:
// out[s][t] = slice s of (transpose ? in[k][b][a] : in[t])
__global__ void k_split64(const double* __restrict__ in, int n, int blocks, int transpose, int slices,
                          long long sstride, __nv_bfloat16* __restrict__ out) {
  long long tot = (long long)blocks * n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    double v;
    if (transpose) {
      int b = (int)(t % n);
      int a = (int)((t / n) % n);
      long long k = t / ((long long)n * n);
      v = in[k * n * n + (long long)b * n + a];
    } else {
      v = in[t];
    }
    // slices of the FP32-rounded value, split in FP32 (exact: three bf16
    // slices hold the 24-bit significand; FP64 arithmetic is slow here)
    float f = (float)v;
    for (int s = 0; s < slices; ++s) {
      const __nv_bfloat16 h = __float2bfloat16_rn(f);
      out[s * sstride + t] = h;
      f -= __bfloat162float(h);
    }
  }
}

// narrow copy of FP64 data (optionally transposed square matrix), scaled
template <typename O>
__global__ void k_narrow64(const double* __restrict__ in, int n, int transpose, double scale, O* __restrict__ out) {
  long long tot = (long long)n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    int b = (int)(t % n), a = (int)(t / n);
    double v = transpose ? in[(long long)b * n + a] : in[t];
    out[t] = to_narrow<O>((float)(v * scale));
  }
}

// d[i] = sum_a U[a + n i] * T[a * n + i]   (U col-major, T row-major)
template <typename T_>
__global__ void k_coldot(const T_* __restrict__ U, const T_* __restrict__ T, int n, double* __restrict__ d) {
  const int i = blockIdx.x;
  double acc = 0.0;
  for (int a = threadIdx.x; a < n; a += blockDim.x)
    acc = fma((double)U[(long long)i * n + a], (double)T[(long long)a * n + i], acc);
  __shared__ double sh[256];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) d[i] = sh[0];
}

// Sigma[i + n_r j] = sum_k dc[k][i] dr[k][j]
__global__ void k_sigma(const double* __restrict__ dc, const double* __restrict__ dr, int n_r, int n_c, int rank,
                        double* __restrict__ S) {
  long long tot = (long long)n_r * n_c;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    int i = (int)(t % n_r), j = (int)(t / n_r);
    double acc = 0.0;
    for (int k = 0; k < rank; ++k) acc += dc[(long long)k * n_r + i] * dr[(long long)k * n_c + j];
    S[t] = acc;
  }
}

__global__ void k_amax64(const double* __restrict__ x, long long n, double* out) {
  double m = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(x[t]));
  __shared__ double sh[256];
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0];
}

}  // namespace

static int grid_for(kp_ctx* ctx, long long n) {
  long long b = (n + 255) / 256;
  long long cap = (long long)ctx->sm_count * 16;
  return (int)std::max(1LL, std::min(b, cap));
}

static bool is_tc(kp_prec p) { return p == KP_BF16 || p == KP_BF16X3 || p == KP_F16 || p == KP_E4M3; }

// projected spectrum factor: d[k][i] = diag(U^T F^(k) V)_i for square n; for
// k = 0 (the factor the SVD is of) that diagonal is the singular values.
// The terms k >= 1 are one stacked product [F^(1); ...; F^(rank-1)] V, in
// FP32 (U32, V32 given) or FP64.
static kp_status projected_diag(kp_ctx* ctx, const double* F, const double* U, const double* V, const float* U32,
                                const float* V32, const double* s, int n, int rank, double* d, void* tmp,
                                float* F32) {
  KP_CUDA(cudaMemcpyAsync(d, s, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  if (rank < 2) return KP_OK;
  const long long blk = (long long)n * n;
  GemmDesc g;
  g.M = (rank - 1) * n;
  g.N = n;
  g.K = n;
  g.A.ld = n;
  g.B.ld = n;  // B[i][b] = V[b, i] (col-major V)
  g.epi.mode = EPI_T;
  g.epi.out = tmp;
  g.epi.ldd = n;
  if (U32 && ctx->setup_tc) {  // tensor cores: FP32-level (3 slices) or half precision (1)
    KP_TRY(tc_product(ctx, F + blk, true, (rank - 1) * n, V, true, n, n, (float*)tmp, ctx->setup_half ? 1 : 3));
  } else if (U32) {
    KP_TRY(convert_f64_to_f32(ctx, F + blk, F32, (rank - 1) * blk));
    g.A.ptr = F32;
    g.B.ptr = V32;
    KP_TRY(simt_gemm<float>(ctx, g));
  } else {
    g.A.ptr = F + blk;
    g.B.ptr = V;
    KP_TRY(simt_gemm<double>(ctx, g));
  }
  for (int k = 1; k < rank; ++k) {
    if (U32)
      k_coldot<float><<<n, 256, 0, ctx->stream>>>(U32, (const float*)tmp + (k - 1) * blk, n, d + (long long)k * n);
    else
      k_coldot<double><<<n, 256, 0, ctx->stream>>>(U, (const double*)tmp + (k - 1) * blk, n, d + (long long)k * n);
    KP_LAUNCHED(ctx);
  }
  KP_CUDA(cudaGetLastError());
  return KP_OK;
}

extern "C" kp_status kp_setup(kp_ctx* ctx, const double* psf, int n_r, int n_c, int center_r, int center_c, kp_bc bc,
                              int op_rank, int pc_rank, kp_prec op_prec, kp_prec pc_prec, kp_prec vec_prec,
                              kp_sigma sigma) {
  if (!ctx) {
    kp_set_error("kp_setup: NULL context");
    return KP_EINVAL;
  }
  if (!psf || n_r < 2 || n_c < 2 || center_r < 0 || center_r >= n_r || center_c < 0 || center_c >= n_c) {
    kp_set_error("kp_setup: bad PSF, size or centre (n_r=%d n_c=%d c=(%d,%d))", n_r, n_c, center_r, center_c);
    return KP_EINVAL;
  }
  if (((uintptr_t)psf & 15) != 0) {
    kp_set_error("kp_setup: psf must be 16-byte aligned");
    return KP_EINVAL;
  }
  if (bc != KP_BC_ZERO && bc != KP_BC_REFLEXIVE) {
    kp_set_error("kp_setup: unknown boundary condition %d", (int)bc);
    return KP_EINVAL;
  }
  if (sigma != KP_SIGMA_PRODUCT && sigma != KP_SIGMA_PROJECTED) {
    kp_set_error("kp_setup: unknown sigma mode %d", (int)sigma);
    return KP_EINVAL;
  }
  const int rmax = std::min(n_r, n_c);
  if (op_rank < 0 || op_rank > rmax) {
    kp_set_error("kp_setup: op_rank %d outside [0, %d]", op_rank, rmax);
    return KP_EINVAL;
  }
  const int rank = op_rank == 0 ? rmax : op_rank;
  if (pc_rank < 1 || pc_rank > rank) {
    kp_set_error("kp_setup: pc_rank %d outside [1, %d] (the operator's terms)", pc_rank, rank);
    return KP_EINVAL;
  }
  // supported precision combinations
  bool okc = false;
  if (op_prec == KP_F64 && pc_prec == KP_F64 && vec_prec == KP_F64) okc = true;
  if (op_prec == KP_F32 && vec_prec == KP_F32 &&
      (pc_prec == KP_F32 || pc_prec == KP_BF16 || pc_prec == KP_F16 || pc_prec == KP_E4M3))
    okc = true;
  if ((op_prec == KP_BF16 || op_prec == KP_BF16X3) && vec_prec == KP_F32 &&
      (pc_prec == KP_F32 || pc_prec == KP_BF16 || pc_prec == KP_F16 || pc_prec == KP_E4M3))
    okc = true;
  if (!okc) {
    kp_set_error("kp_setup: unsupported precision combination op=%d pc=%d vec=%d", (int)op_prec, (int)pc_prec,
                 (int)vec_prec);
    return KP_EINVAL;
  }
  if ((is_tc(op_prec) || is_tc(pc_prec))) {
    if (!tc_device_supported(ctx)) {
      kp_set_error("kp_setup: tensor-core precisions need an sm_103 device");
      return KP_ENOTSUP;
    }
    if (n_r % 16 || n_c % 16) {
      kp_set_error("kp_setup: tensor-core precisions need n_r, n_c multiples of 16");
      return KP_ENOTSUP;
    }
  }
  KP_CUDA(cudaSetDevice(ctx->device));
  KP_TRY(kp_enter(ctx));
  for (auto& e : ctx->ev_setup)
    if (!e) KP_CUDA(cudaEventCreate(&e));
  KP_CUDA(cudaEventRecord(ctx->ev_setup[0], ctx->stream));
  kp_free_all(ctx);
  ctx->n_r = n_r;
  ctx->n_c = n_c;
  ctx->c_r = center_r;
  ctx->c_c = center_c;
  ctx->rank = rank;
  ctx->pc_rank = pc_rank;
  ctx->bc = bc;
  ctx->op_prec = op_prec;
  ctx->op_prec_setup = op_prec;
  ctx->sigma_max = -1.0;
  ctx->pc_prec = pc_prec;
  ctx->vec_prec = vec_prec;
  ctx->sigma_mode = sigma;
  ctx->setup_fp32 = vec_prec == KP_F32 && !ctx->force_setup_fp64;
  ctx->setup_tc = ctx->setup_fp32 && n_r % 16 == 0 && n_c % 16 == 0 && tc_device_supported(ctx);
  ctx->setup_half = ctx->setup_tc && ctx->force_setup_half;
  KP_CUDA(cudaMemsetAsync(ctx->dev_status, 0, sizeof(int), ctx->stream));

  cudaStream_t st = ctx->stream;
  const long long N = (long long)n_r * n_c;
  const int reflexive = bc == KP_BC_REFLEXIVE ? 1 : 0;

  // ---- 1-2: weighted PSF SVD and terms
  double *W, *Uw, *sw, *Vw;
  const int mm = std::max(n_r, n_c), nn = std::min(n_r, n_c);
  KP_TRY(kp_alloc(ctx, (void**)&W, sizeof(double) * N));
  KP_TRY(kp_alloc(ctx, (void**)&Uw, sizeof(double) * (size_t)mm * nn));
  KP_TRY(kp_alloc(ctx, (void**)&sw, sizeof(double) * nn));
  KP_TRY(kp_alloc(ctx, (void**)&Vw, sizeof(double) * (size_t)nn * nn));
  k_weight_psf<<<grid_for(ctx, N), 256, 0, st>>>(psf, n_r, n_c, center_r, center_c, W);
  KP_LAUNCHED(ctx);
  {  // the weighted PSF is finite and nonzero exactly when the PSF is
    double h[2];
    KP_TRY(norm_amax_dev(ctx, W, N, true, ctx->dscal + S_RR));
    KP_CUDA(cudaMemcpyAsync(h, ctx->dscal + S_RR, sizeof(h), cudaMemcpyDeviceToHost, st));
    KP_CUDA(kp_wait(ctx, st));
    if (!std::isfinite(h[0]) || !std::isfinite(h[1])) {
      kp_set_error("kp_setup: the PSF holds a NaN or Inf");
      return KP_ENUMERIC;
    }
    if (!(h[1] > 0.0)) {
      kp_set_error("kp_setup: the PSF is zero");
      return KP_EINVAL;
    }
  }
  double *Uc_w, *Vc_w;  // left (n_r) and right (n_c) singular vectors of W
  const double* Wsrc = W;
  if (n_r < n_c) {  // work on W^T (m >= n)
    double* WT;
    KP_TRY(kp_alloc(ctx, (void**)&WT, sizeof(double) * N));
    k_transpose64<<<grid_for(ctx, N), 256, 0, st>>>(W, n_r, n_c, WT);
    KP_LAUNCHED(ctx);
    Wsrc = WT;
  }
  // few terms: subspace iteration for the leading ones; otherwise the full
  // one-sided Jacobi SVD
  if (4 * rank <= nn && rank + 8 <= 32) {  // few leading terms: subspace iteration (p = rank + 8 <= 32)
    KP_TRY(topr_svd(ctx, Wsrc, mm, nn, rank, Uw, sw, Vw, nullptr));
  } else {
    KP_TRY(jacobi_svd(ctx, Wsrc, mm, nn, Uw, sw, Vw, nullptr));
  }
  if (n_r >= n_c) {
    Uc_w = Uw;
    Vc_w = Vw;
  } else {  // W^T = Uw S Vw^T
    Uc_w = Vw;
    Vc_w = Uw;
  }
  KP_TRY(kp_alloc(ctx, (void**)&ctx->s_terms, sizeof(double) * rank));
  KP_TRY(kp_alloc(ctx, (void**)&ctx->u_terms, sizeof(double) * (size_t)n_r * rank));
  KP_TRY(kp_alloc(ctx, (void**)&ctx->v_terms, sizeof(double) * (size_t)n_c * rank));
  k_terms<<<rank, 256, 0, st>>>(Uc_w, sw, Vc_w, n_r, n_c, center_r, center_c, ctx->u_terms, ctx->v_terms,
                                ctx->s_terms);
  KP_LAUNCHED(ctx);

  // ---- 3: factors (row-major per term)
  KP_TRY(kp_alloc(ctx, (void**)&ctx->Ac64, sizeof(double) * (size_t)rank * n_r * n_r));
  KP_TRY(kp_alloc(ctx, (void**)&ctx->Ar64, sizeof(double) * (size_t)rank * n_c * n_c));
  k_build_factor<<<grid_for(ctx, (long long)rank * n_r * n_r), 256, 0, st>>>(ctx->u_terms, n_r, center_r, rank,
                                                                             reflexive, ctx->Ac64);
  k_build_factor<<<grid_for(ctx, (long long)rank * n_c * n_c), 256, 0, st>>>(ctx->v_terms, n_c, center_c, rank,
                                                                             reflexive, ctx->Ar64);
  ctx->launches += 2;

  // ---- 4: factor SVDs (eq. AKronSVD): A_r^(1) = U_r S_r V_r^T, A_c^(1) = U_c S_c V_c^T
  KP_TRY(kp_alloc(ctx, (void**)&ctx->Ur, sizeof(double) * (size_t)n_c * n_c));
  KP_TRY(kp_alloc(ctx, (void**)&ctx->Vr, sizeof(double) * (size_t)n_c * n_c));
  KP_TRY(kp_alloc(ctx, (void**)&ctx->sr, sizeof(double) * n_c));
  KP_TRY(kp_alloc(ctx, (void**)&ctx->Uc, sizeof(double) * (size_t)n_r * n_r));
  KP_TRY(kp_alloc(ctx, (void**)&ctx->Vc, sizeof(double) * (size_t)n_r * n_r));
  KP_TRY(kp_alloc(ctx, (void**)&ctx->sc, sizeof(double) * n_r));
  const int transform = reflexive ? 0 : 1;
  KP_TRY(factor_svd(ctx, ctx->Ar64, n_c, transform, ctx->Ur, ctx->sr, ctx->Vr, nullptr));
  KP_TRY(factor_svd(ctx, ctx->Ac64, n_r, transform, ctx->Uc, ctx->sc, ctx->Vc, nullptr));
  if (ctx->setup_fp32) {
    KP_TRY(kp_alloc(ctx, (void**)&ctx->Uc32, sizeof(float) * (size_t)n_r * n_r));
    KP_TRY(kp_alloc(ctx, (void**)&ctx->Vc32, sizeof(float) * (size_t)n_r * n_r));
    KP_TRY(kp_alloc(ctx, (void**)&ctx->Ur32, sizeof(float) * (size_t)n_c * n_c));
    KP_TRY(kp_alloc(ctx, (void**)&ctx->Vr32, sizeof(float) * (size_t)n_c * n_c));
    KP_TRY(convert_f64_to_f32(ctx, ctx->Uc, ctx->Uc32, (long long)n_r * n_r));
    KP_TRY(convert_f64_to_f32(ctx, ctx->Vc, ctx->Vc32, (long long)n_r * n_r));
    KP_TRY(convert_f64_to_f32(ctx, ctx->Ur, ctx->Ur32, (long long)n_c * n_c));
    KP_TRY(convert_f64_to_f32(ctx, ctx->Vr, ctx->Vr32, (long long)n_c * n_c));
  }

  // ---- 5: KP spectrum
  KP_TRY(kp_alloc(ctx, (void**)&ctx->Sigma64, sizeof(double) * N));
  KP_TRY(kp_alloc(ctx, (void**)&ctx->Sigma32, sizeof(float) * N));
  {
    double *dc, *dr;
    void* tmp = nullptr;
    float* F32 = nullptr;
    const int nmax = std::max(n_r, n_c);
    const int rk = sigma == KP_SIGMA_PROJECTED ? rank : 1;
    KP_TRY(kp_alloc(ctx, (void**)&dc, sizeof(double) * (size_t)rk * n_r));
    KP_TRY(kp_alloc(ctx, (void**)&dr, sizeof(double) * (size_t)rk * n_c));
    if (sigma == KP_SIGMA_PROJECTED) {
      const size_t stack = (size_t)std::max(rank - 1, 1) * nmax * nmax;
      if (ctx->setup_fp32) {
        KP_TRY(kp_alloc(ctx, &tmp, sizeof(float) * stack));
        KP_TRY(kp_alloc(ctx, (void**)&F32, sizeof(float) * stack));
      } else {
        KP_TRY(kp_alloc(ctx, &tmp, sizeof(double) * stack));
      }
      KP_TRY(projected_diag(ctx, ctx->Ac64, ctx->Uc, ctx->Vc, ctx->Uc32, ctx->Vc32, ctx->sc, n_r, rank, dc, tmp, F32));
      KP_TRY(projected_diag(ctx, ctx->Ar64, ctx->Ur, ctx->Vr, ctx->Ur32, ctx->Vr32, ctx->sr, n_c, rank, dr, tmp, F32));
    } else {
      KP_CUDA(cudaMemcpyAsync(dc, ctx->sc, sizeof(double) * n_r, cudaMemcpyDeviceToDevice, st));
      KP_CUDA(cudaMemcpyAsync(dr, ctx->sr, sizeof(double) * n_c, cudaMemcpyDeviceToDevice, st));
    }
    k_sigma<<<grid_for(ctx, N), 256, 0, st>>>(dc, dr, n_r, n_c, rk, ctx->Sigma64);
    KP_LAUNCHED(ctx);
    KP_TRY(convert_f64_to_f32(ctx, ctx->Sigma64, ctx->Sigma32, N));
  }

  // ---- 6: operator copies
  const long long blk_c = (long long)rank * n_r * n_r, blk_r = (long long)rank * n_c * n_c;
  if (op_prec == KP_F64) {
    ctx->op_slices = 1;
    ctx->opAc = ctx->Ac64;
    ctx->opAr = ctx->Ar64;
    KP_TRY(kp_alloc(ctx, &ctx->opAcT, sizeof(double) * blk_c));
    KP_TRY(kp_alloc(ctx, &ctx->opArT, sizeof(double) * blk_r));
    k_transpose_blocks<double><<<grid_for(ctx, blk_c), 256, 0, st>>>(ctx->Ac64, n_r, rank, (double*)ctx->opAcT);
    k_transpose_blocks<double><<<grid_for(ctx, blk_r), 256, 0, st>>>(ctx->Ar64, n_c, rank, (double*)ctx->opArT);
    ctx->launches += 2;
  } else if (op_prec == KP_F32) {
    ctx->op_slices = 1;
    KP_TRY(kp_alloc(ctx, &ctx->opAc, sizeof(float) * blk_c));
    KP_TRY(kp_alloc(ctx, &ctx->opAr, sizeof(float) * blk_r));
    KP_TRY(kp_alloc(ctx, &ctx->opAcT, sizeof(float) * blk_c));
    KP_TRY(kp_alloc(ctx, &ctx->opArT, sizeof(float) * blk_r));
    k_cast<float><<<grid_for(ctx, blk_c), 256, 0, st>>>(ctx->Ac64, blk_c, (float*)ctx->opAc, 1.0);
    k_cast<float><<<grid_for(ctx, blk_r), 256, 0, st>>>(ctx->Ar64, blk_r, (float*)ctx->opAr, 1.0);
    k_transpose_blocks<float><<<grid_for(ctx, blk_c), 256, 0, st>>>(ctx->Ac64, n_r, rank, (float*)ctx->opAcT);
    k_transpose_blocks<float><<<grid_for(ctx, blk_r), 256, 0, st>>>(ctx->Ar64, n_c, rank, (float*)ctx->opArT);
    ctx->launches += 4;
  } else {
    ctx->op_slices = 3;
    const size_t bc_ = sizeof(__nv_bfloat16) * 3;
    KP_TRY(kp_alloc(ctx, &ctx->opAc, bc_ * blk_c));
    KP_TRY(kp_alloc(ctx, &ctx->opAr, bc_ * blk_r));
    KP_TRY(kp_alloc(ctx, &ctx->opAcT, bc_ * blk_c));
    KP_TRY(kp_alloc(ctx, &ctx->opArT, bc_ * blk_r));
    k_split64<<<grid_for(ctx, blk_c), 256, 0, st>>>(ctx->Ac64, n_r, rank, 0, 3, blk_c, (__nv_bfloat16*)ctx->opAc);
    k_split64<<<grid_for(ctx, blk_r), 256, 0, st>>>(ctx->Ar64, n_c, rank, 0, 3, blk_r, (__nv_bfloat16*)ctx->opAr);
    k_split64<<<grid_for(ctx, blk_c), 256, 0, st>>>(ctx->Ac64, n_r, rank, 1, 3, blk_c, (__nv_bfloat16*)ctx->opAcT);
    k_split64<<<grid_for(ctx, blk_r), 256, 0, st>>>(ctx->Ar64, n_c, rank, 1, 3, blk_r, (__nv_bfloat16*)ctx->opArT);
    ctx->launches += 4;
  }

  // ---- preconditioner copies: row-major V_c^T (= col-major V_c), V_r^T, V_c, V_r
  const long long nc2 = (long long)n_r * n_r, nr2 = (long long)n_c * n_c;
  if (pc_prec == KP_F64) {
    ctx->pcVcT = ctx->Vc;
    ctx->pcVrT = ctx->Vr;
    KP_TRY(kp_alloc(ctx, &ctx->pcVc, sizeof(double) * nc2));
    KP_TRY(kp_alloc(ctx, &ctx->pcVr, sizeof(double) * nr2));
    k_transpose_blocks<double><<<grid_for(ctx, nc2), 256, 0, st>>>(ctx->Vc, n_r, 1, (double*)ctx->pcVc);
    k_transpose_blocks<double><<<grid_for(ctx, nr2), 256, 0, st>>>(ctx->Vr, n_c, 1, (double*)ctx->pcVr);
    ctx->launches += 2;
  } else if (pc_prec == KP_F32) {
    KP_TRY(kp_alloc(ctx, &ctx->pcVcT, sizeof(float) * nc2));
    KP_TRY(kp_alloc(ctx, &ctx->pcVrT, sizeof(float) * nr2));
    KP_TRY(kp_alloc(ctx, &ctx->pcVc, sizeof(float) * nc2));
    KP_TRY(kp_alloc(ctx, &ctx->pcVr, sizeof(float) * nr2));
    k_cast<float><<<grid_for(ctx, nc2), 256, 0, st>>>(ctx->Vc, nc2, (float*)ctx->pcVcT, 1.0);
    k_cast<float><<<grid_for(ctx, nr2), 256, 0, st>>>(ctx->Vr, nr2, (float*)ctx->pcVrT, 1.0);
    k_transpose_blocks<float><<<grid_for(ctx, nc2), 256, 0, st>>>(ctx->Vc, n_r, 1, (float*)ctx->pcVc);
    k_transpose_blocks<float><<<grid_for(ctx, nr2), 256, 0, st>>>(ctx->Vr, n_c, 1, (float*)ctx->pcVr);
    ctx->launches += 4;
  } else {
    const size_t es = pc_prec == KP_E4M3 ? 1 : (pc_prec == KP_BF16 ? 4 : 2);  // BF16: two slices
    KP_TRY(kp_alloc(ctx, &ctx->pcVcT, es * nc2));
    KP_TRY(kp_alloc(ctx, &ctx->pcVrT, es * nr2));
    KP_TRY(kp_alloc(ctx, &ctx->pcVc, es * nc2));
    KP_TRY(kp_alloc(ctx, &ctx->pcVr, es * nr2));
    double sc_c = 1.0, sc_r = 1.0;
    if (pc_prec == KP_E4M3) {
      // power-of-two per-factor scale putting max|V| into [224, 448)
      double* am;
      KP_TRY(kp_alloc(ctx, (void**)&am, 2 * sizeof(double)));
      k_amax64<<<1, 256, 0, st>>>(ctx->Vc, nc2, am);
      k_amax64<<<1, 256, 0, st>>>(ctx->Vr, nr2, am + 1);
      ctx->launches += 2;
      double h[2];
      KP_CUDA(cudaMemcpyAsync(h, am, sizeof(h), cudaMemcpyDeviceToHost, st));
      KP_CUDA(kp_wait(ctx, st));
      int e;
      std::frexp(448.0 / h[0], &e);
      sc_c = std::ldexp(1.0, e - 1);
      std::frexp(448.0 / h[1], &e);
      sc_r = std::ldexp(1.0, e - 1);
    }
    ctx->pc_vscale_c = (float)sc_c;
    ctx->pc_vscale_r = (float)sc_r;
    if (pc_prec == KP_BF16) {
      // bf16 factors as a hi + lo pair (slices at stride n^2): their 8-bit
      // mantissa alone would cost ~4e-3 relative per apply
      k_split64<<<grid_for(ctx, nc2), 256, 0, st>>>(ctx->Vc, n_r, 1, 0, 2, nc2, (__nv_bfloat16*)ctx->pcVcT);
      k_split64<<<grid_for(ctx, nr2), 256, 0, st>>>(ctx->Vr, n_c, 1, 0, 2, nr2, (__nv_bfloat16*)ctx->pcVrT);
      k_split64<<<grid_for(ctx, nc2), 256, 0, st>>>(ctx->Vc, n_r, 1, 1, 2, nc2, (__nv_bfloat16*)ctx->pcVc);
      k_split64<<<grid_for(ctx, nr2), 256, 0, st>>>(ctx->Vr, n_c, 1, 1, 2, nr2, (__nv_bfloat16*)ctx->pcVr);
    } else if (pc_prec == KP_F16) {
      k_narrow64<__half><<<grid_for(ctx, nc2), 256, 0, st>>>(ctx->Vc, n_r, 0, 1.0, (__half*)ctx->pcVcT);
      k_narrow64<__half><<<grid_for(ctx, nr2), 256, 0, st>>>(ctx->Vr, n_c, 0, 1.0, (__half*)ctx->pcVrT);
      k_narrow64<__half><<<grid_for(ctx, nc2), 256, 0, st>>>(ctx->Vc, n_r, 1, 1.0, (__half*)ctx->pcVc);
      k_narrow64<__half><<<grid_for(ctx, nr2), 256, 0, st>>>(ctx->Vr, n_c, 1, 1.0, (__half*)ctx->pcVr);
    } else {
      k_narrow64<__nv_fp8_e4m3><<<grid_for(ctx, nc2), 256, 0, st>>>(ctx->Vc, n_r, 0, sc_c, (__nv_fp8_e4m3*)ctx->pcVcT);
      k_narrow64<__nv_fp8_e4m3><<<grid_for(ctx, nr2), 256, 0, st>>>(ctx->Vr, n_c, 0, sc_r, (__nv_fp8_e4m3*)ctx->pcVrT);
      k_narrow64<__nv_fp8_e4m3><<<grid_for(ctx, nc2), 256, 0, st>>>(ctx->Vc, n_r, 1, sc_c, (__nv_fp8_e4m3*)ctx->pcVc);
      k_narrow64<__nv_fp8_e4m3><<<grid_for(ctx, nr2), 256, 0, st>>>(ctx->Vr, n_c, 1, sc_r, (__nv_fp8_e4m3*)ctx->pcVr);
    }
    ctx->launches += 4;
  }
  KP_CUDA(cudaGetLastError());

  // ---- workspaces and GEMM plans
  KP_TRY(ops_prepare(ctx));
  KP_CUDA(cudaEventRecord(ctx->ev_setup[1], st));
  KP_CUDA(kp_wait(ctx, st));
  KP_TRY(read_status(ctx));
  {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev_setup[0], ctx->ev_setup[1]);
    ctx->last_setup_ms = ms;
  }
  ctx->ready = true;
  return kp_leave(ctx);
}
