// Shared declarations of the vector kernels (kp_vec.cu).
#pragma once
#include "kp_internal.h"

constexpr int VEC_THREADS = 256;

template <typename N>
__device__ __forceinline__ N to_narrow(float v);
template <>
__device__ __forceinline__ __nv_bfloat16 to_narrow<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __half to_narrow<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_fp8_e4m3 to_narrow<__nv_fp8_e4m3>(float v) { return __nv_fp8_e4m3(v); }

// device scalar slots (ctx->dscal) and flag slots (ctx->dflags) of the (F)PCG loop
enum {
  S_RR = 0, S_AMAX = 1, S_PQ = 2, S_ALPHA = 3, S_ZR = 4, S_ZRNEW = 5, S_ZROLD = 6, S_BETA = 7,
  S_RR0 = 8, S_RMAX = 9, S_TOL2 = 10, S_DELTA2 = 11
};
enum { F_PAUSE = 0, F_REASON = 1, F_ITER = 2, F_MAXIT = 3, F_FLEX = 4 };
enum { R_CONV = 1, R_REPLACE = 2, R_MAXIT = 4, R_BREAKDOWN = 8, R_NUMERIC = 16 };

// scalar step run by the last block of a reduction, on its final values:
//   POST_ALPHA  alpha = zr / pq (breakdown / NaN checks)
//   POST_CHECK  iteration count, residual history, convergence / replacement / maxit flags
//   POST_BETA   beta (Fletcher-Reeves or Polak-Ribiere) and zr update
enum { POST_NONE = 0, POST_ALPHA = 1, POST_CHECK = 2, POST_BETA = 3 };
struct PostOp {
  int kind = POST_NONE;
  double* s = nullptr;
  int* f = nullptr;
  double* hist = nullptr;
  int hist_cap = 0;
};

int vec_grid(kp_ctx* ctx, long long n);
kp_status dot2_dev(kp_ctx* ctx, const void* a, const void* b, const void* c, long long n, bool f64, double* out,
                   const int* flags, PostOp post = PostOp());
kp_status norm_amax_dev(kp_ctx* ctx, const void* x, long long n, bool f64, double* out2);
kp_status update_xr_dev(kp_ctx* ctx, void* x, void* r, void* r_old, const void* p, const void* q, long long n,
                        bool f64, const double* alpha_dev, double* out2, const int* flags, PostOp post = PostOp());
kp_status p_update_dev(kp_ctx* ctx, void* p, const void* z, long long n, bool f64, const double* beta_dev,
                       __nv_bfloat16* ps, int slices, long long sstride, const int* flags);
kp_status quantize_dev(kp_ctx* ctx, const void* r, long long n, bool f64, const double* stat, int narrow,
                       double lam2, void* out, float* inv_out, const int* flags, unsigned int* reset = nullptr,
                       int nreset = 0);
kp_status quant8_dev(kp_ctx* ctx, const float* in, long long n, const unsigned int* amax_bits, float* gs, int stage,
                     const float* base, float* inv_out, void* out, const int* flags);
kp_status axpby_dev(kp_ctx* ctx, const void* x, void* y, long long n, bool f64, double alpha, double beta);
kp_status convert_f64_to_f32(kp_ctx* ctx, const double* x, float* y, long long n);
kp_status convert_f32_to_f64(kp_ctx* ctx, const float* x, double* y, long long n);
