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
  S_RR0 = 8, S_RMAX = 9, S_TOL2 = 10, S_DELTA2 = 11,
  S_QPQ = 12, S_QMAX = 13,  // fused iteration: p^T q and max |q| (K application's term sum)
  S_RTPREV = 14             // ||r||^2 of the previous true residual (stagnation test)
};
enum { F_PAUSE = 0, F_REASON = 1, F_ITER = 2, F_MAXIT = 3, F_FLEX = 4, F_STAG = 5, F_SINCE = 6,
       F_SAVED = 7,   // device loop: the reason that triggered a residual replacement
       F_REPL = 8,    // device loop: residual replacements done
       F_NOTDUE = 9,  // batched loop: 1 unless this problem's residual replacement is due (its skip flag)
       F_BLOOP = 10 };  // batched loop: this problem's loop goes on
constexpr int F_GUARD = 15;  // device loop: passes of the loop body
// the multi-term preconditioner's inner PCG keeps its scalars and flags in
// blocks of their own, at these offsets into ctx->dscal / ctx->dflags
constexpr int S_INNER = 64, F_INNER = 16;
constexpr int S_JACOBI = 320;  // setup: the Jacobi thresholds (tol, floor) the sweep kernels read
// a reliable update is also due after this many iterations without one (so a
// recurred residual that stops falling is checked against the true one)
constexpr int REPLACE_EVERY = 50;
enum { R_CONV = 1, R_REPLACE = 2, R_MAXIT = 4, R_BREAKDOWN = 8, R_NUMERIC = 16 };

// scalar step run by the last block of a reduction, on its final values:
//   POST_ALPHA  alpha = zr / pq (breakdown / NaN checks)
//   POST_CHECK  iteration count, residual history, convergence / replacement / maxit flags
//   POST_BETA   beta (Fletcher-Reeves or Polak-Ribiere) and zr update
enum { POST_NONE = 0, POST_ALPHA = 1, POST_CHECK = 2, POST_BETA = 3 };
struct PostOp {
  int kind = POST_NONE;
  // POST_CHECK inside the device-side loop graph: 1 = also set the graph's
  // conditions (residual replacement due; loop continues); 2 = batched loop:
  // write them to F_NOTDUE / F_BLOOP (the loop's own kernels combine the
  // problems' decisions)
  int cond = 0;
  cudaGraphConditionalHandle h_rep = 0, h_loop = 0;
  double* s = nullptr;
  int* f = nullptr;
  double* hist = nullptr;
  int hist_cap = 0;
};

// a K-concatenated GEMM plan (tc_plan_is_kcat) whose epilogue also reduces
// sum(out * aux) as a double-float pair into out2[0] (and max |out| into
// out2[1] when qmax), finished by the last CTA, which runs `post` on them;
// epi must be EPI_F32 with aux
kp_status tc_plan_run_dot(kp_ctx* ctx, TcGemmPlan* plan, const EpiParams& epi, double* out2, double* partials,
                          unsigned int* counter, const PostOp& post, int qmax);

int vec_grid(kp_ctx* ctx, long long n);
kp_status dot2_dev(kp_ctx* ctx, const void* a, const void* b, const void* c, long long n, bool f64, double* out,
                   const int* flags, PostOp post = PostOp());
kp_status norm_amax_dev(kp_ctx* ctx, const void* x, long long n, bool f64, double* out2, const int* flags = nullptr);
kp_status update_xr_dev(kp_ctx* ctx, void* x, void* r, void* r_old, const void* p, const void* q, long long n,
                        bool f64, const double* alpha_dev, double* out2, const int* flags, PostOp post = PostOp());
// The same update, also writing the preconditioner's input narrow(r * s)
// (F16 / BF16), with the power of two s taken from a bound on max |r_new|
// known before the update: max |r| (out2[1], from the previous update) +
// |alpha| max |q| (*qmax_dev).  Writes *inv_out = 1 / (lam2 s).
kp_status update_xr_q_dev(kp_ctx* ctx, void* x, void* r, void* r_old, const void* p, const void* q, long long n,
                          const double* alpha_dev, double* out2, const double* qmax_dev, int narrow, double lam2,
                          void* pc_out, float* inv_out, const int* flags, PostOp post);
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

// ---------------------------------------------------------------- device reductions
// (shared by the vector kernels and the operator's fused term sum)
namespace kpv {

__device__ __forceinline__ bool paused(const int* flags) { return flags != nullptr && *(volatile const int*)flags != 0; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-level reduction of NV sums (+ optional max in slot NV-1 when
// last_is_max) and the cross-block ordered finish.  blockDim.x == VEC_THREADS.
__device__ inline void run_post(const PostOp& po, const double* vals);

// Double-float (hi + lo in FP32) accumulation: FP64 instructions run at a
// small fraction of the FP32 rate on this GPU, so per-element and per-warp
// sums are kept as unevaluated pairs of floats (error-free transformations:
// TwoSum, and the exact FMA residual of each product), ~2^-44 relative, and
// only the per-warp results are converted to FP64.
__device__ __forceinline__ void df_add(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  lo += (hi - (s - bp)) + (x - bp);
  hi = s;
}
__device__ __forceinline__ void df_add_prod(float& hi, float& lo, float a, float b) {
  const float p = a * b;
  lo += fmaf(a, b, -p);
  df_add(hi, lo, p);
}
__device__ __forceinline__ void df_warp_sum(float& hi, float& lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
    float l = lo + ol;
    df_add(hi, l, oh);
    const float t = hi + l;  // renormalise
    lo = l - (t - hi);
    hi = t;
  }
}

// Block-level reduction of NV sums (+ optional max in slot NV-1 when
// last_is_max) and the cross-block ordered finish.  blockDim.x == VEC_THREADS.
// wv: this warp's values (used in lane 0).
template <int NV>
__device__ inline void reduce_tail(const double (&wv)[NV], bool last_is_max, double* partials, unsigned int* counter,
                                   double* out, int nout, const PostOp& po) {
  __shared__ double sh[VEC_THREADS / 32][NV];
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) sh[wid][i] = wv[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 0; i < NV; ++i) {
      const bool mx = last_is_max && i == NV - 1;
      double t = sh[0][i];
      for (int w = 1; w < VEC_THREADS / 32; ++w) t = mx ? fmax(t, sh[w][i]) : t + sh[w][i];
      partials[blockIdx.x * NV + i] = t;
    }
    __threadfence();
    unsigned int prev = atomicAdd(counter, 1u);
    s_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // all of this thread's partials are loaded before any is used (L2 loads,
  // in flight together), then combined in block order
  constexpr int MAXP = 8;
  double pv[MAXP][NV];
#pragma unroll
  for (int u = 0; u < MAXP; ++u) {
    const int b = threadIdx.x + u * VEC_THREADS;
#pragma unroll
    for (int i = 0; i < NV; ++i) pv[u][i] = b < (int)gridDim.x ? __ldcg(partials + b * NV + i) : 0.0;
  }
  double acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    const bool mx = last_is_max && i == NV - 1;
    acc[i] = 0.0;
#pragma unroll
    for (int u = 0; u < MAXP; ++u) acc[i] = mx ? fmax(acc[i], pv[u][i]) : acc[i] + pv[u][i];
  }
  for (int b = threadIdx.x + MAXP * VEC_THREADS; b < (int)gridDim.x; b += VEC_THREADS) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const bool mx = last_is_max && i == NV - 1;
      const double q = __ldcg(partials + b * NV + i);
      acc[i] = mx ? fmax(acc[i], q) : acc[i] + q;
    }
  }
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    const bool mx = last_is_max && i == NV - 1;
    acc[i] = mx ? warp_max(acc[i]) : warp_sum(acc[i]);
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) sh[wid][i] = acc[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double fin[NV];
    for (int i = 0; i < NV; ++i) {
      const bool mx = last_is_max && i == NV - 1;
      double t = sh[0][i];
      for (int w = 1; w < VEC_THREADS / 32; ++w) t = mx ? fmax(t, sh[w][i]) : t + sh[w][i];
      fin[i] = t;
      if (i < nout) out[i] = t;
    }
    *counter = 0u;
    if (po.kind != POST_NONE) run_post(po, fin);
  }
}

template <int NV>
__device__ inline void reduce_finish(double (&v)[NV], bool last_is_max, double* partials, unsigned int* counter,
                                     double* out, int nout, const PostOp& po = PostOp()) {
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    const bool mx = last_is_max && i == NV - 1;
    v[i] = mx ? warp_max(v[i]) : warp_sum(v[i]);
  }
  reduce_tail<NV>(v, last_is_max, partials, counter, out, nout, po);
}

// The same from per-thread double-float sums (a max slot keeps its value in
// hi), kept as float pairs through the block and grid levels; only the final
// values become FP64 (thread 0 of the last block).  partials: 8 bytes per
// value and block, as (hi, lo) float pairs.
template <int NV>
__device__ inline void df_block_sum(float (&hi)[NV], float (&lo)[NV], bool last_is_max) {
  __shared__ float2 shp[VEC_THREADS / 32][NV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    if (last_is_max && i == NV - 1) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) hi[i] = fmaxf(hi[i], __shfl_xor_sync(0xffffffffu, hi[i], o));
      lo[i] = 0.f;
    } else {
      df_warp_sum(hi[i], lo[i]);
    }
    if (lane == 0) shp[wid][i] = make_float2(hi[i], lo[i]);
  }
  __syncthreads();
  if (wid == 0) {  // warp 0 combines the warps' pairs (all lanes take part)
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const float2 t = lane < VEC_THREADS / 32 ? shp[lane][i] : make_float2(0.f, 0.f);
      hi[i] = t.x;
      lo[i] = t.y;
      if (last_is_max && i == NV - 1) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) hi[i] = fmaxf(hi[i], __shfl_xor_sync(0xffffffffu, hi[i], o));
      } else {
        df_warp_sum(hi[i], lo[i]);
      }
    }
  }
}

template <int NV>
__device__ inline void reduce_finish_df(float (&hi)[NV], float (&lo)[NV], bool last_is_max, double* partials,
                                        unsigned int* counter, double* out, int nout, const PostOp& po = PostOp()) {
  __shared__ bool s_last;
  float2* pp = reinterpret_cast<float2*>(partials);
  df_block_sum<NV>(hi, lo, last_is_max);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) pp[blockIdx.x * NV + i] = make_float2(hi[i], lo[i]);
    __threadfence();
    s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    hi[i] = 0.f;
    lo[i] = 0.f;
  }
  for (int b = threadIdx.x; b < (int)gridDim.x; b += VEC_THREADS) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const float2 t = __ldcg(pp + b * NV + i);
      if (last_is_max && i == NV - 1) {
        hi[i] = fmaxf(hi[i], t.x);
      } else {
        lo[i] += t.y;
        df_add(hi[i], lo[i], t.x);
      }
    }
  }
  __syncthreads();  // shared pairs of the first pass are read before they are reused
  df_block_sum<NV>(hi, lo, last_is_max);
  if (threadIdx.x == 0) {
    double fin[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      fin[i] = (double)hi[i] + (double)lo[i];
      if (i < nout) out[i] = fin[i];
    }
    *counter = 0u;
    if (po.kind != POST_NONE) run_post(po, fin);
  }
}

// scalar steps of the iteration (see PostOp); vals = the reduction's results
__device__ inline void run_post(const PostOp& po, const double* vals) {
  double* s = po.s;
  int* f = po.f;
  if (po.kind == POST_ALPHA) {  // vals[0] = p^T K p
    const double pq = vals[0], zr = s[S_ZR];
    if (!isfinite(pq) || !isfinite(zr)) {
      f[F_REASON] |= R_NUMERIC;
      f[F_PAUSE] = 1;
    } else if (!(pq > 0.0) || !(zr > 0.0)) {
      f[F_REASON] |= R_BREAKDOWN;
      f[F_PAUSE] = 1;
    } else {
      s[S_ALPHA] = zr / pq;
    }
  } else if (po.kind == POST_CHECK) {  // vals[0] = ||r||^2
    const int it = ++f[F_ITER];
    const double rr = vals[0];
    if (it < po.hist_cap) po.hist[it] = sqrt(rr / s[S_RR0]);
    int reason = 0;
    if (!isfinite(rr)) reason |= R_NUMERIC;
    else if (rr <= s[S_TOL2]) reason |= R_CONV;
    else if (s[S_DELTA2] > 0.0 && (rr < s[S_DELTA2] * s[S_RMAX] || ++f[F_SINCE] >= REPLACE_EVERY)) reason |= R_REPLACE;
    if (it >= f[F_MAXIT]) reason |= R_MAXIT;
    if (reason) {
      f[F_REASON] |= reason;
      f[F_PAUSE] = 1;
    }
    if (po.cond) {
      // the loop graph's decisions: a reliable update is due (then the
      // replacement's own step decides whether the loop goes on), or the
      // loop stops, or it goes on; the loop also ends a few passes past maxit
      const int rs = f[F_REASON];
      unsigned int repl = 0u, loop = 1u;
      if (f[F_PAUSE]) {
        if (!(rs & (R_NUMERIC | R_BREAKDOWN)) && s[S_DELTA2] > 0.0 && (rs & (R_CONV | R_REPLACE | R_MAXIT))) {
          repl = 1u;
          f[F_SAVED] = rs;
        } else {
          loop = 0u;
        }
      }
      if (++f[F_GUARD] > f[F_MAXIT] + 8) loop = 0u;
      if (po.cond == 1) {
        cudaGraphSetConditional(po.h_rep, repl);
        cudaGraphSetConditional(po.h_loop, loop);
      } else {
        f[F_NOTDUE] = repl ? 0 : 1;
        f[F_BLOOP] = loop;
        if (!loop) f[F_PAUSE] = 1;  // a stopped problem's kernels skip from here on
      }
    }
  } else if (po.kind == POST_BETA) {  // vals[0] = z^T r, vals[1] = z^T r_old
    const double zn = vals[0], zo = vals[1], zr = s[S_ZR];
    if (!isfinite(zn) || !isfinite(zo)) {
      f[F_REASON] |= R_NUMERIC;
      f[F_PAUSE] = 1;
    } else if (!(zn > 0.0)) {
      f[F_REASON] |= R_BREAKDOWN;
      f[F_PAUSE] = 1;
    } else {
      s[S_BETA] = f[F_FLEX] ? (zn - zo) / zr : zn / zr;
      s[S_ZR] = zn;
    }
  }
}

}  // namespace kpv
