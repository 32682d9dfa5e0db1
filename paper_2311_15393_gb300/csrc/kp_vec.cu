// Vector kernels of the (F)PCG loop and helper reductions.
//
// Every inner product and norm is accumulated as a tree: per-thread partial
// sums, warp shuffles, a block reduction, per-block partials, and a final
// ordered reduction by the last block to finish, in FP64 from the warp level
// up.  The result does not depend on block scheduling.  This is the GPU form
// of the pairwise summation the paper uses to limit rounding-error growth in
// inner products (Section 4).  FP32 vectors are processed in FP32 (16-byte
// loads; per-thread partial sums over at most 64 elements before they are
// added into FP64): FP64 arithmetic runs at a small fraction of the FP32 rate
// on this GPU and would bound these memory-bound kernels.  The last block of
// a reduction can run the scalar step of the iteration (alpha, the
// convergence test, beta) on the final values, saving a launch.
#include <type_traits>

#include "kp_group.cuh"
#include "kp_vec.cuh"

namespace kpv {

// 16-byte access to element 4 i of an FP32 vector
__device__ __forceinline__ float4 ld4(const float* p, long long i) { return reinterpret_cast<const float4*>(p)[i]; }
__device__ __forceinline__ void st4(float* p, long long i, float4 v) { reinterpret_cast<float4*>(p)[i] = v; }
constexpr int FLUSH = 16;  // float4 packets per thread between FP64 flushes


// ------------------------------------------------------------- dot products
// out[0] = a.b ; if c != null, out[1] = a.c
template <typename T>
__device__ __forceinline__ void k_dot2_body(const T* __restrict__ a, const T* __restrict__ b,
                                                      const T* __restrict__ c, long long n, int vec4,
                                                      double* partials, unsigned int* counter, double* out,
                                                      const int* flags, PostOp po) {
  KP_PDL_WAIT();
  KP_PDL_TRIGGER();
  if (paused(flags)) return;
  double v[2] = {0.0, 0.0};
  const long long tid = blockIdx.x * (long long)VEC_THREADS + threadIdx.x, stride = (long long)gridDim.x * VEC_THREADS;
  long long i0 = tid;
  if constexpr (std::is_same<T, float>::value) {
    float hi[2] = {0.f, 0.f}, lo[2] = {0.f, 0.f};
    if (vec4) {
      const long long n4 = n >> 2;
      for (long long i = tid; i < n4; i += stride) {
        const float4 x = ld4(a, i), y = ld4(b, i);
        df_add_prod(hi[0], lo[0], x.x, y.x);
        df_add_prod(hi[0], lo[0], x.y, y.y);
        df_add_prod(hi[0], lo[0], x.z, y.z);
        df_add_prod(hi[0], lo[0], x.w, y.w);
        if (c) {
          const float4 z = ld4(c, i);
          df_add_prod(hi[1], lo[1], x.x, z.x);
          df_add_prod(hi[1], lo[1], x.y, z.y);
          df_add_prod(hi[1], lo[1], x.z, z.z);
          df_add_prod(hi[1], lo[1], x.w, z.w);
        }
      }
      i0 = 4 * n4 + tid;
    }
    for (long long i = i0; i < n; i += stride) {
      df_add_prod(hi[0], lo[0], a[i], b[i]);
      if (c) df_add_prod(hi[1], lo[1], a[i], c[i]);
    }
    reduce_finish_df<2>(hi, lo, false, partials, counter, out, c ? 2 : 1, po);
  } else {
    for (long long i = i0; i < n; i += stride) {
      const double ai = (double)a[i];
      v[0] = fma(ai, (double)b[i], v[0]);
      if (c) v[1] = fma(ai, (double)c[i], v[1]);
    }
    reduce_finish<2>(v, false, partials, counter, out, c ? 2 : 1, po);
  }
}
template <typename T>
__global__ void __launch_bounds__(VEC_THREADS) k_dot2(const T* __restrict__ a, const T* __restrict__ b,
                                                      const T* __restrict__ c, long long n, int vec4,
                                                      double* partials, unsigned int* counter, double* out,
                                                      const int* flags, PostOp po) {
  k_dot2_body<T>(a, b, c, n, vec4, partials, counter, out, flags, po);
}

// y = alpha*x + beta*y (scalars from host); used by setup / hooks
template <typename T>
__global__ void k_axpby(const T* __restrict__ x, T* __restrict__ y, long long n, double alpha, double beta) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (T)(alpha * (double)x[i] + beta * (double)y[i]);
}

// ------------------------------------------------------------- PCG updates
// x += alpha p ; r_old = r ; r -= alpha q ; out: rr = ||r||^2, amax(r)
template <typename T>
__global__ void __launch_bounds__(VEC_THREADS) k_update_xr(T* __restrict__ x, T* __restrict__ r,
                                                           T* __restrict__ r_old, const T* __restrict__ p,
                                                           const T* __restrict__ q, long long n, int vec4,
                                                           const double* __restrict__ alpha_dev, double* partials,
                                                           unsigned int* counter, double* out, const int* flags,
                                                           PostOp po) {
  KP_PDL_WAIT();
  KP_PDL_TRIGGER();
  if (paused(flags)) {
    // paused before the update (NaN or breakdown in alpha): inside the loop
    // graph no replacement, and the loop ends
    if (po.cond && blockIdx.x == 0 && threadIdx.x == 0) {
      if (po.cond == 1) {
        cudaGraphSetConditional(po.h_rep, 0u);
        cudaGraphSetConditional(po.h_loop, 0u);
      } else {
        po.f[F_NOTDUE] = 1;
        po.f[F_BLOOP] = 0;
      }
    }
    return;
  }
  double v[2] = {0.0, 0.0};
  const long long tid = blockIdx.x * (long long)VEC_THREADS + threadIdx.x, stride = (long long)gridDim.x * VEC_THREADS;
  if constexpr (std::is_same<T, float>::value) {
    const float al = (float)*alpha_dev;
    long long i0 = tid;
    float hi[2] = {0.f, 0.f}, lo[2] = {0.f, 0.f};  // ||r||^2 (double-float), amax(r)
    if (vec4) {
      const long long n4 = n >> 2;
      for (long long i = tid; i < n4; i += stride) {
        const float4 xi = ld4(x, i), ri = ld4(r, i), pi = ld4(p, i), qi = ld4(q, i);
        st4(x, i, make_float4(fmaf(al, pi.x, xi.x), fmaf(al, pi.y, xi.y), fmaf(al, pi.z, xi.z), fmaf(al, pi.w, xi.w)));
        st4(r_old, i, ri);
        const float4 rn = make_float4(fmaf(-al, qi.x, ri.x), fmaf(-al, qi.y, ri.y), fmaf(-al, qi.z, ri.z),
                                      fmaf(-al, qi.w, ri.w));
        st4(r, i, rn);
        df_add_prod(hi[0], lo[0], rn.x, rn.x);
        df_add_prod(hi[0], lo[0], rn.y, rn.y);
        df_add_prod(hi[0], lo[0], rn.z, rn.z);
        df_add_prod(hi[0], lo[0], rn.w, rn.w);
        hi[1] = fmaxf(hi[1], fmaxf(fmaxf(fabsf(rn.x), fabsf(rn.y)), fmaxf(fabsf(rn.z), fabsf(rn.w))));
      }
      i0 = 4 * n4 + tid;
    }
    for (long long i = i0; i < n; i += stride) {
      const float ri = r[i];
      x[i] = fmaf(al, p[i], x[i]);
      r_old[i] = ri;
      const float rn = fmaf(-al, q[i], ri);
      r[i] = rn;
      df_add_prod(hi[0], lo[0], rn, rn);
      hi[1] = fmaxf(hi[1], fabsf(rn));
    }
    reduce_finish_df<2>(hi, lo, true, partials, counter, out, 2, po);
  } else {
    double v[2] = {0.0, 0.0};
    const double alpha = *alpha_dev;
    for (long long i = tid; i < n; i += stride) {
      T ri = r[i];
      x[i] = (T)((double)x[i] + alpha * (double)p[i]);
      r_old[i] = ri;
      T rn = (T)((double)ri - alpha * (double)q[i]);
      r[i] = rn;
      double d = (double)rn;
      v[0] = fma(d, d, v[0]);
      v[1] = fmax(v[1], fabs(d));
    }
    reduce_finish<2>(v, true, partials, counter, out, 2, po);
  }
}

// p = z + beta p ; optional bf16 split copy of p (slices written at stride).
// With beta_dev null, p = z: the old p is not read (it may be uninitialised).
template <typename T>
__device__ __forceinline__ void k_p_update_body(T* __restrict__ p, const T* __restrict__ z, long long n, int vec4,
                           const double* __restrict__ beta_dev, __nv_bfloat16* __restrict__ ps, int slices,
                           long long sstride, const int* flags) {
  KP_PDL_WAIT();
  KP_PDL_TRIGGER();
  if (paused(flags)) return;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
  if constexpr (std::is_same<T, float>::value) {
    const float be = beta_dev ? (float)*beta_dev : 0.f;
    long long i0 = tid;
    if (vec4) {
      const long long n4 = n >> 2;
      for (long long i = tid; i < n4; i += stride) {
        const float4 zi = ld4(z, i);
        float4 pn = zi;
        if (beta_dev) {
          const float4 pi = ld4(p, i);
          pn = make_float4(fmaf(be, pi.x, zi.x), fmaf(be, pi.y, zi.y), fmaf(be, pi.z, zi.z), fmaf(be, pi.w, zi.w));
        }
        st4(p, i, pn);
        if (ps) {
          float w[4] = {pn.x, pn.y, pn.z, pn.w};
          for (int sl = 0; sl < slices; ++sl) {
            __nv_bfloat162 h0 = __floats2bfloat162_rn(w[0], w[1]);
            __nv_bfloat162 h1 = __floats2bfloat162_rn(w[2], w[3]);
            uint2 pk;
            pk.x = *reinterpret_cast<uint32_t*>(&h0);
            pk.y = *reinterpret_cast<uint32_t*>(&h1);
            *reinterpret_cast<uint2*>(ps + sl * sstride + 4 * i) = pk;
            w[0] -= __bfloat162float(h0.x);
            w[1] -= __bfloat162float(h0.y);
            w[2] -= __bfloat162float(h1.x);
            w[3] -= __bfloat162float(h1.y);
          }
        }
      }
      i0 = 4 * n4 + tid;
    }
    for (long long i = i0; i < n; i += stride) {
      const float pn = beta_dev ? fmaf(be, p[i], z[i]) : z[i];
      p[i] = pn;
      if (ps) {
        float v = pn;
        for (int sl = 0; sl < slices; ++sl) {
          __nv_bfloat16 h = __float2bfloat16_rn(v);
          ps[sl * sstride + i] = h;
          v -= __bfloat162float(h);
        }
      }
    }
  } else {
    const double beta = beta_dev ? *beta_dev : 0.0;
    for (long long i = tid; i < n; i += stride) {
      T pn = beta_dev ? (T)((double)z[i] + beta * (double)p[i]) : z[i];
      p[i] = pn;
      if (ps) {
        float v = (float)pn;
        for (int sl = 0; sl < slices; ++sl) {
          __nv_bfloat16 h = __float2bfloat16_rn(v);
          ps[sl * sstride + i] = h;
          v -= __bfloat162float(h);
        }
      }
    }
  }
}
template <typename T>
__global__ void k_p_update(T* __restrict__ p, const T* __restrict__ z, long long n, int vec4,
                           const double* __restrict__ beta_dev, __nv_bfloat16* __restrict__ ps, int slices,
                           long long sstride, const int* flags) {
  k_p_update_body<T>(p, z, n, vec4, beta_dev, ps, slices, sstride, flags);
}

// bf16 slices of a vector (x -> hi, mid, lo)
template <typename T>
__device__ __forceinline__ void k_split_body(const T* __restrict__ x, long long n, __nv_bfloat16* __restrict__ out, int slices,
                        long long sstride, const int* flags) {
  KP_PDL_WAIT();
  KP_PDL_TRIGGER();
  if (paused(flags)) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float v = (float)x[i];
    for (int s = 0; s < slices; ++s) {
      __nv_bfloat16 h = __float2bfloat16_rn(v);
      out[s * sstride + i] = h;
      v -= __bfloat162float(h);
    }
  }
}
template <typename T>
__global__ void k_split(const T* __restrict__ x, long long n, __nv_bfloat16* __restrict__ out, int slices,
                        long long sstride, const int* flags) {
  k_split_body<T>(x, n, out, slices, sstride, flags);
}

// Quantise r for the reduced-precision preconditioner: out = narrow(r * 2^e)
// with 2^e chosen from amax(r) (stat[1]) so that amax * 2^e lies in
// [target/2, target); writes inv_out = 1 / (lam2 * 2^e) for the last GEMM.
__device__ __forceinline__ float pow2_scale(double amax, double target) {
  if (!(amax > 0.0) || !isfinite(amax)) return 1.f;
  int e;
  frexp(target / amax, &e);  // target/amax = m 2^e, m in [0.5, 1)
  return (float)ldexp(1.0, e - 1);
}
template <typename T, typename N>
__device__ __forceinline__ void k_quantize_body(const T* __restrict__ r, long long n, int vec4, const double* __restrict__ stat,
                           double target, double lam2, N* __restrict__ out, float* __restrict__ inv_out,
                           unsigned int* __restrict__ reset, int nreset, const int* flags) {
  KP_PDL_WAIT();
  KP_PDL_TRIGGER();
  if (paused(flags)) return;
  __shared__ float s_sh;
  if (threadIdx.x == 0) {
    s_sh = pow2_scale(stat[1], target);
    if (blockIdx.x == 0) {
      *inv_out = (float)(1.0 / (lam2 * (double)s_sh));
      for (int i = 0; i < nreset; ++i) reset[i] = 0u;  // per-stage amax slots of this apply
    }
  }
  __syncthreads();
  const float s = s_sh;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
  long long i0 = tid;
  if (vec4) {
    const long long n4 = n >> 2;
    for (long long i = tid; i < n4; i += stride) {
      const float4 v = ld4((const float*)r, i);
      out[4 * i + 0] = to_narrow<N>(v.x * s);
      out[4 * i + 1] = to_narrow<N>(v.y * s);
      out[4 * i + 2] = to_narrow<N>(v.z * s);
      out[4 * i + 3] = to_narrow<N>(v.w * s);
    }
    i0 = 4 * n4 + tid;
  }
  for (long long i = i0; i < n; i += stride) out[i] = to_narrow<N>((float)r[i] * s);
}
template <typename T, typename N>
__global__ void k_quantize(const T* __restrict__ r, long long n, int vec4, const double* __restrict__ stat,
                           double target, double lam2, N* __restrict__ out, float* __restrict__ inv_out,
                           unsigned int* __restrict__ reset, int nreset, const int* flags) {
  k_quantize_body<T, N>(r, n, vec4, stat, target, lam2, out, inv_out, reset, nreset, flags);
}

// two narrow values packed in 32 bits (low half first)
template <typename NQ>
__device__ __forceinline__ uint32_t pack2(float a, float b);
template <>
__device__ __forceinline__ uint32_t pack2<__half>(float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}
template <>
__device__ __forceinline__ uint32_t pack2<__nv_bfloat16>(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// x += alpha p ; r_old = r ; r -= alpha q ; ||r||^2, max |r| (as k_update_xr)
// and the preconditioner input out = narrow(r * s) in the same pass.  The
// scale s is a power of two from the bound max |r| + |alpha| max |q| >=
// max |r_new|, both known before the update, so no extra pass over r is
// needed; the bound (not the exact max) only moves values down in the
// narrow type's range.  out2[1] (max |r| of the previous update) is read by
// every block before the last block overwrites it.
template <typename NQ>
__device__ __forceinline__ void k_update_xr_q_body(float* __restrict__ x, float* __restrict__ r, float* __restrict__ r_old, const float* __restrict__ p,
                  const float* __restrict__ q, long long n, int vec4, const double* __restrict__ alpha_dev,
                  const double* __restrict__ qmax_dev, double lam2, NQ* __restrict__ out, float* __restrict__ inv_out,
                  double* partials, unsigned int* counter, double* out2, const int* flags, PostOp po) {
  KP_PDL_WAIT();
  KP_PDL_TRIGGER();
  if (paused(flags)) {
    if (po.cond && blockIdx.x == 0 && threadIdx.x == 0) {
      if (po.cond == 1) {
        cudaGraphSetConditional(po.h_rep, 0u);
        cudaGraphSetConditional(po.h_loop, 0u);
      } else {  // batched loop: this problem takes no replacement and has stopped
        po.f[F_NOTDUE] = 1;
        po.f[F_BLOOP] = 0;
      }
    }
    return;
  }
  __shared__ float s_sh;
  if (threadIdx.x == 0) {
    const double bound = out2[1] + fabs(*alpha_dev) * *qmax_dev;
    s_sh = pow2_scale(bound * (1.0 + 1e-6), 1.0);
    if (blockIdx.x == 0) *inv_out = (float)(1.0 / (lam2 * (double)s_sh));
  }
  __syncthreads();
  const float sc = s_sh;
  const float al = (float)*alpha_dev;
  const long long tid = blockIdx.x * (long long)VEC_THREADS + threadIdx.x, stride = (long long)gridDim.x * VEC_THREADS;
  long long i0 = tid;
  float hi[2] = {0.f, 0.f}, lo[2] = {0.f, 0.f};
  if (vec4) {
    const long long n4 = n >> 2;
    for (long long i = tid; i < n4; i += stride) {
      const float4 xi = ld4(x, i), ri = ld4(r, i), pi = ld4(p, i), qi = ld4(q, i);
      st4(x, i, make_float4(fmaf(al, pi.x, xi.x), fmaf(al, pi.y, xi.y), fmaf(al, pi.z, xi.z), fmaf(al, pi.w, xi.w)));
      st4(r_old, i, ri);
      const float4 rn = make_float4(fmaf(-al, qi.x, ri.x), fmaf(-al, qi.y, ri.y), fmaf(-al, qi.z, ri.z),
                                    fmaf(-al, qi.w, ri.w));
      st4(r, i, rn);
      *reinterpret_cast<uint2*>(out + 4 * i) = make_uint2(pack2<NQ>(rn.x * sc, rn.y * sc), pack2<NQ>(rn.z * sc, rn.w * sc));
      df_add_prod(hi[0], lo[0], rn.x, rn.x);
      df_add_prod(hi[0], lo[0], rn.y, rn.y);
      df_add_prod(hi[0], lo[0], rn.z, rn.z);
      df_add_prod(hi[0], lo[0], rn.w, rn.w);
      hi[1] = fmaxf(hi[1], fmaxf(fmaxf(fabsf(rn.x), fabsf(rn.y)), fmaxf(fabsf(rn.z), fabsf(rn.w))));
    }
    i0 = 4 * n4 + tid;
  }
  for (long long i = i0; i < n; i += stride) {
    const float ri = r[i];
    x[i] = fmaf(al, p[i], x[i]);
    r_old[i] = ri;
    const float rn = fmaf(-al, q[i], ri);
    r[i] = rn;
    out[i] = to_narrow<NQ>(rn * sc);
    df_add_prod(hi[0], lo[0], rn, rn);
    hi[1] = fmaxf(hi[1], fabsf(rn));
  }
  reduce_finish_df<2>(hi, lo, true, partials, counter, out2, 2, po);
}
template <typename NQ>
__global__ void __launch_bounds__(VEC_THREADS)
    k_update_xr_q(float* __restrict__ x, float* __restrict__ r, float* __restrict__ r_old, const float* __restrict__ p,
                  const float* __restrict__ q, long long n, int vec4, const double* __restrict__ alpha_dev,
                  const double* __restrict__ qmax_dev, double lam2, NQ* __restrict__ out, float* __restrict__ inv_out,
                  double* partials, unsigned int* counter, double* out2, const int* flags, PostOp po) {
  k_update_xr_q_body<NQ>(x, r, r_old, p, q, n, vec4, alpha_dev, qmax_dev, lam2, out, inv_out, partials, counter, out2, flags, po);
}

// One stage of the E4M3 preconditioner solve: the stage's FP32 GEMM output
// (max |.| accumulated by the GEMM epilogue into *amax_bits) is scaled by a
// power of two g putting its maximum into [224, 448) and rounded to E4M3;
// g is kept in gs[stage].  The last stage also writes the scale of the final
// product, inv_out = base / (g_0 g_1 g_2).
__global__ void k_quant8(const float* __restrict__ in, long long n, int vec4, const unsigned int* __restrict__ amax_bits,
                         float* __restrict__ gs, int stage, const float* __restrict__ base, float* __restrict__ inv_out,
                         __nv_fp8_e4m3* __restrict__ out, const int* flags) {
  KP_PDL_WAIT();
  KP_PDL_TRIGGER();
  if (paused(flags)) return;
  __shared__ float g_sh;
  if (threadIdx.x == 0) {
    const float am = __uint_as_float(*amax_bits);
    g_sh = pow2_scale((double)am, 448.0);
    if (blockIdx.x == 0) {
      gs[stage] = g_sh;
      if (stage == 2) *inv_out = *base / (gs[0] * gs[1] * g_sh);
    }
  }
  __syncthreads();
  const float g = g_sh;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
  long long i0 = tid;
  if (vec4) {
    const long long n4 = n >> 2;
    for (long long i = tid; i < n4; i += stride) {
      const float4 v = ld4(in, i);
      const __nv_fp8x4_e4m3 q(make_float4(v.x * g, v.y * g, v.z * g, v.w * g));
      reinterpret_cast<__nv_fp8x4_e4m3*>(out)[i] = q;
    }
    i0 = 4 * n4 + tid;
  }
  for (long long i = i0; i < n; i += stride) out[i] = __nv_fp8_e4m3(in[i] * g);
}

// amax only (for one-off applies outside the loop)
template <typename T>
__device__ __forceinline__ void k_norm_amax_body(const T* __restrict__ x, long long n, double* partials,
                                                           unsigned int* counter, double* out, const int* flags) {
  KP_PDL_WAIT();
  KP_PDL_TRIGGER();
  if (paused(flags)) return;
  double v[2] = {0.0, 0.0};
  const long long tid = blockIdx.x * (long long)VEC_THREADS + threadIdx.x, stride = (long long)gridDim.x * VEC_THREADS;
  if constexpr (std::is_same<T, float>::value) {
    float hi[2] = {0.f, 0.f}, lo[2] = {0.f, 0.f};
    for (long long i = tid; i < n; i += stride) {
      const float d = x[i];
      df_add_prod(hi[0], lo[0], d, d);
      hi[1] = fmaxf(hi[1], fabsf(d));
    }
    reduce_finish_df<2>(hi, lo, true, partials, counter, out, 2);
  } else {
    for (long long i = tid; i < n; i += stride) {
      double d = (double)x[i];
      v[0] = fma(d, d, v[0]);
      v[1] = fmax(v[1], fabs(d));
    }
    reduce_finish<2>(v, true, partials, counter, out, 2);
  }
}
template <typename T>
__global__ void __launch_bounds__(VEC_THREADS) k_norm_amax(const T* __restrict__ x, long long n, double* partials,
                                                           unsigned int* counter, double* out, const int* flags) {
  k_norm_amax_body<T>(x, n, partials, counter, out, flags);
}

template <typename A, typename B>
__global__ void k_convert(const A* __restrict__ x, B* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (B)x[i];
}

}  // namespace kpv

// ------------------------------------------------------------- host wrappers
using namespace kpv;

// bodies of the kernels that batched solves group (kp_group.cuh)
KP_BODY(DotF, kpv::k_dot2_body<float>);
KP_BODY(DotD, kpv::k_dot2_body<double>);
KP_BODY(NormAmaxF, kpv::k_norm_amax_body<float>);
KP_BODY(NormAmaxD, kpv::k_norm_amax_body<double>);
KP_BODY(UpdXrQH, kpv::k_update_xr_q_body<__half>);
KP_BODY(UpdXrQB, kpv::k_update_xr_q_body<__nv_bfloat16>);
KP_BODY(PUpdF, kpv::k_p_update_body<float>);
KP_BODY(PUpdD, kpv::k_p_update_body<double>);
KP_BODY(SplitF, kpv::k_split_body<float>);
KP_BODY(SplitD, kpv::k_split_body<double>);
KP_BODY(QuantB, kpv::k_quantize_body<float, __nv_bfloat16>);
KP_BODY(QuantH, kpv::k_quantize_body<float, __half>);
KP_BODY(Quant8, kpv::k_quantize_body<float, __nv_fp8_e4m3>);

int vec_grid(kp_ctx* ctx, long long n) {
  long long b = (n + VEC_THREADS * 4 - 1) / (VEC_THREADS * 4);
  long long cap = (long long)ctx->sm_count * 4;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

static int aligned16(const void* a, const void* b = nullptr, const void* c = nullptr, const void* d = nullptr,
                     const void* e = nullptr) {
  const uintptr_t m = (uintptr_t)a | (uintptr_t)b | (uintptr_t)c | (uintptr_t)d | (uintptr_t)e;
  return (m & 15) == 0 ? 1 : 0;
}

kp_status dot2_dev(kp_ctx* ctx, const void* a, const void* b, const void* c, long long n, bool f64, double* out,
                   const int* flags, PostOp post) {
  int g = vec_grid(ctx, n);
  if (f64)
    KP_CUDA(kp_launch_g<DotD>(ctx, k_dot2<double>, dim3(g), dim3(VEC_THREADS), 0, (const double*)a, (const double*)b, (const double*)c, n, 0,
                                                       ctx->red_part, ctx->red_count, out, flags, post));
  else
    KP_CUDA(kp_launch_g<DotF>(ctx, k_dot2<float>, dim3(g), dim3(VEC_THREADS), 0, (const float*)a, (const float*)b, (const float*)c, n,
                                                      aligned16(a, b, c), ctx->red_part, ctx->red_count, out, flags,
                                                      post));
  KP_LAUNCHED(ctx);
  KP_CUDA(cudaGetLastError());
  return KP_OK;
}

kp_status dot_dev(kp_ctx* ctx, const void* x, const void* y, long long n, bool f64, double* out_dev) {
  return dot2_dev(ctx, x, y, nullptr, n, f64, out_dev, nullptr);
}

kp_status norm_amax_dev(kp_ctx* ctx, const void* x, long long n, bool f64, double* out2, const int* flags) {
  int g = vec_grid(ctx, n);
  if (f64)
    KP_CUDA(kp_launch_g<NormAmaxD>(ctx, k_norm_amax<double>, dim3(g), dim3(VEC_THREADS), 0, (const double*)x, n, ctx->red_part, ctx->red_count, out2, flags));
  else
    KP_CUDA(kp_launch_g<NormAmaxF>(ctx, k_norm_amax<float>, dim3(g), dim3(VEC_THREADS), 0, (const float*)x, n, ctx->red_part, ctx->red_count, out2, flags));
  KP_LAUNCHED(ctx);
  KP_CUDA(cudaGetLastError());
  return KP_OK;
}

kp_status norm2_dev(kp_ctx* ctx, const void* x, long long n, bool f64, double* out_dev) {
  return dot2_dev(ctx, x, x, nullptr, n, f64, out_dev, nullptr);
}

kp_status update_xr_dev(kp_ctx* ctx, void* x, void* r, void* r_old, const void* p, const void* q, long long n,
                        bool f64, const double* alpha_dev, double* out2, const int* flags, PostOp post) {
  int g = vec_grid(ctx, n);
  if (f64)
    KP_CUDA(kp_launch(ctx, k_update_xr<double>, dim3(g), dim3(VEC_THREADS), 0, (double*)x, (double*)r, (double*)r_old, (const double*)p,
                                                            (const double*)q, n, 0, alpha_dev, ctx->red_part,
                                                            ctx->red_count, out2, flags, post));
  else
    KP_CUDA(kp_launch(ctx, k_update_xr<float>, dim3(g), dim3(VEC_THREADS), 0, (float*)x, (float*)r, (float*)r_old, (const float*)p,
                                                           (const float*)q, n, aligned16(x, r, r_old, p, q),
                                                           alpha_dev, ctx->red_part, ctx->red_count, out2, flags,
                                                           post));
  KP_LAUNCHED(ctx);
  KP_CUDA(cudaGetLastError());
  return KP_OK;
}

kp_status update_xr_q_dev(kp_ctx* ctx, void* x, void* r, void* r_old, const void* p, const void* q, long long n,
                          const double* alpha_dev, double* out2, const double* qmax_dev, int narrow, double lam2,
                          void* pc_out, float* inv_out, const int* flags, PostOp post) {
  const int g = vec_grid(ctx, n);
  const int v4 = aligned16(x, r, r_old, p, q) && (((uintptr_t)pc_out & 7) == 0);
  if (narrow == NT_F16)
    KP_CUDA(kp_launch_g<UpdXrQH>(ctx, k_update_xr_q<__half>, dim3(g), dim3(VEC_THREADS), 0, (float*)x, (float*)r, (float*)r_old,
                      (const float*)p, (const float*)q, n, v4, alpha_dev, qmax_dev, lam2, (__half*)pc_out, inv_out,
                      ctx->red_part, ctx->red_count, out2, flags, post));
  else if (narrow == NT_BF16)
    KP_CUDA(kp_launch_g<UpdXrQB>(ctx, k_update_xr_q<__nv_bfloat16>, dim3(g), dim3(VEC_THREADS), 0, (float*)x, (float*)r,
                      (float*)r_old, (const float*)p, (const float*)q, n, v4, alpha_dev, qmax_dev, lam2,
                      (__nv_bfloat16*)pc_out, inv_out, ctx->red_part, ctx->red_count, out2, flags, post));
  else {
    kp_set_error("update_xr_q: the fused preconditioner input is F16 or BF16");
    return KP_ENOTSUP;
  }
  KP_LAUNCHED(ctx);
  KP_CUDA(cudaGetLastError());
  return KP_OK;
}

kp_status p_update_dev(kp_ctx* ctx, void* p, const void* z, long long n, bool f64, const double* beta_dev,
                       __nv_bfloat16* ps, int slices, long long sstride, const int* flags) {
  int g = vec_grid(ctx, n);
  if (f64)
    KP_CUDA(kp_launch_g<PUpdD>(ctx, k_p_update<double>, dim3(g), dim3(VEC_THREADS), 0, (double*)p, (const double*)z, n, 0, beta_dev, ps, slices,
                                                           sstride, flags));
  else
    KP_CUDA(kp_launch_g<PUpdF>(ctx, k_p_update<float>, dim3(g), dim3(VEC_THREADS), 0, 
        (float*)p, (const float*)z, n, aligned16(p, z) && (((uintptr_t)ps & 7) == 0) && (sstride % 4 == 0), beta_dev,
        ps, slices, sstride, flags));
  KP_LAUNCHED(ctx);
  KP_CUDA(cudaGetLastError());
  return KP_OK;
}

kp_status split_bf16(kp_ctx* ctx, const void* x, bool f64, long long n, void* out, int slices, long long sstride,
                     const int* flags) {
  int g = vec_grid(ctx, n);
  if (f64)
    KP_CUDA(kp_launch_g<SplitD>(ctx, k_split<double>, dim3(g), dim3(VEC_THREADS), 0, (const double*)x, n, (__nv_bfloat16*)out, slices, sstride, flags));
  else
    KP_CUDA(kp_launch_g<SplitF>(ctx, k_split<float>, dim3(g), dim3(VEC_THREADS), 0, (const float*)x, n, (__nv_bfloat16*)out, slices, sstride, flags));
  KP_LAUNCHED(ctx);
  KP_CUDA(cudaGetLastError());
  return KP_OK;
}

kp_status quant8_dev(kp_ctx* ctx, const float* in, long long n, const unsigned int* amax_bits, float* gs, int stage,
                     const float* base, float* inv_out, void* out, const int* flags) {
  int g = vec_grid(ctx, n);
  const int v4 = aligned16(in) && (((uintptr_t)out & 3) == 0);
  KP_CUDA(kp_launch(ctx, k_quant8, dim3(g), dim3(VEC_THREADS), 0, in, n, v4, amax_bits, gs, stage, base, inv_out,
                    (__nv_fp8_e4m3*)out, flags));
  KP_LAUNCHED(ctx);
  return KP_OK;
}

kp_status quantize_dev(kp_ctx* ctx, const void* r, long long n, bool f64, const double* stat, int narrow,
                       double lam2, void* out, float* inv_out, const int* flags, unsigned int* reset, int nreset) {
  int g = vec_grid(ctx, n);
  double target = narrow == NT_E4M3 ? 448.0 : 1.0;
  if (f64) {
    kp_set_error("reduced-precision preconditioner needs FP32 vectors");
    return KP_ENOTSUP;
  }
  const float* rf = (const float*)r;
  const int v4 = aligned16(r);
  if (narrow == NT_BF16)
    KP_CUDA(kp_launch_g<QuantB>(ctx, k_quantize<float, __nv_bfloat16>, dim3(g), dim3(VEC_THREADS), 0, rf, n, v4, stat, target, lam2,
                                                                          (__nv_bfloat16*)out, inv_out, reset, nreset, flags));
  else if (narrow == NT_F16)
    KP_CUDA(kp_launch_g<QuantH>(ctx, k_quantize<float, __half>, dim3(g), dim3(VEC_THREADS), 0, rf, n, v4, stat, target, lam2, (__half*)out,
                                                                   inv_out, reset, nreset, flags));
  else
    KP_CUDA(kp_launch_g<Quant8>(ctx, k_quantize<float, __nv_fp8_e4m3>, dim3(g), dim3(VEC_THREADS), 0, rf, n, v4, stat, target, lam2,
                                                                          (__nv_fp8_e4m3*)out, inv_out, reset, nreset, flags));
  KP_LAUNCHED(ctx);
  KP_CUDA(cudaGetLastError());
  return KP_OK;
}

kp_status copy_vec(kp_ctx* ctx, const void* x, void* y, long long n, bool f64) {
  KP_CUDA(cudaMemcpyAsync(y, x, n * (f64 ? 8 : 4), cudaMemcpyDeviceToDevice, ctx->stream));
  return KP_OK;
}

kp_status axpby_dev(kp_ctx* ctx, const void* x, void* y, long long n, bool f64, double alpha, double beta) {
  int g = vec_grid(ctx, n);
  if (f64)
    k_axpby<double><<<g, VEC_THREADS, 0, ctx->stream>>>((const double*)x, (double*)y, n, alpha, beta);
  else
    k_axpby<float><<<g, VEC_THREADS, 0, ctx->stream>>>((const float*)x, (float*)y, n, alpha, beta);
  KP_LAUNCHED(ctx);
  KP_CUDA(cudaGetLastError());
  return KP_OK;
}

kp_status convert_f64_to_f32(kp_ctx* ctx, const double* x, float* y, long long n) {
  int g = vec_grid(ctx, n);
  k_convert<double, float><<<g, VEC_THREADS, 0, ctx->stream>>>(x, y, n);
  KP_LAUNCHED(ctx);
  KP_CUDA(cudaGetLastError());
  return KP_OK;
}
kp_status convert_f32_to_f64(kp_ctx* ctx, const float* x, double* y, long long n) {
  int g = vec_grid(ctx, n);
  k_convert<float, double><<<g, VEC_THREADS, 0, ctx->stream>>>(x, y, n);
  KP_LAUNCHED(ctx);
  KP_CUDA(cudaGetLastError());
  return KP_OK;
}
