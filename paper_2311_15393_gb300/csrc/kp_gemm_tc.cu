// Tensor-core GEMM for sm_103a: tcgen05.mma with TMEM accumulators, operands
// staged by TMA (cp.async.bulk.tensor) into 128-byte-swizzled shared memory.
//
//   D[m][n] = sum_p sum_k sum_kk A[sa_p * a_terms + k][m][kk] * B[sb_p * b_terms + k][n][kk]
//
// Used for the dense n x n Kronecker contractions of the operator
// (A vec(X) = vec(sum_k A_c^(k) X A_r^(k)^T), Section 3, eq. KronSumDecomp)
// and of the preconditioner solve Z = V_c (S .* (V_c^T R V_r)) V_r^T
// (eq. PreconSolve), in BF16 / FP16 (kind::f16) or FP8 E4M3 (kind::f8f6f4)
// with FP32 accumulation.  Reduced-precision operands split a value into
// bf16 slices (hi + lo + ...) and sum slice products to recover FP32-level
// accuracy where needed.
//
// Persistent kernel, one or two CTAs per SM.  Work units are (128 x BN
// output tile, K split) pairs handed out round-robin over the grid:
//   warp 0      TMA producer (lanes 0 / 1: A / B tiles): STAGES-deep ring
//   warp 1      TMEM allocation + MMA issuer (one thread)
//   warps 2..5  epilogue: tcgen05.ld TMEM -> registers -> fused output
// The accumulator is double-buffered in TMEM (2 x BN columns), so the
// epilogue of one unit overlaps the main loop of the next.  With split-K each
// split writes an FP32 partial tile; the split that arrives last (per-tile
// counter) sums the partials in split order, so results do not depend on
// scheduling, and runs the fused epilogue.  Every wait is bounded; a wait
// that gives up sets DEV_ERR_TIMEOUT in the device status word, and the CTA
// drains and returns.
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "kp_internal.h"
#include "kp_vec.cuh"

namespace {

constexpr int TBM = 128;
constexpr int TC_THREADS = 192;

// Tile configurations: 128 x BN output tiles, CPS CTAs resident per SM.  The
// shared-memory ring is as deep as ~192 KiB per SM allows: the loads of a
// k-step take about a microsecond to arrive, so a deep ring (bytes in
// flight) is what keeps the tensor pipe fed.
//   BN 256, 1 CTA/SM: 4 x 48 KiB     BN 128, 1 CTA/SM: 6 x 32 KiB
//   BN 128, 2 CTAs/SM: 3 x 32 KiB each (one's prologue / epilogue overlaps
//   the other's main loop)            BN 64, 1 CTA/SM: 8 x 24 KiB
// Narrow tiles give the square n x n products enough tiles to occupy the
// SMs without splitting K (split-K partials cost more than they save here).
// A ring stage holds KPS k-blocks (each an A and a B tile of 128-byte rows):
// the producer and MMA threads pay their per-stage costs (barrier waits,
// commits, loop control) once per KPS k-blocks.
template <int BN, int CPS, int KPS = 1>
struct TcCfg {
  static_assert(CPS == 1 || (CPS == 2 && BN <= 128), "TMEM holds 2 x BN columns per CTA");
  static constexpr int A_BYTES = TBM * 128;
  static constexpr int B_BYTES = BN * 128;
  static constexpr int KB_BYTES = A_BYTES + B_BYTES;  // one k-block
  static constexpr int STAGE = KPS * KB_BYTES;
  static constexpr int STAGES = (196608 / CPS) / STAGE;
  static constexpr int SMEM = STAGES * STAGE + 1024 /*align*/ + 512 /*barriers*/;
  static constexpr int TMEM_COLS = 2 * BN;
  static_assert(STAGES >= 2, "ring too shallow");
};

struct TcParams {
  int M, N, K;
  int nkron, npairs, a_terms, b_terms;
  int sa[KP_MAX_PAIRS], sb[KP_MAX_PAIRS];
  int kblocks;      // ceil(K / BK)
  int splits;       // split-K factor over the (pair, term, kblock) steps
  int steps_total;  // npairs * nkron * kblocks (npairs * kblocks when batched)
  int batch_rows;   // > 0: term index = tile row / batch_rows, no sum over terms
  int tiles_m, tiles_n, units;
  uint32_t idesc;
  EpiParams epi;
  float* ws;                // split-K partials [split][M][N]
  unsigned int* counters;   // split-K arrival counters, one per tile (self-resetting)
  const float* alpha_dev;   // optional device scale multiplied into the output
  const int* flags;
  int* status;
  // multicast-cluster kernel only: sum(out * aux) as a double-float pair and
  // max |out| over the whole output into dot_out[0..1] (null: none), the
  // last CTA to finish running dot_po on them
  double* dot_out;
  double* dot_part;
  unsigned int* dot_count;
  PostOp dot_po;
  int dot_qmax;
};

// ------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; returns false (and flags the status word) on give-up
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* status) {
  for (long long i = 0; i < KP_SPIN_LIMIT; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  atomicOr(status, DEV_ERR_TIMEOUT);
  return false;
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms of
// 1024 bytes (stride byte offset), descriptor version 1 (sm_100 family)
__device__ __forceinline__ uint64_t make_sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;            // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024u >> 4) << 32;  // stride byte offset
  d |= (uint64_t)1u << 46;            // version
  d |= (uint64_t)2u << 61;            // SWIZZLE_128B
  return d;
}

template <int KIND>
__device__ __forceinline__ void mma_issue(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accum) {
  if constexpr (KIND == TC_E4M3) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
  }
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------- epilogue
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ uint32_t pack_f16(float a, float b) {
  __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ uint32_t pack_e4m3(float a, float b, float c, float d) {
  __nv_fp8_e4m3 q[4] = {__nv_fp8_e4m3(a), __nv_fp8_e4m3(b), __nv_fp8_e4m3(c), __nv_fp8_e4m3(d)};
  return (uint32_t)q[0].__x | ((uint32_t)q[1].__x << 8) | ((uint32_t)q[2].__x << 16) | ((uint32_t)q[3].__x << 24);
}

// Fused output of one row segment of 32 columns (row gm, columns gn0..gn0+31).
// All indexing is at compile time (the values stay in registers); full
// segments use 16-byte vector accesses, ragged ones predicated scalars.
__device__ __forceinline__ void epi_store32(const EpiParams& e, float scale_dev, int gm, int gn0, int N,
                                            float (&v)[32], float& tmax) {
  const int cnt = min(32, N - gn0);
  if (cnt <= 0) return;
  const long long base = (long long)gm * e.ldd + gn0;
  const float* aux = (const float*)e.aux;
  const long long abase = (long long)gm * e.ld_aux + gn0;
  const bool vec = (cnt == 32) && ((base & 7) == 0) && (aux == nullptr || (abase & 3) == 0);
  const float a = (float)e.alpha * scale_dev;
#pragma unroll
  for (int c = 0; c < 32; ++c) v[c] *= a;
  if (aux) {
    const float bt = (float)e.beta;
    if (vec) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 t = *reinterpret_cast<const float4*>(aux + abase + 4 * q);
        v[4 * q + 0] = fmaf(bt, t.x, v[4 * q + 0]);
        v[4 * q + 1] = fmaf(bt, t.y, v[4 * q + 1]);
        v[4 * q + 2] = fmaf(bt, t.z, v[4 * q + 2]);
        v[4 * q + 3] = fmaf(bt, t.w, v[4 * q + 3]);
      }
    } else {
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c < cnt) v[c] = fmaf(bt, aux[abase + c], v[c]);
    }
  }
  if ((e.mode == EPI_NARROW || e.mode == EPI_F32) && e.sigma32) {
    // S' = lam^2 / (sigma^2 + lam^2) in FP32 (it scales a value about to be
    // rounded to 16 or 8 bits; FP64 arithmetic is slow on this part)
    const float l2 = (float)e.lam2;
    if (vec) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 sg = *reinterpret_cast<const float4*>(e.sigma32 + base + 4 * q);
        v[4 * q + 0] *= __fdividef(l2, fmaf(sg.x, sg.x, l2));
        v[4 * q + 1] *= __fdividef(l2, fmaf(sg.y, sg.y, l2));
        v[4 * q + 2] *= __fdividef(l2, fmaf(sg.z, sg.z, l2));
        v[4 * q + 3] *= __fdividef(l2, fmaf(sg.w, sg.w, l2));
      }
    } else {
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        if (c < cnt) {
          const float sg = e.sigma32[base + c];
          v[c] *= __fdividef(l2, fmaf(sg, sg, l2));
        }
      }
    }
  }
  if (e.mode == EPI_F32) {
    if (e.bias || e.act) {  // the learned-lambda MLP's bias and activation
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        if (c < cnt) {
          if (e.bias) v[c] += e.bias[gn0 + c];
          if (e.act == 1) {
            e.pre[base + c] = v[c];
            v[c] = kp_gelu(v[c]);
          } else if (e.act == 2) {
            v[c] *= kp_gelu_grad(e.pre[base + c]);
          }
        }
      }
    }
    if (e.amax_bits) {
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c < cnt) tmax = fmaxf(tmax, fabsf(v[c]));
    }
    float* out = (float*)e.out + base;
    if (vec) {
#pragma unroll
      for (int q = 0; q < 8; ++q)
        *reinterpret_cast<float4*>(out + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else {
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c < cnt) out[c] = v[c];
    }
  } else if (e.mode == EPI_SLICES) {
    __nv_bfloat16* out = (__nv_bfloat16*)e.out + base;
    for (int s = 0; s < e.slices; ++s) {
      __nv_bfloat16* o = out + s * e.slice_stride;
      if (vec) {
        uint32_t w[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          w[q] = pack_bf16(v[2 * q], v[2 * q + 1]);
          const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&w[q]);
          v[2 * q] -= __bfloat162float(h.x);
          v[2 * q + 1] -= __bfloat162float(h.y);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
          *reinterpret_cast<uint4*>(o + 8 * q) = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
      } else {
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const __nv_bfloat16 h = __float2bfloat16_rn(v[c]);
          if (c < cnt) o[c] = h;
          v[c] -= __bfloat162float(h);
        }
      }
    }
  } else if (e.mode == EPI_NARROW) {
    if (e.narrow == NT_E4M3) {
      uint8_t* o = (uint8_t*)e.out + base;
      if (vec && (base & 15) == 0) {
        uint32_t w[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) w[q] = pack_e4m3(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        *reinterpret_cast<uint4*>(o) = make_uint4(w[0], w[1], w[2], w[3]);
        *reinterpret_cast<uint4*>(o + 16) = make_uint4(w[4], w[5], w[6], w[7]);
      } else {
#pragma unroll
        for (int c = 0; c < 32; ++c)
          if (c < cnt) o[c] = __nv_fp8_e4m3(v[c]).__x;
      }
    } else {
      const bool bf = e.narrow == NT_BF16;
      uint16_t* o = (uint16_t*)e.out + base;
      if (vec) {
        uint32_t w[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) w[q] = bf ? pack_bf16(v[2 * q], v[2 * q + 1]) : pack_f16(v[2 * q], v[2 * q + 1]);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          *reinterpret_cast<uint4*>(o + 8 * q) = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
      } else {
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          if (c < cnt) {
            const uint32_t w = bf ? pack_bf16(v[c], 0.f) : pack_f16(v[c], 0.f);
            o[c] = (uint16_t)(w & 0xFFFFu);
          }
        }
      }
    }
  }
}

// FP32 partial of one 32-column row segment (split-K)
__device__ __forceinline__ void partial_store32(float* w, int cnt, const float (&v)[32]) {
  if (cnt == 32) {
#pragma unroll
    for (int q = 0; q < 8; ++q)
      *reinterpret_cast<float4*>(w + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  } else {
#pragma unroll
    for (int c = 0; c < 32; ++c)
      if (c < cnt) w[c] = v[c];
  }
}
__device__ __forceinline__ void partial_add32(const float* w, int cnt, float (&v)[32]) {
  if (cnt == 32) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 t = __ldcg(reinterpret_cast<const float4*>(w + 4 * q));
      v[4 * q + 0] += t.x;
      v[4 * q + 1] += t.y;
      v[4 * q + 2] += t.z;
      v[4 * q + 3] += t.w;
    }
  } else {
#pragma unroll
    for (int c = 0; c < 32; ++c)
      if (c < cnt) v[c] += __ldcg(w + c);
  }
}

struct Unit {
  int m0, n0, tile, split, step0, nsteps;
};
__device__ __forceinline__ Unit decode_unit(const TcParams& p, int u, int bn) {
  Unit r;
  r.split = u % p.splits;
  r.tile = u / p.splits;
  r.m0 = (r.tile / p.tiles_n) * TBM;
  r.n0 = (r.tile % p.tiles_n) * bn;
  const int per = (p.steps_total + p.splits - 1) / p.splits;
  r.step0 = r.split * per;
  r.nsteps = max(0, min(p.steps_total, r.step0 + per) - r.step0);
  return r;
}

template <int KIND, int BN, int CPS, int KPS>
__global__ void __launch_bounds__(TC_THREADS, CPS)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcParams p) {
  using C = TcCfg<BN, CPS, KPS>;
  if (threadIdx.x == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
  }
  extern __shared__ unsigned char smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + C::STAGES * C::STAGE);
  uint64_t* full = bars;
  uint64_t* empty = bars + C::STAGES;
  uint64_t* tfull = bars + 2 * C::STAGES;   // [2]
  uint64_t* tempty = tfull + 2;             // [2]
  uint32_t* tmem_slot = (uint32_t*)(tempty + 2);
  __shared__ int s_abort;
  __shared__ int s_last;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&tfull[b]), 1);
      mbar_init(smem_u32(&tempty[b]), 128);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int ksh = KIND == TC_E4M3 ? 0 : 1;  // K elements per 128-byte row: 128 >> ksh
  // The prologue above overlaps the previous kernel (programmatic dependent
  // launch).  The A operand of every GEMM here is a constant factor, so the
  // producer also loads the A tiles of the first ring stages before waiting
  // for the previous kernel; everything else waits first.
  bool skip = false;
  if (warp == 0 && lane < 2 * KPS) {
    // ---------------- TMA producer: lane 2q loads the A tile, lane 2q + 1
    // the B tile of k-block q of the stage (all issued by one instruction);
    // lane 0 owns the barriers
    const bool isB = lane & 1;
    const int q = lane >> 1;
    const CUtensorMap* map = isB ? &tmB : &tmA;
    const int nk = p.batch_rows ? 1 : p.nkron;
    const unsigned mask = (1u << (2 * KPS)) - 1u;
    auto load = [&](const Unit& w, int j, int s, bool a_side) {
      // this lane's tile of stage j of unit w (A lanes when a_side, else B lanes)
      const int nkb = min(KPS, w.nsteps - j * KPS);
      if (q >= nkb || isB == a_side) return;
      const int tb = p.batch_rows ? w.m0 / p.batch_rows : 0;
      const int row0 = isB ? w.n0 : w.m0 - tb * p.batch_rows;
      const int stp = w.step0 + j * KPS + q;
      const int kb = stp % p.kblocks;
      const int rest = stp / p.kblocks;
      const int k = rest % nk, pr = rest / nk;
      const int term = (isB ? p.sb[pr] * p.b_terms : p.sa[pr] * p.a_terms) + (p.batch_rows ? tb : k);
      const uint32_t dst = smem_u32(smem + s * C::STAGE + q * C::KB_BYTES) + (isB ? (uint32_t)C::A_BYTES : 0u);
      tma_load_3d(dst, map, (kb * 128) >> ksh, row0, term, smem_u32(&full[s]));
    };
    // prefetch: the first ring stages of the first unit (fresh barriers, free slots)
    int npre = 0;
    Unit w0;
    if ((int)blockIdx.x < p.units) {
      w0 = decode_unit(p, blockIdx.x, BN);
      npre = min(C::STAGES, (w0.nsteps + KPS - 1) / KPS);
      for (int j = 0; j < npre; ++j) {
        if (lane == 0) mbar_expect_tx(smem_u32(&full[j]), (uint32_t)(min(KPS, w0.nsteps - j * KPS) * C::KB_BYTES));
        __syncwarp(mask);
        load(w0, j, j, true);
      }
    }
    KP_PDL_WAIT();
    KP_PDL_TRIGGER();
    skip = p.flags && *(volatile const int*)p.flags;
    // the B tiles of the prefetched stages (also when paused: the stages must fill before the CTA exits)
    for (int j = 0; j < npre; ++j) load(w0, j, j, false);
    if (skip) {
      if (lane == 0)
        for (int j = 0; j < npre; ++j) mbar_wait(smem_u32(&full[j]), 0, p.status);
    } else {
      int it = npre;
      bool run = true;
      for (int u = blockIdx.x; run && u < p.units && !*(volatile int*)&s_abort; u += gridDim.x) {
        const Unit w = decode_unit(p, u, BN);
        for (int j = u == (int)blockIdx.x ? npre : 0; j * KPS < w.nsteps; ++j, ++it) {
          const int s = it % C::STAGES;
          const uint32_t ph = (it / C::STAGES) & 1;
          const int nkb = min(KPS, w.nsteps - j * KPS);  // k-blocks in this stage
          int okw = 1;
          if (lane == 0) {
            okw = mbar_wait(smem_u32(&empty[s]), ph ^ 1, p.status) ? 1 : 0;
            if (okw) mbar_expect_tx(smem_u32(&full[s]), (uint32_t)(nkb * C::KB_BYTES));
          }
          okw = __shfl_sync(mask, okw, 0);
          if (!okw) {
            if (lane == 0) s_abort = 1;
            run = false;
            break;
          }
          load(w, j, s, true);
          load(w, j, s, false);
        }
      }
    }
  } else {
    KP_PDL_WAIT();
    KP_PDL_TRIGGER();
    skip = p.flags && *(volatile const int*)p.flags;
  }

  if (skip || warp == 0) {
    // paused, or the producer (done above): nothing more before the teardown
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      int it = 0, i = 0;
      for (int u = blockIdx.x; u < p.units; u += gridDim.x, ++i) {
        const Unit w = decode_unit(p, u, BN);
        const int buf = i & 1;
        if (*(volatile int*)&s_abort || !mbar_wait(smem_u32(&tempty[buf]), ((i >> 1) & 1) ^ 1, p.status)) {
          s_abort = 1;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * BN);
        bool ok = true;
        for (int j = 0; j * KPS < w.nsteps; ++j, ++it) {
          const int s = it % C::STAGES;
          const uint32_t ph = (it / C::STAGES) & 1;
          if (*(volatile int*)&s_abort || !mbar_wait(smem_u32(&full[s]), ph, p.status)) {
            s_abort = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          const int nkb = min(KPS, w.nsteps - j * KPS);
#pragma unroll
          for (int q = 0; q < KPS; ++q) {
            if (q < nkb) {
              const uint32_t a0 = smem_u32(smem + s * C::STAGE + q * C::KB_BYTES);
              const uint32_t b0 = a0 + C::A_BYTES;
#pragma unroll
              for (int kk = 0; kk < 4; ++kk)  // 4 x 32 bytes of K per 128-byte row
                mma_issue<KIND>(d, make_sdesc(a0 + kk * 32), make_sdesc(b0 + kk * 32), p.idesc,
                                (j > 0 || q > 0 || kk > 0) ? 1u : 0u);
            }
          }
          mma_commit(smem_u32(&empty[s]));
        }
        mma_commit(smem_u32(&tfull[buf]));
        if (!ok) break;
      }
    }
  } else {
    // ---------------- epilogue warps 2..5 -> TMEM lanes 32 * (warp % 4)
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const int etid = threadIdx.x - 64;
    const float sdev = p.alpha_dev ? *p.alpha_dev : 1.f;
    int i = 0;
    for (int u = blockIdx.x; u < p.units; u += gridDim.x, ++i) {
      const Unit w = decode_unit(p, u, BN);
      const int buf = i & 1;
      if (!mbar_wait(smem_u32(&tfull[buf]), (i >> 1) & 1, p.status)) break;
      tc_fence_after();
      const int gm = w.m0 + row;
      const bool row_ok = gm < p.M;
      float tmax = 0.f;
      if (p.splits == 1) {
#pragma unroll 1
        for (int chunk = 0; chunk < BN / 32; ++chunk) {
          float acc[32];
          if (w.nsteps > 0) {
            tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * BN + chunk * 32), acc);
          } else {
#pragma unroll
            for (int c = 0; c < 32; ++c) acc[c] = 0.f;
          }
          const int gn0 = w.n0 + chunk * 32;
          if (row_ok && gn0 < p.N) epi_store32(p.epi, sdev, gm, gn0, p.N, acc, tmax);
        }
        tc_fence_before();
        mbar_arrive(smem_u32(&tempty[buf]));
        if (p.epi.amax_bits) {  // one atomic per warp and unit
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) tmax = fmaxf(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
          if (lane == 0 && tmax > 0.f) atomicMax(p.epi.amax_bits, __float_as_uint(tmax));
        }
      } else {
        // split-K: FP32 partial, then the last split to arrive finishes the tile
#pragma unroll 1
        for (int chunk = 0; chunk < BN / 32; ++chunk) {
          float acc[32];
          if (w.nsteps > 0) {
            tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * BN + chunk * 32), acc);
          } else {
#pragma unroll
            for (int c = 0; c < 32; ++c) acc[c] = 0.f;
          }
          const int gn0 = w.n0 + chunk * 32;
          if (row_ok && gn0 < p.N)
            partial_store32(p.ws + ((long long)w.split * p.M + gm) * p.N + gn0, min(32, p.N - gn0), acc);
        }
        tc_fence_before();
        mbar_arrive(smem_u32(&tempty[buf]));
        __threadfence();
        epi_bar();
        if (etid == 0) {
          const unsigned int prev = atomicAdd(&p.counters[w.tile], 1u);
          s_last = (prev == (unsigned int)(p.splits - 1)) ? 1 : 0;
          if (s_last) p.counters[w.tile] = 0u;
        }
        epi_bar();
        if (s_last) {
          __threadfence();
          if (row_ok) {
#pragma unroll 1
            for (int chunk = 0; chunk < BN / 32; ++chunk) {
              const int gn0 = w.n0 + chunk * 32;
              if (gn0 >= p.N) break;
              const int cnt = min(32, p.N - gn0);
              float acc[32];
#pragma unroll
              for (int c = 0; c < 32; ++c) acc[c] = 0.f;
              for (int s = 0; s < p.splits; ++s) partial_add32(p.ws + ((long long)s * p.M + gm) * p.N + gn0, cnt, acc);
              epi_store32(p.epi, sdev, gm, gn0, p.N, acc, tmax);
            }
          }
          if (p.epi.amax_bits) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) tmax = fmaxf(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
            if (lane == 0 && tmax > 0.f) atomicMax(p.epi.amax_bits, __float_as_uint(tmax));
          }
        }
        epi_bar();  // s_last is reused by the next unit
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS) : "memory");
  }
}

// ------------------------------------------------------------- grouped kernel
// The GEMMs of several independent problems (one plan each: its own tensor
// maps, sizes and epilogue, all in global memory) as one persistent launch:
// the units of all plans are numbered consecutively (ustart[e] is the first
// unit of plan e) and the CTAs take them in turn, so small problems share the
// GPU instead of each filling it with a launch of its own.  A plan whose
// pause flag is set (its problem has stopped) contributes no work: every
// role reads the same flag, written before this launch, and skips its units.
// No split-K; the ring and accumulator phases run on across plans.
struct alignas(128) TcGroupEntry {  // the alignment of CUtensorMap
  CUtensorMap mapA, mapB;
  TcParams p;
};

__device__ __forceinline__ int group_find(const int* __restrict__ ustart, int nent, int u) {
  int lo = 0, hi = nent - 1;  // largest e with ustart[e] <= u
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (ustart[mid] <= u) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int KIND, int BN, int CPS, int KPS>
__global__ void __launch_bounds__(TC_THREADS, CPS)
    tc_gemm_group_kernel(const TcGroupEntry* __restrict__ ents, const int* __restrict__ ustart, int nent,
                         int* status) {
  using C = TcCfg<BN, CPS, KPS>;
  extern __shared__ unsigned char smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + C::STAGES * C::STAGE);
  uint64_t* full = bars;
  uint64_t* empty = bars + C::STAGES;
  uint64_t* tfull = bars + 2 * C::STAGES;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_slot = (uint32_t*)(tempty + 2);
  __shared__ int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&tfull[b]), 1);
      mbar_init(smem_u32(&tempty[b]), 128);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int ksh = KIND == TC_E4M3 ? 0 : 1;
  KP_PDL_WAIT();
  KP_PDL_TRIGGER();
  const int units = ustart[nent];
  // plan of unit u and the unit's index within it; false: the plan is paused
  auto unit_of = [&](int u, const TcGroupEntry*& e, Unit& w) -> bool {
    const int k = group_find(ustart, nent, u);
    e = ents + k;
    if (e->p.flags && *(volatile const int*)e->p.flags) return false;
    w = decode_unit(e->p, u - ustart[k], BN);
    return true;
  };
  if (warp == 0 && lane < 2 * KPS) {
    // ---------------- TMA producer (lanes as in tc_gemm_kernel)
    const bool isB = lane & 1;
    const int q = lane >> 1;
    const unsigned mask = (1u << (2 * KPS)) - 1u;
    int it = 0;
    bool run = true;
    for (int u = blockIdx.x; run && u < units && !*(volatile int*)&s_abort; u += gridDim.x) {
      const TcGroupEntry* e;
      Unit w;
      if (!unit_of(u, e, w)) continue;
      const TcParams& p = e->p;
      const CUtensorMap* map = isB ? &e->mapB : &e->mapA;
      const int nk = p.batch_rows ? 1 : p.nkron;
      for (int j = 0; j * KPS < w.nsteps; ++j, ++it) {
        const int s = it % C::STAGES;
        const uint32_t ph = (it / C::STAGES) & 1;
        const int nkb = min(KPS, w.nsteps - j * KPS);
        int okw = 1;
        if (lane == 0) {
          okw = mbar_wait(smem_u32(&empty[s]), ph ^ 1, status) ? 1 : 0;
          if (okw) mbar_expect_tx(smem_u32(&full[s]), (uint32_t)(nkb * C::KB_BYTES));
        }
        okw = __shfl_sync(mask, okw, 0);
        if (!okw) {
          if (lane == 0) s_abort = 1;
          run = false;
          break;
        }
        if (q < nkb) {
          const int tb = p.batch_rows ? w.m0 / p.batch_rows : 0;
          const int row0 = isB ? w.n0 : w.m0 - tb * p.batch_rows;
          const int stp = w.step0 + j * KPS + q;
          const int kb = stp % p.kblocks;
          const int rest = stp / p.kblocks;
          const int k = rest % nk, pr = rest / nk;
          const int term = (isB ? p.sb[pr] * p.b_terms : p.sa[pr] * p.a_terms) + (p.batch_rows ? tb : k);
          const uint32_t dst =
              smem_u32(smem + s * C::STAGE + q * C::KB_BYTES) + (isB ? (uint32_t)C::A_BYTES : 0u);
          tma_load_3d(dst, map, (kb * 128) >> ksh, row0, term, smem_u32(&full[s]));
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      int it = 0, i = 0;
      for (int u = blockIdx.x; u < units; u += gridDim.x) {
        const TcGroupEntry* e;
        Unit w;
        if (!unit_of(u, e, w)) continue;
        const uint32_t idesc = e->p.idesc;
        const int buf = i & 1;
        if (*(volatile int*)&s_abort || !mbar_wait(smem_u32(&tempty[buf]), ((i >> 1) & 1) ^ 1, status)) {
          s_abort = 1;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * BN);
        bool ok = true;
        for (int j = 0; j * KPS < w.nsteps; ++j, ++it) {
          const int s = it % C::STAGES;
          const uint32_t ph = (it / C::STAGES) & 1;
          if (*(volatile int*)&s_abort || !mbar_wait(smem_u32(&full[s]), ph, status)) {
            s_abort = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          const int nkb = min(KPS, w.nsteps - j * KPS);
#pragma unroll
          for (int q = 0; q < KPS; ++q) {
            if (q < nkb) {
              const uint32_t a0 = smem_u32(smem + s * C::STAGE + q * C::KB_BYTES);
              const uint32_t b0 = a0 + C::A_BYTES;
#pragma unroll
              for (int kk = 0; kk < 4; ++kk)
                mma_issue<KIND>(d, make_sdesc(a0 + kk * 32), make_sdesc(b0 + kk * 32), idesc,
                                (j > 0 || q > 0 || kk > 0) ? 1u : 0u);
            }
          }
          mma_commit(smem_u32(&empty[s]));
        }
        mma_commit(smem_u32(&tfull[buf]));
        ++i;
        if (!ok) break;
      }
    }
  } else if (warp >= 2) {
    // ---------------- epilogue warps 2..5 -> TMEM lanes 32 * (warp % 4)
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    int i = 0;
    for (int u = blockIdx.x; u < units; u += gridDim.x) {
      const TcGroupEntry* e;
      Unit w;
      if (!unit_of(u, e, w)) continue;
      const TcParams& p = e->p;
      const int buf = i & 1;
      if (!mbar_wait(smem_u32(&tfull[buf]), (i >> 1) & 1, status)) break;
      ++i;
      tc_fence_after();
      const float sdev = p.alpha_dev ? *p.alpha_dev : 1.f;
      const int gm = w.m0 + row;
      const bool row_ok = gm < p.M;
      float tmax = 0.f;
#pragma unroll 1
      for (int chunk = 0; chunk < BN / 32; ++chunk) {
        float acc[32];
        if (w.nsteps > 0) {
          tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * BN + chunk * 32), acc);
        } else {
#pragma unroll
          for (int c = 0; c < 32; ++c) acc[c] = 0.f;
        }
        const int gn0 = w.n0 + chunk * 32;
        if (row_ok && gn0 < p.N) epi_store32(p.epi, sdev, gm, gn0, p.N, acc, tmax);
      }
      tc_fence_before();
      mbar_arrive(smem_u32(&tempty[buf]));
      if (p.epi.amax_bits) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tmax = fmaxf(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
        if (lane == 0 && tmax > 0.f) atomicMax(p.epi.amax_bits, __float_as_uint(tmax));
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS) : "memory");
  }
}

// ------------------------------------------------------------- CTA-pair kernel
// The same GEMM on 256 x 256 output tiles computed by a pair of CTAs on two
// SMs (a cluster of 2) with tcgen05.mma.cta_group::2: the MMA of M = 256,
// N = 256 reads 128 rows of A and 128 rows of B from each CTA's shared
// memory and leaves 128 rows x 256 columns of the accumulator in each CTA's
// TMEM.  Each SM then stages 32 KB per 64-wide k-block for 256 x 128 x 64
// MACs of its own accumulator rows, two thirds of the 48 KB a one-CTA
// 128 x 256 tile needs for the same work; the L2 -> shared-memory stream
// is what limits the one-CTA tiles here.
//   rank 0 (leader): lane 0 of warp 0 arms the stage's full barrier with the
//     bytes of both CTAs' loads; lane 0 of warp 1 issues the MMAs and commits
//     them to both CTAs' empty / accumulator-full barriers (multicast)
//   both ranks: warp 0 loads this CTA's halves of A and B (TMA, completion
//     counted on the leader's full barrier); warps 2..5 read this CTA's TMEM
//     rows and arrive on the leader's accumulator-empty barrier
// Every wait is bounded by a time limit; all paths end at a cluster barrier
// before TMEM is freed, so neither CTA leaves while the other may still
// signal its barriers.
constexpr int PAIR_M = 256, PAIR_N = 256;
constexpr unsigned long long KP_WAIT_NS = 500000000ull;  // 0.5 s per wait

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t peer_addr(uint32_t local_shared, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local_shared), "r"(rank));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// wait bounded by a time limit; false (and the status word flagged) on give-up
__device__ __forceinline__ bool mbar_wait_t(uint32_t bar, uint32_t parity, int* status) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned int i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63u) == 0u && global_ns() - t0 > KP_WAIT_NS) {
      atomicOr(status, DEV_ERR_TIMEOUT);
      return false;
    }
  }
}
__device__ __forceinline__ void tma_load_3d_pair(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                                 uint32_t leader_bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
      "%4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(leader_bar)
      : "memory");
}
template <int KIND>
__device__ __forceinline__ void mma_issue_pair(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                               uint32_t accum) {
  if constexpr (KIND == TC_E4M3) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
  }
}
// arrive (once) on the barrier at this address in both CTAs of the pair when
// the MMAs issued so far have completed
__device__ __forceinline__ void mma_commit_pair(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
      "h"((unsigned short)3)
      : "memory");
}

template <int KPS>
struct PairCfg {
  static constexpr int A_BYTES = 128 * 128;  // this CTA's 128 rows of A, one 128-byte k-block row each
  static constexpr int B_BYTES = 128 * 128;  // this CTA's 128 rows (of 256) of B
  static constexpr int KB_BYTES = A_BYTES + B_BYTES;
  static constexpr int STAGE = KPS * KB_BYTES;
  static constexpr int STAGES = 196608 / STAGE;
  static constexpr int SMEM = STAGES * STAGE + 1024 + 512;
  static constexpr int TMEM_COLS = 2 * PAIR_N;
  static_assert(STAGES >= 2, "ring too shallow");
};

struct PairUnit {
  int m0, n0;
};
__device__ __forceinline__ PairUnit decode_pair(const TcParams& p, int u) {
  PairUnit r;
  r.m0 = (u / p.tiles_n) * PAIR_M;
  r.n0 = (u % p.tiles_n) * PAIR_N;
  return r;
}

template <int KIND, int KPS>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(TC_THREADS, 1)
    tc_gemm_pair_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcParams p) {
  using C = PairCfg<KPS>;
  if (threadIdx.x == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
  }
  extern __shared__ unsigned char smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + C::STAGES * C::STAGE);
  uint64_t* full = bars;
  uint64_t* empty = bars + C::STAGES;
  uint64_t* tfull = bars + 2 * C::STAGES;  // [2]
  uint64_t* tempty = tfull + 2;            // [2]
  uint32_t* tmem_slot = (uint32_t*)(tempty + 2);
  __shared__ int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const int cl = blockIdx.x >> 1, ncl = gridDim.x >> 1;
  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&tfull[b]), 1);
      mbar_init(smem_u32(&tempty[b]), 8);  // 4 epilogue warps in each CTA (the leader's is used)
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // barriers of both CTAs initialised before any remote signal
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int ksh = KIND == TC_E4M3 ? 0 : 1;
  const int nk = p.batch_rows ? 1 : p.nkron;
  bool skip = false;
  if (warp == 0 && lane < 2 * KPS) {
    // ---------------- TMA producer of this CTA's halves
    const bool isB = lane & 1;
    const int q = lane >> 1;
    const CUtensorMap* map = isB ? &tmB : &tmA;
    const unsigned mask = (1u << (2 * KPS)) - 1u;
    auto load = [&](const PairUnit& w, int j, int s, bool a_side) {
      const int nkb = min(KPS, p.steps_total - j * KPS);
      if (q >= nkb || isB == a_side) return;
      const int tb = p.batch_rows ? w.m0 / p.batch_rows : 0;
      const int row0 = isB ? w.n0 + 128 * (int)rank : w.m0 + 128 * (int)rank - tb * p.batch_rows;
      const int stp = j * KPS + q;
      const int kb = stp % p.kblocks;
      const int rest = stp / p.kblocks;
      const int k = rest % nk, pr = rest / nk;
      const int term = (isB ? p.sb[pr] * p.b_terms : p.sa[pr] * p.a_terms) + (p.batch_rows ? tb : k);
      const uint32_t dst = smem_u32(smem + s * C::STAGE + q * C::KB_BYTES) + (isB ? (uint32_t)C::A_BYTES : 0u);
      tma_load_3d_pair(dst, map, (kb * 128) >> ksh, row0, term, peer_addr(smem_u32(&full[s]), 0));
    };
    auto arm = [&](int j, int s) {  // leader: both CTAs' bytes of stage j
      const int nkb = min(KPS, p.steps_total - j * KPS);
      mbar_expect_tx(smem_u32(&full[s]), (uint32_t)(2 * nkb * C::KB_BYTES));
    };
    int npre = 0;
    PairUnit w0;
    const int nstages = (p.steps_total + KPS - 1) / KPS;
    if (cl < p.units) {
      w0 = decode_pair(p, cl);
      npre = min(C::STAGES, nstages);
      for (int j = 0; j < npre; ++j) {
        if (leader && lane == 0) arm(j, j);
        __syncwarp(mask);
        load(w0, j, j, true);
      }
    }
    KP_PDL_WAIT();
    KP_PDL_TRIGGER();
    skip = p.flags && *(volatile const int*)p.flags;
    for (int j = 0; j < npre; ++j) load(w0, j, j, false);
    if (skip) {
      if (leader && lane == 0)  // every prefetched stage lands before the pair leaves
        for (int j = 0; j < npre; ++j) mbar_wait_t(smem_u32(&full[j]), 0, p.status);
    } else {
      int it = npre;
      bool run = true;
      for (int u = cl; run && u < p.units && !*(volatile int*)&s_abort; u += ncl) {
        const PairUnit w = decode_pair(p, u);
        for (int j = u == cl ? npre : 0; j < nstages; ++j, ++it) {
          const int s = it % C::STAGES;
          const uint32_t ph = (it / C::STAGES) & 1;
          int okw = 1;
          if (lane == 0) {
            okw = mbar_wait_t(smem_u32(&empty[s]), ph ^ 1, p.status) ? 1 : 0;
            if (okw && leader) arm(j, s);
          }
          okw = __shfl_sync(mask, okw, 0);
          if (!okw) {
            if (lane == 0) s_abort = 1;
            run = false;
            break;
          }
          load(w, j, s, true);
          load(w, j, s, false);
        }
      }
    }
  } else {
    KP_PDL_WAIT();
    KP_PDL_TRIGGER();
    skip = p.flags && *(volatile const int*)p.flags;
  }

  if (skip || warp == 0) {
  } else if (warp == 1) {
    if (leader && lane == 0) {
      // ---------------- MMA issuer (leader CTA only)
      const int nstages = (p.steps_total + KPS - 1) / KPS;
      int it = 0, i = 0;
      for (int u = cl; u < p.units; u += ncl, ++i) {
        const int buf = i & 1;
        if (*(volatile int*)&s_abort || !mbar_wait_t(smem_u32(&tempty[buf]), ((i >> 1) & 1) ^ 1, p.status)) {
          s_abort = 1;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * PAIR_N);
        bool ok = true;
        for (int j = 0; j < nstages; ++j, ++it) {
          const int s = it % C::STAGES;
          const uint32_t ph = (it / C::STAGES) & 1;
          if (*(volatile int*)&s_abort || !mbar_wait_t(smem_u32(&full[s]), ph, p.status)) {
            s_abort = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          const int nkb = min(KPS, p.steps_total - j * KPS);
#pragma unroll
          for (int q = 0; q < KPS; ++q) {
            if (q < nkb) {
              const uint32_t a0 = smem_u32(smem + s * C::STAGE + q * C::KB_BYTES);
              const uint32_t b0 = a0 + C::A_BYTES;
#pragma unroll
              for (int kk = 0; kk < 4; ++kk)
                mma_issue_pair<KIND>(d, make_sdesc(a0 + kk * 32), make_sdesc(b0 + kk * 32), p.idesc,
                                     (j > 0 || q > 0 || kk > 0) ? 1u : 0u);
            }
          }
          mma_commit_pair(smem_u32(&empty[s]));
        }
        mma_commit_pair(smem_u32(&tfull[buf]));
        if (!ok) break;
      }
    }
  } else {
    // ---------------- epilogue warps 2..5: this CTA's 128 accumulator rows
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const float sdev = p.alpha_dev ? *p.alpha_dev : 1.f;
    int i = 0;
    for (int u = cl; u < p.units; u += ncl, ++i) {
      const PairUnit w = decode_pair(p, u);
      const int buf = i & 1;
      if (!mbar_wait_t(smem_u32(&tfull[buf]), (i >> 1) & 1, p.status)) break;
      tc_fence_after();
      const int gm = w.m0 + 128 * (int)rank + row;
      const bool row_ok = gm < p.M;
      float tmax = 0.f;
#pragma unroll 1
      for (int chunk = 0; chunk < PAIR_N / 32; ++chunk) {
        float acc[32];
        tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * PAIR_N + chunk * 32), acc);
        const int gn0 = w.n0 + chunk * 32;
        if (row_ok && gn0 < p.N) epi_store32(p.epi, sdev, gm, gn0, p.N, acc, tmax);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_remote(peer_addr(smem_u32(&tempty[buf]), 0));
      if (p.epi.amax_bits) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tmax = fmaxf(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
        if (lane == 0 && tmax > 0.f) atomicMax(p.epi.amax_bits, __float_as_uint(tmax));
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // both CTAs are done with TMEM and with each other's barriers
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS) : "memory");
  }
}

// ------------------------------------------------------------- K-concatenated products
// A product summed over many k-blocks (the operator's sum over Kronecker
// terms as ONE GEMM over the concatenated K of all terms, the terms summed in
// the TMEM accumulator) on narrow 128 x 64 tiles, so that a 1024 x 1024
// output still gives one tile per SM, and without per-term outputs.  The
// epilogue can also reduce sum(out * aux) (double-float) and max |out| over
// the whole output, finished by the last CTA to arrive (for the operator's
// last GEMM: p^T q, max |q| and the alpha step).
// With CL = 4 the CTAs form clusters of four along N: they compute
// neighbouring tiles of the same 128 output rows, so they read the same A
// tile at every k-block, and each loads one quarter of its rows (32) and
// multicasts it to the whole cluster (12 KiB instead of 24 KiB from L2 per
// CTA and k-block).  A ring slot is then refilled only after the MMAs of
// every CTA of the cluster have read it: each CTA's MMA thread commits its
// reads to that slot's empty barrier in all of them (count CL).  A CTA's
// full barrier counts the bytes landing in its own shared memory (its B tile
// and the slices of A), armed by its own producer; slices from the other
// CTAs may land before it is armed (the barrier's pending arrival keeps the
// phase open until then).
//   warp 0      TMA producer (lanes 2q / 2q + 1: A (slice) / B tile of k-block q)
//   warp 1      TMEM allocation + MMA issuer (one thread)
//   warps 2..5  epilogue; optionally the dot reduction of the output
// Every wait is bounded; the producer waits, before the CTA leaves, until the
// cluster has read every slot it filled, and all CTAs end at a cluster
// barrier, so no CTA leaves while another may still write its shared memory.
constexpr int KC_BN = 64;

template <int KPS, int CL>
struct KcCfg {
  static constexpr int A_BYTES = TBM * 128;     // the whole A tile of a k-block (CL slices)
  static constexpr int A_SLICE = A_BYTES / CL;  // the rows one CTA of the cluster loads
  static constexpr int B_BYTES = KC_BN * 128;
  static constexpr int KB_BYTES = A_BYTES + B_BYTES;
  static constexpr int STAGE = KPS * KB_BYTES;
  static constexpr int STAGES = 196608 / STAGE;
  static constexpr int SMEM = STAGES * STAGE + 1024 + 512;
  static constexpr int TMEM_COLS = 2 * KC_BN;
  static_assert(STAGES >= 2, "ring too shallow");
  static_assert(A_SLICE % 1024 == 0, "A slices must keep the 1024-byte swizzle atoms");
};

__device__ __forceinline__ void tma_load_3d_mc(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                               uint32_t bar, uint16_t cta_mask) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster [%0], [%1, {%2, "
      "%3, %4}], [%5], %6;" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar), "h"(cta_mask)
      : "memory");
}
// arrive (once) on the barrier at this offset in every CTA of the mask when
// the MMAs issued so far have completed
__device__ __forceinline__ void mma_commit_mc(uint32_t bar, uint16_t cta_mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
      "h"(cta_mask)
      : "memory");
}

struct KcUnit {
  int m0, n0;
};
// unit u = one cluster's CL neighbouring tiles of a 128-row block
template <int CL>
__device__ __forceinline__ KcUnit decode_kc(const TcParams& p, int u, int rank) {
  const int groups_n = p.tiles_n / CL;
  KcUnit r;
  r.m0 = (u / groups_n) * TBM;
  r.n0 = ((u % groups_n) * CL + rank) * KC_BN;
  return r;
}

// sum(out * aux) and max |out| of one stored 32-column row segment (out: the
// values epi_store32 wrote, in v)
__device__ __forceinline__ void kc_dot_segment(const EpiParams& e, int gm, int gn0, int N, const float (&v)[32],
                                               float& dh, float& dl, float& mx) {
  const int cnt = min(32, N - gn0);
  const float* aux = (const float*)e.aux + (long long)gm * e.ld_aux + gn0;
  if (cnt == 32 && ((reinterpret_cast<uintptr_t>(aux) & 15) == 0)) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 t = *reinterpret_cast<const float4*>(aux + 4 * q);
      kpv::df_add_prod(dh, dl, v[4 * q + 0], t.x);
      kpv::df_add_prod(dh, dl, v[4 * q + 1], t.y);
      kpv::df_add_prod(dh, dl, v[4 * q + 2], t.z);
      kpv::df_add_prod(dh, dl, v[4 * q + 3], t.w);
    }
#pragma unroll
    for (int c = 0; c < 32; ++c) mx = fmaxf(mx, fabsf(v[c]));
  } else {
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      if (c < cnt) {
        kpv::df_add_prod(dh, dl, v[c], aux[c]);
        mx = fmaxf(mx, fabsf(v[c]));
      }
    }
  }
}

// the epilogue warps' (128 threads, named barrier 1) double-float sum and max:
// within the warp, then over the four warps in a fixed order
__device__ __forceinline__ void kc_epi_reduce(float& h, float& l, float& mx, float2 (*red)[2], int quarter,
                                              int lane) {
  kpv::df_warp_sum(h, l);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) {
    red[quarter][0] = make_float2(h, l);
    red[quarter][1] = make_float2(mx, 0.f);
  }
  epi_bar();
  h = 0.f;
  l = 0.f;
  mx = 0.f;
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    l += red[w][0].y;
    kpv::df_add(h, l, red[w][0].x);
    mx = fmaxf(mx, red[w][1].x);
  }
  epi_bar();  // red is read by every thread before it is written again
}

template <int KIND, int KPS, int CL>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(TC_THREADS, 1)
    tc_gemm_kcat_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcParams p) {
  using C = KcCfg<KPS, CL>;
  if (threadIdx.x == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
  }
  extern __shared__ unsigned char smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + C::STAGES * C::STAGE);
  uint64_t* full = bars;
  uint64_t* empty = bars + C::STAGES;
  uint64_t* tfull = bars + 2 * C::STAGES;  // [2]
  uint64_t* tempty = tfull + 2;            // [2]
  uint32_t* tmem_slot = (uint32_t*)(tempty + 2);
  __shared__ int s_abort;
  __shared__ int s_last;
  __shared__ float2 s_red[4][2];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rank = (int)cluster_rank();
  const int cl = blockIdx.x / CL, ncl = gridDim.x / CL;
  const uint16_t all = (uint16_t)((1u << CL) - 1u);
  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), CL);  // the MMA threads of the whole cluster
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&tfull[b]), 1);
      mbar_init(smem_u32(&tempty[b]), 128);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // every CTA's barriers initialised before any multicast reaches them
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int ksh = KIND == TC_E4M3 ? 0 : 1;
  const int nk = p.nkron;
  const int nstages = (p.steps_total + KPS - 1) / KPS;
  bool skip = false;
  if (warp == 0 && lane < 2 * KPS) {
    // ---------------- TMA producer
    const bool isB = lane & 1;
    const int q = lane >> 1;
    const CUtensorMap* map = isB ? &tmB : &tmA;
    const unsigned mask = (1u << (2 * KPS)) - 1u;
    auto load = [&](const KcUnit& w, int j, int s, bool a_side) {
      const int nkb = min(KPS, p.steps_total - j * KPS);
      if (q >= nkb || isB == a_side) return;
      const int stp = j * KPS + q;
      const int kb = stp % p.kblocks;
      const int rest = stp / p.kblocks;
      const int k = rest % nk, pr = rest / nk;
      const int term = (isB ? p.sb[pr] * p.b_terms : p.sa[pr] * p.a_terms) + k;
      const uint32_t kbase = smem_u32(smem + s * C::STAGE + q * C::KB_BYTES);
      if (isB)
        tma_load_3d(kbase + (uint32_t)C::A_BYTES, map, (kb * 128) >> ksh, w.n0, term, smem_u32(&full[s]));
      else if constexpr (CL == 1)
        tma_load_3d(kbase, map, (kb * 128) >> ksh, w.m0, term, smem_u32(&full[s]));
      else
        tma_load_3d_mc(kbase + (uint32_t)(rank * C::A_SLICE), map, (kb * 128) >> ksh, w.m0 + (TBM / CL) * rank, term,
                       smem_u32(&full[s]), all);
    };
    auto arm = [&](int j, int s) {
      const int nkb = min(KPS, p.steps_total - j * KPS);
      mbar_expect_tx(smem_u32(&full[s]), (uint32_t)(nkb * C::KB_BYTES));
    };
    // prefetch: the A slices (a constant factor) of the first ring stages
    // before waiting for the previous kernel
    int npre = 0;
    KcUnit w0;
    if (cl < p.units) {
      w0 = decode_kc<CL>(p, cl, rank);
      npre = min(C::STAGES, nstages);
      for (int j = 0; j < npre; ++j) {
        if (lane == 0) arm(j, j);
        __syncwarp(mask);
        load(w0, j, j, true);
      }
    }
    KP_PDL_WAIT();
    KP_PDL_TRIGGER();
    skip = p.flags && *(volatile const int*)p.flags;
    for (int j = 0; j < npre; ++j) load(w0, j, j, false);
    if (skip) {
      if (lane == 0)  // every prefetched stage (all CTAs' slices) lands before the CTA leaves
        for (int j = 0; j < npre; ++j) mbar_wait_t(smem_u32(&full[j]), 0, p.status);
    } else {
      int it = npre;
      bool run = true;
      for (int u = cl; run && u < p.units && !*(volatile int*)&s_abort; u += ncl) {
        const KcUnit w = decode_kc<CL>(p, u, rank);
        for (int j = u == cl ? npre : 0; j < nstages; ++j, ++it) {
          const int s = it % C::STAGES;
          const uint32_t ph = (it / C::STAGES) & 1;
          int okw = 1;
          if (lane == 0) {
            okw = mbar_wait_t(smem_u32(&empty[s]), ph ^ 1, p.status) ? 1 : 0;
            if (okw) arm(j, s);
          }
          okw = __shfl_sync(mask, okw, 0);
          if (!okw) {
            if (lane == 0) s_abort = 1;
            run = false;
            break;
          }
          load(w, j, s, true);
          load(w, j, s, false);
        }
      }
      // tail: the whole cluster has read every slot this CTA filled (their
      // commits to this CTA's empty barriers have landed)
      if (run && lane == 0) {
        for (int t = it; t < it + C::STAGES; ++t)
          if (!mbar_wait_t(smem_u32(&empty[t % C::STAGES]), ((t / C::STAGES) & 1) ^ 1, p.status)) break;
      }
    }
  } else {
    KP_PDL_WAIT();
    KP_PDL_TRIGGER();
    skip = p.flags && *(volatile const int*)p.flags;
  }

  if (skip || warp == 0) {
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      int it = 0, i = 0;
      for (int u = cl; u < p.units; u += ncl, ++i) {
        const int buf = i & 1;
        if (*(volatile int*)&s_abort || !mbar_wait_t(smem_u32(&tempty[buf]), ((i >> 1) & 1) ^ 1, p.status)) {
          s_abort = 1;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * KC_BN);
        bool ok = true;
        for (int j = 0; j < nstages; ++j, ++it) {
          const int s = it % C::STAGES;
          const uint32_t ph = (it / C::STAGES) & 1;
          if (*(volatile int*)&s_abort || !mbar_wait_t(smem_u32(&full[s]), ph, p.status)) {
            s_abort = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          const int nkb = min(KPS, p.steps_total - j * KPS);
#pragma unroll
          for (int q = 0; q < KPS; ++q) {
            if (q < nkb) {
              const uint32_t a0 = smem_u32(smem + s * C::STAGE + q * C::KB_BYTES);
              const uint32_t b0 = a0 + C::A_BYTES;
#pragma unroll
              for (int kk = 0; kk < 4; ++kk)
                mma_issue<KIND>(d, make_sdesc(a0 + kk * 32), make_sdesc(b0 + kk * 32), p.idesc,
                                (j > 0 || q > 0 || kk > 0) ? 1u : 0u);
            }
          }
          if constexpr (CL == 1)
            mma_commit(smem_u32(&empty[s]));
          else
            mma_commit_mc(smem_u32(&empty[s]), all);
        }
        mma_commit(smem_u32(&tfull[buf]));
        if (!ok) break;
      }
    }
  } else {
    // ---------------- epilogue warps 2..5 -> TMEM lanes 32 * (warp % 4)
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const int etid = threadIdx.x - 64;
    const float sdev = p.alpha_dev ? *p.alpha_dev : 1.f;
    const bool dot = p.dot_out != nullptr;
    float dh = 0.f, dl = 0.f, dmx = 0.f;
    int i = 0;
    for (int u = cl; u < p.units; u += ncl, ++i) {
      const KcUnit w = decode_kc<CL>(p, u, rank);
      const int buf = i & 1;
      if (!mbar_wait_t(smem_u32(&tfull[buf]), (i >> 1) & 1, p.status)) break;
      tc_fence_after();
      const int gm = w.m0 + row;
      const bool row_ok = gm < p.M;
      float tmax = 0.f;
#pragma unroll 1
      for (int chunk = 0; chunk < KC_BN / 32; ++chunk) {
        float acc[32];
        tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * KC_BN + chunk * 32), acc);
        const int gn0 = w.n0 + chunk * 32;
        if (row_ok && gn0 < p.N) {
          epi_store32(p.epi, sdev, gm, gn0, p.N, acc, tmax);
          if (dot) kc_dot_segment(p.epi, gm, gn0, p.N, acc, dh, dl, dmx);
        }
      }
      tc_fence_before();
      mbar_arrive(smem_u32(&tempty[buf]));
      if (p.epi.amax_bits) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tmax = fmaxf(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
        if (lane == 0 && tmax > 0.f) atomicMax(p.epi.amax_bits, __float_as_uint(tmax));
      }
    }
    if (dot) {
      // this CTA's sums, then the last CTA to arrive adds all CTAs' in order
      kc_epi_reduce(dh, dl, dmx, s_red, quarter, lane);
      float2* pp = reinterpret_cast<float2*>(p.dot_part);
      if (etid == 0) {
        pp[2 * blockIdx.x] = make_float2(dh, dl);
        pp[2 * blockIdx.x + 1] = make_float2(dmx, 0.f);
        __threadfence();
        s_last = atomicAdd(p.dot_count, 1u) == gridDim.x - 1 ? 1 : 0;
      }
      epi_bar();
      if (s_last) {
        __threadfence();
        dh = dl = dmx = 0.f;
        for (int b = etid; b < (int)gridDim.x; b += 128) {
          const float2 t = __ldcg(pp + 2 * b);
          dl += t.y;
          kpv::df_add(dh, dl, t.x);
          dmx = fmaxf(dmx, __ldcg(pp + 2 * b + 1).x);
        }
        kc_epi_reduce(dh, dl, dmx, s_red, quarter, lane);
        if (etid == 0) {
          double fin[2] = {(double)dh + (double)dl, (double)dmx};
          p.dot_out[0] = fin[0];
          if (p.dot_qmax) p.dot_out[1] = fin[1];
          *p.dot_count = 0u;
          if (p.dot_po.kind != POST_NONE) kpv::run_post(p.dot_po, fin);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // no CTA leaves while another may still signal or fill it
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS) : "memory");
  }
}

}  // namespace

// ------------------------------------------------------------- host side
struct TcGemmPlan {
  CUtensorMap mapA, mapB;
  TcParams params;
  int kind;
  int bn;
  int cps;
  int kps;
  bool pair;  // 256 x 256 tiles on CTA pairs (tc_gemm_pair_kernel)
  int kcat;   // > 0: K-concatenated product on tc_gemm_kcat_kernel, clusters of this many CTAs
  dim3 grid;
};

static CUtensorMapDataType tc_dtype(int kind) {
  return kind == TC_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                         : (kind == TC_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8);
}

// cuTensorMapEncodeTiled through the runtime's driver entry-point query, so
// that the library has no link-time dependency on libcuda
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

static kp_status make_map(CUtensorMap* map, const GemmOp& op, int kind, int box_rows) {
  const int esize = kind == TC_E4M3 ? 1 : 2;
  const int bk = 128 / esize;
  cuuint64_t dims[3] = {(cuuint64_t)op.K, (cuuint64_t)op.rows, (cuuint64_t)(op.nterm_idx > 0 ? op.nterm_idx : 1)};
  cuuint64_t strides[2] = {(cuuint64_t)(op.ld * esize), (cuuint64_t)(op.tstride * esize)};
  cuuint32_t box[3] = {(cuuint32_t)bk, (cuuint32_t)box_rows, 1u};
  cuuint32_t estr[3] = {1, 1, 1};
  if (((uintptr_t)op.ptr & 15) || (strides[0] & 15) || (strides[1] & 15)) {
    kp_set_error("tensor map: base or strides not 16-byte aligned (ld=%lld ts=%lld)", op.ld, op.tstride);
    return KP_EINVAL;
  }
  if (dims[2] == 1) strides[1] = strides[0] * dims[1];
  auto enc = encode_fn();
  if (!enc) {
    kp_set_error("cuTensorMapEncodeTiled is not available from the driver");
    return KP_ENOTSUP;
  }
  CUresult r = enc(map, tc_dtype(kind), 3, const_cast<void*>(op.ptr), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    kp_set_error("cuTensorMapEncodeTiled failed with CUresult %d", (int)r);
    return KP_ECUDA;
  }
  return KP_OK;
}

static uint32_t make_idesc(int kind, int bn, int bm) {
  uint32_t d = 0;
  d |= 1u << 4;  // D format F32
  if (kind == TC_BF16) {
    d |= 1u << 7;   // A BF16
    d |= 1u << 10;  // B BF16
  }                 // F16 / E4M3: format code 0
  // K-major A and B (bits 15, 16 = 0)
  d |= (uint32_t)(bn >> 3) << 17;
  d |= (uint32_t)(bm >> 4) << 24;
  return d;
}

bool tc_device_supported(kp_ctx* ctx) {
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, ctx->device);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, ctx->device);
  return major == 10 && minor == 3;
}

// clusters of the K-concatenated kernel that fit on the GPU at once (0: none
// or unknown, then the plan does not use the kernel)
template <int KPS, int CL>
static int kcat_max_clusters(kp_ctx* ctx) {
  static std::atomic<int> cached{-1};
  int v = cached.load();
  if (v >= 0) return v;
  using C = KcCfg<KPS, CL>;
  v = 0;
  if (cudaFuncSetAttribute(tc_gemm_kcat_kernel<TC_BF16, KPS, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           C::SMEM) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL * std::max(1, ctx->sm_count / CL), 1, 1);
    cfg.blockDim = dim3(TC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = ctx->stream;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, tc_gemm_kcat_kernel<TC_BF16, KPS, CL>, &cfg) == cudaSuccess) v = n;
  }
  cudaGetLastError();
  cached = v;
  return v;
}
static int kcat_clusters(kp_ctx* ctx, int kps, int cl) {
  if (cl == 4) return kps == 4 ? kcat_max_clusters<4, 4>(ctx) : (kps == 2 ? kcat_max_clusters<2, 4>(ctx) : kcat_max_clusters<1, 4>(ctx));
  return kps == 4 ? kcat_max_clusters<4, 1>(ctx) : (kps == 2 ? kcat_max_clusters<2, 1>(ctx) : kcat_max_clusters<1, 1>(ctx));
}

static kp_status tc_plan_create_one(kp_ctx* ctx, const GemmDesc& g, int kind, int splits, TcGemmPlan** out) {
  if (g.npairs < 1 || g.npairs > KP_MAX_PAIRS || g.nkron < 1) {
    kp_set_error("tc_plan_create: bad term description");
    return KP_EINVAL;
  }
  const int esize = kind == TC_E4M3 ? 1 : 2;
  if ((g.K * esize) % 16) {
    kp_set_error("tc_plan_create: K * element size must be a multiple of 16 bytes (K=%d)", g.K);
    return KP_ENOTSUP;
  }
  // Tile shape, CTAs per SM and K split.  Wide tiles (most work per byte
  // staged) when they alone give most SMs a tile; else 128-wide tiles, with
  // K split so that about one unit lands on each SM (each split keeping at
  // least 8 k-steps), two CTAs per SM when the tiles outnumber the SMs.
  const int sms = ctx->sm_count;
  const int bk_ = 128 / esize;
  if (g.batch_rows > 0 && (g.batch_rows % TBM != 0 || g.M != g.batch_rows * g.nkron)) {
    kp_set_error("tc_plan_create: batched rows must be a multiple of %d and M = terms x rows", TBM);
    return KP_EINVAL;
  }
  const int steps_all = g.npairs * (g.batch_rows > 0 ? 1 : g.nkron) * ((g.K + bk_ - 1) / bk_);
  const int tm = (g.M + TBM - 1) / TBM;
  auto tiles_of = [&](int w) { return tm * ((g.N + w - 1) / w); };
  int bn = 64;
  if (g.N >= 256 && 4 * tiles_of(256) >= 3 * sms)
    bn = 256;
  else if (g.N >= 128 && 4 * tiles_of(128) >= 3 * sms)
    bn = 128;
  if (ctx->tc_bn_override == 64 || ctx->tc_bn_override == 128 || ctx->tc_bn_override == 256)
    bn = ctx->tc_bn_override;
  // grouped launches of a batched solve with one tile shape for all problems
  // (so that one launch covers every problem's GEMM at that step)
  const bool uniform = ctx->tc_grouping && ctx->tc_group_uniform;
  if (uniform) bn = g.N >= 128 ? 128 : 64;
  const int tiles_bn = tiles_of(bn);
  int cps = (bn == 128 && tiles_bn > sms && !uniform) ? 2 : 1;
  if (bn == 128 && !uniform && (ctx->tc_cps_override == 1 || ctx->tc_cps_override == 2)) cps = ctx->tc_cps_override;
  if (splits < 1) {  // K split only when even 64-wide tiles leave most SMs idle
    splits = 1;
    if (2 * tiles_bn < sms && !ctx->tc_grouping)
      splits = std::max(1, std::min({4, sms / tiles_bn, steps_all / 16}));
  }
  // CTA pairs (256 x 256 tiles, cta_group::2) for BF16 GEMMs without a K
  // split whose pair tiles fill most SM pairs; option tc_pair: 1 = never,
  // 2 = whenever the shape allows
  const int pair_tiles = ((g.M + PAIR_M - 1) / PAIR_M) * ((g.N + PAIR_N - 1) / PAIR_N);
  const bool pair_ok = kind == TC_BF16 && splits == 1 && g.N >= PAIR_N &&
                       (g.batch_rows == 0 || g.batch_rows % PAIR_M == 0) && g.M >= PAIR_M;
  // (plans of a batched solve run in grouped launches: one-CTA tiles, no K split)
  const bool pair = pair_ok && !ctx->tc_grouping && ctx->tc_pair_override != 1 &&
                    (ctx->tc_pair_override == 2 || (ctx->tc_bn_override == 0 && 4 * pair_tiles >= 3 * (sms / 2)));
  // a K-concatenated product on 128 x 64 tiles (clusters of g.kcat CTAs along
  // N) where those tiles fill most SMs (option tc_kcat 2: wherever the shape
  // allows)
  const int kc_kps = (ctx->tc_kps_override == 1 || ctx->tc_kps_override == 2) ? ctx->tc_kps_override : 4;
  const int kc_cl = g.kcat == 4 ? 4 : 1;
  int kc_maxc = 0;
  bool kcat = false;
  if (g.kcat && kind == TC_BF16 && splits <= 1 && g.batch_rows == 0 && !ctx->tc_grouping &&
      (kc_cl == 1 || g.N % (KC_BN * kc_cl) == 0)) {
    const int kc_tiles = tm * ((g.N + KC_BN - 1) / KC_BN);
    kc_maxc = kcat_clusters(ctx, kc_kps, kc_cl);
    kcat = kc_maxc > 0 && (ctx->tc_kcat == 2 || 4 * kc_tiles >= 3 * sms);
  }
  TcGemmPlan* pl = new TcGemmPlan();
  pl->pair = pair && !kcat;
  pl->kcat = kcat ? kc_cl : 0;
  if (kcat) {
    splits = 1;
    bn = KC_BN;
    cps = 1;
  } else if (pair) {
    splits = 1;
    bn = PAIR_N;
  }
  kp_status st = make_map(&pl->mapA, g.A, kind, kcat ? TBM / kc_cl : TBM);
  if (st == KP_OK) st = make_map(&pl->mapB, g.B, kind, pl->pair ? PAIR_N / 2 : bn);
  if (st != KP_OK) {
    delete pl;
    return st;
  }
  TcParams& p = pl->params;
  p.M = g.M;
  p.N = g.N;
  p.K = g.K;
  p.nkron = g.nkron;
  p.npairs = g.npairs;
  p.a_terms = g.a_terms;
  p.b_terms = g.b_terms;
  for (int i = 0; i < KP_MAX_PAIRS; ++i) {
    p.sa[i] = g.sa[i];
    p.sb[i] = g.sb[i];
  }
  const int bk = 128 / esize;
  p.kblocks = (g.K + bk - 1) / bk;
  p.batch_rows = g.batch_rows;
  p.steps_total = g.npairs * (g.batch_rows > 0 ? 1 : g.nkron) * p.kblocks;
  p.tiles_m = pl->pair ? (g.M + PAIR_M - 1) / PAIR_M : (g.M + TBM - 1) / TBM;
  p.tiles_n = (g.N + bn - 1) / bn;
  const int tiles = p.tiles_m * p.tiles_n;
  splits = std::min(splits, p.steps_total);
  p.splits = splits;
  p.units = kcat ? tiles / kc_cl : tiles * splits;  // K-concatenated: one unit per cluster's tiles
  p.idesc = make_idesc(kind, bn, pl->pair ? PAIR_M : TBM);
  p.dot_out = nullptr;
  p.dot_part = nullptr;
  p.dot_count = nullptr;
  p.dot_po = PostOp();
  p.dot_qmax = 0;
  p.epi = g.epi;
  if (p.epi.ld_aux == 0) p.epi.ld_aux = p.epi.ldd;
  p.ws = ctx->w_split;
  p.counters = nullptr;
  p.alpha_dev = nullptr;
  p.flags = g.flags;
  p.status = ctx->dev_status;
  if (splits > 1) {
    if ((long long)splits * g.M * g.N > ctx->w_split_elems) {
      delete pl;
      kp_set_error("tc_plan_create: split-K workspace too small");
      return KP_EINVAL;
    }
    kp_status as = kp_alloc(ctx, (void**)&p.counters, sizeof(unsigned int) * tiles);
    if (as != KP_OK) {
      delete pl;
      return as;
    }
    cudaMemsetAsync(p.counters, 0, sizeof(unsigned int) * tiles, ctx->stream);
  }
  pl->kind = kind;
  pl->bn = bn;
  pl->cps = cps;
  // k-blocks per ring stage: 2, or 4 for 64-wide tiles (the producer's and
  // MMA thread's per-stage costs otherwise bound the main loop); 1 with two
  // CTAs per SM
  pl->kps = bn == 64 ? 4 : ((bn == 128 && cps == 2) ? 1 : 2);
  if (ctx->tc_kps_override == 1 || (ctx->tc_kps_override == 2 && !(bn == 128 && cps == 2)) ||
      (ctx->tc_kps_override == 4 && bn == 64))
    pl->kps = ctx->tc_kps_override;
  pl->grid = dim3(std::min(p.units, ctx->sm_count * cps), 1, 1);
  if (pl->pair) {
    pl->kps = (ctx->tc_kps_override == 1) ? 1 : 2;
    pl->grid = dim3(2 * std::min(p.units, ctx->sm_count / 2), 1, 1);
  }
  if (kcat) {
    pl->kps = kc_kps;
    pl->grid = dim3(kc_cl * std::min(p.units, kc_maxc), 1, 1);
  }
  ctx->tc_plans.push_back(pl);
  *out = pl;
  return KP_OK;
}

namespace {
// bf16 slices of FP64 or FP32 data (the FP32-rounded value, split exactly
// into `slices` parts): out[s * n + t]
template <typename T>
__global__ void k_to_bf16_slices(const T* __restrict__ in, long long n, int slices, __nv_bfloat16* __restrict__ out) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    float v = (float)in[t];
    for (int sl = 0; sl < slices; ++sl) {
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      out[sl * n + t] = h;
      v -= __bfloat162float(h);
    }
  }
}
}  // namespace

kp_status tc_operand_slices(kp_ctx* ctx, const void* in, bool f64, long long n, int slices, void* out) {
  const int g = (int)std::max(1LL, std::min((n + 255) / 256, (long long)ctx->sm_count * 16));
  if (f64)
    k_to_bf16_slices<double><<<g, 256, 0, ctx->stream>>>((const double*)in, n, slices, (__nv_bfloat16*)out);
  else
    k_to_bf16_slices<float><<<g, 256, 0, ctx->stream>>>((const float*)in, n, slices, (__nv_bfloat16*)out);
  KP_LAUNCHED(ctx);
  KP_CUDA(cudaGetLastError());
  return KP_OK;
}

kp_status tc_product_plan(kp_ctx* ctx, const void* a16, int rows_a, const void* b16, int rows_b, int K, int slices,
                          float* D, TcGemmPlan** out) {
  static const int acc_a[6] = {0, 0, 1, 0, 1, 2}, acc_b[6] = {0, 1, 0, 2, 1, 0};
  GemmDesc g;
  g.M = rows_a;
  g.N = rows_b;
  g.K = K;
  g.npairs = slices == 3 ? 6 : 1;
  for (int q = 0; q < g.npairs; ++q) {
    g.sa[q] = acc_a[q];
    g.sb[q] = acc_b[q];
  }
  g.A.ptr = a16;
  g.A.rows = rows_a;
  g.A.K = K;
  g.A.ld = K;
  g.A.tstride = (long long)rows_a * K;
  g.A.nterm_idx = slices;
  g.B.ptr = b16;
  g.B.rows = rows_b;
  g.B.K = K;
  g.B.ld = K;
  g.B.tstride = (long long)rows_b * K;
  g.B.nterm_idx = slices;
  g.epi.mode = EPI_F32;
  g.epi.out = D;
  g.epi.ldd = rows_b;
  return tc_plan_create(ctx, g, TC_BF16, 1, out);
}

// D = A B^T on the tensor cores: A rows_a x K and B rows_b x K (FP64 or FP32,
// K-major, leading dimension K), D row-major rows_a x rows_b FP32; the
// inputs as `slices` bf16 slices (1: half-precision inputs; 3: an exact
// split of the FP32 values, six slice products, FP32-level result), FP32
// accumulation.  K a multiple of 8.
kp_status tc_product(kp_ctx* ctx, const void* A, bool a64, int rows_a, const void* B, bool b64, int rows_b, int K,
                     float* D, int slices) {
  __nv_bfloat16 *a16 = nullptr, *b16 = nullptr;
  const long long na = (long long)rows_a * K, nb = (long long)rows_b * K;
  KP_TRY(kp_alloc(ctx, (void**)&a16, sizeof(__nv_bfloat16) * na * slices));
  KP_TRY(kp_alloc(ctx, (void**)&b16, sizeof(__nv_bfloat16) * nb * slices));
  KP_TRY(tc_operand_slices(ctx, A, a64, na, slices, a16));
  KP_TRY(tc_operand_slices(ctx, B, b64, nb, slices, b16));
  TcGemmPlan* pl = nullptr;
  KP_TRY(tc_product_plan(ctx, a16, rows_a, b16, rows_b, K, slices, D, &pl));
  return tc_plan_run(ctx, pl, nullptr);
}

kp_status half_product(kp_ctx* ctx, const double* A, int rows_a, const double* B, int rows_b, int K, float* D) {
  return tc_product(ctx, A, true, rows_a, B, true, rows_b, K, D, 1);
}

// ------------------------------------------------------------- tile autotuner
// With the option tc_autotune, each GEMM shape's tile configuration (tile
// width, CTAs per SM, k-blocks per ring stage, CTA pairs) is picked by
// timing the candidates: each runs once to warm up and three times between
// CUDA events on the context's stream, writing an FP32 scratch output.  The
// winners are kept per process and, when the environment variable
// KPSVD_TUNE_CACHE names a file, read from and appended to it, one line per
// shape: "kind M N K pairs terms batch_rows splits sms bn cps kps pair".
namespace {
struct TuneCfg {
  int bn, cps, kps, pair;
};
std::mutex g_tune_mutex;
std::map<std::string, TuneCfg> g_tune_cache;
bool g_tune_loaded = false;

std::string tune_key(const GemmDesc& g, int kind, int splits, int sms) {
  char b[160];
  std::snprintf(b, sizeof(b), "%d %d %d %d %d %d %d %d %d", kind, g.M, g.N, g.K, g.npairs, g.nkron, g.batch_rows,
                splits, sms);
  return b;
}

void tune_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = std::getenv("KPSVD_TUNE_CACHE");
  if (!path || !*path) return;
  std::FILE* f = std::fopen(path, "r");
  if (!f) return;
  int v[13];
  while (std::fscanf(f, "%d %d %d %d %d %d %d %d %d %d %d %d %d", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5], &v[6],
                     &v[7], &v[8], &v[9], &v[10], &v[11], &v[12]) == 13) {
    char b[160];
    std::snprintf(b, sizeof(b), "%d %d %d %d %d %d %d %d %d", v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7], v[8]);
    g_tune_cache[b] = TuneCfg{v[9], v[10], v[11], v[12]};
  }
  std::fclose(f);
}

void tune_store(const std::string& key, const TuneCfg& c) {
  g_tune_cache[key] = c;
  const char* path = std::getenv("KPSVD_TUNE_CACHE");
  if (!path || !*path) return;
  std::FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %d %d %d %d\n", key.c_str(), c.bn, c.cps, c.kps, c.pair);
  std::fclose(f);
}

// the context's tile overrides set to one configuration, restored on exit
struct OverrideScope {
  kp_ctx* c;
  int bn, cps, kps, pair;
  OverrideScope(kp_ctx* ctx, const TuneCfg& t)
      : c(ctx), bn(ctx->tc_bn_override), cps(ctx->tc_cps_override), kps(ctx->tc_kps_override),
        pair(ctx->tc_pair_override) {
    c->tc_bn_override = t.bn;
    c->tc_cps_override = t.cps;
    c->tc_kps_override = t.kps;
    c->tc_pair_override = t.pair ? 2 : 1;
  }
  ~OverrideScope() {
    c->tc_bn_override = bn;
    c->tc_cps_override = cps;
    c->tc_kps_override = kps;
    c->tc_pair_override = pair;
  }
};

void plan_discard(kp_ctx* ctx, TcGemmPlan* pl) {
  auto& v = ctx->tc_plans;
  v.erase(std::remove(v.begin(), v.end(), pl), v.end());
  delete pl;
}
}  // namespace

kp_status tc_plan_create(kp_ctx* ctx, const GemmDesc& g, int kind, int splits, TcGemmPlan** out) {
  if (!ctx->tc_autotune || g.kcat) return tc_plan_create_one(ctx, g, kind, splits, out);
  const std::string key = tune_key(g, kind, splits, ctx->sm_count);
  TuneCfg best{0, 0, 0, 0};
  bool have = false;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    tune_load();
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      best = it->second;
      have = true;
    }
  }
  if (!have) {
    // candidates; configurations the shape does not allow fall back inside
    // tc_plan_create_one and are skipped as duplicates of what it built
    std::vector<TuneCfg> cand;
    for (int bn : {64, 128, 256})
      for (int cps : {1, 2})
        for (int kps : {1, 2, 4}) {
          if (cps == 2 && bn != 128) continue;
          if (kps == 4 && bn != 64) continue;
          if (bn > 64 && bn > g.N) continue;
          cand.push_back(TuneCfg{bn, cps, kps, 0});
        }
    for (int kps : {1, 2}) cand.push_back(TuneCfg{256, 1, kps, 1});
    float* scratch = nullptr;
    KP_TRY(kp_alloc(ctx, (void**)&scratch, sizeof(float) * (size_t)g.M * g.N));
    EpiParams e;
    e.mode = EPI_F32;
    e.out = scratch;
    e.ldd = g.N;
    cudaEvent_t e0, e1;
    KP_CUDA(cudaEventCreate(&e0));
    KP_CUDA(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    std::vector<TuneCfg> seen;
    kp_status res = KP_OK;
    for (const TuneCfg& c : cand) {
      TcGemmPlan* pl = nullptr;
      {
        OverrideScope os(ctx, c);
        res = tc_plan_create_one(ctx, g, kind, splits, &pl);
      }
      if (res != KP_OK) break;
      const TuneCfg got{pl->bn, pl->cps, pl->kps, pl->pair ? 1 : 0};
      bool dup = false;
      for (const TuneCfg& q : seen) dup |= q.bn == got.bn && q.cps == got.cps && q.kps == got.kps && q.pair == got.pair;
      if (!dup && !(c.pair && !got.pair)) {
        seen.push_back(got);
        tc_plan_set_runtime(pl, nullptr, nullptr);
        res = tc_plan_run(ctx, pl, &e);
        if (res == KP_OK) res = cudaEventRecord(e0, ctx->stream) == cudaSuccess ? KP_OK : KP_ECUDA;
        for (int r = 0; r < 3 && res == KP_OK; ++r) res = tc_plan_run(ctx, pl, &e);
        if (res == KP_OK && (cudaEventRecord(e1, ctx->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
          res = KP_ECUDA;
        float ms = 0.f;
        if (res == KP_OK) cudaEventElapsedTime(&ms, e0, e1);
        if (res == KP_OK && ms < best_ms) {
          best_ms = ms;
          best = got;
        }
      }
      plan_discard(ctx, pl);
      if (res != KP_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    KP_TRY(res);
    KP_TRY(read_status(ctx));
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    tune_store(key, best);
  }
  OverrideScope os(ctx, best);
  return tc_plan_create_one(ctx, g, kind, splits, out);
}

void tc_plan_set_epi(TcGemmPlan* plan, const EpiParams& e) {
  plan->params.epi = e;
  if (plan->params.epi.ld_aux == 0) plan->params.epi.ld_aux = plan->params.epi.ldd;
}

void tc_plan_set_runtime(TcGemmPlan* plan, const float* alpha_dev, const int* flags) {
  plan->params.alpha_dev = alpha_dev;
  plan->params.flags = flags;
}

template <int KIND, int BN, int CPS, int KPS>
static kp_status launch_kind(kp_ctx* ctx, TcGemmPlan* pl, const TcParams& p) {
  using C = TcCfg<BN, CPS, KPS>;
  static std::atomic<bool> attr_set{false};  // contexts on several host threads launch this
  if (!attr_set.load()) {
    KP_CUDA(cudaFuncSetAttribute(tc_gemm_kernel<KIND, BN, CPS, KPS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 C::SMEM));
    attr_set = true;
  }
  KP_CUDA(kp_launch(ctx, tc_gemm_kernel<KIND, BN, CPS, KPS>, pl->grid, dim3(TC_THREADS), C::SMEM, pl->mapA, pl->mapB,
                    p));
  KP_LAUNCHED(ctx);
  return KP_OK;
}

template <int KIND, int KPS>
static kp_status launch_pair(kp_ctx* ctx, TcGemmPlan* pl, const TcParams& p) {
  using C = PairCfg<KPS>;
  static std::atomic<bool> attr_set{false};
  if (!attr_set.load()) {
    KP_CUDA(cudaFuncSetAttribute(tc_gemm_pair_kernel<KIND, KPS>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    attr_set = true;
  }
  KP_CUDA(kp_launch(ctx, tc_gemm_pair_kernel<KIND, KPS>, pl->grid, dim3(TC_THREADS), C::SMEM, pl->mapA, pl->mapB, p));
  KP_LAUNCHED(ctx);
  return KP_OK;
}

template <int KIND, int KPS, int CL>
static kp_status launch_kcat(kp_ctx* ctx, TcGemmPlan* pl, const TcParams& p) {
  using C = KcCfg<KPS, CL>;
  static std::atomic<bool> attr_set{false};
  if (!attr_set.load()) {
    KP_CUDA(cudaFuncSetAttribute(tc_gemm_kcat_kernel<KIND, KPS, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 C::SMEM));
    attr_set = true;
  }
  KP_CUDA(kp_launch(ctx, tc_gemm_kcat_kernel<KIND, KPS, CL>, pl->grid, dim3(TC_THREADS), C::SMEM, pl->mapA, pl->mapB,
                    p));
  KP_LAUNCHED(ctx);
  return KP_OK;
}

// recorded launches of a batched solve (see KpRec): the records of one
// kernel configuration at one position become one tc_gemm_group_kernel launch
template <int KIND, int BN, int CPS, int KPS>
struct GemmGroup {
  static size_t bytes(int n) { return sizeof(TcGroupEntry) * (size_t)n + sizeof(int) * (size_t)(n + 1); }
  static int units_of(const KpRec* r) {
    TcGroupEntry e;
    std::memcpy(&e, r->blob.data(), sizeof(e));
    return e.p.units;
  }
  static void table(const KpRec* const* r, int n, unsigned char* dst) {
    // (before the graph capture that launches it)
    static std::atomic<bool> attr_set{false};
    if (!attr_set.load()) {
      cudaFuncSetAttribute(tc_gemm_group_kernel<KIND, BN, CPS, KPS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           TcCfg<BN, CPS, KPS>::SMEM);
      attr_set = true;
    }
    int* us = reinterpret_cast<int*>(dst + sizeof(TcGroupEntry) * (size_t)n);
    int acc = 0;
    for (int i = 0; i < n; ++i) {
      std::memcpy(dst + sizeof(TcGroupEntry) * (size_t)i, r[i]->blob.data(), sizeof(TcGroupEntry));
      us[i] = acc;
      acc += units_of(r[i]);
    }
    us[n] = acc;
  }
  static kp_status launch(kp_ctx* ctx, const KpRec* const* r, int n, const void* dev) {
    using C = TcCfg<BN, CPS, KPS>;
    long long total = 0;
    for (int i = 0; i < n; ++i) total += units_of(r[i]);
    TcGroupEntry e0;
    std::memcpy(&e0, r[0]->blob.data(), sizeof(e0));
    const int grid = (int)std::max(1LL, std::min(total, (long long)ctx->sm_count * CPS));
    const TcGroupEntry* ents = reinterpret_cast<const TcGroupEntry*>(dev);
    const int* us = reinterpret_cast<const int*>(reinterpret_cast<const unsigned char*>(dev) +
                                                 sizeof(TcGroupEntry) * (size_t)n);
    KP_CUDA(kp_launch(ctx, tc_gemm_group_kernel<KIND, BN, CPS, KPS>, dim3(grid), dim3(TC_THREADS), C::SMEM, ents, us,
                      n, e0.p.status));
    KP_LAUNCHED(ctx);
    return KP_OK;
  }
  static void record(kp_ctx* ctx, const TcGemmPlan* pl, const TcParams& p) {
    TcGroupEntry e;
    e.mapA = pl->mapA;
    e.mapB = pl->mapB;
    e.p = p;
    KpRec rec;
    rec.key = reinterpret_cast<const void*>(tc_gemm_group_kernel<KIND, BN, CPS, KPS>);
    rec.table_bytes = &bytes;
    rec.table = &table;
    rec.launch = &launch;
    rec.grid = pl->grid;
    rec.block = dim3(TC_THREADS);
    rec.smem = TcCfg<BN, CPS, KPS>::SMEM;
    rec.blob.resize(sizeof(e));
    std::memcpy(rec.blob.data(), &e, sizeof(e));
    ctx->rec->recs.push_back(std::move(rec));
  }
};

template <int KIND>
static kp_status record_cfg(kp_ctx* ctx, TcGemmPlan* pl, const TcParams& p) {
  if (pl->pair || pl->kcat || p.splits != 1) {
    kp_set_error("batched solve: a CTA-pair, K-concatenated or split-K GEMM plan cannot be grouped");
    return KP_ENOTSUP;
  }
  if (pl->bn == 256) {
    if (pl->kps == 2) GemmGroup<KIND, 256, 1, 2>::record(ctx, pl, p);
    else GemmGroup<KIND, 256, 1, 1>::record(ctx, pl, p);
  } else if (pl->bn == 64) {
    if (pl->kps == 4) GemmGroup<KIND, 64, 1, 4>::record(ctx, pl, p);
    else if (pl->kps == 2) GemmGroup<KIND, 64, 1, 2>::record(ctx, pl, p);
    else GemmGroup<KIND, 64, 1, 1>::record(ctx, pl, p);
  } else if (pl->cps == 2) {
    GemmGroup<KIND, 128, 2, 1>::record(ctx, pl, p);
  } else if (pl->kps == 2) {
    GemmGroup<KIND, 128, 1, 2>::record(ctx, pl, p);
  } else {
    GemmGroup<KIND, 128, 1, 1>::record(ctx, pl, p);
  }
  return KP_OK;
}

template <int KIND>
static kp_status launch_cfg(kp_ctx* ctx, TcGemmPlan* pl, const TcParams& p) {
  if (ctx->rec) return record_cfg<KIND>(ctx, pl, p);
  if (pl->kcat) {
    if constexpr (KIND == TC_BF16) {
      if (pl->kcat == 4) {
        if (pl->kps == 4) return launch_kcat<KIND, 4, 4>(ctx, pl, p);
        return pl->kps == 2 ? launch_kcat<KIND, 2, 4>(ctx, pl, p) : launch_kcat<KIND, 1, 4>(ctx, pl, p);
      }
      if (pl->kps == 4) return launch_kcat<KIND, 4, 1>(ctx, pl, p);
      return pl->kps == 2 ? launch_kcat<KIND, 2, 1>(ctx, pl, p) : launch_kcat<KIND, 1, 1>(ctx, pl, p);
    } else {
      kp_set_error("tensor-core GEMM: K-concatenated products are built for BF16 only");
      return KP_ENOTSUP;
    }
  }
  if (pl->pair) {
    if constexpr (KIND == TC_BF16) {
      return pl->kps == 1 ? launch_pair<KIND, 1>(ctx, pl, p) : launch_pair<KIND, 2>(ctx, pl, p);
    } else {
      kp_set_error("tensor-core GEMM: CTA-pair tiles are built for BF16 only");
      return KP_ENOTSUP;
    }
  }
  if (pl->bn == 256) return pl->kps == 2 ? launch_kind<KIND, 256, 1, 2>(ctx, pl, p) : launch_kind<KIND, 256, 1, 1>(ctx, pl, p);
  if (pl->bn == 64) {
    if (pl->kps == 4) return launch_kind<KIND, 64, 1, 4>(ctx, pl, p);
    return pl->kps == 2 ? launch_kind<KIND, 64, 1, 2>(ctx, pl, p) : launch_kind<KIND, 64, 1, 1>(ctx, pl, p);
  }
  if (pl->cps == 2) return launch_kind<KIND, 128, 2, 1>(ctx, pl, p);
  return pl->kps == 2 ? launch_kind<KIND, 128, 1, 2>(ctx, pl, p) : launch_kind<KIND, 128, 1, 1>(ctx, pl, p);
}

kp_status tc_plan_run(kp_ctx* ctx, TcGemmPlan* pl, const EpiParams* epi_override) {
  TcParams p = pl->params;
  if (epi_override) {
    p.epi = *epi_override;
    if (p.epi.ld_aux == 0) p.epi.ld_aux = p.epi.ldd;
  }
  kp_status st;
  if (pl->kind == TC_BF16)
    st = launch_cfg<TC_BF16>(ctx, pl, p);
  else if (pl->kind == TC_F16)
    st = launch_cfg<TC_F16>(ctx, pl, p);
  else
    st = launch_cfg<TC_E4M3>(ctx, pl, p);
  KP_TRY(st);
  KP_CUDA(cudaGetLastError());
  return KP_OK;
}

bool tc_plan_is_kcat(const TcGemmPlan* plan) { return plan && plan->kcat > 0; }

void tc_plan_release(kp_ctx* ctx, TcGemmPlan* plan) {
  if (plan) plan_discard(ctx, plan);
}

kp_status tc_plan_run_dot(kp_ctx* ctx, TcGemmPlan* pl, const EpiParams& epi, double* out2, double* partials,
                          unsigned int* counter, const PostOp& post, int qmax) {
  if (!pl->kcat || epi.mode != EPI_F32 || !epi.aux || !out2 || !partials || !counter) {
    kp_set_error("tc_plan_run_dot: needs a K-concatenated plan, an FP32 output with aux and the reduction buffers");
    return KP_EINVAL;
  }
  TcParams p = pl->params;
  p.epi = epi;
  if (p.epi.ld_aux == 0) p.epi.ld_aux = p.epi.ldd;
  p.dot_out = out2;
  p.dot_part = partials;
  p.dot_count = counter;
  p.dot_po = post;
  p.dot_qmax = qmax;
  KP_TRY(launch_cfg<TC_BF16>(ctx, pl, p));
  KP_CUDA(cudaGetLastError());
  return KP_OK;
}

void tc_plans_free(kp_ctx* ctx) {
  for (auto* p : ctx->tc_plans) delete p;
  ctx->tc_plans.clear();
}
