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
// One CTA computes one 128 x 128 output tile (optionally one K-range of it
// when split-K is used):
//   warp 0      TMA producer (one elected thread)
//   warp 1      TMEM allocation + MMA issuer (one elected thread)
//   warps 2..5  epilogue: tcgen05.ld TMEM -> registers -> fused output
// STAGES-deep shared-memory ring with full / empty mbarriers.  Every wait is
// bounded; a wait that gives up sets DEV_ERR_TIMEOUT in the device status
// word and the CTA drains and returns.
#include <cudaTypedefs.h>

#include "kp_internal.h"
#include "kp_vec.cuh"

namespace {

constexpr int TBM = 128, TBN = 128;
constexpr int STAGES = 4;
constexpr int TILE_BYTES = 128 * 128;           // 128 rows x 128 bytes
constexpr int STAGE_BYTES = 2 * TILE_BYTES;     // A + B
constexpr int TC_THREADS = 192;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;

struct TcParams {
  int M, N, K;
  int nkron, npairs, a_terms, b_terms;
  int sa[KP_MAX_PAIRS], sb[KP_MAX_PAIRS];
  int kblocks;      // ceil(K / BK)
  int splits;       // split-K factor over the (pair, term, kblock) steps
  int steps_total;  // npairs * nkron * kblocks
  uint32_t idesc;
  EpiParams epi;
  float* ws;        // split-K partials [split][M][N]
  const float* alpha_dev;  // optional device scale multiplied into the output
  const int* flags;
  int* status;
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
// Fused output of one row segment of 32 columns (row gm, columns gn0..gn0+31).
// Full, 16-byte aligned segments use vector loads and stores.
__device__ __forceinline__ void epi_store32(const EpiParams& e, float scale_dev, int gm, int gn0, int N,
                                            const float (&acc)[32]) {
  const long long base = (long long)gm * e.ldd + gn0;
  const int cnt = min(32, N - gn0);
  if (cnt <= 0) return;
  const float* aux = (const float*)e.aux;
  const long long abase = (long long)gm * e.ld_aux + gn0;
  const bool vec = (cnt == 32) && ((base & 7) == 0) && (aux == nullptr || (abase & 3) == 0);
  float v[32];
  const float a = (float)e.alpha * scale_dev;
#pragma unroll
  for (int c = 0; c < 32; ++c) v[c] = a * acc[c];
  if (aux) {
    if (vec) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float4 t = *reinterpret_cast<const float4*>(aux + abase + 4 * q);
        v[4 * q + 0] = fmaf((float)e.beta, t.x, v[4 * q + 0]);
        v[4 * q + 1] = fmaf((float)e.beta, t.y, v[4 * q + 1]);
        v[4 * q + 2] = fmaf((float)e.beta, t.z, v[4 * q + 2]);
        v[4 * q + 3] = fmaf((float)e.beta, t.w, v[4 * q + 3]);
      }
    } else {
      for (int c = 0; c < cnt; ++c) v[c] = fmaf((float)e.beta, aux[abase + c], v[c]);
    }
  }
  if (e.mode == EPI_NARROW && e.sigma32) {
    for (int c = 0; c < cnt; ++c) {
      const double sg = (double)e.sigma32[base + c];
      v[c] = v[c] * (float)(e.lam2 / (sg * sg + e.lam2));
    }
  }
  switch (e.mode) {
    case EPI_F32: {
      float* out = (float*)e.out + base;
      if (vec) {
#pragma unroll
        for (int q = 0; q < 8; ++q)
          *reinterpret_cast<float4*>(out + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      } else {
        for (int c = 0; c < cnt; ++c) out[c] = v[c];
      }
      break;
    }
    case EPI_SLICES: {
      __nv_bfloat16* out = (__nv_bfloat16*)e.out + base;
      for (int s = 0; s < e.slices; ++s) {
        __align__(16) __nv_bfloat16 h[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          h[c] = __float2bfloat16_rn(v[c]);
          v[c] -= __bfloat162float(h[c]);
        }
        __nv_bfloat16* o = out + s * e.slice_stride;
        if (vec) {
#pragma unroll
          for (int q = 0; q < 4; ++q) *reinterpret_cast<uint4*>(o + 8 * q) = *reinterpret_cast<const uint4*>(h + 8 * q);
        } else {
          for (int c = 0; c < cnt; ++c) o[c] = h[c];
        }
      }
      break;
    }
    case EPI_NARROW: {
      if (e.narrow == NT_E4M3) {
        __align__(16) __nv_fp8_e4m3 h[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) h[c] = __nv_fp8_e4m3(v[c]);
        __nv_fp8_e4m3* o = (__nv_fp8_e4m3*)e.out + base;
        if (vec && (base & 15) == 0) {
          *reinterpret_cast<uint4*>(o) = *reinterpret_cast<const uint4*>(h);
          *reinterpret_cast<uint4*>(o + 16) = *reinterpret_cast<const uint4*>(h + 16);
        } else {
          for (int c = 0; c < cnt; ++c) o[c] = h[c];
        }
      } else {
        __align__(16) uint16_t h[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          if (e.narrow == NT_BF16) {
            __nv_bfloat16 b = __float2bfloat16_rn(v[c]);
            h[c] = *reinterpret_cast<uint16_t*>(&b);
          } else {
            __half b = __float2half_rn(v[c]);
            h[c] = *reinterpret_cast<uint16_t*>(&b);
          }
        }
        uint16_t* o = (uint16_t*)e.out + base;
        if (vec) {
#pragma unroll
          for (int q = 0; q < 4; ++q) *reinterpret_cast<uint4*>(o + 8 * q) = *reinterpret_cast<const uint4*>(h + 8 * q);
        } else {
          for (int c = 0; c < cnt; ++c) o[c] = h[c];
        }
      }
      break;
    }
    default:
      break;
  }
}

template <int KIND>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcParams p) {
  if (p.flags && *(volatile const int*)p.flags) return;
  extern __shared__ unsigned char smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint64_t* full = bars;
  uint64_t* empty = bars + STAGES;
  uint64_t* tfull = bars + 2 * STAGES;
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * STAGES + 1);
  __shared__ int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;
  const int split = blockIdx.z;
  const int per = (p.steps_total + p.splits - 1) / p.splits;
  const int step0 = split * per;
  const int step1 = min(p.steps_total, step0 + per);
  const int nsteps = max(0, step1 - step0);

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(tfull), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TBN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      for (int it = 0; it < nsteps; ++it) {
        const int stp = step0 + it;
        const int kb = stp % p.kblocks;
        const int rest = stp / p.kblocks;
        const int k = rest % p.nkron;
        const int pr = rest / p.nkron;
        const int ta = p.sa[pr] * p.a_terms + k;
        const int tb = p.sb[pr] * p.b_terms + k;
        const int s = it % STAGES;
        const uint32_t ph = (it / STAGES) & 1;
        if (!mbar_wait(smem_u32(&empty[s]), ph ^ 1, p.status)) {
          s_abort = 1;
          break;
        }
        const uint32_t fb = smem_u32(&full[s]);
        mbar_expect_tx(fb, STAGE_BYTES);
        const int kc = kb * 128 / (KIND == TC_E4M3 ? 1 : 2);
        tma_load_3d(smem_u32(smem + s * STAGE_BYTES), &tmA, kc, m0, ta, fb);
        tma_load_3d(smem_u32(smem + s * STAGE_BYTES + TILE_BYTES), &tmB, kc, n0, tb, fb);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      for (int it = 0; it < nsteps; ++it) {
        const int s = it % STAGES;
        const uint32_t ph = (it / STAGES) & 1;
        if (*(volatile int*)&s_abort || !mbar_wait(smem_u32(&full[s]), ph, p.status)) {
          s_abort = 1;
          break;
        }
        tc_fence_after();
        const uint32_t a0 = smem_u32(smem + s * STAGE_BYTES);
        const uint32_t b0 = a0 + TILE_BYTES;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {  // 4 x 32 bytes of K per 128-byte row
          mma_issue<KIND>(tmem, make_sdesc(a0 + kk * 32), make_sdesc(b0 + kk * 32), p.idesc,
                          (it > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(smem_u32(&empty[s]));
      }
      mma_commit(smem_u32(tfull));
    }
  } else {
    // ---------------- epilogue warps 2..5 -> TMEM lanes 32 * (warp % 4)
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const int gm = m0 + row;
    bool ok = mbar_wait(smem_u32(tfull), 0, p.status);
    tc_fence_after();
    if (ok) {
      const float sdev = p.alpha_dev ? *p.alpha_dev : 1.f;
#pragma unroll 1
      for (int chunk = 0; chunk < TBN / 32; ++chunk) {
        float acc[32];
        if (nsteps > 0) {
          tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + chunk * 32, acc);
        } else {
#pragma unroll
          for (int c = 0; c < 32; ++c) acc[c] = 0.f;
        }
        const int gn0 = n0 + chunk * 32;
        if (gm < p.M && gn0 < p.N) {
          if (p.epi.mode == EPI_PARTIAL) {
            float* w = p.ws + ((long long)split * p.M + gm) * p.N + gn0;
            const int cnt = min(32, p.N - gn0);
            for (int c = 0; c < cnt; ++c) w[c] = acc[c];
          } else {
            epi_store32(p.epi, sdev, gm, gn0, p.N, acc);
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TBN) : "memory");
  }
}

// split-K finish: sum partials in split order, then the fused epilogue
__global__ void k_splitk_finish(const float* __restrict__ ws, int splits, int M, int N, EpiParams e,
                                const float* alpha_dev, const int* flags) {
  if (flags && *(volatile const int*)flags) return;
  const float sdev = alpha_dev ? *alpha_dev : 1.f;
  const long long tot = (long long)M * ((N + 31) / 32);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int gm = (int)(t / ((N + 31) / 32));
    const int gn0 = (int)(t % ((N + 31) / 32)) * 32;
    float acc[32];
    const int cnt = min(32, N - gn0);
#pragma unroll
    for (int c = 0; c < 32; ++c) acc[c] = 0.f;
    for (int s = 0; s < splits; ++s) {
      const float* w = ws + ((long long)s * M + gm) * N + gn0;
      for (int c = 0; c < cnt; ++c) acc[c] += w[c];
    }
    epi_store32(e, sdev, gm, gn0, N, acc);
  }
}

}  // namespace

// ------------------------------------------------------------- host side
struct TcGemmPlan {
  CUtensorMap mapA, mapB;
  TcParams params;
  int kind;
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

static kp_status make_map(CUtensorMap* map, const GemmOp& op, int kind) {
  const int esize = kind == TC_E4M3 ? 1 : 2;
  const int bk = 128 / esize;
  cuuint64_t dims[3] = {(cuuint64_t)op.K, (cuuint64_t)op.rows, (cuuint64_t)(op.nterm_idx > 0 ? op.nterm_idx : 1)};
  cuuint64_t strides[2] = {(cuuint64_t)(op.ld * esize), (cuuint64_t)(op.tstride * esize)};
  cuuint32_t box[3] = {(cuuint32_t)bk, 128u, 1u};
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

static uint32_t make_idesc(int kind) {
  uint32_t d = 0;
  d |= 1u << 4;  // D format F32
  if (kind == TC_BF16) {
    d |= 1u << 7;   // A BF16
    d |= 1u << 10;  // B BF16
  }                 // F16 / E4M3: format code 0
  // K-major A and B (bits 15, 16 = 0)
  d |= (uint32_t)(TBN >> 3) << 17;
  d |= (uint32_t)(TBM >> 4) << 24;
  return d;
}

bool tc_device_supported(kp_ctx* ctx) {
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, ctx->device);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, ctx->device);
  return major == 10 && minor == 3;
}

kp_status tc_plan_create(kp_ctx* ctx, const GemmDesc& g, int kind, int splits, TcGemmPlan** out) {
  if (g.npairs < 1 || g.npairs > KP_MAX_PAIRS || g.nkron < 1) {
    kp_set_error("tc_plan_create: bad term description");
    return KP_EINVAL;
  }
  const int esize = kind == TC_E4M3 ? 1 : 2;
  if ((g.K * esize) % 16) {
    kp_set_error("tc_plan_create: K * element size must be a multiple of 16 bytes (K=%d)", g.K);
    return KP_ENOTSUP;
  }
  TcGemmPlan* pl = new TcGemmPlan();
  kp_status st = make_map(&pl->mapA, g.A, kind);
  if (st == KP_OK) st = make_map(&pl->mapB, g.B, kind);
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
  p.steps_total = g.npairs * g.nkron * p.kblocks;
  if (splits < 1) splits = 1;
  if (splits > p.steps_total) splits = p.steps_total;
  p.splits = splits;
  p.idesc = make_idesc(kind);
  p.epi = g.epi;
  if (p.epi.ld_aux == 0) p.epi.ld_aux = p.epi.ldd;
  p.ws = ctx->w_split;
  p.alpha_dev = nullptr;
  p.flags = g.flags;
  p.status = ctx->dev_status;
  if (splits > 1 && (long long)splits * g.M * g.N > ctx->w_split_elems) {
    delete pl;
    kp_set_error("tc_plan_create: split-K workspace too small");
    return KP_EINVAL;
  }
  pl->kind = kind;
  pl->grid = dim3((g.N + TBN - 1) / TBN, (g.M + TBM - 1) / TBM, splits);
  ctx->tc_plans.push_back(pl);
  *out = pl;
  return KP_OK;
}

void tc_plan_set_epi(TcGemmPlan* plan, const EpiParams& e) {
  plan->params.epi = e;
  if (plan->params.epi.ld_aux == 0) plan->params.epi.ld_aux = plan->params.epi.ldd;
}

void tc_plan_set_runtime(TcGemmPlan* plan, const float* alpha_dev, const int* flags) {
  plan->params.alpha_dev = alpha_dev;
  plan->params.flags = flags;
}

template <int KIND>
static kp_status launch_kind(kp_ctx* ctx, TcGemmPlan* pl, const TcParams& p) {
  static bool attr_set = false;
  if (!attr_set) {
    KP_CUDA(cudaFuncSetAttribute(tc_gemm_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    attr_set = true;
  }
  tc_gemm_kernel<KIND><<<pl->grid, TC_THREADS, SMEM_BYTES, ctx->stream>>>(pl->mapA, pl->mapB, p);
  KP_LAUNCHED(ctx);
  return KP_OK;
}

kp_status tc_plan_run(kp_ctx* ctx, TcGemmPlan* pl, const EpiParams* epi_override) {
  TcParams p = pl->params;
  if (epi_override) {
    p.epi = *epi_override;
    if (p.epi.ld_aux == 0) p.epi.ld_aux = p.epi.ldd;
  }
  const EpiParams final_epi = p.epi;
  if (p.splits > 1) p.epi.mode = EPI_PARTIAL;
  if (pl->kind == TC_BF16)
    KP_TRY(launch_kind<TC_BF16>(ctx, pl, p));
  else if (pl->kind == TC_F16)
    KP_TRY(launch_kind<TC_F16>(ctx, pl, p));
  else
    KP_TRY(launch_kind<TC_E4M3>(ctx, pl, p));
  KP_CUDA(cudaGetLastError());
  if (p.splits > 1) {
    long long tot = (long long)p.M * ((p.N + 31) / 32);
    int blocks = (int)std::min<long long>((tot + 255) / 256, (long long)ctx->sm_count * 8);
    k_splitk_finish<<<blocks, 256, 0, ctx->stream>>>(p.ws, p.splits, p.M, p.N, final_epi, p.alpha_dev, p.flags);
    KP_LAUNCHED(ctx);
    KP_CUDA(cudaGetLastError());
  }
  return KP_OK;
}

void tc_plans_free(kp_ctx* ctx) {
  for (auto* p : ctx->tc_plans) delete p;
  ctx->tc_plans.clear();
}
