// C ABI entry points: context lifetime, errors, options, getters.
// The operations themselves are in kp_setup.cu, kp_solver.cu, kp_lambda.cu.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <mutex>
#include <string>

#include <algorithm>

#include <cmath>

#include "kp_internal.h"

static thread_local std::string g_last_error;

void kp_set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

extern "C" const char* kp_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* kp_status_str(kp_status s) {
  switch (s) {
    case KP_OK: return "KP_OK";
    case KP_EINVAL: return "KP_EINVAL: invalid argument";
    case KP_ENOMEM: return "KP_ENOMEM: out of memory";
    case KP_ECUDA: return "KP_ECUDA: CUDA error";
    case KP_ENOTSUP: return "KP_ENOTSUP: unsupported";
    case KP_ENOCONV: return "KP_ENOCONV: not converged";
    case KP_EBREAKDOWN: return "KP_EBREAKDOWN: PCG breakdown";
    case KP_ENUMERIC: return "KP_ENUMERIC: NaN or Inf";
    case KP_ENOROOT: return "KP_ENOROOT: no root";
    case KP_ETIMEOUT: return "KP_ETIMEOUT: device wait timed out";
    case KP_ESTATE: return "KP_ESTATE: call out of order";
  }
  return "unknown status";
}

// Host-side fault injection: with KPSVD_FAULT=alloc:N in the environment the
// N-th device allocation after the variable was set (or changed) fails as if
// cudaMalloc had, so the error paths can be tested without touching the GPU.
static bool injected_alloc_failure() {
  static std::mutex mu;
  static std::string last;
  static long count = 0;
  const char* v = std::getenv("KPSVD_FAULT");
  std::lock_guard<std::mutex> lock(mu);
  const std::string cur = v ? v : "";
  if (cur != last) {
    last = cur;
    count = 0;
  }
  if (cur.compare(0, 6, "alloc:") != 0) return false;
  const long n = std::atol(cur.c_str() + 6);
  return n > 0 && ++count == n;
}

kp_status kp_alloc(kp_ctx* ctx, void** p, size_t bytes) {
  *p = nullptr;
  if (injected_alloc_failure()) {
    kp_set_error("device allocation of %zu bytes failed (injected by KPSVD_FAULT)", bytes);
    return KP_ENOMEM;
  }
  bytes = (std::max<size_t>(bytes, 16) + 255) & ~(size_t)255;
  // smallest pooled block that fits and wastes at most half of itself
  auto it = ctx->pool.lower_bound(bytes);
  if (it != ctx->pool.end() && it->first <= 2 * bytes) {
    *p = it->second;
    ctx->allocs.emplace_back(it->second, it->first);
    ctx->pool.erase(it);
    return KP_OK;
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess && !ctx->pool.empty()) {  // give the pool back and retry once
    cudaGetLastError();
    kp_pool_release(ctx);
    e = cudaMalloc(p, bytes);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    kp_set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    return KP_ENOMEM;
  }
  ctx->allocs.emplace_back(*p, bytes);
  return KP_OK;
}

void kp_pool_release(kp_ctx* ctx) {
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (auto& b : ctx->pool) cudaFree(b.second);
  ctx->pool.clear();
}

void tc_plans_free(kp_ctx* ctx);

void ops_state_free(kp_ctx* ctx);

kp_status kp_enter(kp_ctx* ctx) {
  KP_CUDA(cudaSetDevice(ctx->device));
  if (!ctx->own_stream) return KP_OK;
  KP_CUDA(cudaEventRecord(ctx->ev_in, ctx->user_stream));
  KP_CUDA(cudaStreamWaitEvent(ctx->stream, ctx->ev_in, 0));
  return KP_OK;
}

kp_status kp_leave(kp_ctx* ctx) {
  if (!ctx->own_stream) return KP_OK;
  KP_CUDA(cudaEventRecord(ctx->ev_out, ctx->stream));
  KP_CUDA(cudaStreamWaitEvent(ctx->user_stream, ctx->ev_out, 0));
  return KP_OK;
}

void kp_free_all(kp_ctx* ctx) {
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  ops_state_free(ctx);
  for (auto& b : ctx->allocs) ctx->pool.emplace(b.second, b.first);
  ctx->allocs.clear();
  tc_plans_free(ctx);
  for (auto& t : ctx->lam_tc) t = kp_ctx::LamTc();
  ctx->lam_img16 = ctx->lam_t16 = nullptr;
  ctx->lam_t32 = ctx->lam_o32 = nullptr;
  ctx->lam_ws = nullptr;
  ctx->simt_ws = nullptr;
  ctx->simt_ws_bytes = 0;
  ctx->lam_sigma_ready = false;
  ctx->Uc32 = ctx->Ur32 = ctx->Vc32 = ctx->Vr32 = nullptr;
  ctx->ready = false;
}

namespace {
// a wait on an mbarrier that nothing arrives on, bounded by limit_ns (the
// global timer): on give-up the status word's timeout bit is set
__global__ void k_bounded_wait(int* status, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(&bar));
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(1u) : "memory");
  unsigned long long t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(0u)
        : "memory");
    if (ok) return;
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > limit_ns) {
      atomicOr(status, DEV_ERR_TIMEOUT);
      return;
    }
  }
}
}  // namespace

// Test hook: one bounded device wait that nothing releases, so that the
// timeout path (status word -> KP_ETIMEOUT, context still usable) can be
// exercised without a GPU fault.
extern "C" kp_status kp_test_bounded_wait(kp_ctx* ctx, double limit_ms) {
  if (!ctx || !(limit_ms > 0.0) || limit_ms > 10000.0) {
    kp_set_error("kp_test_bounded_wait: need a context and 0 < limit_ms <= 10000");
    return KP_EINVAL;
  }
  KP_CUDA(cudaSetDevice(ctx->device));
  KP_TRY(kp_enter(ctx));
  KP_CUDA(cudaMemsetAsync(ctx->dev_status, 0, sizeof(int), ctx->stream));
  k_bounded_wait<<<1, 1, 0, ctx->stream>>>(ctx->dev_status, (unsigned long long)(limit_ms * 1e6));
  KP_LAUNCHED(ctx);
  KP_CUDA(cudaGetLastError());
  const kp_status st = read_status(ctx);
  KP_CUDA(cudaMemsetAsync(ctx->dev_status, 0, sizeof(int), ctx->stream));
  KP_CUDA(cudaStreamSynchronize(ctx->stream));
  const kp_status l = kp_leave(ctx);
  return st != KP_OK ? st : l;
}

cudaError_t kp_wait(kp_ctx* ctx, cudaStream_t st) {
  if (!ctx->yield) return cudaStreamSynchronize(st);
  if (!ctx->ev_wait) {
    const cudaError_t e = cudaEventCreateWithFlags(&ctx->ev_wait, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaEventRecord(ctx->ev_wait, st);
  if (e != cudaSuccess) return e;
  while ((e = cudaEventQuery(ctx->ev_wait)) == cudaErrorNotReady) ctx->yield(ctx->yield_arg);
  return e;
}

kp_status read_status(kp_ctx* ctx) {
  int h = 0;
  KP_CUDA(cudaMemcpyAsync(&h, ctx->dev_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  KP_CUDA(kp_wait(ctx, ctx->stream));
  if (h & DEV_ERR_TIMEOUT) {
    kp_set_error("a bounded device-side wait gave up (status word 0x%x)", h);
    return KP_ETIMEOUT;
  }
  if (h & DEV_ERR_BOUNDS) {
    kp_set_error("device-side bounds check failed (status word 0x%x)", h);
    return KP_EINVAL;
  }
  return KP_OK;
}

extern "C" kp_status kp_create(kp_ctx** out, int device, void* cuda_stream) {
  if (!out) {
    kp_set_error("kp_create: out is NULL");
    return KP_EINVAL;
  }
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    kp_set_error("kp_create: no CUDA device (%s)", cudaGetErrorString(e));
    return KP_ECUDA;
  }
  if (device < 0 || device >= ndev) {
    kp_set_error("kp_create: device %d out of range [0, %d)", device, ndev);
    return KP_EINVAL;
  }
  KP_CUDA(cudaSetDevice(device));
  kp_ctx* ctx = new kp_ctx();
  ctx->device = device;
  ctx->user_stream = (cudaStream_t)cuda_stream;
  // a caller's stream is used directly; the legacy default stream (NULL) can
  // not be captured into graphs, so then work runs on a private stream
  // ordered with it through events
  ctx->own_stream = cuda_stream == nullptr;
  if (!ctx->own_stream) ctx->stream = ctx->user_stream;
  if ((ctx->own_stream && cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) ||
      cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    kp_set_error("kp_create: stream / event creation failed");
    return KP_ECUDA;
  }
  cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
  // context-level buffers (not released by a new kp_setup)
  void* p = nullptr;
  const size_t bytes = 4096 + 64 * 1024 * sizeof(double) + 256;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    kp_set_error("kp_create: cudaMalloc failed");
    return KP_ENOMEM;
  }
  cudaMemset(p, 0, bytes);
  ctx->dev_status = (int*)p;                                   // [0..63] bytes: status word
  ctx->dflags = (int*)((char*)p + 64);                         // [64..255] bytes: solver flags
  ctx->red_count = (unsigned int*)((char*)p + 256);            // reduction counter
  ctx->dscal = (double*)((char*)p + 1024);                     // 384 doubles of scalars
  ctx->red_part = (double*)((char*)p + 4096);                  // reduction partials
  ctx->ctx_block = p;
  *out = ctx;
  return KP_OK;
}

extern "C" void kp_destroy(kp_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  kp_free_all(ctx);
  kp_pool_release(ctx);
  if (ctx->hmirror) cudaFreeHost(ctx->hmirror);
  for (auto& e : ctx->ev_setup)
    if (e) cudaEventDestroy(e);
  for (auto& e : ctx->ev_blk)
    if (e) cudaEventDestroy(e);
  if (ctx->ev_wait) cudaEventDestroy(ctx->ev_wait);
  jacobi_cache_free(ctx);
  if (ctx->ctx_block) cudaFree(ctx->ctx_block);
  if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
  if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
  if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
  if (ctx->stream && ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

extern "C" kp_status kp_set_option(kp_ctx* ctx, const char* name, double value) {
  if (!ctx || !name) {
    kp_set_error("kp_set_option: NULL argument");
    return KP_EINVAL;
  }
  if (!strcmp(name, "reliable_delta")) {
    if (value < 0 || value >= 1) {
      kp_set_error("reliable_delta must be in [0, 1)");
      return KP_EINVAL;
    }
    ctx->reliable_delta = value;
  } else if (!strcmp(name, "check_every")) {
    if (value < 1 || value > 64) {
      kp_set_error("check_every must be in [1, 64]");
      return KP_EINVAL;
    }
    ctx->check_every = (int)value;
  } else if (!strcmp(name, "pc_lambda_ratio")) {
    if (!(value > 0) || !std::isfinite(value)) {
      kp_set_error("pc_lambda_ratio must be > 0");
      return KP_EINVAL;
    }
    ctx->pc_lambda_ratio = value;
  } else if (!strcmp(name, "op_auto_cond")) {
    if (!(value >= 0)) {
      kp_set_error("op_auto_cond must be >= 0");
      return KP_EINVAL;
    }
    ctx->op_auto_cond = value;
  } else if (!strcmp(name, "cg_fuse")) {
    if (value != 0 && value != 1) {
      kp_set_error("cg_fuse must be 0 or 1");
      return KP_EINVAL;
    }
    ctx->cg_fuse = value != 0;
  } else if (!strcmp(name, "jacobi_tol")) {
    if (!(value > 0 && value < 1e-3)) {
      kp_set_error("jacobi_tol must be in (0, 1e-3)");
      return KP_EINVAL;
    }
    ctx->jacobi_tol = value;
  } else if (!strcmp(name, "jacobi_max_sweeps")) {
    if (value < 1 || value > 1000) {
      kp_set_error("jacobi_max_sweeps must be in [1, 1000]");
      return KP_EINVAL;
    }
    ctx->jacobi_max_sweeps = (int)value;
  } else if (!strcmp(name, "jacobi_block")) {
    if (value != 0 && value != 1) {
      kp_set_error("jacobi_block must be 0 or 1");
      return KP_EINVAL;
    }
    ctx->jacobi_block = value != 0;
  } else if (!strcmp(name, "jacobi_warm_u")) {
    if (value != 0 && value != 1) {
      kp_set_error("jacobi_warm_u must be 0 or 1");
      return KP_EINVAL;
    }
    ctx->jacobi_warm_u = value != 0;
  } else if (!strcmp(name, "splitk")) {
    ctx->splitk_override = (int)value;
  } else if (!strcmp(name, "pdl")) {
    ctx->pdl = value != 0.0;
  } else if (!strcmp(name, "device_loop")) {
    ctx->device_loop = value != 0.0;
  } else if (!strcmp(name, "tc_bn")) {
    ctx->tc_bn_override = (int)value;
  } else if (!strcmp(name, "tc_kblocks_per_stage")) {
    ctx->tc_kps_override = (int)value;
  } else if (!strcmp(name, "tc_ctas_per_sm")) {
    ctx->tc_cps_override = (int)value;
  } else if (!strcmp(name, "pc_inner_iters")) {
    if (!(value >= 1.0 && value <= 64.0)) {
      kp_set_error("pc_inner_iters must be in [1, 64]");
      return KP_EINVAL;
    }
    ctx->pc_inner_iters = (int)value;
  } else if (!strcmp(name, "tc_autotune")) {
    ctx->tc_autotune = value != 0.0;
  } else if (!strcmp(name, "tc_pair")) {
    ctx->tc_pair_override = (int)value;
  } else if (!strcmp(name, "tc_kcat")) {
    if (value != 0.0 && value != 1.0 && value != 2.0) {
      kp_set_error("tc_kcat must be 0, 1 or 2");
      return KP_EINVAL;
    }
    ctx->tc_kcat = (int)value;
  } else if (!strcmp(name, "tc_kcat_cluster")) {
    if (value != 1.0 && value != 4.0) {
      kp_set_error("tc_kcat_cluster must be 1 or 4");
      return KP_EINVAL;
    }
    ctx->tc_kcat_cluster = (int)value;
  } else if (!strcmp(name, "setup_fp64")) {
    ctx->force_setup_fp64 = value != 0.0;
  } else if (!strcmp(name, "setup_half")) {
    ctx->force_setup_half = value != 0.0;
  } else {
    kp_set_error("kp_set_option: unknown option '%s'", name);
    return KP_EINVAL;
  }
  return KP_OK;
}

extern "C" long long kp_launch_count(kp_ctx* ctx, int reset) {
  if (!ctx) return -1;
  long long n = ctx->launches;
  if (reset) ctx->launches = 0;
  return n;
}

static kp_status need_ready(kp_ctx* ctx) {
  if (!ctx) {
    kp_set_error("NULL context");
    return KP_EINVAL;
  }
  if (!ctx->ready) {
    kp_set_error("kp_setup has not completed on this context");
    return KP_ESTATE;
  }
  cudaSetDevice(ctx->device);
  return KP_OK;
}

extern "C" kp_status kp_get_rank(kp_ctx* ctx, int* op_rank) {
  KP_TRY(need_ready(ctx));
  if (!op_rank) {
    kp_set_error("kp_get_rank: NULL output");
    return KP_EINVAL;
  }
  *op_rank = ctx->rank;
  return KP_OK;
}

extern "C" kp_status kp_get_spectrum(kp_ctx* ctx, double* sigma) {
  KP_TRY(need_ready(ctx));
  if (!sigma) {
    kp_set_error("kp_get_spectrum: NULL output");
    return KP_EINVAL;
  }
  KP_CUDA(cudaMemcpyAsync(sigma, ctx->Sigma64, sizeof(double) * ctx->n_r * ctx->n_c, cudaMemcpyDeviceToHost,
                          ctx->stream));
  KP_CUDA(cudaStreamSynchronize(ctx->stream));
  return KP_OK;
}

extern "C" kp_status kp_get_terms(kp_ctx* ctx, double* s, double* u, double* v) {
  KP_TRY(need_ready(ctx));
  const int r = ctx->rank;
  if (s) KP_CUDA(cudaMemcpyAsync(s, ctx->s_terms, sizeof(double) * r, cudaMemcpyDeviceToHost, ctx->stream));
  if (u) KP_CUDA(cudaMemcpyAsync(u, ctx->u_terms, sizeof(double) * r * ctx->n_r, cudaMemcpyDeviceToHost, ctx->stream));
  if (v) KP_CUDA(cudaMemcpyAsync(v, ctx->v_terms, sizeof(double) * r * ctx->n_c, cudaMemcpyDeviceToHost, ctx->stream));
  KP_CUDA(cudaStreamSynchronize(ctx->stream));
  return KP_OK;
}

extern "C" kp_status kp_get_kpsvd(kp_ctx* ctx, double* sr, double* Ur, double* Vr, double* sc, double* Uc,
                                  double* Vc) {
  KP_TRY(need_ready(ctx));
  const size_t nr = ctx->n_r, nc = ctx->n_c;
  cudaStream_t st = ctx->stream;
  if (sr) KP_CUDA(cudaMemcpyAsync(sr, ctx->sr, sizeof(double) * nc, cudaMemcpyDeviceToHost, st));
  if (Ur) KP_CUDA(cudaMemcpyAsync(Ur, ctx->Ur, sizeof(double) * nc * nc, cudaMemcpyDeviceToHost, st));
  if (Vr) KP_CUDA(cudaMemcpyAsync(Vr, ctx->Vr, sizeof(double) * nc * nc, cudaMemcpyDeviceToHost, st));
  if (sc) KP_CUDA(cudaMemcpyAsync(sc, ctx->sc, sizeof(double) * nr, cudaMemcpyDeviceToHost, st));
  if (Uc) KP_CUDA(cudaMemcpyAsync(Uc, ctx->Uc, sizeof(double) * nr * nr, cudaMemcpyDeviceToHost, st));
  if (Vc) KP_CUDA(cudaMemcpyAsync(Vc, ctx->Vc, sizeof(double) * nr * nr, cudaMemcpyDeviceToHost, st));
  KP_CUDA(cudaStreamSynchronize(st));
  return KP_OK;
}

kp_status kp_check_ready(kp_ctx* ctx) { return need_ready(ctx); }
