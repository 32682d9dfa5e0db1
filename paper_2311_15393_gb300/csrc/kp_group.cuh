// Grouped launches of the vector kernels (batched solves).
//
// A vector kernel is written as a device body plus a thin __global__
// wrapper.  In recording mode (ctx->rec set) kp_launch_g keeps the launch's
// arguments instead of running it; the records of several problems at one
// position of their iteration then run as ONE launch of k_grouped, whose
// blockIdx.y selects the problem's argument set and whose blockIdx.x /
// gridDim.x are what the body sees (grid.x is the largest of the records':
// the bodies stride over their elements by gridDim.x and finish their
// reductions with the last of gridDim.x blocks, so a larger grid changes
// only the order of the partial sums).
#pragma once
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "kp_internal.h"

// a plain argument tuple (trivially copyable: it crosses to the device as bytes)
template <typename... T>
struct KTuple {
  template <class F, class... X>
  __device__ __forceinline__ void call(F f, const X&... x) const {
    f(x...);
  }
};
template <typename H, typename... T>
struct KTuple<H, T...> {
  H h;
  KTuple<T...> t;
  template <class F, class... X>
  __device__ __forceinline__ void call(F f, const X&... x) const {
    t.call(f, x..., h);
  }
};
inline KTuple<> make_ktuple() { return {}; }
template <typename H, typename... T>
inline KTuple<H, T...> make_ktuple(H h, T... t) {
  KTuple<H, T...> r;
  r.h = h;
  r.t = make_ktuple(t...);
  return r;
}

template <class BODY, typename... A>
__global__ void k_grouped(const KTuple<A...>* __restrict__ argv) {
  argv[blockIdx.y].call(BODY{});
}

template <class BODY, typename... A>
struct VecGroup {
  using Tup = KTuple<A...>;
  static size_t bytes(int n) { return sizeof(Tup) * (size_t)n; }
  static void table(const KpRec* const* r, int n, unsigned char* dst) {
    for (int i = 0; i < n; ++i) std::memcpy(dst + sizeof(Tup) * i, r[i]->blob.data(), sizeof(Tup));
  }
  static kp_status launch(kp_ctx* ctx, const KpRec* const* r, int n, const void* dev) {
    dim3 g = r[0]->grid;
    size_t sm = r[0]->smem;
    for (int i = 1; i < n; ++i) {
      g.x = std::max(g.x, r[i]->grid.x);
      sm = std::max(sm, r[i]->smem);
    }
    g.y = (unsigned)n;
    KP_CUDA(kp_launch(ctx, k_grouped<BODY, A...>, g, r[0]->block, sm, (const Tup*)dev));
    KP_LAUNCHED(ctx);
    return KP_OK;
  }
};

// kp_launch, or (recording) the launch kept for a grouped launch
template <class BODY, typename... KArgs, typename... Args>
inline cudaError_t kp_launch_g(kp_ctx* ctx, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                               Args&&... args) {
  if (!ctx->rec) return kp_launch(ctx, kernel, grid, block, smem, std::forward<Args>(args)...);
  using G = VecGroup<BODY, std::remove_cv_t<KArgs>...>;
  const typename G::Tup t = make_ktuple<std::remove_cv_t<KArgs>...>(std::remove_cv_t<KArgs>(args)...);
  KpRec r;
  r.key = reinterpret_cast<const void*>(kernel);
  r.table_bytes = &G::bytes;
  r.table = &G::table;
  r.launch = &G::launch;
  r.grid = grid;
  r.block = block;
  r.smem = smem;
  r.blob.resize(sizeof(t));
  std::memcpy(r.blob.data(), &t, sizeof(t));
  ctx->rec->recs.push_back(std::move(r));
  return cudaSuccess;
}

// functor calling a kernel body (template arguments in the body's name)
#define KP_BODY(NAME, ...)                                      \
  struct NAME {                                                 \
    template <class... X>                                       \
    __device__ __forceinline__ void operator()(X... x) const {  \
      __VA_ARGS__(x...);                                        \
    }                                                           \
  }
