// kp_apply_Minv_noalloc: the FP32 preconditioner solve
//   z = V_c (S .* (V_c^T R V_r)) V_r^T,  S = 1 / (Sigma^2 + lambda^2),
// for callers that cannot allocate device memory.
//
// Everything it needs besides the caller's inputs and outputs lives in one
// file-scope device array of fixed size, so the call makes no allocation of
// any kind.  Host code cannot use the array's name as a device address: at
// the first call on a device the address is looked up with
// cudaGetSymbolAddress (with that device current) and cached per device.
// Every call shares the array, so calls that overlap on the GPU (e.g. on
// two streams at once) race with each other.
#include <mutex>

#include "kp_internal.h"

// largest image this entry point accepts, and the scratch it needs:
// three n_r x n_c intermediates plus transposed copies of V_c and V_r
#define KP_NOALLOC_MAX_SIDE 512
#define KP_NOALLOC_MAX_PIXELS (KP_NOALLOC_MAX_SIDE * KP_NOALLOC_MAX_SIDE)
#define KP_NOALLOC_SCRATCH_FLOATS (5 * KP_NOALLOC_MAX_PIXELS)  // 5 MiB

static __device__ __align__(256) float g_noalloc_scratch[KP_NOALLOC_SCRATCH_FLOATS];

namespace {

constexpr int KP_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
float* g_noalloc_ptr[KP_MAX_DEVICES] = {nullptr};

// out (row-major n x n) = in (column-major n x n), i.e. out[a][b] = in[a + n b]
__global__ void k_noalloc_transpose(const float* __restrict__ in, int n, float* __restrict__ out) {
  const long long tot = (long long)n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(t / n), b = (int)(t % n);
    out[t] = in[a + (long long)n * b];
  }
}

// device address of the scratch array for the current device (looked up once)
kp_status scratch_address(float** out) {
  int dev = 0;
  KP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= KP_MAX_DEVICES) {
    kp_set_error("kp_apply_Minv_noalloc: device index %d out of range", dev);
    return KP_ENOTSUP;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      kp_set_error("kp_apply_Minv_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return KP_ECUDA;
    }
    g_noalloc_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return KP_OK;
}

}  // namespace

extern "C" kp_status kp_apply_Minv_noalloc(const float* Vc, const float* Vr, const double* sigma, int n_r, int n_c,
                                           double lambda, const float* r, float* z, void* cuda_stream) {
  if (!Vc || !Vr || !sigma || !r || !z || r == z) {
    kp_set_error("kp_apply_Minv_noalloc: NULL or aliased pointer");
    return KP_EINVAL;
  }
  if (!(lambda > 0.0)) {
    kp_set_error("kp_apply_Minv_noalloc: need lambda > 0");
    return KP_EINVAL;
  }
  if (n_r < 1 || n_c < 1 || n_r > KP_NOALLOC_MAX_SIDE || n_c > KP_NOALLOC_MAX_SIDE) {
    kp_set_error("kp_apply_Minv_noalloc: image %d x %d exceeds the fixed scratch (at most %d x %d)", n_r, n_c,
                 KP_NOALLOC_MAX_SIDE, KP_NOALLOC_MAX_SIDE);
    return KP_EINVAL;
  }
  {  // the scratch address is per device: the stream must run on the current one
    int cur = 0, sdev = 0;
    KP_CUDA(cudaGetDevice(&cur));
    KP_CUDA(cudaStreamGetDevice(static_cast<cudaStream_t>(cuda_stream), &sdev));
    if (sdev != cur) {
      kp_set_error("kp_apply_Minv_noalloc: the stream belongs to device %d, the current device is %d", sdev, cur);
      return KP_EINVAL;
    }
  }
  float* scratch = nullptr;
  KP_TRY(scratch_address(&scratch));
  const long long N = (long long)n_r * n_c;
  float* t1 = scratch;                   // V_c^T R          (row-major n_r x n_c)
  float* t2 = t1 + N;                    // S .* (T1 V_r)     (column-major)
  float* t3 = t2 + N;                    // V_c W             (row-major)
  float* vc_rm = t3 + N;                 // V_c row-major (n_r x n_r)
  float* vr_rm = vc_rm + (long long)n_r * n_r;  // V_r row-major (n_c x n_c)

  // a stack context carries the stream for the GEMM launcher; it owns no memory
  kp_ctx host;
  host.stream = static_cast<cudaStream_t>(cuda_stream);
  const int g = 256;
  k_noalloc_transpose<<<g, 256, 0, host.stream>>>(Vc, n_r, vc_rm);
  k_noalloc_transpose<<<g, 256, 0, host.stream>>>(Vr, n_c, vr_rm);
  KP_CUDA(cudaGetLastError());

  // the four products of the preconditioner solve, all operands K-major
  for (int w = 0; w < 4; ++w) {
    GemmDesc d;
    d.epi.mode = EPI_T;
    if (w == 0 || w == 2) {  // T1 = V_c^T R ; T3 = V_c W
      d.M = n_r;
      d.N = n_c;
      d.K = n_r;
      d.A.ptr = w == 0 ? Vc : vc_rm;  // V_c^T row-major is V_c column-major
      d.A.ld = n_r;
      d.B.ptr = w == 0 ? r : t2;
      d.B.ld = n_r;
      d.epi.out = w == 0 ? t1 : t3;
      d.epi.ldd = n_c;
    } else {  // T2^T = V_r^T T1^T (scaled by S) ; Z^T = V_r T3^T
      d.M = n_c;
      d.N = n_r;
      d.K = n_c;
      d.A.ptr = w == 1 ? Vr : vr_rm;
      d.A.ld = n_c;
      d.B.ptr = w == 1 ? t1 : t3;
      d.B.ld = n_c;
      d.epi.out = w == 1 ? t2 : z;
      d.epi.ldd = n_r;
      if (w == 1) {
        d.epi.sigma64 = sigma;
        d.epi.lam2 = lambda * lambda;
      } else {
        d.epi.alpha = 1.0 / (lambda * lambda);
      }
    }
    KP_TRY(simt_gemm<float>(&host, d));
  }
  return KP_OK;
}
