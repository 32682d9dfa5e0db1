// One-sided (Hestenes) Jacobi SVD in FP64 for the KP-SVD setup
// (eq. AKronSVD needs the SVDs of A_r and A_c; the paper used MATLAB's svd).
//
// A (m x n, column-major, m >= n) is orthogonalised column pair by column
// pair: for a pair (i, j) with alpha = |a_i|^2, beta = |a_j|^2,
// gamma = a_i . a_j, the plane rotation with
//   zeta = (beta - alpha) / (2 gamma), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
//   c = 1 / sqrt(1 + t^2), s = c t
// makes the two columns orthogonal; it is applied to A and accumulated in V.
// Pairs are visited in the round-robin (circle) order: each of the n - 1
// rounds holds n / 2 disjoint pairs, one per thread block, and a sweep is the
// n - 1 rounds, captured once as a CUDA graph.  Sweeps repeat until no pair
// needs a rotation (|gamma| <= tol sqrt(alpha beta)).  Then
// sigma_i = |a_i|, u_i = a_i / sigma_i, and the triplets are sorted by
// decreasing sigma.
#include "kp_internal.h"

namespace {

constexpr int JT = 256;

__device__ __forceinline__ double jwarp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// pair p of round `round` for npad players (circle method)
__device__ __forceinline__ int rr_player(int t, int round, int npad) {
  return t == 0 ? 0 : 1 + ((t - 1 + round) % (npad - 1));
}

__global__ void __launch_bounds__(JT) k_jacobi_round(double* __restrict__ W, double* __restrict__ V, int m, int n,
                                                     int npad, int round, double tol,
                                                     unsigned int* __restrict__ rot_count) {
  const int pidx = blockIdx.x;
  int i = rr_player(pidx, round, npad);
  int j = rr_player(npad - 1 - pidx, round, npad);
  if (i > j) {
    int t = i;
    i = j;
    j = t;
  }
  if (j >= n) return;  // pair with the padding column
  double* a = W + (long long)i * m;
  double* b = W + (long long)j * m;
  double sa = 0.0, sb = 0.0, sg = 0.0;
  for (int r = threadIdx.x; r < m; r += JT) {
    double x = a[r], y = b[r];
    sa = fma(x, x, sa);
    sb = fma(y, y, sb);
    sg = fma(x, y, sg);
  }
  __shared__ double sh[3][JT / 32];
  __shared__ double cs[2];
  sa = jwarp_sum(sa);
  sb = jwarp_sum(sb);
  sg = jwarp_sum(sg);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sh[0][wid] = sa;
    sh[1][wid] = sb;
    sh[2][wid] = sg;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double al = 0, be = 0, ga = 0;
    for (int w = 0; w < JT / 32; ++w) {
      al += sh[0][w];
      be += sh[1][w];
      ga += sh[2][w];
    }
    double c = 1.0, s = 0.0;
    if (ga != 0.0 && fabs(ga) > tol * sqrt(al) * sqrt(be)) {
      double zeta = (be - al) / (2.0 * ga);
      double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
      c = 1.0 / sqrt(1.0 + t * t);
      s = c * t;
      atomicAdd(rot_count, 1u);
    }
    cs[0] = c;
    cs[1] = s;
  }
  __syncthreads();
  const double c = cs[0], s = cs[1];
  if (s == 0.0) return;
  for (int r = threadIdx.x; r < m; r += JT) {
    double x = a[r], y = b[r];
    a[r] = c * x - s * y;
    b[r] = s * x + c * y;
  }
  double* va = V + (long long)i * n;
  double* vb = V + (long long)j * n;
  for (int r = threadIdx.x; r < n; r += JT) {
    double x = va[r], y = vb[r];
    va[r] = c * x - s * y;
    vb[r] = s * x + c * y;
  }
}

__global__ void k_set_identity(double* V, int n) {
  long long tot = (long long)n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x)
    V[t] = (t / n == t % n) ? 1.0 : 0.0;
}

__global__ void k_zero_u32(unsigned int* p) { *p = 0u; }

// column norms -> sigma (unsorted)
__global__ void __launch_bounds__(JT) k_col_norms(const double* __restrict__ W, int m, double* __restrict__ s) {
  const double* a = W + (long long)blockIdx.x * m;
  double v = 0.0;
  for (int r = threadIdx.x; r < m; r += JT) v = fma(a[r], a[r], v);
  __shared__ double sh[JT / 32];
  v = jwarp_sum(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < JT / 32; ++w) t += sh[w];
    s[blockIdx.x] = sqrt(t);
  }
}

// sort indices by decreasing sigma (ties: smaller index first); one block,
// bitonic sort of npow2 keys in shared memory
__global__ void k_sort_desc(const double* __restrict__ s, int n, int npow2, int* __restrict__ perm) {
  extern __shared__ unsigned char smem_raw[];
  double* key = (double*)smem_raw;
  int* idx = (int*)(key + npow2);
  for (int t = threadIdx.x; t < npow2; t += blockDim.x) {
    key[t] = t < n ? s[t] : -1.0;
    idx[t] = t;
  }
  __syncthreads();
  for (int k = 2; k <= npow2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < npow2; t += blockDim.x) {
        int u = t ^ j;
        if (u > t) {
          bool desc = ((t & k) == 0);
          // "a before b" when key larger, or equal key and smaller index
          double ka = key[t], kb = key[u];
          int ia = idx[t], ib = idx[u];
          bool a_first = (ka > kb) || (ka == kb && ia < ib);
          bool swap = desc ? !a_first : a_first;
          if (swap) {
            key[t] = kb;
            key[u] = ka;
            idx[t] = ib;
            idx[u] = ia;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < n; t += blockDim.x) perm[t] = idx[t];
}

// U[:, c] = W[:, perm[c]] / sigma, V_out[:, c] = V[:, perm[c]], s_out[c]
__global__ void k_gather(const double* __restrict__ W, const double* __restrict__ V, const double* __restrict__ s,
                         const int* __restrict__ perm, int m, int n, double* __restrict__ U, double* __restrict__ Vo,
                         double* __restrict__ so) {
  const int c = blockIdx.x;
  const int src = perm[c];
  const double sg = s[src];
  const double inv = sg > 0.0 ? 1.0 / sg : 0.0;
  for (int r = threadIdx.x; r < m; r += blockDim.x) U[(long long)c * m + r] = W[(long long)src * m + r] * inv;
  for (int r = threadIdx.x; r < n; r += blockDim.x) Vo[(long long)c * n + r] = V[(long long)src * n + r];
  if (threadIdx.x == 0) so[c] = sg;
}

}  // namespace

kp_status jacobi_svd(kp_ctx* ctx, const double* A, int m, int n, double* U, double* s, double* V, int* sweeps_out) {
  if (m < n || n < 1) {
    kp_set_error("jacobi_svd: need m >= n >= 1 (m=%d n=%d)", m, n);
    return KP_EINVAL;
  }
  cudaStream_t st = ctx->stream;
  double *W = nullptr, *Vw = nullptr, *sw = nullptr;
  int* perm = nullptr;
  unsigned int* cnt = nullptr;
  KP_TRY(kp_alloc(ctx, (void**)&W, sizeof(double) * (size_t)m * n));
  KP_TRY(kp_alloc(ctx, (void**)&Vw, sizeof(double) * (size_t)n * n));
  KP_TRY(kp_alloc(ctx, (void**)&sw, sizeof(double) * n));
  KP_TRY(kp_alloc(ctx, (void**)&perm, sizeof(int) * n));
  KP_TRY(kp_alloc(ctx, (void**)&cnt, sizeof(unsigned int)));
  KP_CUDA(cudaMemcpyAsync(W, A, sizeof(double) * (size_t)m * n, cudaMemcpyDeviceToDevice, st));
  k_set_identity<<<ctx->sm_count * 2, 256, 0, st>>>(Vw, n);
  KP_LAUNCHED(ctx);
  const int npad = n + (n & 1);
  int sweeps = 0;
  if (npad >= 2) {
    // capture one sweep
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    KP_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    k_zero_u32<<<1, 1, 0, st>>>(cnt);
    for (int round = 0; round < npad - 1; ++round)
      k_jacobi_round<<<npad / 2, JT, 0, st>>>(W, Vw, m, n, npad, round, ctx->jacobi_tol, cnt);
    cudaError_t ce = cudaStreamEndCapture(st, &graph);
    if (ce != cudaSuccess) {
      kp_set_error("jacobi_svd: capture failed: %s", cudaGetErrorString(ce));
      return KP_ECUDA;
    }
    KP_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    unsigned int h_cnt = 1;
    for (sweeps = 0; sweeps < ctx->jacobi_max_sweeps; ++sweeps) {
      KP_CUDA(cudaGraphLaunch(exec, st));
      ctx->launches += npad;
      KP_CUDA(cudaMemcpyAsync(&h_cnt, cnt, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
      KP_CUDA(cudaStreamSynchronize(st));
      if (h_cnt == 0) {
        ++sweeps;
        break;
      }
    }
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    if (h_cnt != 0) {
      kp_set_error("jacobi_svd: no convergence after %d sweeps (%u rotations in the last)", sweeps, h_cnt);
      return KP_ENOCONV;
    }
  }
  k_col_norms<<<n, JT, 0, st>>>(W, m, sw);
  KP_LAUNCHED(ctx);
  int npow2 = 1;
  while (npow2 < n) npow2 <<= 1;
  size_t shm = (size_t)npow2 * (sizeof(double) + sizeof(int));
  if (shm > 48 * 1024) KP_CUDA(cudaFuncSetAttribute(k_sort_desc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  k_sort_desc<<<1, 1024, shm, st>>>(sw, n, npow2, perm);
  KP_LAUNCHED(ctx);
  k_gather<<<n, 256, 0, st>>>(W, Vw, sw, perm, m, n, U, V, s);
  KP_LAUNCHED(ctx);
  KP_CUDA(cudaGetLastError());
  if (sweeps_out) *sweeps_out = sweeps;
  return KP_OK;
}
