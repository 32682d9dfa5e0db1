// SIMT GEMM (FP64 / FP32) over a sum of term blocks:
//   D[m][n] = sum_p sum_k sum_kk A[sa_p * a_terms + k][m][kk] * B[sb_p * b_terms + k][n][kk]
// with A and B K-major.  This is the all-FP64 / all-FP32 form of the
// Kronecker-sum contractions A vec(X) = vec(sum_k A_c^(k) X A_r^(k)^T)
// (Section 3; eq. KronSumDecomp) and of the preconditioner solve
// (eq. PreconSolve); the tensor-core path is in kp_gemm_tc.cu.
#include <algorithm>

#include "kp_internal.h"

namespace {

constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
constexpr int THREADS = (BM / TM) * (BN / TN);  // 256

template <typename T>
struct SimtParams {
  const T* A;
  const T* B;
  int M, N, K;
  long long lda, ldb, a_ts, b_ts;
  int nkron, npairs, a_terms, b_terms;
  int sa[KP_MAX_PAIRS], sb[KP_MAX_PAIRS];
  EpiParams epi;
  const int* flags;
  // > 1: the (pair, term, k-tile) steps are split over blockIdx.z; split s
  // writes its partial tile to ws[s][M][N] and simt_split_finish adds the
  // splits in order and applies the epilogue
  int splits;
  T* ws;
};

// fused output of one element (the epilogue of both forms)
template <typename T>
__device__ __forceinline__ void simt_store(const SimtParams<T>& p, int gm, int gn, T accv) {
  const EpiParams& e = p.epi;
  T* out = (T*)e.out;
  const T* aux = (const T*)e.aux;
  const long long idx = (long long)gm * e.ldd + gn;
  double v = (double)e.alpha * (double)accv;
  if (aux) v += (double)e.beta * (double)aux[(long long)gm * e.ld_aux + gn];
  if (e.sigma64) {
    double s = e.sigma64[idx];
    v *= e.lam2 / (s * s + e.lam2);
  }
  out[idx] = (T)v;
}

template <typename T>
__global__ void __launch_bounds__(THREADS) simt_gemm_kernel(SimtParams<T> p) {
  if (p.flags && *(volatile const int*)p.flags) return;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

  // this block's steps: pairs outermost, then terms, then k-tiles (with one
  // split, the order of the unsplit sum)
  const int ktiles = (p.K + BK - 1) / BK;
  const int steps = p.npairs * p.nkron * ktiles;
  const int per = (steps + p.splits - 1) / p.splits;
  const int st0 = blockIdx.z * per, st1 = min(steps, st0 + per);
  // loader mapping: 64 rows x 16 k = 1024 elements, 4 per thread (same row)
  const int lr = tid / 4, lk = (tid % 4) * 4;
  for (int st = st0; st < st1; ++st) {
    const int k0 = (st % ktiles) * BK;
    const int rest = st / ktiles;
    const int k = rest % p.nkron, pr = rest / p.nkron;
    const T* Ab = p.A + (long long)(p.sa[pr] * p.a_terms + k) * p.a_ts;
    const T* Bb = p.B + (long long)(p.sb[pr] * p.b_terms + k) * p.b_ts;
    {
      const int gm = m0 + lr;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int gk = k0 + lk + u;
        As[lk + u][lr] = (gm < p.M && gk < p.K) ? Ab[(long long)gm * p.lda + gk] : T(0);
      }
      const int gn = n0 + lr;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int gk = k0 + lk + u;
        Bs[lk + u][lr] = (gn < p.N && gk < p.K) ? Bb[(long long)gn * p.ldb + gk] : T(0);
      }
    }
    __syncthreads();
    // blocked summation: each k-tile of BK products is summed on its own
    // and then added to the running sum, so rounding errors grow with
    // BK + K / BK additions instead of K (the blocked / pairwise
    // summation argument of Section 4)
    T part[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) part[i][j] = T(0);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) part[i][j] = fma(a[i], b[j], part[i][j]);
    }
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] += part[i][j];
    __syncthreads();
  }
  // epilogue, or this split's partial tile
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gm = m0 + ty * TM + i;
    if (gm >= p.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = n0 + tx * TN + j;
      if (gn >= p.N) continue;
      if (p.splits > 1)
        p.ws[((long long)blockIdx.z * p.M + gm) * p.N + gn] = acc[i][j];
      else
        simt_store(p, gm, gn, acc[i][j]);
    }
  }
}

// the splits' partial tiles added in split order, then the epilogue
template <typename T>
__global__ void simt_split_finish(SimtParams<T> p) {
  if (p.flags && *(volatile const int*)p.flags) return;
  const long long mn = (long long)p.M * p.N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < mn; i += (long long)gridDim.x * blockDim.x) {
    T a = p.ws[i];
    for (int s = 1; s < p.splits; ++s) a += p.ws[(long long)s * mn + i];
    simt_store(p, (int)(i / p.N), (int)(i % p.N), a);
  }
}

}  // namespace

template <typename T>
kp_status simt_gemm(kp_ctx* ctx, const GemmDesc& g) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0) return KP_OK;
  if (g.epi.mode != EPI_T && g.epi.mode != EPI_F32) {
    kp_set_error("SIMT GEMM supports plain epilogues only");
    return KP_ENOTSUP;
  }
  SimtParams<T> p;
  p.A = (const T*)g.A.ptr;
  p.B = (const T*)g.B.ptr;
  p.M = g.M;
  p.N = g.N;
  p.K = g.K;
  p.lda = g.A.ld;
  p.ldb = g.B.ld;
  p.a_ts = g.A.tstride;
  p.b_ts = g.B.tstride;
  p.nkron = g.nkron;
  p.npairs = g.npairs;
  p.a_terms = g.a_terms;
  p.b_terms = g.b_terms;
  for (int i = 0; i < KP_MAX_PAIRS; ++i) {
    p.sa[i] = g.sa[i];
    p.sb[i] = g.sb[i];
  }
  p.epi = g.epi;
  if (p.epi.ld_aux == 0) p.epi.ld_aux = p.epi.ldd;
  p.flags = g.flags;
  dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM);
  // fewer output tiles than SMs: split the steps over blocks (FP64 runs at a
  // small fraction of the FP32 rate, so one block per tile would leave most
  // SMs idle for the whole sum), as many splits as the workspace holds
  const long long tiles = (long long)grid.x * grid.y;
  const long long steps = (long long)g.npairs * g.nkron * ((g.K + BK - 1) / BK);
  const long long mn = (long long)g.M * g.N;
  p.splits = 1;
  p.ws = nullptr;
  if (ctx->simt_ws && tiles < ctx->sm_count) {
    const long long cap = (long long)(ctx->simt_ws_bytes / sizeof(T)) / mn;
    const long long sp = std::min({(long long)ctx->sm_count / tiles, steps, cap, 256LL});
    if (sp > 1) {
      p.splits = (int)sp;
      p.ws = (T*)ctx->simt_ws;
    }
  }
  grid.z = p.splits;
  simt_gemm_kernel<T><<<grid, THREADS, 0, ctx->stream>>>(p);
  KP_LAUNCHED(ctx);
  KP_CUDA(cudaGetLastError());
  if (p.splits > 1) {
    const int fb = (int)std::min<long long>((mn + 255) / 256, (long long)ctx->sm_count * 4);
    simt_split_finish<T><<<fb, 256, 0, ctx->stream>>>(p);
    KP_LAUNCHED(ctx);
    KP_CUDA(cudaGetLastError());
  }
  return KP_OK;
}

template kp_status simt_gemm<double>(kp_ctx*, const GemmDesc&);
template kp_status simt_gemm<float>(kp_ctx*, const GemmDesc&);
