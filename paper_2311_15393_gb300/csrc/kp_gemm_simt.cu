// SIMT GEMM (FP64 / FP32) over a sum of term blocks:
//   D[m][n] = sum_p sum_k sum_kk A[sa_p * a_terms + k][m][kk] * B[sb_p * b_terms + k][n][kk]
// with A and B K-major.  This is the all-FP64 / all-FP32 form of the
// Kronecker-sum contractions A vec(X) = vec(sum_k A_c^(k) X A_r^(k)^T)
// (Section 3; eq. KronSumDecomp) and of the preconditioner solve
// (eq. PreconSolve); the tensor-core path is in kp_gemm_tc.cu.
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
};

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

  // loader mapping: 64 rows x 16 k = 1024 elements, 4 per thread (same row)
  const int lr = tid / 4, lk = (tid % 4) * 4;
  for (int pr = 0; pr < p.npairs; ++pr) {
    for (int k = 0; k < p.nkron; ++k) {
      const T* Ab = p.A + (long long)(p.sa[pr] * p.a_terms + k) * p.a_ts;
      const T* Bb = p.B + (long long)(p.sb[pr] * p.b_terms + k) * p.b_ts;
      for (int k0 = 0; k0 < p.K; k0 += BK) {
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
    }
  }
  // epilogue
  const EpiParams& e = p.epi;
  T* out = (T*)e.out;
  const T* aux = (const T*)e.aux;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gm = m0 + ty * TM + i;
    if (gm >= p.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = n0 + tx * TN + j;
      if (gn >= p.N) continue;
      const long long idx = (long long)gm * e.ldd + gn;
      double v = (double)e.alpha * (double)acc[i][j];
      if (aux) v += (double)e.beta * (double)aux[(long long)gm * e.ld_aux + gn];
      if (e.sigma64) {
        double s = e.sigma64[idx];
        v *= e.lam2 / (s * s + e.lam2);
      }
      out[idx] = (T)v;
    }
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
  simt_gemm_kernel<T><<<grid, THREADS, 0, ctx->stream>>>(p);
  KP_LAUNCHED(ctx);
  KP_CUDA(cudaGetLastError());
  return KP_OK;
}

template kp_status simt_gemm<double>(kp_ctx*, const GemmDesc&);
template kp_status simt_gemm<float>(kp_ctx*, const GemmDesc&);
