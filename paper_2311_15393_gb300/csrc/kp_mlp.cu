// Learned lambda: a multilayer perceptron mapping the spectral features of a
// problem (kp_lambda_features) to log10(lambda), trained on problems labelled
// by the discrepancy principle.  Not part of the paper, which only asks for a
// systematic choice of the regularisation parameter (Section 5).
//
//   x -> (x - mean) * inv_std -> [Linear(in, W) -> GELU] x depth -> Linear(W, 1)
//
// Weights: FP32 masters (for Adam) and bf16 copies used by the products;
// biases and every activation and accumulation in FP32.  GELU(z) = z Phi(z).
// Loss: mean squared error of log10(lambda).  Adam with bias correction.
// The width x width products of the hidden layers (forward, weight
// gradients, input gradients) run on the tcgen05 tensor cores: FP32
// activations and gradients enter as three bf16 slices each (an exact split
// of the FP32 value), weights as their bf16 copy, with FP32 accumulation in
// TMEM, so the products keep FP32 accuracy; bias, GELU and GELU' are fused
// into the GEMM epilogue.  The scalar output layer (width -> 1) and the
// column sums of the bias gradients are small SIMT kernels.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "kp_internal.h"

struct kp_mlp {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int n_in = 256, width = 0, depth = 0, max_batch = 0, L = 0;
  std::vector<int> in, out;                      // per layer
  std::vector<float*> Wm, c, mW, vW, mc, vc, gW, gc;
  std::vector<__nv_bfloat16*> Wb;
  std::vector<float*> act, pre;                  // act[l]: input of layer l (batch x in[l]); pre[l]: its output before GELU
  float *mean = nullptr, *inv_std = nullptr;
  float *g0 = nullptr, *g1 = nullptr;            // backward ping-pong (batch x max width)
  double* loss_dev = nullptr;
  int t = 0;
  std::vector<void*> allocs;
  // tensor-core products of the hidden layers
  kp_ctx* tc = nullptr;                          // context that owns the GEMM plans (its stream is ours)
  int bpad = 0;                                  // max_batch rounded up to 8 (16-byte rows of bf16 over the batch)
  std::vector<__nv_bfloat16*> actS, actT;        // per hidden layer l: act[l] as 3 bf16 slices, and transposed
  __nv_bfloat16 *gS = nullptr, *gT = nullptr;    // the backward gradient as 3 bf16 slices, and transposed
  std::vector<__nv_bfloat16*> WbT;               // per layer: bf16 W^T (in x out)
  struct Plans {
    std::vector<TcGemmPlan*> fwd, dW, dX;
  };
  std::map<int, Plans> plans;                    // per batch size
};

namespace {

constexpr int MT = 32, NT = 32, KT = 16, MLP_THREADS = 256;

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }


enum { MEPI_STORE = 0, MEPI_BIAS = 1, MEPI_BIAS_GELU = 2, MEPI_GELU_GRAD = 3 };

// C[m][n] = sum_k A(m, k) B(k, n), A(m, k) = A[m * sam + k * sak], B(k, n) =
// B[k * sbk + n * sbn]; epilogue: + bias[n] (and GELU, keeping the sum in
// pre), or * GELU'(aux[m * ldc + n]).  32 x 32 tiles, 4 outputs per thread.
template <typename TB>
__global__ void __launch_bounds__(MLP_THREADS)
    k_mlp_gemm(int M, int N, int K, const float* __restrict__ A, long long sam, long long sak,
               const TB* __restrict__ B, long long sbk, long long sbn, float* __restrict__ C, int ldc, int epi,
               const float* __restrict__ bias, float* __restrict__ pre, const float* __restrict__ aux) {
  __shared__ float As[KT][MT + 1];
  __shared__ float Bs[KT][NT + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // 16 x 16 threads, 2 x 2 outputs each
  const int m0 = blockIdx.y * MT, n0 = blockIdx.x * NT;
  float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  for (int k0 = 0; k0 < K; k0 += KT) {
    for (int e = threadIdx.x; e < KT * MT; e += MLP_THREADS) {
      const int kk = e / MT, mm = e % MT;
      const int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < M && k < K) ? A[m * sam + k * sak] : 0.f;
    }
    for (int e = threadIdx.x; e < KT * NT; e += MLP_THREADS) {
      const int kk = e / NT, nn = e % NT;
      const int n = n0 + nn, k = k0 + kk;
      Bs[kk][nn] = (n < N && k < K) ? to_f(B[k * sbk + n * sbn]) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KT; ++kk) {
      const float a0 = As[kk][ty], a1 = As[kk][ty + 16];
      const float b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
      acc[0][0] = fmaf(a0, b0, acc[0][0]);
      acc[0][1] = fmaf(a0, b1, acc[0][1]);
      acc[1][0] = fmaf(a1, b0, acc[1][0]);
      acc[1][1] = fmaf(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (m >= M || n >= N) continue;
      float v = acc[i][j];
      const long long o = (long long)m * ldc + n;
      if (epi == MEPI_BIAS || epi == MEPI_BIAS_GELU) v += bias[n];
      if (epi == MEPI_BIAS_GELU) {
        pre[o] = v;
        v = kp_gelu(v);
      } else if (epi == MEPI_GELU_GRAD) {
        v *= kp_gelu_grad(aux[o]);
      }
      C[o] = v;
    }
  }
}

// out[b][i] = (X[b][i] - mean[i]) * inv_std[i]
__global__ void k_mlp_normalize(const float* __restrict__ X, int batch, int n, const float* __restrict__ mean,
                                const float* __restrict__ inv_std, float* __restrict__ out) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)batch * n;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % n);
    out[t] = (X[t] - mean[i]) * inv_std[i];
  }
}

// loss = mean (pred - y)^2 (FP64 sum in one block, fixed order); g = 2 (pred - y) / batch
__global__ void k_mlp_loss(const float* __restrict__ pred, const float* __restrict__ y, int batch,
                           float* __restrict__ g, double* __restrict__ loss) {
  __shared__ double sh[MLP_THREADS];
  double a = 0.0;
  for (int b = threadIdx.x; b < batch; b += blockDim.x) {
    const float d = pred[b] - y[b];
    g[b] = 2.f * d / (float)batch;
    a += (double)d * (double)d;
  }
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = sh[0] / batch;
}

// gc[o] = sum_b g[b][o]
__global__ void k_mlp_colsum(const float* __restrict__ g, int batch, int n, float* __restrict__ out) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  float a = 0.f;
  for (int b = 0; b < batch; ++b) a += g[(long long)b * n + o];
  out[o] = a;
}

// Adam on one parameter array; wb (nullable) receives the bf16 copy and wbt
// (nullable) its transpose (w is rows x cols, row-major)
__global__ void k_mlp_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ g, long long n, float lr, float b1, float b2, float eps,
                           float c1, float c2, __nv_bfloat16* __restrict__ wb, __nv_bfloat16* __restrict__ wbt,
                           int rows, int cols) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    const __nv_bfloat16 h = __float2bfloat16_rn(wi);
    if (wb) wb[i] = h;
    if (wbt) wbt[(i % cols) * rows + i / cols] = h;
  }
}

// X (rows x cols FP32, row-major) as three bf16 slices x = s0 + s1 + s2 (an
// exact split of the FP32 value): S[s][r][c] for r < rows (row stride cols,
// slice stride s_stride) and T[s][c][r] for r < rows_pad (zero for r >=
// rows; row stride t_ld, slice stride t_stride)
__global__ void k_mlp_slices(const float* __restrict__ X, int rows, int cols, int rows_pad,
                             __nv_bfloat16* __restrict__ S, long long s_stride, __nv_bfloat16* __restrict__ T,
                             int t_ld, long long t_stride) {
  const long long tot = (long long)rows_pad * cols;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t / cols), c = (int)(t % cols);
    float v = r < rows ? X[t] : 0.f;
    for (int sl = 0; sl < 3; ++sl) {
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      v -= __bfloat162float(h);
      if (S && r < rows) S[sl * s_stride + t] = h;
      if (T) T[sl * t_stride + (long long)c * t_ld + r] = h;
    }
  }
}

// bf16 copy of w (rows x cols, row-major) and of its transpose
__global__ void k_mlp_to_bf16(const float* __restrict__ w, long long n, __nv_bfloat16* __restrict__ wb,
                              __nv_bfloat16* __restrict__ wbt, int rows, int cols) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const __nv_bfloat16 h = __float2bfloat16_rn(w[i]);
    wb[i] = h;
    wbt[(i % cols) * rows + i / cols] = h;
  }
}

template <typename TB>
kp_status gemm(kp_mlp* p, int M, int N, int K, const float* A, long long sam, long long sak, const TB* B, long long sbk,
               long long sbn, float* C, int ldc, int epi, const float* bias, float* pre, const float* aux) {
  dim3 grid((N + NT - 1) / NT, (M + MT - 1) / MT);
  k_mlp_gemm<TB><<<grid, MLP_THREADS, 0, p->stream>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, epi, bias, pre, aux);
  KP_CUDA(cudaGetLastError());
  return KP_OK;
}

// operand of a tensor-core product: rows x K bf16, `slices` blocks of
// `tstride` elements
GemmOp op_of(const void* ptr, int rows, int K, long long ld, long long tstride, int slices) {
  GemmOp o;
  o.ptr = ptr;
  o.rows = rows;
  o.K = K;
  o.ld = ld;
  o.tstride = tstride;
  o.nterm_idx = slices;
  return o;
}

// the tensor-core plans of one batch size (built at its first use)
kp_status plans_for(kp_mlp* p, int batch, kp_mlp::Plans** out) {
  auto it = p->plans.find(batch);
  if (it != p->plans.end()) {
    *out = &it->second;
    return KP_OK;
  }
  kp_mlp::Plans P;
  const int bp = (batch + 7) / 8 * 8;
  const int w = p->width;
  static const int acc_a[6] = {0, 0, 1, 0, 1, 2}, acc_b[6] = {0, 1, 0, 2, 1, 0};
  for (int l = 0; l < p->L - 1; ++l) {
    const int in = p->in[l];
    // forward: act[l + 1] = GELU(sum_s S_s(act[l]) W_l^T + c_l), pre[l] keeps the sum
    GemmDesc f;
    f.M = batch;
    f.N = w;
    f.K = in;
    f.npairs = 3;
    for (int q = 0; q < 3; ++q) {
      f.sa[q] = q;
      f.sb[q] = 0;
    }
    f.A = op_of(p->actS[l], batch, in, in, (long long)p->bpad * in, 3);
    f.B = op_of(p->Wb[l], w, in, in, (long long)w * in, 1);
    f.epi.mode = EPI_F32;
    f.epi.out = p->act[l + 1];
    f.epi.ldd = w;
    f.epi.bias = p->c[l];
    f.epi.pre = p->pre[l];
    f.epi.act = 1;
    TcGemmPlan* pf = nullptr;
    KP_TRY(tc_plan_create(p->tc, f, TC_BF16, 1, &pf));
    P.fwd.push_back(pf);
    // weight gradient: gW_l[o][i] = sum_b g[b][o] act_l[b][i] over the padded batch (six slice pairs)
    GemmDesc d;
    d.M = w;
    d.N = in;
    d.K = bp;
    d.npairs = 6;
    for (int q = 0; q < 6; ++q) {
      d.sa[q] = acc_a[q];
      d.sb[q] = acc_b[q];
    }
    d.A = op_of(p->gT, w, bp, p->bpad, (long long)w * p->bpad, 3);
    d.B = op_of(p->actT[l], in, bp, p->bpad, (long long)in * p->bpad, 3);
    d.epi.mode = EPI_F32;
    d.epi.out = p->gW[l];
    d.epi.ldd = in;
    TcGemmPlan* pd = nullptr;
    KP_TRY(tc_plan_create(p->tc, d, TC_BF16, 1, &pd));
    P.dW.push_back(pd);
    // input gradient (l > 0): gn[b][i] = (sum_o g[b][o] W_l[o][i]) GELU'(pre_(l-1)[b][i])
    TcGemmPlan* px = nullptr;
    if (l > 0) {
      GemmDesc x;
      x.M = batch;
      x.N = in;
      x.K = w;
      x.npairs = 3;
      for (int q = 0; q < 3; ++q) {
        x.sa[q] = q;
        x.sb[q] = 0;
      }
      x.A = op_of(p->gS, batch, w, w, (long long)p->bpad * w, 3);
      x.B = op_of(p->WbT[l], in, w, w, (long long)in * w, 1);
      x.epi.mode = EPI_F32;
      x.epi.out = nullptr;  // set per call (ping-pong buffer)
      x.epi.ldd = in;
      x.epi.pre = p->pre[l - 1];
      x.epi.act = 2;
      KP_TRY(tc_plan_create(p->tc, x, TC_BF16, 1, &px));
    }
    P.dX.push_back(px);
  }
  auto ins = p->plans.emplace(batch, P);
  *out = &ins.first->second;
  return KP_OK;
}

kp_status slices(kp_mlp* p, const float* X, int batch, int cols, __nv_bfloat16* S, __nv_bfloat16* T) {
  const int bp = (batch + 7) / 8 * 8;
  const long long tot = (long long)bp * cols;
  const int g = (int)std::max(1LL, std::min((tot + 255) / 256, 2048LL));
  k_mlp_slices<<<g, 256, 0, p->stream>>>(X, batch, cols, bp, S, (long long)p->bpad * cols, T, p->bpad,
                                         (long long)cols * p->bpad);
  KP_CUDA(cudaGetLastError());
  return KP_OK;
}

kp_status forward(kp_mlp* p, const float* X, int batch) {
  const int g = std::max(1, std::min((batch * p->n_in + 255) / 256, 1024));
  k_mlp_normalize<<<g, 256, 0, p->stream>>>(X, batch, p->n_in, p->mean, p->inv_std, p->act[0]);
  kp_mlp::Plans* P = nullptr;
  KP_TRY(plans_for(p, batch, &P));
  for (int l = 0; l < p->L - 1; ++l) {
    // act[l + 1] = GELU(act[l] W_l^T + c_l) on the tensor cores (pre[l] keeps the sum)
    KP_TRY(slices(p, p->act[l], batch, p->in[l], p->actS[l], p->actT[l]));
    KP_TRY(tc_plan_run(p->tc, P->fwd[l], nullptr));
  }
  // the scalar output layer: act[L] = act[L - 1] W^T + c (no GELU)
  const int l = p->L - 1;
  KP_TRY(gemm<__nv_bfloat16>(p, batch, p->out[l], p->in[l], p->act[l], p->in[l], 1, p->Wb[l], 1, p->in[l],
                             p->act[l + 1], p->out[l], MEPI_BIAS, p->c[l], p->pre[l], nullptr));
  return KP_OK;
}

// loss and the gradients of every weight and bias into gW / gc
kp_status backward(kp_mlp* p, const float* X, const float* y, int batch) {
  KP_TRY(forward(p, X, batch));
  kp_mlp::Plans* P = nullptr;
  KP_TRY(plans_for(p, batch, &P));
  float* g = p->g0;
  float* gn = p->g1;
  k_mlp_loss<<<1, MLP_THREADS, 0, p->stream>>>(p->act[p->L], y, batch, g, p->loss_dev);
  for (int l = p->L - 1; l >= 0; --l) {
    if (l == p->L - 1) {
      // the scalar output layer (SIMT): gW[0][i] = sum_b g[b] act_l[b][i]
      KP_TRY(gemm<float>(p, p->out[l], p->in[l], batch, g, 1, p->out[l], p->act[l], p->in[l], 1, p->gW[l], p->in[l],
                         MEPI_STORE, nullptr, nullptr, nullptr));
    } else {
      // gW_l[o][i] = sum_b g[b][o] act_l[b][i] on the tensor cores
      KP_TRY(slices(p, g, batch, p->out[l], p->gS, p->gT));
      KP_TRY(tc_plan_run(p->tc, P->dW[l], nullptr));
    }
    // gc_l[o] = sum_b g[b][o]
    k_mlp_colsum<<<(p->out[l] + 255) / 256, 256, 0, p->stream>>>(g, batch, p->out[l], p->gc[l]);
    if (l > 0) {
      // gn[b][i] = (sum_o g[b][o] W_l[o][i]) GELU'(pre_(l-1)[b][i])
      if (l == p->L - 1) {
        KP_TRY(gemm<__nv_bfloat16>(p, batch, p->in[l], p->out[l], g, p->out[l], 1, p->Wb[l], p->in[l], 1, gn,
                                   p->in[l], MEPI_GELU_GRAD, nullptr, nullptr, p->pre[l - 1]));
      } else {
        EpiParams e;
        e.mode = EPI_F32;
        e.out = gn;
        e.ldd = p->in[l];
        e.pre = p->pre[l - 1];
        e.act = 2;
        KP_TRY(tc_plan_run(p->tc, P->dX[l], &e));
      }
      std::swap(g, gn);
    }
  }
  KP_CUDA(cudaGetLastError());
  return KP_OK;
}

kp_status mlp_alloc(kp_mlp* p, void** ptr, size_t bytes) {
  if (cudaMalloc(ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    kp_set_error("kp_mlp: cudaMalloc of %zu bytes failed", bytes);
    return KP_ENOMEM;
  }
  p->allocs.push_back(*ptr);
  KP_CUDA(cudaMemsetAsync(*ptr, 0, bytes, p->stream));
  return KP_OK;
}

long long param_count(const kp_mlp* p) {
  long long n = 2LL * p->n_in;
  for (int l = 0; l < p->L; ++l) n += (long long)p->out[l] * p->in[l] + p->out[l];
  return n;
}

}  // namespace

extern "C" kp_status kp_mlp_create(kp_mlp** out, int device, void* cuda_stream, int width, int depth, int max_batch) {
  if (!out || width < 1 || width > 4096 || depth < 1 || depth > 16 || max_batch < 1 || max_batch > 65536) {
    kp_set_error("kp_mlp_create: need out, 1 <= width <= 4096, 1 <= depth <= 16, 1 <= max_batch <= 65536");
    return KP_EINVAL;
  }
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) {
    kp_set_error("kp_mlp_create: cudaSetDevice(%d) failed", device);
    return KP_ECUDA;
  }
  kp_mlp* p = new kp_mlp();
  p->device = device;
  p->width = width;
  p->depth = depth;
  p->max_batch = max_batch;
  p->L = depth + 1;
  if (cuda_stream) {
    p->stream = (cudaStream_t)cuda_stream;
  } else {
    p->own_stream = true;
    if (cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete p;
      kp_set_error("kp_mlp_create: stream creation failed");
      return KP_ECUDA;
    }
  }
  for (int l = 0; l < p->L; ++l) {
    p->in.push_back(l == 0 ? p->n_in : width);
    p->out.push_back(l == p->L - 1 ? 1 : width);
  }
  auto fail = [&](kp_status s) {
    kp_mlp_destroy(p);
    return s;
  };
  auto af = [&](float** q, long long n) { return mlp_alloc(p, (void**)q, sizeof(float) * (size_t)n); };
  kp_status s = KP_OK;
  s = af(&p->mean, p->n_in);
  if (s == KP_OK) s = af(&p->inv_std, p->n_in);
  const int wmax = std::max(width, p->n_in);
  if (s == KP_OK) s = af(&p->g0, (long long)max_batch * wmax);
  if (s == KP_OK) s = af(&p->g1, (long long)max_batch * wmax);
  if (s == KP_OK) s = mlp_alloc(p, (void**)&p->loss_dev, sizeof(double));
  p->act.assign(p->L + 1, nullptr);
  p->pre.assign(p->L, nullptr);
  for (int l = 0; l <= p->L && s == KP_OK; ++l) s = af(&p->act[l], (long long)max_batch * (l < p->L ? p->in[l] : 1));
  for (int l = 0; l < p->L && s == KP_OK; ++l) {
    const long long nw = (long long)p->out[l] * p->in[l];
    float *w, *cc, *m1, *v1, *m2, *v2, *gw, *gcc, *pr;
    __nv_bfloat16* wb;
    s = af(&w, nw);
    if (s == KP_OK) s = af(&cc, p->out[l]);
    if (s == KP_OK) s = af(&m1, nw);
    if (s == KP_OK) s = af(&v1, nw);
    if (s == KP_OK) s = af(&m2, p->out[l]);
    if (s == KP_OK) s = af(&v2, p->out[l]);
    if (s == KP_OK) s = af(&gw, nw);
    if (s == KP_OK) s = af(&gcc, p->out[l]);
    if (s == KP_OK) s = af(&pr, (long long)max_batch * p->out[l]);
    if (s == KP_OK) s = mlp_alloc(p, (void**)&wb, sizeof(__nv_bfloat16) * (size_t)nw);
    if (s != KP_OK) break;
    p->Wm.push_back(w);
    p->c.push_back(cc);
    p->mW.push_back(m1);
    p->vW.push_back(v1);
    p->mc.push_back(m2);
    p->vc.push_back(v2);
    p->gW.push_back(gw);
    p->gc.push_back(gcc);
    p->pre[l] = pr;
    p->Wb.push_back(wb);
  }
  // tensor-core products: the context that owns their plans, the operand slices
  p->bpad = (max_batch + 7) / 8 * 8;
  if (s == KP_OK) s = kp_create(&p->tc, device, p->stream);
  if (s == KP_OK && !tc_device_supported(p->tc)) {
    kp_set_error("kp_mlp_create: the tensor-core products need an sm_103 device");
    s = KP_ENOTSUP;
  }
  auto ab = [&](__nv_bfloat16** q, long long n) { return mlp_alloc(p, (void**)q, sizeof(__nv_bfloat16) * (size_t)n); };
  for (int l = 0; l < p->L - 1 && s == KP_OK; ++l) {
    __nv_bfloat16 *aS = nullptr, *aT = nullptr;
    s = ab(&aS, 3LL * p->bpad * p->in[l]);
    if (s == KP_OK) s = ab(&aT, 3LL * p->bpad * p->in[l]);
    p->actS.push_back(aS);
    p->actT.push_back(aT);
  }
  if (s == KP_OK) s = ab(&p->gS, 3LL * p->bpad * width);
  if (s == KP_OK) s = ab(&p->gT, 3LL * p->bpad * width);
  for (int l = 0; l < p->L && s == KP_OK; ++l) {
    __nv_bfloat16* t = nullptr;
    s = ab(&t, (long long)p->out[l] * p->in[l]);
    p->WbT.push_back(t);
  }
  if (s != KP_OK) return fail(s);
  *out = p;
  return KP_OK;
}

extern "C" void kp_mlp_destroy(kp_mlp* p) {
  if (!p) return;
  cudaSetDevice(p->device);
  if (p->stream) cudaStreamSynchronize(p->stream);
  if (p->tc) kp_destroy(p->tc);
  for (void* a : p->allocs) cudaFree(a);
  if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
  delete p;
}

extern "C" long long kp_mlp_param_count(const kp_mlp* p) { return p ? param_count(p) : -1; }

// parameter vector: mean (n_in), inv_std (n_in), then per layer W (out x in,
// row-major) and c (out)
extern "C" kp_status kp_mlp_set_params(kp_mlp* p, const float* params) {
  if (!p || !params) {
    kp_set_error("kp_mlp_set_params: NULL argument");
    return KP_EINVAL;
  }
  cudaSetDevice(p->device);
  const float* q = params;
  KP_CUDA(cudaMemcpyAsync(p->mean, q, sizeof(float) * p->n_in, cudaMemcpyHostToDevice, p->stream));
  q += p->n_in;
  KP_CUDA(cudaMemcpyAsync(p->inv_std, q, sizeof(float) * p->n_in, cudaMemcpyHostToDevice, p->stream));
  q += p->n_in;
  for (int l = 0; l < p->L; ++l) {
    const long long nw = (long long)p->out[l] * p->in[l];
    KP_CUDA(cudaMemcpyAsync(p->Wm[l], q, sizeof(float) * nw, cudaMemcpyHostToDevice, p->stream));
    q += nw;
    KP_CUDA(cudaMemcpyAsync(p->c[l], q, sizeof(float) * p->out[l], cudaMemcpyHostToDevice, p->stream));
    q += p->out[l];
    k_mlp_to_bf16<<<std::max(1LL, std::min((nw + 255) / 256, 1024LL)), 256, 0, p->stream>>>(p->Wm[l], nw, p->Wb[l],
                                                                                              p->WbT[l], p->out[l],
                                                                                              p->in[l]);
    KP_CUDA(cudaMemsetAsync(p->mW[l], 0, sizeof(float) * nw, p->stream));
    KP_CUDA(cudaMemsetAsync(p->vW[l], 0, sizeof(float) * nw, p->stream));
    KP_CUDA(cudaMemsetAsync(p->mc[l], 0, sizeof(float) * p->out[l], p->stream));
    KP_CUDA(cudaMemsetAsync(p->vc[l], 0, sizeof(float) * p->out[l], p->stream));
  }
  p->t = 0;
  KP_CUDA(cudaStreamSynchronize(p->stream));  // params is a host buffer the caller may reuse
  return KP_OK;
}

extern "C" kp_status kp_mlp_get_params(kp_mlp* p, float* params) {
  if (!p || !params) {
    kp_set_error("kp_mlp_get_params: NULL argument");
    return KP_EINVAL;
  }
  cudaSetDevice(p->device);
  float* q = params;
  KP_CUDA(cudaMemcpyAsync(q, p->mean, sizeof(float) * p->n_in, cudaMemcpyDeviceToHost, p->stream));
  q += p->n_in;
  KP_CUDA(cudaMemcpyAsync(q, p->inv_std, sizeof(float) * p->n_in, cudaMemcpyDeviceToHost, p->stream));
  q += p->n_in;
  for (int l = 0; l < p->L; ++l) {
    const long long nw = (long long)p->out[l] * p->in[l];
    KP_CUDA(cudaMemcpyAsync(q, p->Wm[l], sizeof(float) * nw, cudaMemcpyDeviceToHost, p->stream));
    q += nw;
    KP_CUDA(cudaMemcpyAsync(q, p->c[l], sizeof(float) * p->out[l], cudaMemcpyDeviceToHost, p->stream));
    q += p->out[l];
  }
  KP_CUDA(cudaStreamSynchronize(p->stream));
  return KP_OK;
}

static kp_status check_batch(kp_mlp* p, const void* X, int batch, const char* who) {
  if (!p || !X || batch < 1 || batch > p->max_batch) {
    kp_set_error("%s: need a model, X and 1 <= batch <= max_batch", who);
    return KP_EINVAL;
  }
  if (cudaSetDevice(p->device) != cudaSuccess) {
    kp_set_error("%s: cudaSetDevice failed", who);
    return KP_ECUDA;
  }
  return KP_OK;
}

extern "C" kp_status kp_mlp_forward(kp_mlp* p, const float* X, int batch, float* y) {
  KP_TRY(check_batch(p, X, batch, "kp_mlp_forward"));
  if (!y) {
    kp_set_error("kp_mlp_forward: NULL output");
    return KP_EINVAL;
  }
  KP_TRY(forward(p, X, batch));
  KP_CUDA(cudaMemcpyAsync(y, p->act[p->L], sizeof(float) * batch, cudaMemcpyDeviceToDevice, p->stream));
  return KP_OK;
}

extern "C" kp_status kp_mlp_gradients(kp_mlp* p, const float* X, const float* y, int batch, float* grads,
                                      double* loss) {
  KP_TRY(check_batch(p, X, batch, "kp_mlp_gradients"));
  if (!y || !grads) {
    kp_set_error("kp_mlp_gradients: NULL argument");
    return KP_EINVAL;
  }
  KP_TRY(backward(p, X, y, batch));
  float* q = grads;
  std::memset(q, 0, sizeof(float) * 2 * p->n_in);  // no gradient for the fixed normalisation
  q += 2 * p->n_in;
  for (int l = 0; l < p->L; ++l) {
    const long long nw = (long long)p->out[l] * p->in[l];
    KP_CUDA(cudaMemcpyAsync(q, p->gW[l], sizeof(float) * nw, cudaMemcpyDeviceToHost, p->stream));
    q += nw;
    KP_CUDA(cudaMemcpyAsync(q, p->gc[l], sizeof(float) * p->out[l], cudaMemcpyDeviceToHost, p->stream));
    q += p->out[l];
  }
  if (loss) KP_CUDA(cudaMemcpyAsync(loss, p->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  KP_CUDA(cudaStreamSynchronize(p->stream));
  return KP_OK;
}

extern "C" kp_status kp_mlp_train_step(kp_mlp* p, const float* X, const float* y, int batch, float lr,
                                       double* loss) {
  KP_TRY(check_batch(p, X, batch, "kp_mlp_train_step"));
  if (!y || !(lr > 0.f)) {
    kp_set_error("kp_mlp_train_step: need y and lr > 0");
    return KP_EINVAL;
  }
  KP_TRY(backward(p, X, y, batch));
  ++p->t;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = (float)(1.0 - std::pow(0.9, p->t)), c2 = (float)(1.0 - std::pow(0.999, p->t));
  for (int l = 0; l < p->L; ++l) {
    const long long nw = (long long)p->out[l] * p->in[l];
    k_mlp_adam<<<std::max(1LL, std::min((nw + 255) / 256, 1024LL)), 256, 0, p->stream>>>(
        p->Wm[l], p->mW[l], p->vW[l], p->gW[l], nw, lr, b1, b2, eps, c1, c2, p->Wb[l], p->WbT[l], p->out[l],
        p->in[l]);
    k_mlp_adam<<<1, 256, 0, p->stream>>>(p->c[l], p->mc[l], p->vc[l], p->gc[l], p->out[l], lr, b1, b2, eps, c1, c2,
                                         nullptr, nullptr, 1, p->out[l]);
  }
  KP_CUDA(cudaGetLastError());
  if (loss) {
    KP_CUDA(cudaMemcpyAsync(loss, p->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    KP_CUDA(cudaStreamSynchronize(p->stream));
  }
  return KP_OK;
}
