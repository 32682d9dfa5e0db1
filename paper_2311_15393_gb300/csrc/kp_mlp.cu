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
// All products are small (batch x 256 x 256), so one tiled SIMT kernel with
// strided operand access serves the forward pass and both backward products.
#include <algorithm>
#include <cmath>
#include <cstring>
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
};

namespace {

constexpr int MT = 32, NT = 32, KT = 16, MLP_THREADS = 256;

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ float phi(float z) { return 0.5f * erfcf(-z * 0.70710678118654752f); }
__device__ __forceinline__ float gelu(float z) { return z * phi(z); }
__device__ __forceinline__ float gelu_grad(float z) {
  return phi(z) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

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
        v = gelu(v);
      } else if (epi == MEPI_GELU_GRAD) {
        v *= gelu_grad(aux[o]);
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

// Adam on one parameter array; wb (nullable) receives the bf16 copy
__global__ void k_mlp_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ g, long long n, float lr, float b1, float b2, float eps,
                           float c1, float c2, __nv_bfloat16* __restrict__ wb) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16_rn(wi);
  }
}

__global__ void k_mlp_to_bf16(const float* __restrict__ w, long long n, __nv_bfloat16* __restrict__ wb) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    wb[i] = __float2bfloat16_rn(w[i]);
}

template <typename TB>
kp_status gemm(kp_mlp* p, int M, int N, int K, const float* A, long long sam, long long sak, const TB* B, long long sbk,
               long long sbn, float* C, int ldc, int epi, const float* bias, float* pre, const float* aux) {
  dim3 grid((N + NT - 1) / NT, (M + MT - 1) / MT);
  k_mlp_gemm<TB><<<grid, MLP_THREADS, 0, p->stream>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, epi, bias, pre, aux);
  KP_CUDA(cudaGetLastError());
  return KP_OK;
}

kp_status forward(kp_mlp* p, const float* X, int batch) {
  const int g = std::max(1, std::min((batch * p->n_in + 255) / 256, 1024));
  k_mlp_normalize<<<g, 256, 0, p->stream>>>(X, batch, p->n_in, p->mean, p->inv_std, p->act[0]);
  for (int l = 0; l < p->L; ++l) {
    const bool last = l == p->L - 1;
    // act[l + 1] = GELU(act[l] W_l^T + c_l) (pre[l] keeps the sum); the last layer has no GELU
    KP_TRY(gemm<__nv_bfloat16>(p, batch, p->out[l], p->in[l], p->act[l], p->in[l], 1, p->Wb[l], 1, p->in[l],
                               p->act[l + 1], p->out[l], last ? MEPI_BIAS : MEPI_BIAS_GELU, p->c[l], p->pre[l],
                               nullptr));
  }
  return KP_OK;
}

// loss and the gradients of every weight and bias into gW / gc
kp_status backward(kp_mlp* p, const float* X, const float* y, int batch) {
  KP_TRY(forward(p, X, batch));
  float* g = p->g0;
  float* gn = p->g1;
  k_mlp_loss<<<1, MLP_THREADS, 0, p->stream>>>(p->act[p->L], y, batch, g, p->loss_dev);
  for (int l = p->L - 1; l >= 0; --l) {
    // gW_l[o][i] = sum_b g[b][o] act_l[b][i] ; gc_l[o] = sum_b g[b][o]
    KP_TRY(gemm<float>(p, p->out[l], p->in[l], batch, g, 1, p->out[l], p->act[l], p->in[l], 1, p->gW[l], p->in[l],
                       MEPI_STORE, nullptr, nullptr, nullptr));
    k_mlp_colsum<<<(p->out[l] + 255) / 256, 256, 0, p->stream>>>(g, batch, p->out[l], p->gc[l]);
    if (l > 0) {
      // gn[b][i] = (sum_o g[b][o] W_l[o][i]) GELU'(pre_(l-1)[b][i])
      KP_TRY(gemm<__nv_bfloat16>(p, batch, p->in[l], p->out[l], g, p->out[l], 1, p->Wb[l], p->in[l], 1, gn,
                                 p->in[l], MEPI_GELU_GRAD, nullptr, nullptr, p->pre[l - 1]));
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
  if (s != KP_OK) return fail(s);
  *out = p;
  return KP_OK;
}

extern "C" void kp_mlp_destroy(kp_mlp* p) {
  if (!p) return;
  cudaSetDevice(p->device);
  if (p->stream) cudaStreamSynchronize(p->stream);
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
    k_mlp_to_bf16<<<std::max(1LL, std::min((nw + 255) / 256, 1024LL)), 256, 0, p->stream>>>(p->Wm[l], nw, p->Wb[l]);
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
        p->Wm[l], p->mW[l], p->vW[l], p->gW[l], nw, lr, b1, b2, eps, c1, c2, p->Wb[l]);
    k_mlp_adam<<<1, 256, 0, p->stream>>>(p->c[l], p->mc[l], p->vc[l], p->gc[l], p->out[l], lr, b1, b2, eps, c1, c2,
                                         nullptr);
  }
  KP_CUDA(cudaGetLastError());
  if (loss) {
    KP_CUDA(cudaMemcpyAsync(loss, p->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    KP_CUDA(cudaStreamSynchronize(p->stream));
  }
  return KP_OK;
}
