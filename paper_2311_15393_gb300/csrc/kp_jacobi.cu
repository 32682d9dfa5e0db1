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
// n - 1 rounds, captured once as a CUDA graph (a sweep that would rotate no
// pair is replaced by the same test on the Gram matrix W^T W, one FP64
// GEMM, before the first sweep and after sweeps with few rotations).  Sweeps
// repeat until no pair
// needs a rotation: |gamma| <= tol sqrt(alpha beta) (tol >= m eps), or
// |gamma| <= m eps ||A||_F max(|a_i|, |a_j|), i.e. what would be removed is
// below the rounding noise every column carries (without this absolute
// floor, columns of singular values below eps ||A|| never settle).  Then
// sigma_i = |a_i|, u_i = a_i / sigma_i, and the triplets are sorted by
// decreasing sigma.  For FP32 vectors the blur-factor SVDs take their O(n^3)
// products (the transform F C and the Gram test) in FP32 and use eps = 2^-23
// in both thresholds; rotations stay FP64.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <cmath>
#include <vector>

#include "kp_internal.h"
#include "kp_vec.cuh"

namespace {

constexpr int JT = 256;

__device__ __forceinline__ double jwarp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T jwsum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
struct Eps;
template <>
struct Eps<double> {
  static constexpr double v = 2.220446049250313e-16;
};
template <>
struct Eps<float> {
  static constexpr double v = 1.1920928955078125e-07;
};

// pair p of round `round` for npad players (circle method)
__device__ __forceinline__ int rr_player(int t, int round, int npad) {
  return t == 0 ? 0 : 1 + ((t - 1 + round) % (npad - 1));
}

// One round of the one-sided Jacobi sweep in T arithmetic (FP64, or FP32 for
// the FP32-vector setup, whose tolerance is FP32-level anyway)
template <typename T>
__global__ void __launch_bounds__(JT) k_jacobi_round(T* __restrict__ W, T* __restrict__ V, int m, int n, int npad,
                                                     int round, const double* __restrict__ thr,
                                                     unsigned int* __restrict__ rot_count) {
  const double tol = thr[0], floor = thr[1];  // (in device memory: a captured sweep serves any matrix)
  const int pidx = blockIdx.x;
  int i = rr_player(pidx, round, npad);
  int j = rr_player(npad - 1 - pidx, round, npad);
  if (i > j) {
    int t = i;
    i = j;
    j = t;
  }
  if (j >= n) return;  // pair with the padding column
  T* a = W + (long long)i * m;
  T* b = W + (long long)j * m;
  T sa = 0, sb = 0, sg = 0;
  for (int r = threadIdx.x; r < m; r += JT) {
    const T x = a[r], y = b[r];
    sa = fma(x, x, sa);
    sb = fma(y, y, sb);
    sg = fma(x, y, sg);
  }
  __shared__ T sh[3][JT / 32];
  __shared__ T cs[2];
  sa = jwsum<T>(sa);
  sb = jwsum<T>(sb);
  sg = jwsum<T>(sg);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sh[0][wid] = sa;
    sh[1][wid] = sb;
    sh[2][wid] = sg;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    T al = 0, be = 0, ga = 0;
    for (int w = 0; w < JT / 32; ++w) {
      al += sh[0][w];
      be += sh[1][w];
      ga += sh[2][w];
    }
    T c = 1, s = 0;
    // rotate only if the pair is not orthogonal to relative precision tol and
    // the projection of the smaller column on the larger, |gamma| / |a_max|,
    // is above the noise floor m eps ||A||_F that rounding leaves in any column
    if (ga != T(0) && fabs(ga) > T(tol) * sqrt(al) * sqrt(be) && fabs(ga) > T(floor) * sqrt(fmax(al, be))) {
      const T zeta = (be - al) / (T(2) * ga);
      const T t = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
      c = T(1) / sqrt(T(1) + t * t);
      s = c * t;
      atomicAdd(rot_count, 1u);
    }
    cs[0] = c;
    cs[1] = s;
  }
  __syncthreads();
  const T c = cs[0], s = cs[1];
  if (s == T(0)) return;
  for (int r = threadIdx.x; r < m; r += JT) {
    const T x = a[r], y = b[r];
    a[r] = c * x - s * y;
    b[r] = s * x + c * y;
  }
  T* va = V + (long long)i * n;
  T* vb = V + (long long)j * n;
  for (int r = threadIdx.x; r < n; r += JT) {
    const T x = va[r], y = vb[r];
    va[r] = c * x - s * y;
    vb[r] = s * x + c * y;
  }
}

// Block form of the FP32 sweep with the columns in registers.  A round of
// k_jacobi_round streams all of W and V through L2 for one rotation per
// column; here the n columns form nb blocks of RB_JB, a launch pairs the
// blocks in the same round-robin order (nb - 1 launches per sweep), and each
// thread block runs one full cyclic sweep over its 2 RB_JB columns (2 RB_JB
// - 1 rounds of RB_JB disjoint pairs) with every thread holding rows
// t, t + RB_T, ... of all of them in registers: a round is RB_JB x 3 dot
// products (reduced across the block through shared memory) and the
// rotations in registers.  Rotation and threshold are k_jacobi_round's.
constexpr int RB_T = 128;
constexpr int RB_JB = 4;
__host__ __device__ constexpr int rb_player(int t, int round) {  // players 0 .. 2 RB_JB - 1
  return t == 0 ? 0 : 1 + ((t - 1 + round) % (2 * RB_JB - 1));
}
__host__ __device__ constexpr int rb_lo(int p, int round) {
  return rb_player(p, round) < rb_player(2 * RB_JB - 1 - p, round) ? rb_player(p, round)
                                                                   : rb_player(2 * RB_JB - 1 - p, round);
}
__host__ __device__ constexpr int rb_hi(int p, int round) {
  return rb_player(p, round) < rb_player(2 * RB_JB - 1 - p, round) ? rb_player(2 * RB_JB - 1 - p, round)
                                                                   : rb_player(p, round);
}

template <int R>  // rows per thread: m, n <= R RB_T
__global__ void __launch_bounds__(RB_T) k_jacobi_rblock(float* __restrict__ W, float* __restrict__ V, int m, int n,
                                                        int nb, int round, const double* __restrict__ thr,
                                                        unsigned int* __restrict__ rot_count) {
  const float tol = (float)thr[0], floor = (float)thr[1];
  constexpr int C = 2 * RB_JB;
  constexpr int NW = RB_T / 32;
  __shared__ float red[NW][RB_JB][3];
  __shared__ float rot[RB_JB][2];
  __shared__ unsigned int s_rot;
  const int bi = rr_player(blockIdx.x, round, nb);
  const int bj = rr_player(nb - 1 - blockIdx.x, round, nb);
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  auto gcol = [&](int c) -> int {
    const int g = c < RB_JB ? bi * RB_JB + c : bj * RB_JB + c - RB_JB;
    return g < n ? g : -1;
  };
  float w[C][R], v[C][R];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int g = gcol(c);
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int r = t + k * RB_T;
      w[c][k] = (g >= 0 && r < m) ? W[(long long)g * m + r] : 0.f;
      v[c][k] = (g >= 0 && r < n) ? V[(long long)g * n + r] : 0.f;
    }
  }
  if (t == 0) s_rot = 0u;
#pragma unroll
  for (int rd = 0; rd < C - 1; ++rd) {
    float part[RB_JB][3];
#pragma unroll
    for (int p = 0; p < RB_JB; ++p) {
      const int i = rb_lo(p, rd), j = rb_hi(p, rd);
      float sa = 0.f, sb = 0.f, sg = 0.f;
#pragma unroll
      for (int k = 0; k < R; ++k) {
        sa = fmaf(w[i][k], w[i][k], sa);
        sb = fmaf(w[j][k], w[j][k], sb);
        sg = fmaf(w[i][k], w[j][k], sg);
      }
      part[p][0] = sa;
      part[p][1] = sb;
      part[p][2] = sg;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int p = 0; p < RB_JB; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) part[p][q] += __shfl_xor_sync(0xffffffffu, part[p][q], o);
    if (lane == 0)
#pragma unroll
      for (int p = 0; p < RB_JB; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) red[wid][p][q] = part[p][q];
    __syncthreads();
    if (t < RB_JB) {
      const int p = t;
      float al = 0.f, be = 0.f, ga = 0.f;
#pragma unroll
      for (int x = 0; x < NW; ++x) {
        al += red[x][p][0];
        be += red[x][p][1];
        ga += red[x][p][2];
      }
      float c = 1.f, s = 0.f;
      const bool valid = gcol(rb_lo(p, rd)) >= 0 && gcol(rb_hi(p, rd)) >= 0;
      if (valid && ga != 0.f && fabsf(ga) > tol * sqrtf(al) * sqrtf(be) && fabsf(ga) > floor * sqrtf(fmaxf(al, be))) {
        const float zeta = (be - al) / (2.f * ga);
        const float tt = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
        c = 1.f / sqrtf(1.f + tt * tt);
        s = c * tt;
        atomicAdd(&s_rot, 1u);
      }
      rot[p][0] = c;
      rot[p][1] = s;
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < RB_JB; ++p) {
      const float c = rot[p][0], s = rot[p][1];
      if (s != 0.f) {
        const int i = rb_lo(p, rd), j = rb_hi(p, rd);
#pragma unroll
        for (int k = 0; k < R; ++k) {
          const float x = w[i][k], y = w[j][k];
          w[i][k] = c * x - s * y;
          w[j][k] = s * x + c * y;
          const float a = v[i][k], b = v[j][k];
          v[i][k] = c * a - s * b;
          v[j][k] = s * a + c * b;
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int g = gcol(c);
    if (g < 0) continue;
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int r = t + k * RB_T;
      if (r < m) W[(long long)g * m + r] = w[c][k];
      if (r < n) V[(long long)g * n + r] = v[c][k];
    }
  }
  if (t == 0 && s_rot) atomicAdd(rot_count, s_rot);
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

// orthogonal transform that nearly diagonalises the blur factors:
// DCT-II (reflexive BC) or DST-I (zero BC), column-major n x n.  The entries
// are scale * trig(pi q / P) for an integer q reduced mod 2P, so one table of
// 2P values (k_trig_table) serves all n^2 entries.
//   DCT-II: C[j][k] = sqrt(2/n) cos(pi (2j+1) k / (2n)) (k = 0 row x 1/sqrt 2), P = 2n
//   DST-I:  C[j][k] = sqrt(2/(n+1)) sin(pi (j+1)(k+1) / (n+1)),                 P = n+1
__global__ void k_trig_table(int P, int kind, double* __restrict__ tab) {
  const double pi = 3.141592653589793238462643;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < 2 * P; q += gridDim.x * blockDim.x)
    tab[q] = kind == 0 ? cos(pi * q / P) : sin(pi * q / P);
}
__global__ void k_transform(int n, int kind, const double* __restrict__ tab, double scale, double* __restrict__ C) {
  const long long tot = (long long)n * n;
  const long long P2 = kind == 0 ? 4LL * n : 2LL * (n + 1);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const long long j = t % n, k = t / n;
    if (kind == 0) {
      const double v = scale * tab[((2 * j + 1) * k) % P2];
      C[t] = k == 0 ? v * 0.70710678118654752440 : v;
    } else {
      C[t] = scale * tab[((j + 1) * (k + 1)) % P2];
    }
  }
}

// fill C (n x n) with the transform: table, then the gather
static kp_status make_transform(kp_ctx* ctx, int n, int kind, double* C) {
  const int P = kind == 0 ? 2 * n : n + 1;
  double* tab = nullptr;
  KP_TRY(kp_alloc(ctx, (void**)&tab, sizeof(double) * 2 * (size_t)P));
  k_trig_table<<<(2 * P + 255) / 256, 256, 0, ctx->stream>>>(P, kind, tab);
  const long long nn = (long long)n * n;
  const int g = std::max(1, std::min((int)((nn + 255) / 256), ctx->sm_count * 16));
  const double scale = kind == 0 ? std::sqrt(2.0 / n) : std::sqrt(2.0 / (n + 1.0));
  k_transform<<<g, 256, 0, ctx->stream>>>(n, kind, tab, scale, C);
  ctx->launches += 2;
  KP_CUDA(cudaGetLastError());
  return KP_OK;
}

// B (n x m col-major) = A^T for A m x n col-major
template <typename T>
__global__ void k_transpose_cm(const T* __restrict__ A, int m, int n, T* __restrict__ B) {
  long long tot = (long long)m * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % m), j = (int)(t / m);
    B[j + (long long)n * i] = A[t];
  }
}

// flip column c of U when it points against column c of R (one block per column)
__global__ void k_align_signs(double* __restrict__ U, const double* __restrict__ R, int m) {
  const int c = blockIdx.x;
  double v = 0.0;
  for (int r = threadIdx.x; r < m; r += blockDim.x) v = fma(U[(long long)c * m + r], R[(long long)c * m + r], v);
  __shared__ double sh[JT / 32];
  v = jwarp_sum(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  __shared__ double tot;
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < JT / 32; ++w) t += sh[w];
    tot = t;
  }
  __syncthreads();
  if (tot < 0)
    for (int r = threadIdx.x; r < m; r += blockDim.x) U[(long long)c * m + r] = -U[(long long)c * m + r];
}

// count entries with F[i][j] != F[j][i] (exact comparison)
__global__ void k_asym_count(const double* __restrict__ F, int n, unsigned int* __restrict__ count) {
  const long long tot = (long long)n * n;
  unsigned int local = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / n), j = (int)(t % n);
    if (i < j && F[t] != F[(long long)j * n + i]) ++local;
  }
  if (local) atomicAdd(count, local);
}

// count pairs (i < j) of the Gram matrix G = W^T W that still need a rotation
// (same test as k_jacobi_round: relative and absolute floors)
template <typename T>
__global__ void k_gram_violations(const T* __restrict__ G, int n, double tol, double floor,
                                  unsigned int* __restrict__ count) {
  const long long tot = (long long)n * n;
  unsigned int local = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), j = (int)(t / n);
    if (i >= j) continue;
    // |g| > tol sqrt(a b) and |g| > floor sqrt(max(a, b)), compared squared
    const T ga = G[t], al = G[(long long)i * n + i], be = G[(long long)j * n + j];
    const T g2 = ga * ga;
    if (ga != T(0) && g2 > T(tol * tol) * al * be && g2 > T(floor * floor) * (al > be ? al : be)) ++local;
  }
  if (local) atomicAdd(count, local);
}


// out[j + k ldo] = sum_i X[i + j ldx] Y[i + k ldy] for j < ncol, k < p: the
// tall-skinny products of the subspace iteration, one warp per column j
constexpr int SK_CHUNK = 8;
template <typename T>
__global__ void __launch_bounds__(256) k_skinny_tn(const T* __restrict__ X, long long ldx,
                                                   const T* __restrict__ Y, long long ldy, int m, int ncol,
                                                   int p, T* __restrict__ out, long long ldo) {
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= ncol) return;
  const T* x = X + warp * ldx;
  for (int k0 = 0; k0 < p; k0 += SK_CHUNK) {
    const int kn = min(SK_CHUNK, p - k0);
    T acc[SK_CHUNK];
#pragma unroll
    for (int q = 0; q < SK_CHUNK; ++q) acc[q] = T(0);
    for (int i = lane; i < m; i += 32) {
      const T xv = x[i];
#pragma unroll
      for (int q = 0; q < SK_CHUNK; ++q)
        if (q < kn) acc[q] = fma(xv, Y[i + (long long)(k0 + q) * ldy], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < SK_CHUNK; ++q) acc[q] = jwsum<T>(acc[q]);
    if (lane == 0)
#pragma unroll
      for (int q = 0; q < SK_CHUNK; ++q)
        if (q < kn) out[warp + (long long)(k0 + q) * ldo] = acc[q];
  }
}

// out (m x r col-major) = Q (m x p col-major) B[:, :r] (B p x p col-major)
template <typename T>
__global__ void k_small_right(const T* __restrict__ Q, int m, int p, const T* __restrict__ B, int r,
                              T* __restrict__ out) {
  const long long tot = (long long)m * r;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % m), c = (int)(t / m);
    T acc = T(0);
    for (int j = 0; j < p; ++j) acc = fma(Q[i + (long long)j * m], B[j + (long long)c * p], acc);
    out[t] = acc;
  }
}

// Orthonormalise the p columns of Q (m x p col-major) in place by classical
// Gram-Schmidt with each projection done twice (CGS2: all dots against the
// previous columns in one block reduction); a column that vanishes (rank
// deficiency) is replaced by a unit vector e_t and orthogonalised again.
// With R non-null, also the triangular factor of Q_in = Q_out R (p x p
// col-major; a vanished column keeps its small remaining norm on the
// diagonal).  One block of CG_T threads runs the column sweeps; with one
// warp per scheduler it issued an instruction every ~4.4 cycles (measured),
// so the block is wide (16 warps, each thread ~m / 512 rows) and the warps'
// reductions overlap.  With `staged`, Q is copied into shared memory (m p
// elements of dynamic shared memory) and back, so the sweeps read shared
// memory instead of waiting on global loads.
constexpr int CG_T = 512;
constexpr int CG_CH = 16;  // dots per block reduction

// Warp sums of 16 values at once: four halving exchanges (8 + 4 + 2 + 1
// shuffles) leave each lane pair with one value index, and a last exchange
// adds the pair: 16 shuffles instead of 16 x 5.  Returns the warp sum of
// value cg_index(lane); v is consumed.
__device__ __forceinline__ int cg_index(int lane) {
  return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}
template <typename T>
__device__ __forceinline__ T warp_sum16(T (&v)[CG_CH], int lane) {
#pragma unroll
  for (int h = 8; h >= 1; h >>= 1) {
    const bool up = (lane & (2 * h)) != 0;  // exchange across lane bit 2h: keep the upper or lower half
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const T send = up ? v[i] : v[i + h];
      const T keep = up ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 2 * h);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}
constexpr int CG_SMEM_MAX = 200 * 1024;
template <typename T>
__global__ void __launch_bounds__(CG_T) k_cgs2(T* __restrict__ Qg, int m, int p, T* __restrict__ R, int staged) {
  constexpr int NW = CG_T / 32;
  __shared__ T sh[NW][CG_CH + 1];
  __shared__ T dsh[CG_CH];
  __shared__ T tot;
  extern __shared__ __align__(16) unsigned char cg_dyn[];
  const int mp = m * p;
  T* Q = staged ? reinterpret_cast<T*>(cg_dyn) : Qg;
  if (staged) {
    for (int i = threadIdx.x; i < mp; i += CG_T) Q[i] = Qg[i];
    __syncthreads();
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  auto bsum = [&](T v) -> T {
    v = jwsum<T>(v);
    __syncthreads();
    if (lane == 0) sh[wid][0] = v;
    __syncthreads();
    if (wid == 0) {
      T t = lane < NW ? sh[lane][0] : T(0);
      t = jwsum<T>(t);
      if (lane == 0) tot = t;
    }
    __syncthreads();
    return tot;
  };
  for (int k = 0; k < p; ++k) {
    T* qk = Q + k * m;
    T n0 = 0;
    for (int r = threadIdx.x; r < m; r += CG_T) n0 = fma(qk[r], qk[r], n0);
    n0 = sqrt(bsum(n0));
    for (int attempt = 0; attempt < 3; ++attempt) {
      for (int pass = 0; pass < 2; ++pass) {
        for (int j0 = 0; j0 < k; j0 += CG_CH) {
          const int jn = min(CG_CH, k - j0);
          const T* Qj = Q + j0 * m;
          T d[CG_CH];
#pragma unroll
          for (int q = 0; q < CG_CH; ++q) d[q] = T(0);
          for (int r = threadIdx.x; r < m; r += CG_T) {
            const T x = qk[r];
#pragma unroll
            for (int q = 0; q < CG_CH; ++q)
              if (q < jn) d[q] = fma(Qj[r + q * m], x, d[q]);
          }
          {
            const T v = warp_sum16<T>(d, lane);
            if ((lane & 1) == 0) sh[wid][cg_index(lane)] = v;
          }
          __syncthreads();
          if (threadIdx.x < jn) {
            T t = 0;
            for (int w = 0; w < NW; ++w) t += sh[w][threadIdx.x];
            dsh[threadIdx.x] = t;
            if (R && attempt == 0) {
              T* rr = R + k * p + j0 + threadIdx.x;
              *rr = (pass == 0 ? T(0) : *rr) + t;
            }
          }
          __syncthreads();
          for (int r = threadIdx.x; r < m; r += CG_T) {
            T x = qk[r];
            for (int q = 0; q < jn; ++q) x = fma(-dsh[q], Qj[r + q * m], x);
            qk[r] = x;
          }
          __syncthreads();
        }
      }
      T nk = 0;
      for (int r = threadIdx.x; r < m; r += CG_T) nk = fma(qk[r], qk[r], nk);
      nk = sqrt(bsum(nk));
      if (R && attempt == 0 && threadIdx.x == 0) {
        for (int j = k + 1; j < p; ++j) R[k * p + j] = T(0);
        R[k * p + k] = nk;
      }
      if (nk > T(sizeof(T) == 8 ? 1e-10 : 1e-4) * n0 && nk > T(0)) {
        const T inv = T(1) / nk;  // one division per column, not per entry
        for (int r = threadIdx.x; r < m; r += CG_T) qk[r] *= inv;
        __syncthreads();
        break;
      }
      const int t = (int)(((long long)(k + 1) * 7919 + attempt * 104729) % m);
      for (int r = threadIdx.x; r < m; r += CG_T) qk[r] = (r == t) ? T(1) : T(0);
      n0 = T(1);
      __syncthreads();
    }
  }
  if (staged) {
    __syncthreads();
    for (int i = threadIdx.x; i < mp; i += CG_T) Qg[i] = Q[i];
  }
}

// One-sided Jacobi SVD of a narrow A (m x p col-major, p <= 32) held in
// shared memory by one block: the same rotations, thresholds and round-robin
// order as the multi-block sweep, every sweep in this launch, one warp per
// pair.  Writes U = A V / sigma (m x p), sigma (p) and V (p x p) sorted by
// decreasing sigma; *status = 1 if max_sweeps sweeps did not converge.
constexpr int SJ_T = 1024;
constexpr int SJ_MAXP = 32;
template <typename T>
__global__ void __launch_bounds__(SJ_T) k_jacobi_small(const T* __restrict__ A, int m, int p, T tol_in,
                                                       int max_sweeps, T* __restrict__ U,
                                                       T* __restrict__ s_out, T* __restrict__ V_out,
                                                       int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_j[];
  T* W = reinterpret_cast<T*>(smem_j);                    // m x p
  T* V = W + (long long)m * p;      // p x p
  __shared__ T red[SJ_T / 32];
  __shared__ T sg[SJ_MAXP];
  __shared__ int perm[SJ_MAXP];
  __shared__ unsigned int rot;
  __shared__ T floor_sh;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T f2 = T(0);
  for (long long t = threadIdx.x; t < (long long)m * p; t += SJ_T) {
    const T x = A[t];
    W[t] = x;
    f2 = fma(x, x, f2);
  }
  for (int t = threadIdx.x; t < p * p; t += SJ_T) V[t] = (t / p == t % p) ? T(1) : T(0);
  f2 = jwsum<T>(f2);
  if (lane == 0) red[wid] = f2;
  __syncthreads();
  if (threadIdx.x == 0) {
    T t = 0;
    for (int w = 0; w < SJ_T / 32; ++w) t += red[w];
    floor_sh = T((double)m * Eps<T>::v) * sqrt(t);
  }
  __syncthreads();
  const T floor = floor_sh;
  const T tol = tol_in > T((double)m * Eps<T>::v) ? tol_in : T((double)m * Eps<T>::v);
  const int npad = p + (p & 1);
  int sweep = 0;
  bool done = npad < 2;
  for (; !done && sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) rot = 0u;
    __syncthreads();
    for (int round = 0; round < npad - 1; ++round) {
      if (wid < npad / 2) {
        int i = rr_player(wid, round, npad);
        int j = rr_player(npad - 1 - wid, round, npad);
        if (i > j) {
          const int t = i;
          i = j;
          j = t;
        }
        if (j < p) {
          T* a = W + (long long)i * m;
          T* b = W + (long long)j * m;
          T al = T(0), be = T(0), ga = T(0);
          for (int r = lane; r < m; r += 32) {
            const T x = a[r], y = b[r];
            al = fma(x, x, al);
            be = fma(y, y, be);
            ga = fma(x, y, ga);
          }
          al = jwsum<T>(al);
          be = jwsum<T>(be);
          ga = jwsum<T>(ga);
          if (ga != T(0) && fabs(ga) > tol * sqrt(al) * sqrt(be) && fabs(ga) > floor * sqrt(al > be ? al : be)) {
            const T zeta = (be - al) / (T(2) * ga);
            const T t = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
            const T c = T(1) / sqrt(T(1) + t * t), sn = c * t;
            for (int r = lane; r < m; r += 32) {
              const T x = a[r], y = b[r];
              a[r] = c * x - sn * y;
              b[r] = sn * x + c * y;
            }
            T* va = V + (long long)i * p;
            T* vb = V + (long long)j * p;
            for (int r = lane; r < p; r += 32) {
              const T x = va[r], y = vb[r];
              va[r] = c * x - sn * y;
              vb[r] = sn * x + c * y;
            }
            if (lane == 0) atomicAdd(&rot, 1u);
          }
        }
      }
      __syncthreads();
    }
    done = rot == 0u;
    __syncthreads();
  }
  if (!done && threadIdx.x == 0) *status = 1;
  // sigma = column norms, then sort (descending; ties keep the smaller index)
  for (int c = wid; c < p; c += SJ_T / 32) {
    T v = T(0);
    for (int r = lane; r < m; r += 32) v = fma(W[(long long)c * m + r], W[(long long)c * m + r], v);
    v = jwsum<T>(v);
    if (lane == 0) sg[c] = sqrt(v);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int c = 0; c < p; ++c) perm[c] = c;
    for (int a = 1; a < p; ++a) {
      const int x = perm[a];
      int b = a - 1;
      while (b >= 0 && sg[perm[b]] < sg[x]) {
        perm[b + 1] = perm[b];
        --b;
      }
      perm[b + 1] = x;
    }
  }
  __syncthreads();
  for (int c = wid; c < p; c += SJ_T / 32) {
    const int src = perm[c];
    const T sv = sg[src];
    const T inv = sv > T(0) ? T(1) / sv : T(0);
    for (int r = lane; r < m; r += 32) U[(long long)c * m + r] = W[(long long)src * m + r] * inv;
    for (int r = lane; r < p; r += 32) V_out[(long long)c * p + r] = V[(long long)src * p + r];
    if (lane == 0) s_out[c] = sv;
  }
}


}  // namespace

// instantiated sweep graphs of a context (at most 16; the oldest is dropped)
struct JacobiCache {
  struct Entry {
    const void* w;
    const void* v;
    const void* cnt;
    int m, n, kind;
    cudaGraphExec_t exec;
  };
  std::vector<Entry> entries;
};
static JacobiCache* jacobi_cache(kp_ctx* ctx) {
  if (!ctx->jac_cache) ctx->jac_cache = new JacobiCache();
  return static_cast<JacobiCache*>(ctx->jac_cache);
}
static void jacobi_cache_put(JacobiCache* jc, const JacobiCache::Entry& e) {
  if (jc->entries.size() >= 16) {
    cudaGraphExecDestroy(jc->entries.front().exec);
    jc->entries.erase(jc->entries.begin());
  }
  jc->entries.push_back(e);
}
void jacobi_cache_free(kp_ctx* ctx) {
  if (!ctx->jac_cache) return;
  auto* jc = static_cast<JacobiCache*>(ctx->jac_cache);
  for (auto& e : jc->entries) cudaGraphExecDestroy(e.exec);
  delete jc;
  ctx->jac_cache = nullptr;
}

// Sweeps on W (m x n col-major, in place) accumulating into V (n x n,
// holding its initial value); then sigma, sorting, U = W / sigma.
static kp_status jacobi_run(kp_ctx* ctx, double* W, int m, int n, double* Vw, double* U, double* s, double* V,
                            int* sweeps_out, bool fast = false) {
  cudaStream_t st = ctx->stream;
  double *sw = nullptr, *nrm = nullptr;
  int* perm = nullptr;
  unsigned int* cnt = nullptr;
  KP_TRY(kp_alloc(ctx, (void**)&sw, sizeof(double) * n));
  KP_TRY(kp_alloc(ctx, (void**)&perm, sizeof(int) * n));
  KP_TRY(kp_alloc(ctx, (void**)&cnt, sizeof(unsigned int)));
  KP_TRY(kp_alloc(ctx, (void**)&nrm, sizeof(double)));
  // noise floor m eps ||A||_F; eps is the unit of the arithmetic W came from
  // (FP32 when the products of the setup run in FP32)
  KP_TRY(dot_dev(ctx, W, W, (long long)m * n, true, nrm));
  double fro2 = 0.0;
  KP_CUDA(cudaMemcpyAsync(&fro2, nrm, sizeof(double), cudaMemcpyDeviceToHost, st));
  KP_CUDA(kp_wait(ctx, st));
  const double eps = fast ? 1.1920928955078125e-07 : 2.220446049250313e-16;
  const double floor = (double)m * eps * sqrt(fro2);
  // pairs count as orthogonal at |gamma| <= tol sqrt(alpha beta); below m eps
  // the inner products are rounding noise and rotations would never stop
  const double tol = std::max(ctx->jacobi_tol, (double)m * eps);
  const int npad = n + (n & 1);
  int sweeps = 0;
  if (npad >= 2) {
    // Before the first sweep, and instead of a sweep that would only confirm
    // convergence, count the pairs that need a rotation on G = W^T W (one
    // GEMM): a sweep over a matrix with no such pair rotates nothing.
    double* G = nullptr;
    float *G32 = nullptr, *W32 = nullptr, *V32 = nullptr;
    if (fast) {  // the sweeps rotate FP32 copies of W and Vw (copied back below)
      KP_TRY(kp_alloc(ctx, (void**)&G32, sizeof(float) * (size_t)n * n));
      KP_TRY(kp_alloc(ctx, (void**)&W32, sizeof(float) * (size_t)m * n));
      KP_TRY(kp_alloc(ctx, (void**)&V32, sizeof(float) * (size_t)n * n));
      KP_TRY(convert_f64_to_f32(ctx, W, W32, (long long)m * n));
      KP_TRY(convert_f64_to_f32(ctx, Vw, V32, (long long)n * n));
    } else {
      KP_TRY(kp_alloc(ctx, (void**)&G, sizeof(double) * (size_t)n * n));
    }
    auto gram_clean = [&](bool* clean) -> kp_status {
      GemmDesc gd;  // G[i][j] = sum_r W[r, i] W[r, j]
      gd.M = n;
      gd.N = n;
      gd.K = m;
      gd.A.ld = m;
      gd.B.ld = m;
      gd.epi.mode = EPI_T;
      gd.epi.ldd = n;
      const int gb = std::max(1, std::min((int)(((long long)n * n + 255) / 256), ctx->sm_count * 8));
      KP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned int), st));
      if (fast) {
        if (ctx->setup_tc && m % 8 == 0) {  // FP32-level product on the tensor cores
          KP_TRY(tc_product(ctx, W32, false, n, W32, false, n, m, G32, 3));
        } else {
          gd.A.ptr = W32;
          gd.B.ptr = W32;
          gd.epi.out = G32;
          KP_TRY(simt_gemm<float>(ctx, gd));
        }
        k_gram_violations<float><<<gb, 256, 0, st>>>(G32, n, tol, floor, cnt);
      } else {
        gd.A.ptr = W;
        gd.B.ptr = W;
        gd.epi.out = G;
        KP_TRY(simt_gemm<double>(ctx, gd));
        k_gram_violations<double><<<gb, 256, 0, st>>>(G, n, tol, floor, cnt);
      }
      KP_LAUNCHED(ctx);
      unsigned int h = 0;
      KP_CUDA(cudaMemcpyAsync(&h, cnt, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
      KP_CUDA(kp_wait(ctx, st));
      *clean = h == 0;
      return KP_OK;
    };
    unsigned int h_cnt = 1;
    bool clean = false;
    KP_TRY(gram_clean(&clean));
    if (clean) h_cnt = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    kp_status gst = KP_OK;
    // FP32 sweeps in the register block form where the rows fit (m, n <= 8 RB_T)
    const int mx = std::max(m, n);
    const int rneed = (mx + RB_T - 1) / RB_T;
    const int rsel = rneed <= 1 ? 1 : rneed <= 2 ? 2 : rneed <= 4 ? 4 : rneed <= 6 ? 6 : rneed <= 8 ? 8 : 0;
    const bool blocked = fast && ctx->jacobi_block && rsel > 0;
    const int nbl = (n + RB_JB - 1) / RB_JB;
    const int nb = nbl + (nbl & 1);
    const int rounds = blocked ? nb - 1 : npad - 1;
    // the thresholds live in device memory, so a captured sweep depends only on
    // the buffers and sizes: the sweep graphs are kept per context and reused
    // whenever the same buffers come back (repeated setups of equal sizes)
    double* thr = ctx->dscal + S_JACOBI;
    {
      const double th[2] = {tol, floor};
      KP_CUDA(cudaMemcpyAsync(thr, th, sizeof(th), cudaMemcpyHostToDevice, st));
      KP_CUDA(kp_wait(ctx, st));  // th is a host stack value
    }
    JacobiCache* jc = jacobi_cache(ctx);
    const void* kw = fast ? (const void*)W32 : (const void*)W;
    const void* kv = fast ? (const void*)V32 : (const void*)Vw;
    const int kind = blocked ? rsel : (fast ? -1 : -2);
    for (const auto& e : jc->entries)
      if (e.w == kw && e.v == kv && e.cnt == cnt && e.m == m && e.n == n && e.kind == kind) exec = e.exec;
    for (sweeps = 0; !clean && sweeps < ctx->jacobi_max_sweeps; ++sweeps) {
      if (!exec) {  // one sweep (n - 1 rounds, or nb - 1 block rounds) as a graph, built at the first sweep
        KP_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        k_zero_u32<<<1, 1, 0, st>>>(cnt);
        for (int round = 0; round < rounds; ++round) {
          if (blocked) {
            switch (rsel) {
              case 1: k_jacobi_rblock<1><<<nb / 2, RB_T, 0, st>>>(W32, V32, m, n, nb, round, thr, cnt); break;
              case 2: k_jacobi_rblock<2><<<nb / 2, RB_T, 0, st>>>(W32, V32, m, n, nb, round, thr, cnt); break;
              case 4: k_jacobi_rblock<4><<<nb / 2, RB_T, 0, st>>>(W32, V32, m, n, nb, round, thr, cnt); break;
              case 6: k_jacobi_rblock<6><<<nb / 2, RB_T, 0, st>>>(W32, V32, m, n, nb, round, thr, cnt); break;
              default: k_jacobi_rblock<8><<<nb / 2, RB_T, 0, st>>>(W32, V32, m, n, nb, round, thr, cnt); break;
            }
          } else if (fast) {
            k_jacobi_round<float><<<npad / 2, JT, 0, st>>>(W32, V32, m, n, npad, round, thr, cnt);
          } else {
            k_jacobi_round<double><<<npad / 2, JT, 0, st>>>(W, Vw, m, n, npad, round, thr, cnt);
          }
        }
        cudaError_t ce = cudaStreamEndCapture(st, &graph);
        if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) {
          cudaGraphDestroy(graph);
          graph = nullptr;
        }
        if (ce != cudaSuccess) {
          kp_set_error("jacobi_svd: sweep graph capture failed: %s", cudaGetErrorString(ce));
          gst = KP_ECUDA;
          break;
        }
        jacobi_cache_put(jc, JacobiCache::Entry{kw, kv, cnt, m, n, kind, exec});
      }
      cudaError_t ce = cudaGraphLaunch(exec, st);
      if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h_cnt, cnt, sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
      if (ce == cudaSuccess) ce = kp_wait(ctx, st);
      if (ce != cudaSuccess) {
        kp_set_error("jacobi_svd: sweep failed: %s", cudaGetErrorString(ce));
        gst = KP_ECUDA;
        break;
      }
      ctx->launches += rounds + 1;
      if (h_cnt == 0) {
        ++sweeps;
        break;
      }
      // few rotations: the next sweep is likely only a confirmation
      if ((long long)h_cnt * 8 < (long long)npad) {
        gst = gram_clean(&clean);
        if (gst != KP_OK) break;
        if (clean) {
          h_cnt = 0;
          ++sweeps;
          break;
        }
      }
    }
    if (graph) cudaGraphDestroy(graph);
    KP_TRY(gst);
    if (fast && sweeps > 0) {
      KP_TRY(convert_f32_to_f64(ctx, W32, W, (long long)m * n));
      KP_TRY(convert_f32_to_f64(ctx, V32, Vw, (long long)n * n));
    }
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
  if (shm > 48 * 1024) {  // raise the kernel's limit, never lower it (other threads may launch it meanwhile)
    static std::mutex mu;
    static size_t shm_set = 48 * 1024;
    std::lock_guard<std::mutex> lock(mu);
    if (shm > shm_set) {
      KP_CUDA(cudaFuncSetAttribute(k_sort_desc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
      shm_set = shm;
    }
  }
  k_sort_desc<<<1, 1024, shm, st>>>(sw, n, npow2, perm);
  KP_LAUNCHED(ctx);
  k_gather<<<n, 256, 0, st>>>(W, Vw, sw, perm, m, n, U, V, s);
  KP_LAUNCHED(ctx);
  KP_CUDA(cudaGetLastError());
  if (sweeps_out) *sweeps_out = sweeps;
  return KP_OK;
}

kp_status jacobi_svd(kp_ctx* ctx, const double* A, int m, int n, double* U, double* s, double* V, int* sweeps_out) {
  if (m < n || n < 1) {
    kp_set_error("jacobi_svd: need m >= n >= 1 (m=%d n=%d)", m, n);
    return KP_EINVAL;
  }
  double *W = nullptr, *Vw = nullptr;
  KP_TRY(kp_alloc(ctx, (void**)&W, sizeof(double) * (size_t)m * n));
  KP_TRY(kp_alloc(ctx, (void**)&Vw, sizeof(double) * (size_t)n * n));
  KP_CUDA(cudaMemcpyAsync(W, A, sizeof(double) * (size_t)m * n, cudaMemcpyDeviceToDevice, ctx->stream));
  k_set_identity<<<ctx->sm_count * 2, 256, 0, ctx->stream>>>(Vw, n);
  KP_LAUNCHED(ctx);
  return jacobi_run(ctx, W, m, n, Vw, U, s, V, sweeps_out);
}

// SVD of a square blur factor F (n x n, given row-major) with an orthogonal
// transform C that nearly diagonalises it: one-sided Jacobi on F C with V
// starting at C (so V ends as C Q, exact for any orthogonal C); the
// transform only shortens the sweeps (DCT-II for reflexive BC, DST-I for
// zero BC).  U must be orthonormal also where sigma is below the noise floor:
// for a symmetric F it is V with column signs; otherwise a second run on F^T
// gives U as accumulated rotations.  Either way its columns are sign-aligned
// with F v_i / sigma_i of the first run.
kp_status factor_svd(kp_ctx* ctx, const double* F_rm, int n, int transform, double* U, double* s, double* V,
                     int* sweeps_out) {
  cudaStream_t st = ctx->stream;
  const bool fast = ctx->setup_fp32;
  const long long nn = (long long)n * n;
  double *C, *W, *Vw, *FT_rm, *U1, *s2;
  KP_TRY(kp_alloc(ctx, (void**)&C, sizeof(double) * nn));
  KP_TRY(kp_alloc(ctx, (void**)&W, sizeof(double) * nn));
  KP_TRY(kp_alloc(ctx, (void**)&Vw, sizeof(double) * nn));
  KP_TRY(kp_alloc(ctx, (void**)&FT_rm, sizeof(double) * nn));
  KP_TRY(kp_alloc(ctx, (void**)&U1, sizeof(double) * nn));
  KP_TRY(kp_alloc(ctx, (void**)&s2, sizeof(double) * n));
  float *C32 = nullptr, *F32 = nullptr, *W32 = nullptr;
  if (fast) {
    KP_TRY(kp_alloc(ctx, (void**)&C32, sizeof(float) * nn));
    KP_TRY(kp_alloc(ctx, (void**)&F32, sizeof(float) * nn));
    KP_TRY(kp_alloc(ctx, (void**)&W32, sizeof(float) * nn));
  }
  const int g = std::max(1, std::min((int)((nn + 255) / 256), ctx->sm_count * 16));
  KP_TRY(make_transform(ctx, n, transform, C));
  if (fast) KP_TRY(convert_f64_to_f32(ctx, C, C32, nn));
  // W (col-major) = X R for X given row-major and R col-major (R = C, or V
  // of the first run), computed as the row-major product D[k][i] = sum_j
  // R[j,k] X[i,j]; FP32 products are widened to FP64
  const double* R = C;
  const float* R32 = C32;
  auto mul = [&](const double* X_rm, double* out) -> kp_status {
    GemmDesc gd;
    gd.M = n;
    gd.N = n;
    gd.K = n;
    gd.A.ld = n;
    gd.B.ld = n;
    gd.epi.mode = EPI_T;
    gd.epi.ldd = n;
    if (ctx->setup_tc) {  // tensor cores: FP32-level (3 slices) or half precision (1)
      KP_TRY(tc_product(ctx, R, true, n, X_rm, true, n, n, W32, ctx->setup_half ? 1 : 3));
      return convert_f32_to_f64(ctx, W32, out, nn);
    }
    if (fast) {
      KP_TRY(convert_f64_to_f32(ctx, X_rm, F32, nn));
      gd.A.ptr = R32;
      gd.B.ptr = F32;
      gd.epi.out = W32;
      KP_TRY(simt_gemm<float>(ctx, gd));
      return convert_f32_to_f64(ctx, W32, out, nn);
    }
    gd.A.ptr = R;
    gd.B.ptr = X_rm;
    gd.epi.out = out;
    return simt_gemm<double>(ctx, gd);
  };
  int sw1 = 0, sw2 = 0;
  // run 1: F = U1 S V^T
  KP_TRY(mul(F_rm, W));
  KP_CUDA(cudaMemcpyAsync(Vw, C, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st));
  KP_TRY(jacobi_run(ctx, W, n, n, Vw, U1, s, V, &sw1, fast));
  // A symmetric factor F = Q L Q^T (reflexive BC with a PSF symmetric about its
  // centre gives one) has U = V sign(L): the columns of U1 = F V / sigma are
  // +-V where sigma is above rounding level, and any sign pairs with sigma ~ 0.
  unsigned int* cnt;
  KP_TRY(kp_alloc(ctx, (void**)&cnt, sizeof(unsigned int)));
  KP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned int), st));
  k_asym_count<<<g, 256, 0, st>>>(F_rm, n, cnt);
  KP_LAUNCHED(ctx);
  unsigned int asym = 1;
  KP_CUDA(cudaMemcpyAsync(&asym, cnt, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
  KP_CUDA(kp_wait(ctx, st));
  if (asym == 0) {
    KP_CUDA(cudaMemcpyAsync(U, V, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st));
  } else {
    // run 2: F^T = V' S U^T  (F^T row-major = F column-major = transpose of F_rm),
    // started from the first run's V instead of the transform: exactly
    // orthogonal, and for the nearly symmetric (or antisymmetric) factors of
    // a PSF symmetric about its centre F^T V = V S U^T V is nearly orthogonal
    // already (U ~ +-V), so the sweeps only finish what the boundary rows of
    // the factor make asymmetric
    k_transpose_cm<double><<<g, 256, 0, st>>>(F_rm, n, n, FT_rm);
    KP_LAUNCHED(ctx);
    if (ctx->jacobi_warm_u) {
      R = V;
      if (fast && !ctx->setup_tc) {
        KP_TRY(convert_f64_to_f32(ctx, V, C32, nn));
        R32 = C32;
      }
    }
    KP_TRY(mul(FT_rm, W));
    KP_CUDA(cudaMemcpyAsync(Vw, R, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st));
    KP_TRY(jacobi_run(ctx, W, n, n, Vw, FT_rm /* scratch */, s2, U, &sw2, fast));
  }
  k_align_signs<<<n, JT, 0, st>>>(U, U1, n);
  KP_LAUNCHED(ctx);
  KP_CUDA(cudaGetLastError());
  if (sweeps_out) *sweeps_out = sw1 + sw2;
  return KP_OK;
}

// Subspace iteration for the leading r singular triplets, in T arithmetic
// (FP64, or FP32 for the FP32-vector setup); p <= SJ_MAXP.  W (m x n col-major)
// and WT = W^T are T; outputs (T): U (m x r), s (r), V (n x r).
// CGS2 launch: Q staged in shared memory when m p elements fit
template <typename T>
static kp_status cgs2(kp_ctx* ctx, T* Q, int m, int p, T* R) {
  static std::atomic<bool> attr_set{false};  // contexts on several host threads launch this
  const size_t bytes = sizeof(T) * (size_t)m * p;
  const bool staged = bytes <= (size_t)CG_SMEM_MAX;
  if (staged && !attr_set.load()) {
    KP_CUDA(cudaFuncSetAttribute(k_cgs2<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, CG_SMEM_MAX));
    attr_set = true;
  }
  k_cgs2<T><<<1, CG_T, staged ? bytes : 0, ctx->stream>>>(Q, m, p, R, staged ? 1 : 0);
  KP_LAUNCHED(ctx);
  KP_CUDA(cudaGetLastError());
  return KP_OK;
}

template <typename T>
static kp_status topr_run(kp_ctx* ctx, const T* W, const T* WT, int m, int n, int r, int p, T* U, T* s, T* V,
                          int* iters_out) {
  cudaStream_t st = ctx->stream;
  T *Q, *Z, *Uz, *sz, *Vz, *Rz, *UR;
  int* jstat;
  KP_TRY(kp_alloc(ctx, (void**)&Q, sizeof(T) * (size_t)m * p));
  KP_TRY(kp_alloc(ctx, (void**)&Z, sizeof(T) * (size_t)n * p));
  KP_TRY(kp_alloc(ctx, (void**)&Uz, sizeof(T) * (size_t)n * p));
  KP_TRY(kp_alloc(ctx, (void**)&sz, sizeof(T) * p));
  KP_TRY(kp_alloc(ctx, (void**)&Vz, sizeof(T) * (size_t)p * p));
  KP_TRY(kp_alloc(ctx, (void**)&Rz, sizeof(T) * (size_t)p * p));
  KP_TRY(kp_alloc(ctx, (void**)&UR, sizeof(T) * (size_t)p * p));
  KP_TRY(kp_alloc(ctx, (void**)&jstat, sizeof(int)));
  KP_CUDA(cudaMemsetAsync(jstat, 0, sizeof(int), st));
  {  // start vectors: the first p columns of the m x m DCT-II matrix (smooth, orthonormal)
    double* C;
    KP_TRY(kp_alloc(ctx, (void**)&C, sizeof(double) * (size_t)m * m));
    KP_TRY(make_transform(ctx, m, 0, C));
    if (sizeof(T) == sizeof(double))
      KP_CUDA(cudaMemcpyAsync(Q, C, sizeof(double) * (size_t)m * p, cudaMemcpyDeviceToDevice, st));
    else
      KP_TRY(convert_f64_to_f32(ctx, C, (float*)Q, (long long)m * p));
  }
  // the Ritz step: Z = Q_z R_z (CGS2), then the one-block Jacobi SVD of the
  // p x p factor R_z = U_R S V_R^T, so that U_z = Q_z U_R, V_z = V_R
  const size_t small_smem = sizeof(T) * 2 * (size_t)p * p;
  const int gz = std::max(1, std::min((int)(((long long)n * p + 255) / 256), ctx->sm_count * 4));
  auto skinny = [&](const T* X, int rows, int ncol, const T* Y, T* out) -> kp_status {
    const long long threads = (long long)ncol * 32;
    k_skinny_tn<T><<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(X, rows, Y, rows, rows, ncol, p, out, ncol);
    KP_LAUNCHED(ctx);
    return KP_OK;
  };
  // settled when the leading Ritz values stop moving, relative to the largest:
  // 4 eps in FP64, 64 eps in FP32 (whose rounding noise is sqrt(n) eps)
  const double settle = (sizeof(T) == sizeof(double) ? 4.0 : 64.0) * Eps<T>::v;
  std::vector<T> prev(r, T(0)), cur(r, T(0));
  int it = 0;
  const int maxit = 200;
  for (it = 0; it < maxit; ++it) {
    if (it > 0) {  // the start vectors are orthonormal already
      KP_TRY(cgs2<T>(ctx, Q, m, p, nullptr));
    }
    KP_TRY(skinny(W, m, n, Q, Z));  // Z (n x p) = W^T Q
    KP_TRY(cgs2<T>(ctx, Z, n, p, Rz));  // Z <- Q_z
    k_jacobi_small<T><<<1, SJ_T, small_smem, st>>>(Rz, p, p, (T)ctx->jacobi_tol, ctx->jacobi_max_sweeps, UR, sz, Vz,
                                                   jstat);
    k_small_right<T><<<gz, 256, 0, st>>>(Z, n, p, UR, p, Uz);
    ctx->launches += 3;
    KP_CUDA(cudaMemcpyAsync(cur.data(), sz, sizeof(T) * r, cudaMemcpyDeviceToHost, st));
    KP_CUDA(kp_wait(ctx, st));
    double d = 0.0;
    for (int k = 0; k < r; ++k)
      d = std::max(d, std::fabs((double)cur[k] - (double)prev[k]) / std::max((double)cur[0], 1e-300));
    if (it > 0 && d <= settle) break;
    prev = cur;
    // Q (m x p) = W U_z, the span of W Z, with its columns already in the
    // order of the Ritz values
    KP_TRY(skinny(WT, n, m, Uz, Q));
  }
  if (it == maxit) {
    kp_set_error("topr_svd: subspace iteration did not settle in %d iterations", maxit);
    return KP_ENOCONV;
  }
  int h = 0;
  KP_CUDA(cudaMemcpyAsync(&h, jstat, sizeof(int), cudaMemcpyDeviceToHost, st));
  KP_CUDA(kp_wait(ctx, st));
  if (h) {
    kp_set_error("topr_svd: Ritz-step Jacobi did not converge in %d sweeps", ctx->jacobi_max_sweeps);
    return KP_ENOCONV;
  }
  // Z = W^T Q = V_W S (Q^T U_W)^T: U_z holds right singular vectors of W,
  // sz the values, V_z (p x p) gives the left vectors U = Q V_z
  KP_CUDA(cudaMemcpyAsync(V, Uz, sizeof(T) * (size_t)n * r, cudaMemcpyDeviceToDevice, st));
  KP_CUDA(cudaMemcpyAsync(s, sz, sizeof(T) * r, cudaMemcpyDeviceToDevice, st));
  const int gr = std::max(1, std::min((int)(((long long)m * r + 255) / 256), ctx->sm_count * 16));
  k_small_right<T><<<gr, 256, 0, st>>>(Q, m, p, Vz, r, U);
  KP_LAUNCHED(ctx);
  KP_CUDA(cudaGetLastError());
  if (iters_out) *iters_out = it + 1;
  return KP_OK;
}

kp_status topr_svd(kp_ctx* ctx, const double* W, int m, int n, int r, double* U, double* s, double* V,
                   int* iters_out) {
  cudaStream_t st = ctx->stream;
  const int p = std::min(n, r + 8);
  const long long mn = (long long)m * n;
  const int g = std::max(1, std::min((int)((mn + 255) / 256), ctx->sm_count * 16));
  if (p > SJ_MAXP) {  // wide subspace: Ritz values of Z by the multi-block Jacobi (FP64)
    kp_set_error("topr_svd: subspace of %d columns exceeds %d", p, SJ_MAXP);
    return KP_ENOTSUP;
  }
  if (!ctx->setup_fp32) {
    double* WT;
    KP_TRY(kp_alloc(ctx, (void**)&WT, sizeof(double) * mn));
    k_transpose_cm<double><<<g, 256, 0, st>>>(W, m, n, WT);
    KP_LAUNCHED(ctx);
    return topr_run<double>(ctx, W, WT, m, n, r, p, U, s, V, iters_out);
  }
  // FP32 arithmetic for FP32 vectors: the PSF terms to FP32 accuracy
  float *W32, *WT32, *U32, *s32, *V32;
  KP_TRY(kp_alloc(ctx, (void**)&W32, sizeof(float) * mn));
  KP_TRY(kp_alloc(ctx, (void**)&WT32, sizeof(float) * mn));
  KP_TRY(kp_alloc(ctx, (void**)&U32, sizeof(float) * (size_t)m * r));
  KP_TRY(kp_alloc(ctx, (void**)&s32, sizeof(float) * r));
  KP_TRY(kp_alloc(ctx, (void**)&V32, sizeof(float) * (size_t)n * r));
  KP_TRY(convert_f64_to_f32(ctx, W, W32, mn));
  k_transpose_cm<float><<<g, 256, 0, st>>>(W32, m, n, WT32);
  KP_LAUNCHED(ctx);
  KP_TRY(topr_run<float>(ctx, W32, WT32, m, n, r, p, U32, s32, V32, iters_out));
  KP_TRY(convert_f32_to_f64(ctx, U32, U, (long long)m * r));
  KP_TRY(convert_f32_to_f64(ctx, s32, s, r));
  return convert_f32_to_f64(ctx, V32, V, (long long)n * r);
}
