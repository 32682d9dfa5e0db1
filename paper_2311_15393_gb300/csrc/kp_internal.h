// Internal declarations of the KP-SVD deblurring library (sm_103a).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <utility>
#include <vector>

#include "../../include/kpsvd.h"

// ---------------------------------------------------------------- errors
void kp_set_error(const char* fmt, ...);

#define KP_CUDA(call)                                                                 \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      kp_set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
      return KP_ECUDA;                                                                \
    }                                                                                 \
  } while (0)

#define KP_TRY(call)              \
  do {                            \
    kp_status s_ = (call);        \
    if (s_ != KP_OK) return s_;   \
  } while (0)

#define KP_LAUNCHED(ctx) \
  do { (ctx)->launches++; } while (0)

// device status word bits (written by kernels, read by the host at sync points)
enum : int { DEV_ERR_TIMEOUT = 1, DEV_ERR_NUMERIC = 2, DEV_ERR_BREAKDOWN = 4, DEV_ERR_BOUNDS = 8 };

// Programmatic dependent launch.  Kernels of the iteration are launched with
// programmatic stream serialization, so a kernel's launch and prologue
// overlap the tail of the one before it.  Each such kernel executes
// KP_PDL_WAIT() (wait until the preceding grid has completed and its writes
// are visible) before it reads or writes anything another kernel touches,
// and before any early return; KP_PDL_TRIGGER() lets the next grid launch.
#define KP_PDL_WAIT() asm volatile("griddepcontrol.wait;" ::: "memory")
#define KP_PDL_TRIGGER() asm volatile("griddepcontrol.launch_dependents;" ::: "memory")

// bounded spin limit for device-side waits (each try_wait already suspends
// for a hardware-defined interval, so this is a few seconds at most)
constexpr long long KP_SPIN_LIMIT = 1LL << 24;

// ---------------------------------------------------------------- GEMM descriptors
// D[m][n] = sum_{pair p} sum_{term k} sum_kk A[ta][m][kk] * B[tb][n][kk],
// ta = sa[p] * a_terms + k, tb = sb[p] * b_terms + k; A and B are K-major
// (row-major rows x K with leading dimension ld, one block per term index).
enum EpiMode : int {
  EPI_F32 = 0,     // out_f32 = alpha * acc + beta * aux           (aux optional)
  EPI_SLICES = 1,  // v = alpha * acc + beta * aux; out = ns bf16 slices of v
  EPI_NARROW = 2,  // v = alpha * acc [* lam2 / (sigma^2 + lam2)]; out = narrow type
  EPI_T = 3,       // SIMT: out_T = alpha * acc + beta * aux [* sigma factor]
  EPI_PARTIAL = 4  // split-K partial: ws[split][m][n] = acc (fp32)
};
enum NarrowType : int { NT_BF16 = 0, NT_F16 = 1, NT_E4M3 = 2 };

constexpr int KP_MAX_PAIRS = 6;

struct GemmOp {
  const void* ptr = nullptr;
  int rows = 0;           // M (A) or N (B)
  int K = 0;
  long long ld = 0;       // elements between rows
  long long tstride = 0;  // elements between term blocks
  int nterm_idx = 0;      // number of term blocks present (for the TMA map)
};

struct EpiParams {
  int mode = EPI_F32;
  void* out = nullptr;
  long long ldd = 0;
  int slices = 1;
  long long slice_stride = 0;
  double alpha = 1.0, beta = 0.0;
  const void* aux = nullptr;  // same index as out (T or float)
  long long ld_aux = 0;
  const float* sigma32 = nullptr;
  const double* sigma64 = nullptr;
  double lam2 = 0.0;
  int narrow = NT_BF16;
  unsigned int* amax_bits = nullptr;  // EPI_F32: atomicMax of max |out| (bits of a non-negative float)
  // EPI_F32 only (the learned-lambda MLP): + bias[n]; act 1: pre[m][n] =
  // the value, out = GELU(value); act 2: out = value * GELU'(pre[m][n]);
  // pre has the indexing of out
  const float* bias = nullptr;
  float* pre = nullptr;
  int act = 0;
};

// GELU(z) = z Phi(z) with the normal CDF Phi, and its derivative
__device__ __forceinline__ float kp_phi(float z) { return 0.5f * erfcf(-z * 0.70710678118654752f); }
__device__ __forceinline__ float kp_gelu(float z) { return z * kp_phi(z); }
__device__ __forceinline__ float kp_gelu_grad(float z) {
  return kp_phi(z) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

struct GemmDesc {
  int M = 0, N = 0, K = 0;
  int nkron = 1;        // k runs over [0, nkron)
  int npairs = 1;
  int sa[KP_MAX_PAIRS] = {0}, sb[KP_MAX_PAIRS] = {0};
  int a_terms = 1, b_terms = 1;  // term blocks per slice
  GemmOp A, B;
  EpiParams epi;
  const int* flags = nullptr;  // when non-null and *flags != 0 the launch does nothing
  // > 0: batched over terms instead of summed: output rows [k * batch_rows,
  // (k + 1) * batch_rows) are the product with term k alone (M = nkron *
  // batch_rows); the caller sums the per-term outputs
  int batch_rows = 0;
  // > 0: one product summed over all k-blocks on 128 x 64 tiles
  // (tc_gemm_kcat_kernel), in clusters of this many CTAs (1 or 4; 4: the A
  // tile shared by multicast), where the shape allows it (BF16, no K split,
  // not batched, whole clusters of tiles along N); otherwise the plan falls
  // back to the usual choice
  int kcat = 0;
};

// ---------------------------------------------------------------- context
struct TcGemmPlan;  // prepared tensor-core GEMM (tensor maps + params)

struct kp_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;       // private work stream (capturable)
  cudaStream_t user_stream = nullptr;  // caller's stream, ordered with `stream` by events
  bool own_stream = false;             // `stream` is private (caller passed the legacy stream)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  void* ops_state = nullptr;
  int* dflags = nullptr;               // device solver flags
  int sm_count = 0;
  long long launches = 0;

  // problem
  bool ready = false;
  int n_r = 0, n_c = 0, c_r = 0, c_c = 0, rank = 0;
  int pc_rank = 1;          // Kronecker terms behind the preconditioner (1: the KP-SVD solve)
  int pc_inner_iters = 2;   // inner PCG steps of a multi-term preconditioner
  kp_bc bc = KP_BC_ZERO;
  kp_prec op_prec = KP_F64, pc_prec = KP_F64, vec_prec = KP_F64;
  kp_prec op_prec_setup = KP_F64;  // op_prec given to kp_setup (op_prec may be raised per solve)
  double sigma_max = -1.0;         // max |Sigma| of the current setup (< 0: not computed yet)
  kp_sigma sigma_mode = KP_SIGMA_PROJECTED;

  // options
  double reliable_delta = -1.0;  // < 0: default for the operator precision
  int check_every = 2;
  double pc_lambda_ratio = 1.0;  // preconditioner lambda / system lambda
  double op_auto_cond = 0.0;  // > 0: BF16 inner operator raised to BF16X3 when cond(K) exceeds it
  bool cg_fuse = true;  // the x / r update also writes the preconditioner's narrow input (where possible)
  double jacobi_tol = 1e-15;  // raised to m * eps inside the SVD
  int jacobi_max_sweeps = 40;
  bool jacobi_block = true;   // FP32 sweeps in the register block form (k_jacobi_rblock) where it fits
  bool jacobi_warm_u = true;  // second factor-SVD run (U from F^T) starts from the first run's V
  bool pdl = true;           // programmatic dependent launch in the iteration
  bool device_loop = true;   // (F)PCG loop as a device-side graph while loop (host loop: false)
  cudaStream_t aux_stream = nullptr;  // second capture stream (nested graph bodies)
  void* hmirror = nullptr;   // pinned host copies of the solver flags / scalars (2 slots)
  cudaEvent_t ev_blk[2] = {nullptr, nullptr};
  cudaEvent_t ev_setup[2] = {nullptr, nullptr};  // timing of kp_setup
  double last_setup_ms = 0.0;                     // device time of the last kp_setup
  int splitk_override = 0;  // > 0: fixed split-K factor for the square GEMMs
  int tc_bn_override = 0;   // 128 / 256: fixed tensor-core tile width
  int tc_cps_override = 0;  // 1 / 2: fixed CTAs per SM for 128-wide tiles
  int tc_kps_override = 0;  // 1 / 2: fixed k-blocks per ring stage
  int tc_pair_override = 0;  // 1: no CTA-pair tiles; 2: CTA-pair tiles wherever the shape allows
  int tc_kcat = 0;  // G2 / G4 of the inner operator as one K-concatenated GEMM: 0 never, 1 where its tiles fill most SMs, 2 wherever the shape allows
  int tc_kcat_cluster = 1;  // CTAs per cluster of those GEMMs: 1, or 4 (A tiles shared by multicast)
  bool tc_autotune = false;  // pick each GEMM shape's tile configuration by timing (cached)

  // device allocations: ctx_block lives with the context, allocs with the
  // problem; a new kp_setup returns the previous problem's blocks to `pool`,
  // from which kp_alloc serves requests before calling cudaMalloc
  void* ctx_block = nullptr;
  std::vector<std::pair<void*, size_t>> allocs;
  std::multimap<size_t, void*> pool;
  // FP32 arithmetic for the O(n^3) products of the setup and of the spectral
  // coefficients (factor SVD products, projected spectrum, U^T B U): on for
  // FP32 vectors unless the "setup_fp64" option is set
  bool setup_fp32 = false;
  bool force_setup_fp64 = false;
  // half-precision setup (the paper's future work, Section 3 after eq.
  // PreconSolve): the products that form V_c, V_r and the spectrum take bf16
  // inputs with FP32 accumulation on the tensor cores (FP32 vectors only)
  bool setup_half = false;
  bool force_setup_half = false;
  // the setup's FP32 products on the tensor cores (inputs as three bf16
  // slices, six slice products): FP32 vectors, a tcgen05 device, sizes
  // multiples of 16
  bool setup_tc = false;
  // choose_lambda's spectral coefficients on the tensor cores (built once
  // per setup): per basis (0: U, 1: V) the bases' slices and the two plans
  struct LamTc {
    void* L16 = nullptr;
    void* R16 = nullptr;
    TcGemmPlan* p1 = nullptr;
    TcGemmPlan* p2 = nullptr;
  } lam_tc[2];
  void* lam_img16 = nullptr;  // slices of the image and of the intermediate
  void* lam_t16 = nullptr;
  float* lam_t32 = nullptr;   // FP32 intermediate and result
  float* lam_o32 = nullptr;
  int* dev_status = nullptr;     // device status word
  double* dscal = nullptr;       // device scalars (see kp_solver.cu)
  double* red_part = nullptr;    // reduction partials
  unsigned int* red_count = nullptr;

  // FP64 masters
  double* s_terms = nullptr;  // rank
  double* u_terms = nullptr;  // n_r x rank (col-major)
  double* v_terms = nullptr;  // n_c x rank
  double* Ac64 = nullptr;     // [rank][n_r][n_r] row-major A_c^(k)
  double* Ar64 = nullptr;     // [rank][n_c][n_c] row-major A_r^(k)
  double *Ur = nullptr, *Vr = nullptr, *sr = nullptr;  // col-major n_c x n_c
  double *Uc = nullptr, *Vc = nullptr, *sc = nullptr;  // col-major n_r x n_r
  double* Sigma64 = nullptr;  // n_r x n_c col-major
  float* Sigma32 = nullptr;
  // FP32 copies of the factor bases (setup_fp32 only), col-major
  float *Uc32 = nullptr, *Ur32 = nullptr, *Vc32 = nullptr, *Vr32 = nullptr;

  // operator factors in the four GEMM layouts (T = op type, or bf16 slices)
  void* opAc = nullptr;   // G1: [slice][k][i'][i] = A_c^(k)[i', i]
  void* opAr = nullptr;   // G2: [slice][k][l][j]  = A_r^(k)[l, j]
  void* opAcT = nullptr;  // G3: [slice][k][i'][i] = A_c^(k)[i, i']
  void* opArT = nullptr;  // G4: [slice][k][l][j]  = A_r^(k)[j, l]
  int op_slices = 1;
  // preconditioner factors (pc type), row-major
  void* pcVcT = nullptr;  // P1 A: V_c^T
  void* pcVrT = nullptr;  // P2 A: V_r^T
  void* pcVc = nullptr;   // P3 A: V_c
  void* pcVr = nullptr;   // P4 A: V_r
  float pc_vscale_c = 1.f, pc_vscale_r = 1.f;  // power-of-two factor scales (E4M3)

  // workspaces (sized by kp_setup)
  void* w_stack = nullptr;   // G1/G3 outputs: [slices][rank * n_r][n_c]
  void* w_img = nullptr;     // G2 outputs / inputs of G3: [slices][n_r * n_c]
  void* w_img2 = nullptr;    // p slices (inner operator input)
  void* w_img3 = nullptr;    // x slices (accurate operator input)
  double* hist = nullptr;    // residual history (device)
  void* lam_ws = nullptr;    // choose_lambda scratch (allocated at its first call)
  bool lam_sigma_ready = false;  // spectrum-only part of lam_ws filled (once per setup)
  double lam_sigma_ext[2] = {0.0, 0.0};  // max |Sigma|, min |Sigma| > 0
  int hist_cap = 0;
  float* w_split = nullptr;  // split-K partials
  long long w_split_elems = 0;
  // SIMT GEMMs with fewer output tiles than SMs split their (pair, term,
  // k-tile) steps over blocks; partial tiles go here (null: no split)
  void* simt_ws = nullptr;
  size_t simt_ws_bytes = 0;
  void* pc_in = nullptr;     // quantised residual R
  void* pc_t1 = nullptr;     // P1 out
  void* pc_t2 = nullptr;     // P2 out
  void* pc_t3 = nullptr;     // P3 out
  float* pc_f32 = nullptr;   // FP32 staging for E4M3 dynamic scaling
  void* vbuf[10] = {nullptr};  // solver vectors (vec type)
  void* pc_inner[5] = {nullptr};  // multi-term preconditioner's inner r, r_old, p, q, z
  void* tmp_img = nullptr;   // vec-type scratch image
  void* tmp_img2 = nullptr;

  // prepared tensor-core GEMM plans
  std::vector<TcGemmPlan*> tc_plans;

  // batched solves: while set, launches are recorded here instead of run
  struct KpRecorder* rec = nullptr;
  // batched solves: the setups of several problems run as cooperative fibers
  // on one host thread; while `yield` is set, kp_wait hands the thread to the
  // other problems instead of blocking
  void* jac_cache = nullptr;  // instantiated Jacobi sweep graphs (kp_jacobi.cu)
  void (*yield)(void*) = nullptr;
  void* yield_arg = nullptr;
  cudaEvent_t ev_wait = nullptr;
  bool tc_group = false;     // batched solve: the operator's and preconditioner's plans run in grouped launches
  bool tc_grouping = false;  // set while those plans are made: no K split, no CTA pairs
  bool tc_group_uniform = true;  // ... and one tile shape (128 wide, one CTA per SM) for all problems
};

// ---------------------------------------------------------------- recorded launches
// A batched solve runs one iteration of each problem in recording mode: each
// launch becomes a KpRec (its arguments as bytes) instead of running.  The
// records at the same position of the problems' sequences that share a
// kernel (`key`) then become one grouped launch: `table` writes their
// arguments into a device table (before graph capture), `launch` runs the
// grouped kernel over them.
struct KpRec {
  const void* key = nullptr;
  size_t (*table_bytes)(int n) = nullptr;
  void (*table)(const KpRec* const* recs, int n, unsigned char* host_dst) = nullptr;
  kp_status (*launch)(kp_ctx* ctx, const KpRec* const* recs, int n, const void* dev_table) = nullptr;
  dim3 grid, block;
  size_t smem = 0;
  std::vector<unsigned char> blob;
};
struct KpRecorder {
  std::vector<KpRec> recs;
};

// one problem's solve around a grouped loop (kp_solver.cu; driven by kp_batch.cu)
struct BatchRun;
kp_status batch_begin(kp_ctx* ctx, const void* b, double lambda, double tol, int maxit, int flexible, void* x,
                      BatchRun** out);
bool batch_groupable(const BatchRun* br);
bool batch_needs_loop(const BatchRun* br);
kp_status batch_record(kp_ctx* ctx, BatchRun* br, KpRecorder* seg_a, KpRecorder* seg_r, KpRecorder* seg_b);
kp_status batch_arm(kp_ctx* ctx, BatchRun* br);
kp_status batch_finish(kp_ctx* ctx, BatchRun* br, kp_solve_info* info);
void batch_discard(BatchRun* br);

// launch with programmatic stream serialization (when ctx->pdl); the kernel
// must begin with KP_PDL_WAIT()
template <typename... KArgs, typename... Args>
inline cudaError_t kp_launch(const kp_ctx* ctx, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                             Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = ctx->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = ctx->pdl ? 1 : 0;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// allocation helper: registers the pointer with the context
kp_status kp_alloc(kp_ctx* ctx, void** p, size_t bytes);
void kp_free_all(kp_ctx* ctx);    // problem blocks -> pool
void kp_pool_release(kp_ctx* ctx);  // cudaFree the pool

// ---------------------------------------------------------------- kernels (host launchers)
// SIMT GEMM (double or float)
template <typename T>
kp_status simt_gemm(kp_ctx* ctx, const GemmDesc& g);

// tensor-core GEMM: prepare a plan (tensor maps) once, run it many times
enum TcKind : int { TC_BF16 = 0, TC_F16 = 1, TC_E4M3 = 2 };
kp_status tc_plan_create(kp_ctx* ctx, const GemmDesc& g, int kind, int splits, TcGemmPlan** out);
kp_status tc_plan_run(kp_ctx* ctx, TcGemmPlan* plan, const EpiParams* epi_override);
void tc_plan_set_epi(TcGemmPlan* plan, const EpiParams& e);
bool tc_device_supported(kp_ctx* ctx);
// D (rows_a x rows_b row-major FP32) = A B^T, A rows_a x K and B rows_b x K
// FP64 K-major, with bf16 inputs and FP32 accumulation on the tensor cores
kp_status half_product(kp_ctx* ctx, const double* A, int rows_a, const double* B, int rows_b, int K, float* D);
// the same with FP64 or FP32 inputs as 1 (half precision) or 3 (exact FP32
// split, six slice products) bf16 slices
kp_status tc_product(kp_ctx* ctx, const void* A, bool a64, int rows_a, const void* B, bool b64, int rows_b, int K,
                     float* D, int slices);
// pieces of tc_product for reuse: bf16 slices of an operand (out: slices x n)
// and the plan of D = A B^T from sliced operands
kp_status tc_operand_slices(kp_ctx* ctx, const void* in, bool f64, long long n, int slices, void* out);
kp_status tc_product_plan(kp_ctx* ctx, const void* a16, int rows_a, const void* b16, int rows_b, int K, int slices,
                          float* D, TcGemmPlan** out);

// one-sided Jacobi SVD (FP64): A (m x n col-major, m >= n) -> U (m x n), s (n), V (n x n)
kp_status jacobi_svd(kp_ctx* ctx, const double* A, int m, int n, double* U, double* s, double* V,
                     int* sweeps_out);
// SVD F = U diag(s) V^T of a square blur factor given row-major; transform 0 =
// DCT-II (reflexive BC), 1 = DST-I (zero BC) preconditioning
kp_status factor_svd(kp_ctx* ctx, const double* F_rm, int n, int transform, double* U, double* s, double* V,
                     int* sweeps_out);
// leading r singular triplets of W (m x n col-major, m >= n) by subspace iteration
kp_status topr_svd(kp_ctx* ctx, const double* W, int m, int n, int r, double* U, double* s, double* V,
                   int* iters_out);

// vector / reduction helpers (kp_vec.cu)
kp_status dot_dev(kp_ctx* ctx, const void* x, const void* y, long long n, bool f64, double* out_dev);
kp_status norm2_dev(kp_ctx* ctx, const void* x, long long n, bool f64, double* out_dev);
kp_status split_bf16(kp_ctx* ctx, const void* x, bool f64, long long n, void* out, int slices,
                     long long slice_stride, const int* flags = nullptr);
kp_status copy_vec(kp_ctx* ctx, const void* x, void* y, long long n, bool f64);
kp_status read_status(kp_ctx* ctx);
// wait until the work queued on st so far is done (cudaStreamSynchronize, or,
// inside a batched solve's fiber, yield to the other fibers until it is)
cudaError_t kp_wait(kp_ctx* ctx, cudaStream_t st);
void jacobi_cache_free(kp_ctx* ctx);
kp_status kp_check_ready(kp_ctx* ctx);
kp_status kp_enter(kp_ctx* ctx);   // order the work stream after the caller's stream
kp_status kp_leave(kp_ctx* ctx);   // order the caller's stream after the work stream
void tc_plan_set_runtime(TcGemmPlan* plan, const float* alpha_dev, const int* flags);
// whether the plan is a K-concatenated product (tc_gemm_kcat_kernel, which
// can fuse the output's dot reduction into its epilogue: tc_plan_run_dot in
// kp_vec.cuh)
bool tc_plan_is_kcat(const TcGemmPlan* plan);
void tc_plan_release(kp_ctx* ctx, TcGemmPlan* plan);  // free a plan before the context does
