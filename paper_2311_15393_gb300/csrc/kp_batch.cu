// Batched independent deblurring problems of uneven sizes (kp_solve_batch).
//
// Each problem is what kp_setup + choose_lambda + tik_pcg compute for it
// alone (Sections 3-5: KP-SVD preconditioned (F)PCG on the Tikhonov normal
// equations, lambda by GCV / discrepancy / ...).  Concurrency: `workers` host
// threads, each with its own context on its own non-blocking stream, take
// the problems largest first from a shared counter, so the GPU overlaps the
// kernels (and the host round trips) of different problems; results do not
// depend on which worker ran a problem.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "kp_internal.h"

namespace {

struct WorkerResult {
  kp_status first = KP_OK;
  int first_idx = -1;
  std::string msg;
};

void run_worker(int device, kp_problem* probs, const std::vector<int>& order, std::atomic<int>* next,
                const kp_batch_opts& o, WorkerResult* res) {
  auto fail = [&](int idx, kp_status s) {
    if (res->first_idx < 0 || idx < res->first_idx) {
      res->first = s;
      res->first_idx = idx;
      res->msg = kp_last_error();
    }
  };
  if (cudaSetDevice(device) != cudaSuccess) {
    kp_set_error("kp_solve_batch: cudaSetDevice(%d) failed", device);
    fail(order.empty() ? 0 : order[0], KP_ECUDA);
    return;
  }
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    kp_set_error("kp_solve_batch: stream creation failed");
    fail(order.empty() ? 0 : order[0], KP_ECUDA);
    return;
  }
  kp_ctx* ctx = nullptr;
  kp_status cs = kp_create(&ctx, device, st);
  // ill-conditioned problems of a BF16-operator batch get the BF16X3 inner
  // operator (one threshold for all problems; see op_auto_cond)
  const double auto_cond = 1e4;
  const bool bf16 = o.op_prec == KP_BF16;
  if (cs == KP_OK && bf16) cs = kp_set_option(ctx, "op_auto_cond", auto_cond);
  for (;;) {
    const int k = next->fetch_add(1);
    if (k >= (int)order.size()) break;
    const int i = order[k];
    kp_problem& p = probs[i];
    kp_status s = cs;
    if (s == KP_OK)
      s = kp_setup(ctx, p.psf, p.n_r, p.n_c, p.center_r, p.center_c, p.bc, p.op_rank, 1, o.op_prec, o.pc_prec,
                   o.vec_prec, o.sigma);
    double lam = p.lambda;
    if (s == KP_OK && !(lam > 0.0)) s = choose_lambda(ctx, p.b, o.method, p.lambda_param, nullptr, &lam);
    if (s == KP_OK) {
      p.lambda = lam;
      s = tik_pcg(ctx, p.b, lam, o.tol, o.maxit, o.flexible, p.x, 0, &p.info);
      if (bf16 && ctx->op_prec == KP_BF16 && (s == KP_ENOCONV || s == KP_EBREAKDOWN || s == KP_ENUMERIC)) {
        // the BF16 inner operator stalled or broke down below the threshold:
        // solve again from x = 0 with the BF16X3 inner operator
        kp_status so = kp_set_option(ctx, "op_auto_cond", 1.0);
        if (so == KP_OK) s = tik_pcg(ctx, p.b, lam, o.tol, o.maxit, o.flexible, p.x, 0, &p.info);
        kp_set_option(ctx, "op_auto_cond", auto_cond);
      }
    } else {
      p.info.status = s;
    }
    if (s != KP_OK) fail(i, s);
  }
  if (ctx) kp_destroy(ctx);
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
}

}  // namespace

extern "C" kp_status kp_solve_batch(int device, kp_problem* probs, int nprob, const kp_batch_opts* opts,
                                    double* ms_total) {
  if (!opts || nprob < 0 || (nprob > 0 && !probs)) {
    kp_set_error("kp_solve_batch: NULL argument or nprob < 0");
    return KP_EINVAL;
  }
  for (int i = 0; i < nprob; ++i) {
    if (!probs[i].psf || !probs[i].b || !probs[i].x || probs[i].n_r < 1 || probs[i].n_c < 1) {
      kp_set_error("kp_solve_batch: problem %d has a NULL pointer or an empty size", i);
      return KP_EINVAL;
    }
    probs[i].info.status = KP_OK;
    probs[i].info.iters = 0;
    probs[i].info.replacements = 0;
  }
  const auto t0 = std::chrono::steady_clock::now();
  // largest problems first (the longest run in the tail is then a small one)
  std::vector<int> order(nprob);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (long long)probs[a].n_r * probs[a].n_c > (long long)probs[b].n_r * probs[b].n_c;
  });
  const int nw = std::max(1, std::min(opts->workers > 0 ? opts->workers : 8, std::max(nprob, 1)));
  std::atomic<int> next{0};
  std::vector<WorkerResult> res(nw);
  std::vector<std::thread> threads;
  threads.reserve(nw);
  for (int w = 0; w < nw; ++w)
    threads.emplace_back(run_worker, device, probs, std::cref(order), &next, std::cref(*opts), &res[w]);
  for (auto& t : threads) t.join();
  if (ms_total)
    *ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  const WorkerResult* first = nullptr;
  for (const auto& r : res)
    if (r.first_idx >= 0 && (!first || r.first_idx < first->first_idx)) first = &r;
  if (first) {
    kp_set_error("kp_solve_batch: problem %d: %s", first->first_idx, first->msg.c_str());
    return first->first;
  }
  return KP_OK;
}
