// Batched independent deblurring problems of uneven sizes (kp_solve_batch).
//
// Each problem is what kp_setup + choose_lambda + tik_pcg compute for it
// alone (Sections 3-5: KP-SVD preconditioned (F)PCG on the Tikhonov normal
// equations, lambda by GCV / discrepancy / ...).
//
// Default (grouped): one host thread and one context per problem.  Setup,
// lambda and the steps before the iterations run problem by problem; then
// one iteration of every problem is recorded (kp_group.cuh: launches kept as
// argument records), and the records at each position of the iteration
// become ONE launch over all problems: a persistent tensor-core GEMM over
// the (problem, tile) units of all problems' plans (tc_gemm_group_kernel,
// per-problem tensor maps in a device table), or a vector kernel with one
// blockIdx.y per problem.  The whole iteration of all problems is one CUDA
// graph with a device-side while loop; each problem's flags say whether it
// still runs (a stopped problem's launches do no work), whether its residual
// replacement is due (the replacement runs inside an if node, skipped by the
// problems for which none is due), and the loop ends when no problem runs.
// Tile shapes are each plan's (the per-shape choice, or the timed one with
// the tc_autotune option and its cache file).
//
// workers > 0: the former form, `workers` host threads, each with its own
// context on its own stream, taking the problems largest first.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include <sys/mman.h>
#include <ucontext.h>
#include <unistd.h>

#include "kp_internal.h"
#include "kp_vec.cuh"

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

static kp_status solve_grouped(int device, kp_problem* probs, int nprob, const kp_batch_opts* opts);

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
  if (opts->workers <= 0) {
    const kp_status gs = solve_grouped(device, probs, nprob, opts);
    if (ms_total)
      *ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return gs;
  }
  // largest problems first (the longest run in the tail is then a small one)
  std::vector<int> order(nprob);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (long long)probs[a].n_r * probs[a].n_c > (long long)probs[b].n_r * probs[b].n_c;
  });
  const int nw = std::max(1, std::min(opts->workers, std::max(nprob, 1)));
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

// ---------------------------------------------------------------- grouped form
namespace {

// The loop condition of the grouped graph: h = whether any problem's flag
// `slot` is nonzero (want_zero: is zero).  With `passes` (the while loop's
// condition), also a bound on the passes, so that the loop ends even if a
// problem's flags never stop it (each problem also stops itself a few
// passes past maxit).
__global__ void k_batch_any(int* const* __restrict__ flags, int n, int slot, int want_zero, int* passes,
                            int max_passes, cudaGraphConditionalHandle h) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int v = *(volatile const int*)(flags[i] + slot);
    if (want_zero ? v == 0 : v != 0) any = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int go = any ? 1u : 0u;
    if (passes && ++*passes > max_passes) go = 0u;
    cudaGraphSetConditional(h, go);
  }
}

// Contexts and buffers kept from one call to the next on a device (the
// problems' buffers are reused when the sizes repeat); kp_batch_release
// frees them.
struct GroupPool {
  std::mutex mu;
  std::vector<kp_ctx*> ctxs;
  unsigned char* dev = nullptr;
  size_t dev_bytes = 0;
  int last_grouped = 0;  // problems the last call's grouped loop ran
  int last_passes = 0;   // passes of that loop
  double last_ms[3] = {0.0, 0.0, 0.0};  // host wall time: before the loop, building it, running it
  int last_shape[6] = {0, 0, 0, 0, 0, 0};  // first epoch: launch positions and grouped launches per
                                           // pass (outside the replacement), the same inside it;
                                           // then the setups' fibers (1: ran as fibers) and yields
};
long long g_yields = 0;
std::mutex g_pools_mu;
std::map<int, GroupPool*> g_pools;

GroupPool* group_pool(int device) {
  std::lock_guard<std::mutex> lock(g_pools_mu);
  auto it = g_pools.find(device);
  if (it != g_pools.end()) return it->second;
  GroupPool* p = new GroupPool();
  g_pools[device] = p;
  return p;
}

// one grouped launch: the records of one kernel at one position
struct Group {
  std::vector<const KpRec*> recs;
  size_t off = 0;  // its table in the device buffer
};

// Positions of one segment across the problems: the records at position k
// of every problem, split by kernel.
kp_status plan_segment(const std::vector<KpRecorder*>& segs, std::vector<Group>* out, size_t* bytes) {
  const size_t len = segs[0]->recs.size();
  for (size_t k = 0; k < len; ++k) {
    std::vector<const void*> keys;
    std::vector<Group> gs;
    for (KpRecorder* r : segs) {
      const KpRec* rec = &r->recs[k];
      size_t g = 0;
      while (g < keys.size() && keys[g] != rec->key) ++g;
      if (g == keys.size()) {
        keys.push_back(rec->key);
        gs.emplace_back();
      }
      gs[g].recs.push_back(rec);
    }
    for (Group& g : gs) {
      g.off = *bytes;
      *bytes += (g.recs[0]->table_bytes((int)g.recs.size()) + 255) & ~(size_t)255;
      out->push_back(std::move(g));
    }
  }
  return KP_OK;
}

kp_status launch_groups(kp_ctx* dctx, const std::vector<Group>& gs, const unsigned char* dev) {
  for (const Group& g : gs) KP_TRY(g.recs[0]->launch(dctx, g.recs.data(), (int)g.recs.size(), dev + g.off));
  return KP_OK;
}

}  // namespace

extern "C" int kp_batch_grouped(int device, int* passes, double* ms, int* shape) {
  GroupPool* p = group_pool(device);
  std::lock_guard<std::mutex> lock(p->mu);
  if (passes) *passes = p->last_passes;
  if (ms)
    for (int i = 0; i < 3; ++i) ms[i] = p->last_ms[i];
  if (shape)
    for (int i = 0; i < 6; ++i) shape[i] = p->last_shape[i];
  return p->last_grouped;
}

extern "C" void kp_batch_release(int device) {
  GroupPool* p = group_pool(device);
  std::lock_guard<std::mutex> lock(p->mu);
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  for (kp_ctx* c : p->ctxs) kp_destroy(c);
  p->ctxs.clear();
  if (p->dev) cudaFree(p->dev);
  p->dev = nullptr;
  p->dev_bytes = 0;
  if (prev >= 0) cudaSetDevice(prev);
}

// ---- cooperative fibers (one host thread): run work[k] on ctxs[k] as fibers
// that yield at their GPU waits (kp_wait); the scheduler resumes them in turn
// until all have finished.  Each fiber has its own stack with a guard page.
struct Fiber {
  ucontext_t uc;
  void* mem = nullptr;
  size_t bytes = 0;
  std::function<void()>* fn = nullptr;
  bool done = false;
  ucontext_t* main = nullptr;
};
static void fiber_entry(unsigned lo, unsigned hi) {
  Fiber* f = reinterpret_cast<Fiber*>((uintptr_t)lo | ((uintptr_t)hi << 32));
  (*f->fn)();
  f->done = true;
  swapcontext(&f->uc, f->main);
}
static void fiber_yield(void* arg) {
  Fiber* f = static_cast<Fiber*>(arg);
  ++g_yields;
  swapcontext(&f->uc, f->main);
}
static kp_status run_fibers(std::vector<std::function<void()>>& work, const std::vector<kp_ctx*>& ctxs) {
  constexpr size_t STACK = 2u << 20;
  const size_t page = (size_t)sysconf(_SC_PAGESIZE);
  const int n = (int)work.size();
  std::vector<Fiber> fs(n);
  ucontext_t main_uc;
  kp_status st = KP_OK;
  for (int k = 0; k < n && st == KP_OK; ++k) {
    Fiber& f = fs[k];
    f.bytes = STACK + page;
    f.mem = mmap(nullptr, f.bytes, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    if (f.mem == MAP_FAILED) {
      f.mem = nullptr;
      st = KP_ENOMEM;
      break;
    }
    mprotect(f.mem, page, PROT_NONE);  // guard page below the stack
    if (getcontext(&f.uc) != 0) {
      st = KP_EINVAL;
      break;
    }
    f.uc.uc_stack.ss_sp = static_cast<char*>(f.mem) + page;
    f.uc.uc_stack.ss_size = STACK;
    f.uc.uc_link = nullptr;
    f.fn = &work[k];
    f.main = &main_uc;
    const uintptr_t a = reinterpret_cast<uintptr_t>(&f);
    makecontext(&f.uc, reinterpret_cast<void (*)()>(fiber_entry), 2, (unsigned)(a & 0xffffffffu), (unsigned)(a >> 32));
  }
  if (st == KP_OK) {
    for (int k = 0; k < n; ++k) {
      ctxs[k]->yield = fiber_yield;
      ctxs[k]->yield_arg = &fs[k];
    }
    for (int left = n; left > 0;) {
      left = 0;
      for (int k = 0; k < n; ++k) {
        if (fs[k].done) continue;
        swapcontext(&main_uc, &fs[k].uc);
        if (!fs[k].done) ++left;
      }
    }
    for (int k = 0; k < n; ++k) {
      ctxs[k]->yield = nullptr;
      ctxs[k]->yield_arg = nullptr;
    }
  }
  for (Fiber& f : fs)
    if (f.mem) munmap(f.mem, f.bytes);
  return st;
}

// One epoch of the grouped loop over the problems `act` (all armed, their
// iterations of equal shape): record one iteration of each, build the graph
// while (any runs and fewer than max_passes) { first halves; if (any
// replacement due) { replacements }; second halves }, run it; *done = passes.
static kp_status run_epoch(GroupPool* pool, const std::vector<int>& act, const std::vector<BatchRun*>& runs,
                           int max_passes, int* done) {
  using clk = std::chrono::steady_clock;
  const clk::time_point t0 = clk::now();
  *done = 0;
  const int n = (int)act.size();
  std::vector<KpRecorder> ra(n), rr(n), rb(n);
  for (int j = 0; j < n; ++j) KP_TRY(batch_record(pool->ctxs[act[j]], runs[act[j]], &ra[j], &rr[j], &rb[j]));
  std::vector<KpRecorder*> sa, sr, sb;
  for (int j = 0; j < n; ++j) {
    sa.push_back(&ra[j]);
    sr.push_back(&rr[j]);
    sb.push_back(&rb[j]);
  }
  std::vector<Group> ga, gr, gb;
  size_t bytes = 0;
  plan_segment(sa, &ga, &bytes);
  plan_segment(sr, &gr, &bytes);
  plan_segment(sb, &gb, &bytes);
  if (pool->last_shape[0] == 0) {
    pool->last_shape[0] = (int)(ra[0].recs.size() + rb[0].recs.size());
    pool->last_shape[1] = (int)(ga.size() + gb.size());
    pool->last_shape[2] = (int)rr[0].recs.size();
    pool->last_shape[3] = (int)gr.size();
  }
  const size_t off_flags = bytes;
  bytes += sizeof(int*) * n + sizeof(int) * 64;
  const size_t off_passes = off_flags + sizeof(int*) * n;
  if (bytes > pool->dev_bytes) {
    if (pool->dev) cudaFree(pool->dev);
    pool->dev = nullptr;
    pool->dev_bytes = 0;
    KP_CUDA(cudaMalloc((void**)&pool->dev, bytes));
    pool->dev_bytes = bytes;
  }
  std::vector<unsigned char> host(bytes, 0);
  for (auto* gs : {&ga, &gr, &gb})
    for (const Group& g : *gs) g.recs[0]->table(g.recs.data(), (int)g.recs.size(), host.data() + g.off);
  for (int j = 0; j < n; ++j) {
    int* fp = pool->ctxs[act[j]]->dflags;
    std::memcpy(host.data() + off_flags + sizeof(int*) * j, &fp, sizeof(fp));
  }
  KP_CUDA(cudaMemcpy(pool->dev, host.data(), bytes, cudaMemcpyHostToDevice));
  int* const* dflags = reinterpret_cast<int* const*>(pool->dev + off_flags);
  int* passes = reinterpret_cast<int*>(pool->dev + off_passes);
  kp_ctx* dctx = pool->ctxs[act[0]];
  cudaStream_t s0 = dctx->stream;
  if (!dctx->aux_stream) KP_CUDA(cudaStreamCreateWithFlags(&dctx->aux_stream, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  KP_CUDA(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h_loop, h_rep;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h_loop, g, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams wp = {};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = h_loop;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wnode;
  if (e == cudaSuccess) e = cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &wp);
  cudaGraph_t body = e == cudaSuccess ? wp.conditional.phGraph_out[0] : nullptr;
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h_rep, body, 0, 0);
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(s0, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    kp_set_error("kp_solve_batch: loop graph: %s", cudaGetErrorString(e));
    return KP_ECUDA;
  }
  kp_status cs = launch_groups(dctx, ga, pool->dev);
  if (cs == KP_OK) {
    k_batch_any<<<1, 256, 0, s0>>>(dflags, n, F_NOTDUE, 1, nullptr, 0, h_rep);
    cudaStreamCaptureStatus cst;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* ed = nullptr;
    size_t nd = 0;
    cudaGraphNodeParams ip = {};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = h_rep;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t inode;
    e = cudaStreamGetCaptureInfo(s0, &cst, nullptr, &cg, &deps, &ed, &nd);
    if (e == cudaSuccess) e = cudaGraphAddNode(&inode, cg, deps, ed, nd, &ip);
    if (e == cudaSuccess)
      e = cudaStreamUpdateCaptureDependencies(s0, &inode, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess)
      e = cudaStreamBeginCaptureToGraph(dctx->aux_stream, ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      kp_set_error("kp_solve_batch: loop graph (replacement): %s", cudaGetErrorString(e));
      cs = KP_ECUDA;
    } else {
      dctx->stream = dctx->aux_stream;
      cs = launch_groups(dctx, gr, pool->dev);
      dctx->stream = s0;
      cudaGraph_t tmp = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(dctx->aux_stream, &tmp);
      if (cs == KP_OK && e2 != cudaSuccess) {
        kp_set_error("kp_solve_batch: loop graph (replacement): %s", cudaGetErrorString(e2));
        cs = KP_ECUDA;
      }
    }
  }
  if (cs == KP_OK) cs = launch_groups(dctx, gb, pool->dev);
  if (cs == KP_OK) k_batch_any<<<1, 256, 0, s0>>>(dflags, n, F_BLOOP, 0, passes, max_passes, h_loop);
  {
    cudaGraph_t tmp = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(s0, &tmp);
    if (cs == KP_OK && ee != cudaSuccess) {
      kp_set_error("kp_solve_batch: loop graph capture: %s", cudaGetErrorString(ee));
      cs = KP_ECUDA;
    }
  }
  if (cs == KP_OK && cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) {
    kp_set_error("kp_solve_batch: loop graph instantiation failed");
    cs = KP_ECUDA;
  }
  const clk::time_point t1 = clk::now();
  if (cs == KP_OK) {
    int hp = 0;
    cudaError_t le = cudaMemsetAsync(passes, 0, sizeof(int), s0);
    if (le == cudaSuccess) le = cudaGraphLaunch(ge, s0);
    if (le == cudaSuccess) le = cudaMemcpyAsync(&hp, passes, sizeof(int), cudaMemcpyDeviceToHost, s0);
    if (le == cudaSuccess) le = cudaStreamSynchronize(s0);
    if (le != cudaSuccess) {
      kp_set_error("kp_solve_batch: grouped loop: %s", cudaGetErrorString(le));
      cs = KP_ECUDA;
    }
    *done = hp;
  }
  if (ge) cudaGraphExecDestroy(ge);
  cudaGraphDestroy(g);
  pool->last_ms[1] += std::chrono::duration<double, std::milli>(t1 - t0).count();
  pool->last_ms[2] += std::chrono::duration<double, std::milli>(clk::now() - t1).count();
  return cs;
}

static kp_status solve_grouped(int device, kp_problem* probs, int nprob, const kp_batch_opts* o) {
  GroupPool* pool = group_pool(device);
  std::lock_guard<std::mutex> lock(pool->mu);
  pool->last_grouped = 0;
  pool->last_passes = 0;
  for (double& v : pool->last_ms) v = 0.0;
  for (int& v : pool->last_shape) v = 0;
  KP_CUDA(cudaSetDevice(device));
  using clk = std::chrono::steady_clock;
  auto ms_since = [](clk::time_point t) { return std::chrono::duration<double, std::milli>(clk::now() - t).count(); };
  const clk::time_point t_begin = clk::now();
  clk::time_point t_mark = t_begin;
  const bool bf16 = o->op_prec == KP_BF16;
  const double auto_cond = 1e4;  // ill-conditioned problems of a BF16 batch: BF16X3 inner operator
  while ((int)pool->ctxs.size() < nprob) {
    kp_ctx* c = nullptr;
    KP_TRY(kp_create(&c, device, nullptr));
    pool->ctxs.push_back(c);
  }
  std::vector<BatchRun*> runs(nprob, nullptr);
  std::vector<kp_status> st(nprob, KP_OK);
  std::vector<std::string> msg(nprob);
  std::vector<char> entered(nprob, 0);
  auto fail = [&](int i, kp_status s) {
    st[i] = s;
    msg[i] = kp_last_error();
    probs[i].info.status = s;
  };
  // setup, lambda and the steps before the iterations of every problem, each
  // problem in a fiber of its own on this thread: where its host code waits
  // for the GPU (a convergence test read back, a scalar), it yields, and the
  // other problems' work is queued meanwhile, so the GPU runs many setups at
  // once (largest problems first)
  auto phase1 = [&](int i) {
    kp_problem& p = probs[i];
    kp_ctx* ctx = pool->ctxs[i];
    kp_status s = kp_set_option(ctx, "op_auto_cond", bf16 ? auto_cond : 0.0);
    ctx->tc_group = true;  // grouped GEMMs: one-CTA tiles, no K split
    ctx->tc_group_uniform = o->autotune == 0;
    if (s == KP_OK) s = kp_set_option(ctx, "tc_autotune", o->autotune == 1 ? 1 : 0);
    entered[i] = 0;
    if (s == KP_OK)
      s = kp_setup(ctx, p.psf, p.n_r, p.n_c, p.center_r, p.center_c, p.bc, p.op_rank, 1, o->op_prec, o->pc_prec,
                   o->vec_prec, o->sigma);
    double lam = p.lambda;
    if (s == KP_OK && !(lam > 0.0)) s = choose_lambda(ctx, p.b, o->method, p.lambda_param, nullptr, &lam);
    if (s == KP_OK) {
      p.lambda = lam;
      if (!p.b || !p.x || ((uintptr_t)p.b & 15) || ((uintptr_t)p.x & 15)) {
        kp_set_error("kp_solve_batch: problem %d: b and x must be 16-byte aligned device pointers", i);
        s = KP_EINVAL;
      }
    }
    if (s == KP_OK && !(o->tol >= 0.0 && o->maxit >= 1)) {
      kp_set_error("kp_solve_batch: need tol >= 0 and maxit >= 1");
      s = KP_EINVAL;
    }
    if (s == KP_OK) {
      s = kp_enter(ctx);
      entered[i] = 1;
    }
    if (s == KP_OK) s = batch_begin(ctx, p.b, lam, o->tol, o->maxit, o->flexible, p.x, &runs[i]);
    if (s != KP_OK) fail(i, s);
  };
  {
    std::vector<int> order(nprob);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      return (long long)probs[a].n_r * probs[a].n_c > (long long)probs[b].n_r * probs[b].n_c;
    });
    std::vector<std::function<void()>> work;
    for (int i : order) work.push_back([&, i]() { phase1(i); });
    std::vector<kp_ctx*> cs;
    for (int i : order) cs.push_back(pool->ctxs[i]);
    g_yields = 0;
    const kp_status fs = run_fibers(work, cs);
    if (fs != KP_OK) {  // no fibers: the same work, one problem after another
      for (int i : order) phase1(i);
    }
    pool->last_shape[4] = fs == KP_OK ? 1 : 0;
    pool->last_shape[5] = (int)std::min<long long>(g_yields, 2000000000LL);
  }
  pool->last_ms[0] = ms_since(t_begin);
  t_mark = clk::now();
  // record one iteration of every problem whose loop can run grouped
  std::vector<int> grp;
  std::string record_msg;
  std::vector<KpRecorder> ra(nprob), rr(nprob), rb(nprob);
  for (int i = 0; i < nprob; ++i) {
    if (!runs[i] || !batch_groupable(runs[i])) continue;
    const kp_status s = batch_record(pool->ctxs[i], runs[i], &ra[i], &rr[i], &rb[i]);
    if (s == KP_OK) {
      grp.push_back(i);
    } else {
      cudaGetLastError();
      if (record_msg.empty()) record_msg = kp_last_error();
    }
  }
  // the grouped problems' iterations must line up launch by launch; the
  // largest set of equal lengths runs grouped, the rest alone
  {
    std::map<std::vector<size_t>, std::vector<int>> by_len;
    for (int i : grp) by_len[{ra[i].recs.size(), rr[i].recs.size(), rb[i].recs.size()}].push_back(i);
    std::vector<int> best;
    for (auto& kv : by_len)
      if (kv.second.size() > best.size()) best = kv.second;
    grp = best;
  }
  std::vector<char> in_grp(nprob, 0);
  for (int i : grp) in_grp[i] = 1;
  kp_status gst = KP_OK;
  pool->last_ms[1] = ms_since(t_mark);
  if (!grp.empty()) {
    // Epochs of 16, 32, 64, ... passes; after each, the graph is rebuilt for
    // the problems still running, so that the long tail of a few slow
    // problems does not pay for the launches of the ones that stopped.
    for (int i : grp)
      if (gst == KP_OK) gst = batch_arm(pool->ctxs[i], runs[i]);
    std::vector<int> act = grp;
    int total = 0, epoch = 16;
    while (gst == KP_OK && !act.empty()) {
      const int left = o->maxit + 16 - total;
      if (left <= 0) break;
      int done = 0;
      gst = run_epoch(pool, act, runs, std::min(epoch, left), &done);
      total += done;
      epoch *= 2;
      if (gst != KP_OK) break;
      std::vector<int> still;
      std::vector<int> go(act.size(), 0);
      cudaStream_t s0 = pool->ctxs[act[0]]->stream;
      for (size_t j = 0; j < act.size(); ++j)
        KP_CUDA(cudaMemcpyAsync(&go[j], pool->ctxs[act[j]]->dflags + F_BLOOP, sizeof(int), cudaMemcpyDeviceToHost,
                                s0));
      KP_CUDA(cudaStreamSynchronize(s0));
      for (size_t j = 0; j < act.size(); ++j)
        if (go[j]) still.push_back(act[j]);
      act.swap(still);
    }
    pool->last_passes = total;
    if (gst == KP_OK) pool->last_grouped = (int)grp.size();
  }
  // results; problems outside the grouped loop run it alone; a BF16 inner
  // operator that stalled or broke down is retried with BF16X3 (as alone)
  for (int i = 0; i < nprob; ++i) {
    if (!runs[i]) continue;
    kp_problem& p = probs[i];
    kp_ctx* ctx = pool->ctxs[i];
    kp_status s;
    if (in_grp[i] && gst == KP_OK) {
      s = batch_finish(ctx, runs[i], &p.info);
    } else if (!batch_needs_loop(runs[i])) {
      s = batch_finish(ctx, runs[i], &p.info);
    } else {
      batch_discard(runs[i]);
      s = tik_pcg(ctx, p.b, p.lambda, o->tol, o->maxit, o->flexible, p.x, 0, &p.info);
    }
    runs[i] = nullptr;
    if (bf16 && ctx->op_prec == KP_BF16 && (s == KP_ENOCONV || s == KP_EBREAKDOWN || s == KP_ENUMERIC)) {
      kp_status so = kp_set_option(ctx, "op_auto_cond", 1.0);
      if (so == KP_OK) s = tik_pcg(ctx, p.b, p.lambda, o->tol, o->maxit, o->flexible, p.x, 0, &p.info);
      kp_set_option(ctx, "op_auto_cond", auto_cond);
    }
    p.info.status = s;
    if (s != KP_OK) fail(i, s);
  }
  for (int i = 0; i < nprob; ++i)
    if (entered[i]) kp_leave(pool->ctxs[i]);
  if (gst != KP_OK) {
    kp_set_error("kp_solve_batch: grouped loop: %s", kp_last_error());
    return gst;
  }
  for (int i = 0; i < nprob; ++i)
    if (st[i] != KP_OK) {
      kp_set_error("kp_solve_batch: problem %d: %s", i, msg[i].c_str());
      return st[i];
    }
  // (a problem that could not be recorded ran alone; say why, without failing)
  if (!record_msg.empty()) kp_set_error("kp_solve_batch: ran alone: %s", record_msg.c_str());
  return KP_OK;
}
