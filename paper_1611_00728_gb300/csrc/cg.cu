// Solver drivers: single-mass CG (FP64, or mixed FP32/FP64 with reliable
// updates) and multi-mass (multi-shift) CG (paper Sec. 3-4: the single- and
// multi-mass staggered CG; the multi-mass form is the benchmarked routine).
//
// All Krylov scalars stay in device memory (SolverState). The whole loop is
// one CUDA graph launch: a WHILE conditional node runs the iteration body
// until the device-side state says done (or a hard iteration bound is hit);
// the FP64 reliable update is an IF node inside the body. The host reads the
// state once, after the loop.
#include <chrono>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "sqcg_internal.cuh"

namespace {

constexpr int kCGKernelsPerIter = 7;  // enqueue_cg_head (3 + 2 finishers) + xpay + loop control
constexpr int kCGKernelsPerUpdate = 3;  // enqueue_cg_reliable (2 + finisher)
constexpr int kMSKernelsPerIter = 7;  // enqueue_ms_iteration (4 + 2 finishers) + loop control
constexpr int kSRKernelsPerIter = 4;  // enqueue_sr_head (2 + finisher) + the update
// Steps of the single-reduction loop per pass of its WHILE node. Each pass ends with the reliable-update
// IF node and the loop control; a step that asks for a reliable update closes the pass (the steps
// after it are skipped by their gate), and the IF node completes it. On the GB300 an IF node costs
// about 3.4 us and a WHILE pass 3.5 us (a CUDA-graph probe of empty bodies), against ~200 us a step
// at 32^4; the 32^4 mixed solve took 44.6, 43.5, 43.0 and 42.9 ms with 1, 2, 4 and 8 steps a pass.
constexpr int kSRUnroll = 8;
// the persistent loop runs where a parity has at most this many 128-site tiles a SM (measured
// crossover on the GB300: 20^4, 4.1 tiles a SM, gains; 24^4, 8.5, loses)
constexpr int kPersistentMaxTilesPerSM = 5;
constexpr int kSRKernelsPerUpdatePersistent = 4;  // flush, Dslash pair, finisher (no head)
constexpr int kSRKernelsPerUpdate = 7;  // enqueue_sr_reliable: flush, 2 FP64 + finisher, 2 FP32 + finisher

// KIND_CG: Hestenes-Stiefel CG (FP64 mode); KIND_MS: multi-shift; KIND_SR: single-reduction mixed CG
enum { KIND_CG = 0, KIND_MS = 1, KIND_SR = 2 };

}  // namespace

struct CGGraph {
  int kind, mixed, nshift;
  const void* b;
  void* x[SQCG_MAX_SHIFTS];
  cudaGraphExec_t exec;
  cudaGraphConditionalHandle h_while, h_if;
  CGGraph* next;
};

void free_graphs(sqcg_ctx* ctx) {
  CGGraph* g = ctx->graphs;
  while (g) {
    CGGraph* n = g->next;
    cudaGraphExecDestroy(g->exec);
    free(g);
    g = n;
  }
  ctx->graphs = nullptr;
}

namespace {

CGGraph* find_graph(sqcg_ctx* ctx, int kind, int mixed, const void* b, void* const* x, int nx) {
  for (CGGraph* g = ctx->graphs; g; g = g->next) {
    if (g->kind != kind || g->mixed != mixed || g->b != b || g->nshift != nx) continue;
    bool same = true;
    for (int j = 0; j < nx; ++j) same = same && g->x[j] == x[j];
    if (same) return g;
  }
  return nullptr;
}

void add_graph(sqcg_ctx* ctx, CGGraph* g) {
  // keep at most 8 cached graphs: drop the oldest
  int n = 0;
  CGGraph** pp = &ctx->graphs;
  while (*pp) {
    if (++n >= 8) {
      CGGraph* victim = *pp;
      *pp = victim->next;
      cudaGraphExecDestroy(victim->exec);
      free(victim);
      continue;
    }
    pp = &(*pp)->next;
  }
  g->next = ctx->graphs;
  ctx->graphs = g;
}

// Kernels of one single-mass CG iteration, before the reliable-update node:
// tmp = D_oe p; Ap = sigma p - D_eo tmp with alpha = |r|^2/<p,Ap>;
// x += alpha p, r -= alpha Ap with beta and the reliable-update decision.
int enqueue_cg_head(sqcg_ctx* ctx, int mixed, void* x, cudaStream_t s) {
  const int wp = mixed ? SQCG_F32 : SQCG_F64;
  void* p = mixed ? (void*)ctx->p32 : (void*)ctx->p64;
  void* Ap = mixed ? (void*)ctx->Ap32 : (void*)ctx->Ap64;
  void* tmp = mixed ? (void*)ctx->tmp32 : (void*)ctx->tmp64;
  DslashLaunch L = {};
  L.out_parity = 1; L.prec = L.out_prec = wp; L.epi = EPI_PLAIN; L.in = p; L.out = tmp; L.gate = GATE_ITER;
  SQCG_TRY(launch_dslash(ctx, L, s));
  L = DslashLaunch{};
  L.out_parity = 0; L.prec = L.out_prec = wp; L.epi = EPI_NORMAL_DOT; L.in = tmp; L.out = Ap; L.y = p;
  L.sigma_dev = &ctx->st->sigma; L.gate = GATE_ITER; L.fin = FIN_PAP; L.pdl = 1;
  SQCG_TRY(launch_dslash(ctx, L, s));
  SQCG_TRY(launch_cg_update_x(ctx, mixed, (double2*)x, s));
  return SQCG_OK;
}

// Body of the reliable-update IF node: r = b - A x in FP64 (written to the
// working r), which also confirms convergence on the true residual.
int enqueue_cg_reliable(sqcg_ctx* ctx, int mixed, const void* b, void* x, cudaStream_t s) {
  void* r = mixed ? (void*)ctx->r32 : (void*)ctx->r64;
  DslashLaunch L = {};
  L.out_parity = 1; L.prec = L.out_prec = SQCG_F64; L.epi = EPI_PLAIN; L.in = x; L.out = ctx->tmp64;
  L.gate = GATE_UPDATE;
  SQCG_TRY(launch_dslash(ctx, L, s));
  L = DslashLaunch{};
  L.out_parity = 0; L.prec = SQCG_F64; L.out_prec = mixed ? SQCG_F32 : SQCG_F64; L.epi = EPI_TRUE_RESID;
  L.in = ctx->tmp64; L.out = r; L.y = x; L.b = b; L.sigma_dev = &ctx->st->sigma; L.gate = GATE_UPDATE;
  L.fin = FIN_TRUE_RESID;
  SQCG_TRY(launch_dslash(ctx, L, s));
  return SQCG_OK;
}

// Single-reduction mixed CG, head of one iteration: tmp = D_oe r; s = sigma r - D_eo tmp (into Ap32)
// with <r, s> and |r|^2 from its epilogue and <r, q> from the previous update kernel (or, right after a
// reliable update replaced r, from this epilogue: after_update); the finisher decides on convergence
// and the reliable update and, without one, computes alpha and beta.
int enqueue_sr_head(sqcg_ctx* ctx, cudaStream_t s, bool after_update = false, bool after_kernel = false) {
  DslashLaunch L = {};
  L.out_parity = 1; L.prec = L.out_prec = SQCG_F32; L.epi = EPI_PLAIN; L.in = ctx->r32; L.out = ctx->tmp32;
  L.gate = GATE_STEP; L.pdl = after_kernel;
  SQCG_TRY(launch_dslash(ctx, L, s));
  L = DslashLaunch{};
  L.out_parity = 0; L.prec = L.out_prec = SQCG_F32; L.epi = after_update ? EPI_SR_DOTS : EPI_SR_DOTS2;
  L.in = ctx->tmp32; L.out = ctx->Ap32;
  L.y = ctx->r32; L.y3 = ctx->q32; L.sigma_dev = &ctx->st->sigma; L.gate = GATE_STEP;
  L.fin = FIN_SR_STEP; L.pdl = 1;
  return launch_dslash(ctx, L, s);
}

// Single-reduction mixed CG, reliable update (IF-node body): x += xh, then r = b - A x (also the
// convergence check), then A r and the step's scalars again from the true residual. The true residual's
// Dslash pair runs in float-float (default) or FP64 arithmetic (sqcg_set_update_arithmetic); the sum
// b - sigma x + D x and its norm are FP64 either way.
int enqueue_sr_reliable(sqcg_ctx* ctx, const void* b, void* x, cudaStream_t s, bool head = true) {
  if (ctx->ru_arith == SQCG_FF) {
    SQCG_TRY(launch_flush_split(ctx, (double2*)x, ctx->xh32, ctx->xff, GATE_UPDATE, s));
    FFLaunch F = {};
    F.out_parity = 1; F.in = ctx->xff; F.out_ff = ctx->tmp64; F.gate = GATE_UPDATE;  // tmp64 holds float4 [3][Vh]
    SQCG_TRY(launch_dslash_ff(ctx, F, s));
    F = FFLaunch{};
    F.out_parity = 0; F.true_resid = 1; F.in = ctx->tmp64; F.out32 = ctx->r32; F.x = x; F.b = b;
    F.sigma_dev = &ctx->st->sigma; F.gate = GATE_UPDATE; F.fin = FIN_TRUE_RESID;
    SQCG_TRY(launch_dslash_ff(ctx, F, s));
    return head ? enqueue_sr_head(ctx, s, true, true) : SQCG_OK;
  }
  SQCG_TRY(launch_flush_partial_x(ctx, (double2*)x, GATE_UPDATE, s));
  DslashLaunch L = {};
  L.out_parity = 1; L.prec = L.out_prec = SQCG_F64; L.epi = EPI_PLAIN; L.in = x; L.out = ctx->tmp64;
  L.gate = GATE_UPDATE;
  SQCG_TRY(launch_dslash(ctx, L, s));
  L = DslashLaunch{};
  L.out_parity = 0; L.prec = SQCG_F64; L.out_prec = SQCG_F32; L.epi = EPI_TRUE_RESID;
  L.in = ctx->tmp64; L.out = ctx->r32; L.y = x; L.b = b; L.sigma_dev = &ctx->st->sigma; L.gate = GATE_UPDATE;
  L.fin = FIN_TRUE_RESID;
  SQCG_TRY(launch_dslash(ctx, L, s));
  return head ? enqueue_sr_head(ctx, s, true, true) : SQCG_OK;  // gated on the loop going on (GATE_STEP)
}

int enqueue_ms_iteration(sqcg_ctx* ctx, int mixed, int nshift, double2* const* x, cudaStream_t s) {
  const int wp = mixed ? SQCG_F32 : SQCG_F64;
  void* p = mixed ? (void*)ctx->p32 : (void*)ctx->p64;
  void* Ap = mixed ? (void*)ctx->Ap32 : (void*)ctx->Ap64;
  void* tmp = mixed ? (void*)ctx->tmp32 : (void*)ctx->tmp64;
  DslashLaunch L = {};
  L.out_parity = 1; L.prec = L.out_prec = wp; L.epi = EPI_PLAIN; L.in = p; L.out = tmp; L.gate = GATE_ITER;
  SQCG_TRY(launch_dslash(ctx, L, s));
  L = DslashLaunch{};
  L.out_parity = 0; L.prec = L.out_prec = wp; L.epi = EPI_NORMAL_DOT; L.in = tmp; L.out = Ap; L.y = p;
  L.sigma_dev = &ctx->st->sigma; L.gate = GATE_ITER; L.fin = FIN_MS_PAP; L.pdl = 1;
  SQCG_TRY(launch_dslash(ctx, L, s));
  SQCG_TRY(launch_ms_update_x(ctx, mixed, nshift, x, s));
  SQCG_TRY(launch_ms_xpay(ctx, mixed, nshift, x, s));
  return SQCG_OK;
}

// Build the solver graph: one WHILE node whose body is one iteration (kSRUnroll
// steps for the single-reduction loop) followed by the loop-control kernel. For
// single-mass CG the reliable update sits in an IF node inside the body, so
// iterations without an update launch none of its kernels. The conditional
// handles are passed to the kernels through the device state (h_while, h_if).
int capture_body(sqcg_ctx* ctx, int kind, int mixed, const void* b, void* const* x, int nx, cudaGraph_t body,
                 cudaGraphConditionalHandle* hif, cudaGraph_t* ifbody) {
  cudaStream_t cs = ctx->cap_stream;
  SQCG_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  int rc = SQCG_OK;
  if (kind == KIND_SR) {  // kSRUnroll steps, each skipped once a reliable update is pending
    for (int k = 0; k < kSRUnroll && rc == SQCG_OK; ++k) {
      rc = enqueue_sr_head(ctx, cs, false, k > 0);
      if (rc == SQCG_OK) rc = launch_sr_update(ctx, cs, true);
    }
  }
  if (kind == KIND_CG || kind == KIND_SR) {
    if (kind == KIND_CG) rc = enqueue_cg_head(ctx, mixed, x[0], cs);
    if (rc == SQCG_OK) {
      cudaStreamCaptureStatus status;
      cudaGraph_t capg = nullptr;
      const cudaGraphNode_t* deps = nullptr;
      size_t ndeps = 0;
      cudaGraphNode_t inode = nullptr;
      cudaGraphNodeParams ip = {};
      if (cudaStreamGetCaptureInfo(cs, &status, nullptr, &capg, &deps, nullptr, &ndeps) != cudaSuccess ||
          cudaGraphConditionalHandleCreate(hif, capg, 0, 0) != cudaSuccess) {
        rc = SQCG_ERR_CUDA;
      } else {
        ip.type = cudaGraphNodeTypeConditional;
        ip.conditional.handle = *hif;
        ip.conditional.type = cudaGraphCondTypeIf;
        ip.conditional.size = 1;
        if (cudaGraphAddNode(&inode, capg, deps, nullptr, ndeps, &ip) != cudaSuccess ||
            cudaStreamUpdateCaptureDependencies(cs, &inode, nullptr, 1, cudaStreamSetCaptureDependencies) !=
                cudaSuccess)
          rc = SQCG_ERR_CUDA;
        else
          *ifbody = ip.conditional.phGraph_out[0];
      }
    }
    if (rc == SQCG_OK && kind == KIND_CG) rc = launch_cg_xpay(ctx, mixed, cs);
  } else {
    rc = enqueue_ms_iteration(ctx, mixed, nx, (double2* const*)x, cs);
  }
  if (rc == SQCG_OK) rc = launch_loop_control(ctx, cs);
  cudaGraph_t out = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &out);
  if (rc == SQCG_ERR_CUDA) sqcg_set_last_cuda_error(cudaGetLastError(), "conditional node", __FILE__, __LINE__);
  if (rc != SQCG_OK) return rc;
  if (e != cudaSuccess) { sqcg_set_last_cuda_error(e, "cudaStreamEndCapture", __FILE__, __LINE__); return SQCG_ERR_CUDA; }
  if (kind == KIND_CG || kind == KIND_SR) {
    SQCG_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, *ifbody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    if (kind == KIND_CG) {
      rc = enqueue_cg_reliable(ctx, mixed, b, x[0], cs);
    } else {  // the update, the step's head again from the true residual, and the step's vector update
      rc = enqueue_sr_reliable(ctx, b, x[0], cs);
      if (rc == SQCG_OK) rc = launch_sr_update(ctx, cs, true);
    }
    e = cudaStreamEndCapture(cs, &out);
    if (rc != SQCG_OK) return rc;
    if (e != cudaSuccess) { sqcg_set_last_cuda_error(e, "cudaStreamEndCapture", __FILE__, __LINE__); return SQCG_ERR_CUDA; }
  }
  return SQCG_OK;
}

int capture_new(sqcg_ctx* ctx, int kind, int mixed, const void* b, void* const* x, int nx, CGGraph** out) {
  cudaGraph_t top = nullptr;
  SQCG_CUDA_TRY(cudaGraphCreate(&top, 0));
  cudaGraphConditionalHandle hw = 0, hif = 0;
  cudaGraph_t ifbody = nullptr;
  int rc = SQCG_OK;
  cudaGraphNodeParams wp = {};
  cudaGraphNode_t wnode = nullptr;
  if (cudaGraphConditionalHandleCreate(&hw, top, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
    rc = SQCG_ERR_CUDA;
  } else {
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = hw;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    if (cudaGraphAddNode(&wnode, top, nullptr, nullptr, 0, &wp) != cudaSuccess) rc = SQCG_ERR_CUDA;
  }
  if (rc == SQCG_ERR_CUDA) sqcg_set_last_cuda_error(cudaGetLastError(), "WHILE node", __FILE__, __LINE__);
  if (rc == SQCG_OK) rc = capture_body(ctx, kind, mixed, b, x, nx, wp.conditional.phGraph_out[0], &hif, &ifbody);
  cudaGraphExec_t exec = nullptr;
  if (rc == SQCG_OK) {
    cudaError_t e = cudaGraphInstantiate(&exec, top, 0);
    if (e != cudaSuccess) { sqcg_set_last_cuda_error(e, "cudaGraphInstantiate", __FILE__, __LINE__); rc = SQCG_ERR_CUDA; }
  }
  cudaGraphDestroy(top);
  if (rc != SQCG_OK) return rc;
  CGGraph* g = (CGGraph*)calloc(1, sizeof(CGGraph));
  if (!g) { cudaGraphExecDestroy(exec); return SQCG_ERR_NO_MEMORY; }
  g->kind = kind; g->mixed = mixed; g->nshift = nx; g->b = b; g->exec = exec;
  g->h_while = hw; g->h_if = hif;
  for (int j = 0; j < nx; ++j) g->x[j] = x[j];
  add_graph(ctx, g);
  *out = g;
  return SQCG_OK;
}

// The cached graph of this loop, or a new capture. Programmatic edges inside a conditional node's body
// need a recent driver: if the capture with them fails, the context drops programmatic dependent launch
// and captures again with plain edges (same kernels, same results).
int capture(sqcg_ctx* ctx, int kind, int mixed, const void* b, void* const* x, int nx, CGGraph** out) {
  CGGraph* g = find_graph(ctx, kind, mixed, b, x, nx);
  if (g) { *out = g; return SQCG_OK; }
  int rc = capture_new(ctx, kind, mixed, b, x, nx, out);
  if (rc == SQCG_ERR_CUDA && ctx->pdl) {
    cudaGetLastError();
    ctx->pdl = 0;
    rc = capture_new(ctx, kind, mixed, b, x, nx, out);
  }
  return rc;
}

int read_state(sqcg_ctx* ctx, cudaStream_t s) {
  SQCG_CUDA_TRY(cudaMemcpyAsync(ctx->st_host, ctx->st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
  SQCG_CUDA_TRY(cudaStreamSynchronize(s));
  return SQCG_OK;
}

int write_state(sqcg_ctx* ctx, cudaStream_t s) {
  SQCG_CUDA_TRY(cudaMemcpyAsync(ctx->st, ctx->st_host, sizeof(SolverState), cudaMemcpyHostToDevice, s));
  return SQCG_OK;
}

// Run the whole device-side loop with one graph launch, then read the state.
// *iters_run = WHILE-loop iterations executed (for the launch count).
int run_loop(sqcg_ctx* ctx, CGGraph* g, int max_iter, cudaStream_t s, int* iters_run) {
  SolverState* h = ctx->st_host;
  h->h_while = g->h_while;
  h->h_if = g->h_if;
  h->use_if = (g->kind == KIND_CG || g->kind == KIND_SR) ? 1 : 0;
  h->loop_count = 0;
  h->loop_limit = max_iter + 4;
  SQCG_TRY(write_state(ctx, s));
  SQCG_CUDA_TRY(cudaGraphLaunch(g->exec, s));
  SQCG_TRY(read_state(ctx, s));
  *iters_run = h->loop_count;
  return SQCG_OK;
}

// The same iterations launched one kernel at a time, with the host reading
// the device state after each step (SQCG_LAUNCH_MODE=eager). Kernel-level
// profilers do not see kernels inside conditional graph nodes; this mode
// gives them the identical kernel sequence to list. Results are the same.
bool eager_mode() {
  const char* m = getenv("SQCG_LAUNCH_MODE");
  return m && strcmp(m, "eager") == 0;
}

int run_eager(sqcg_ctx* ctx, int kind, int mixed, const void* b, void* const* x, int nx, int max_iter,
              cudaStream_t s, int* iters_run) {
  SolverState* h = ctx->st_host;
  h->use_if = 0;  // no graph: the kernels must not touch conditional handles
  SQCG_TRY(write_state(ctx, s));
  int it = 0;
  for (; it < max_iter + 4; ++it) {
    if (kind == KIND_CG) {
      SQCG_TRY(enqueue_cg_head(ctx, mixed, x[0], s));
      SQCG_TRY(read_state(ctx, s));
      if (!h->done && h->need_update) {
        SQCG_TRY(enqueue_cg_reliable(ctx, mixed, b, x[0], s));
        SQCG_TRY(read_state(ctx, s));
      }
      if (h->done) break;
      SQCG_TRY(launch_cg_xpay(ctx, mixed, s));
    } else if (kind == KIND_SR) {
      SQCG_TRY(enqueue_sr_head(ctx, s));
      SQCG_TRY(read_state(ctx, s));
      if (!h->done && h->need_update) {
        SQCG_TRY(enqueue_sr_reliable(ctx, b, x[0], s));
        SQCG_TRY(read_state(ctx, s));
      }
      if (h->done) break;
      SQCG_TRY(launch_sr_update(ctx, s));
    } else {
      SQCG_TRY(enqueue_ms_iteration(ctx, mixed, nx, (double2* const*)x, s));
      SQCG_TRY(read_state(ctx, s));
      if (h->done || (h->ms_ru && h->need_update)) break;  // finished, or paused for the host-driven update
    }
  }
  *iters_run = it + 1;
  return SQCG_OK;
}

// The single-reduction mixed loop as the persistent kernel (cg_persistent.cu): one launch runs the
// iterations up to the next reliable update; the host reads the state, runs the true-residual pass
// and launches again. *segments = persistent launches, *updates_run = true-residual passes.
//
// Which loop runs: the persistent kernel where every 128-site tile of a parity has its own resident
// block (each phase is one wave, so a grid barrier replaces a kernel boundary at no cost in balance,
// and the launch and finisher latency it removes dominates small lattices); the graph-launched
// loop on larger lattices, where a phase takes several waves and the barrier across all resident
// blocks costs more than the kernel boundaries it replaces. SQCG_PERSISTENT=0 or 1 forces one.
bool use_persistent(sqcg_ctx* ctx) {
  const char* m = getenv("SQCG_PERSISTENT");
  if (m && strcmp(m, "0") == 0) return false;
  const int G = persistent_grid(ctx);
  if (G <= 0) return false;
  if (m && strcmp(m, "1") == 0) return true;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const int ntiles = grid_for(ctx->g.Vh, 128);
  return G >= ntiles && ntiles <= kPersistentMaxTilesPerSM * nsm;  // one block a tile, few a SM
}

int run_persistent(sqcg_ctx* ctx, const void* b, void* x, int max_iter, cudaStream_t s, int* segments,
                   int* updates_run) {
  SolverState* h = ctx->st_host;
  h->use_if = 0;
  SQCG_TRY(write_state(ctx, s));
  *segments = 0;
  *updates_run = 0;
  for (int k = 0; k < max_iter + 4; ++k) {
    SQCG_TRY(launch_sr_persistent(ctx, max_iter + 2 - h->iter, s));
    *segments += 1;
    SQCG_TRY(read_state(ctx, s));
    if (h->done || !h->need_update) break;
    SQCG_TRY(enqueue_sr_reliable(ctx, b, x, s, false));
    *updates_run += 1;
  }
  return SQCG_OK;
}

int validate_vec(const void* p, int prec) {
  if (!p) return SQCG_ERR_INVALID_ARG;
  const uintptr_t a = (uintptr_t)p;
  return (a % (prec == SQCG_F64 ? 16 : 8)) ? SQCG_ERR_INVALID_ARG : SQCG_OK;
}

}  // namespace

// CG on (sigma - D_eo D_oe) x = b; x: initial guess in, solution out.
int cg_solve_sigma(sqcg_ctx* ctx, double sigma, const void* b, void* x, double tol, int max_iter, int mode,
                   sqcg_info* info) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!ctx) return SQCG_ERR_INVALID_ARG;
  if (!(tol > 0) || max_iter <= 0 || (mode != SQCG_MODE_F64 && mode != SQCG_MODE_MIXED) || !isfinite(sigma) ||
      b == x)
    return SQCG_ERR_INVALID_ARG;
  SQCG_TRY(validate_vec(b, SQCG_F64));
  SQCG_TRY(validate_vec(x, SQCG_F64));
  if (!ctx->have_links) return SQCG_ERR_NO_LINKS;
  SQCG_TRY(ensure_workspace(ctx));
  const int mixed = (mode == SQCG_MODE_MIXED);
  cudaStream_t s = ctx->stream;

  SolverState* h = ctx->st_host;
  memset(h, 0, sizeof(SolverState));
  h->sigma = sigma;
  h->stop_rr = tol * tol;  // times |b|^2 on the device
  h->delta2 = ctx->ru_delta * ctx->ru_delta;
  h->max_iter = max_iter;
  h->update_interval = mixed ? ctx->ru_interval : (1 << 30);
  h->mixed = mixed;
  h->sr = mixed;  // mixed mode runs the single-reduction loop; FP64 mode the Hestenes-Stiefel loop
  h->status = SQCG_OK;
  SQCG_TRY(write_state(ctx, s));
  SQCG_TRY(launch_norm2_f64(ctx, (const double2*)b, FIN_BB, s));
  // |x0|^2: for a zero initial guess (the usual start) the initial residual is exactly b,
  // and the two FP64 Dslash passes of b - A x0 are skipped
  SQCG_TRY(launch_norm2_f64(ctx, (const double2*)x, FIN_STORE, s));
  SQCG_TRY(read_state(ctx, s));
  void* r0 = mixed ? (void*)ctx->r32 : (void*)ctx->r64;
  void* p0 = mixed ? (void*)ctx->p32 : (void*)ctx->p64;
  int launches = 4;
  if (h->pAp == 0.0) {
    const int wp = mixed ? SQCG_F32 : SQCG_F64;
    SQCG_TRY(layout_convert(ctx, SQCG_F64, b, wp, r0, s));
    SQCG_TRY(layout_convert(ctx, SQCG_F64, b, wp, p0, s));
    // the initial-residual step of the device state, with |r|^2 = |b|^2
    const double v = h->bb;
    if (!isfinite(v)) {
      h->status = SQCG_ERR_BREAKDOWN;
      h->done = 1;
      h->need_update = 0;
    } else {
      h->rr = h->rr_true = h->rr_max = h->rr_prev = v;
      h->iter_last_update = 0;
      if (v <= h->stop_rr) h->done = 1;
    }
    SQCG_TRY(write_state(ctx, s));
    launches += 2;
  } else {
    // r = b - A x0 (FP64), p = r, both in the working precision
    DslashLaunch L = {};
    L.out_parity = 1; L.prec = L.out_prec = SQCG_F64; L.epi = EPI_PLAIN; L.in = x; L.out = ctx->tmp64;
    SQCG_TRY(launch_dslash(ctx, L, s));
    L = DslashLaunch{};
    L.out_parity = 0; L.prec = SQCG_F64; L.out_prec = mixed ? SQCG_F32 : SQCG_F64; L.epi = EPI_TRUE_RESID;
    L.in = ctx->tmp64; L.out = r0; L.out2 = p0;
    L.y = x; L.b = b; L.sigma = sigma; L.fin = FIN_INIT;
    SQCG_TRY(launch_dslash(ctx, L, s));
    SQCG_TRY(read_state(ctx, s));
    launches += 3;
  }

  int status = SQCG_OK;
  int loops = 0;
  if (h->bb == 0.0) {  // b = 0: the solution is x = 0
    SQCG_CUDA_TRY(cudaMemsetAsync(x, 0, (size_t)ctx->g.Vh * 3 * sizeof(double2), s));
    SQCG_CUDA_TRY(cudaStreamSynchronize(s));
    if (info) {
      info->iters = 0; info->reliable_updates = 0; info->status = SQCG_OK; info->true_rel_resid = 0.0;
      info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      info->launches = launches;
    }
    return SQCG_OK;
  }
  if (!h->done) {
    void* xs[1] = {x};
    const int kind = mixed ? KIND_SR : KIND_CG;
    if (mixed) {  // p, q, the FP32 partial solution and the first step's <r, q> partials start at zero
      const size_t wb = (size_t)ctx->g.Vh * 3 * sizeof(float2);
      SQCG_CUDA_TRY(cudaMemsetAsync(ctx->p32, 0, wb, s));
      SQCG_CUDA_TRY(cudaMemsetAsync(ctx->q32, 0, wb, s));
      SQCG_CUDA_TRY(cudaMemsetAsync(ctx->xh32, 0, wb, s));
      SQCG_CUDA_TRY(cudaMemsetAsync(ctx->partials + sr_update_partials(ctx), 0,
                                    (size_t)ctx->max_blocks * sizeof(double), s));
    }
    int segments = -1, pupdates = 0;
    if (mixed && !eager_mode() && use_persistent(ctx)) {
      SQCG_TRY(run_persistent(ctx, b, x, max_iter, s, &segments, &pupdates));
    } else if (eager_mode()) {
      SQCG_TRY(run_eager(ctx, kind, mixed, b, xs, 1, max_iter, s, &loops));
    } else {
      CGGraph* g = nullptr;
      SQCG_TRY(capture(ctx, kind, mixed, b, xs, 1, &g));
      SQCG_TRY(run_loop(ctx, g, max_iter, s, &loops));
    }
    if (mixed) {  // whatever the partial solution still holds (nothing after a converged update)
      SQCG_TRY(launch_flush_partial_x(ctx, (double2*)x, GATE_NONE, s));
      SQCG_CUDA_TRY(cudaStreamSynchronize(s));
      if (segments >= 0)  // persistent launches, true-residual passes, final flush
        launches += segments + pupdates * kSRKernelsPerUpdatePersistent + 1;
      else
        launches += eager_mode() ? loops * kSRKernelsPerIter + h->updates * kSRKernelsPerUpdate + 1
                                 : loops * (kSRUnroll * kSRKernelsPerIter + 1) +  // passes: steps, control
                                       h->updates * (kSRKernelsPerUpdate + 1) + 1;  // IF bodies; final flush
    } else {
      launches += loops * kCGKernelsPerIter + h->updates * kCGKernelsPerUpdate;
    }
    status = h->done ? h->status : SQCG_ERR_NOT_CONVERGED;
  } else {
    status = h->status;  // x0 already solves the system (or breakdown on a non-finite residual)
  }
  if (info) {
    info->iters = h->iter;
    info->reliable_updates = h->updates;
    info->status = status;
    info->true_rel_resid = sqrt(h->rr_true / h->bb);
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    info->launches = launches;
  }
  return status;
}

extern "C" int sqcg_cg_solve(sqcg_ctx* ctx, double mass, const void* b, void* x, double tol, int max_iter, int mode,
                             sqcg_info* info) {
  if (!isfinite(mass)) return SQCG_ERR_INVALID_ARG;
  return cg_solve_sigma(ctx, 4.0 * mass * mass, b, x, tol, max_iter, mode, info);
}

namespace {

// Shift-aware reliable update of the multi-shift loop (SQCG_MS_SHIFT_RU), run by the host while the
// loop is paused after a whole iteration (x_s, r and the directions all at step k + 1), in FP64:
// r_0 = b - A_0 x_0; for every shift still iterating r_s = b - A_s x_s, the least-squares factor
// zeta'_s = Re<r_0, r_s> / |r_0|^2 and the loss |r_s - zeta'_s r_0|. A shift whose loss is at most
// half its tolerance continues from zeta'_s: zeta_{k+1} and zeta_k both scale by zeta'_s / zeta_s
// (the zeta recurrence is homogeneous of degree one in the pair, so alpha_s and beta_s keep their
// values), and its stopping threshold drops by the loss, which later steps in the shared Krylov
// space do not remove. Then r_0 replaces the iterated base residual and every moving direction takes
// the change, p_s += zeta_s (r_0 - r). sig, tl: shifts and tolerances in the loop's order (base
// first); perm maps that order to the caller's. ru_count[j] counts the updates shift j continued from.
// shifts_too = 0 (the mixed mode's base updates) skips the shifts' residuals: only the base residual is replaced,
// in mixed mode computed with the float-float Dslash (as the single-mass reliable update) when that is
// the context's update arithmetic, and written as FP32 into the free A p vector.
int ms_shift_aware_update(sqcg_ctx* ctx, int mixed, int nshift, const double* sig, const double* tl,
                          const int* perm, const void* b, void* const* xs, cudaStream_t s, int* ru_count,
                          int* launches, bool shifts_too) {
  SolverState* h = ctx->st_host;
  const size_t n = (size_t)ctx->g.Vh * 3;
  if (!shifts_too && mixed && ctx->ru_arith == SQCG_FF) {
    SQCG_TRY(launch_split_ff((const double2*)xs[0], ctx->xff, n, s));
    FFLaunch F = {};
    F.out_parity = 1; F.in = ctx->xff; F.out_ff = ctx->tmp64;  // tmp64 holds float4 [3][Vh]
    SQCG_TRY(launch_dslash_ff(ctx, F, s));
    F = FFLaunch{};
    F.out_parity = 0; F.true_resid = 1; F.in = ctx->tmp64; F.out32 = ctx->Ap32; F.x = xs[0]; F.b = b;
    F.sigma = sig[0]; F.fin = FIN_STORE;  // |r_0|^2 (FP64 sum) into st->pAp, free while the loop pauses
    SQCG_TRY(launch_dslash_ff(ctx, F, s));
    *launches += 4;
    SQCG_TRY(read_state(ctx, s));
    const double r0n = h->pAp;
    const int u = ctx->ms_rec_n++;
    if (u < SQCG_MS_RU_RECORD) {
      ctx->ms_rec_iter[u] = h->iter;
      ctx->ms_rec_base[u] = sqrt(r0n / h->bb);
      for (int j = 0; j < nshift; ++j) ctx->ms_rec_loss[u][perm[j]] = (j == 0) ? 0.0 : NAN;
    }
    if (!isfinite(r0n)) {
      h->status = SQCG_ERR_BREAKDOWN;
      h->done = 1;
      h->need_update = 0;
      return write_state(ctx, s);
    }
    ru_count[0] += 1;
    h->rr = h->rr_true = h->rr_max = r0n;
    h->need_update = 0;
    h->updates += 1;
    SQCG_TRY(write_state(ctx, s));
    *launches += 1;
    return launch_ms_ru_fix(ctx, mixed, nshift, ctx->Ap32, SQCG_F32, s);
  }
  if (!ctx->ms_ru_vec && cudaMalloc(&ctx->ms_ru_vec, 2 * n * sizeof(double2)) != cudaSuccess) {
    cudaGetLastError();
    return SQCG_ERR_NO_MEMORY;
  }
  double2* r0 = ctx->ms_ru_vec;
  double2* rs = ctx->ms_ru_vec + n;
  auto true_resid = [&](const void* x, double sigma, double2* out) -> int {  // out = b - A_sigma x, FP64
    DslashLaunch L = {};
    L.out_parity = 1; L.prec = L.out_prec = SQCG_F64; L.epi = EPI_PLAIN; L.in = x; L.out = ctx->tmp64;
    SQCG_TRY(launch_dslash(ctx, L, s));
    L = DslashLaunch{};
    L.out_parity = 0; L.prec = L.out_prec = SQCG_F64; L.epi = EPI_TRUE_RESID; L.in = ctx->tmp64; L.out = out;
    L.y = x; L.b = b; L.sigma = sigma;
    *launches += 2;
    return launch_dslash(ctx, L, s);
  };
  SQCG_TRY(true_resid(xs[0], sig[0], r0));
  SQCG_TRY(launch_ms_ru_sums(ctx, r0, r0, 0.0, s));
  *launches += 2;
  SQCG_TRY(read_state(ctx, s));
  const double r0n = h->ms_sums[2], bb = h->bb;
  const int u = ctx->ms_rec_n++;
  if (u < SQCG_MS_RU_RECORD) {
    ctx->ms_rec_iter[u] = h->iter;
    ctx->ms_rec_base[u] = sqrt(r0n / bb);
    for (int j = 0; j < nshift; ++j) ctx->ms_rec_loss[u][perm[j]] = (j == 0) ? 0.0 : NAN;
  }
  if (!isfinite(r0n)) {
    h->status = SQCG_ERR_BREAKDOWN;
    h->done = 1;
    h->need_update = 0;
    return write_state(ctx, s);
  }
  double scale[SQCG_MAX_SHIFTS], l2s[SQCG_MAX_SHIFTS];
  int keep[SQCG_MAX_SHIFTS] = {};
  for (int j = 1; j < nshift && shifts_too; ++j) {
    if (h->active[j] != 1) continue;
    SQCG_TRY(true_resid(xs[j], sig[j], rs));
    SQCG_TRY(launch_ms_ru_sums(ctx, r0, rs, 0.0, s));
    SQCG_TRY(read_state(ctx, s));
    const double zp = r0n > 0.0 ? h->ms_sums[0] / r0n : 0.0;
    SQCG_TRY(launch_ms_ru_sums(ctx, r0, rs, zp, s));
    SQCG_TRY(read_state(ctx, s));
    *launches += 4;
    const double l2 = h->ms_sums[1], loss = sqrt(l2 / bb);
    if (u < SQCG_MS_RU_RECORD) ctx->ms_rec_loss[u][perm[j]] = loss;
    if (isfinite(loss) && loss <= 0.5 * tl[j] && zp != 0.0 && h->zeta[j] != 0.0) {
      keep[j] = 1;
      scale[j] = zp / h->zeta[j];
      l2s[j] = l2;
    }
  }
  // the state read last is the device's: apply the decisions to it
  for (int j = 1; j < nshift; ++j) {
    if (!keep[j]) continue;
    h->zeta[j] *= scale[j];
    h->zeta_prev[j] *= scale[j];
    h->stop_rr_s[j] = tl[j] * tl[j] * bb - l2s[j];
    ru_count[j] += 1;
  }
  ru_count[0] += 1;
  h->rr = h->rr_true = h->rr_max = r0n;
  h->need_update = 0;
  h->updates += 1;
  SQCG_TRY(write_state(ctx, s));
  *launches += 1;
  return launch_ms_ru_fix(ctx, mixed, nshift, r0, SQCG_F64, s);
}

}  // namespace

// Multi-shift CG: (sigma_s - D_eo D_oe) x_s = b for all shifts from one Krylov
// space built on the smallest shift; FP64 scalar recurrences. In mixed mode
// each shift whose FP64 true residual is above its tolerance is then refined
// by mixed-precision CG started from x_s.
extern "C" int sqcg_multishift_cg_solve(sqcg_ctx* ctx, int nshift, const double* shifts, const void* b,
                                        void* const* x, const double* tol, int max_iter, int mode,
                                        sqcg_info* info) {
  const auto t0 = std::chrono::steady_clock::now();
  const int ru_shifts = (mode & SQCG_MS_SHIFT_RU) != 0, no_ru = (mode & SQCG_MS_NO_RU) != 0;
  mode &= ~(SQCG_MS_SHIFT_RU | SQCG_MS_NO_RU);
  if (ru_shifts && no_ru) return SQCG_ERR_INVALID_ARG;
  // mixed: base reliable updates unless SQCG_MS_NO_RU; FP64: only with SQCG_MS_SHIFT_RU
  const int ru = ru_shifts || (mode == SQCG_MODE_MIXED && !no_ru);
  if (!ctx || nshift < 1 || nshift > SQCG_MAX_SHIFTS || !shifts || !x || !tol || max_iter <= 0 ||
      (mode != SQCG_MODE_F64 && mode != SQCG_MODE_MIXED))
    return SQCG_ERR_INVALID_ARG;
  SQCG_TRY(validate_vec(b, SQCG_F64));
  for (int j = 0; j < nshift; ++j) {
    if (!isfinite(shifts[j]) || shifts[j] < 0 || !(tol[j] > 0)) return SQCG_ERR_INVALID_ARG;
    SQCG_TRY(validate_vec(x[j], SQCG_F64));
    if (x[j] == b) return SQCG_ERR_INVALID_ARG;
    for (int k = 0; k < j; ++k)
      if (x[k] == x[j]) return SQCG_ERR_INVALID_ARG;
  }
  if (!ctx->have_links) return SQCG_ERR_NO_LINKS;
  SQCG_TRY(ensure_workspace(ctx));
  const int mixed = (mode == SQCG_MODE_MIXED);
  cudaStream_t s = ctx->stream;
  const size_t n = (size_t)ctx->g.Vh * 3;
  const size_t wbytes = n * (mixed ? sizeof(float2) : sizeof(double2));

  // order the shifts: the smallest is the base system (index 0)
  int perm[SQCG_MAX_SHIFTS];
  for (int j = 0; j < nshift; ++j) perm[j] = j;
  for (int j = 1; j < nshift; ++j)
    for (int k = j; k > 0 && shifts[perm[k]] < shifts[perm[k - 1]]; --k) {
      int t = perm[k]; perm[k] = perm[k - 1]; perm[k - 1] = t;
    }
  void* xs[SQCG_MAX_SHIFTS];
  for (int j = 0; j < nshift; ++j) xs[j] = x[perm[j]];

  // per-shift directions p_s (s >= 1) in the working precision; p_0 is the base p
  if (ctx->ms_nalloc < nshift || ctx->ms_prec != mixed) {
    for (int j = 1; j < ctx->ms_nalloc; ++j) cudaFree(ctx->ms_p[j]);
    ctx->ms_nalloc = 0;
    free_graphs(ctx);
    for (int j = 1; j < nshift; ++j) {
      if (cudaMalloc(&ctx->ms_p[j], wbytes) != cudaSuccess) {
        cudaGetLastError();
        for (int k = 1; k < j; ++k) cudaFree(ctx->ms_p[k]);
        return SQCG_ERR_NO_MEMORY;
      }
    }
    ctx->ms_nalloc = nshift;
    ctx->ms_prec = mixed;
  }
  ctx->ms_p[0] = mixed ? (void*)ctx->p32 : (void*)ctx->p64;

  SolverState* h = ctx->st_host;
  memset(h, 0, sizeof(SolverState));
  const double sigma0 = shifts[perm[0]];
  h->sigma = sigma0;
  h->stop_rr = 0.0;
  h->max_iter = max_iter;
  h->mixed = mixed;
  h->nshift = nshift;
  h->alpha_prev = 1.0;
  h->beta_prev = 0.0;
  h->ms_ru = ru;
  h->delta2 = ctx->ru_delta * ctx->ru_delta;
  ctx->ms_rec_n = 0;
  ctx->ms_rec_nshift = nshift;
  for (int j = 0; j < nshift; ++j) {
    h->active[j] = 1;
    h->dsig[j] = shifts[perm[j]] - sigma0;
    h->stop_rr_s[j] = tol[perm[j]] * tol[perm[j]];
    h->zeta[j] = h->zeta_prev[j] = 1.0;
  }
  SQCG_TRY(write_state(ctx, s));
  for (int j = 0; j < nshift; ++j) SQCG_CUDA_TRY(cudaMemsetAsync(xs[j], 0, n * sizeof(double2), s));
  SQCG_TRY(launch_norm2_f64(ctx, (const double2*)b, FIN_BB, s));
  // r = p = p_s = b (x_s = 0)
  const int wp = mixed ? SQCG_F32 : SQCG_F64;
  void* r = mixed ? (void*)ctx->r32 : (void*)ctx->r64;
  SQCG_TRY(layout_convert(ctx, SQCG_F64, b, wp, r, s));
  for (int j = 0; j < nshift; ++j) SQCG_TRY(layout_convert(ctx, SQCG_F64, b, wp, ctx->ms_p[j], s));
  SQCG_TRY(read_state(ctx, s));
  if (h->bb == 0.0) {
    SQCG_CUDA_TRY(cudaStreamSynchronize(s));
    for (int j = 0; j < nshift; ++j)
      if (info) info[j] = sqcg_info{0, 0, SQCG_OK, 0.0, 0.0, 3 + nshift};
    return SQCG_OK;
  }
  h->rr = h->rr_prev = h->rr_max = h->bb;
  SQCG_TRY(write_state(ctx, s));

  // the shared loop; it pauses for each reliable update (base, or shift-aware with SQCG_MS_SHIFT_RU)
  int loops = 0, ru_launches = 0;
  int ru_count[SQCG_MAX_SHIFTS] = {};
  double sig_l[SQCG_MAX_SHIFTS], tol_l[SQCG_MAX_SHIFTS];
  for (int j = 0; j < nshift; ++j) {
    sig_l[j] = shifts[perm[j]];
    tol_l[j] = tol[perm[j]];
  }
  const bool eager = eager_mode();
  CGGraph* g = nullptr;
  if (!eager) SQCG_TRY(capture(ctx, KIND_MS, mixed, b, xs, nshift, &g));
  for (;;) {
    int seg = 0;
    if (eager) SQCG_TRY(run_eager(ctx, KIND_MS, mixed, b, xs, nshift, max_iter, s, &seg));
    else SQCG_TRY(run_loop(ctx, g, max_iter, s, &seg));
    loops += seg;
    if (h->done || !(h->ms_ru && h->need_update)) break;
    SQCG_TRY(ms_shift_aware_update(ctx, mixed, nshift, sig_l, tol_l, perm, b, xs, s, ru_count, &ru_launches,
                                   ru_shifts != 0));
  }
  int launches = 2 + 1 + nshift + loops * kMSKernelsPerIter + ru_launches;
  const int loop_status = h->done ? h->status : SQCG_ERR_NOT_CONVERGED;
  int iters_s[SQCG_MAX_SHIFTS];
  for (int j = 0; j < nshift; ++j) iters_s[j] = h->iters_s[j];

  // Per-shift FP64 true residual and refinement. Each refinement CG starts by
  // computing r = b - (sigma_s - D_eo D_oe) x_s in FP64 and stops there when
  // x_s already meets its tolerance. Mixed mode refines all shifts together as
  // one batched mixed-precision CG (one RHS per shift, per-RHS sigma, shared
  // source), so the links are read once per block of shifts.
  int left = 1;
  for (int j = 0; j < nshift; ++j)
    if (max_iter - iters_s[j] > left) left = max_iter - iters_s[j];
  int worst = SQCG_OK;
  sqcg_info ri[SQCG_MAX_SHIFTS] = {};
  if (loop_status == SQCG_ERR_BREAKDOWN) {  // no refinement from a broken-down Krylov space
    for (int j = 0; j < nshift; ++j) {
      ri[j].status = SQCG_ERR_BREAKDOWN;
      ri[j].true_rel_resid = NAN;
    }
  } else if (mixed) {
    // library-owned copies (solutions stacked, then the source) keep the cached batched plan
    // valid across calls whatever buffers the caller passes
    if (ctx->ms_stack_n != nshift) {
      SQCG_CUDA_TRY(cudaStreamSynchronize(s));
      cudaFree(ctx->ms_stack);
      ctx->ms_stack = nullptr;
      ctx->ms_stack_n = 0;
      if (cudaMalloc(&ctx->ms_stack, (size_t)(nshift + 1) * n * sizeof(double2)) != cudaSuccess) {
        cudaGetLastError();
        return SQCG_ERR_NO_MEMORY;
      }
      ctx->ms_stack_n = nshift;
    }
    double sig[SQCG_MAX_SHIFTS], tl[SQCG_MAX_SHIFTS];
    for (int j = 0; j < nshift; ++j) {
      sig[j] = shifts[perm[j]];
      tl[j] = tol[perm[j]];
      SQCG_CUDA_TRY(cudaMemcpyAsync(ctx->ms_stack + (size_t)j * n, xs[j], n * sizeof(double2),
                                    cudaMemcpyDeviceToDevice, s));
    }
    double2* bcopy = ctx->ms_stack + (size_t)nshift * n;
    SQCG_CUDA_TRY(cudaMemcpyAsync(bcopy, b, n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    sqcg_ctx* cl[1] = {ctx};
    const int nr[1] = {nshift};
    const void* bl[1] = {bcopy};
    void* xl[1] = {ctx->ms_stack};
    const int st = batched_solve(1, cl, nr, sig, tl, bl, 1, xl, left, ri);
    if (st == SQCG_ERR_CUDA || st == SQCG_ERR_INVALID_ARG || st == SQCG_ERR_NO_MEMORY) return st;
    for (int j = 0; j < nshift; ++j)
      SQCG_CUDA_TRY(cudaMemcpyAsync(xs[j], ctx->ms_stack + (size_t)j * n, n * sizeof(double2),
                                    cudaMemcpyDeviceToDevice, s));
    SQCG_CUDA_TRY(cudaStreamSynchronize(s));
    launches += ri[0].launches + 2 * nshift;
  } else {
    for (int j = 0; j < nshift; ++j) {
      const int st = cg_solve_sigma(ctx, shifts[perm[j]], b, xs[j], tol[perm[j]], left, mode, &ri[j]);
      if (st == SQCG_ERR_CUDA || st == SQCG_ERR_INVALID_ARG || st == SQCG_ERR_NO_MEMORY) return st;
      ri[j].status = st;
      launches += ri[j].launches;
    }
  }
  for (int j = 0; j < nshift; ++j) {
    const int u = perm[j];
    const int st = ri[j].status;
    if (info) {
      info[u].iters = iters_s[j] + ri[j].iters;
      info[u].reliable_updates = ri[j].reliable_updates + ru_count[j];
      info[u].status = st;
      info[u].true_rel_resid = ri[j].true_rel_resid;
    }
    if (st != SQCG_OK && worst == SQCG_OK) worst = st;
  }
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info)
    for (int j = 0; j < nshift; ++j) {
      info[j].seconds = secs;
      info[j].launches = launches;
    }
  return worst;
}

extern "C" int sqcg_multishift_ru_record(const sqcg_ctx* ctx, int max_updates, int* nupdates, int* nshift_out,
                                         int* iter, double* base, double* loss) {
  if (!ctx || !nupdates || !nshift_out || max_updates < 0) return SQCG_ERR_INVALID_ARG;
  *nupdates = ctx->ms_rec_n;
  *nshift_out = ctx->ms_rec_nshift;
  int m = ctx->ms_rec_n < max_updates ? ctx->ms_rec_n : max_updates;
  if (m > SQCG_MS_RU_RECORD) m = SQCG_MS_RU_RECORD;
  const int ns = ctx->ms_rec_nshift;
  for (int u = 0; u < m; ++u) {
    if (iter) iter[u] = ctx->ms_rec_iter[u];
    if (base) base[u] = ctx->ms_rec_base[u];
    if (loss)
      for (int j = 0; j < ns; ++j) loss[(size_t)u * ns + j] = ctx->ms_rec_loss[u][j];
  }
  return SQCG_OK;
}

// ---------------------------------------------------------------------------
// rational-function application (the multi-mass CG's use inside RHMC)
// ---------------------------------------------------------------------------
namespace {

struct Coeffs {
  const double2* x[SQCG_MAX_SHIFTS];
  double a[SQCG_MAX_SHIFTS];
};

// out = a0 b + sum_s a_s x_s, FP64
__global__ void k_rational_combine(Coeffs C, int nshift, double a0, const double2* __restrict__ b,
                                   double2* __restrict__ out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 bv = b[i];
  double re = a0 * bv.x, im = a0 * bv.y;
  for (int j = 0; j < nshift; ++j) {
    const double2 v = C.x[j][i];
    re = fma(C.a[j], v.x, re);
    im = fma(C.a[j], v.y, im);
  }
  out[i] = make_double2(re, im);
}

}  // namespace

extern "C" int sqcg_rational_apply(sqcg_ctx* ctx, int nshift, const double* shifts, const double* residues, double a0,
                                   const void* b, void* out, double tol, int max_iter, int mode, sqcg_info* info) {
  if (!ctx || nshift < 1 || nshift > SQCG_MAX_SHIFTS || !shifts || !residues || !isfinite(a0) || !out || out == b ||
      !(tol > 0))
    return SQCG_ERR_INVALID_ARG;
  SQCG_TRY(validate_vec(b, SQCG_F64));
  SQCG_TRY(validate_vec(out, SQCG_F64));
  for (int j = 0; j < nshift; ++j)
    if (!isfinite(residues[j])) return SQCG_ERR_INVALID_ARG;
  if (!ctx->have_links) return SQCG_ERR_NO_LINKS;
  // per-shift solutions in library-owned FP64 buffers
  const size_t bytes = (size_t)ctx->g.Vh * 3 * sizeof(double2);
  if (ctx->rat_n < nshift) {
    SQCG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    for (int j = 0; j < ctx->rat_n; ++j) cudaFree(ctx->rat_x[j]);
    ctx->rat_n = 0;
    free_graphs(ctx);
    for (int j = 0; j < nshift; ++j) {
      if (cudaMalloc(&ctx->rat_x[j], bytes) != cudaSuccess) {
        cudaGetLastError();
        for (int k = 0; k < j; ++k) cudaFree(ctx->rat_x[k]);
        return SQCG_ERR_NO_MEMORY;
      }
    }
    ctx->rat_n = nshift;
  }
  double tols[SQCG_MAX_SHIFTS];
  for (int j = 0; j < nshift; ++j) tols[j] = tol;
  const int rc = sqcg_multishift_cg_solve(ctx, nshift, shifts, b, ctx->rat_x, tols, max_iter, mode, info);
  if (rc == SQCG_ERR_CUDA || rc == SQCG_ERR_INVALID_ARG || rc == SQCG_ERR_NO_MEMORY) return rc;
  Coeffs C;
  for (int j = 0; j < nshift; ++j) {
    C.x[j] = (const double2*)ctx->rat_x[j];
    C.a[j] = residues[j];
  }
  const int n = ctx->g.Vh * 3;
  k_rational_combine<<<grid_for(n, 256), 256, 0, ctx->stream>>>(C, nshift, a0, (const double2*)b, (double2*)out, n);
  SQCG_CUDA_TRY(cudaGetLastError());
  SQCG_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return rc;
}
