// Solver drivers: single-mass CG (FP64, or mixed FP32/FP64 with reliable
// updates) and multi-mass (multi-shift) CG (paper Sec. 3-4: the single- and
// multi-mass staggered CG; the multi-mass form is the benchmarked routine).
//
// All Krylov scalars stay in device memory (SolverState). The iteration is
// captured once into a CUDA graph of kChunk iterations; every kernel in it is
// gated on the device-side state, so iterations after convergence cost only
// empty launches. The host reads the state once per chunk.
#include <chrono>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "sqcg_internal.cuh"

namespace {

constexpr int kChunk = 16;
constexpr int kCGKernelsPerIter = 6;  // enqueue_cg_iteration
constexpr int kMSKernelsPerIter = 4;  // enqueue_ms_iteration

enum { KIND_CG = 0, KIND_MS = 1 };

}  // namespace

struct CGGraph {
  int kind, mixed, nshift;
  const void* b;
  void* x[SQCG_MAX_SHIFTS];
  cudaGraphExec_t exec;
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

// kernels of one single-mass CG iteration (see FIN_* in solver_device.cuh)
int enqueue_cg_iteration(sqcg_ctx* ctx, int mixed, const void* b, void* x, cudaStream_t s) {
  const int wp = mixed ? SQCG_F32 : SQCG_F64;
  void* p = mixed ? (void*)ctx->p32 : (void*)ctx->p64;
  void* Ap = mixed ? (void*)ctx->Ap32 : (void*)ctx->Ap64;
  void* tmp = mixed ? (void*)ctx->tmp32 : (void*)ctx->tmp64;
  void* r = mixed ? (void*)ctx->r32 : (void*)ctx->r64;
  const double* sigma_dev = &ctx->st->sigma;

  DslashLaunch L = {};
  // tmp_o = D_oe p
  L.out_parity = 1; L.prec = L.out_prec = wp; L.epi = EPI_PLAIN; L.in = p; L.out = tmp; L.gate = GATE_ITER;
  SQCG_TRY(launch_dslash(ctx, L, s));
  // Ap = sigma p - D_eo tmp; alpha = |r|^2 / <p, Ap>
  L = DslashLaunch{};
  L.out_parity = 0; L.prec = L.out_prec = wp; L.epi = EPI_NORMAL_DOT; L.in = tmp; L.out = Ap; L.y = p;
  L.sigma_dev = sigma_dev; L.gate = GATE_ITER; L.fin = FIN_PAP;
  SQCG_TRY(launch_dslash(ctx, L, s));
  // x += alpha p; r -= alpha Ap; beta, convergence / reliable-update trigger
  SQCG_TRY(launch_cg_update_x(ctx, mixed, (double2*)x, s));
  // reliable update / final check: r = b - A x in FP64
  L = DslashLaunch{};
  L.out_parity = 1; L.prec = L.out_prec = SQCG_F64; L.epi = EPI_PLAIN; L.in = x; L.out = ctx->tmp64;
  L.gate = GATE_UPDATE;
  SQCG_TRY(launch_dslash(ctx, L, s));
  L = DslashLaunch{};
  L.out_parity = 0; L.prec = SQCG_F64; L.out_prec = wp; L.epi = EPI_TRUE_RESID; L.in = ctx->tmp64; L.out = r;
  L.y = x; L.b = b; L.sigma_dev = sigma_dev; L.gate = GATE_UPDATE; L.fin = FIN_TRUE_RESID;
  SQCG_TRY(launch_dslash(ctx, L, s));
  // p = r + beta p
  SQCG_TRY(launch_cg_xpay(ctx, mixed, s));
  return SQCG_OK;
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
  L.sigma_dev = &ctx->st->sigma; L.gate = GATE_ITER; L.fin = FIN_MS_PAP;
  SQCG_TRY(launch_dslash(ctx, L, s));
  SQCG_TRY(launch_ms_update_x(ctx, mixed, nshift, x, s));
  SQCG_TRY(launch_ms_xpay(ctx, mixed, nshift, s));
  return SQCG_OK;
}

int capture(sqcg_ctx* ctx, int kind, int mixed, const void* b, void* const* x, int nx, CGGraph** out) {
  CGGraph* g = find_graph(ctx, kind, mixed, b, x, nx);
  if (g) { *out = g; return SQCG_OK; }
  cudaStream_t cs = ctx->cap_stream;
  SQCG_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  int rc = SQCG_OK;
  for (int k = 0; k < kChunk && rc == SQCG_OK; ++k) {
    if (kind == KIND_CG) rc = enqueue_cg_iteration(ctx, mixed, b, x[0], cs);
    else rc = enqueue_ms_iteration(ctx, mixed, nx, (double2* const*)x, cs);
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &graph);
  if (rc != SQCG_OK) { if (graph) cudaGraphDestroy(graph); return rc; }
  if (e != cudaSuccess) { sqcg_set_last_cuda_error(e, "cudaStreamEndCapture", __FILE__, __LINE__); return SQCG_ERR_CUDA; }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) { sqcg_set_last_cuda_error(e, "cudaGraphInstantiate", __FILE__, __LINE__); return SQCG_ERR_CUDA; }
  g = (CGGraph*)calloc(1, sizeof(CGGraph));
  if (!g) { cudaGraphExecDestroy(exec); return SQCG_ERR_NO_MEMORY; }
  g->kind = kind; g->mixed = mixed; g->nshift = nx; g->b = b; g->exec = exec;
  for (int j = 0; j < nx; ++j) g->x[j] = x[j];
  add_graph(ctx, g);
  *out = g;
  return SQCG_OK;
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

// run chunks of the captured loop until the device state says done; *chunks = graphs launched
int run_loop(sqcg_ctx* ctx, CGGraph* g, int max_iter, cudaStream_t s, int* chunks) {
  const long max_chunks = (long)max_iter / kChunk + 8;
  *chunks = 0;
  for (long c = 0; c < max_chunks; ++c) {
    SQCG_CUDA_TRY(cudaGraphLaunch(g->exec, s));
    *chunks += 1;
    SQCG_TRY(read_state(ctx, s));
    if (ctx->st_host->done) return SQCG_OK;
  }
  return SQCG_OK;
}

// |b - (sigma - D_eo D_oe) x|^2 in FP64 (r64 as scratch); result in *rr
int true_residual2(sqcg_ctx* ctx, double sigma, const void* b, const void* x, double* rr, cudaStream_t s) {
  DslashLaunch L = {};
  L.out_parity = 1; L.prec = L.out_prec = SQCG_F64; L.epi = EPI_PLAIN; L.in = x; L.out = ctx->tmp64;
  SQCG_TRY(launch_dslash(ctx, L, s));
  L = DslashLaunch{};
  L.out_parity = 0; L.prec = L.out_prec = SQCG_F64; L.epi = EPI_TRUE_RESID; L.in = ctx->tmp64; L.out = ctx->r64;
  L.y = x; L.b = b; L.sigma = sigma; L.fin = FIN_STORE;
  SQCG_TRY(launch_dslash(ctx, L, s));
  SQCG_TRY(read_state(ctx, s));
  *rr = ctx->st_host->pAp;
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
  h->delta2 = 0.1 * 0.1;
  h->max_iter = max_iter;
  h->update_interval = mixed ? 100 : (1 << 30);
  h->mixed = mixed;
  h->status = SQCG_OK;
  SQCG_TRY(write_state(ctx, s));
  SQCG_TRY(launch_norm2_f64(ctx, (const double2*)b, FIN_BB, s));
  // r = b - A x0 (FP64), p = r, both in the working precision
  DslashLaunch L = {};
  L.out_parity = 1; L.prec = L.out_prec = SQCG_F64; L.epi = EPI_PLAIN; L.in = x; L.out = ctx->tmp64;
  SQCG_TRY(launch_dslash(ctx, L, s));
  L = DslashLaunch{};
  L.out_parity = 0; L.prec = SQCG_F64; L.out_prec = mixed ? SQCG_F32 : SQCG_F64; L.epi = EPI_TRUE_RESID;
  L.in = ctx->tmp64; L.out = mixed ? (void*)ctx->r32 : (void*)ctx->r64;
  L.out2 = mixed ? (void*)ctx->p32 : (void*)ctx->p64;
  L.y = x; L.b = b; L.sigma = sigma; L.fin = FIN_INIT;
  SQCG_TRY(launch_dslash(ctx, L, s));
  SQCG_TRY(read_state(ctx, s));

  int status = SQCG_OK;
  int launches = 3, chunks = 0;
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
    CGGraph* g = nullptr;
    void* xs[1] = {x};
    SQCG_TRY(capture(ctx, KIND_CG, mixed, b, xs, 1, &g));
    SQCG_TRY(run_loop(ctx, g, max_iter, s, &chunks));
    launches += chunks * kChunk * kCGKernelsPerIter;
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

// Multi-shift CG: (sigma_s - D_eo D_oe) x_s = b for all shifts from one Krylov
// space built on the smallest shift; FP64 scalar recurrences. In mixed mode
// each shift whose FP64 true residual is above its tolerance is then refined
// by mixed-precision CG started from x_s.
extern "C" int sqcg_multishift_cg_solve(sqcg_ctx* ctx, int nshift, const double* shifts, const void* b,
                                        void* const* x, const double* tol, int max_iter, int mode,
                                        sqcg_info* info) {
  const auto t0 = std::chrono::steady_clock::now();
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
  h->rr = h->rr_prev = h->bb;
  SQCG_TRY(write_state(ctx, s));

  CGGraph* g = nullptr;
  SQCG_TRY(capture(ctx, KIND_MS, mixed, b, xs, nshift, &g));
  int chunks = 0;
  SQCG_TRY(run_loop(ctx, g, max_iter, s, &chunks));
  int launches = 1 + 1 + nshift + chunks * kChunk * kMSKernelsPerIter;
  const int loop_status = h->done ? h->status : SQCG_ERR_NOT_CONVERGED;
  int iters_s[SQCG_MAX_SHIFTS];
  for (int j = 0; j < nshift; ++j) iters_s[j] = h->iters_s[j];
  const double bb = h->bb;

  // per-shift FP64 true residual, refinement where needed
  int worst = SQCG_OK;
  for (int j = 0; j < nshift; ++j) {
    const int u = perm[j];
    const double sig = shifts[u];
    double rr = 0.0;
    int st = (loop_status == SQCG_ERR_BREAKDOWN) ? SQCG_ERR_BREAKDOWN : SQCG_OK;
    SQCG_TRY(true_residual2(ctx, sig, b, xs[j], &rr, s));
    launches += 2;
    double rel = sqrt(rr / bb);
    int extra = 0, updates = 0;
    if (st == SQCG_OK && !(rel <= tol[u])) {
      sqcg_info ri;
      const int left = max_iter - iters_s[j] > 0 ? max_iter - iters_s[j] : 1;
      st = cg_solve_sigma(ctx, sig, b, xs[j], tol[u], left, mode, &ri);
      if (st == SQCG_ERR_CUDA || st == SQCG_ERR_INVALID_ARG || st == SQCG_ERR_NO_MEMORY) return st;
      extra = ri.iters;
      updates = ri.reliable_updates;
      launches += ri.launches;
      rel = ri.true_rel_resid;
    }
    if (info) {
      info[u].iters = iters_s[j] + extra;
      info[u].reliable_updates = updates;
      info[u].status = st;
      info[u].true_rel_resid = rel;
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
