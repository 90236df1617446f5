// C ABI entry points: context lifetime, links, colour-vector packing, Dslash
// and normal operator. Solvers are in cg.cu.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "sqcg_internal.cuh"

static thread_local char g_last_cuda_error[256] = "";

void sqcg_set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s (%s) at %s:%d", cudaGetErrorString(e), what, file,
           line);
}

int ensure_workspace(sqcg_ctx* ctx) {
  if (ctx->st) return SQCG_OK;
  const size_t n = (size_t)ctx->g.Vh * 3;
  // the largest grid of any reducing kernel: Dslash uses 128-thread blocks
  ctx->max_blocks = grid_for(ctx->g.Vh, 128);
  bool ok = cudaMalloc((void**)&ctx->r64, n * sizeof(double2)) == cudaSuccess &&
            cudaMalloc((void**)&ctx->p64, n * sizeof(double2)) == cudaSuccess &&
            cudaMalloc((void**)&ctx->Ap64, n * sizeof(double2)) == cudaSuccess &&
            cudaMalloc((void**)&ctx->tmp64, n * sizeof(double2)) == cudaSuccess &&
            cudaMalloc((void**)&ctx->r32, n * sizeof(float2)) == cudaSuccess &&
            cudaMalloc((void**)&ctx->p32, n * sizeof(float2)) == cudaSuccess &&
            cudaMalloc((void**)&ctx->Ap32, n * sizeof(float2)) == cudaSuccess &&
            cudaMalloc((void**)&ctx->tmp32, n * sizeof(float2)) == cudaSuccess &&
            cudaMalloc((void**)&ctx->q32, n * sizeof(float2)) == cudaSuccess &&
            cudaMalloc((void**)&ctx->xh32, n * sizeof(float2)) == cudaSuccess &&
            cudaMalloc((void**)&ctx->xff, n * sizeof(float4)) == cudaSuccess &&
            cudaMalloc((void**)&ctx->partials, 4 * (size_t)ctx->max_blocks * sizeof(double)) == cudaSuccess &&
            cudaMalloc((void**)&ctx->fin_aux, 64 * sizeof(float2)) == cudaSuccess &&
            cudaMalloc((void**)&ctx->fin_cnt, 32 * sizeof(unsigned)) == cudaSuccess &&
            cudaMalloc((void**)&ctx->st, sizeof(SolverState)) == cudaSuccess &&
            cudaMallocHost((void**)&ctx->st_host, sizeof(SolverState)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_workspace(ctx);
    return SQCG_ERR_NO_MEMORY;
  }
  SQCG_CUDA_TRY(cudaMemsetAsync(ctx->st, 0, sizeof(SolverState), ctx->stream));
  SQCG_CUDA_TRY(cudaMemsetAsync(ctx->fin_cnt, 0, 32 * sizeof(unsigned), ctx->stream));
  return SQCG_OK;
}

void free_workspace(sqcg_ctx* ctx) {
  cudaFree(ctx->r64); cudaFree(ctx->p64); cudaFree(ctx->Ap64); cudaFree(ctx->tmp64);
  cudaFree(ctx->r32); cudaFree(ctx->p32); cudaFree(ctx->Ap32); cudaFree(ctx->tmp32);
  cudaFree(ctx->q32); cudaFree(ctx->xh32); cudaFree(ctx->xff);
  cudaFree(ctx->partials); cudaFree(ctx->st);
  cudaFree(ctx->fin_aux); cudaFree(ctx->fin_cnt);
  ctx->fin_aux = nullptr;
  ctx->fin_cnt = nullptr;
  cudaFree(ctx->pers_part); cudaFree(ctx->pers_bar); cudaFree(ctx->pers_rq);
  ctx->pers_rq = nullptr;
  ctx->pers_part = nullptr;
  ctx->pers_bar = nullptr;
  ctx->pers_grid = 0;
  if (ctx->st_host) cudaFreeHost(ctx->st_host);
  ctx->r64 = ctx->p64 = ctx->Ap64 = ctx->tmp64 = nullptr;
  ctx->r32 = ctx->p32 = ctx->Ap32 = ctx->tmp32 = nullptr;
  ctx->q32 = ctx->xh32 = nullptr;
  ctx->xff = nullptr;
  ctx->partials = nullptr;
  ctx->st = nullptr;
  ctx->st_host = nullptr;
  for (int j = 1; j < ctx->ms_nalloc; ++j) cudaFree(ctx->ms_p[j]);
  for (int j = 0; j < SQCG_MAX_SHIFTS; ++j) ctx->ms_p[j] = nullptr;
  ctx->ms_nalloc = 0;
  for (int j = 0; j < ctx->rat_n; ++j) cudaFree(ctx->rat_x[j]);
  for (int j = 0; j < SQCG_MAX_SHIFTS; ++j) ctx->rat_x[j] = nullptr;
  cudaFree(ctx->ms_stack);
  ctx->ms_stack = nullptr;
  ctx->ms_stack_n = 0;
  cudaFree(ctx->ms_ru_vec);
  ctx->ms_ru_vec = nullptr;
  ctx->rat_n = 0;
}

extern "C" {

int sqcg_create(const int dims[4], int flags, void* cuda_stream, sqcg_ctx** out) {
  if (!dims || !out) return SQCG_ERR_INVALID_ARG;
  *out = nullptr;
  if (flags & ~(SQCG_ANTIPERIODIC_T | SQCG_PHASES_FOLDED)) return SQCG_ERR_INVALID_ARG;
  long V = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (dims[mu] < 4 || (dims[mu] & 1)) return SQCG_ERR_INVALID_ARG;
    V *= dims[mu];
  }
  // device indices are 32-bit: keep 4 V (link-pack threads) and 9 Vh * 8 well inside int range
  if (V > (1L << 28)) return SQCG_ERR_INVALID_ARG;
  sqcg_ctx* c = (sqcg_ctx*)calloc(1, sizeof(sqcg_ctx));
  if (!c) return SQCG_ERR_NO_MEMORY;
  memcpy(c->L, dims, sizeof(c->L));
  c->flags = flags;
  Geom& g = c->g;
  g.Lx = dims[0];
  g.Ly = dims[1];
  g.Lz = dims[2];
  g.Lt = dims[3];
  g.Lxh = dims[0] / 2;
  g.Vh = (int)(V / 2);
  g.sy = g.Lxh;
  g.sz = g.Lxh * g.Ly;
  g.st = g.Lxh * g.Ly * g.Lz;
  g.apbc = (flags & SQCG_ANTIPERIODIC_T) ? 1 : 0;
  c->stream = (cudaStream_t)cuda_stream;
  c->ru_arith = SQCG_FF;
  {  // SQCG_PDL=0: launch the loop kernels without programmatic dependent launch
    const char* pdl = getenv("SQCG_PDL");
    c->pdl = (pdl && strcmp(pdl, "0") == 0) ? 0 : 1;
  }
  c->ru_delta = 0.001;
  c->ru_interval = 100;
  if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    sqcg_set_last_cuda_error(cudaGetLastError(), "cudaStreamCreate", __FILE__, __LINE__);
    free(c);
    return SQCG_ERR_CUDA;
  }
  *out = c;
  return SQCG_OK;
}

int sqcg_destroy(sqcg_ctx* ctx) {
  if (!ctx) return SQCG_OK;
  cudaStreamSynchronize(ctx->stream);
  free_graphs(ctx);
  free_batch_plan(ctx);
  free_workspace(ctx);
  cudaFree(ctx->fat64); cudaFree(ctx->lng64); cudaFree(ctx->fat32); cudaFree(ctx->lng32);
  cudaFree(ctx->fatb32); cudaFree(ctx->lngb32);
  cudaFree(ctx->fatff); cudaFree(ctx->lngff);
  cudaFree(ctx->stage);
  cudaStreamDestroy(ctx->cap_stream);
  free(ctx);
  return SQCG_OK;
}

int sqcg_set_stream(sqcg_ctx* ctx, void* cuda_stream) {
  if (!ctx) return SQCG_ERR_INVALID_ARG;
  ctx->stream = (cudaStream_t)cuda_stream;
  return SQCG_OK;
}

int sqcg_set_reliable_update(sqcg_ctx* ctx, double delta, int interval) {
  if (!ctx || !(delta > 0.0) || !(delta < 1.0) || interval < 1) return SQCG_ERR_INVALID_ARG;
  ctx->ru_delta = delta;
  ctx->ru_interval = interval;
  return SQCG_OK;
}

int sqcg_set_update_arithmetic(sqcg_ctx* ctx, int prec) {
  if (!ctx || (prec != SQCG_F64 && prec != SQCG_FF)) return SQCG_ERR_INVALID_ARG;
  if (prec != ctx->ru_arith) free_graphs(ctx);  // captured loops hold the old kernels
  ctx->ru_arith = prec;
  return SQCG_OK;
}

int sqcg_spinor_bytes(const sqcg_ctx* ctx, int prec, size_t* bytes) {
  if (!ctx || !bytes || (prec != SQCG_F64 && prec != SQCG_F32 && prec != SQCG_FF)) return SQCG_ERR_INVALID_ARG;
  *bytes = (size_t)ctx->g.Vh * 3 * (prec == SQCG_F32 ? sizeof(float2) : sizeof(double2));
  return SQCG_OK;
}

int sqcg_load_links(sqcg_ctx* ctx, const double* fat, const double* lng, int opts) {
  if (!ctx) return SQCG_ERR_INVALID_ARG;
  return layout_load_links(ctx, fat, lng, opts);
}

int sqcg_pack_spinor(sqcg_ctx* ctx, int prec, const double* host, void* dev) {
  if (!ctx) return SQCG_ERR_INVALID_ARG;
  return layout_pack_spinor(ctx, prec, host, dev);
}

int sqcg_unpack_spinor(sqcg_ctx* ctx, int prec, const void* dev, double* host) {
  if (!ctx) return SQCG_ERR_INVALID_ARG;
  return layout_unpack_spinor(ctx, prec, dev, host);
}

int sqcg_dslash(sqcg_ctx* ctx, int out_parity, int prec, const void* in, void* out) {
  if (!ctx || !in || !out || in == out) return SQCG_ERR_INVALID_ARG;
  if (prec == SQCG_FF) {
    if (((uintptr_t)in | (uintptr_t)out) % 16) return SQCG_ERR_INVALID_ARG;
    FFLaunch F = {};
    F.out_parity = out_parity;
    F.in = in;
    F.out_ff = out;
    return launch_dslash_ff(ctx, F, ctx->stream);
  }
  if (prec != SQCG_F64 && prec != SQCG_F32) return SQCG_ERR_INVALID_ARG;
  DslashLaunch L = {};
  L.out_parity = out_parity;
  L.prec = L.out_prec = prec;
  L.epi = EPI_PLAIN;
  L.in = in;
  L.out = out;
  return launch_dslash(ctx, L, ctx->stream);
}

int sqcg_normal_op(sqcg_ctx* ctx, double sigma, int prec, const void* x, void* y) {
  if (!ctx || !x || !y || x == y) return SQCG_ERR_INVALID_ARG;
  if (prec != SQCG_F64 && prec != SQCG_F32) return SQCG_ERR_INVALID_ARG;
  if (!ctx->have_links) return SQCG_ERR_NO_LINKS;
  SQCG_TRY(ensure_workspace(ctx));
  void* tmp = (prec == SQCG_F64) ? (void*)ctx->tmp64 : (void*)ctx->tmp32;
  DslashLaunch L = {};
  L.out_parity = 1;
  L.prec = L.out_prec = prec;
  L.epi = EPI_PLAIN;
  L.in = x;
  L.out = tmp;
  SQCG_TRY(launch_dslash(ctx, L, ctx->stream));
  L.out_parity = 0;
  L.epi = EPI_NORMAL;
  L.in = tmp;
  L.out = y;
  L.y = x;
  L.sigma = sigma;
  return launch_dslash(ctx, L, ctx->stream);
}

const char* sqcg_strerror(int status) {
  switch (status) {
    case SQCG_OK: return "ok";
    case SQCG_ERR_INVALID_ARG: return "invalid argument";
    case SQCG_ERR_CUDA: return g_last_cuda_error[0] ? g_last_cuda_error : "CUDA error";
    case SQCG_ERR_NOT_CONVERGED: return "not converged within max_iter";
    case SQCG_ERR_BREAKDOWN: return "breakdown: <p,Ap> <= 0 or non-finite reduction";
    case SQCG_ERR_RECON_REJECTED: return "12-real long links rejected: links are not a global scale times SU(3)";
    case SQCG_ERR_NO_LINKS: return "no links loaded";
    case SQCG_ERR_NO_MEMORY: return "device allocation failed";
    case SQCG_ERR_SCRATCH_TOO_SMALL:
      return "lattice too large for the fixed 8 MiB scratch of sqcg_normal_op_noalloc "
             "(at most 174762 sites per parity in FP64, 349525 in FP32)";
    default: return "unknown status";
  }
}

}  // extern "C"
