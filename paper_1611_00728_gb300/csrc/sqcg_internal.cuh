// Internal declarations of the sqcg CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/sqcg.h"

// ---------------------------------------------------------------------------
// error plumbing: every CUDA call is checked, the code turns into SQCG_ERR_CUDA
// ---------------------------------------------------------------------------
#define SQCG_CUDA_TRY(expr)                                   \
  do {                                                        \
    cudaError_t _e = (expr);                                  \
    if (_e != cudaSuccess) {                                  \
      sqcg_set_last_cuda_error(_e, #expr, __FILE__, __LINE__); \
      return SQCG_ERR_CUDA;                                   \
    }                                                         \
  } while (0)

#define SQCG_TRY(expr)         \
  do {                         \
    int _s = (expr);           \
    if (_s != SQCG_OK) return _s; \
  } while (0)

void sqcg_set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);

// ---------------------------------------------------------------------------
// geometry of the even-odd half lattice
// ---------------------------------------------------------------------------
struct Geom {
  int Lx, Ly, Lz, Lt;
  int Lxh;         // Lx / 2
  int Vh;          // sites per parity
  int sy, sz, st;  // half-lattice index strides of y, z, t: Lxh, Lxh*Ly, Lxh*Ly*Lz
  int apbc;        // antiperiodic time direction
};

// Link storage per field: [parity][mu][elem][Vh] complex, elem = 9 (full) or 6 (two rows).
template <typename R2>
struct LinkField {
  const R2* par[2];  // base of each parity
  int nelem;         // 9 or 6
};

// ---------------------------------------------------------------------------
// solver state kept in device memory (scalars never leave the GPU inside a solve)
// ---------------------------------------------------------------------------
#define SQCG_MAX_SHIFTS 32

struct SolverState {
  double sigma;    // diagonal term of the Krylov system
  double bb;       // |b|^2
  double stop_rr;  // tol^2 |b|^2
  double rr;       // current iterated |r|^2
  double rr_prev;  // |r|^2 of the previous iteration
  double rr_true;  // last FP64 true residual |b - A x|^2
  double rr_max;   // max iterated |r|^2 since the last reliable update
  double delta2;   // reliable-update trigger: update when |r|^2 < delta2 * rr_max
  // stop_rr is set to tol^2 by the host and multiplied by |b|^2 in FIN_BB
  double pAp, alpha, beta;
  int iter, max_iter;
  int iter_last_update, update_interval;
  int done;         // loop finished (converged, breakdown or out of iterations)
  int status;       // SQCG_OK / SQCG_ERR_*
  int need_update;  // the FP64 true-residual pass runs in this iteration
  int updates;      // reliable updates performed inside the loop
  int mixed;        // working vectors are FP32
  int vh;           // sites per parity (network input scale)
  int use_if;       // the reliable-update pass is an IF node whose condition FIN_UPDATE sets
  int loop_count;        // iterations of the device-side WHILE loop so far
  int loop_limit;        // hard bound on loop_count (the loop always ends)
  unsigned long long h_while;  // conditional handle of the WHILE node (cudaGraphConditionalHandle)
  unsigned long long h_if;     // conditional handle of the reliable-update IF node

  // single-reduction CG (mixed mode): one reduction per iteration, <r, A r> and |r|^2 together
  int sr;            // the loop is the single-reduction form
  int after_update;  // the next FIN_SR_STEP follows a reliable update (its residual is the true one)
  double sr_alpha_prev;  // alpha of the previous iteration

  // flexible CG with the network preconditioner
  double rz;          // <z_k, r_k>
  double nn_s;        // network input scale sqrt(3 Vh) / |r|
  double nn_inv_s;    // 1 / nn_s

  // multi-shift CG (Jegerlehner recurrences; shift s uses sigma + dsig[s])
  int nshift;
  int ms_final;  // the loop has just ended: the fused update still applies the last x_s updates
  int active[SQCG_MAX_SHIFTS];  // 1 iterating, 2 converged with its last x update pending, 0 done
  double dsig[SQCG_MAX_SHIFTS];
  double stop_rr_s[SQCG_MAX_SHIFTS];
  double zeta[SQCG_MAX_SHIFTS], zeta_prev[SQCG_MAX_SHIFTS];
  double alpha_s[SQCG_MAX_SHIFTS], beta_s[SQCG_MAX_SHIFTS];
  double alpha_prev, beta_prev;
  int iters_s[SQCG_MAX_SHIFTS];
  int ms_ru;           // shift-aware reliable updates: the loop pauses when need_update is set
  double ms_sums[3];   // the host-driven update's sums (k_ms_ru_sum3)
};

// ---------------------------------------------------------------------------
// batched multi-RHS CG over several lattices (one state entry per RHS)
// ---------------------------------------------------------------------------
#define SQCG_MS_RU_RECORD 16  // shift-aware reliable updates recorded per multi-shift solve
#define SQCG_MAX_BATCH_RHS 256
#define SQCG_MAX_LATTICES 16

struct RhsScalars {
  double sigma, bb, stop_rr, rr, rr_prev, rr_true, rr_max, pAp, alpha, beta;
  int iter, iter_last_update, active, status, need_update, updates;
};

struct BatchState {
  int nrhs, nblk;   // right-hand sides; FP32 RHS blocks over all lattices
  int max_iter, update_interval;
  double delta2;
  int loop_count, loop_limit;
  int if_runs;    // executions of the reliable-update IF body
  int use_graph;  // the control kernels set the graph's conditional handles (0: eager launches)
  unsigned long long h_while, h_if;
  RhsScalars r[SQCG_MAX_BATCH_RHS];
  int blk_active[SQCG_MAX_BATCH_RHS];  // RHS block has an active RHS
  int blk_update[SQCG_MAX_BATCH_RHS];  // RHS block runs the FP64 reliable update
};

struct BatchPlan;  // defined in batched.cu

// gates: which kernels of a captured iteration actually run
// GATE_ITER: the loop goes on; GATE_UPDATE: a reliable update is due; GATE_STEP: the loop goes on and
// no reliable update is pending (the unrolled single-reduction body, whose IF node comes after K steps)
enum Gate { GATE_NONE = 0, GATE_ITER = 1, GATE_UPDATE = 2, GATE_STEP = 3 };

// what the finisher of a grid reduction does with the total
enum Finisher {
  FIN_NONE = 0,
  FIN_STORE = 1,       // store the total in state->pAp (generic scalar result slot)
  FIN_BB = 2,          // |b|^2 and the stopping threshold
  FIN_PAP = 3,         // alpha = rr / <p, A p>
  FIN_UPDATE = 4,      // new |r|^2, beta, convergence / reliable-update trigger
  FIN_TRUE_RESID = 5,  // FP64 true residual inside the loop
  FIN_INIT = 6,        // initial residual r = b - A x0
  FIN_MS_PAP = 7,      // multi-shift: alpha and the zeta recurrences of every shift
  FIN_MS_UPDATE = 8,   // multi-shift: new |r|^2, beta, per-shift convergence
  FIN_NN_SCALE = 9,    // network input scale from |r|^2
  FIN_FCG_PAP = 10,    // flexible CG: alpha = <z,r> / <p,Ap>
  FIN_FCG_BETA = 11,   // flexible CG (two sums): beta = (<z,r> - <z,r_old>) / <z_old,r_old>
  FIN_FCG_INIT = 12,   // flexible CG: <z_0, r_0>
  FIN_SR_STEP = 13,    // single-reduction CG (three sums, see EPI_SR_DOTS): convergence / reliable-update
                       // decision, then alpha and beta of the iteration
};

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct CGGraph;

struct sqcg_ctx {
  int L[4];
  int flags;
  Geom g;
  cudaStream_t stream;
  cudaStream_t cap_stream;  // private stream used only to capture graphs

  bool have_links;
  bool recon;
  unsigned long long links_gen;  // process-wide counter value of the last sqcg_load_links
  double long_scale;  // global real scale s0 of the long links (recon)

  // device links, [parity][mu][elem][Vh]
  double2* fat64;
  double2* lng64;
  float2* fat32;
  float2* lng32;
  // float-float copy of the FP64 links (hi, lo floats per real; float4 per complex), same layout
  float4* fatff;
  float4* lngff;
  // 8-way option (FP32 only): backward links -F_mu(n-mu)^+, -L_mu(n-3mu)^+ stored at n
  bool eightway;
  float2* fatb32;
  float2* lngb32;

  // host-copy staging for pack/unpack
  void* stage;
  size_t stage_bytes;

  // solver workspace (allocated on first solve)
  double2 *r64, *p64, *Ap64, *tmp64;
  float2 *r32, *p32, *Ap32, *tmp32;
  float2 *q32, *xh32;  // single-reduction mixed CG: q = A p, and the FP32 partial solution
  float4* xff;         // float-float copy of x for the reliable update (its odd intermediate lives in tmp64)
  double* partials;    // 4 * max_blocks: three sums of a Dslash epilogue, then the update kernel's sum
  float2* fin_aux;     // the single-reduction finisher's per-block totals (3 float-float slots a block)
  unsigned* fin_cnt;   // ... and its arrival counter (zero between launches)
  int max_blocks;
  int blas_grid;  // blocks of the streaming BLAS kernels (0 until first use)
  int pers_grid;        // blocks of the persistent CG loop (0 until first use, -1 unavailable)
  double* pers_part;    // its partial sums: [3][pers_grid] step sums, [2][pers_grid] cross terms
  unsigned* pers_bar;   // its grid-barrier words
  float2* pers_rq;      // its second buffers of r and q ([3][Vh] each)
  SolverState* st;       // device
  SolverState* st_host;  // pinned host mirror

  // multi-shift workspace
  void* ms_p[SQCG_MAX_SHIFTS];  // per-shift search directions (working precision)
  void* rat_x[SQCG_MAX_SHIFTS];  // per-shift solutions of sqcg_rational_apply (FP64)
  int rat_n;
  double2* ms_stack;  // batched refinement (FP64): per-shift solutions [nshift][3][Vh], then a copy of b
  int ms_stack_n;
  // shift-aware reliable updates of the multi-shift loop (SQCG_MS_SHIFT_RU)
  double2* ms_ru_vec;  // FP64 [2][3][Vh]: the base true residual r_0, then one shift's r_s
  int ms_rec_n, ms_rec_nshift;  // updates recorded by the last multi-shift solve; its shift count
  int ms_rec_iter[SQCG_MS_RU_RECORD];
  double ms_rec_base[SQCG_MS_RU_RECORD];
  double ms_rec_loss[SQCG_MS_RU_RECORD][SQCG_MAX_SHIFTS];  // caller's shift order
  int ms_nalloc;
  int ms_prec;

  int ru_arith;        // arithmetic of the mixed solvers' true residuals: SQCG_F64 or SQCG_FF (default)
  int pdl;             // launch the loop kernels that follow a kernel with programmatic dependent launch
  double ru_delta;     // reliable update when |r| < ru_delta * max |r| since the last one
  int ru_interval;     // ... or after this many iterations
  CGGraph* graphs;  // cached captured solver loops
  BatchPlan* batch;  // cached batched-solve workspace and graph (owned by the first context of a batch)
};

void free_batch_plan(sqcg_ctx* ctx);
// batched mixed-precision CG with per-RHS shifts sigma[] and tolerances tol[] (RHS in lattice order);
// b_shared: all RHS of lattice k solve for the one source b[k] (batched.cu)
int batched_solve(int nctx, sqcg_ctx* const* ctx, const int* nrhs, const double* sigma, const double* tol,
                  const void* const* b, int b_shared, void* const* x, int max_iter, sqcg_info* info);

// ---------------------------------------------------------------------------
// launchers (defined in dslash.cu / blas.cu / layout.cu)
// ---------------------------------------------------------------------------
enum DslashEpi {
  EPI_PLAIN = 0,          // out = D in
  EPI_NORMAL = 1,         // out = sigma*y - D in
  EPI_NORMAL_DOT = 2,     // out = sigma*y - D in, reduce Re<y, out>
  EPI_TRUE_RESID = 3,     // out = b - sigma*y + D in (b, y FP64), reduce |out|^2
  EPI_SR_DOTS = 4,        // single-reduction CG: s = sigma*r - D in (r = y, q = y3 on the output parity);
                          // three sums Re<r,s>, Re<r,q>, |r|^2 (after a reliable update)
  EPI_SR_DOTS2 = 5,       // the same without q: sums Re<r,s> and |r|^2; Re<r,q> comes from the update kernel
};

struct DslashLaunch {
  int out_parity;
  int prec;      // SQCG_F64 / SQCG_F32: precision of links, in and the arithmetic
  int out_prec;  // precision of out (differs from prec only for EPI_TRUE_RESID)
  int epi;
  const void* in;
  void* out;
  void* out2;        // EPI_TRUE_RESID: optional second copy of out (same precision as out)
  const void* y;     // EPI_NORMAL*: vector on out_parity (precision prec); EPI_TRUE_RESID: FP64 x
  const void* y3;    // EPI_SR_DOTS: q on out_parity
  const void* b;     // EPI_TRUE_RESID: FP64 right-hand side
  double sigma;
  const double* sigma_dev;  // if non-null, sigma is read from here (solver state)
  int gate;
  int fin;
  int pdl;  // the kernel before it on the stream is a kernel: launch with programmatic dependent launch
};

int launch_dslash(sqcg_ctx* ctx, const DslashLaunch& L, cudaStream_t s);

int launch_cg_update_x(sqcg_ctx* ctx, int mixed, double2* x, cudaStream_t s);
int launch_loop_control(sqcg_ctx* ctx, cudaStream_t s);
// blocks of the streaming BLAS kernels (one wave on every SM; each thread loops over sites)
int blas_grid(sqcg_ctx* ctx);
// Launch kern<<<grid, block, smem, s>>>(args...), with the programmatic-serialization attribute when pdl
// is set (the kernel must then call pdl_wait() before it reads what the kernel before it wrote).
template <typename... KArgs, typename... Args>
cudaError_t launch_kernel(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                          Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

int launch_finish(sqcg_ctx* ctx, int nblocks, int fin, int gate, cudaStream_t s, bool pdl = false);
// the same for float-float partials (ffs slots; the FP32 Dslash's EPI_NORMAL_DOT, k_ms_update<float>)
int launch_finish_ffs(sqcg_ctx* ctx, int nblocks, int fin, int gate, cudaStream_t s, bool pdl = false);
// persistent single-reduction mixed CG (cg_persistent.cu): grid size (0: unavailable) and one launch,
// which runs iterations until the state asks for a reliable update or the solve ends
int persistent_grid(sqcg_ctx* ctx);
int launch_sr_persistent(sqcg_ctx* ctx, int max_steps, cudaStream_t s);
int launch_finish2(sqcg_ctx* ctx, int nblocks, int fin, int gate, cudaStream_t s);
// the single-reduction step's finisher: sums <r,s> = partials[0, n), <r,q> = partials[coff, coff + cn),
// |r|^2 = partials[2n, 3n)
int launch_finish_sr(sqcg_ctx* ctx, int nblocks, int coff, int cn, int gate, cudaStream_t s, bool pdl = false);
// offset of the update kernel's partials of <r_new, q> in ctx->partials
inline int sr_update_partials(const sqcg_ctx* ctx) { return 3 * ctx->max_blocks; }
int launch_cg_xpay(sqcg_ctx* ctx, int mixed, cudaStream_t s);
// single-reduction mixed CG: p = r + beta p, q = s + beta q, xh += alpha p, r -= alpha q (s in Ap32), with
// the WHILE-loop control of the captured loop in one thread
// (after_kernel: a kernel precedes it on the stream; it then launches with programmatic dependent launch)
int launch_sr_update(sqcg_ctx* ctx, cudaStream_t s, bool after_kernel = false);
// x += xh (FP64 += FP32), xh = 0
int launch_flush_partial_x(sqcg_ctx* ctx, double2* x, int gate, cudaStream_t s);
int launch_norm2_f64(sqcg_ctx* ctx, const double2* v, int fin, cudaStream_t s);
int launch_scale_copy_f64(sqcg_ctx* ctx, const double2* src, double2* dst, double a, cudaStream_t s);

int launch_ms_update_x(sqcg_ctx* ctx, int mixed, int nshift, double2* const* x, cudaStream_t s);

int launch_ms_xpay(sqcg_ctx* ctx, int mixed, int nshift, double2* const* x, cudaStream_t s);
// shift-aware reliable update of the multi-shift loop: Re<a, b>, |b - z a|^2 and |a|^2 (FP64 vectors) into
// st->ms_sums; then r <- rt (FP64, or FP32 in mixed mode) with p_s += zeta_s (rt - r) for every direction
// still moving
int launch_ms_ru_sums(sqcg_ctx* ctx, const double2* a, const double2* b, double z, cudaStream_t s);
int launch_ms_ru_fix(sqcg_ctx* ctx, int mixed, int nshift, const void* rt, int rt_prec, cudaStream_t s);

// float-float Dslash (dslash_ff.cu): in and out_ff are float4 [3][Vh] (re_hi, re_lo, im_hi, im_lo);
// true_resid: out32 (FP32) = b - sigma x + D in with |.|^2 reduced in FP64 (x, b FP64)
struct FFLaunch {
  int out_parity;
  int true_resid;
  const void* in;
  void* out_ff;
  void* out32;
  const void* x;
  const void* b;
  double sigma;
  const double* sigma_dev;
  int gate;
  int fin;
};
int launch_dslash_ff(sqcg_ctx* ctx, const FFLaunch& L, cudaStream_t s);
int launch_split_ff(const double2* in, float4* out, size_t n, cudaStream_t s);
// x += xh (if xh), xh = 0, xff = float-float copy of x
int launch_flush_split(sqcg_ctx* ctx, double2* x, float2* xh, float4* xff, int gate, cudaStream_t s);

int layout_load_links(sqcg_ctx* ctx, const double* fat, const double* lng, int opts);
// the same from links already in device memory (host order [V][4][3][3] complex)
int layout_load_links_device(sqcg_ctx* ctx, const double* fat, const double* lng, int opts);
int layout_pack_spinor(sqcg_ctx* ctx, int prec, const double* host, void* dev);
int layout_unpack_spinor(sqcg_ctx* ctx, int prec, const void* dev, double* host);
int layout_convert(sqcg_ctx* ctx, int from_prec, const void* src, int to_prec, void* dst, cudaStream_t s);

int ensure_workspace(sqcg_ctx* ctx);
void free_workspace(sqcg_ctx* ctx);
void free_graphs(sqcg_ctx* ctx);

inline int grid_for(int n, int threads) { return (n + threads - 1) / threads; }
