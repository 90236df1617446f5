/*
 * sqcg.h -- C ABI of the GB300 improved-staggered CG library.
 *
 * The library solves the even-odd preconditioned improved-staggered normal
 * equation (sigma - D_eo D_oe) x = b, sigma = 4 m^2, and its multi-shift form,
 * on one CUDA GPU (the single- and multi-mass staggered CG of arXiv:1611.00728,
 * Sec. 3; the benchmarked double-precision multi-mass CG of Sec. 4). D is the
 * staggered Dslash with fat one-hop and long (Naik) three-hop links (Sec. 3,
 * the generated "staggered dslash" kernel):
 *
 *   (D psi)(n) = sum_mu [  s F_mu(n) psi(n+mu) - s' F_mu(n-mu)^+ psi(n-mu)
 *                        + s L_mu(n) psi(n+3mu) - s' L_mu(n-3mu)^+ psi(n-3mu) ]
 *
 * s, s' = eta_mu * boundary sign of the forward hop (eta_x = 1,
 * eta_y = (-1)^x, eta_z = (-1)^(x+y), eta_t = (-1)^(x+y+z); -1 for a forward
 * hop across the last time slice when the time direction is antiperiodic).
 *
 * Conventions shared by every call:
 *  - Lattice extents dims = {Lx, Ly, Lz, Lt}, all even and >= 4. Sites are
 *    numbered lex = x + Lx*(y + Ly*(z + Lz*t)); parity = (x+y+z+t) mod 2;
 *    V = Lx*Ly*Lz*Lt, Vh = V/2.
 *  - Host gauge fields: double [V][4][3][3][2] (complex, row-major 3x3,
 *    direction order x, y, z, t, forward links only: the standard MILC storage
 *    the paper contrasts with its 8-way layout, Sec. 3).
 *  - Host colour vectors on one parity: double [Vh][3][2], sites of that parity
 *    in increasing lex order (index lex/2).
 *  - Device colour vectors on one parity (what sqcg_dslash and the solvers
 *    take): structure of arrays [3 colour][Vh] of complex, i.e. double2
 *    (SQCG_F64) or float2 (SQCG_F32); 16-byte (F64) / 8-byte (F32) aligned.
 *    The caller allocates and owns them (e.g. torch tensors).
 *  - All work is queued on the context's CUDA stream (set at creation or by
 *    sqcg_set_stream). Calls that return results to the host (solver info)
 *    synchronise that stream before returning.
 *  - Return value: SQCG_OK (0) or a negative SQCG_ERR_* code; sqcg_strerror
 *    gives a message. Nothing aborts the process and no kernel traps.
 *  - A context is not thread-safe: one host thread at a time per context.
 *  - Solver loops run on the device as one CUDA graph launch (conditional
 *    WHILE/IF nodes). With the environment variable SQCG_LAUNCH_MODE=eager
 *    every solver (single-mass, multi-shift with its refinement, batched,
 *    flexible CG) launches the same kernels one at a time with a host round
 *    trip per iteration instead (kernel-level profilers do not list kernels
 *    inside conditional graph nodes); results are identical.
 */
#ifndef SQCG_H
#define SQCG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define SQCG_OK 0
#define SQCG_ERR_INVALID_ARG (-1)    /* odd or too small extent, null pointer, bad flag, tol <= 0 ... */
#define SQCG_ERR_CUDA (-2)           /* a CUDA runtime call failed */
#define SQCG_ERR_NOT_CONVERGED (-3)  /* max_iter reached; x holds the last iterate, info is filled */
#define SQCG_ERR_BREAKDOWN (-4)      /* <p, A p> <= 0, or NaN/Inf in a reduction */
#define SQCG_ERR_RECON_REJECTED (-5) /* 12-real long links requested but the links fail the test */
#define SQCG_ERR_NO_LINKS (-6)       /* operator used before sqcg_load_links */
#define SQCG_ERR_NO_MEMORY (-7)      /* device allocation failed */
#define SQCG_ERR_SCRATCH_TOO_SMALL (-8) /* lattice larger than the fixed scratch of sqcg_normal_op_noalloc */

/* ---- sqcg_create flags ---- */
#define SQCG_ANTIPERIODIC_T 1 /* extra -1 on forward hops across the last time slice */
#define SQCG_PHASES_FOLDED 2  /* links passed to sqcg_load_links already carry eta and the boundary sign */

/* ---- sqcg_load_links options ---- */
#define SQCG_RECON12_LONG 1 /* FP32 long links as 2 rows (12 reals), row 3 rebuilt on the fly */
#define SQCG_EIGHT_WAY 2    /* FP32 copy also stores the backward links -F(n-mu)^+, -L(n-3mu)^+ at n */

/* ---- precisions ---- */
#define SQCG_F64 0
#define SQCG_F32 1
/* Float-float ("double-single"): each real is an unevaluated sum hi + lo of
 * two floats (about 48 significand bits). A device colour vector is
 * [3][Vh] of float4 (re_hi, re_lo, im_hi, im_lo), 16 bytes per complex like
 * SQCG_F64, 16-byte aligned. The Dslash in this arithmetic runs on the FP32
 * pipe with error-free products and sums (relative error of order 1e-14,
 * tested against the FP64 oracle at 1e-12); on the GB300, whose FP64 FMA rate
 * is 1/64 of FP32, it is bound by memory instead of FP64 arithmetic. Accepted
 * by sqcg_dslash, sqcg_pack_spinor, sqcg_unpack_spinor, sqcg_spinor_bytes and
 * sqcg_set_update_arithmetic. Not in the paper, whose kernels are FP64. */
#define SQCG_FF 2

/* ---- solver modes ---- */
#define SQCG_MODE_F64 0   /* everything in FP64 */
#define SQCG_MODE_MIXED 1 /* FP32 Dslash and vectors; FP64 x and scalars; grid sums in float-float;
                             true residuals of the reliable updates in float-float (SQCG_FF, default) or
                             FP64 arithmetic, summed in FP64 */
/* Multi-shift only: OR-ed into the mode of sqcg_multishift_cg_solve (and
 * sqcg_rational_apply), shift-aware reliable updates of the shared Krylov loop.
 * Each time the base residual has fallen by the reliable-update factor (1e-3
 * by default), the loop pauses and, in FP64: r_0 = b - A_0 x_0 replaces the
 * iterated base residual; every shift still iterating gets its true residual
 * r_s = b - A_s x_s, the least-squares factor zeta'_s = Re<r_0, r_s> / |r_0|^2
 * and the collinearity loss |r_s - zeta'_s r_0| / |b|. Where that loss is at
 * most tol_s / 2 the shift continues from zeta'_s (its zeta recurrence
 * rescaled, its stopping threshold lowered by the loss, which later iterations
 * of the shared space do not remove); otherwise it continues unchanged and is
 * refined after the loop as without the flag. The losses are kept for
 * sqcg_multishift_ru_record. Not in the paper (its multi-mass CG is FP64). */
#define SQCG_MS_SHIFT_RU 0x10
/* Multi-shift only, OR-ed into the mode: no reliable updates in the shared
 * loop. Without this flag (and without SQCG_MS_SHIFT_RU) the mixed multi-shift
 * takes base reliable updates: the same pauses, but only the base residual is
 * recomputed (with the context's update arithmetic, float-float by default)
 * and replaces the iterated one, every moving direction taking the change; no
 * shift's residual is formed and no zeta changes. Either way every shift is
 * then checked and refined. The FP64 mode has no reliable updates unless
 * SQCG_MS_SHIFT_RU asks for them. */
#define SQCG_MS_NO_RU 0x20

typedef struct sqcg_ctx sqcg_ctx; /* opaque, library-owned */

typedef struct {
  int iters;             /* CG iterations (Dslash pairs in the Krylov loop) */
  int reliable_updates;  /* FP64 true-residual recomputations inside the loop */
  int status;            /* SQCG_OK or SQCG_ERR_* for this system */
  double true_rel_resid; /* |b - A x| / |b| recomputed in FP64 from the returned x */
  double seconds;        /* wall time of the solve on the host, including the final sync */
  int launches;          /* kernels this call launched (including gated-off ones in a captured loop) */
  int fallback;          /* sqcg_fcg_solve_nn only: 1 if plain CG took over from the flexible CG */
} sqcg_info;

/* Create a context for one lattice geometry. dims: 4 extents, all even and
 * >= 4. flags: SQCG_ANTIPERIODIC_T | SQCG_PHASES_FOLDED. cuda_stream: a
 * cudaStream_t (NULL = legacy default stream). On success *out owns device
 * memory until sqcg_destroy. Errors: INVALID_ARG, CUDA. */
int sqcg_create(const int dims[4], int flags, void* cuda_stream, sqcg_ctx** out);

/* Free everything the context owns (device links, workspace, graphs). NULL is a no-op. */
int sqcg_destroy(sqcg_ctx* ctx);

/* Change the stream later calls queue their work on. */
int sqcg_set_stream(sqcg_ctx* ctx, void* cuda_stream);

/* Reliable-update trigger of the mixed-precision solvers on this context: the
 * FP64 true residual is recomputed when the iterated |r| falls below
 * delta * (max |r| since the last update), or after `interval` iterations,
 * whichever comes first (0 < delta < 1, interval >= 1; defaults 0.001 and 100).
 * The batched solve uses the settings of its first context. The multi-shift
 * loop's reliable updates use delta only. */
int sqcg_set_reliable_update(sqcg_ctx* ctx, double delta, int interval);

/* Arithmetic of the true-residual recomputations (reliable updates and the
 * final convergence check) of the single-mass mixed-precision solve, and of the
 * mixed multi-shift loop's base reliable updates, on this context: SQCG_FF
 * (default; float-float Dslash from float-float copies of the FP64 links, the
 * sum b - sigma x + D x and the norm in FP64) or SQCG_F64 (the FP64 Dslash).
 * The FP64 solver mode, and the shift-aware updates (SQCG_MS_SHIFT_RU), always
 * use FP64. Not in the paper. */
int sqcg_set_update_arithmetic(sqcg_ctx* ctx, int prec);

/* Bytes of one device colour vector on one parity in precision prec (Vh * 3 * 2 * sizeof(real);
 * SQCG_FF: Vh * 3 * 16). */
int sqcg_spinor_bytes(const sqcg_ctx* ctx, int prec, size_t* bytes);

/* Load fat (one-hop) and long (three-hop) links from host memory in the host
 * gauge format above. The library folds eta and the boundary sign into its
 * copies unless the context has SQCG_PHASES_FOLDED, converts them to its
 * parity-split structure-of-arrays layout and keeps an FP64, an FP32 and a
 * float-float (SQCG_FF) copy on the device (owned by the context, replacing
 * earlier links). The host arrays
 * are only read during the call.
 * opts: SQCG_RECON12_LONG stores the FP32 copy of the long links as their
 * first two rows (the FP32 Dslash rebuilds the third); it is accepted only if
 * every long link is s * W with W in SU(3) and one global real |s| (checked to
 * 1e-12), else SQCG_ERR_RECON_REJECTED and nothing is loaded. The FP64 copy
 * and the fat links are always stored in full (the FP64 Dslash is bound by
 * FP64 arithmetic, which the reconstruction would add to).
 * SQCG_EIGHT_WAY additionally stores, for the FP32 copy, the daggered and
 * negated backward links at the site that uses them (the paper's 8-way gauge
 * storage, Sec. 3): every FP32 link read is then at the thread's own index, at
 * twice the FP32 link memory. Combined with SQCG_RECON12_LONG the backward
 * long links are stored as two rows too. */
int sqcg_load_links(sqcg_ctx* ctx, const double* fat, const double* lng, int opts);

/* Copy one host colour vector (parity order, complex double [Vh][3]) into a
 * device vector of precision prec (rounded to nearest for SQCG_F32; for
 * SQCG_FF hi = fl32(v), lo = fl32(v - hi)). */
int sqcg_pack_spinor(sqcg_ctx* ctx, int prec, const double* host, void* dev);

/* Copy a device vector of precision prec back to host parity order (complex
 * double [Vh][3]; SQCG_FF: hi + lo in FP64). Synchronises the stream. */
int sqcg_unpack_spinor(sqcg_ctx* ctx, int prec, const void* dev, double* host);

/* out = D in on the sites of parity out_parity, reading in on the other
 * parity (paper Sec. 3, staggered dslash). in and out are device vectors of
 * precision prec; they must not alias. Asynchronous on the stream. */
int sqcg_dslash(sqcg_ctx* ctx, int out_parity, int prec, const void* in, void* out);

/* y = (sigma - D_eo D_oe) x on the even sites, FP64 or FP32 device vectors
 * (x, y must not alias). Asynchronous. */
int sqcg_normal_op(sqcg_ctx* ctx, double sigma, int prec, const void* x, void* y);

/* Same result as sqcg_normal_op, but this call allocates no device memory.
 * The paper has no counterpart: it exists for callers that cannot call
 * cudaMalloc when they apply the operator, such as host applications that give
 * all device memory to their own allocator or pool up front (a new cudaMalloc
 * would fail or break their budget) and latency-bound loops that cannot accept
 * an allocation, which may synchronise the device. sqcg_normal_op keeps its
 * intermediate D_oe x in the context's workspace, which is allocated on first
 * use; this call keeps it in one fixed 8 MiB array compiled into the library
 * (held on every GPU that loads the library until the process exits), so the
 * lattice may have at most 174762 sites per parity in SQCG_F64 and 349525 in
 * SQCG_F32; larger lattices get SQCG_ERR_SCRATCH_TOO_SMALL. The context must
 * already exist with its links loaded; x and y are the caller's device vectors
 * as for sqcg_normal_op. The first call on each device looks up the device
 * address of that array (cudaGetSymbolAddress, with that device current); make
 * that first call before any stream capture. Every call on a device shares the
 * array and it keeps the last call's contents (nothing in it has to start at
 * zero: each call overwrites what it reads); calls that overlap on the GPU
 * (other streams or host threads) race on it. Asynchronous on the stream. */
int sqcg_normal_op_noalloc(sqcg_ctx* ctx, double sigma, int prec, const void* x, void* y);

/* Solve (4 mass^2 - D_eo D_oe) x = b on the even sites by CG (paper Sec. 3,
 * single-mass CG). b, x: FP64 device vectors; x holds the initial guess on
 * entry (zero it for x0 = 0) and the solution on return. A zero guess is
 * detected (|x0| = 0) and its initial residual is b itself, with no FP64
 * operator application; any other guess starts from r = b - A x0 in FP64.
 * Stops when the FP64
 * true relative residual |b - A x|/|b| <= tol, or after max_iter iterations
 * (SQCG_ERR_NOT_CONVERGED, x = last iterate). mode: SQCG_MODE_F64 or
 * SQCG_MODE_MIXED (FP32 Krylov vectors with reliable updates). The FP64 mode
 * runs as one CUDA graph launch; the mixed mode too (eight steps per WHILE
 * pass), except on lattices of at most five 128-site tiles per SM, where one
 * persistent cooperative kernel runs each segment between reliable updates
 * (environment SQCG_PERSISTENT=0 or 1 forces one form; SQCG_LAUNCH_MODE=eager
 * launches the graph's kernels one at a time, for profilers; SQCG_PDL=0, read
 * when a context is created, launches without programmatic dependent launch).
 * A persistent grid barrier that waits past its bound ends the solve with
 * SQCG_ERR_CUDA. info may be NULL. Synchronises the stream. */
int sqcg_cg_solve(sqcg_ctx* ctx, double mass, const void* b, void* x, double tol, int max_iter,
                  int mode, sqcg_info* info);

/* Solve (shifts[s] - D_eo D_oe) x[s] = b for nshift shifts at once (1 <= nshift
 * <= 32) from one Krylov space (paper Sec. 3-4, the multi-mass CG; shifts[s]
 * plays the role of 4 m_s^2, all >= 0). The smallest shift is the base system;
 * the shifted systems follow from collinear residuals r_s = zeta_s r with the
 * FP64 zeta/alpha/beta recurrences of Jegerlehner (hep-lat/9612014). b: FP64
 * device vector; x: host array of nshift distinct FP64 device vectors
 * (overwritten; the multi-shift start is x_s = 0); tol[s]: per-shift
 * tolerance on the FP64 true relative residual. A shift stops when its
 * iterated residual |zeta_s| |r| / |b| <= tol[s]. Each x_s is then checked on
 * its FP64 true residual; where that is above tol[s] (expected with FP32
 * vectors) it is refined from x_s: in mixed mode all shifts together as one
 * batched mixed-precision CG (one right-hand side per shift, held in the
 * context's batched workspace), in FP64 mode by one CG per shift. mode:
 * SQCG_MODE_F64 or SQCG_MODE_MIXED, either optionally | SQCG_MS_SHIFT_RU (the
 * shift-aware reliable updates above; info[s].reliable_updates then also
 * counts the updates in which shift s continued from zeta'_s) or
 * | SQCG_MS_NO_RU (mixed mode without its base reliable updates).
 * info: NULL or an array of nshift (per-shift iterations including refinement,
 * status, true residual; seconds = whole call). Returns SQCG_OK when every
 * shift converged, else the first failing status. Synchronises the stream. */
int sqcg_multishift_cg_solve(sqcg_ctx* ctx, int nshift, const double* shifts, const void* b,
                             void* const* x, const double* tol, int max_iter, int mode,
                             sqcg_info* info);

/* The reliable updates of the last multi-shift solve on ctx (SQCG_MS_SHIFT_RU,
 * or the mixed mode's base updates). *nupdates = how many ran. For update
 * u < min(*nupdates, max_updates, 16): iter[u] = the loop iteration it followed,
 * base[u] = |r_0| / |b| (FP64 true base residual), loss[u * nshift + s] =
 * |r_s - zeta'_s r_0| / |b| for shift s in the order the caller passed them
 * (0 for the base system; NaN where not measured: a shift that had already
 * stopped, or every other shift in a base update). *nshift_out
 * = that solve's shift count; loss holds max_updates * nshift entries. iter, base
 * and loss may be NULL. Host-only: reads what the solve left. */
int sqcg_multishift_ru_record(const sqcg_ctx* ctx, int max_updates, int* nupdates, int* nshift_out, int* iter,
                              double* base, double* loss);

/* Rational-function application, the multi-mass CG's use inside RHMC evolution
 * (paper Sec. 4: su3_rhmc_hisq, about nine masses):
 *   out = a0 b + sum_s residues[s] (shifts[s] - D_eo D_oe)^-1 b,
 * from one multi-shift solve (sqcg_multishift_cg_solve rules: shifts >= 0, each
 * shift solved to FP64 true relative residual tol, mixed mode refined as
 * needed), combined in FP64. For a rational approximation
 * r(x) = a0 + sum_s a_s / (x + beta_s) of a function of M^+M = 4 m^2 - D_eo D_oe
 * the shifts are 4 m^2 + beta_s. b, out: FP64 device vectors (distinct). The
 * per-shift solutions are kept in library-owned buffers (freed with the
 * context). info: NULL or nshift entries. Synchronises the stream. */
int sqcg_rational_apply(sqcg_ctx* ctx, int nshift, const double* shifts, const double* residues, double a0,
                        const void* b, void* out, double tol, int max_iter, int mode, sqcg_info* info);

/* Batched CG: solve (4 mass[k]^2 - D_eo D_oe) x = b for nrhs[k] right-hand
 * sides on each of nctx lattices (1 <= nctx <= 16, sum of nrhs <= 256) in one
 * device-side loop, mixed precision (FP32 Dslash and Krylov vectors, FP64 x,
 * reductions and reliable updates). This applies the paper's single-mass CG
 * (Sec. 3) to many sources at once; batching is not in the paper. Each link is
 * loaded once per block of W right-hand sides. W (1..16), the RHS per thread,
 * the site-block size, the warp shape and the shared-memory carveout are picked on the first
 * call for a given set of lattices by timing the multi-RHS Dslash (cached per
 * process, and in the file named by the environment variable SQCG_TUNE_CACHE
 * if set; SQCG_TUNE_VERBOSE=1 prints each timed candidate to stderr), unless
 * sqcg_batched_pin_tuning has fixed them.
 * ctx[k]: distinct contexts with links loaded, all on the current device; the
 * work runs on ctx[0]'s stream. b[k], x[k]: device arrays of nrhs[k]
 * consecutive FP64 device vectors ([nrhs][3][Vh] complex double); x[k] holds
 * the initial guesses and receives the solutions (when every guess is zero the
 * initial residuals are the b[k] themselves; otherwise r = b - A x0 in FP64 for
 * all). tol: FP64 true relative residual target for every RHS. info: NULL or
 * sum(nrhs) entries, lattice-major. Workspace (per site and RHS: 96 bytes of
 * FP32 vectors, for an RHS count rounded up to even, and 48 bytes of FP64) is
 * cached with ctx[0] for repeated calls with the same arguments. Returns
 * SQCG_OK when every RHS converged, else the first failing status.
 * Synchronises the stream. */
int sqcg_cg_solve_batched(int nctx, sqcg_ctx* const* ctx, const int* nrhs, const double* mass,
                          const void* const* b, void* const* x, double tol, int max_iter,
                          sqcg_info* info);

/* ---- learned gauge-covariant preconditioner and flexible CG ----
 * Not in the paper: a learned preconditioner for a flexible CG built around
 * the paper's single-mass CG (Sec. 3). The network N has three
 * parallel-transport convolution layers over the fat links (channels
 * 1 -> 8 -> 8 -> 1; taps: self and the 8 one-hop neighbours; complex weights
 * that mix channels only, stored in BF16 with FP32 accumulation), a gate
 * h <- h sigmoid(a |h|^2 + b) after layers 1 and 2, and an input scaled to
 * unit RMS with the output scaled back, so N(c r) = c N(r). It is exactly
 * gauge covariant. Parameters (SQCG_NN_NPARAMS floats, host layout):
 *   [0, 144)     layer 1 weights [tap][out 8][in 1][re, im]
 *   [144, 1296)  layer 2 weights [tap][out 8][in 8][re, im]
 *   [1296, 1440) layer 3 weights [tap][out 1][in 8][re, im]
 *   [1440, 1472) gate 1 a[8], b[8], gate 2 a[8], b[8]
 * taps: 0 self, 1 + 2 mu = F_mu(n) h(n + mu), 2 + 2 mu = F_mu(n - mu)^+ h(n - mu),
 * with F the fat links carrying the staggered phases and boundary sign.
 * Vectors given to these calls are FP32 device vectors on the even sites. */
typedef struct sqcg_nn sqcg_nn;
#define SQCG_NN_NPARAMS 1472

/* Network bound to ctx (its links and geometry); parameters start at zero.
 * After sqcg_destroy(ctx) the only valid call on its networks is
 * sqcg_nn_destroy, which does not touch the context (it waits for the whole
 * device before freeing the network's buffers). */
int sqcg_nn_create(sqcg_ctx* ctx, sqcg_nn** out);
int sqcg_nn_destroy(sqcg_nn* nn);
int sqcg_nn_nparams(void);
/* Copy parameters in (host floats, layout above; resets the optimiser state) or
 * out (bf16_rounded != 0: the weights as the forward pass uses them). */
int sqcg_nn_set_params(sqcg_nn* nn, const float* params);
int sqcg_nn_get_params(const sqcg_nn* nn, float* params, int bf16_rounded);
/* z = N(r). Asynchronous. */
int sqcg_nn_apply(sqcg_nn* nn, const void* r, void* z);
/* Arithmetic of the 8 -> 8 layer's channel mixing in inference (sqcg_nn_apply and the flexible
 * CG): SQCG_NN_MIX_FP32 (default; FP32 on the CUDA cores, the results of the training forward pass)
 * or SQCG_NN_MIX_BF16 (warp-level tensor-core MMAs, m16n8k16: the transported activations rounded
 * to BF16, the BF16 weights as they are, FP32 accumulation; a relative change of the layer's output
 * of order 2^-9). Training always uses FP32. A captured flexible-CG loop is recaptured after a
 * change. SQCG_ERR_INVALID_ARG for another mode. */
#define SQCG_NN_MIX_FP32 0
#define SQCG_NN_MIX_BF16 1
int sqcg_nn_set_mixing(sqcg_nn* nn, int mode);
/* Training loss of one (residual r, error e) pair, d = N(r) - e,
 * A = sigma - D_eo D_oe, in the norm chosen by sqcg_nn_set_loss:
 *   1 (default): L = <d, A d> / <e, r>  (A-norm of the error relative to that of e)
 *   2:           L = <A d, A d> / <r, r> (A^2-norm: |A N(r) - r|^2 / |r|^2, since A e = r)
 * and its gradient (host floats, parameter layout, complex entries as
 * dL/dRe + i dL/dIm). Synchronises. */
int sqcg_nn_set_loss(sqcg_nn* nn, int norm);
int sqcg_nn_loss_grad(sqcg_nn* nn, double sigma, const void* r, const void* e, double* loss, float* grad);
/* Adam (lr, beta1 0.9, beta2 0.999) over `steps` mini-batches of `batch` pairs
 * drawn from npairs pairs (r, e: npairs consecutive FP32 even vectors each)
 * with a seeded generator. loss_first / loss_last: mean batch loss of the
 * first and last step. Synchronises. */
int sqcg_nn_train(sqcg_nn* nn, double sigma, int npairs, const void* r, const void* e, int steps, int batch,
                  double lr, unsigned long long seed, double* loss_first, double* loss_last);
/* One training pair from a CG iterate: r = b - (sigma - D_eo D_oe) x_k in FP64,
 * e = x_star - x_k, both rounded to FP32 (b, x_k, x_star: FP64 device vectors). */
int sqcg_make_training_pair(sqcg_ctx* ctx, double sigma, const void* b, const void* x_k, const void* x_star,
                            void* r_out, void* e_out);
/* Flexible CG (Notay's FCG with one stored direction, Polak-Ribiere beta)
 * preconditioned by nn, FP32 vectors with FP64 x and reliable updates, for
 * (4 mass^2 - D_eo D_oe) x = b (FP64 device vectors; x = initial guess in,
 * solution out). On breakdown (<p,Ap> <= 0, <z,r> <= 0, non-finite) or
 * without convergence it hands over to the mixed-precision CG from the
 * current iterate (info->fallback = 1), which also confirms the answer on the
 * FP64 true residual. nn must be bound to ctx. The captured solver loop is
 * kept with nn and reused while b, x and the context's links stay the same
 * (the weights and the mass are read on the device, so they may change).
 * A zero initial guess starts from r = b. Synchronises. */
int sqcg_fcg_solve_nn(sqcg_ctx* ctx, sqcg_nn* nn, double mass, const void* b, void* x, double tol, int max_iter,
                      sqcg_info* info);

/* ---- HISQ link construction (the action of the paper's benchmark application, Sec. 4:
 * su3_rhmc_hisq; construction of Follana et al., hep-lat/0610092). Thin links U
 * -> V = smear(U, level1) -> W = V (V^+ V)^(-1/2) (U(3) projection) ->
 * fat = smear(W, level2), long = naik W_mu(n) W_mu(n+mu) W_mu(n+2mu).
 * smear(X)_mu(n) = one_link X_mu(n) + three_staple (sum of the 6 3-link staples)
 *   + five_staple (24 5-link) + seven_staple (48 7-link) + lepage (6 5-link
 *   staples that step twice in the same direction and sign), every staple
 *   running from n to n+mu through the other directions.
 * Coefficients are for unphased links (periodic in every direction); the
 * staggered phases and the time-boundary sign are applied when the result is
 * loaded. Everything in FP64. */
typedef struct {
  double one_link, three_staple, five_staple, seven_staple, lepage;
} sqcg_smear_level;
typedef struct {
  sqcg_smear_level level1, level2;
  double naik;
} sqcg_hisq_coeffs;
/* NULL coefficients mean the HISQ values: level1 = fat7 (1/8, 1/16, 1/64,
 * 1/384, 0), level2 = (1, 1/16, 1/64, 1/384, -1/8), naik = -1/24. The level-2
 * one-link value follows from tree-level improvement of the free dispersion
 * (fat + 3 naik = 1 and fat + 27 naik = 0 for unit thin links). */

/* Device workspace sqcg_hisq_smear needs for this lattice (0 for bad dims). */
size_t sqcg_hisq_workspace_bytes(const int dims[4]);

/* Thin -> fat, long on the device. thin, fat, lng: device arrays in the host
 * link order [V][4][3][3] complex double (lex sites, directions x, y, z, t);
 * fat may alias thin (thin is consumed first), lng must not alias either.
 * workspace: device memory of at least sqcg_hisq_workspace_bytes (caller
 * owned, 16-byte aligned). Work goes on `stream` (a cudaStream_t, NULL =
 * default); the call synchronises it. Returns SQCG_ERR_BREAKDOWN when a
 * level-1 link is singular or non-finite (the U(3) projection is undefined);
 * the outputs are then not meaningful. */
int sqcg_hisq_smear(const int dims[4], const void* thin, void* fat, void* lng, const sqcg_hisq_coeffs* coeffs,
                    void* workspace, size_t workspace_bytes, void* stream);

/* HISQ links from host thin links, installed as the context's links as by
 * sqcg_load_links (opts: SQCG_EIGHT_WAY; SQCG_RECON12_LONG is checked as
 * usual and fails for HISQ long links, which are U(3), not SU(3) up to a real
 * scale). The context must not have SQCG_PHASES_FOLDED. fat_out, lng_out:
 * NULL or host arrays [V][4][3][3] complex double that receive the unphased
 * links. Allocates and frees its own device memory; synchronises the stream. */
int sqcg_hisq_load_links(sqcg_ctx* ctx, const double* thin, const sqcg_hisq_coeffs* coeffs, int opts,
                         double* fat_out, double* lng_out);

/* RHS block width W and site-block size T chosen by the autotuner for the
 * batched solve cached with ctx (the ctx passed first to the last batched call). */
int sqcg_batched_tuning(const sqcg_ctx* ctx, int* W, int* T);

/* The full FP32 Dslash configuration of that batched solve: RHS block width W,
 * right-hand sides per thread WT (W / WT thread groups per site block), site
 * block T, shared-memory carveout in percent (-1 = the driver's default) and
 * warp_sites, the consecutive sites one warp covers: 32 (one RHS group per
 * warp), or 16 (two RHS groups per warp, whose link reads from shared memory
 * are then one broadcast access for both). Any output pointer may be NULL. */
int sqcg_batched_tuning_ex(const sqcg_ctx* ctx, int* W, int* WT, int* T, int* carve, int* warp_sites);

/* Pin the FP32 Dslash configuration of batched solves planned from now on in
 * this process instead of autotuning it (plans already cached with a context
 * keep theirs); W = 0 returns to autotuning. Requirements: W in {1, 2, 4, 8,
 * 12, 16}; WT in {1, 2, 4}, WT <= W and dividing W; T a multiple of 32 in [32, 128] with
 * T * W / WT <= 512; carve -1 or 0..100; warp_sites 32 (or 0, the same) or 16
 * with W / WT even. SQCG_ERR_INVALID_ARG otherwise (nothing changes).
 * Thread-safe. */
int sqcg_batched_pin_tuning(int W, int WT, int T, int carve, int warp_sites);

const char* sqcg_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* SQCG_H */
