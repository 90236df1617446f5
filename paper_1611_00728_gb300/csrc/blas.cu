// Fused BLAS-1 kernels of the CG iteration (the vector updates and global
// reductions around the Dslash; paper Sec. 4 notes that multi-mass CG is even
// more bandwidth bound than CG because of them). Each kernel streams its
// vectors once; norms and dot products are accumulated in FP64 and reduced
// deterministically (warp shuffle -> block partial -> one finisher block that
// adds the partials in index order), and the scalar CG step runs in that
// finisher.
#include "solver_device.cuh"
#include "sqcg_internal.cuh"

namespace {

constexpr int kThreads = 256;

template <typename R> struct V2;
template <> struct V2<double> { typedef double2 T; };
template <> struct V2<float> { typedef float2 T; };

// x += alpha p (x FP64); r -= alpha Ap; reduce |r|^2 -> FIN_UPDATE. Held to 5 blocks of 256 a SM: the
// one-wave grid of blas_grid() is sized by this kernel's FP32 instance, and the FP64 one (64 registers
// unbounded) would run it as 1.25 waves.
template <typename R>
__global__ void __launch_bounds__(kThreads, 5)
k_cg_update(double2* __restrict__ x, typename V2<R>::T* __restrict__ r, const typename V2<R>::T* __restrict__ p,
            const typename V2<R>::T* __restrict__ Ap, int Vh, SolverState* st, double* partials) {
  typedef typename V2<R>::T R2;
  if (!gate_open(st, GATE_ITER)) return;
  const double alpha = st->alpha;
  const R ra = (R)alpha;
  double nrm = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Vh; i += gridDim.x * blockDim.x) {
    // all loads before any store: the colour offsets of one array are not provably distinct,
    // so interleaved stores would hold back the next colour's loads
    R2 pc[3], apc[3], rc[3];
    double2 xc[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t k = (size_t)c * Vh + i;
      pc[c] = p[k];
      apc[c] = Ap[k];
      rc[c] = r[k];
      xc[c] = x[k];
    }
    R part = R(0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t k = (size_t)c * Vh + i;
      xc[c].x = fma(alpha, (double)pc[c].x, xc[c].x);
      xc[c].y = fma(alpha, (double)pc[c].y, xc[c].y);
      x[k] = xc[c];
      rc[c].x = fma(-ra, apc[c].x, rc[c].x);
      rc[c].y = fma(-ra, apc[c].y, rc[c].y);
      r[k] = rc[c];
      part = fma(rc[c].x, rc[c].x, fma(rc[c].y, rc[c].y, part));
    }
    nrm += (double)part;
  }
  block_partial(nrm, partials);
}

// p = r + beta p
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_cg_xpay(const typename V2<R>::T* __restrict__ r, typename V2<R>::T* __restrict__ p, int Vh, const SolverState* st) {
  typedef typename V2<R>::T R2;
  if (!gate_open(st, GATE_ITER)) return;
  const R beta = (R)st->beta;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Vh; i += gridDim.x * blockDim.x) {
    R2 rc[3], pc[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      rc[c] = r[(size_t)c * Vh + i];
      pc[c] = p[(size_t)c * Vh + i];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      pc[c].x = fma(beta, pc[c].x, rc[c].x);
      pc[c].y = fma(beta, pc[c].y, rc[c].y);
      p[(size_t)c * Vh + i] = pc[c];
    }
  }
}

// Single-reduction CG update, one pass over five FP32 vectors (s = A r, written by the Dslash epilogue):
//   p = r + beta p,  q = s + beta q  (= A p),  xh += alpha p,  r -= alpha q,
// and the block partials of Re<r_new, q_new>, the next step's cross term (the next Dslash epilogue then
// reads only r). xh is the FP32 partial solution, flushed into the FP64 x at every reliable update.
// Skipped (uniformly) when the step before it asked for a reliable update or ended the solve. Held to
// the residency of k_cg_update (5 blocks of 256 a SM), which sizes the one-wave grid of blas_grid():
// with 64 registers it fit 4, and that grid ran as 1.25 waves.
__global__ void __launch_bounds__(kThreads, 5)
k_sr_update(float2* __restrict__ r, const float2* __restrict__ sv, float2* __restrict__ p, float2* __restrict__ q,
            float2* __restrict__ xh, int Vh, SolverState* st, double* cpart) {
  pdl_wait();
  const volatile SolverState* vs = st;
  if (vs->done || vs->need_update) return;  // uniform over the grid: the step did not complete
  const float alpha = (float)st->alpha, beta = (float)st->beta;
  float2 cross[1] = {make_float2(0.f, 0.f)};  // float-float, as the step's other sums
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Vh; i += gridDim.x * blockDim.x) {
    float2 rc[3], sc[3], pc[3], qc[3], xc[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {  // all loads before any store (see k_cg_update)
      const size_t k = (size_t)c * Vh + i;
      rc[c] = r[k];
      sc[c] = sv[k];
      pc[c] = p[k];
      qc[c] = q[k];
      xc[c] = xh[k];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t k = (size_t)c * Vh + i;
      pc[c].x = fmaf(beta, pc[c].x, rc[c].x);
      pc[c].y = fmaf(beta, pc[c].y, rc[c].y);
      qc[c].x = fmaf(beta, qc[c].x, sc[c].x);
      qc[c].y = fmaf(beta, qc[c].y, sc[c].y);
      xc[c].x = fmaf(alpha, pc[c].x, xc[c].x);
      xc[c].y = fmaf(alpha, pc[c].y, xc[c].y);
      rc[c].x = fmaf(-alpha, qc[c].x, rc[c].x);
      rc[c].y = fmaf(-alpha, qc[c].y, rc[c].y);
      p[k] = pc[c];
      q[k] = qc[c];
      xh[k] = xc[c];
      r[k] = rc[c];
    }
    float rq = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) rq = fmaf(rc[c].x, qc[c].x, fmaf(rc[c].y, qc[c].y, rq));
    cross[0] = ffs_add(cross[0], make_float2(rq, 0.f));
  }
  block_sum_ffs<1>(cross);
  if (threadIdx.x == 0) ffs_slots(cpart)[blockIdx.x] = cross[0];
}

// x += xh (the FP32 partial solution, added in FP64), xh = 0
__global__ void __launch_bounds__(kThreads)
k_flush_partial_x(double2* __restrict__ x, float2* __restrict__ xh, int n, const SolverState* st, int gate) {
  if (!gate_open(st, gate)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float2 h = xh[i];
    double2 v = x[i];
    v.x += (double)h.x;
    v.y += (double)h.y;
    x[i] = v;
    xh[i] = make_float2(0.f, 0.f);
  }
}

__global__ void __launch_bounds__(kThreads)
k_norm2_f64(const double2* __restrict__ v, int Vh, SolverState* st, double* partials, int fin) {
  double nrm = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Vh; i += gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double2 a = v[(size_t)c * Vh + i];
      nrm = fma(a.x, a.x, fma(a.y, a.y, nrm));
    }
  }
  block_partial(nrm, partials);
}

__global__ void __launch_bounds__(kThreads)
k_scale_copy_f64(const double2* __restrict__ src, double2* __restrict__ dst, double a, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 s = src[i];
  dst[i] = make_double2(a * s.x, a * s.y);
}

// ---------------------------------------------------------------------------
// multi-shift CG: the base r update with the x_s updates of all shifts, and
// the p_s updates. The shift scalars come from SolverState (FP64).
// ---------------------------------------------------------------------------
struct MSPtrs {
  double2* x[SQCG_MAX_SHIFTS];
  void* p[SQCG_MAX_SHIFTS];
};

// r -= alpha Ap (base), reduce |r|^2 -> FIN_MS_UPDATE
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_ms_update(typename V2<R>::T* __restrict__ r, const typename V2<R>::T* __restrict__ Ap, int Vh, SolverState* st,
            double* partials) {
  typedef typename V2<R>::T R2;
  if (!gate_open(st, GATE_ITER)) return;
  const R ra = (R)st->alpha;
  double nrm = 0.0;                             // FP64 vectors: FP64 partials
  float2 nrm_ff[1] = {make_float2(0.f, 0.f)};  // FP32 vectors: float-float partials
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Vh; i += gridDim.x * blockDim.x) {
    R2 rc[3], apc[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      rc[c] = r[(size_t)c * Vh + i];
      apc[c] = Ap[(size_t)c * Vh + i];
    }
    R part = R(0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      rc[c].x = fma(-ra, apc[c].x, rc[c].x);
      rc[c].y = fma(-ra, apc[c].y, rc[c].y);
      r[(size_t)c * Vh + i] = rc[c];
      part = fma(rc[c].x, rc[c].x, fma(rc[c].y, rc[c].y, part));
    }
    if constexpr (sizeof(R) == 4)
      nrm_ff[0] = ffs_add(nrm_ff[0], make_float2(part, 0.f));
    else
      nrm += (double)part;
  }
  if constexpr (sizeof(R) == 4) {
    block_sum_ffs<1>(nrm_ff);
    if (threadIdx.x == 0) ffs_slots(partials)[blockIdx.x] = nrm_ff[0];
  } else {
    block_partial(nrm, partials);
  }
}

// One pass over every shift's direction: x_s += alpha_s p_s (the old p_s; for
// every shift with an update this iteration, including one that just
// converged), then p_s = zeta_s r + beta_s p_s for shifts still iterating.
// Shift 0 is the base system: its direction is the base p = r + beta p.
// Runs while the loop goes on, and once more in the iteration that ends it.
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_ms_xpay(MSPtrs P, const typename V2<R>::T* __restrict__ r, typename V2<R>::T* __restrict__ p, int Vh,
          const SolverState* st) {
  typedef typename V2<R>::T R2;
  const volatile SolverState* vs = st;
  const int done = vs->done;
  if (done && !vs->ms_final) return;
  const int ns = st->nshift;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Vh; i += gridDim.x * blockDim.x) {
    R2 rc[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) rc[c] = r[(size_t)c * Vh + i];
    for (int j = 0; j < ns; ++j) {
      const int act = st->active[j];
      const bool upd_p = !done && (j == 0 || act == 1);  // the base direction moves while the loop runs
      if (!act && !upd_p) continue;
      R2* ps = (j == 0) ? p : static_cast<R2*>(P.p[j]);
      const double as = st->alpha_s[j];
      const R z = (j == 0) ? R(1) : (R)st->zeta[j];
      const R bs = (j == 0) ? (R)st->beta : (R)st->beta_s[j];
      double2* xs = P.x[j];
      R2 pc[3];
      double2 xc[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {  // loads before stores (see k_cg_update)
        pc[c] = ps[(size_t)c * Vh + i];
        if (act) xc[c] = xs[(size_t)c * Vh + i];
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const size_t k = (size_t)c * Vh + i;
        if (act) {
          xc[c].x = fma(as, (double)pc[c].x, xc[c].x);
          xc[c].y = fma(as, (double)pc[c].y, xc[c].y);
          xs[k] = xc[c];
        }
        if (upd_p) {
          R2 pn;
          pn.x = fma(bs, pc[c].x, z * rc[c].x);
          pn.y = fma(bs, pc[c].y, z * rc[c].y);
          ps[k] = pn;
        }
      }
    }
  }
}

// Shift-aware reliable update of the multi-shift loop (host-driven, a few times a solve; FP64 on
// FP64 vectors): the block partials of Re<a, b>, |b - z a|^2 and |a|^2 at partials[0, nb, 2 nb).
__global__ void __launch_bounds__(kThreads)
k_ms_ru_dots(const double2* __restrict__ a, const double2* __restrict__ b, double z, int Vh, double* partials) {
  double ab = 0.0, d2 = 0.0, aa = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Vh; i += gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double2 u = a[(size_t)c * Vh + i], v = b[(size_t)c * Vh + i];
      ab = fma(u.x, v.x, fma(u.y, v.y, ab));
      const double dx = fma(-z, u.x, v.x), dy = fma(-z, u.y, v.y);
      d2 = fma(dx, dx, fma(dy, dy, d2));
      aa = fma(u.x, u.x, fma(u.y, u.y, aa));
    }
  }
  block_sum3(ab, d2, aa);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = ab;
    partials[gridDim.x + blockIdx.x] = d2;
    partials[2 * gridDim.x + blockIdx.x] = aa;
  }
}

// ... and their totals, in block order, into the device state for the host to read
__global__ void __launch_bounds__(kFinishThreads) k_ms_ru_sum3(SolverState* st, const double* partials, int n) {
  double a = 0.0, b = 0.0, c = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    a += partials[j];
    b += partials[n + j];
    c += partials[2 * n + j];
  }
  block_sum3(a, b, c);
  if (threadIdx.x == 0) {
    st->ms_sums[0] = a;
    st->ms_sums[1] = b;
    st->ms_sums[2] = c;
  }
}

// The FP64 base residual r_t replaces the iterated r, and every direction still moving takes the
// same change scaled by its shift's zeta (the base direction's is 1): p_s += zeta_s (r_t - r).
template <typename R, typename RT>
__global__ void __launch_bounds__(kThreads)
k_ms_ru_fix(MSPtrs P, typename V2<R>::T* __restrict__ r, const RT* __restrict__ rt, int Vh, const SolverState* st) {
  typedef typename V2<R>::T R2;
  const int ns = st->nshift;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Vh; i += gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t k = (size_t)c * Vh + i;
      const double2 t = make_double2((double)rt[k].x, (double)rt[k].y);
      R2 rc = r[k];
      const double dx = t.x - (double)rc.x, dy = t.y - (double)rc.y;
      rc.x = (R)t.x;
      rc.y = (R)t.y;
      r[k] = rc;
      for (int j = 0; j < ns; ++j) {
        if (j > 0 && st->active[j] != 1) continue;
        R2* ps = static_cast<R2*>(P.p[j]);
        const double z = (j == 0) ? 1.0 : st->zeta[j];
        R2 pc = ps[k];
        pc.x = (R)fma(z, dx, (double)pc.x);
        pc.y = (R)fma(z, dy, (double)pc.y);
        ps[k] = pc;
      }
    }
  }
}

// Second stage of a grid reduction: sum the block partials, run the scalar step.
__global__ void __launch_bounds__(kFinishThreads) k_finish(SolverState* st, const double* partials, int n, int fin,
                                                           int gate) {
  pdl_wait();
  if (!gate_open(st, gate)) return;
  finish_partials(st, partials, n, fin);
}

__global__ void __launch_bounds__(kFinishThreads) k_finish_ffs(SolverState* st, const double* partials, int n, int fin,
                                                               int gate) {
  pdl_wait();
  if (!gate_open(st, gate)) return;
  finish_partials_ffs(st, partials, n, fin);
}

__global__ void __launch_bounds__(kFinishThreads) k_finish2(SolverState* st, const double* partials, int n, int fin,
                                                            int gate) {
  if (!gate_open(st, gate)) return;
  finish_partials2(st, partials, n, fin);
}

__global__ void __launch_bounds__(kFinishSRThreads) k_finish_sr(SolverState* st, const double* partials, int n,
                                                                int coff, int cn, int gate, float2* aux,
                                                                unsigned* cnt) {
  pdl_wait();
  if (!gate_open(st, gate)) return;  // uniform over the grid
  finish_partials_sr(st, partials, n, coff, cn, aux, cnt);
}

// One thread: count the WHILE-loop iterations and set its condition. The loop
// continues while the solve is not done and the hard bound is not reached.
__global__ void k_loop_control(SolverState* st) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  st->loop_count += 1;
  // a multi-shift loop with shift-aware reliable updates pauses for the host-driven update
  const int pause = st->ms_ru && st->need_update && !st->done;
  int go = !st->done && !pause && st->loop_count < st->loop_limit;
  if (!go && !st->done && !pause) {
    st->done = 1;
    st->status = SQCG_ERR_NOT_CONVERGED;
  }
  cudaGraphSetConditional((cudaGraphConditionalHandle)st->h_while, go ? 1u : 0u);
}

}  // namespace

// Grid of the streaming BLAS kernels: one wave of resident blocks on every SM, each
// thread looping over sites (no partially filled last wave). Fixed per context, so
// the reductions stay deterministic.
int blas_grid(sqcg_ctx* ctx) {
  if (ctx->blas_grid > 0) return ctx->blas_grid;
  int dev = 0, nsm = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_update<float>, kThreads, 0) != cudaSuccess ||
      nsm < 1 || per_sm < 1) {
    cudaGetLastError();
    nsm = 1;
    per_sm = 1 << 20;  // fall back to one thread per site
  }
  const long g = (long)nsm * per_sm;
  const int full = grid_for(ctx->g.Vh, kThreads);
  ctx->blas_grid = g < full ? (int)g : full;
  return ctx->blas_grid;
}

int launch_finish(sqcg_ctx* ctx, int nblocks, int fin, int gate, cudaStream_t s, bool pdl) {
  SQCG_CUDA_TRY(launch_kernel(k_finish, 1, kFinishThreads, 0, s, pdl, ctx->st, ctx->partials, nblocks, fin, gate));
  return SQCG_OK;
}

int launch_finish_ffs(sqcg_ctx* ctx, int nblocks, int fin, int gate, cudaStream_t s, bool pdl) {
  SQCG_CUDA_TRY(launch_kernel(k_finish_ffs, 1, kFinishThreads, 0, s, pdl, ctx->st, ctx->partials, nblocks, fin, gate));
  return SQCG_OK;
}

int launch_finish2(sqcg_ctx* ctx, int nblocks, int fin, int gate, cudaStream_t s) {
  k_finish2<<<1, kFinishThreads, 0, s>>>(ctx->st, ctx->partials, nblocks, fin, gate);
  SQCG_CUDA_TRY(cudaGetLastError());
  return SQCG_OK;
}

int launch_finish_sr(sqcg_ctx* ctx, int nblocks, int coff, int cn, int gate, cudaStream_t s, bool pdl) {
  SQCG_CUDA_TRY(launch_kernel(k_finish_sr, kFinishSRBlocks, kFinishSRThreads, 0, s, pdl, ctx->st, ctx->partials,
                              nblocks, coff, cn, gate, ctx->fin_aux, ctx->fin_cnt));
  return SQCG_OK;
}

int launch_loop_control(sqcg_ctx* ctx, cudaStream_t s) {
  k_loop_control<<<1, 32, 0, s>>>(ctx->st);
  SQCG_CUDA_TRY(cudaGetLastError());
  return SQCG_OK;
}

// variant with an explicit x (the solver's output vector)
int launch_cg_update_x(sqcg_ctx* ctx, int mixed, double2* x, cudaStream_t s) {
  const int Vh = ctx->g.Vh, grid = blas_grid(ctx);
  if (grid > ctx->max_blocks) return SQCG_ERR_INVALID_ARG;
  if (mixed)
    k_cg_update<float><<<grid, kThreads, 0, s>>>(x, ctx->r32, ctx->p32, ctx->Ap32, Vh, ctx->st, ctx->partials);
  else
    k_cg_update<double><<<grid, kThreads, 0, s>>>(x, ctx->r64, ctx->p64, ctx->Ap64, Vh, ctx->st, ctx->partials);
  SQCG_CUDA_TRY(cudaGetLastError());
  return launch_finish(ctx, grid, FIN_UPDATE, GATE_ITER, s);
}

int launch_cg_xpay(sqcg_ctx* ctx, int mixed, cudaStream_t s) {
  const int Vh = ctx->g.Vh, grid = blas_grid(ctx);
  if (mixed)
    k_cg_xpay<float><<<grid, kThreads, 0, s>>>(ctx->r32, ctx->p32, Vh, ctx->st);
  else
    k_cg_xpay<double><<<grid, kThreads, 0, s>>>(ctx->r64, ctx->p64, Vh, ctx->st);
  SQCG_CUDA_TRY(cudaGetLastError());
  return SQCG_OK;
}

int launch_sr_update(sqcg_ctx* ctx, cudaStream_t s, bool after_kernel) {
  const int Vh = ctx->g.Vh, grid = blas_grid(ctx);
  if (grid > ctx->max_blocks) return SQCG_ERR_INVALID_ARG;
  SQCG_CUDA_TRY(launch_kernel(k_sr_update, grid, kThreads, 0, s, after_kernel && ctx->pdl, ctx->r32, ctx->Ap32,
                              ctx->p32, ctx->q32, ctx->xh32, Vh, ctx->st, ctx->partials + sr_update_partials(ctx)));
  return SQCG_OK;
}

int launch_flush_partial_x(sqcg_ctx* ctx, double2* x, int gate, cudaStream_t s) {
  const int n = ctx->g.Vh * 3;
  k_flush_partial_x<<<blas_grid(ctx), kThreads, 0, s>>>(x, ctx->xh32, n, ctx->st, gate);
  SQCG_CUDA_TRY(cudaGetLastError());
  return SQCG_OK;
}

int launch_norm2_f64(sqcg_ctx* ctx, const double2* v, int fin, cudaStream_t s) {
  const int Vh = ctx->g.Vh, grid = blas_grid(ctx);
  if (grid > ctx->max_blocks) return SQCG_ERR_INVALID_ARG;
  k_norm2_f64<<<grid, kThreads, 0, s>>>(v, Vh, ctx->st, ctx->partials, fin);
  SQCG_CUDA_TRY(cudaGetLastError());
  return launch_finish(ctx, grid, fin, GATE_NONE, s);
}

int launch_scale_copy_f64(sqcg_ctx* ctx, const double2* src, double2* dst, double a, cudaStream_t s) {
  const int n = ctx->g.Vh * 3;
  k_scale_copy_f64<<<grid_for(n, kThreads), kThreads, 0, s>>>(src, dst, a, n);
  SQCG_CUDA_TRY(cudaGetLastError());
  return SQCG_OK;
}

int launch_ms_update_x(sqcg_ctx* ctx, int mixed, int nshift, double2* const* x, cudaStream_t s) {
  // one thread per site: measured faster here than the one-wave grid of the CG kernels
  const int Vh = ctx->g.Vh, grid = grid_for(Vh, kThreads);
  if (grid > ctx->max_blocks || nshift < 1 || nshift > ctx->ms_nalloc) return SQCG_ERR_INVALID_ARG;
  (void)x;  // the x_s updates run in k_ms_xpay
  if (mixed)
    k_ms_update<float><<<grid, kThreads, 0, s>>>(ctx->r32, ctx->Ap32, Vh, ctx->st, ctx->partials);
  else
    k_ms_update<double><<<grid, kThreads, 0, s>>>(ctx->r64, ctx->Ap64, Vh, ctx->st, ctx->partials);
  SQCG_CUDA_TRY(cudaGetLastError());
  return mixed ? launch_finish_ffs(ctx, grid, FIN_MS_UPDATE, GATE_ITER, s)
               : launch_finish(ctx, grid, FIN_MS_UPDATE, GATE_ITER, s);
}

int launch_ms_ru_sums(sqcg_ctx* ctx, const double2* a, const double2* b, double z, cudaStream_t s) {
  const int Vh = ctx->g.Vh, grid = blas_grid(ctx);
  if (3 * grid > 4 * ctx->max_blocks) return SQCG_ERR_INVALID_ARG;  // partials hold 4 * max_blocks
  k_ms_ru_dots<<<grid, kThreads, 0, s>>>(a, b, z, Vh, ctx->partials);
  SQCG_CUDA_TRY(cudaGetLastError());
  k_ms_ru_sum3<<<1, kFinishThreads, 0, s>>>(ctx->st, ctx->partials, grid);
  SQCG_CUDA_TRY(cudaGetLastError());
  return SQCG_OK;
}

int launch_ms_ru_fix(sqcg_ctx* ctx, int mixed, int nshift, const void* rt, int rt_prec, cudaStream_t s) {
  const int Vh = ctx->g.Vh, grid = blas_grid(ctx);
  if (nshift < 1 || nshift > ctx->ms_nalloc) return SQCG_ERR_INVALID_ARG;
  MSPtrs P;
  for (int j = 0; j < SQCG_MAX_SHIFTS; ++j) {
    P.x[j] = nullptr;
    P.p[j] = (j < nshift) ? ctx->ms_p[j] : nullptr;
  }
  const double2* t64 = static_cast<const double2*>(rt);
  const float2* t32 = static_cast<const float2*>(rt);
  if (mixed && rt_prec == SQCG_F32)
    k_ms_ru_fix<float, float2><<<grid, kThreads, 0, s>>>(P, ctx->r32, t32, Vh, ctx->st);
  else if (mixed)
    k_ms_ru_fix<float, double2><<<grid, kThreads, 0, s>>>(P, ctx->r32, t64, Vh, ctx->st);
  else if (rt_prec == SQCG_F64)
    k_ms_ru_fix<double, double2><<<grid, kThreads, 0, s>>>(P, ctx->r64, t64, Vh, ctx->st);
  else
    return SQCG_ERR_INVALID_ARG;
  SQCG_CUDA_TRY(cudaGetLastError());
  return SQCG_OK;
}

int launch_ms_xpay(sqcg_ctx* ctx, int mixed, int nshift, double2* const* x, cudaStream_t s) {
  const int Vh = ctx->g.Vh, grid = grid_for(Vh, kThreads);
  if (nshift < 1 || nshift > ctx->ms_nalloc) return SQCG_ERR_INVALID_ARG;
  MSPtrs P;
  for (int j = 0; j < SQCG_MAX_SHIFTS; ++j) {
    P.x[j] = (j < nshift) ? x[j] : nullptr;
    P.p[j] = (j < nshift) ? ctx->ms_p[j] : nullptr;
  }
  if (mixed)
    k_ms_xpay<float><<<grid, kThreads, 0, s>>>(P, ctx->r32, ctx->p32, Vh, ctx->st);
  else
    k_ms_xpay<double><<<grid, kThreads, 0, s>>>(P, ctx->r64, ctx->p64, Vh, ctx->st);
  SQCG_CUDA_TRY(cudaGetLastError());
  return SQCG_OK;
}
