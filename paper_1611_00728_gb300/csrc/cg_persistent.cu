// Persistent single-reduction mixed-precision CG: the whole Krylov loop between two reliable updates
// in one cooperative kernel, one resident grid that stays on the GPU from one reliable update to the
// next (arXiv:1611.00728 Sec. 4: the CG of the staggered normal equations, with the Dslash as its
// kernel).
//
// Each iteration is the single-reduction step of the graph-launched loop (cg.cu), in three phases
// separated by two grid-wide barriers instead of kernel boundaries:
//   A  the previous step's vector update on this block's even tiles, p = r + beta p, q = s + beta q,
//      xh += alpha p, r -= alpha q, with the block partials of <r_new, q> (this step's cross term), and
//      tmp = D_oe r_new on its odd tiles, each neighbour's r_new formed on the fly from the previous
//      r, s and q with the same two FMAs its owner uses (so the values agree bit for bit). r and q
//      alternate between two buffers by step, so no block overwrites what another still reads; the
//      first step of a launch has no update pending and applies D_oe to r alone
//   B  s = sigma r - D_eo tmp, block partials of <r,s>, |r|^2 (and <r,q> right after a reliable update)
//   C  every block adds the partials in index order and runs the scalar step (convergence, reliable-
//      update trigger, alpha, beta) on its own copy of the solver state in shared memory: the sums
//      and the step are the same instructions on the same data in every block, so every copy is
//      identical and no broadcast is needed. The cross-term partials alternate between two buffers
//      by step as well.
// The kernel returns when the step asks for a reliable update or the solve is done, with r and q
// copied back to the context's buffers; block 0 writes its state copy back. The host then runs the true-residual pass (float-float or FP64 Dslash pair)
// and launches the kernel again, which starts with the three-sum phase B.
//
// Every phase reads the vectors other blocks wrote in the phase before through coherent loads (not
// the read-only path); the links are read-only and keep it. The grid barrier is one arrival counter
// and one generation word: each block's thread 0 fences, arrives, and waits for the generation to
// move, at most kBarrierSpins polls, after which it records the time-out, the grid leaves the loop
// and the state reports SQCG_ERR_CUDA. The launch is cooperative, so the runtime refuses a grid
// that cannot be resident at once instead of starting it.
#include <stdlib.h>
#include <string.h>

#include "dslash_core.cuh"

namespace {

using namespace dcore;

// Registers for 5 resident blocks of 128 a SM (102 a thread). The loop runs only where a parity has at
// most five 128-site tiles a SM (cg.cu), so 5 blocks a SM hold every tile.
constexpr int kPersistentThreadsPerSM = 640;
// a wait gives up after this many polls, 64 ns sleeps apart: well under a second, and more than a
// thousand times the longest phase a barrier waits for in a solve
constexpr unsigned kBarrierSpins = 1u << 22;

struct PArgs {
  DArgs<float> d1;  // tmp = D_oe r  (output parity 1, in = r, out = tmp)
  DArgs<float> d2;  // s = sigma r - D_eo tmp  (output parity 0, in = tmp, out = s)
  float2* r;   // r and q of even steps (the context's buffers, in and out)
  float2* r1;  // ... and of odd steps
  float2* s;
  float2* p;
  float2* q;
  float2* q1;
  float2* xh;
  float2* tmp;
  int Vh, ntiles;
  SolverState* st;
  double* part;     // float-float slots: [3 G] phase-B sums, then [2][G] cross-term partials
  unsigned* bar;    // [0] arrivals, [1] generation, [2] time-out flag
  int max_steps;    // bound on the iterations of one launch (the solver state ends the loop sooner)
  unsigned arrivals;  // blocks a barrier waits for: the grid (one more only in the time-out test)
};

// Grid-wide barrier with release/acquire fences; false when a wait timed out (here or elsewhere).
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;  // the generation cannot move before this block arrives
    __threadfence();
    int good = 1;
    if (atomicAdd(bar, 1u) == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned spins = 0;
      while (*gen == g && *(volatile unsigned*)(bar + 2) == 0u) {
        if (++spins > kBarrierSpins) {
          atomicExch(bar + 2, 1u);
          good = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok = good && *(volatile unsigned*)(bar + 2) == 0u;
  }
  __syncthreads();
  return ok != 0;
}

// r_new = r - alpha (s + beta q) at a neighbour, with the FMAs of the vector update
struct UpdatedIn {
  const float2* r;
  const float2* s;
  const float2* q;
  int Vh;
  float alpha, beta;
  __device__ __forceinline__ void operator()(float2 (&v)[3], int idx) const {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t k = (size_t)c * Vh + idx;
      const float2 rc = r[k], sc = s[k], qc = q[k];
      const float qx = fmaf(beta, qc.x, sc.x), qy = fmaf(beta, qc.y, sc.y);
      v[c] = make_float2(fmaf(-alpha, qx, rc.x), fmaf(-alpha, qy, rc.y));
    }
  }
};

template <bool RECON, bool EIGHT, int PT>
__global__ void __launch_bounds__(PT, kPersistentThreadsPerSM / PT) k_sr_persistent(PArgs a) {
  __shared__ SolverState ss;
  typedef unsigned long long W;
  constexpr int kWords = sizeof(SolverState) / sizeof(W);
  static_assert(sizeof(SolverState) % sizeof(W) == 0, "state copied as 8-byte words");
  for (int k = threadIdx.x; k < kWords; k += PT) reinterpret_cast<W*>(&ss)[k] = reinterpret_cast<const W*>(a.st)[k];
  __syncthreads();
  if (threadIdx.x == 0) ss.use_if = 0;
  const int G = gridDim.x, Vh = a.Vh;
  double* dpart = a.part;
  double* cpart = a.part + 3 * (size_t)G;
  bool timed_out = false;
  int n = 0;
  __syncthreads();
  int cur = 0;  // buffer of the current r and q
  if (!ss.done && !ss.need_update) {
    for (; n < a.max_steps; ++n) {
      const int cb = n & 1;  // this step's buffer
      float2* rn = cb ? a.r1 : a.r;
      float2* qn = cb ? a.q1 : a.q;
      if (n == 0) {
        // A: tmp = D_oe r
        for (int t = blockIdx.x; t < a.ntiles; t += G) {
          const int i = t * PT + threadIdx.x;
          if (i < Vh) {
            float2 acc[3];
            dslash_site<float, RECON, EIGHT, false>(a.d1, i, acc);
#pragma unroll
            for (int c = 0; c < 3; ++c) a.tmp[(size_t)c * Vh + i] = acc[c];
          }
        }
      } else {
        // A: the previous step's update on the even tiles, with the partials of <r_new, q>
        const float2* ro = cb ? a.r : a.r1;
        const float2* qo = cb ? a.q : a.q1;
        const float alpha = (float)ss.alpha, beta = (float)ss.beta;
        float2 cross[1] = {make_float2(0.f, 0.f)};
        for (int t = blockIdx.x; t < a.ntiles; t += G) {
          const int i = t * PT + threadIdx.x;
          if (i < Vh) {
            float2 rc[3], sc[3], pc[3], qc[3], xc[3];
#pragma unroll
            for (int col = 0; col < 3; ++col) {  // all loads before any store
              const size_t k = (size_t)col * Vh + i;
              rc[col] = ro[k];
              sc[col] = a.s[k];
              pc[col] = a.p[k];
              qc[col] = qo[k];
              xc[col] = a.xh[k];
            }
            float rq = 0.f;
#pragma unroll
            for (int col = 0; col < 3; ++col) {
              const size_t k = (size_t)col * Vh + i;
              pc[col].x = fmaf(beta, pc[col].x, rc[col].x);
              pc[col].y = fmaf(beta, pc[col].y, rc[col].y);
              qc[col].x = fmaf(beta, qc[col].x, sc[col].x);
              qc[col].y = fmaf(beta, qc[col].y, sc[col].y);
              xc[col].x = fmaf(alpha, pc[col].x, xc[col].x);
              xc[col].y = fmaf(alpha, pc[col].y, xc[col].y);
              rc[col].x = fmaf(-alpha, qc[col].x, rc[col].x);
              rc[col].y = fmaf(-alpha, qc[col].y, rc[col].y);
              a.p[k] = pc[col];
              qn[k] = qc[col];
              a.xh[k] = xc[col];
              rn[k] = rc[col];
            }
#pragma unroll
            for (int col = 0; col < 3; ++col) rq = fmaf(rc[col].x, qc[col].x, fmaf(rc[col].y, qc[col].y, rq));
            cross[0] = ffs_add(cross[0], make_float2(rq, 0.f));
          }
        }
        block_sum_ffs<1>(cross);
        if (threadIdx.x == 0) ffs_slots(cpart)[(size_t)cb * G + blockIdx.x] = cross[0];
        // ... and tmp = D_oe r_new on the odd tiles, r_new formed at each neighbour from the previous step
        const UpdatedIn in_at{ro, a.s, qo, Vh, alpha, beta};
        for (int t = blockIdx.x; t < a.ntiles; t += G) {
          const int i = t * PT + threadIdx.x;
          if (i < Vh) {
            float2 acc[3];
            dslash_site_in<float, RECON, EIGHT>(a.d1, i, acc, in_at);
#pragma unroll
            for (int c = 0; c < 3; ++c) a.tmp[(size_t)c * Vh + i] = acc[c];
          }
        }
      }
      cur = cb;
      if (!grid_barrier(a.bar, a.arrivals)) { timed_out = true; break; }
      // B: s = sigma r - D_eo tmp with <r,s>, |r|^2 and, after a reliable update, <r,q>
      const bool after = ss.after_update != 0;
      const float sig = (float)ss.sigma;
      __shared__ float2 tot[3];  // the block's totals so far (thread 0; in shared memory, not live in registers)
      if (threadIdx.x == 0) tot[0] = tot[1] = tot[2] = make_float2(0.f, 0.f);
      for (int t = blockIdx.x; t < a.ntiles; t += G) {
        const int i = t * PT + threadIdx.x;
        float rs = 0.f, rq = 0.f, rr = 0.f;
        if (i < Vh) {
          float2 acc[3];
          dslash_site<float, RECON, EIGHT, false>(a.d2, i, acc);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const size_t k = (size_t)c * Vh + i;
            const float2 rc = rn[k];
            const float2 o = make_float2(sig * rc.x - acc[c].x, sig * rc.y - acc[c].y);
            a.s[k] = o;
            rs = fmaf(rc.x, o.x, fmaf(rc.y, o.y, rs));
            rr = fmaf(rc.x, rc.x, fmaf(rc.y, rc.y, rr));
            if (after) {
              const float2 qc = qn[k];
              rq = fmaf(rc.x, qc.x, fmaf(rc.y, qc.y, rq));
            }
          }
        }
        // the tile's sums (one tree per tile keeps nothing live across the next tile's Dslash)
        float2 v[3] = {make_float2(rs, 0.f), make_float2(rq, 0.f), make_float2(rr, 0.f)};
        block_sum_ffs<3>(v);
        if (threadIdx.x == 0)
#pragma unroll
          for (int k = 0; k < 3; ++k) tot[k] = ffs_add(tot[k], v[k]);
      }
      if (threadIdx.x == 0) {
        float2* slot = ffs_slots(dpart);
        slot[blockIdx.x] = tot[0];
        slot[G + blockIdx.x] = tot[1];
        slot[2 * G + blockIdx.x] = tot[2];
      }
      if (!grid_barrier(a.bar, a.arrivals)) { timed_out = true; break; }
      // C: the step's sums, in the same order in every block, and the scalar step on the block's copy
      double d, c, g;
      ffs_sum_partials3(a.part, 0, after ? G : 3 * G + cb * G, G, 2 * G, G, d, c, g);
      if (threadIdx.x == 0) sr_step(&ss, d, c, g);
      __syncthreads();
      if (ss.done || ss.need_update) break;  // the same decision in every block
    }
  }
  // r and q back into the context's buffers (each block copies the even tiles it wrote; nothing reads
  // them any more in this launch)
  if (cur == 1) {
    for (int t = blockIdx.x; t < a.ntiles; t += G) {
      const int i = t * PT + threadIdx.x;
      if (i < Vh) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const size_t k = (size_t)c * Vh + i;
          a.r[k] = a.r1[k];
          a.q[k] = a.q1[k];
        }
      }
    }
  }
  if (blockIdx.x != 0) return;
  __syncthreads();
  if (threadIdx.x == 0) {
    if (timed_out) {
      ss.status = SQCG_ERR_CUDA;
      ss.done = 1;
      ss.need_update = 0;
    } else if (n >= a.max_steps && !ss.done && !ss.need_update) {
      ss.status = SQCG_ERR_NOT_CONVERGED;
      ss.done = 1;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < kWords; k += PT) reinterpret_cast<W*>(a.st)[k] = reinterpret_cast<const W*>(&ss)[k];
}

constexpr int kPT = 128;

template <bool RECON, bool EIGHT>
void* kernel_for() {
  return reinterpret_cast<void*>(k_sr_persistent<RECON, EIGHT, kPT>);
}

void* persistent_kernel(const sqcg_ctx* ctx) {
  if (ctx->eightway) return ctx->recon ? kernel_for<true, true>() : kernel_for<false, true>();
  return ctx->recon ? kernel_for<true, false>() : kernel_for<false, false>();
}

DArgs<float> dargs(const sqcg_ctx* ctx, int par, const float2* in, float2* out) {
  DArgs<float> a = {};
  const size_t Vh = ctx->g.Vh;
  const int p = par, q = 1 - par;
  const int nl = ctx->recon ? 6 : 9;
  const float2* fat = reinterpret_cast<const float2*>(ctx->fat32);
  const float2* lng = reinterpret_cast<const float2*>(ctx->lng32);
  a.g = ctx->g;
  a.par = par;
  a.fat_p = fat + (size_t)p * 4 * 9 * Vh;
  a.fat_q = fat + (size_t)q * 4 * 9 * Vh;
  a.lng_p = lng + (size_t)p * 4 * nl * Vh;
  a.lng_q = lng + (size_t)q * 4 * nl * Vh;
  a.fatb_p = ctx->eightway ? reinterpret_cast<const float2*>(ctx->fatb32) + (size_t)p * 4 * 9 * Vh : nullptr;
  a.lngb_p = ctx->eightway ? reinterpret_cast<const float2*>(ctx->lngb32) + (size_t)p * 4 * nl * Vh : nullptr;
  a.nl = nl;
  a.inv_s0 = (float)(ctx->recon ? 1.0 / ctx->long_scale : 1.0);
  a.in = in;
  a.out = out;
  return a;
}

}  // namespace

// Grid of the persistent loop for the context's link form (0: not available): every SM filled with
// resident blocks, never more blocks than tiles. Allocates the kernel's partials (for the largest
// grid, one block a tile) and barrier words on first use.
int persistent_grid(sqcg_ctx* ctx) {
  if (ctx->pers_grid < 0) return 0;
  int dev = 0, coop = 0, nsm = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_kernel(ctx), kPT, 0) != cudaSuccess) {
    cudaGetLastError();
    ctx->pers_grid = -1;
    return 0;
  }
  if (!coop || nsm < 1 || per_sm < 1) {
    ctx->pers_grid = -1;
    return 0;
  }
  const int ntiles = grid_for(ctx->g.Vh, kPT);
  if (!ctx->pers_part) {
    const size_t nv = (size_t)3 * ctx->g.Vh;
    if (cudaMalloc(&ctx->pers_part, (size_t)5 * ntiles * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&ctx->pers_bar, 4 * sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(&ctx->pers_rq, 2 * nv * sizeof(float2)) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(ctx->pers_part);
      cudaFree(ctx->pers_bar);
      cudaFree(ctx->pers_rq);
      ctx->pers_part = nullptr;
      ctx->pers_bar = nullptr;
      ctx->pers_rq = nullptr;
      ctx->pers_grid = -1;
      return 0;
    }
  }
  const long want = (long)nsm * per_sm;
  ctx->pers_grid = (int)(want < ntiles ? want : ntiles);
  return ctx->pers_grid;
}

// One launch of the persistent loop on the solver workspace (r32, Ap32 as s, p32, q32, xh32, tmp32).
int launch_sr_persistent(sqcg_ctx* ctx, int max_steps, cudaStream_t s) {
  const int G = persistent_grid(ctx);
  if (G <= 0) return SQCG_ERR_INVALID_ARG;
  PArgs a = {};
  a.d1 = dargs(ctx, 1, ctx->r32, ctx->tmp32);
  a.d2 = dargs(ctx, 0, ctx->tmp32, ctx->Ap32);
  a.r = ctx->r32;
  a.r1 = ctx->pers_rq;
  a.s = ctx->Ap32;
  a.p = ctx->p32;
  a.q = ctx->q32;
  a.q1 = ctx->pers_rq + (size_t)3 * ctx->g.Vh;
  a.xh = ctx->xh32;
  a.tmp = ctx->tmp32;
  a.Vh = ctx->g.Vh;
  a.ntiles = grid_for(ctx->g.Vh, kPT);
  a.st = ctx->st;
  a.part = ctx->pers_part;
  a.bar = ctx->pers_bar;
  a.max_steps = max_steps;
  // SQCG_TEST_BARRIER_TIMEOUT=1 makes every barrier wait for one block more than the grid has, so each
  // wait runs out: the test of the bounded waits (the solve then returns SQCG_ERR_CUDA, nothing hangs)
  const char* t = getenv("SQCG_TEST_BARRIER_TIMEOUT");
  a.arrivals = (unsigned)G + ((t && strcmp(t, "1") == 0) ? 1u : 0u);
  SQCG_CUDA_TRY(cudaMemsetAsync(ctx->pers_bar, 0, 4 * sizeof(unsigned), s));
  void* args[] = {&a};
  SQCG_CUDA_TRY(cudaLaunchCooperativeKernel(persistent_kernel(ctx), dim3(G), dim3(kPT), args, 0, s));
  return SQCG_OK;
}
