// Device-side solver control: gates, deterministic grid reductions and the
// scalar steps of CG and multi-shift CG, which one thread of the finisher
// kernel (the second stage of a reduction) runs. All scalars live in
// SolverState in device memory, so a captured solver iteration needs no host
// round trip.
#pragma once

#include <math.h>

#include "sqcg_internal.cuh"

// Programmatic dependent launch (PTX griddepcontrol, sm_90 and later). A kernel launched with the
// programmatic-serialization attribute may be scheduled while the kernel before it on the stream still
// drains its last wave; pdl_wait() blocks until that kernel has completed and its writes are visible,
// and pdl_launch_dependents() lets the next such kernel be scheduled once every block of this one has
// issued it. Both are no-ops in a kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ bool gate_open(const SolverState* st, int gate) {
  if (gate == GATE_NONE) return true;
  const volatile SolverState* v = st;
  if (v->done) return false;
  if (gate == GATE_UPDATE) return v->need_update != 0;
  if (gate == GATE_STEP) return v->need_update == 0;
  return true;
}

// sum over the block; the result is valid in thread 0. blockDim.x must be a
// multiple of 32 and at most 1024. Fixed reduction tree -> deterministic.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double warp_part[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();  // warp_part may still be read by an earlier call
  if (lane == 0) warp_part[wid] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  v = (threadIdx.x < nw) ? warp_part[threadIdx.x] : 0.0;
  if (wid == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

// ---------------------------------------------------------------------------
// scalar steps (run by thread 0 of the finisher, after the partials are summed;
// the multi-shift steps run on the whole block, see solver_finish_ms)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void finish_breakdown(SolverState* s) {
  s->status = SQCG_ERR_BREAKDOWN;
  s->done = 1;
  s->need_update = 0;
}

__device__ inline void solver_finish(SolverState* s, int fin, double v) {
  switch (fin) {
    case FIN_STORE:
      s->pAp = v;
      break;
    case FIN_BB:  // stop thresholds arrive as tol^2 and become tol^2 |b|^2
      s->bb = v;
      s->stop_rr *= v;
      for (int j = 0; j < s->nshift; ++j) s->stop_rr_s[j] *= v;
      break;
    case FIN_INIT:  // r = b - A x0 has just been written
      if (!isfinite(v)) { finish_breakdown(s); break; }
      s->rr = s->rr_true = s->rr_max = v;
      s->rr_prev = v;
      s->iter_last_update = 0;
      if (v <= s->stop_rr) s->done = 1;
      break;
    case FIN_PAP:  // alpha_k = |r_k|^2 / <p_k, A p_k>
      s->pAp = v;
      if (!(v > 0.0) || !isfinite(v)) { finish_breakdown(s); break; }
      s->alpha = s->rr / v;
      break;
    case FIN_UPDATE: {  // |r_{k+1}|^2 after r -= alpha A p
      if (!isfinite(v)) { finish_breakdown(s); break; }
      s->iter += 1;
      s->rr_prev = s->rr;
      s->rr = v;
      s->beta = v / s->rr_prev;
      if (v > s->rr_max) s->rr_max = v;
      if (v <= s->stop_rr) {
        s->need_update = 1;  // confirm on the FP64 true residual
      } else if (s->mixed && (v < s->delta2 * s->rr_max ||
                              s->iter - s->iter_last_update >= s->update_interval)) {
        s->need_update = 1;  // reliable update
      }
      if (s->iter >= s->max_iter) s->need_update = 1;  // final true residual, then stop
      if (s->use_if) cudaGraphSetConditional((cudaGraphConditionalHandle)s->h_if, s->need_update ? 1u : 0u);
      break;
    }
    case FIN_TRUE_RESID: {  // r = b - A x recomputed in FP64 and copied to the working r
      if (!isfinite(v)) { finish_breakdown(s); break; }
      s->rr_true = v;
      s->need_update = 0;
      s->updates += 1;
      s->iter_last_update = s->iter;
      s->rr_max = v;
      if (v <= s->stop_rr) {
        s->done = 1;
        s->status = SQCG_OK;
      } else if (s->iter >= s->max_iter) {
        s->done = 1;
        s->status = SQCG_ERR_NOT_CONVERGED;
      } else if (s->sr) {
        s->after_update = 1;  // the single-reduction step recomputes alpha and beta from A r_true
      } else {
        s->beta = v / s->rr_prev;  // continue from the true residual
        s->rr = v;
      }
      break;
    }
    case FIN_NN_SCALE:  // |r|^2 of the network input
      if (!(v > 0.0) || !isfinite(v)) { finish_breakdown(s); s->nn_s = s->nn_inv_s = 0.0; break; }
      s->nn_s = sqrt(3.0 * (double)s->vh / v);
      s->nn_inv_s = 1.0 / s->nn_s;
      break;
    case FIN_FCG_PAP:  // alpha = <z_k, r_k> / <p_k, A p_k>
      s->pAp = v;
      if (!(v > 0.0) || !isfinite(v)) { finish_breakdown(s); break; }
      s->alpha = s->rz / v;
      break;
    case FIN_FCG_INIT:
      if (!(v > 0.0) || !isfinite(v)) { finish_breakdown(s); break; }
      s->rz = v;
      break;
    default:
      break;
  }
}

// The multi-shift scalar steps, run by the whole finisher block: thread j < nshift
// advances shift j's recurrences, thread 0 the base system's scalars. v is the
// block's total (the same in every thread).
__device__ inline void solver_finish_ms(SolverState* s, int fin, double v) {
  const int j = threadIdx.x;
  const bool own = j < s->nshift;
  if (fin == FIN_MS_PAP) {  // base alpha_k, then zeta_{k+1} and alpha^s_k for every shift
    const bool bad = !(v > 0.0) || !isfinite(v);
    const double a = s->rr / v;
    if (own) {
      int act = s->active[j];
      if (act == 2) s->active[j] = act = 0;  // its final x update was applied last iteration
      if (!bad) {
        if (!act) {
          s->alpha_s[j] = 0.0;
        } else {
          const double zk = s->zeta[j], zkm = s->zeta_prev[j];
          const double den = a * s->beta_prev * (zkm - zk) + zkm * s->alpha_prev * (1.0 + s->dsig[j] * a);
          const double znext = zk * zkm * s->alpha_prev / den;
          s->alpha_s[j] = a * znext / zk;
          s->beta_s[j] = znext;  // holds zeta_{k+1} until the update step
        }
      }
    }
    __syncthreads();  // every thread has read the base scalars before thread 0 writes them
    if (j == 0) {
      s->pAp = v;
      if (bad) finish_breakdown(s);
      else s->alpha = a;
    }
  } else if (fin == FIN_MS_UPDATE) {  // |r_{k+1}|^2, beta_k, beta^s_k, per-shift convergence
    const bool bad = !isfinite(v);
    const double b = v / s->rr;
    const int it = s->iter + 1;
    int any = 0;
    if (own && !bad && s->active[j] == 1) {
      const double zk = s->zeta[j], znext = s->beta_s[j];
      s->zeta_prev[j] = zk;
      s->zeta[j] = znext;
      s->beta_s[j] = b * (znext / zk) * (znext / zk);
      s->iters_s[j] = it;
      // shift residual = zeta * r; a converged shift still takes this iteration's x update (state 2)
      if (znext * znext * v <= s->stop_rr_s[j]) s->active[j] = 2;
      else any = 1;
    }
    any = __syncthreads_or(any);  // also: every thread has read the base scalars
    if (j == 0) {
      if (bad) {
        finish_breakdown(s);
      } else {
        s->iter = it;
        s->rr_prev = s->rr;
        s->rr = v;
        s->beta = b;
        s->alpha_prev = s->alpha;
        s->beta_prev = b;
        if (!any) { s->done = 1; s->status = SQCG_OK; s->ms_final = 1; }
        else if (it >= s->max_iter) { s->done = 1; s->status = SQCG_ERR_NOT_CONVERGED; s->ms_final = 1; }
        else if (s->ms_ru) {  // shift-aware reliable update: the loop pauses after this iteration
          if (v > s->rr_max) s->rr_max = v;
          if (v < s->delta2 * s->rr_max) s->need_update = 1;
        }
      }
    }
  }
}

// Single-reduction CG step (Chronopoulos and Gear's form of CG, one reduction per iteration). The
// iteration carries p, q = A p (recursively) and r; one Dslash pass gives s = A r_k, and its epilogue
// reduces gamma = |r_k|^2, d = Re<r_k, s> and c = Re<r_k, q_{k-1}>. Then beta_k = gamma_k / gamma_{k-1}
// (beta_0 = 0), and the new p_k = r_k + beta p_{k-1}, q_k = s + beta q_{k-1} have
//   <p_k, q_k> = d + 2 beta c + beta^2 <p_{k-1}, q_{k-1}>
// (A is Hermitian, so Re<p_{k-1}, A r_k> = Re<q_{k-1}, r_k>, and <p_{k-1}, q_{k-1}> is the previous step's
// value), and alpha_k = gamma_k / <p_k, q_k>. The cross term is measured, not taken from the textbook
// shortcut <r_k, q_{k-1}> = -gamma_k / alpha_{k-1}, which assumes r_k orthogonal to r_{k-1}: with FP32
// vectors that loses its sign after long stretches without a reliable update. Before that, gamma_k
// decides convergence and the reliable update (an FP64 true residual, after which the step runs again
// on r_true).
__device__ inline void sr_step(SolverState* s, double d, double c, double g) {
  if (!isfinite(d) || !isfinite(c) || !isfinite(g)) { finish_breakdown(s); return; }
  if (s->after_update) {  // r was just replaced by the FP64 true residual (not converged)
    s->after_update = 0;
    s->rr = g;
  } else {
    s->rr_prev = s->rr;
    s->rr = g;
    if (g > s->rr_max) s->rr_max = g;
    if (g <= s->stop_rr) {
      s->need_update = 1;  // confirm on the FP64 true residual
    } else if (g < s->delta2 * s->rr_max || s->iter - s->iter_last_update >= s->update_interval) {
      s->need_update = 1;  // reliable update
    }
    if (s->iter >= s->max_iter) s->need_update = 1;  // final true residual, then stop
    if (s->use_if) cudaGraphSetConditional((cudaGraphConditionalHandle)s->h_if, s->need_update ? 1u : 0u);
    if (s->need_update) return;  // the step runs again after the update
  }
  const double beta = (s->iter > 0) ? g / s->rr_prev : 0.0;
  const double pAp = (s->iter > 0) ? d + beta * (2.0 * c + beta * s->pAp) : d;
  if (!(pAp > 0.0) || !isfinite(pAp)) { finish_breakdown(s); return; }
  s->beta = beta;
  s->pAp = pAp;
  s->alpha = g / pAp;
  s->sr_alpha_prev = s->alpha;
  s->iter += 1;  // the update kernel that follows makes iterate number iter
}

// scalar steps that take two sums (a = first, b = second)
__device__ inline void solver_finish2(SolverState* s, int fin, double a, double b) {
  if (fin == FIN_FCG_BETA) {  // a = <z_{k+1}, r_{k+1}>, b = <z_{k+1}, r_k>
    if (!(a > 0.0) || !isfinite(a) || !isfinite(b)) { finish_breakdown(s); return; }
    s->beta = (a - b) / s->rz;  // Polak-Ribiere (flexible) beta
    s->rz = a;
  }
}

// First stage of a grid-wide sum: each block writes its partial sum to
// partials[blockIdx.x]. The second stage is k_finish (one block, launched
// right after on the same stream), which adds the partials in index order and
// runs the scalar step, so the total does not depend on timing. The kernel
// boundary makes the partials visible without fences or atomics.
__device__ __forceinline__ void block_partial(double v, double* partials) {
  const double b = block_sum(v);
  if (threadIdx.x == 0) partials[blockIdx.x] = b;
}

// Second stage: one block of kFinishThreads threads (each adds only a few partials).
constexpr int kFinishThreads = 1024;
// the single-reduction step's finisher: a few blocks share the partial sums (finish_partials_sr)
constexpr int kFinishSRBlocks = 8;
constexpr int kFinishSRThreads = 256;
static_assert(3 * kFinishSRBlocks <= 64, "the finisher's per-block slots (fin_aux holds 64)");

__device__ __forceinline__ void finish_partials(SolverState* st, const double* partials, int n, int fin) {
  double s = 0.0;
#pragma unroll 4
  for (int j = threadIdx.x; j < n; j += blockDim.x) s += partials[j];
  s = block_sum(s);
  if (fin == FIN_MS_PAP || fin == FIN_MS_UPDATE) {
    __shared__ double total;
    if (threadIdx.x == 0) total = s;
    __syncthreads();
    solver_finish_ms(st, fin, total);
  } else if (threadIdx.x == 0) {
    solver_finish(st, fin, s);
  }
}

// two sums at once: block partials of the second sum follow those of the first (offset n)
__device__ __forceinline__ void block_partial2(double v, double w, double* partials) {
  const double a = block_sum(v);
  const double b = block_sum(w);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = a;
    partials[gridDim.x + blockIdx.x] = b;
  }
}

// Three sums of a block in one pass (warp shuffles, one shared-memory exchange): the totals are valid in
// thread 0. blockDim.x a multiple of 32, at most 1024. Fixed tree -> deterministic.
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c) {
  __shared__ double part3[3][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  __syncthreads();  // part3 may still be read by an earlier call
  if (lane == 0) { part3[0][wid] = a; part3[1][wid] = b; part3[2][wid] = c; }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    a = lane < nw ? part3[0][lane] : 0.0;
    b = lane < nw ? part3[1][lane] : 0.0;
    c = lane < nw ? part3[2][lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
      c += __shfl_down_sync(0xffffffffu, c, o);
    }
  }
}

// ---------------------------------------------------------------------------
// Float-float sums for the single-reduction step. On the GB300 an FP64 add issues at 1/64 of the
// FP32 rate (about two per clock on an SM), so a one-block tree over thousands of FP64 partials
// (measured: 13 us for the 10.6 k partials of a 32^4 step, with the FP64 pipe the stall) and the
// per-block FP64 trees are bound by it. The step's sums instead carry each value as an unevaluated
// sum hi + lo of two floats: a sum of two such pairs is TwoSum of the high parts (Knuth, TAOCP
// vol. 2, 4.2.2) with both low parts added to its error term, then renormalised (Dekker's
// add): about 2^-44 relative per addition, on the FP32 pipe. A partial is stored as a float2 in
// one 8-byte slot of the partials array. Site values are FP32 (as before); the totals become FP64
// only for the scalar step.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 ffs_add(float2 a, float2 b) {
  const float s = __fadd_rn(a.x, b.x);
  const float v = __fsub_rn(s, a.x);
  float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, v)), __fsub_rn(b.x, v));
  e = __fadd_rn(e, __fadd_rn(a.y, b.y));
  const float h = __fadd_rn(s, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, s)));
}

__device__ __forceinline__ double ffs_value(float2 v) { return (double)v.x + (double)v.y; }

__device__ __forceinline__ float2* ffs_slots(double* partials) { return reinterpret_cast<float2*>(partials); }
__device__ __forceinline__ const float2* ffs_slots(const double* partials) {
  return reinterpret_cast<const float2*>(partials);
}

// N float-float sums over the block in one pass; the totals are valid in thread 0. blockDim.x a
// multiple of 32 and at most 1024; a fixed tree (deterministic).
template <int N>
__device__ __forceinline__ void block_sum_ffs(float2 (&v)[N]) {
  __shared__ float2 part[N][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < N; ++k)
      v[k] = ffs_add(v[k], make_float2(__shfl_down_sync(0xffffffffu, v[k].x, o), __shfl_down_sync(0xffffffffu, v[k].y, o)));
  __syncthreads();  // part may still be read by an earlier call
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < N; ++k) part[k][wid] = v[k];
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = lane < nw ? part[k][lane] : make_float2(0.f, 0.f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int k = 0; k < N; ++k)
        v[k] = ffs_add(v[k], make_float2(__shfl_down_sync(0xffffffffu, v[k].x, o), __shfl_down_sync(0xffffffffu, v[k].y, o)));
  }
}

// Three float-float sums over slots [o0, o0 + n), [o1, o1 + n1), [o2, o2 + n) of ffs partials, each
// thread taking every blockDim.x-th slot into four interleaved accumulators (four rows of loads in
// flight), merged in a fixed order; then the block tree. Totals in thread 0 as FP64.
__device__ __forceinline__ void ffs_block_sums3(const double* partials, int o0, int o1, int n1, int o2, int n,
                                                float2 (&v)[3]) {
  const float2* p = ffs_slots(partials);
  const int bd = blockDim.x;
  float2 z = make_float2(0.f, 0.f);
  float2 a4[4] = {z, z, z, z}, b4[4] = {z, z, z, z}, c4[4] = {z, z, z, z};
  int j = threadIdx.x;
  for (; j + 3 * bd < n; j += 4 * bd)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a4[u] = ffs_add(a4[u], p[o0 + j + u * bd]);
      c4[u] = ffs_add(c4[u], p[o2 + j + u * bd]);
    }
#pragma unroll
  for (int u = 0; u < 3; ++u)
    if (j + u * bd < n) {
      a4[u] = ffs_add(a4[u], p[o0 + j + u * bd]);
      c4[u] = ffs_add(c4[u], p[o2 + j + u * bd]);
    }
  j = threadIdx.x;
  for (; j + 3 * bd < n1; j += 4 * bd)
#pragma unroll
    for (int u = 0; u < 4; ++u) b4[u] = ffs_add(b4[u], p[o1 + j + u * bd]);
#pragma unroll
  for (int u = 0; u < 3; ++u)
    if (j + u * bd < n1) b4[u] = ffs_add(b4[u], p[o1 + j + u * bd]);
  v[0] = ffs_add(ffs_add(a4[0], a4[1]), ffs_add(a4[2], a4[3]));
  v[1] = ffs_add(ffs_add(b4[0], b4[1]), ffs_add(b4[2], b4[3]));
  v[2] = ffs_add(ffs_add(c4[0], c4[1]), ffs_add(c4[2], c4[3]));
  block_sum_ffs<3>(v);
}

__device__ __forceinline__ void ffs_sum_partials3(const double* partials, int o0, int o1, int n1, int o2, int n,
                                                  double& a, double& b, double& c) {
  float2 v[3];
  ffs_block_sums3(partials, o0, o1, n1, o2, n, v);
  a = ffs_value(v[0]);
  b = ffs_value(v[1]);
  c = ffs_value(v[2]);
}

// One float-float sum over slots [0, n) of ffs partials (same order rules); total in thread 0 as FP64.
__device__ __forceinline__ double ffs_sum_partials1(const double* partials, int n) {
  const float2* p = ffs_slots(partials);
  const int bd = blockDim.x;
  const float2 z = make_float2(0.f, 0.f);
  float2 a4[4] = {z, z, z, z};
  int j = threadIdx.x;
  for (; j + 3 * bd < n; j += 4 * bd)
#pragma unroll
    for (int u = 0; u < 4; ++u) a4[u] = ffs_add(a4[u], p[j + u * bd]);
#pragma unroll
  for (int u = 0; u < 3; ++u)
    if (j + u * bd < n) a4[u] = ffs_add(a4[u], p[j + u * bd]);
  float2 v[1] = {ffs_add(ffs_add(a4[0], a4[1]), ffs_add(a4[2], a4[3]))};
  block_sum_ffs<1>(v);
  return ffs_value(v[0]);
}

// finish_partials for float-float partials (the FP32 passes of the mixed multi-shift loop)
__device__ __forceinline__ void finish_partials_ffs(SolverState* st, const double* partials, int n, int fin) {
  const double s = ffs_sum_partials1(partials, n);
  if (fin == FIN_MS_PAP || fin == FIN_MS_UPDATE) {
    __shared__ double total;
    if (threadIdx.x == 0) total = s;
    __syncthreads();
    solver_finish_ms(st, fin, total);
  } else if (threadIdx.x == 0) {
    solver_finish(st, fin, s);
  }
}

// The single-reduction step's finisher, spread over the blocks of its grid: d = sum of slots [0, n),
// c = sum of [coff, coff + cn), g = sum of [2n, 3n) (ffs partials). Block b adds the b-th of gridDim.x
// equal contiguous ranges of each; the last block to arrive (an atomic counter, after a fence; a
// handful of arrivals) adds the blocks' totals in block order and runs the scalar step. The ranges and
// both orders are fixed, so the result does not depend on which block comes last. aux holds 3 slots a
// block; *cnt is zero before and after.
__device__ __forceinline__ void finish_partials_sr(SolverState* st, const double* partials, int n, int coff, int cn,
                                                   float2* aux, unsigned* cnt) {
  const int b = blockIdx.x, nb = gridDim.x;
  const int a0 = (int)((long)n * b / nb), a1 = (int)((long)n * (b + 1) / nb);
  const int c0 = (int)((long)cn * b / nb), c1 = (int)((long)cn * (b + 1) / nb);
  float2 v[3];
  ffs_block_sums3(partials, a0, coff + c0, c1 - c0, 2 * n + a0, a1 - a0, v);  // v = {d, c, g} of the range
  __shared__ int last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 3; ++k) aux[3 * b + k] = v[k];
    __threadfence();
    last = atomicAdd(cnt, 1u) == (unsigned)nb - 1u;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  float2 t[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  for (int j = 0; j < nb; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k) t[k] = ffs_add(t[k], __ldcg(&aux[3 * j + k]));
  *cnt = 0u;
  sr_step(st, ffs_value(t[0]), ffs_value(t[1]), ffs_value(t[2]));
}

__device__ __forceinline__ void finish_partials2(SolverState* st, const double* partials, int n, int fin) {
  double a = 0.0, b = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    a += partials[j];
    b += partials[n + j];
  }
  a = block_sum(a);
  b = block_sum(b);
  if (threadIdx.x == 0) solver_finish2(st, fin, a, b);
}
