// Batched multi-RHS CG over several lattices of different volumes in one
// device-side loop (the single-mass CG of arXiv:1611.00728 Sec. 3 applied to
// many sources at once; mixed precision with FP64 reliable updates).
//
// Work decomposition: a tile is (lattice, RHS block of width W, block of T
// sites). One launch per phase covers the tiles of every lattice, so the small
// lattices ride along with the large one instead of paying their own launch
// and tail. The FP32 Dslash block first stages the 16 links of each of its
// sites in shared memory, then its W / WT thread groups apply them to WT
// right-hand sides each, so the link stream (96% of the single-RHS bytes) is
// read from HBM once per W sources: 1152/W + 48 bytes per site-RHS. The FP32
// work vectors hold the RHS in pairs (see pv), so a thread's two RHS of one
// site and colour are one 16-byte gather.
//
// Every RHS has its own CG scalars in BatchState; the per-RHS dot products are
// reduced deterministically in two stages (warp shuffle -> block partial per
// tile, then one block per RHS adds the partials in site-block order). The
// BLAS kernels use their own 256-site tiles, independent of the Dslash tile.
// The loop is one CUDA graph: a WHILE node around [D_oe p, A p with <p,Ap>,
// x/r update, IF(reliable update in FP64), p update, loop control], or the
// same kernels launched one at a time (SQCG_LAUNCH_MODE=eager). W, WT, T and
// the shared-memory carveout are chosen by a small autotuner that times the
// FP32 multi-RHS Dslash over the whole batch and caches the choice (or are
// pinned by sqcg_batched_pin_tuning).
#include <chrono>
#include <map>
#include <math.h>
#include <mutex>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <string>

#include "ff_arith.cuh"
#include "solver_device.cuh"
#include "sqcg_internal.cuh"

namespace {

constexpr int kMaxT = 256;    // largest site block (threads along x)
constexpr int kMaxThreads = 512;  // largest CTA (site block x RHS groups)
constexpr int kMaxTSmem = 128;    // largest site block of the shared-memory FP32 Dslash (144 KB of links)
constexpr int kMinT = 32;     // smallest site block
constexpr int kW64 = 4;       // RHS per pass in the FP64 kernels (register budget)
constexpr int kTB = 256;      // site block of the BLAS kernels (independent of the tuned Dslash tile)

struct LatDev {
  Geom g;
  const float2* fat32[2];
  const float2* lng32[2];
  const double2* fat64[2];
  const double2* lng64[2];
  int nl32, recon;  // the 12-real long-link form exists for the FP32 copy only
  float inv_s0_f;
  double inv_s0_d;
  int rhs0, nrhs;  // global index of the first RHS, count
  int nsb;         // site blocks of T sites
  int nrb, rb0;    // FP32 RHS blocks of width W, global index of the first
  int nrb64, rb640;  // FP64 RHS blocks of width min(W, kW64)
  int tile0, tile640;  // first FP32 / FP64 tile
  int nsb_b, tile0_b;  // BLAS tiling: site blocks of kTB sites, first BLAS tile
  int sbt0;            // first BLAS site block of this lattice over all lattices
  float2 *r, *p, *Ap, *tmp;  // RHS pairs: element (w, c, i) at pv(w, c, i, Vh)
  float2* xh;                // FP32 partial solutions (RHS pairs), flushed into x at each reliable update
  double2* x;
  double2* tmp64;       // FP64 intermediate, or the float-float one (float4 [w][c][Vh]) of the float-float passes
  const float4* fatff[2];  // float-float links (reliable updates in float-float arithmetic)
  const float4* lngff[2];
  float4* xff;          // float-float copy of x for those passes ([w][c][Vh])
  const double2* b;
  size_t b_stride;  // elements between the sources of consecutive RHS: 3 Vh, or 0 when all share one source
};

// The FP32 work vectors r, p, Ap and tmp hold the right-hand sides of a lattice in pairs:
// element (RHS w, colour c, site i) is float2 number ((w/2)*3 + c)*2Vh + 2i + w%2, so the two
// RHS of a pair at one site and colour form one 16-byte word (one gather for a thread that
// holds both). An odd RHS count leaves the second half of the last pair zero. The FP64
// vectors (x, b, tmp64) keep the caller's [w][c][Vh] order.
__host__ __device__ __forceinline__ size_t pv(int w, int c, int i, int Vh) {
  return (((size_t)(w >> 1) * 3 + c) * Vh + i) * 2 + (w & 1);
}

// v[w] = element (w0 + w, c, i) for w < WT; zero where w >= nw. WT = 1, or WT even with w0 even.
template <int WT>
__device__ __forceinline__ void pv_load(const float2* __restrict__ base, int w0, int nw, int c, int i, int Vh,
                                        float2 (&v)[WT]) {
  if constexpr (WT == 1) {
    v[0] = nw > 0 ? __ldg(base + pv(w0, c, i, Vh)) : make_float2(0.f, 0.f);
  } else {
#pragma unroll
    for (int q = 0; q < WT / 2; ++q) {
      float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
      if (2 * q < nw) t = __ldg(reinterpret_cast<const float4*>(base) + ((size_t)((w0 >> 1) + q) * 3 + c) * Vh + i);
      v[2 * q] = make_float2(t.x, t.y);
      v[2 * q + 1] = make_float2(t.z, t.w);
    }
  }
}

// element (w0 + w, c, i) = v[w] for w < nw (the same layouts as pv_load)
template <int WT>
__device__ __forceinline__ void pv_store(float2* __restrict__ base, int w0, int nw, int c, int i, int Vh,
                                         const float2 (&v)[WT]) {
  if constexpr (WT == 1) {
    if (nw > 0) base[pv(w0, c, i, Vh)] = v[0];
  } else {
#pragma unroll
    for (int q = 0; q < WT / 2; ++q) {
      if (2 * q + 1 < nw)
        reinterpret_cast<float4*>(base)[((size_t)((w0 >> 1) + q) * 3 + c) * Vh + i] =
            make_float4(v[2 * q].x, v[2 * q].y, v[2 * q + 1].x, v[2 * q + 1].y);
      else if (2 * q < nw)
        base[pv(w0 + 2 * q, c, i, Vh)] = v[2 * q];
    }
  }
}

template <typename R> struct V2;
template <> struct V2<double> { typedef double2 T; };
template <> struct V2<float> { typedef float2 T; };

template <typename R2>
__device__ __forceinline__ R2 mk2(decltype(R2().x) a, decltype(R2().x) b) { R2 r; r.x = a; r.y = b; return r; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// decode a tile into (lattice, RHS block, site block); RHS blocks fastest
__device__ __forceinline__ int find_lat(const LatDev* lats, int nlat, int tile, bool fp64) {
  int k = 0;
  for (int j = 1; j < nlat; ++j)
    if (tile >= (fp64 ? lats[j].tile640 : lats[j].tile0)) k = j;
  return k;
}

// ---------------------------------------------------------------------------
// per-RHS CG scalar steps (same rules as the single-mass solver)
// ---------------------------------------------------------------------------
enum BFin { BFIN_BB = 1, BFIN_INIT = 2, BFIN_PAP = 3, BFIN_UPDATE = 4, BFIN_TRUE = 5, BFIN_XX = 6 };

__device__ void rhs_finish(RhsScalars& s, const BatchState* st, int fin, double v) {
  switch (fin) {
    case BFIN_BB:
      s.bb = v;
      s.stop_rr *= v;
      break;
    case BFIN_XX:  // |x0|^2, parked in pAp until the first iteration overwrites it
      s.pAp = v;
      break;
    case BFIN_INIT:
      if (!isfinite(v)) { s.status = SQCG_ERR_BREAKDOWN; s.active = 0; break; }
      s.rr = s.rr_true = s.rr_max = s.rr_prev = v;
      s.iter_last_update = 0;
      if (v <= s.stop_rr) { s.active = 0; s.status = SQCG_OK; }
      break;
    case BFIN_PAP:
      if (!s.active) break;
      s.pAp = v;
      if (!(v > 0.0) || !isfinite(v)) { s.status = SQCG_ERR_BREAKDOWN; s.active = 0; s.need_update = 0; break; }
      s.alpha = s.rr / v;
      break;
    case BFIN_UPDATE:
      if (!s.active) break;
      if (!isfinite(v)) { s.status = SQCG_ERR_BREAKDOWN; s.active = 0; s.need_update = 0; break; }
      s.iter += 1;
      s.rr_prev = s.rr;
      s.rr = v;
      s.beta = v / s.rr_prev;
      if (v > s.rr_max) s.rr_max = v;
      if (v <= s.stop_rr || v < st->delta2 * s.rr_max || s.iter - s.iter_last_update >= st->update_interval ||
          s.iter >= st->max_iter)
        s.need_update = 1;
      break;
    case BFIN_TRUE:  // only the RHS that asked for the update were recomputed
      if (!s.need_update || !s.active) break;
      if (!isfinite(v)) { s.status = SQCG_ERR_BREAKDOWN; s.active = 0; s.need_update = 0; break; }
      s.rr_true = v;
      s.need_update = 0;
      s.updates += 1;
      s.iter_last_update = s.iter;
      s.rr_max = v;
      if (v <= s.stop_rr) { s.active = 0; s.status = SQCG_OK; }
      else if (s.iter >= st->max_iter) { s.active = 0; s.status = SQCG_ERR_NOT_CONVERGED; }
      else { s.beta = v / s.rr_prev; s.rr = v; }
      break;
    default:
      break;
  }
}

// First stage of the per-RHS sums: reduce the tile's values per RHS and write
// partials[rhs][site block]. Blocks are (sites x RHS groups): thread (x, y)
// holds the WT values of RHS y*WT .. y*WT+WT-1 of the tile; blockDim.x is a
// multiple of 32, so every warp belongs to one group. The second stage is
// k_batch_finish, launched right after on the same stream.
template <int WT>
__device__ void rhs_block_partial(double (&v)[WT], const LatDev& L, int wbase, int nw_tile, int sb,
                                  double* partials, int max_nsb) {
  __shared__ double red[16][kMaxT / 32];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, wx = threadIdx.x >> 5, nwx = blockDim.x >> 5;
#pragma unroll
  for (int w = 0; w < WT; ++w) {
    const double t = warp_sum(v[w]);
    if (lane == 0) red[threadIdx.y * WT + w][wx] = t;
  }
  __syncthreads();
  if (tid < nw_tile) {
    double t = 0.0;
    for (int j = 0; j < nwx; ++j) t += red[tid][j];
    partials[(size_t)(L.rhs0 + wbase + tid) * max_nsb + sb] = t;
  }
}

// Second stage: one block per RHS adds its partials in site-block order and
// runs the per-RHS scalar step (deterministic). blas: the partials come from
// the BLAS tiling (nsb_b site blocks) rather than the Dslash tiling (nsb).
constexpr int kBatchFinishThreads = 1024;

__global__ void __launch_bounds__(kBatchFinishThreads) k_batch_finish(BatchState* st, const LatDev* lats, int nlat,
                                                                      const double* partials, int max_nsb, int fin,
                                                                      int blas) {
  const int g = blockIdx.x;
  int k = 0;
  for (int j = 1; j < nlat; ++j)
    if (g >= lats[j].rhs0) k = j;
  const LatDev& L = lats[k];
  const int n = blas ? L.nsb_b : L.nsb;
  // four independent sums per thread keep several loads in flight (the Dslash leaves up to
  // one partial per 32 sites); the assignment of partials to sums is fixed -> deterministic
  const double* pp = partials + (size_t)g * max_nsb;
  const int B = blockDim.x;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int j = threadIdx.x;
  for (; j + 3 * B < n; j += 4 * B) {
    s0 += pp[j];
    s1 += pp[j + B];
    s2 += pp[j + 2 * B];
    s3 += pp[j + 3 * B];
  }
  for (; j < n; j += B) s0 += pp[j];
  const double s = block_sum((s0 + s1) + (s2 + s3));
  if (threadIdx.x == 0) rhs_finish(st->r[g], st, fin, s);
}

// ---------------------------------------------------------------------------
// multi-RHS Dslash
// ---------------------------------------------------------------------------
template <typename R, bool RECONS>
__device__ __forceinline__ void load_link_m(typename V2<R>::T (&U)[9], const typename V2<R>::T* __restrict__ base,
                                            int Vh, int idx, bool recon, R inv_s) {
  typedef typename V2<R>::T R2;
  if (!recon) {
#pragma unroll
    for (int e = 0; e < 9; ++e) U[e] = __ldg(base + (size_t)e * Vh + idx);
  } else {
#pragma unroll
    for (int e = 0; e < 6; ++e) U[e] = __ldg(base + (size_t)e * Vh + idx);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int k = (j + 1) % 3, l = (j + 2) % 3;
      const R2 ak = U[k], al = U[l], bk = U[3 + k], bl = U[3 + l];
      const R re = ak.x * bl.x - ak.y * bl.y - (al.x * bk.x - al.y * bk.y);
      const R im = ak.x * bl.y + ak.y * bl.x - (al.x * bk.y + al.y * bk.x);
      U[6 + j] = mk2<R2>(re * inv_s, -im * inv_s);
    }
  }
}

template <typename R, int W, bool DAG>
__device__ __forceinline__ void apply_w(typename V2<R>::T (&acc)[W][3], const typename V2<R>::T (&U)[9],
                                        const typename V2<R>::T* __restrict__ in, int Vh, int idx, int nw,
                                        unsigned mask = 0xffffffffu) {
  typedef typename V2<R>::T R2;
#pragma unroll
  for (int w = 0; w < W; ++w) {
    if (w < nw && ((mask >> w) & 1u)) {
      R2 v[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) v[c] = __ldg(in + ((size_t)w * 3 + c) * Vh + idx);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          if (!DAG) {
            const R2 u = U[a * 3 + b];
            acc[w][a].x = fma(u.x, v[b].x, acc[w][a].x);
            acc[w][a].x = fma(-u.y, v[b].y, acc[w][a].x);
            acc[w][a].y = fma(u.x, v[b].y, acc[w][a].y);
            acc[w][a].y = fma(u.y, v[b].x, acc[w][a].y);
          } else {
            const R2 u = U[b * 3 + a];
            acc[w][a].x = fma(-u.x, v[b].x, acc[w][a].x);
            acc[w][a].x = fma(-u.y, v[b].y, acc[w][a].x);
            acc[w][a].y = fma(-u.x, v[b].y, acc[w][a].y);
            acc[w][a].y = fma(u.y, v[b].x, acc[w][a].y);
          }
        }
      }
    }
  }
}

// acc[w] = D in[w] at site i of parity par, for nw <= W right-hand sides
template <typename R, int W>
__device__ __forceinline__ void dslash_mrhs_site(const LatDev& L, int par, int i, const typename V2<R>::T* in,
                                                 int nw, typename V2<R>::T (&acc)[W][3],
                                                 unsigned mask = 0xffffffffu) {
  typedef typename V2<R>::T R2;
  const Geom& g = L.g;
  const int Vh = g.Vh;
  const int xh = i % g.Lxh;
  int rr = i / g.Lxh;
  const int y = rr % g.Ly;
  rr /= g.Ly;
  const int z = rr % g.Lz;
  const int t = rr / g.Lz;
  const int x = 2 * xh + ((y + z + t + par) & 1);
  const int row = i - xh;
#pragma unroll
  for (int w = 0; w < W; ++w)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[w][c] = mk2<R2>(R(0), R(0));
  const R2* fat_p;
  const R2* fat_q;
  const R2* lng_p;
  const R2* lng_q;
  R inv_s0;
  if constexpr (sizeof(R) == 8) {
    fat_p = L.fat64[par]; fat_q = L.fat64[1 - par]; lng_p = L.lng64[par]; lng_q = L.lng64[1 - par];
    inv_s0 = (R)L.inv_s0_d;
  } else {
    fat_p = L.fat32[par]; fat_q = L.fat32[1 - par]; lng_p = L.lng32[par]; lng_q = L.lng32[1 - par];
    inv_s0 = (R)L.inv_s0_f;
  }
  const bool recon = (sizeof(R) == 4) && L.recon != 0;
  const int nl = recon ? 6 : 9;
  R2 U[9];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    R inv_f = inv_s0, inv_b = inv_s0;
    if (recon) {
      int e = 0;
      if (mu == 1) e = x;
      if (mu == 2) e = x + y;
      if (mu == 3) e = x + y + z;
      if (e & 1) { inv_f = -inv_f; inv_b = -inv_b; }
      if (mu == 3 && g.apbc) {
        if (t + 3 >= g.Lt) inv_f = -inv_f;
        if (t < 3) inv_b = -inv_b;
      }
    }
    const int cmu = (mu == 0) ? x : (mu == 1) ? y : (mu == 2) ? z : t;
    const int Lmu = (mu == 0) ? g.Lx : (mu == 1) ? g.Ly : (mu == 2) ? g.Lz : g.Lt;
    const int smu = (mu == 1) ? g.sy : (mu == 2) ? g.sz : g.st;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int d = (k == 0) ? 1 : 3;
      int fwd, bwd;
      if (mu == 0) {
        int xp = x + d; if (xp >= g.Lx) xp -= g.Lx;
        int xm = x - d; if (xm < 0) xm += g.Lx;
        fwd = row + (xp >> 1);
        bwd = row + (xm >> 1);
      } else {
        fwd = i + d * smu; if (cmu + d >= Lmu) fwd -= Lmu * smu;
        bwd = i - d * smu; if (cmu - d < 0) bwd += Lmu * smu;
      }
      if (k == 0) {
        load_link_m<R, false>(U, fat_p + (size_t)mu * 9 * Vh, Vh, i, false, R(1));
        apply_w<R, W, false>(acc, U, in, Vh, fwd, nw, mask);
        load_link_m<R, false>(U, fat_q + (size_t)mu * 9 * Vh, Vh, bwd, false, R(1));
        apply_w<R, W, true>(acc, U, in, Vh, bwd, nw, mask);
      } else {
        load_link_m<R, true>(U, lng_p + (size_t)mu * nl * Vh, Vh, i, recon, inv_f);
        apply_w<R, W, false>(acc, U, in, Vh, fwd, nw, mask);
        load_link_m<R, true>(U, lng_q + (size_t)mu * nl * Vh, Vh, bwd, recon, inv_b);
        apply_w<R, W, true>(acc, U, in, Vh, bwd, nw, mask);
      }
    }
  }
}

enum MEpi { M_PLAIN = 0, M_NORMAL_DOT = 1, M_TRUE_RESID = 2 };
enum MVec { V_P = 0, V_TMP = 1, V_X = 2, V_TMP64 = 3, V_XFF = 4 };

struct MArgs {
  const LatDev* lats;
  int nlat;
  int par;       // output parity
  int in_vec;    // MVec of the input
  int epi;
  int gate;      // GATE_NONE, GATE_ITER (RHS block active), GATE_UPDATE (RHS block needs update)
  BatchState* st;
  double* partials;
  int max_nsb;
  int W;         // RHS block width of the FP32 blocks (gates refer to these blocks)
  int write_p;   // M_TRUE_RESID at initialisation: also copy r into p
  int ntiles;    // tiles of the launch (float-float kernel: several tiles per CTA)
};

// Thread (x, y) of a tile: site sb*blockDim.x + x, right-hand sides y*WT .. y*WT+WT-1
// of the tile's RHS block (width WT*blockDim.y). The groups y of one site
// block load the same links, which the first group brings into L1.
template <typename R, int WT>
__global__ void __launch_bounds__(kMaxThreads) k_mrhs_dslash(MArgs a) {
  typedef typename V2<R>::T R2;
  constexpr bool F64 = sizeof(R) == 8;
  static_assert(F64, "the FP32 batched Dslash is k_mrhs_dslash_smem");
  const int tile = blockIdx.x;
  const int k = find_lat(a.lats, a.nlat, tile, F64);
  const LatDev& L = a.lats[k];
  const int local = tile - (F64 ? L.tile640 : L.tile0);
  const int nrb = F64 ? L.nrb64 : L.nrb;
  const int rb = local % nrb, sb = local / nrb;
  const int Wtile = WT * blockDim.y;
  const int wbase = rb * Wtile;
  const int nw_tile = min(Wtile, L.nrhs - wbase);
  const int w0 = wbase + threadIdx.y * WT;            // first RHS of this thread (within the lattice)
  const int nw = max(0, min(WT, L.nrhs - w0));
  const int blk = L.rb0 + wbase / a.W;  // FP32 block that holds these RHS
  if (a.gate == GATE_ITER && !a.st->blk_active[blk]) return;
  if (a.gate == GATE_UPDATE && !a.st->blk_update[blk]) return;
  const int Vh = L.g.Vh;
  const int i = sb * blockDim.x + threadIdx.x;
  double part[WT];
#pragma unroll
  for (int w = 0; w < WT; ++w) part[w] = 0.0;
  const R2* in = (a.in_vec == V_X ? (const R2*)L.x : (const R2*)L.tmp64) + (size_t)w0 * 3 * Vh;
  // in a reliable-update pass only the RHS that asked for one are computed (FP64 work is the cost here)
  unsigned mask = 0xffffffffu;
  if (a.gate == GATE_UPDATE) {
    mask = 0u;
#pragma unroll
    for (int w = 0; w < WT; ++w)
      if (w < nw && a.st->r[L.rhs0 + w0 + w].need_update && a.st->r[L.rhs0 + w0 + w].active) mask |= 1u << w;
  }
  if (i < Vh && nw > 0 && mask) {
    R2 acc[WT][3];
    dslash_mrhs_site<R, WT>(L, a.par, i, in, nw, acc, mask);
    if (a.epi == M_PLAIN) {
      R2* out = (R2*)L.tmp64 + (size_t)w0 * 3 * Vh;
#pragma unroll
      for (int w = 0; w < WT; ++w)
        if (w < nw && ((mask >> w) & 1u))
#pragma unroll
          for (int c = 0; c < 3; ++c) out[((size_t)w * 3 + c) * Vh + i] = acc[w][c];
    } else {  // M_TRUE_RESID: r = b - sigma x + D tmp64, |r|^2; r (FP32) and optionally p
      const double2* xb = L.x + (size_t)w0 * 3 * Vh;
      const double2* bb = L.b + (size_t)w0 * L.b_stride;
#pragma unroll
      for (int w = 0; w < WT; ++w) {
        if (w < nw && ((mask >> w) & 1u)) {
          const double sig = a.st->r[L.rhs0 + w0 + w].sigma;
          double n2 = 0.0;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const size_t o = ((size_t)w * 3 + c) * Vh + i;
            const double2 xc = __ldg(xb + o), bc = __ldg(bb + (size_t)w * L.b_stride + (size_t)c * Vh + i);
            const double re = bc.x - sig * xc.x + (double)acc[w][c].x;
            const double im = bc.y - sig * xc.y + (double)acc[w][c].y;
            const float2 f = make_float2((float)re, (float)im);
            L.r[pv(w0 + w, c, i, Vh)] = f;
            if (a.write_p) L.p[pv(w0 + w, c, i, Vh)] = f;
            n2 += re * re + im * im;
          }
          part[w] = n2;
        }
      }
    }
  }
  if (a.epi != M_PLAIN) {
    const int fin = (a.epi == M_NORMAL_DOT) ? BFIN_PAP : (a.write_p ? BFIN_INIT : BFIN_TRUE);
    (void)fin;
    rhs_block_partial<WT>(part, L, wbase, nw_tile, sb, a.partials, a.max_nsb);
  }
}

// The reliable-update passes in float-float arithmetic (ff_arith.cuh): the same tiles, gates and
// epilogues as k_mrhs_dslash<double, WT>, with links and vectors as float4 (hi, lo) pairs. On this GPU
// the FP64 kernel is bound by the FP64 FMA rate (1/64 of FP32); this one runs on the FP32 pipe.
// Per-RHS partials of a CTA that holds NB = blockDim.y independent tiles of blockDim.x sites (slice y is
// tile tile0 + y): each slice reduces its WT sums over its sites (warp shuffles, then a fixed-order sum
// over the slice's warps) and writes partials[rhs][sb]. Every thread of the CTA must call it.
template <int WT>
__device__ void slice_partials(double (&v)[WT], const LatDev* L, int wbase, int nw_tile, int sb, double* partials,
                               int max_nsb) {
  __shared__ double red[4][4][WT];  // [slice][warp of the slice][rhs]; blockDim.x * blockDim.y <= 128
  const int lane = threadIdx.x & 31, wx = threadIdx.x >> 5, nwx = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int w = 0; w < WT; ++w) {
    double t = v[w];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) red[threadIdx.y][wx][w] = t;
  }
  __syncthreads();
  if (L && (int)threadIdx.x < nw_tile) {
    double t = 0.0;
    for (int j = 0; j < nwx; ++j) t += red[threadIdx.y][j][threadIdx.x];
    partials[(size_t)(L->rhs0 + wbase + threadIdx.x) * max_nsb + sb] = t;
  }
}

// 128 threads per CTA and at least 6 CTAs per SM: at most 80 registers per thread, so 24 warps per SM
// keep the gathers in flight (at 4 RHS per thread in registers this kernel needed 128 and held 16)
template <int WT>
__global__ void __launch_bounds__(128, 6) k_mrhs_dslash_ff(MArgs a) {
  // slice y of the CTA is one tile (blockDim.x sites x WT right-hand sides); no early return before the
  // partials, whose reduction synchronises the CTA
  const int tile = blockIdx.x * blockDim.y + threadIdx.y;
  const bool have_tile = tile < a.ntiles;
  const int k = have_tile ? find_lat(a.lats, a.nlat, tile, true) : 0;
  const LatDev& L = a.lats[k];
  const int local = tile - L.tile640;
  const int rb = have_tile ? local % L.nrb64 : 0, sb = have_tile ? local / L.nrb64 : 0;
  const int wbase = rb * WT;
  const int nw_tile = have_tile ? min(WT, L.nrhs - wbase) : 0;
  const int w0 = wbase;
  const int nw = have_tile ? max(0, min(WT, L.nrhs - w0)) : 0;
  const int blk = L.rb0 + wbase / a.W;
  bool run = have_tile && !(a.gate == GATE_UPDATE && !a.st->blk_update[blk]);
  const Geom& g = L.g;
  const int Vh = g.Vh;
  const int i = sb * blockDim.x + threadIdx.x;
  double part[WT];
#pragma unroll
  for (int w = 0; w < WT; ++w) part[w] = 0.0;
  unsigned mask = 0xffffffffu;
  if (run && a.gate == GATE_UPDATE) {
    mask = 0u;
#pragma unroll
    for (int w = 0; w < WT; ++w)
      if (w < nw && a.st->r[L.rhs0 + w0 + w].need_update && a.st->r[L.rhs0 + w0 + w].active) mask |= 1u << w;
  }
  if (run && i < Vh && nw > 0 && mask) {
    const int xh = i % g.Lxh;
    int rr = i / g.Lxh;
    const int y = rr % g.Ly;
    rr /= g.Ly;
    const int z = rr % g.Lz;
    const int t = rr / g.Lz;
    const int x = 2 * xh + ((y + z + t + a.par) & 1);
    const int row = i - xh;
    // one RHS at a time: the registers of the single-RHS float-float kernel, so the CTA keeps many warps
    // resident; the tile's links come from HBM for its first RHS and from L1/L2 for the others
#pragma unroll 1
    for (int w = 0; w < WT; ++w) {
      if (!(w < nw && ((mask >> w) & 1u))) continue;
      const float4* in = (a.in_vec == V_XFF ? (const float4*)L.xff : (const float4*)L.tmp64) +
                         (size_t)(w0 + w) * 3 * Vh;
      float4 acc[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
      float4 U[9], v[3];
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) {
        const int cmu = (mu == 0) ? x : (mu == 1) ? y : (mu == 2) ? z : t;
        const int Lmu = (mu == 0) ? g.Lx : (mu == 1) ? g.Ly : (mu == 2) ? g.Lz : g.Lt;
        const int smu = (mu == 1) ? g.sy : (mu == 2) ? g.sz : g.st;
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          const int d = (kk == 0) ? 1 : 3;
          int fwd, bwd;
          if (mu == 0) {
            int xp = x + d; if (xp >= g.Lx) xp -= g.Lx;
            int xm = x - d; if (xm < 0) xm += g.Lx;
            fwd = row + (xp >> 1);
            bwd = row + (xm >> 1);
          } else {
            fwd = i + d * smu; if (cmu + d >= Lmu) fwd -= Lmu * smu;
            bwd = i - d * smu; if (cmu - d < 0) bwd += Lmu * smu;
          }
          const float4* fl = (kk == 0) ? L.fatff[a.par] : L.lngff[a.par];
          const float4* bl = (kk == 0) ? L.fatff[1 - a.par] : L.lngff[1 - a.par];
#pragma unroll
          for (int e = 0; e < 9; ++e) U[e] = __ldg(fl + ((size_t)mu * 9 + e) * Vh + i);
#pragma unroll
          for (int c = 0; c < 3; ++c) v[c] = __ldg(in + (size_t)c * Vh + fwd);
          ff_mv(acc, U, v);
#pragma unroll
          for (int e = 0; e < 9; ++e) U[e] = __ldg(bl + ((size_t)mu * 9 + e) * Vh + bwd);
#pragma unroll
          for (int c = 0; c < 3; ++c) v[c] = __ldg(in + (size_t)c * Vh + bwd);
          ff_mdv_sub(acc, U, v);
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        ff_norm(acc[c].x, acc[c].y);
        ff_norm(acc[c].z, acc[c].w);
      }
      if (a.epi == M_PLAIN) {
        float4* out = (float4*)L.tmp64 + (size_t)(w0 + w) * 3 * Vh;
#pragma unroll
        for (int c = 0; c < 3; ++c) out[(size_t)c * Vh + i] = acc[c];
      } else {  // M_TRUE_RESID: r = b - sigma x + D tmp, the sum in FP64; r (FP32) and optionally p
        const double2* xb = L.x + (size_t)(w0 + w) * 3 * Vh;
        const double2* bb = L.b + (size_t)(w0 + w) * L.b_stride;
        const double sig = a.st->r[L.rhs0 + w0 + w].sigma;
        double n2 = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const double2 xc = __ldg(xb + (size_t)c * Vh + i), bc = __ldg(bb + (size_t)c * Vh + i);
          const double2 dv = join_ff(acc[c]);
          const double re = bc.x - sig * xc.x + dv.x;
          const double im = bc.y - sig * xc.y + dv.y;
          const float2 f = make_float2((float)re, (float)im);
          L.r[pv(w0 + w, c, i, Vh)] = f;
          if (a.write_p) L.p[pv(w0 + w, c, i, Vh)] = f;
          n2 += re * re + im * im;
        }
        part[w] = n2;  // one local-memory store per RHS (a register array would cost the loop registers)
      }
    }
  }
  if (a.epi != M_PLAIN) slice_partials<WT>(part, run ? &L : nullptr, wbase, nw_tile, sb, a.partials, a.max_nsb);
}

// For every RHS that takes the reliable update (all RHS when not gated): x += xh (the FP32 partial
// solution, added in FP64), xh = 0, and, with float-float updates (split), xff = the float-float copy of
// the new x. Ungated without split, it is the final flush after the loop.
__global__ void k_mrhs_flush_x(const LatDev* lats, int nlat, const BatchState* st, int gated, int split) {
  const int g = blockIdx.y;
  int k = 0;
  for (int j = 1; j < nlat; ++j)
    if (g >= lats[j].rhs0) k = j;
  const LatDev& L = lats[k];
  const int w = g - L.rhs0;
  if (w >= L.nrhs) return;
  if (gated && !(st->r[g].need_update && st->r[g].active)) return;
  const int Vh = L.g.Vh;
  const size_t n = (size_t)3 * Vh, off = (size_t)w * n;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx / Vh), i = (int)(idx % Vh);
    float2* hp = L.xh + pv(w, c, i, Vh);
    const float2 h = *hp;
    double2 v = L.x[off + idx];
    v.x += (double)h.x;
    v.y += (double)h.y;
    L.x[off + idx] = v;
    *hp = make_float2(0.f, 0.f);
    if (split) L.xff[off + idx] = split_ff(v);
  }
}

// Per-RHS block partial of a kernel whose warps hold SUB consecutive sites of 32 / SUB RHS groups:
// thread (site ax, group ay) holds v[w] for RHS ay * WT + w of the tile. Segmented warp sums over the
// SUB sites, then a fixed-order sum over the site chunks -> deterministic.
template <int WT, int SUB>
__device__ void rhs_block_partial_m(double (&v)[WT], const LatDev& L, int wbase, int nw_tile, int sb, int ax, int ay,
                                    double* partials, int max_nsb) {
  __shared__ double red[16][kMaxTSmem / 16];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31;
  const int nchunk = blockDim.x / SUB;
#pragma unroll
  for (int w = 0; w < WT; ++w) {
    double t = v[w];
#pragma unroll
    for (int o = SUB / 2; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o, SUB);
    if ((lane & (SUB - 1)) == 0) red[ay * WT + w][ax / SUB] = t;
  }
  __syncthreads();
  if (tid < nw_tile) {
    double t = 0.0;
    for (int j = 0; j < nchunk; ++j) t += red[tid][j];
    partials[(size_t)(L.rhs0 + wbase + tid) * max_nsb + sb] = t;
  }
}

// half-lattice coordinates of site i of parity par
struct SiteXY {
  int x, y, z, t, row;
};

__device__ __forceinline__ SiteXY site_of(const Geom& g, int i, int par) {
  SiteXY c;
  const int xh = i % g.Lxh;
  int rr = i / g.Lxh;
  c.y = rr % g.Ly;
  rr /= g.Ly;
  c.z = rr % g.Lz;
  c.t = rr / g.Lz;
  c.x = 2 * xh + ((c.y + c.z + c.t + par) & 1);
  c.row = i - xh;
  return c;
}

// half index of n + d mu for the site (i, c)
__device__ __forceinline__ int nbr_of(const Geom& g, int i, const SiteXY& c, int mu, int d) {
  if (mu == 0) {
    int xp = c.x + d;
    if (xp >= g.Lx) xp -= g.Lx;
    if (xp < 0) xp += g.Lx;
    return c.row + (xp >> 1);
  }
  const int cc = (mu == 1) ? c.y : (mu == 2) ? c.z : c.t;
  const int Lm = (mu == 1) ? g.Ly : (mu == 2) ? g.Lz : g.Lt;
  const int sm = (mu == 1) ? g.sy : (mu == 2) ? g.sz : g.st;
  int j = i + d * sm;
  if (cc + d >= Lm) j -= Lm * sm;
  if (cc + d < 0) j += Lm * sm;
  return j;
}

// FP32 multi-RHS Dslash with the links of the tile staged in shared memory.
// A block covers T = blockDim.x sites and the tile's W = WT * G right-hand sides
// (G = blockDim.y groups of WT). First the block copies the 16 links of each of
// its sites (8 fat, 8 long; 12-real long links rebuilt here) from global memory
// into shared memory, thread (x, y) staging site x for hops y, y + G, ...; then
// every (site, group) thread applies them to its WT right-hand sides. Each link
// is read from global memory once per RHS block, whatever W is.
// SUB = 32: a warp holds 32 consecutive sites of one group. SUB = 16 (G even):
// a warp holds 16 sites of two groups, so each link element a warp reads from
// shared memory serves both groups in one access (a broadcast), which halves the
// shared-memory wavefronts of the link reads; the neighbour gathers are the same.
constexpr int kHops = 16;

template <int WT, int SUB>
__global__ void __launch_bounds__(kMaxThreads) k_mrhs_dslash_smem(MArgs a) {
  extern __shared__ float2 sU[];  // [kHops][9][blockDim.x]
  const int tile = blockIdx.x;
  const int k = find_lat(a.lats, a.nlat, tile, false);
  const LatDev& L = a.lats[k];
  const int local = tile - L.tile0;
  const int rb = local % L.nrb, sb = local / L.nrb;
  const int TX = blockDim.x, G = blockDim.y;
  const int Wtile = WT * G;
  const int wbase = rb * Wtile;
  const int nw_tile = min(Wtile, L.nrhs - wbase);
  const int blk = L.rb0 + rb;
  if (a.gate == GATE_ITER && !a.st->blk_active[blk]) return;
  const Geom& g = L.g;
  const int Vh = g.Vh;
  const int par = a.par, q = 1 - par;
  // ---- stage the links: thread (x, y) stages site x for hops h = y, y + G, ... ----
  // hop h = 4 * mu + 2 * (long) + (backward)
  {
    const int i = sb * TX + threadIdx.x;
    const bool valid = i < Vh;
    const SiteXY c = valid ? site_of(g, i, par) : SiteXY{0, 0, 0, 0, 0};
    const bool recon = L.recon != 0;
    const int nl = recon ? 6 : 9;
    for (int h = threadIdx.y; h < kHops; h += G) {
      const int mu = h >> 2, lng = (h >> 1) & 1, bwd = h & 1;
      const int d = lng ? 3 : 1;
      float2 u[9];
      if (valid) {
        const float2* base = lng ? (bwd ? L.lng32[q] : L.lng32[par]) : (bwd ? L.fat32[q] : L.fat32[par]);
        base += (size_t)mu * (lng ? nl : 9) * Vh;
        const int idx = bwd ? nbr_of(g, i, c, mu, -d) : i;
        const int ne = lng ? nl : 9;
#pragma unroll
        for (int e = 0; e < 9; ++e)
          if (e < ne) u[e] = __ldg(base + (size_t)e * Vh + idx);
        if (lng && recon) {  // third row = conj(row0 x row1) / s, s = s0 * eta_mu * boundary sign
          int ep = 0;
          if (mu == 1) ep = c.x;
          if (mu == 2) ep = c.x + c.y;
          if (mu == 3) ep = c.x + c.y + c.z;
          float inv_s = (ep & 1) ? -L.inv_s0_f : L.inv_s0_f;
          if (mu == 3 && g.apbc && (bwd ? (c.t < 3) : (c.t + 3 >= g.Lt))) inv_s = -inv_s;
#pragma unroll
          for (int jj = 0; jj < 3; ++jj) {
            const int kk = (jj + 1) % 3, ll = (jj + 2) % 3;
            const float2 ak = u[kk], al = u[ll], bk = u[3 + kk], bl = u[3 + ll];
            const float re = ak.x * bl.x - ak.y * bl.y - (al.x * bk.x - al.y * bk.y);
            const float im = ak.x * bl.y + ak.y * bl.x - (al.x * bk.y + al.y * bk.x);
            u[6 + jj] = make_float2(re * inv_s, -im * inv_s);
          }
        }
      } else {
#pragma unroll
        for (int e = 0; e < 9; ++e) u[e] = make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int e = 0; e < 9; ++e) sU[(h * 9 + e) * TX + threadIdx.x] = u[e];
    }
  }
  __syncthreads();
  // ---- apply to this thread's right-hand sides: thread (site ax, group ay) ----
  int ax = threadIdx.x, ay = threadIdx.y;
  if constexpr (SUB == 16) {
    const int tid = threadIdx.x + TX * threadIdx.y;
    const int lane = tid & 31, warp = tid >> 5, cpr = TX / 16;
    ax = (warp % cpr) * 16 + (lane & 15);
    ay = (warp / cpr) * 2 + (lane >> 4);
  }
  const int w0 = wbase + ay * WT;
  const int nw = max(0, min(WT, L.nrhs - w0));
  const int i = sb * TX + ax;
  const bool valid = i < Vh;
  double part[WT];
#pragma unroll
  for (int w = 0; w < WT; ++w) part[w] = 0.0;
  const float2* in = (a.in_vec == V_P ? (const float2*)L.p : (const float2*)L.tmp);
  if (valid && nw > 0) {
    const SiteXY c = site_of(g, i, par);
    float2 acc[WT][3];
#pragma unroll
    for (int w = 0; w < WT; ++w)
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) acc[w][cc] = make_float2(0.f, 0.f);
    // one-hop software pipeline: the next hop's neighbour vectors are in flight while
    // this hop's products run (the gathers, not the FMAs, set the pace of this kernel)
    float2 vin[WT][3], vnx[WT][3];
    auto gather = [&](int h, float2 (&v)[WT][3]) {
      const int mu = h >> 2, lng = (h >> 1) & 1, bwd = h & 1;
      const int j = nbr_of(g, i, c, mu, bwd ? (lng ? -3 : -1) : (lng ? 3 : 1));
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        float2 t[WT];
        pv_load<WT>(in, w0, nw, cc, j, Vh, t);  // one 16-byte gather per RHS pair
#pragma unroll
        for (int w = 0; w < WT; ++w) v[w][cc] = t[w];
      }
    };
    gather(0, vin);
#pragma unroll
    for (int h = 0; h < kHops; ++h) {
      if (h + 1 < kHops) gather(h + 1, vnx);
      const bool bwd = h & 1;
      float2 U[9];
#pragma unroll
      for (int e = 0; e < 9; ++e) U[e] = sU[(h * 9 + e) * TX + ax];
#pragma unroll
      for (int w = 0; w < WT; ++w)
#pragma unroll
        for (int aa = 0; aa < 3; ++aa)
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            const float2 v = vin[w][b];
            if (!bwd) {
              const float2 u = U[aa * 3 + b];
              acc[w][aa].x = fmaf(u.x, v.x, acc[w][aa].x);
              acc[w][aa].x = fmaf(-u.y, v.y, acc[w][aa].x);
              acc[w][aa].y = fmaf(u.x, v.y, acc[w][aa].y);
              acc[w][aa].y = fmaf(u.y, v.x, acc[w][aa].y);
            } else {
              const float2 u = U[b * 3 + aa];
              acc[w][aa].x = fmaf(-u.x, v.x, acc[w][aa].x);
              acc[w][aa].x = fmaf(-u.y, v.y, acc[w][aa].x);
              acc[w][aa].y = fmaf(-u.x, v.y, acc[w][aa].y);
              acc[w][aa].y = fmaf(u.y, v.x, acc[w][aa].y);
            }
          }
      if (h + 1 < kHops)
#pragma unroll
        for (int w = 0; w < WT; ++w)
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) vin[w][cc] = vnx[w][cc];
    }
    if (a.epi == M_PLAIN) {
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        float2 t[WT];
#pragma unroll
        for (int w = 0; w < WT; ++w) t[w] = acc[w][cc];
        pv_store<WT>(L.tmp, w0, nw, cc, i, Vh, t);
      }
    } else {  // M_NORMAL_DOT: Ap = sigma p - D tmp, <p, Ap>
      float sig[WT], dot[WT];
#pragma unroll
      for (int w = 0; w < WT; ++w) {
        sig[w] = w < nw ? (float)a.st->r[L.rhs0 + w0 + w].sigma : 0.f;
        dot[w] = 0.f;
      }
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        float2 yc[WT], v[WT];
        pv_load<WT>(L.p, w0, nw, cc, i, Vh, yc);
#pragma unroll
        for (int w = 0; w < WT; ++w) {
          v[w] = make_float2(sig[w] * yc[w].x - acc[w][cc].x, sig[w] * yc[w].y - acc[w][cc].y);
          dot[w] = fmaf(yc[w].x, v[w].x, fmaf(yc[w].y, v[w].y, dot[w]));
        }
        pv_store<WT>(L.Ap, w0, nw, cc, i, Vh, v);
      }
#pragma unroll
      for (int w = 0; w < WT; ++w)
        if (w < nw) part[w] = (double)dot[w];
    }
  }
  if (a.epi != M_PLAIN)
    rhs_block_partial_m<WT, SUB>(part, L, wbase, nw_tile, sb, ax, ay, a.partials, a.max_nsb);
}

// ---------------------------------------------------------------------------
// multi-RHS BLAS: x += alpha p, r -= alpha Ap (|r|^2); p = r + beta p; |b|^2
// ---------------------------------------------------------------------------
// B_NORM_X: |x0|^2; B_INIT_B: r = p = b (FP32) with |b|^2, the exact initial residual for x0 = 0
enum MBlas { B_UPDATE = 0, B_XPAY = 1, B_NORM_B = 2, B_NORM_X = 3, B_INIT_B = 4 };

struct BArgs {
  const LatDev* lats;
  int nlat;
  int op;
  BatchState* st;
  double* partials;
  int max_nsb;
  int W;
};

// One thread per (site, RHS pair): blockIdx.x runs over the kTB-site blocks of all lattices,
// blockIdx.y over the RHS pairs of a lattice. A thread streams the three colour components
// of both RHS (16-byte words of the paired FP32 vectors), so all loads of a block are
// independent and in flight together. An RHS that is not running keeps its values. Per-RHS
// sums go to partials[rhs][site block] for k_batch_finish.
__global__ void __launch_bounds__(kTB) k_mrhs_blas(BArgs a) {
  int k = 0;
  for (int j = 1; j < a.nlat; ++j)
    if ((int)blockIdx.x >= a.lats[j].sbt0) k = j;
  const LatDev& L = a.lats[k];
  const int w0 = 2 * blockIdx.y;
  if (w0 >= L.nrhs) return;
  const int nw = min(2, L.nrhs - w0);
  const int sb = blockIdx.x - L.sbt0;
  const bool all = (a.op == B_NORM_B || a.op == B_NORM_X || a.op == B_INIT_B);
  bool act[2];
  double alpha[2], beta[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int rhs = L.rhs0 + w0 + u;
    act[u] = u < nw && (all || (a.st->blk_active[L.rb0 + (w0 + u) / a.W] && a.st->r[rhs].active));
    alpha[u] = act[u] ? a.st->r[rhs].alpha : 0.0;
    beta[u] = act[u] ? a.st->r[rhs].beta : 0.0;
  }
  if (!act[0] && !act[1]) return;
  const int Vh = L.g.Vh;
  const int i = sb * blockDim.x + threadIdx.x;
  double part[2] = {0.0, 0.0};
  if (i < Vh) {
    if (all) {
      float2 f[3][2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (!act[u]) continue;
        const double2* v = (a.op == B_NORM_X) ? L.x + (size_t)(w0 + u) * 3 * Vh : L.b + (size_t)(w0 + u) * L.b_stride;
        double2 vc[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) vc[c] = v[(size_t)c * Vh + i];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          part[u] = fma(vc[c].x, vc[c].x, fma(vc[c].y, vc[c].y, part[u]));
          f[c][u] = make_float2((float)vc[c].x, (float)vc[c].y);
        }
      }
      if (a.op == B_INIT_B)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          pv_store<2>(L.r, w0, nw, c, i, Vh, f[c]);
          pv_store<2>(L.p, w0, nw, c, i, Vh, f[c]);
        }
    } else if (a.op == B_UPDATE) {
      float2 pc[3][2], apc[3][2], rc[3][2];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        pv_load<2>(L.p, w0, nw, c, i, Vh, pc[c]);
        pv_load<2>(L.Ap, w0, nw, c, i, Vh, apc[c]);
        pv_load<2>(L.r, w0, nw, c, i, Vh, rc[c]);
      }
      float2 xc[3][2];  // the FP32 partial solutions of the pair (flushed into x at reliable updates)
#pragma unroll
      for (int c = 0; c < 3; ++c) pv_load<2>(L.xh, w0, nw, c, i, Vh, xc[c]);
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (!act[u]) continue;
        const float fa = (float)alpha[u];
        float n2 = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          xc[c][u].x = fmaf(fa, pc[c][u].x, xc[c][u].x);
          xc[c][u].y = fmaf(fa, pc[c][u].y, xc[c][u].y);
          rc[c][u].x = fmaf(-fa, apc[c][u].x, rc[c][u].x);
          rc[c][u].y = fmaf(-fa, apc[c][u].y, rc[c][u].y);
          n2 = fmaf(rc[c][u].x, rc[c][u].x, fmaf(rc[c][u].y, rc[c][u].y, n2));
        }
        part[u] = (double)n2;
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        pv_store<2>(L.r, w0, nw, c, i, Vh, rc[c]);
        pv_store<2>(L.xh, w0, nw, c, i, Vh, xc[c]);
      }
    } else {  // B_XPAY
      float2 rc[3][2], pc[3][2];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        pv_load<2>(L.r, w0, nw, c, i, Vh, rc[c]);
        pv_load<2>(L.p, w0, nw, c, i, Vh, pc[c]);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (!act[u]) continue;
        const float be = (float)beta[u];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          pc[c][u].x = fmaf(be, pc[c][u].x, rc[c][u].x);
          pc[c][u].y = fmaf(be, pc[c][u].y, rc[c][u].y);
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) pv_store<2>(L.p, w0, nw, c, i, Vh, pc[c]);
    }
  }
  if (a.op != B_XPAY) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const double t = block_sum(part[u]);
      if (threadIdx.x == 0 && act[u]) a.partials[(size_t)(L.rhs0 + w0 + u) * a.max_nsb + sb] = t;
    }
  }
}

// One thread: which RHS blocks need the FP64 reliable update -> IF condition
__global__ void k_batch_ctl_update(BatchState* st, const LatDev* lats, int nlat, int W) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int any = 0;
  for (int k = 0; k < nlat; ++k) {
    const LatDev& L = lats[k];
    for (int rb = 0; rb < L.nrb; ++rb) {
      int u = 0;
      for (int w = rb * W; w < min((rb + 1) * W, L.nrhs); ++w) u |= st->r[L.rhs0 + w].need_update;
      st->blk_update[L.rb0 + rb] = u;
      any |= u;
    }
  }
  st->if_runs += any;
  if (st->use_graph) cudaGraphSetConditional((cudaGraphConditionalHandle)st->h_if, any ? 1u : 0u);
}

// One thread: active RHS blocks, loop count and the WHILE condition
__global__ void k_batch_ctl_loop(BatchState* st, const LatDev* lats, int nlat, int W) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  st->loop_count += 1;
  int any = 0;
  for (int k = 0; k < nlat; ++k) {
    const LatDev& L = lats[k];
    for (int rb = 0; rb < L.nrb; ++rb) {
      int a = 0;
      for (int w = rb * W; w < min((rb + 1) * W, L.nrhs); ++w) a |= st->r[L.rhs0 + w].active;
      st->blk_active[L.rb0 + rb] = a;
      any |= a;
    }
  }
  const int go = any && st->loop_count < st->loop_limit;
  if (!go && any) {  // hard bound reached: stop every RHS that is still running
    for (int j = 0; j < st->nrhs; ++j)
      if (st->r[j].active) { st->r[j].active = 0; st->r[j].status = SQCG_ERR_NOT_CONVERGED; }
  }
  if (st->use_graph) cudaGraphSetConditional((cudaGraphConditionalHandle)st->h_while, go ? 1u : 0u);
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct BatchPlan {
  int nlat;
  sqcg_ctx* ctx[SQCG_MAX_LATTICES];
  unsigned long long gen[SQCG_MAX_LATTICES];
  int nrhs[SQCG_MAX_LATTICES];
  const void* b[SQCG_MAX_LATTICES];
  void* x[SQCG_MAX_LATTICES];
  int b_shared;          // every RHS of a lattice reads the same source b[k]
  int ff;                // reliable updates in float-float arithmetic (else FP64)
  int W, T;              // tuned RHS block width and site block (threads along x)
  int carve;             // tuned shared-memory carveout of the FP32 Dslash (percent; -1 = driver default)
  int WT;                // RHS per thread in the FP32 Dslash (W / WT thread groups per site block)
  int sub;               // sites per warp row of the FP32 Dslash: 32, or 16 (two RHS groups per warp)
  int ntiles, ntiles64;  // FP32 / FP64 tiles over all lattices
  int ntiles_b;          // BLAS tiles over all lattices
  int nblk;              // FP32 RHS blocks over all lattices
  int max_nsb;
  int nrhs_total;
  LatDev host[SQCG_MAX_LATTICES];
  LatDev* dev;           // device copy of host[]
  void* work[SQCG_MAX_LATTICES];  // per lattice: r, p, Ap, tmp, xh (FP32), tmp64 and xff
  double* partials;
  BatchState* st;
  BatchState* st_host;
  cudaGraphExec_t exec;
  cudaGraphConditionalHandle h_while, h_if;
};

extern unsigned long long sqcg_links_generation(const sqcg_ctx* ctx);

namespace {

struct TuneChoice {
  int W, WT, T, carve, sub;
};

// shape rules of the FP32 Dslash: T a multiple of 32 up to kMaxTSmem, T * W / WT threads at most
// kMaxThreads, SUB = 16 only with an even number of RHS groups
bool smem_shape_ok(int W, int WT, int T, int sub) {
  if (WT < 1 || W % WT) return false;
  const int G = W / WT;
  if (T < 32 || T % 32 || T > kMaxTSmem || T * G > kMaxThreads) return false;
  return sub == 32 || (sub == 16 && G % 2 == 0);
}


// Guards the process-wide tuning state (the cache and file, and the per-kernel shared-memory
// attributes) when several host threads run batched solves on their own contexts.
std::recursive_mutex& tune_mutex() {
  static std::recursive_mutex m;
  return m;
}

TuneChoice& tune_pin() {  // W = 0: autotune
  static TuneChoice c = {0, 0, 0, -1, 32};
  return c;
}

std::map<std::string, TuneChoice>& tune_cache() {
  static std::map<std::string, TuneChoice> m;
  return m;
}

bool tune_file_loaded = false;

void tune_file_load() {
  if (tune_file_loaded) return;
  tune_file_loaded = true;
  const char* path = getenv("SQCG_TUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char line[768], key[512];
  while (fgets(line, sizeof(line), f)) {
    int W, WT, T, carve = -1, sub = 32;
    const int got = sscanf(line, "%511s %d %d %d %d %d", key, &W, &WT, &T, &carve, &sub);
    if (got >= 4 && smem_shape_ok(W, WT, T, got == 6 ? sub : 32))
      tune_cache()[key] = {W, WT, T, got >= 5 ? carve : -1, got == 6 ? sub : 32};
  }
  fclose(f);
}

void tune_file_store(const std::string& key, const TuneChoice& c) {
  const char* path = getenv("SQCG_TUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %d %d %d %d\n", key.c_str(), c.W, c.WT, c.T, c.carve, c.sub);
  fclose(f);
}

std::string tune_key(const BatchPlan& P) {
  std::string k = "mrhs_dslash_smem_f32";
  char buf[128];
  for (int j = 0; j < P.nlat; ++j) {
    const Geom& g = P.host[j].g;
    snprintf(buf, sizeof(buf), ":%dx%dx%dx%d/r%d/n%d", g.Lx, g.Ly, g.Lz, g.Lt, P.host[j].recon, P.nrhs[j]);
    k += buf;
  }
  return k;
}

// tiles, blocks and first indices for a given W and T
void layout_tiles(BatchPlan& P, int W, int WT, int T) {
  int tile = 0, tile64 = 0, tileb = 0, rb0 = 0, rb640 = 0, sbt = 0;
  const int W64 = W < kW64 ? W : kW64;
  for (int k = 0; k < P.nlat; ++k) {
    LatDev& L = P.host[k];
    L.nsb = grid_for(L.g.Vh, T);
    L.nrb = grid_for(L.nrhs, W);
    L.nrb64 = grid_for(L.nrhs, W64);
    L.rb0 = rb0;
    L.rb640 = rb640;
    L.tile0 = tile;
    L.tile640 = tile64;
    L.nsb_b = grid_for(L.g.Vh, kTB);
    L.tile0_b = tileb;
    L.sbt0 = sbt;
    sbt += L.nsb_b;
    tileb += L.nsb_b * L.nrb;
    tile += L.nsb * L.nrb;
    tile64 += L.nsb * L.nrb64;
    rb0 += L.nrb;
    rb640 += L.nrb64;
  }
  P.W = W;
  P.WT = WT;
  P.T = T;
  P.ntiles = tile;
  P.ntiles64 = tile64;
  P.ntiles_b = tileb;
  P.nblk = rb0;
}

template <typename R>
int launch_mrhs_dslash_w(int WT, int G, int grid, int T, cudaStream_t s, const MArgs& a) {
  const dim3 block(T, G);
  if (T * G > kMaxThreads || T % 32) return SQCG_ERR_INVALID_ARG;
  switch (WT) {
    case 1: k_mrhs_dslash<R, 1><<<grid, block, 0, s>>>(a); break;
    case 2: k_mrhs_dslash<R, 2><<<grid, block, 0, s>>>(a); break;
    case 4: k_mrhs_dslash<R, 4><<<grid, block, 0, s>>>(a); break;
    default: return SQCG_ERR_INVALID_ARG;
  }
  SQCG_CUDA_TRY(cudaGetLastError());
  return SQCG_OK;
}

int launch_mrhs_blas(const BatchPlan& P, int op, cudaStream_t s) {
  BArgs a;
  a.lats = P.dev; a.nlat = P.nlat; a.op = op; a.st = P.st; a.partials = P.partials; a.max_nsb = P.max_nsb; a.W = P.W;
  int maxr = 0, nsb = 0;
  for (int k = 0; k < P.nlat; ++k) {
    maxr = P.nrhs[k] > maxr ? P.nrhs[k] : maxr;
    nsb += P.host[k].nsb_b;
  }
  k_mrhs_blas<<<dim3(nsb, (maxr + 1) / 2), kTB, 0, s>>>(a);
  SQCG_CUDA_TRY(cudaGetLastError());
  return SQCG_OK;
}

MArgs margs(const BatchPlan& P, int par, int in_vec, int epi, int gate, int write_p) {
  MArgs a;
  a.lats = P.dev; a.nlat = P.nlat; a.par = par; a.in_vec = in_vec; a.epi = epi; a.gate = gate; a.st = P.st;
  a.partials = P.partials; a.max_nsb = P.max_nsb; a.W = P.W; a.write_p = write_p;
  a.ntiles = 0;
  return a;
}

int launch_finish_b(const BatchPlan& P, int fin, int blas, cudaStream_t s) {
  k_batch_finish<<<P.nrhs_total, kBatchFinishThreads, 0, s>>>(P.st, P.dev, P.nlat, P.partials, P.max_nsb, fin, blas);
  SQCG_CUDA_TRY(cudaGetLastError());
  return SQCG_OK;
}

// The FP32 Dslash instantiations: (WT, SUB) for WT in {1, 2, 4} and SUB in {32, 16}.
typedef void (*SmemKernel)(MArgs);
int smem_index(int WT, int sub) {
  const int k = WT == 1 ? 0 : WT == 2 ? 1 : WT == 4 ? 2 : -1;
  if (k < 0 || (sub != 32 && sub != 16)) return -1;
  return 2 * k + (sub == 16 ? 1 : 0);
}
SmemKernel smem_kernel(int idx) {
  static const SmemKernel fns[6] = {k_mrhs_dslash_smem<1, 32>, k_mrhs_dslash_smem<1, 16>,
                                    k_mrhs_dslash_smem<2, 32>, k_mrhs_dslash_smem<2, 16>,
                                    k_mrhs_dslash_smem<4, 32>, k_mrhs_dslash_smem<4, 16>};
  return fns[idx];
}

// The shared-memory carveout of each FP32 Dslash instantiation: a smaller carveout leaves
// more of the SM's 256 KB to L1, which serves the neighbour gathers, at fewer resident blocks.
// Set outside graph capture (by the tuner, before the plan's graph is captured).
int set_carve(int WT, int sub, int carve) {
  std::lock_guard<std::recursive_mutex> lock(tune_mutex());
  static int cur[6] = {-2, -2, -2, -2, -2, -2};
  const int k = smem_index(WT, sub);
  if (k < 0) return SQCG_ERR_INVALID_ARG;
  if (cur[k] == carve) return SQCG_OK;
  SQCG_CUDA_TRY(cudaFuncSetAttribute((const void*)smem_kernel(k), cudaFuncAttributePreferredSharedMemoryCarveout,
                                     carve));
  cur[k] = carve;
  return SQCG_OK;
}

int launch_f32(const BatchPlan& P, int par, int in_vec, int epi, int gate, cudaStream_t s) {
  const int G = P.W / P.WT, T = P.T;
  if (!smem_shape_ok(P.W, P.WT, T, P.sub)) return SQCG_ERR_INVALID_ARG;
  const size_t smem = (size_t)kHops * 9 * T * sizeof(float2);
  std::lock_guard<std::recursive_mutex> lock(tune_mutex());
  static bool attr_set[6] = {false, false, false, false, false, false};  // per instantiation
  const int k = smem_index(P.WT, P.sub);
  if (k < 0) return SQCG_ERR_INVALID_ARG;
  if (!attr_set[k]) {
    SQCG_CUDA_TRY(cudaFuncSetAttribute((const void*)smem_kernel(k), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kHops * 9 * kMaxTSmem * (int)sizeof(float2)));
    attr_set[k] = true;
  }
  const MArgs a = margs(P, par, in_vec, epi, gate, 0);
  smem_kernel(k)<<<P.ntiles, dim3(T, G), smem, s>>>(a);
  SQCG_CUDA_TRY(cudaGetLastError());
  return SQCG_OK;
}

int launch_f64(const BatchPlan& P, int par, int in_vec, int epi, int gate, int write_p, cudaStream_t s) {
  const int W64 = P.W < kW64 ? P.W : kW64;
  return launch_mrhs_dslash_w<double>(W64, 1, P.ntiles64, P.T, s, margs(P, par, in_vec, epi, gate, write_p));
}

// x += xh for the RHS that take the reliable update (gated) or for all (the initial residual, and the
// final flush after the loop); split: also their float-float copies
int launch_flush_x(const BatchPlan& P, int gated, int split, cudaStream_t s) {
  int max_vh = 0;
  for (int k = 0; k < P.nlat; ++k) max_vh = P.host[k].g.Vh > max_vh ? P.host[k].g.Vh : max_vh;
  const int gx = (int)(((size_t)3 * max_vh + 255) / 256 < 1024 ? ((size_t)3 * max_vh + 255) / 256 : 1024);
  k_mrhs_flush_x<<<dim3(gx, P.nrhs_total), 256, 0, s>>>(P.dev, P.nlat, P.st, gated, split);
  SQCG_CUDA_TRY(cudaGetLastError());
  return SQCG_OK;
}

// The true-residual pass r = b - A x of the RHS that asked for it (gate = GATE_UPDATE) or of all of them
// (GATE_NONE, the initial residual), after x += xh: FP64 kernels, or the float-float ones.
int launch_true_resid_pass(const BatchPlan& P, int gate, int write_p, cudaStream_t s) {
  SQCG_TRY(launch_flush_x(P, gate == GATE_UPDATE ? 1 : 0, P.ff, s));
  if (!P.ff) {
    SQCG_TRY(launch_f64(P, 1, V_X, M_PLAIN, gate, 0, s));
    return launch_f64(P, 0, V_TMP64, M_TRUE_RESID, gate, write_p, s);
  }
  const int W64 = P.W < kW64 ? P.W : kW64;
  // several tiles per CTA (128 threads): the kernel keeps 128 registers per thread, and one-tile CTAs of
  // 32 threads would leave most warp slots empty
  if (P.T > 128 || 128 % P.T) return SQCG_ERR_INVALID_ARG;
  const int NB = 128 / P.T;
  const dim3 block(P.T, NB);
  const int grid = (P.ntiles64 + NB - 1) / NB;
  for (int pass = 0; pass < 2; ++pass) {
    MArgs a = pass == 0 ? margs(P, 1, V_XFF, M_PLAIN, gate, 0) : margs(P, 0, V_TMP64, M_TRUE_RESID, gate, write_p);
    a.ntiles = P.ntiles64;
    switch (W64) {
      case 1: k_mrhs_dslash_ff<1><<<grid, block, 0, s>>>(a); break;
      case 2: k_mrhs_dslash_ff<2><<<grid, block, 0, s>>>(a); break;
      case 4: k_mrhs_dslash_ff<4><<<grid, block, 0, s>>>(a); break;
      default: return SQCG_ERR_INVALID_ARG;
    }
    SQCG_CUDA_TRY(cudaGetLastError());
  }
  return SQCG_OK;
}

int upload_lats(BatchPlan& P, cudaStream_t s) {
  SQCG_CUDA_TRY(cudaMemcpyAsync(P.dev, P.host, sizeof(LatDev) * P.nlat, cudaMemcpyHostToDevice, s));
  return SQCG_OK;
}

// time the FP32 multi-RHS Dslash over the batch for each (W, WT, T); keep the fastest
int autotune(BatchPlan& P, cudaStream_t s) {
  std::lock_guard<std::recursive_mutex> lock(tune_mutex());
  tune_file_load();
  const std::string key = tune_key(P);
  auto it = tune_cache().find(key);
  int maxr = 0;
  for (int k = 0; k < P.nlat; ++k) maxr = P.nrhs[k] > maxr ? P.nrhs[k] : maxr;
  if (tune_pin().W > 0) {
    const TuneChoice& c = tune_pin();
    layout_tiles(P, c.W, c.WT, c.T);
    P.carve = c.carve;
    P.sub = c.sub;
    SQCG_TRY(set_carve(P.WT, P.sub, P.carve));
    return upload_lats(P, s);
  }
  if (it != tune_cache().end()) {
    layout_tiles(P, it->second.W, it->second.WT, it->second.T);
    P.carve = it->second.carve;
    P.sub = it->second.sub;
    SQCG_TRY(set_carve(P.WT, P.sub, P.carve));
    return upload_lats(P, s);
  }
  cudaEvent_t e0, e1;
  SQCG_CUDA_TRY(cudaEventCreate(&e0));
  SQCG_CUDA_TRY(cudaEventCreate(&e1));
  float best = 1e30f;
  TuneChoice bestc = {1, 1, 128, -1, 32};
  // 12 for batches of 9 to 12 right-hand sides (the 11-shift refinement, 12-pole rational
  // functions), where a block of 16 would leave a quarter of its RHS groups empty
  const int Ws[] = {1, 2, 4, 8, 12, 16};
  const int WTs[] = {1, 2, 4};
  const int Ts[] = {32, 64, 128, 256};
  int rc = SQCG_OK;
  // time one configuration (5 launches after 2 warm-up launches); keep it if fastest
  auto trial = [&](int W, int WT, int T, int carve, int sub) {
    layout_tiles(P, W, WT, T);
    P.carve = carve;
    P.sub = sub;
    if ((rc = set_carve(WT, sub, carve)) != SQCG_OK) return;
    if ((rc = upload_lats(P, s)) != SQCG_OK) return;
    for (int rep = 0; rep < 2 && rc == SQCG_OK; ++rep) rc = launch_f32(P, 1, V_P, M_PLAIN, GATE_NONE, s);
    if (rc != SQCG_OK) return;
    cudaEventRecord(e0, s);
    for (int rep = 0; rep < 5 && rc == SQCG_OK; ++rep) rc = launch_f32(P, 1, V_P, M_PLAIN, GATE_NONE, s);
    cudaEventRecord(e1, s);
    if (rc != SQCG_OK) return;
    if (cudaEventSynchronize(e1) != cudaSuccess) { rc = SQCG_ERR_CUDA; return; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (getenv("SQCG_TUNE_VERBOSE"))
      fprintf(stderr, "sqcg tune %s W=%d WT=%d T=%d carve=%d sub=%d %.4f ms\n", key.c_str(), W, WT, T, carve, sub,
              ms / 5);
    if (ms < best) { best = ms; bestc = {W, WT, T, carve, sub}; }
  };
  // 1: block shapes at the driver's default carveout
  for (int W : Ws) {
    if (W > 1 && W / 2 >= maxr) break;  // wider blocks than any lattice's RHS count only add idle lanes
    for (int WT : WTs) {
      if (WT > W) break;
      const int G = W / WT;
      for (int T : Ts) {
        if (T * G > kMaxThreads || T > kMaxTSmem) break;
        for (int sub : {32, 16}) {
          if (!smem_shape_ok(W, WT, T, sub)) continue;
          trial(W, WT, T, -1, sub);
          if (rc != SQCG_OK) break;
        }
        if (rc != SQCG_OK) break;
      }
      if (rc != SQCG_OK) break;
    }
    if (rc != SQCG_OK) break;
  }
  // 2: the best W and WT again with smaller shared-memory carveouts (more L1 for the gathers)
  if (rc == SQCG_OK) {
    const int W = bestc.W, WT = bestc.WT, G = W / WT, sub = bestc.sub;
    const int carves[] = {25, 50, 75};
    for (int T : Ts) {
      if (T * G > kMaxThreads || T > kMaxTSmem) break;
      for (int cv : carves) {
        trial(W, WT, T, cv, sub);
        if (rc != SQCG_OK) break;
      }
      if (rc != SQCG_OK) break;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != SQCG_OK) return rc;
  tune_cache()[key] = bestc;
  tune_file_store(key, bestc);
  layout_tiles(P, bestc.W, bestc.WT, bestc.T);
  P.carve = bestc.carve;
  P.sub = bestc.sub;
  SQCG_TRY(set_carve(P.WT, P.sub, P.carve));
  return upload_lats(P, s);
}

// per lattice: r, p, Ap, tmp and the partial solutions xh in RHS pairs (FP32), tmp64 (FP64 or
// float-float) and, with float-float reliable updates, xff
size_t work_bytes(int nrhs, size_t Vh, int ff) {
  const size_t nf = (size_t)((nrhs + 1) / 2) * 2 * 3 * Vh;
  return 5 * nf * sizeof(float2) + (size_t)(ff ? 2 : 1) * nrhs * 3 * Vh * sizeof(double2);
}

void destroy_plan(BatchPlan* P) {
  if (!P) return;
  if (P->exec) cudaGraphExecDestroy(P->exec);
  for (int k = 0; k < P->nlat; ++k) cudaFree(P->work[k]);
  cudaFree(P->dev);
  cudaFree(P->partials);
  cudaFree(P->st);
  if (P->st_host) cudaFreeHost(P->st_host);
  free(P);
}

int build_plan(int nctx, sqcg_ctx* const* ctx, const int* nrhs, const void* const* b, int b_shared, void* const* x,
               BatchPlan** out, cudaStream_t s) {
  BatchPlan* P = (BatchPlan*)calloc(1, sizeof(BatchPlan));
  if (!P) return SQCG_ERR_NO_MEMORY;
  P->nlat = nctx;
  P->b_shared = b_shared;
  P->ff = ctx[0]->ru_arith == SQCG_FF ? 1 : 0;
  int total = 0, max_vh = 0;
  for (int k = 0; k < nctx; ++k) {
    sqcg_ctx* c = ctx[k];
    P->ctx[k] = c;
    P->gen[k] = sqcg_links_generation(c);
    P->nrhs[k] = nrhs[k];
    P->b[k] = b[k];
    P->x[k] = x[k];
    LatDev& L = P->host[k];
    L.g = c->g;
    const size_t Vh = c->g.Vh;
    const int nl32 = c->recon ? 6 : 9;
    for (int par = 0; par < 2; ++par) {
      L.fat32[par] = c->fat32 + (size_t)par * 4 * 9 * Vh;
      L.lng32[par] = c->lng32 + (size_t)par * 4 * nl32 * Vh;
      L.fat64[par] = c->fat64 + (size_t)par * 4 * 9 * Vh;
      L.lng64[par] = c->lng64 + (size_t)par * 4 * 9 * Vh;
      L.fatff[par] = c->fatff + (size_t)par * 4 * 9 * Vh;
      L.lngff[par] = c->lngff + (size_t)par * 4 * 9 * Vh;
    }
    L.nl32 = nl32;
    L.recon = c->recon ? 1 : 0;
    L.inv_s0_f = (float)(c->recon ? 1.0 / c->long_scale : 1.0);
    L.inv_s0_d = c->recon ? 1.0 / c->long_scale : 1.0;
    L.rhs0 = total;
    L.nrhs = nrhs[k];
    L.b = (const double2*)b[k];
    L.b_stride = b_shared ? 0 : 3 * Vh;
    L.x = (double2*)x[k];
    // FP32 vectors: (nrhs + 1) / 2 RHS pairs each (see pv); FP64 tmp64: nrhs vectors
    if (cudaMalloc(&P->work[k], work_bytes(nrhs[k], Vh, P->ff)) != cudaSuccess) {
      cudaGetLastError();
      destroy_plan(P);
      return SQCG_ERR_NO_MEMORY;
    }
    const size_t nf = (size_t)((nrhs[k] + 1) / 2) * 2 * 3 * Vh;
    float2* w = (float2*)P->work[k];
    L.r = w; L.p = w + nf; L.Ap = w + 2 * nf; L.tmp = w + 3 * nf; L.xh = w + 4 * nf;
    L.tmp64 = (double2*)(w + 5 * nf);
    L.xff = P->ff ? (float4*)(L.tmp64 + (size_t)nrhs[k] * 3 * Vh) : nullptr;
    total += nrhs[k];
    if ((int)Vh > max_vh) max_vh = (int)Vh;
  }
  P->nrhs_total = total;
  P->max_nsb = grid_for(max_vh, kMinT);  // the smallest site block the tuner tries
  bool ok = cudaMalloc((void**)&P->dev, sizeof(LatDev) * nctx) == cudaSuccess &&
            cudaMalloc((void**)&P->partials, sizeof(double) * (size_t)total * P->max_nsb) == cudaSuccess &&
            cudaMalloc((void**)&P->st, sizeof(BatchState)) == cudaSuccess &&
            cudaMallocHost((void**)&P->st_host, sizeof(BatchState)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    destroy_plan(P);
    return SQCG_ERR_NO_MEMORY;
  }
  SQCG_CUDA_TRY(cudaMemsetAsync(P->st, 0, sizeof(BatchState), s));
  for (int k = 0; k < nctx; ++k)
    SQCG_CUDA_TRY(cudaMemsetAsync(P->work[k], 0, work_bytes(nrhs[k], ctx[k]->g.Vh, P->ff), s));
  int rc = autotune(*P, s);
  if (rc != SQCG_OK) { destroy_plan(P); return rc; }
  *out = P;
  return SQCG_OK;
}

// One iteration in three parts: head (D_oe p; A p + <p,Ap>; x, r update; ctl), the FP64
// reliable update r = b - A x of the blocks that asked for it, tail (p update; loop ctl)
int enqueue_head(BatchPlan& P, cudaStream_t s) {
  SQCG_TRY(launch_f32(P, 1, V_P, M_PLAIN, GATE_ITER, s));
  SQCG_TRY(launch_f32(P, 0, V_TMP, M_NORMAL_DOT, GATE_ITER, s));
  SQCG_TRY(launch_finish_b(P, BFIN_PAP, 0, s));
  SQCG_TRY(launch_mrhs_blas(P, B_UPDATE, s));
  SQCG_TRY(launch_finish_b(P, BFIN_UPDATE, 1, s));
  k_batch_ctl_update<<<1, 32, 0, s>>>(P.st, P.dev, P.nlat, P.W);
  SQCG_CUDA_TRY(cudaGetLastError());
  return SQCG_OK;
}

int enqueue_reliable(BatchPlan& P, cudaStream_t s) {
  SQCG_TRY(launch_true_resid_pass(P, GATE_UPDATE, 0, s));
  return launch_finish_b(P, BFIN_TRUE, 0, s);
}

int enqueue_tail(BatchPlan& P, cudaStream_t s) {
  SQCG_TRY(launch_mrhs_blas(P, B_XPAY, s));
  k_batch_ctl_loop<<<1, 32, 0, s>>>(P.st, P.dev, P.nlat, P.W);
  SQCG_CUDA_TRY(cudaGetLastError());
  return SQCG_OK;
}

// The same loop launched one kernel at a time (SQCG_LAUNCH_MODE=eager), the host reading the
// state where the graph's conditional nodes would branch. Kernel-level profilers do not see
// kernels inside conditional graph nodes; this gives them the identical kernel sequence.
int run_eager(BatchPlan& P, cudaStream_t s) {
  BatchState* h = P.st_host;
  auto read = [&]() -> int {
    SQCG_CUDA_TRY(cudaMemcpyAsync(h, P.st, sizeof(BatchState), cudaMemcpyDeviceToHost, s));
    SQCG_CUDA_TRY(cudaStreamSynchronize(s));
    return SQCG_OK;
  };
  const int limit = h->loop_limit;  // the host bounds the loop too, whatever the device state says
  for (int it = 0; it < limit; ++it) {
    SQCG_TRY(enqueue_head(P, s));
    SQCG_TRY(read());
    int upd = 0;
    for (int j = 0; j < P.nblk; ++j) upd |= h->blk_update[j];
    if (upd) SQCG_TRY(enqueue_reliable(P, s));
    SQCG_TRY(enqueue_tail(P, s));
    SQCG_TRY(read());
    int act = 0;
    for (int j = 0; j < P.nblk; ++j) act |= h->blk_active[j];
    if (!act || h->loop_count >= h->loop_limit) break;  // the WHILE condition of k_batch_ctl_loop
  }
  return SQCG_OK;
}

// Capture the loop: WHILE { head; IF { reliable }; tail }
int capture_plan(BatchPlan& P) {
  cudaStream_t cs = P.ctx[0]->cap_stream;
  cudaGraph_t top = nullptr;
  SQCG_CUDA_TRY(cudaGraphCreate(&top, 0));
  int rc = SQCG_OK;
  cudaGraphConditionalHandle hw = 0, hif = 0;
  cudaGraphNodeParams wp = {};
  cudaGraphNode_t wnode = nullptr;
  cudaGraph_t ifbody = nullptr;
  do {
    if (cudaGraphConditionalHandleCreate(&hw, top, 1, cudaGraphCondAssignDefault) != cudaSuccess) { rc = SQCG_ERR_CUDA; break; }
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = hw;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    if (cudaGraphAddNode(&wnode, top, nullptr, nullptr, 0, &wp) != cudaSuccess) { rc = SQCG_ERR_CUDA; break; }
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { rc = SQCG_ERR_CUDA; break; }
    rc = enqueue_head(P, cs);
    if (rc == SQCG_OK) {
      cudaStreamCaptureStatus status;
      cudaGraph_t capg = nullptr;
      const cudaGraphNode_t* deps = nullptr;
      size_t ndeps = 0;
      cudaGraphNodeParams ip = {};
      cudaGraphNode_t inode = nullptr;
      if (cudaStreamGetCaptureInfo(cs, &status, nullptr, &capg, &deps, nullptr, &ndeps) != cudaSuccess ||
          cudaGraphConditionalHandleCreate(&hif, capg, 0, 0) != cudaSuccess) {
        rc = SQCG_ERR_CUDA;
      } else {
        ip.type = cudaGraphNodeTypeConditional;
        ip.conditional.handle = hif;
        ip.conditional.type = cudaGraphCondTypeIf;
        ip.conditional.size = 1;
        if (cudaGraphAddNode(&inode, capg, deps, nullptr, ndeps, &ip) != cudaSuccess ||
            cudaStreamUpdateCaptureDependencies(cs, &inode, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess)
          rc = SQCG_ERR_CUDA;
        else
          ifbody = ip.conditional.phGraph_out[0];
      }
    }
    if (rc == SQCG_OK) rc = enqueue_tail(P, cs);
    cudaGraph_t got = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &got);
    if (rc != SQCG_OK) break;
    if (e != cudaSuccess) { rc = SQCG_ERR_CUDA; break; }
    if (cudaStreamBeginCaptureToGraph(cs, ifbody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { rc = SQCG_ERR_CUDA; break; }
    rc = enqueue_reliable(P, cs);
    e = cudaStreamEndCapture(cs, &got);
    if (rc != SQCG_OK) break;
    if (e != cudaSuccess) { rc = SQCG_ERR_CUDA; break; }
    if (cudaGraphInstantiate(&P.exec, top, 0) != cudaSuccess) { rc = SQCG_ERR_CUDA; break; }
  } while (0);
  if (rc == SQCG_ERR_CUDA) sqcg_set_last_cuda_error(cudaGetLastError(), "batched graph", __FILE__, __LINE__);
  cudaGraphDestroy(top);
  P.h_while = hw;
  P.h_if = hif;
  return rc;
}

bool plan_matches(const BatchPlan* P, int nctx, sqcg_ctx* const* ctx, const int* nrhs, const void* const* b,
                  int b_shared, void* const* x) {
  if (!P || P->nlat != nctx || P->b_shared != b_shared) return false;
  if (P->ff != (ctx[0]->ru_arith == SQCG_FF ? 1 : 0)) return false;
  for (int k = 0; k < nctx; ++k)
    if (P->ctx[k] != ctx[k] || P->gen[k] != sqcg_links_generation(ctx[k]) || P->nrhs[k] != nrhs[k] ||
        P->b[k] != b[k] || P->x[k] != x[k])
      return false;
  return true;
}

}  // namespace

void free_batch_plan(sqcg_ctx* ctx) {
  destroy_plan(ctx->batch);
  ctx->batch = nullptr;
}

// The batched loop over explicit per-RHS shifts and tolerances (RHS in lattice
// order). b_shared: every RHS of a lattice solves for the same source b[k].
int batched_solve(int nctx, sqcg_ctx* const* ctx, const int* nrhs, const double* sigma, const double* tol,
                  const void* const* b, int b_shared, void* const* x, int max_iter, sqcg_info* info) {
  const auto t0 = std::chrono::steady_clock::now();
  if (nctx < 1 || nctx > SQCG_MAX_LATTICES || !ctx || !nrhs || !sigma || !tol || !b || !x || max_iter <= 0)
    return SQCG_ERR_INVALID_ARG;
  int total = 0;
  for (int k = 0; k < nctx; ++k) {
    if (!ctx[k] || nrhs[k] < 1 || !b[k] || !x[k] || b[k] == x[k]) return SQCG_ERR_INVALID_ARG;
    if (((uintptr_t)b[k] | (uintptr_t)x[k]) & 15) return SQCG_ERR_INVALID_ARG;
    if (!ctx[k]->have_links) return SQCG_ERR_NO_LINKS;
    for (int j = 0; j < k; ++j)
      if (ctx[j] == ctx[k] || x[j] == x[k]) return SQCG_ERR_INVALID_ARG;
    total += nrhs[k];
    if (total > SQCG_MAX_BATCH_RHS) return SQCG_ERR_INVALID_ARG;
  }
  for (int j = 0; j < total; ++j)
    if (!isfinite(sigma[j]) || sigma[j] < 0 || !(tol[j] > 0)) return SQCG_ERR_INVALID_ARG;
  sqcg_ctx* c0 = ctx[0];
  cudaStream_t s = c0->stream;
  if (!plan_matches(c0->batch, nctx, ctx, nrhs, b, b_shared, x)) {
    SQCG_CUDA_TRY(cudaStreamSynchronize(s));
    free_batch_plan(c0);
    SQCG_TRY(build_plan(nctx, ctx, nrhs, b, b_shared, x, &c0->batch, s));
  }
  BatchPlan& P = *c0->batch;

  // state: per-RHS scalars
  BatchState* h = P.st_host;
  memset(h, 0, sizeof(BatchState));
  h->nrhs = total;
  h->nblk = P.nblk;
  h->max_iter = max_iter;
  h->update_interval = c0->ru_interval;
  h->delta2 = c0->ru_delta * c0->ru_delta;
  for (int k = 0; k < nctx; ++k)
    for (int j = 0; j < nrhs[k]; ++j) {
      const int g = P.host[k].rhs0 + j;
      RhsScalars& r = h->r[g];
      r.sigma = sigma[g];
      r.stop_rr = tol[g] * tol[g];
      r.active = 1;
      r.status = SQCG_OK;
    }
  for (int j = 0; j < P.nblk; ++j) h->blk_active[j] = 1;
  SQCG_CUDA_TRY(cudaMemcpyAsync(P.st, h, sizeof(BatchState), cudaMemcpyHostToDevice, s));
  for (int k = 0; k < nctx; ++k)  // the FP32 partial solutions start at zero
    SQCG_CUDA_TRY(cudaMemsetAsync(P.host[k].xh, 0,
                                  (size_t)((nrhs[k] + 1) / 2) * 2 * 3 * ctx[k]->g.Vh * sizeof(float2), s));
  // |b|^2 per RHS; r = b - A x0 in FP64 (x holds the initial guess), p = r
  SQCG_TRY(launch_mrhs_blas(P, B_NORM_B, s));
  SQCG_TRY(launch_finish_b(P, BFIN_BB, 1, s));
  // |x0|^2 per RHS: when every initial guess is zero (the usual start) the initial residual
  // is exactly b, and the FP64 passes of b - A x0 are skipped
  SQCG_TRY(launch_mrhs_blas(P, B_NORM_X, s));
  SQCG_TRY(launch_finish_b(P, BFIN_XX, 1, s));
  SQCG_CUDA_TRY(cudaMemcpyAsync(h, P.st, sizeof(BatchState), cudaMemcpyDeviceToHost, s));
  SQCG_CUDA_TRY(cudaStreamSynchronize(s));
  bool x0_zero = true;
  for (int j = 0; j < total; ++j) x0_zero = x0_zero && h->r[j].pAp == 0.0;
  int launches = 4;
  if (x0_zero) {
    SQCG_TRY(launch_mrhs_blas(P, B_INIT_B, s));
    SQCG_TRY(launch_finish_b(P, BFIN_INIT, 1, s));
    launches += 2;
  } else {
    for (int j = 0; j < P.nblk; ++j) h->blk_update[j] = 1;
    SQCG_CUDA_TRY(cudaMemcpyAsync(P.st->blk_update, h->blk_update, sizeof(int) * P.nblk, cudaMemcpyHostToDevice, s));
    SQCG_TRY(launch_true_resid_pass(P, GATE_NONE, 1, s));
    SQCG_TRY(launch_finish_b(P, BFIN_INIT, 0, s));
    launches += 3;
  }
  SQCG_CUDA_TRY(cudaMemcpyAsync(h, P.st, sizeof(BatchState), cudaMemcpyDeviceToHost, s));
  SQCG_CUDA_TRY(cudaStreamSynchronize(s));
  int any = 0;
  for (int j = 0; j < total; ++j) {
    if (h->r[j].bb == 0.0 && h->r[j].active) {  // b = 0: x = 0 is the solution
      h->r[j].active = 0;
      h->r[j].status = SQCG_OK;
    }
    any |= h->r[j].active;
  }
  for (int k = 0; k < nctx; ++k)
    for (int j = 0; j < nrhs[k]; ++j)
      if (h->r[P.host[k].rhs0 + j].bb == 0.0)
        SQCG_CUDA_TRY(cudaMemsetAsync((double2*)x[k] + (size_t)j * 3 * ctx[k]->g.Vh, 0,
                                      (size_t)3 * ctx[k]->g.Vh * sizeof(double2), s));
  if (any) {
    const char* mode = getenv("SQCG_LAUNCH_MODE");
    const bool eager = mode && strcmp(mode, "eager") == 0;
    if (!eager && !P.exec) SQCG_TRY(capture_plan(P));
    for (int k = 0; k < P.nlat; ++k)
      for (int rb = 0; rb < P.host[k].nrb; ++rb) {
        int a = 0;
        for (int w = rb * P.W; w < (rb + 1) * P.W && w < P.host[k].nrhs; ++w) a |= h->r[P.host[k].rhs0 + w].active;
        h->blk_active[P.host[k].rb0 + rb] = a;
      }
    for (int j = 0; j < P.nblk; ++j) h->blk_update[j] = 0;
    for (int j = 0; j < total; ++j) h->r[j].need_update = 0;
    h->h_while = P.h_while;
    h->h_if = P.h_if;
    h->loop_count = 0;
    h->loop_limit = max_iter + 4;
    h->use_graph = eager ? 0 : 1;
    SQCG_CUDA_TRY(cudaMemcpyAsync(P.st, h, sizeof(BatchState), cudaMemcpyHostToDevice, s));
    if (eager) {
      SQCG_TRY(run_eager(P, s));
    } else {
      SQCG_CUDA_TRY(cudaGraphLaunch(P.exec, s));
      SQCG_CUDA_TRY(cudaMemcpyAsync(h, P.st, sizeof(BatchState), cudaMemcpyDeviceToHost, s));
      SQCG_CUDA_TRY(cudaStreamSynchronize(s));
    }
    // whatever the partial solutions still hold (nothing for an RHS whose last update converged)
    SQCG_TRY(launch_flush_x(P, 0, 0, s));
    SQCG_CUDA_TRY(cudaStreamSynchronize(s));
    launches += h->loop_count * 8 + h->if_runs * 4 + 1;
  }
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  int worst = SQCG_OK;
  for (int j = 0; j < total; ++j) {
    const RhsScalars& r = h->r[j];
    int st = r.active ? SQCG_ERR_NOT_CONVERGED : r.status;
    if (info) {
      info[j].iters = r.iter;
      info[j].reliable_updates = r.updates;
      info[j].status = st;
      info[j].true_rel_resid = r.bb > 0 ? sqrt(r.rr_true / r.bb) : 0.0;
      info[j].seconds = secs;
      info[j].launches = launches;
    }
    if (st != SQCG_OK && worst == SQCG_OK) worst = st;
  }
  return worst;
}

extern "C" int sqcg_cg_solve_batched(int nctx, sqcg_ctx* const* ctx, const int* nrhs, const double* mass,
                                     const void* const* b, void* const* x, double tol, int max_iter,
                                     sqcg_info* info) {
  if (nctx < 1 || nctx > SQCG_MAX_LATTICES || !ctx || !nrhs || !mass || !(tol > 0)) return SQCG_ERR_INVALID_ARG;
  double sig[SQCG_MAX_BATCH_RHS], tols[SQCG_MAX_BATCH_RHS];
  int total = 0;
  for (int k = 0; k < nctx; ++k) {
    if (nrhs[k] < 1 || !isfinite(mass[k]) || total + nrhs[k] > SQCG_MAX_BATCH_RHS) return SQCG_ERR_INVALID_ARG;
    for (int j = 0; j < nrhs[k]; ++j, ++total) {
      sig[total] = 4.0 * mass[k] * mass[k];
      tols[total] = tol;
    }
  }
  return batched_solve(nctx, ctx, nrhs, sig, tols, b, 0, x, max_iter, info);
}

extern "C" int sqcg_batched_tuning(const sqcg_ctx* ctx, int* W, int* T) {
  if (!ctx || !ctx->batch || !W || !T) return SQCG_ERR_INVALID_ARG;
  *W = ctx->batch->W;
  *T = ctx->batch->T;
  return SQCG_OK;
}

extern "C" int sqcg_batched_tuning_ex(const sqcg_ctx* ctx, int* W, int* WT, int* T, int* carve, int* warp_sites) {
  if (!ctx || !ctx->batch) return SQCG_ERR_INVALID_ARG;
  const BatchPlan& P = *ctx->batch;
  if (W) *W = P.W;
  if (WT) *WT = P.WT;
  if (T) *T = P.T;
  if (carve) *carve = P.carve;
  if (warp_sites) *warp_sites = P.sub;
  return SQCG_OK;
}

extern "C" int sqcg_batched_pin_tuning(int W, int WT, int T, int carve, int warp_sites) {
  std::lock_guard<std::recursive_mutex> lock(tune_mutex());
  if (W == 0) {
    tune_pin() = {0, 0, 0, -1, 32};
    return SQCG_OK;
  }
  if (warp_sites == 0) warp_sites = 32;
  if ((W != 1 && W != 2 && W != 4 && W != 8 && W != 12 && W != 16) || (WT != 1 && WT != 2 && WT != 4) || WT > W)
    return SQCG_ERR_INVALID_ARG;
  if (!smem_shape_ok(W, WT, T, warp_sites)) return SQCG_ERR_INVALID_ARG;
  if (carve < -1 || carve > 100) return SQCG_ERR_INVALID_ARG;
  tune_pin() = {W, WT, T, carve, warp_sites};
  return SQCG_OK;
}
