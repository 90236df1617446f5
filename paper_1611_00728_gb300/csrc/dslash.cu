// Improved-staggered Dslash on CUDA cores (arXiv:1611.00728 Sec. 3: the
// generated "staggered dslash" kernel; Sec. 4: its least-data model bandwidth).
//
//   (D psi)(n) = sum_mu [ F_mu(n) psi(n+mu) - F_mu(n-mu)^+ psi(n-mu)
//                       + L_mu(n) psi(n+3mu) - L_mu(n-3mu)^+ psi(n-3mu) ]
//
// with eta_mu and the boundary sign already folded into F and L at load time.
// One thread computes one output site of one parity. Links are stored
// [parity][mu][elem][Vh] so that a warp reads each matrix element of 32
// consecutive sites as one contiguous segment; colour vectors are [3][Vh].
// The backward hop reads the forward link of the neighbour and applies the
// dagger in registers (forward-only storage, the standard MILC layout), or,
// with the 8-way option of the FP32 copy, reads -U^+ stored at the site itself.
// Neighbour indices are computed from the site coordinates (no index tables).
// With 12-real long links (FP32 copy only) the third row is rebuilt as
// conj(row0 x row1) / s, s = s0 * eta_mu * boundary sign of that link.
#include "dslash_core.cuh"
namespace {

using namespace dcore;

constexpr int kThreads = 128;

template <typename R, typename RO, bool RECON, bool EIGHT, int EPI>
__global__ void __launch_bounds__(kThreads, (sizeof(R) == 4 && EPI == EPI_SR_DOTS2) ? 9 : 0) k_dslash(DArgs<R> a) {
  typedef typename V2<R>::T R2;
  typedef typename V2<RO>::T O2;
  pdl_wait();
  pdl_launch_dependents();
  if (!gate_open(a.st, a.gate)) return;
  const int Vh = a.g.Vh;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double part = 0.0;
  float srs = 0.f, srq = 0.f, srr = 0.f;  // EPI_SR_DOTS*: the site's <r,s>, <r,q>, |r|^2 (FP32)
  float sdot = 0.f;                       // EPI_NORMAL_DOT with FP32 vectors: the site's dot
  if (i < Vh) {
    R2 acc[3];
    dslash_site<R, RECON, EIGHT>(a, i, acc);
    O2* out = static_cast<O2*>(a.out);
    if constexpr (EPI == EPI_PLAIN) {
#pragma unroll
      for (int c = 0; c < 3; ++c) out[(size_t)c * Vh + i] = mk<O2>((RO)acc[c].x, (RO)acc[c].y);
    } else if constexpr (EPI == EPI_NORMAL || EPI == EPI_NORMAL_DOT) {
      const R sig = (R)(a.sigma_dev ? *a.sigma_dev : a.sigma);
      const R2* yv = static_cast<const R2*>(a.y);
      R dot = R(0);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const R2 yc = ldg2(yv + (size_t)c * Vh + i);
        O2 o = mk<O2>((RO)(sig * yc.x - acc[c].x), (RO)(sig * yc.y - acc[c].y));
        out[(size_t)c * Vh + i] = o;
        dot = fma(yc.x, o.x, fma(yc.y, o.y, dot));
      }
      part = (double)dot;
      sdot = (float)dot;
    } else if constexpr (EPI == EPI_SR_DOTS || EPI == EPI_SR_DOTS2) {  // s = sigma r - D in; <r,s>, [<r,q>], |r|^2
      const R sig = (R)(a.sigma_dev ? *a.sigma_dev : a.sigma);
      const R2* rv = static_cast<const R2*>(a.y);
      const R2* qv = static_cast<const R2*>(a.y3);
      R rs = R(0), rq = R(0), rr = R(0);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const size_t k = (size_t)c * Vh + i;
        const R2 rc = ldg2(rv + k);
        O2 o = mk<O2>((RO)(sig * rc.x - acc[c].x), (RO)(sig * rc.y - acc[c].y));
        out[k] = o;
        rs = fma(rc.x, o.x, fma(rc.y, o.y, rs));
        rr = fma(rc.x, rc.x, fma(rc.y, rc.y, rr));
        if constexpr (EPI == EPI_SR_DOTS) {
          const R2 qc = ldg2(qv + k);
          rq = fma(rc.x, qc.x, fma(rc.y, qc.y, rq));
        }
      }
      srs = rs;
      srq = rq;
      srr = rr;
    } else {  // EPI_TRUE_RESID: out = b - sigma*x + D in, in FP64
      const double sig = a.sigma_dev ? *a.sigma_dev : a.sigma;
      const double2* xv = static_cast<const double2*>(a.y);
      O2* out2 = static_cast<O2*>(a.out2);
      double nrm = 0.0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double2 xc = __ldg(xv + (size_t)c * Vh + i);
        const double2 bc = __ldg(a.b + (size_t)c * Vh + i);
        const double re = bc.x - sig * xc.x + (double)acc[c].x;
        const double im = bc.y - sig * xc.y + (double)acc[c].y;
        O2 o = mk<O2>((RO)re, (RO)im);
        out[(size_t)c * Vh + i] = o;
        if (out2) out2[(size_t)c * Vh + i] = o;
        nrm += re * re + im * im;
      }
      part = nrm;
    }
  }
  if constexpr ((EPI == EPI_NORMAL_DOT && sizeof(R) == 8) || EPI == EPI_TRUE_RESID) {
    if (a.fin != FIN_NONE) block_partial(part, a.partials);
  } else if constexpr (EPI == EPI_NORMAL_DOT) {  // FP32: the site's dot is FP32; float-float partials
    if (a.fin != FIN_NONE) {
      float2 v[1] = {make_float2(sdot, 0.f)};
      block_sum_ffs<1>(v);
      if (threadIdx.x == 0) ffs_slots(a.partials)[blockIdx.x] = v[0];
    }
  }
  if constexpr (EPI == EPI_SR_DOTS) {  // float-float partials of the three sums
    if (a.fin != FIN_NONE) {
      float2 v[3] = {make_float2(srs, 0.f), make_float2(srq, 0.f), make_float2(srr, 0.f)};
      block_sum_ffs<3>(v);
      if (threadIdx.x == 0) {
        float2* slot = ffs_slots(a.partials);
        slot[blockIdx.x] = v[0];
        slot[gridDim.x + blockIdx.x] = v[1];
        slot[2 * gridDim.x + blockIdx.x] = v[2];
      }
    }
  } else if constexpr (EPI == EPI_SR_DOTS2) {  // sums 1 and 3 (the second comes from the update kernel)
    if (a.fin != FIN_NONE) {
      float2 v[2] = {make_float2(srs, 0.f), make_float2(srr, 0.f)};
      block_sum_ffs<2>(v);
      if (threadIdx.x == 0) {
        float2* slot = ffs_slots(a.partials);
        slot[blockIdx.x] = v[0];
        slot[2 * gridDim.x + blockIdx.x] = v[1];
      }
    }
  }
  (void)srs; (void)srq; (void)srr; (void)sdot;
}

template <typename R, typename RO, bool RECON, bool EIGHT>
int launch_t(sqcg_ctx* ctx, const DslashLaunch& L, cudaStream_t s) {
  typedef typename V2<R>::T R2;
  DArgs<R> a;
  a.g = ctx->g;
  a.par = L.out_parity;
  const int p = L.out_parity, q = 1 - L.out_parity;
  const size_t Vh = ctx->g.Vh;
  const int nl = RECON ? 6 : 9;  // the 12-real form exists for the FP32 copy only
  const R2* fat = reinterpret_cast<const R2*>(L.prec == SQCG_F64 ? (const void*)ctx->fat64 : (const void*)ctx->fat32);
  const R2* lng = reinterpret_cast<const R2*>(L.prec == SQCG_F64 ? (const void*)ctx->lng64 : (const void*)ctx->lng32);
  a.fat_p = fat + (size_t)p * 4 * 9 * Vh;
  a.fat_q = fat + (size_t)q * 4 * 9 * Vh;
  a.lng_p = lng + (size_t)p * 4 * nl * Vh;
  a.lng_q = lng + (size_t)q * 4 * nl * Vh;
  a.fatb_p = EIGHT ? reinterpret_cast<const R2*>(ctx->fatb32) + (size_t)p * 4 * 9 * Vh : nullptr;
  a.lngb_p = EIGHT ? reinterpret_cast<const R2*>(ctx->lngb32) + (size_t)p * 4 * nl * Vh : nullptr;
  a.nl = nl;
  a.inv_s0 = (R)(RECON ? 1.0 / ctx->long_scale : 1.0);
  a.in = static_cast<const R2*>(L.in);
  a.out = L.out;
  a.out2 = L.out2;
  a.y = L.y;
  a.y3 = L.y3;
  a.b = static_cast<const double2*>(L.b);
  a.sigma = L.sigma;
  a.sigma_dev = L.sigma_dev;
  a.st = ctx->st;
  a.partials = ctx->partials;
  a.gate = L.gate;
  a.fin = L.fin;
  if ((L.gate != GATE_NONE || L.fin != FIN_NONE) && (ctx->st == nullptr || ctx->partials == nullptr))
    return SQCG_ERR_INVALID_ARG;
  const int grid = grid_for(ctx->g.Vh, kThreads);
  const bool sr = L.epi == EPI_SR_DOTS || L.epi == EPI_SR_DOTS2;
  const bool reduces = (L.epi == EPI_NORMAL_DOT || sr || L.epi == EPI_TRUE_RESID) && L.fin != FIN_NONE;
  if (reduces && grid > ctx->max_blocks) return SQCG_ERR_INVALID_ARG;  // partials hold 3 sums and more
  // programmatic dependent launch where the caller says a kernel precedes this one, and for the
  // finisher, which always follows the Dslash
  const bool pdl = L.pdl && ctx->pdl, fpdl = ctx->pdl != 0;
  void (*kern)(DArgs<R>) = nullptr;
  switch (L.epi) {
    case EPI_PLAIN: kern = k_dslash<R, RO, RECON, EIGHT, EPI_PLAIN>; break;
    case EPI_NORMAL: kern = k_dslash<R, RO, RECON, EIGHT, EPI_NORMAL>; break;
    case EPI_NORMAL_DOT: kern = k_dslash<R, RO, RECON, EIGHT, EPI_NORMAL_DOT>; break;
    case EPI_TRUE_RESID: kern = k_dslash<R, RO, RECON, EIGHT, EPI_TRUE_RESID>; break;
    case EPI_SR_DOTS: kern = k_dslash<R, RO, RECON, EIGHT, EPI_SR_DOTS>; break;
    case EPI_SR_DOTS2: kern = k_dslash<R, RO, RECON, EIGHT, EPI_SR_DOTS2>; break;
    default: return SQCG_ERR_INVALID_ARG;
  }
  SQCG_CUDA_TRY(launch_kernel(kern, grid, kThreads, 0, s, pdl, a));
  if (reduces)
    return L.epi == EPI_SR_DOTS ? launch_finish_sr(ctx, grid, grid, grid, L.gate, s, fpdl)
           : L.epi == EPI_SR_DOTS2
               ? launch_finish_sr(ctx, grid, sr_update_partials(ctx), blas_grid(ctx), L.gate, s, fpdl)
           : (L.epi == EPI_NORMAL_DOT && sizeof(R) == 4) ? launch_finish_ffs(ctx, grid, L.fin, L.gate, s, fpdl)
                                                          : launch_finish(ctx, grid, L.fin, L.gate, s, fpdl);
  return SQCG_OK;
}

template <typename R, typename RO>
int launch_r(sqcg_ctx* ctx, const DslashLaunch& L, cudaStream_t s) {
  if constexpr (sizeof(R) == 4) {  // 12-real and 8-way forms exist for the FP32 copy only
    if (ctx->eightway)
      return ctx->recon ? launch_t<R, RO, true, true>(ctx, L, s) : launch_t<R, RO, false, true>(ctx, L, s);
    if (ctx->recon) return launch_t<R, RO, true, false>(ctx, L, s);
  }
  return launch_t<R, RO, false, false>(ctx, L, s);
}

}  // namespace

int launch_dslash(sqcg_ctx* ctx, const DslashLaunch& L, cudaStream_t s) {
  if (!ctx->have_links) return SQCG_ERR_NO_LINKS;
  if (L.out_parity != 0 && L.out_parity != 1) return SQCG_ERR_INVALID_ARG;
  if (L.epi == EPI_TRUE_RESID) {
    if (L.prec != SQCG_F64 || !L.b || !L.y) return SQCG_ERR_INVALID_ARG;
    return L.out_prec == SQCG_F64 ? launch_r<double, double>(ctx, L, s) : launch_r<double, float>(ctx, L, s);
  }
  if (L.out_prec != L.prec) return SQCG_ERR_INVALID_ARG;
  if ((L.epi == EPI_NORMAL || L.epi == EPI_NORMAL_DOT || L.epi == EPI_SR_DOTS || L.epi == EPI_SR_DOTS2) && !L.y)
    return SQCG_ERR_INVALID_ARG;
  if (L.epi == EPI_SR_DOTS && !L.y3) return SQCG_ERR_INVALID_ARG;
  if (L.prec == SQCG_F64) return launch_r<double, double>(ctx, L, s);
  if (L.prec == SQCG_F32) return launch_r<float, float>(ctx, L, s);
  return SQCG_ERR_INVALID_ARG;
}
