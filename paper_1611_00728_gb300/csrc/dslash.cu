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
#include "solver_device.cuh"
#include "sqcg_internal.cuh"

namespace {

template <typename R> struct V2;
template <> struct V2<double> { typedef double2 T; };
template <> struct V2<float> { typedef float2 T; };

template <typename R2>
__device__ __forceinline__ R2 ldg2(const R2* p) { return __ldg(p); }

template <typename R2>
__device__ __forceinline__ R2 mk(decltype(R2().x) a, decltype(R2().x) b) { R2 r; r.x = a; r.y = b; return r; }

// acc += U v   (U row-major 3x3 complex)
template <typename R, typename R2>
__device__ __forceinline__ void acc_mv(R2 (&acc)[3], const R2 (&U)[9], const R2 (&v)[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const R2 u = U[a * 3 + b];
      acc[a].x = fma(u.x, v[b].x, acc[a].x);
      acc[a].x = fma(-u.y, v[b].y, acc[a].x);
      acc[a].y = fma(u.x, v[b].y, acc[a].y);
      acc[a].y = fma(u.y, v[b].x, acc[a].y);
    }
  }
}

// acc -= U^dagger v
template <typename R, typename R2>
__device__ __forceinline__ void sub_mdv(R2 (&acc)[3], const R2 (&U)[9], const R2 (&v)[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const R2 u = U[b * 3 + a];  // conj(U[b][a]) v[b]
      acc[a].x = fma(-u.x, v[b].x, acc[a].x);
      acc[a].x = fma(-u.y, v[b].y, acc[a].x);
      acc[a].y = fma(-u.x, v[b].y, acc[a].y);
      acc[a].y = fma(u.y, v[b].x, acc[a].y);
    }
  }
}

template <typename R, typename R2, bool RECON>
__device__ __forceinline__ void load_link(R2 (&U)[9], const R2* __restrict__ base, int stride, int idx, R inv_s) {
  if (!RECON) {
#pragma unroll
    for (int e = 0; e < 9; ++e) U[e] = ldg2(base + (size_t)e * stride + idx);
  } else {
#pragma unroll
    for (int e = 0; e < 6; ++e) U[e] = ldg2(base + (size_t)e * stride + idx);
    // row2 = conj(row0 x row1) / s
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int k = (j + 1) % 3, l = (j + 2) % 3;
      const R2 ak = U[k], al = U[l], bk = U[3 + k], bl = U[3 + l];
      R re = ak.x * bl.x - ak.y * bl.y - (al.x * bk.x - al.y * bk.y);
      R im = ak.x * bl.y + ak.y * bl.x - (al.x * bk.y + al.y * bk.x);
      U[6 + j] = mk<R2>(re * inv_s, -im * inv_s);
    }
  }
}

template <typename R2>
__device__ __forceinline__ void load_vec(R2 (&v)[3], const R2* __restrict__ in, int Vh, int idx) {
#pragma unroll
  for (int c = 0; c < 3; ++c) v[c] = ldg2(in + (size_t)c * Vh + idx);
}

template <typename R>
struct DArgs {
  Geom g;
  int par;                         // output parity
  const typename V2<R>::T* fat_p;  // fat links of the output parity
  const typename V2<R>::T* fat_q;  // fat links of the input parity
  const typename V2<R>::T* lng_p;
  const typename V2<R>::T* lng_q;
  const typename V2<R>::T* fatb_p;  // 8-way: -F_mu(n - mu)^+ stored at the output site n
  const typename V2<R>::T* lngb_p;  // 8-way: -L_mu(n - 3mu)^+ stored at n
  int nl;                          // elements per long link (9 or 6)
  R inv_s0;                        // 1 / global long-link scale (recon)
  const typename V2<R>::T* in;
  void* out;
  void* out2;
  const void* y;
  const void* y3;
  const double2* b;
  double sigma;
  const double* sigma_dev;
  SolverState* st;
  double* partials;
  int gate, fin;
};

// D at output site i of parity a.par; returns the three colour components.
// EIGHT: the backward links are read, already daggered and negated, at i.
template <typename R, bool RECON, bool EIGHT>
__device__ __forceinline__ void dslash_site(const DArgs<R>& a, int i, typename V2<R>::T (&acc)[3]) {
  typedef typename V2<R>::T R2;
  const Geom& g = a.g;
  const int Vh = g.Vh;
  const int xh = i % g.Lxh;
  int r = i / g.Lxh;
  const int y = r % g.Ly;
  r /= g.Ly;
  const int z = r % g.Lz;
  const int t = r / g.Lz;
  const int x = 2 * xh + ((y + z + t + a.par) & 1);
  const int row = i - xh;  // half index of (0, y, z, t)

#pragma unroll
  for (int c = 0; c < 3; ++c) acc[c] = mk<R2>(R(0), R(0));

  R2 U[9], v[3];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    // eta_mu(n) and the boundary signs, needed only to rebuild 12-real long links
    R inv_s_f = R(1), inv_s_b = R(1);
    if (RECON) {
      int e = 0;
      if (mu == 1) e = x;
      if (mu == 2) e = x + y;
      if (mu == 3) e = x + y + z;
      const R eta = (e & 1) ? R(-1) : R(1);
      inv_s_f = eta * a.inv_s0;
      inv_s_b = eta * a.inv_s0;
      if (mu == 3 && g.apbc) {
        if (t + 3 >= g.Lt) inv_s_f = -inv_s_f;
        if (t < 3) inv_s_b = -inv_s_b;
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
        load_link<R, R2, false>(U, a.fat_p + (size_t)mu * 9 * Vh, Vh, i, R(1));
        load_vec(v, a.in, Vh, fwd);
        acc_mv<R>(acc, U, v);
        load_vec(v, a.in, Vh, bwd);
        if (EIGHT) {
          load_link<R, R2, false>(U, a.fatb_p + (size_t)mu * 9 * Vh, Vh, i, R(1));
          acc_mv<R>(acc, U, v);
        } else {
          load_link<R, R2, false>(U, a.fat_q + (size_t)mu * 9 * Vh, Vh, bwd, R(1));
          sub_mdv<R>(acc, U, v);
        }
      } else {
        load_link<R, R2, RECON>(U, a.lng_p + (size_t)mu * a.nl * Vh, Vh, i, inv_s_f);
        load_vec(v, a.in, Vh, fwd);
        acc_mv<R>(acc, U, v);
        load_vec(v, a.in, Vh, bwd);
        if (EIGHT) {  // -L^+ = (-s) V^+: its third row is rebuilt with the scale -s
          load_link<R, R2, RECON>(U, a.lngb_p + (size_t)mu * a.nl * Vh, Vh, i, -inv_s_b);
          acc_mv<R>(acc, U, v);
        } else {
          load_link<R, R2, RECON>(U, a.lng_q + (size_t)mu * a.nl * Vh, Vh, bwd, inv_s_b);
          sub_mdv<R>(acc, U, v);
        }
      }
    }
  }
}

constexpr int kThreads = 128;

template <typename R, typename RO, bool RECON, bool EIGHT, int EPI>
__global__ void __launch_bounds__(kThreads, (sizeof(R) == 4 && EPI == EPI_SR_DOTS2) ? 9 : 0) k_dslash(DArgs<R> a) {
  typedef typename V2<R>::T R2;
  typedef typename V2<RO>::T O2;
  if (!gate_open(a.st, a.gate)) return;
  const int Vh = a.g.Vh;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double part = 0.0, part2 = 0.0, part3 = 0.0;
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
      part = (double)rs;
      part2 = (double)rq;
      part3 = (double)rr;
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
  if constexpr (EPI == EPI_NORMAL_DOT || EPI == EPI_TRUE_RESID) {
    if (a.fin != FIN_NONE) block_partial(part, a.partials);
  }
  if constexpr (EPI == EPI_SR_DOTS) {
    if (a.fin != FIN_NONE) block_partial3(part, part2, part3, a.partials);
  } else if constexpr (EPI == EPI_SR_DOTS2) {  // sums 1 and 3 (the second comes from the update kernel)
    if (a.fin != FIN_NONE) {
      block_sum2(part, part3);
      if (threadIdx.x == 0) {
        a.partials[blockIdx.x] = part;
        a.partials[2 * gridDim.x + blockIdx.x] = part3;
      }
    }
  }
  (void)part2; (void)part3;
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
  switch (L.epi) {
    case EPI_PLAIN: k_dslash<R, RO, RECON, EIGHT, EPI_PLAIN><<<grid, kThreads, 0, s>>>(a); break;
    case EPI_NORMAL: k_dslash<R, RO, RECON, EIGHT, EPI_NORMAL><<<grid, kThreads, 0, s>>>(a); break;
    case EPI_NORMAL_DOT: k_dslash<R, RO, RECON, EIGHT, EPI_NORMAL_DOT><<<grid, kThreads, 0, s>>>(a); break;
    case EPI_TRUE_RESID: k_dslash<R, RO, RECON, EIGHT, EPI_TRUE_RESID><<<grid, kThreads, 0, s>>>(a); break;
    case EPI_SR_DOTS: k_dslash<R, RO, RECON, EIGHT, EPI_SR_DOTS><<<grid, kThreads, 0, s>>>(a); break;
    case EPI_SR_DOTS2: k_dslash<R, RO, RECON, EIGHT, EPI_SR_DOTS2><<<grid, kThreads, 0, s>>>(a); break;
    default: return SQCG_ERR_INVALID_ARG;
  }
  SQCG_CUDA_TRY(cudaGetLastError());
  if (reduces)
    return L.epi == EPI_SR_DOTS    ? launch_finish_sr(ctx, grid, grid, grid, L.gate, s)
           : L.epi == EPI_SR_DOTS2 ? launch_finish_sr(ctx, grid, sr_update_partials(ctx), blas_grid(ctx), L.gate, s)
                                   : launch_finish(ctx, grid, L.fin, L.gate, s);
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
