// Improved-staggered Dslash in float-float ("double-single") arithmetic, for
// the passes that need more than FP32: the reliable-update recomputation of the
// true residual r = b - A x in the mixed-precision solvers.
//
// Why: the operator is the same 16-hop sum as the FP32 and FP64 kernels
// (arXiv:1611.00728 Sec. 3, the staggered dslash), but on this GPU FP64 FMAs
// issue at 1/64 of the FP32 rate, so the FP64 Dslash (576 FMAs per site) is
// bound by arithmetic at about 0.5 ms on a 32^4 lattice, 2.6x slower than its
// 2400 bytes per site take from HBM. Here every real number is an unevaluated
// sum hi + lo of two floats (a 48-bit significand), and each product is
// accumulated with error-free transformations on the FP32 pipe:
//   TwoProduct(a, b) = (p, e): p = fl(a b), e = fma(a, b, -p)  (exact: a b = p + e; Dekker 1971, with FMA)
//   TwoSum(s, p)     = (s', t): s' = fl(s + p), t = (s - (s' - b')) + (p - b'), b' = s' - s  (exact; Knuth)
// The cross terms a_hi b_lo + a_lo b_hi go straight into the low word: their
// rounding is of order 2^-48 relative. The result carries a relative error of
// order 1e-14 (checked against the FP64 oracle at 1e-12), far below what a
// true residual at a 1e-8 tolerance needs.
//
// Storage: a complex number is a float4 (re_hi, re_lo, im_hi, im_lo), 16 bytes
// like a double2, so links ([parity][mu][9][Vh], forward only, phases folded)
// and vectors ([3][Vh]) have the FP64 layout and the kernel moves the FP64
// bytes: 2400 per output site. One thread computes one output site.
#include "ff_arith.cuh"
#include "solver_device.cuh"
#include "sqcg_internal.cuh"

namespace {

constexpr int kThreads = 128;

__device__ __forceinline__ void ld_link(float4 (&U)[9], const float4* __restrict__ base, int Vh, int idx) {
#pragma unroll
  for (int e = 0; e < 9; ++e) U[e] = __ldg(base + (size_t)e * Vh + idx);
}

__device__ __forceinline__ void ld_vec(float4 (&v)[3], const float4* __restrict__ in, int Vh, int idx) {
#pragma unroll
  for (int c = 0; c < 3; ++c) v[c] = __ldg(in + (size_t)c * Vh + idx);
}

struct FArgs {
  Geom g;
  int par;
  const float4* fat_p;  // forward links of the output parity
  const float4* fat_q;  // forward links of the input parity (backward hops)
  const float4* lng_p;
  const float4* lng_q;
  const float4* in;     // float-float input vector on the other parity
  float4* out_ff;       // FFE_PLAIN: float-float output
  float2* out32;        // FFE_TRUE_RESID: r = b - sigma x + D in, rounded to FP32
  const double2* x;     // FFE_TRUE_RESID: FP64 x on the output parity
  const double2* b;     // FFE_TRUE_RESID: FP64 right-hand side
  double sigma;
  const double* sigma_dev;
  SolverState* st;
  double* partials;
  int gate, fin;
};

enum { FFE_PLAIN = 0, FFE_TRUE_RESID = 1 };

template <int EPI>
__global__ void __launch_bounds__(kThreads) k_dslash_ff(FArgs a) {
  if (!gate_open(a.st, a.gate)) return;
  const Geom& g = a.g;
  const int Vh = g.Vh;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double part = 0.0;
  if (i < Vh) {
    const int xh = i % g.Lxh;
    int r = i / g.Lxh;
    const int y = r % g.Ly;
    r /= g.Ly;
    const int z = r % g.Lz;
    const int t = r / g.Lz;
    const int x = 2 * xh + ((y + z + t + a.par) & 1);
    const int row = i - xh;
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
        const float4* fl = (k == 0) ? a.fat_p : a.lng_p;
        const float4* bl = (k == 0) ? a.fat_q : a.lng_q;
        ld_link(U, fl + (size_t)mu * 9 * Vh, Vh, i);
        ld_vec(v, a.in, Vh, fwd);
        ff_mv(acc, U, v);
        ld_link(U, bl + (size_t)mu * 9 * Vh, Vh, bwd);
        ld_vec(v, a.in, Vh, bwd);
        ff_mdv_sub(acc, U, v);
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      ff_norm(acc[c].x, acc[c].y);
      ff_norm(acc[c].z, acc[c].w);
    }
    if constexpr (EPI == FFE_PLAIN) {
#pragma unroll
      for (int c = 0; c < 3; ++c) a.out_ff[(size_t)c * Vh + i] = acc[c];
    } else {  // r = b - sigma x + D in, the sum formed in FP64
      const double sig = a.sigma_dev ? *a.sigma_dev : a.sigma;
      double nrm = 0.0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double2 xc = __ldg(a.x + (size_t)c * Vh + i);
        const double2 bc = __ldg(a.b + (size_t)c * Vh + i);
        const double re = bc.x - sig * xc.x + ((double)acc[c].x + (double)acc[c].y);
        const double im = bc.y - sig * xc.y + ((double)acc[c].z + (double)acc[c].w);
        a.out32[(size_t)c * Vh + i] = make_float2((float)re, (float)im);
        nrm += re * re + im * im;
      }
      part = nrm;
    }
  }
  if constexpr (EPI == FFE_TRUE_RESID) {
    if (a.fin != FIN_NONE) block_partial(part, a.partials);
  }
}

__global__ void k_split_ff(const double2* __restrict__ in, float4* __restrict__ out, size_t n) {
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
    out[k] = split_ff(in[k]);
}

// x += xh (FP32 partial solution, added in FP64), xh = 0, and x_ff = the float-float copy of the new x
__global__ void k_flush_split(double2* __restrict__ x, float2* __restrict__ xh, float4* __restrict__ xff, int n,
                              const SolverState* st, int gate) {
  if (!gate_open(st, gate)) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    double2 v = x[k];
    if (xh) {
      const float2 h = xh[k];
      v.x += (double)h.x;
      v.y += (double)h.y;
      x[k] = v;
      xh[k] = make_float2(0.f, 0.f);
    }
    xff[k] = split_ff(v);
  }
}

}  // namespace

int launch_dslash_ff(sqcg_ctx* ctx, const FFLaunch& L, cudaStream_t s) {
  if (!ctx->have_links || !ctx->fatff) return SQCG_ERR_NO_LINKS;
  if ((L.out_parity != 0 && L.out_parity != 1) || !L.in) return SQCG_ERR_INVALID_ARG;
  FArgs a = {};
  a.g = ctx->g;
  a.par = L.out_parity;
  const size_t Vh = ctx->g.Vh;
  const int p = L.out_parity, q = 1 - L.out_parity;
  a.fat_p = ctx->fatff + (size_t)p * 4 * 9 * Vh;
  a.fat_q = ctx->fatff + (size_t)q * 4 * 9 * Vh;
  a.lng_p = ctx->lngff + (size_t)p * 4 * 9 * Vh;
  a.lng_q = ctx->lngff + (size_t)q * 4 * 9 * Vh;
  a.in = static_cast<const float4*>(L.in);
  a.sigma = L.sigma;
  a.sigma_dev = L.sigma_dev;
  a.st = ctx->st;
  a.partials = ctx->partials;
  a.gate = L.gate;
  a.fin = L.fin;
  if ((L.gate != GATE_NONE || L.fin != FIN_NONE) && (!ctx->st || !ctx->partials)) return SQCG_ERR_INVALID_ARG;
  const int grid = grid_for(ctx->g.Vh, kThreads);
  if (L.true_resid) {
    if (!L.out32 || !L.x || !L.b) return SQCG_ERR_INVALID_ARG;
    if (L.fin != FIN_NONE && grid > ctx->max_blocks) return SQCG_ERR_INVALID_ARG;
    a.out32 = static_cast<float2*>(L.out32);
    a.x = static_cast<const double2*>(L.x);
    a.b = static_cast<const double2*>(L.b);
    k_dslash_ff<FFE_TRUE_RESID><<<grid, kThreads, 0, s>>>(a);
    SQCG_CUDA_TRY(cudaGetLastError());
    if (L.fin != FIN_NONE) return launch_finish(ctx, grid, L.fin, L.gate, s);
    return SQCG_OK;
  }
  if (!L.out_ff) return SQCG_ERR_INVALID_ARG;
  a.out_ff = static_cast<float4*>(L.out_ff);
  k_dslash_ff<FFE_PLAIN><<<grid, kThreads, 0, s>>>(a);
  SQCG_CUDA_TRY(cudaGetLastError());
  return SQCG_OK;
}

int launch_split_ff(const double2* in, float4* out, size_t n, cudaStream_t s) {
  const size_t want = (n + 255) / 256;
  const int grid = (int)(want < 65535 ? want : 65535);
  k_split_ff<<<grid > 0 ? grid : 1, 256, 0, s>>>(in, out, n);
  SQCG_CUDA_TRY(cudaGetLastError());
  return SQCG_OK;
}

int launch_flush_split(sqcg_ctx* ctx, double2* x, float2* xh, float4* xff, int gate, cudaStream_t s) {
  const int n = ctx->g.Vh * 3;
  k_flush_split<<<blas_grid(ctx), 256, 0, s>>>(x, xh, xff, n, ctx->st, gate);
  SQCG_CUDA_TRY(cudaGetLastError());
  return SQCG_OK;
}
