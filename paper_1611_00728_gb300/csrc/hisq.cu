// HISQ link construction on the GPU: thin links -> fat and long links in FP64.
//
// The paper's benchmark application evolves the HISQ action (Sec. 4), whose CG
// consumes these links; the construction is that of the HISQ action (Follana
// et al., hep-lat/0610092):
//   V = smear(U, level 1)  one link + 3-, 5-, 7-link staples (fat7)
//   W = V (V^+ V)^(-1/2)   U(3) projection
//   fat = smear(W, level 2) the same staples + the Lepage 5-link staple
//   long = naik W_mu(n) W_mu(n+mu) W_mu(n+2mu)
// Links are unphased and periodic; the staggered phases and the time-boundary
// sign are folded in afterwards, when the result is loaded into a context.
//
// One smearing level is three kernels over full-lattice structure-of-arrays
// fields [field][element][V] (site fastest, coalesced):
//   A: S^s_{mu nu}(n), the single-sign 3-staples (24 fields), and their sums
//      S3_{mu nu} = S^+ + S^- (12 fields);
//   B: Z_{mu nu}(n) = c5 (S3_{mu rho} + S3_{mu sig})(n)
//                    + c7 (wrap_rho S3_{mu sig} + wrap_sig S3_{mu rho})(n),
//      with S3 = S^+ + S^- and {rho, sig} the two directions other than mu, nu;
//   C: F_mu(n) = c1 U_mu(n) + sum_{nu,s} [ c3 S^s_{mu nu}(n)
//                + wrap^s_nu( Z_{mu nu} + cL S^s_{mu nu} )(n) ],
// where wrap^+_d X (n) = U_d(n) X(n+d) U_d(n+mu)^+ and
//       wrap^-_d X (n) = U_d(n-d)^+ X(n-d) U_d(n-d+mu).
// Expanding C gives every 5-link staple (outer nu, inner rho) with c5, every
// 7-link staple (outer nu, middle rho, inner sig) with c7 and every Lepage
// staple (nu twice, same sign) with cL, at 48 3x3 products per link per level
// (12 in A, 24 in B, 12 in C).
//
// Arithmetic: on this GPU an FP64 FMA issues at 1/64 of the FP32 rate, and the FP64 version of these
// kernels ran with the FP64 pipe 90-97% busy. The staple products therefore run in float-float
// arithmetic: every real is an unevaluated sum hi + lo of two floats (48-bit significand), a complex
// number a float4 (re_hi, re_lo, im_hi, im_lo) of the same 16 bytes as a double2, and each product
// is accumulated by error-free transformations on the FP32 pipe (ff_arith.cuh: TwoProduct with an
// FMA, Dekker 1971; TwoSum, Knuth). The fields in the workspace are float-float; the thin links are
// split at the first kernel, the U(3) projection runs in FP64 on the joined values (its Newton
// steps need division and square roots), and the outputs are joined back to FP64.
#include <math.h>
#include <string.h>

#include "ff_arith.cuh"
#include "sqcg_internal.cuh"

namespace {

constexpr int kThreads = 128;

struct Lat {
  int L[4];
  long V;
};

// ---- float-float 3x3 complex matrices (the staple products) ----
struct F3 {
  float4 e[9];
};

// acc += a b, acc += a conj(b), acc += conj(a) b (float-float complex; the low words are not
// renormalised in between: fnorm after a few terms)
__device__ __forceinline__ void fcfma(float4& acc, float4 a, float4 b) {
  ff_acc(acc.x, acc.y, a.x, a.y, b.x, b.y);
  ff_acc(acc.x, acc.y, -a.z, -a.w, b.z, b.w);
  ff_acc(acc.z, acc.w, a.x, a.y, b.z, b.w);
  ff_acc(acc.z, acc.w, a.z, a.w, b.x, b.y);
}
__device__ __forceinline__ void fcfma_cb(float4& acc, float4 a, float4 b) {
  ff_acc(acc.x, acc.y, a.x, a.y, b.x, b.y);
  ff_acc(acc.x, acc.y, a.z, a.w, b.z, b.w);
  ff_acc(acc.z, acc.w, a.z, a.w, b.x, b.y);
  ff_acc(acc.z, acc.w, -a.x, -a.y, b.z, b.w);
}
__device__ __forceinline__ void fcfma_ca(float4& acc, float4 a, float4 b) {
  ff_acc(acc.x, acc.y, a.x, a.y, b.x, b.y);
  ff_acc(acc.x, acc.y, a.z, a.w, b.z, b.w);
  ff_acc(acc.z, acc.w, a.x, a.y, b.z, b.w);
  ff_acc(acc.z, acc.w, -a.z, -a.w, b.x, b.y);
}
__device__ __forceinline__ void fnorm(float4& v) {
  ff_norm(v.x, v.y);
  ff_norm(v.z, v.w);
}
__device__ __forceinline__ F3 fzero() {
  F3 m;
#pragma unroll
  for (int e = 0; e < 9; ++e) m.e[e] = make_float4(0.f, 0.f, 0.f, 0.f);
  return m;
}

__device__ __forceinline__ F3 fmm(const F3& A, const F3& B) {  // A B
  F3 C;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int k = 0; k < 3; ++k) fcfma(s, A.e[i * 3 + k], B.e[k * 3 + j]);
      fnorm(s);
      C.e[i * 3 + j] = s;
    }
  return C;
}
__device__ __forceinline__ F3 fmm_nd(const F3& A, const F3& B) {  // A B^+
  F3 C;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int k = 0; k < 3; ++k) fcfma_cb(s, A.e[i * 3 + k], B.e[j * 3 + k]);
      fnorm(s);
      C.e[i * 3 + j] = s;
    }
  return C;
}
__device__ __forceinline__ F3 fmm_dn(const F3& A, const F3& B) {  // A^+ B
  F3 C;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int k = 0; k < 3; ++k) fcfma_ca(s, A.e[k * 3 + i], B.e[k * 3 + j]);
      fnorm(s);
      C.e[i * 3 + j] = s;
    }
  return C;
}
// C += A B and C += A B^+, renormalised after the three terms of each element
__device__ __forceinline__ void fmm_acc(F3& C, const F3& A, const F3& B) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
#pragma unroll
      for (int k = 0; k < 3; ++k) fcfma(C.e[i * 3 + j], A.e[i * 3 + k], B.e[k * 3 + j]);
      fnorm(C.e[i * 3 + j]);
    }
}
__device__ __forceinline__ void fmm_nd_acc(F3& C, const F3& A, const F3& B) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
#pragma unroll
      for (int k = 0; k < 3; ++k) fcfma_cb(C.e[i * 3 + j], A.e[i * 3 + k], B.e[j * 3 + k]);
      fnorm(C.e[i * 3 + j]);
    }
}
// Y += a X for a float-float real a = (ah, al)
__device__ __forceinline__ void faxpy(F3& Y, float2 a, const F3& X) {
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    ff_acc(Y.e[e].x, Y.e[e].y, a.x, a.y, X.e[e].x, X.e[e].y);
    ff_acc(Y.e[e].z, Y.e[e].w, a.x, a.y, X.e[e].z, X.e[e].w);
    fnorm(Y.e[e]);
  }
}
// Y += X (float-float: TwoSum of the high words, low words added to the error, renormalised)
__device__ __forceinline__ void ff_add(float& h, float& l, float bh, float bl) {
  const float s = __fadd_rn(h, bh);
  const float v = __fsub_rn(s, h);
  float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, v)), __fsub_rn(bh, v));
  e = __fadd_rn(e, __fadd_rn(l, bl));
  h = __fadd_rn(s, e);
  l = __fsub_rn(e, __fsub_rn(h, s));
}
__device__ __forceinline__ void faddto(F3& Y, const F3& X) {
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    ff_add(Y.e[e].x, Y.e[e].y, X.e[e].x, X.e[e].y);
    ff_add(Y.e[e].z, Y.e[e].w, X.e[e].z, X.e[e].w);
  }
}

// field k of a structure-of-arrays float-float buffer: elements [k][e][V]
__device__ __forceinline__ F3 fld(const float4* __restrict__ f, int k, long V, long n) {
  F3 m;
  const float4* p = f + (size_t)k * 9 * V + n;
#pragma unroll
  for (int e = 0; e < 9; ++e) m.e[e] = __ldg(p + (size_t)e * V);
  return m;
}
__device__ __forceinline__ void fst(float4* __restrict__ f, int k, long V, long n, const F3& m) {
  float4* p = f + (size_t)k * 9 * V + n;
#pragma unroll
  for (int e = 0; e < 9; ++e) p[(size_t)e * V] = m.e[e];
}

__device__ __forceinline__ void coords(const Lat& g, long n, int c[4]) {
  c[0] = (int)(n % g.L[0]);
  n /= g.L[0];
  c[1] = (int)(n % g.L[1]);
  n /= g.L[1];
  c[2] = (int)(n % g.L[2]);
  c[3] = (int)(n / g.L[2]);
}
// lex index of c + k1 e_d1 + k2 e_d2 (periodic; |k| <= 3 < L)
__device__ __forceinline__ long nb(const Lat& g, const int c[4], int d1, int k1, int d2 = 0, int k2 = 0) {
  int cc[4] = {c[0], c[1], c[2], c[3]};
  cc[d1] += k1;
  cc[d2] += k2;
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    if (cc[d] < 0) cc[d] += g.L[d];
    if (cc[d] >= g.L[d]) cc[d] -= g.L[d];
  }
  return cc[0] + (long)g.L[0] * (cc[1] + (long)g.L[1] * (cc[2] + (long)g.L[2] * cc[3]));
}
// the i-th direction other than mu (increasing order), and the inverse
__device__ __forceinline__ int other(int mu, int i) { return i + (i >= mu ? 1 : 0); }
__device__ __forceinline__ int other_index(int mu, int d) { return d - (d > mu ? 1 : 0); }
// staple fields: single-sign S^s_{mu d} at (mu*3 + index of d)*2 + s, their sum S3_{mu d} at 24 + mu*3 + index
constexpr int kNumS = 36;
__device__ __forceinline__ int s3_field(int mu, int d) { return 24 + mu * 3 + other_index(mu, d); }

// wrap^s_d X (n) for the direction-mu field X given at the displaced site
__device__ __forceinline__ F3 wrap(const Lat& g, const float4* __restrict__ U, const int c[4], long n, int mu, int d,
                                   int s, const F3& Xd) {
  if (s == 0) {
    const F3 a = fld(U, d, g.V, n);
    const F3 b = fld(U, d, g.V, nb(g, c, mu, 1));
    return fmm_nd(fmm(a, Xd), b);
  }
  const F3 a = fld(U, d, g.V, nb(g, c, d, -1));
  const F3 b = fld(U, d, g.V, nb(g, c, d, -1, mu, 1));
  return fmm(fmm_dn(a, Xd), b);
}

// acc += wrap^s_d X (n)
__device__ __forceinline__ void wrap_acc(F3& acc, const Lat& g, const float4* __restrict__ U, const int c[4], long n,
                                         int mu, int d, int s, const F3& Xd) {
  if (s == 0) {
    const F3 a = fld(U, d, g.V, n);
    const F3 b = fld(U, d, g.V, nb(g, c, mu, 1));
    fmm_nd_acc(acc, fmm(a, Xd), b);
    return;
  }
  const F3 a = fld(U, d, g.V, nb(g, c, d, -1));
  const F3 b = fld(U, d, g.V, nb(g, c, d, -1, mu, 1));
  fmm_acc(acc, fmm_dn(a, Xd), b);
}

// host AoS [V][4][9] (FP64) -> [mu][e][V] (float-float)
__global__ void __launch_bounds__(kThreads) k_links_to_fields(Lat g, const double2* __restrict__ aos,
                                                              float4* __restrict__ U) {
  const long n = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.V) return;
  const int mu = blockIdx.y;
#pragma unroll
  for (int e = 0; e < 9; ++e) U[((size_t)mu * 9 + e) * g.V + n] = split_ff(aos[((size_t)n * 4 + mu) * 9 + e]);
}

// A: 3-staples S^+_{mu nu}, S^-_{mu nu} (s = 0 forward, 1 backward) and S3_{mu nu} = S^+ + S^-
__global__ void __launch_bounds__(kThreads) k_staple3(Lat g, const float4* __restrict__ U, float4* __restrict__ S) {
  const long n = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.V) return;
  const int f = blockIdx.y;  // mu*3 + nu index
  const int mu = f / 3, nu = other(mu, f % 3);
  int c[4];
  coords(g, n, c);
  const F3 sp = wrap(g, U, c, n, mu, nu, 0, fld(U, mu, g.V, nb(g, c, nu, 1)));
  fst(S, 2 * f, g.V, n, sp);
  F3 sm = wrap(g, U, c, n, mu, nu, 1, fld(U, mu, g.V, nb(g, c, nu, -1)));
  fst(S, 2 * f + 1, g.V, n, sm);
  faddto(sm, sp);
  fst(S, 24 + f, g.V, n, sm);
}

// B: Z_{mu nu} = c5 (S3_{mu rho} + S3_{mu sig}) + c7 (wrap_rho S3_{mu sig} + wrap_sig S3_{mu rho})
// (c5, c7 as float-float pairs; a zero coefficient skips its term)
__global__ void __launch_bounds__(kThreads) k_staple57(Lat g, const float4* __restrict__ U,
                                                       const float4* __restrict__ S, float2 c5, float2 c7,
                                                       float4* __restrict__ Z) {
  const long n = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.V) return;
  const int f = blockIdx.y;  // mu*3 + nu index
  const int mu = f / 3, nu = other(mu, f % 3);
  int rs[2], k = 0;
  for (int d = 0; d < 4; ++d)
    if (d != mu && d != nu) rs[k++] = d;
  int c[4];
  coords(g, n, c);
  F3 z = fzero();
  if (c5.x != 0.f) {
    F3 t = fld(S, s3_field(mu, rs[0]), g.V, n);
    faddto(t, fld(S, s3_field(mu, rs[1]), g.V, n));
    faxpy(z, c5, t);
  }
  if (c7.x != 0.f) {
    F3 w = fzero();
    for (int q = 0; q < 2; ++q) {
      const int d = rs[q], inner = rs[1 - q];
      for (int s = 0; s < 2; ++s) {
        const F3 x = fld(S, s3_field(mu, inner), g.V, nb(g, c, d, s == 0 ? 1 : -1));
        wrap_acc(w, g, U, c, n, mu, d, s, x);
      }
    }
    faxpy(z, c7, w);
  }
  fst(Z, f, g.V, n, z);
}

// C: F_mu = c1 U_mu + sum_{nu,s} [ c3 S^s_{mu nu} + wrap^s_nu (Z_{mu nu} + cL S^s_{mu nu}) ]
// out: float-float structure of arrays [mu][e][V], or FP64 in the host order [V][4][9] when aos != 0
__global__ void __launch_bounds__(kThreads) k_smear_links(Lat g, const float4* __restrict__ U,
                                                          const float4* __restrict__ S,
                                                          const float4* __restrict__ Z, float2 c1, float2 c3,
                                                          float2 cL, int use_z, int aos, void* __restrict__ out) {
  const long n = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.V) return;
  const int mu = blockIdx.y;
  int c[4];
  coords(g, n, c);
  F3 F = fzero();
  faxpy(F, c1, fld(U, mu, g.V, n));
  for (int i = 0; i < 3; ++i) {
    const int nu = other(mu, i);
    if (c3.x != 0.f) faxpy(F, c3, fld(S, 24 + mu * 3 + i, g.V, n));  // both signs: S3_{mu nu}
    for (int s = 0; s < 2; ++s) {
      const int fs = (mu * 3 + i) * 2 + s;
      if (!use_z && cL.x == 0.f) continue;
      const long y = nb(g, c, nu, s == 0 ? 1 : -1);
      F3 x;
      if (use_z) {
        x = fld(Z, mu * 3 + i, g.V, y);
        if (cL.x != 0.f) faxpy(x, cL, fld(S, fs, g.V, y));
      } else {
        x = fzero();
        faxpy(x, cL, fld(S, fs, g.V, y));
      }
      wrap_acc(F, g, U, c, n, mu, nu, s, x);
    }
  }
  if (aos) {
    double2* p = static_cast<double2*>(out) + ((size_t)n * 4 + mu) * 9;
#pragma unroll
    for (int e = 0; e < 9; ++e) p[e] = join_ff(F.e[e]);
  } else {
    fst(static_cast<float4*>(out), mu, g.V, n, F);
  }
}

// U(3) projection W = V (V^+ V)^(-1/2): the unitary polar factor of V, by Newton's
// iteration X <- (g X + X^{-+} / g) / 2 with Frobenius-norm scaling g while far from
// convergence (Higham, SIAM J. Sci. Stat. Comput. 7 (1986) 1160). X^{-+} is the
// conjugated cofactor matrix over conj(det X). At most kMaxPolar steps; a singular or
// non-finite link, or no convergence, sets *err and leaves the link as it is.
// The matrix arithmetic (cofactors, determinant, update) is float-float. Any g > 0 keeps the
// polar factor, so g comes from FP32 norms; X^{-+} must be exact to the working precision, so
// 1 / |det|^2 is one FP64 division on the joined value, split back. The step size is measured in
// FP32 from the float-float differences.
constexpr int kMaxPolar = 40;

__device__ __forceinline__ float4 fneg(float4 a) { return make_float4(-a.x, -a.y, -a.z, -a.w); }

__global__ void __launch_bounds__(kThreads) k_u3_project(Lat g, float4* __restrict__ F, int* __restrict__ err) {
  const long n = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.V) return;
  const int mu = blockIdx.y;
  F3 X = fld(F, mu, g.V, n);
  bool ok = false;
  for (int it = 0; it < kMaxPolar; ++it) {
    // cofactors C_ij = X_{i1 j1} X_{i2 j2} - X_{i1 j2} X_{i2 j1} and det = sum_j X_0j C_0j
    F3 C;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        fcfma(a, X.e[i1 * 3 + j1], X.e[i2 * 3 + j2]);
        fcfma(a, fneg(X.e[i1 * 3 + j2]), X.e[i2 * 3 + j1]);
        fnorm(a);
        C.e[i * 3 + j] = a;
      }
    float4 det = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int j = 0; j < 3; ++j) fcfma(det, X.e[j], C.e[j]);
    fnorm(det);
    const double2 dd = join_ff(det);
    const double dn = dd.x * dd.x + dd.y * dd.y;
    if (!(dn > 0.0) || !isfinite(dn)) break;
    const double inv_dn = 1.0 / dn;
    float nx = 0.f, nc = 0.f;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      nx = fmaf(X.e[e].x, X.e[e].x, fmaf(X.e[e].z, X.e[e].z, nx));
      nc = fmaf(C.e[e].x, C.e[e].x, fmaf(C.e[e].z, C.e[e].z, nc));
    }
    // Frobenius scaling gamma = sqrt(|X^-1|_F / |X|_F) = (|C|_F^2 / (|det|^2 |X|_F^2))^(1/4)
    const float gam = sqrtf(sqrtf(nc * (float)inv_dn / nx));
    const bool scale = fabsf(gam - 1.f) > 1e-3f;
    const float g1 = scale ? 0.5f * gam : 0.5f, g2 = scale ? 0.5f / gam : 0.5f;
    // X^{-+} = conj(C) det / |det|^2, elementwise; q = g2 det / |det|^2 (float-float)
    const float4 q = split_ff(make_double2((double)g2 * dd.x * inv_dn, (double)g2 * dd.y * inv_dn));
    const float4 g1c = make_float4(g1, 0.f, 0.f, 0.f);
    float diff = 0.f;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      float4 xn = make_float4(0.f, 0.f, 0.f, 0.f);
      fcfma(xn, g1c, X.e[e]);
      fcfma_ca(xn, C.e[e], q);
      fnorm(xn);
      const float dx = __fadd_rn(__fsub_rn(xn.x, X.e[e].x), __fsub_rn(xn.y, X.e[e].y));
      const float dy = __fadd_rn(__fsub_rn(xn.z, X.e[e].z), __fsub_rn(xn.w, X.e[e].w));
      diff = fmaf(dx, dx, fmaf(dy, dy, diff));
      X.e[e] = xn;
    }
    if (!isfinite(diff)) break;
    // unscaled and the step below 1e-9: Newton's quadratic convergence leaves an error ~1e-18
    if (!scale && diff < 1e-18f) {
      ok = true;
      break;
    }
  }
  if (!ok) {
    atomicExch(err, 1);
    return;
  }
  fst(F, mu, g.V, n, X);
}

// long_mu(n) = naik W_mu(n) W_mu(n+mu) W_mu(n+2mu), written in FP64 in host order [V][4][9]
__global__ void __launch_bounds__(kThreads) k_naik(Lat g, const float4* __restrict__ W, double naik,
                                                   double2* __restrict__ out) {
  const long n = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.V) return;
  const int mu = blockIdx.y;
  int c[4];
  coords(g, n, c);
  const F3 a = fld(W, mu, g.V, n);
  const F3 b = fld(W, mu, g.V, nb(g, c, mu, 1));
  const F3 d = fld(W, mu, g.V, nb(g, c, mu, 2));
  const F3 p = fmm(fmm(a, b), d);
  double2* o = out + ((size_t)n * 4 + mu) * 9;
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    const double2 v = join_ff(p.e[e]);
    o[e] = make_double2(naik * v.x, naik * v.y);
  }
}

int check_dims(const int dims[4], Lat* g) {
  if (!dims) return SQCG_ERR_INVALID_ARG;
  long V = 1;
  for (int d = 0; d < 4; ++d) {
    if (dims[d] < 4 || (dims[d] & 1)) return SQCG_ERR_INVALID_ARG;
    g->L[d] = dims[d];
    V *= dims[d];
  }
  if (V > (1L << 30)) return SQCG_ERR_INVALID_ARG;
  g->V = V;
  return SQCG_OK;
}

const sqcg_hisq_coeffs kDefaultCoeffs = {
    {1.0 / 8.0, 1.0 / 16.0, 1.0 / 64.0, 1.0 / 384.0, 0.0},
    {1.0, 1.0 / 16.0, 1.0 / 64.0, 1.0 / 384.0, -1.0 / 8.0},
    -1.0 / 24.0,
};

bool finite_level(const sqcg_smear_level& l) {
  return isfinite(l.one_link) && isfinite(l.three_staple) && isfinite(l.five_staple) && isfinite(l.seven_staple) &&
         isfinite(l.lepage);
}

// a coefficient as a float-float pair (hi = fl32(c), lo = fl32(c - hi)); zero stays (0, 0)
float2 ff_coeff(double c) {
  const float h = (float)c;
  return make_float2(h, (float)(c - (double)h));
}

// one smearing level: U (float-float fields) -> out (float-float fields, or FP64 host order when aos)
int smear_level(const Lat& g, const float4* U, float4* S, float4* Z, const sqcg_smear_level& c, int aos, void* out,
                cudaStream_t s) {
  const dim3 blk(kThreads);
  const unsigned gx = (unsigned)((g.V + kThreads - 1) / kThreads);
  const bool need_s = c.three_staple != 0.0 || c.five_staple != 0.0 || c.seven_staple != 0.0 || c.lepage != 0.0;
  const bool use_z = c.five_staple != 0.0 || c.seven_staple != 0.0;
  if (need_s) k_staple3<<<dim3(gx, 12), blk, 0, s>>>(g, U, S);
  if (use_z)
    k_staple57<<<dim3(gx, 12), blk, 0, s>>>(g, U, S, ff_coeff(c.five_staple), ff_coeff(c.seven_staple), Z);
  k_smear_links<<<dim3(gx, 4), blk, 0, s>>>(g, U, S, Z, ff_coeff(c.one_link), ff_coeff(c.three_staple),
                                             ff_coeff(c.lepage), use_z ? 1 : 0, aos, out);
  return cudaGetLastError() == cudaSuccess ? SQCG_OK : SQCG_ERR_CUDA;
}

}  // namespace

extern "C" size_t sqcg_hisq_workspace_bytes(const int dims[4]) {
  Lat g;
  if (check_dims(dims, &g) != SQCG_OK) return 0;
  // thin fields (4) + staples (kNumS) + Z (12) + level-1 result / projected links (4), then an error flag
  return (size_t)(4 + kNumS + 12 + 4) * 9 * g.V * sizeof(double2) + 256;
}

extern "C" int sqcg_hisq_smear(const int dims[4], const void* thin, void* fat, void* lng, const sqcg_hisq_coeffs* coeffs,
                               void* workspace, size_t workspace_bytes, void* stream) {
  Lat g;
  SQCG_TRY(check_dims(dims, &g));
  if (!thin || !fat || !lng || !workspace || fat == lng || thin == lng) return SQCG_ERR_INVALID_ARG;
  if ((((uintptr_t)thin) | ((uintptr_t)fat) | ((uintptr_t)lng) | ((uintptr_t)workspace)) & 15)
    return SQCG_ERR_INVALID_ARG;
  if (workspace_bytes < sqcg_hisq_workspace_bytes(dims)) return SQCG_ERR_INVALID_ARG;
  const sqcg_hisq_coeffs& c = coeffs ? *coeffs : kDefaultCoeffs;
  if (!finite_level(c.level1) || !finite_level(c.level2) || !isfinite(c.naik)) return SQCG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nf = 9 * (size_t)g.V;
  float4* U = (float4*)workspace;  // float-float fields, 16 bytes per complex element
  float4* S = U + 4 * nf;
  float4* Z = S + kNumS * nf;
  float4* W = Z + 12 * nf;
  int* err = (int*)(W + 4 * nf);
  const unsigned gx = (unsigned)((g.V + kThreads - 1) / kThreads);
  SQCG_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
  k_links_to_fields<<<dim3(gx, 4), kThreads, 0, s>>>(g, (const double2*)thin, U);
  SQCG_CUDA_TRY(cudaGetLastError());
  SQCG_TRY(smear_level(g, U, S, Z, c.level1, 0, W, s));
  k_u3_project<<<dim3(gx, 4), kThreads, 0, s>>>(g, W, err);
  SQCG_CUDA_TRY(cudaGetLastError());
  SQCG_TRY(smear_level(g, W, S, Z, c.level2, 1, fat, s));
  k_naik<<<dim3(gx, 4), kThreads, 0, s>>>(g, W, c.naik, (double2*)lng);
  SQCG_CUDA_TRY(cudaGetLastError());
  int h_err = 0;
  SQCG_CUDA_TRY(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  SQCG_CUDA_TRY(cudaStreamSynchronize(s));
  return h_err ? SQCG_ERR_BREAKDOWN : SQCG_OK;
}

extern "C" int sqcg_hisq_load_links(sqcg_ctx* ctx, const double* thin, const sqcg_hisq_coeffs* coeffs, int opts,
                                    double* fat_out, double* lng_out) {
  if (!ctx || !thin) return SQCG_ERR_INVALID_ARG;
  if (ctx->flags & SQCG_PHASES_FOLDED) return SQCG_ERR_INVALID_ARG;  // the smearing takes unphased thin links
  if (opts & ~(SQCG_RECON12_LONG | SQCG_EIGHT_WAY)) return SQCG_ERR_INVALID_ARG;
  const size_t V = 2 * (size_t)ctx->g.Vh;
  const size_t bytes = V * 4 * 9 * sizeof(double2);
  const size_t wsb = sqcg_hisq_workspace_bytes(ctx->L);
  cudaStream_t s = ctx->stream;
  void *fat = nullptr, *lng = nullptr, *ws = nullptr;
  if (cudaMalloc(&fat, bytes) != cudaSuccess || cudaMalloc(&lng, bytes) != cudaSuccess ||
      cudaMalloc(&ws, wsb) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(fat); cudaFree(lng); cudaFree(ws);
    return SQCG_ERR_NO_MEMORY;
  }
  int rc = SQCG_OK;
  do {
    // the thin links are staged in the fat output buffer: the first kernel consumes them
    if (cudaMemcpyAsync(fat, thin, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) { rc = SQCG_ERR_CUDA; break; }
    if ((rc = sqcg_hisq_smear(ctx->L, fat, fat, lng, coeffs, ws, wsb, s)) != SQCG_OK) break;
    cudaFree(ws);
    ws = nullptr;
    if (fat_out && cudaMemcpyAsync(fat_out, fat, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) { rc = SQCG_ERR_CUDA; break; }
    if (lng_out && cudaMemcpyAsync(lng_out, lng, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) { rc = SQCG_ERR_CUDA; break; }
    if (cudaStreamSynchronize(s) != cudaSuccess) { rc = SQCG_ERR_CUDA; break; }
    rc = layout_load_links_device(ctx, (const double*)fat, (const double*)lng, opts);
  } while (0);
  if (rc == SQCG_ERR_CUDA) sqcg_set_last_cuda_error(cudaGetLastError(), "hisq_load_links", __FILE__, __LINE__);
  cudaStreamSynchronize(s);
  cudaFree(fat);
  cudaFree(lng);
  cudaFree(ws);
  return rc;
}
