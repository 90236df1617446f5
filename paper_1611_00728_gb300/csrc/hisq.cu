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
// (12 in A, 24 in B, 12 in C). The work is FP64 arithmetic bound on this GPU.
#include <math.h>
#include <string.h>

#include "sqcg_internal.cuh"

namespace {

constexpr int kThreads = 128;

struct Lat {
  int L[4];
  long V;
};

struct M3 {
  double2 e[9];
};

__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {  // acc += a b
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
__device__ __forceinline__ void cfma_cb(double2& acc, double2 a, double2 b) {  // acc += a conj(b)
  acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
  acc.y = fma(a.y, b.x, fma(-a.x, b.y, acc.y));
}
__device__ __forceinline__ void cfma_ca(double2& acc, double2 a, double2 b) {  // acc += conj(a) b
  acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
}

__device__ __forceinline__ M3 mm(const M3& A, const M3& B) {  // A B
  M3 C;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double2 s = make_double2(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < 3; ++k) cfma(s, A.e[i * 3 + k], B.e[k * 3 + j]);
      C.e[i * 3 + j] = s;
    }
  return C;
}
__device__ __forceinline__ M3 mm_nd(const M3& A, const M3& B) {  // A B^+
  M3 C;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double2 s = make_double2(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < 3; ++k) cfma_cb(s, A.e[i * 3 + k], B.e[j * 3 + k]);
      C.e[i * 3 + j] = s;
    }
  return C;
}
__device__ __forceinline__ M3 mm_dn(const M3& A, const M3& B) {  // A^+ B
  M3 C;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double2 s = make_double2(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < 3; ++k) cfma_ca(s, A.e[k * 3 + i], B.e[k * 3 + j]);
      C.e[i * 3 + j] = s;
    }
  return C;
}
// C += A B and C += A B^+ (the product accumulated into C directly)
__device__ __forceinline__ void mm_acc(M3& C, const M3& A, const M3& B) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < 3; ++k) cfma(C.e[i * 3 + j], A.e[i * 3 + k], B.e[k * 3 + j]);
}
__device__ __forceinline__ void mm_nd_acc(M3& C, const M3& A, const M3& B) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < 3; ++k) cfma_cb(C.e[i * 3 + j], A.e[i * 3 + k], B.e[j * 3 + k]);
}
__device__ __forceinline__ void axpy(M3& Y, double a, const M3& X) {
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    Y.e[e].x = fma(a, X.e[e].x, Y.e[e].x);
    Y.e[e].y = fma(a, X.e[e].y, Y.e[e].y);
  }
}
__device__ __forceinline__ void addto(M3& Y, const M3& X) {
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    Y.e[e].x += X.e[e].x;
    Y.e[e].y += X.e[e].y;
  }
}

// field k of a structure-of-arrays buffer: elements [k][e][V]
__device__ __forceinline__ M3 ld(const double2* __restrict__ f, int k, long V, long n) {
  M3 m;
  const double2* p = f + (size_t)k * 9 * V + n;
#pragma unroll
  for (int e = 0; e < 9; ++e) m.e[e] = __ldg(p + (size_t)e * V);
  return m;
}
__device__ __forceinline__ void st(double2* __restrict__ f, int k, long V, long n, const M3& m) {
  double2* p = f + (size_t)k * 9 * V + n;
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
__device__ __forceinline__ M3 wrap(const Lat& g, const double2* __restrict__ U, const int c[4], long n, int mu,
                                   int d, int s, const M3& Xd) {
  if (s == 0) {
    const M3 a = ld(U, d, g.V, n);
    const M3 b = ld(U, d, g.V, nb(g, c, mu, 1));
    return mm_nd(mm(a, Xd), b);
  }
  const M3 a = ld(U, d, g.V, nb(g, c, d, -1));
  const M3 b = ld(U, d, g.V, nb(g, c, d, -1, mu, 1));
  return mm(mm_dn(a, Xd), b);
}

// acc += wrap^s_d X (n)
__device__ __forceinline__ void wrap_acc(M3& acc, const Lat& g, const double2* __restrict__ U, const int c[4], long n,
                                         int mu, int d, int s, const M3& Xd) {
  if (s == 0) {
    const M3 a = ld(U, d, g.V, n);
    const M3 b = ld(U, d, g.V, nb(g, c, mu, 1));
    mm_nd_acc(acc, mm(a, Xd), b);
    return;
  }
  const M3 a = ld(U, d, g.V, nb(g, c, d, -1));
  const M3 b = ld(U, d, g.V, nb(g, c, d, -1, mu, 1));
  mm_acc(acc, mm_dn(a, Xd), b);
}

// host AoS [V][4][9] -> [mu][e][V]
__global__ void __launch_bounds__(kThreads) k_links_to_fields(Lat g, const double2* __restrict__ aos,
                                                              double2* __restrict__ U) {
  const long n = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.V) return;
  const int mu = blockIdx.y;
#pragma unroll
  for (int e = 0; e < 9; ++e) U[((size_t)mu * 9 + e) * g.V + n] = aos[((size_t)n * 4 + mu) * 9 + e];
}

// A: 3-staples S^+_{mu nu}, S^-_{mu nu} (s = 0 forward, 1 backward) and S3_{mu nu} = S^+ + S^-
__global__ void __launch_bounds__(kThreads) k_staple3(Lat g, const double2* __restrict__ U, double2* __restrict__ S) {
  const long n = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.V) return;
  const int f = blockIdx.y;  // mu*3 + nu index
  const int mu = f / 3, nu = other(mu, f % 3);
  int c[4];
  coords(g, n, c);
  const M3 sp = wrap(g, U, c, n, mu, nu, 0, ld(U, mu, g.V, nb(g, c, nu, 1)));
  st(S, 2 * f, g.V, n, sp);
  M3 sm = wrap(g, U, c, n, mu, nu, 1, ld(U, mu, g.V, nb(g, c, nu, -1)));
  st(S, 2 * f + 1, g.V, n, sm);
  addto(sm, sp);
  st(S, 24 + f, g.V, n, sm);
}

// B: Z_{mu nu} = c5 (S3_{mu rho} + S3_{mu sig}) + c7 (wrap_rho S3_{mu sig} + wrap_sig S3_{mu rho})
__global__ void __launch_bounds__(kThreads) k_staple57(Lat g, const double2* __restrict__ U,
                                                       const double2* __restrict__ S, double c5, double c7,
                                                       double2* __restrict__ Z) {
  const long n = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.V) return;
  const int f = blockIdx.y;  // mu*3 + nu index
  const int mu = f / 3, nu = other(mu, f % 3);
  int rs[2], k = 0;
  for (int d = 0; d < 4; ++d)
    if (d != mu && d != nu) rs[k++] = d;
  int c[4];
  coords(g, n, c);
  M3 z;
#pragma unroll
  for (int e = 0; e < 9; ++e) z.e[e] = make_double2(0.0, 0.0);
  if (c5 != 0.0) {
    M3 t = ld(S, s3_field(mu, rs[0]), g.V, n);
    addto(t, ld(S, s3_field(mu, rs[1]), g.V, n));
    axpy(z, c5, t);
  }
  if (c7 != 0.0) {
    M3 w;
#pragma unroll
    for (int e = 0; e < 9; ++e) w.e[e] = make_double2(0.0, 0.0);
    for (int q = 0; q < 2; ++q) {
      const int d = rs[q], inner = rs[1 - q];
      for (int s = 0; s < 2; ++s) {
        const M3 x = ld(S, s3_field(mu, inner), g.V, nb(g, c, d, s == 0 ? 1 : -1));
        wrap_acc(w, g, U, c, n, mu, d, s, x);
      }
    }
    axpy(z, c7, w);
  }
  st(Z, f, g.V, n, z);
}

// C: F_mu = c1 U_mu + sum_{nu,s} [ c3 S^s_{mu nu} + wrap^s_nu (Z_{mu nu} + cL S^s_{mu nu}) ]
// out: structure of arrays [mu][e][V], or the host order [V][4][9] when aos != 0
__global__ void __launch_bounds__(kThreads) k_smear_links(Lat g, const double2* __restrict__ U,
                                                          const double2* __restrict__ S,
                                                          const double2* __restrict__ Z, double c1, double c3,
                                                          double cL, int use_z, int aos, double2* __restrict__ out) {
  const long n = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.V) return;
  const int mu = blockIdx.y;
  int c[4];
  coords(g, n, c);
  M3 F = ld(U, mu, g.V, n);
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    F.e[e].x *= c1;
    F.e[e].y *= c1;
  }
  for (int i = 0; i < 3; ++i) {
    const int nu = other(mu, i);
    if (c3 != 0.0) axpy(F, c3, ld(S, 24 + mu * 3 + i, g.V, n));  // both signs: S3_{mu nu}
    for (int s = 0; s < 2; ++s) {
      const int fs = (mu * 3 + i) * 2 + s;
      if (!use_z && cL == 0.0) continue;
      const long y = nb(g, c, nu, s == 0 ? 1 : -1);
      M3 x;
      if (use_z) {
        x = ld(Z, mu * 3 + i, g.V, y);
        if (cL != 0.0) axpy(x, cL, ld(S, fs, g.V, y));
      } else {
        x = ld(S, fs, g.V, y);
#pragma unroll
        for (int e = 0; e < 9; ++e) {
          x.e[e].x *= cL;
          x.e[e].y *= cL;
        }
      }
      wrap_acc(F, g, U, c, n, mu, nu, s, x);
    }
  }
  if (aos) {
    double2* p = out + ((size_t)n * 4 + mu) * 9;
#pragma unroll
    for (int e = 0; e < 9; ++e) p[e] = F.e[e];
  } else {
    st(out, mu, g.V, n, F);
  }
}

// U(3) projection W = V (V^+ V)^(-1/2): the unitary polar factor of V, by Newton's
// iteration X <- (g X + X^{-+} / g) / 2 with Frobenius-norm scaling g while far from
// convergence (Higham, SIAM J. Sci. Stat. Comput. 7 (1986) 1160). X^{-+} is the
// conjugated cofactor matrix over conj(det X). At most kMaxPolar steps; a singular or
// non-finite link, or no convergence, sets *err and leaves the link as it is.
constexpr int kMaxPolar = 40;

__global__ void __launch_bounds__(kThreads) k_u3_project(Lat g, double2* __restrict__ F, int* __restrict__ err) {
  const long n = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.V) return;
  const int mu = blockIdx.y;
  M3 X = ld(F, mu, g.V, n);
  bool ok = false;
  for (int it = 0; it < kMaxPolar; ++it) {
    // cofactors C_ij and det = sum_j X_0j C_0j
    M3 C;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
        double2 a = make_double2(0.0, 0.0);
        cfma(a, X.e[i1 * 3 + j1], X.e[i2 * 3 + j2]);
        const double2 b = X.e[i1 * 3 + j2], d = X.e[i2 * 3 + j1];
        a.x -= b.x * d.x - b.y * d.y;
        a.y -= b.x * d.y + b.y * d.x;
        C.e[i * 3 + j] = a;
      }
    double2 det = make_double2(0.0, 0.0);
#pragma unroll
    for (int j = 0; j < 3; ++j) cfma(det, X.e[j], C.e[j]);
    const double dn = det.x * det.x + det.y * det.y;
    if (!(dn > 0.0) || !isfinite(dn)) break;
    const double inv_dn = 1.0 / dn;
    double nx = 0.0, nc = 0.0;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      nx += X.e[e].x * X.e[e].x + X.e[e].y * X.e[e].y;
      nc += C.e[e].x * C.e[e].x + C.e[e].y * C.e[e].y;
    }
    // Frobenius scaling gamma = sqrt(|X^-1|_F / |X|_F) = (|C|_F^2 / (|det|^2 |X|_F^2))^(1/4)
    const double gam = sqrt(sqrt(nc * inv_dn / nx));
    const bool scale = fabs(gam - 1.0) > 1e-3;
    const double g1 = scale ? 0.5 * gam : 0.5, g2 = scale ? 0.5 / gam : 0.5;
    // X^{-+} = conj(C) det / |det|^2, elementwise; q = g2 det / |det|^2
    const double2 q = make_double2(g2 * det.x * inv_dn, g2 * det.y * inv_dn);
    double diff = 0.0;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      const double2 cc = C.e[e];
      const double2 xn = make_double2(fma(g1, X.e[e].x, cc.x * q.x + cc.y * q.y),
                                      fma(g1, X.e[e].y, cc.x * q.y - cc.y * q.x));
      const double dx = xn.x - X.e[e].x, dy = xn.y - X.e[e].y;
      diff += dx * dx + dy * dy;
      X.e[e] = xn;
    }
    if (!isfinite(diff)) break;
    // unscaled and the step below 1e-9: Newton's quadratic convergence leaves an error ~1e-18
    if (!scale && diff < 1e-18) {
      ok = true;
      break;
    }
  }
  if (!ok) {
    atomicExch(err, 1);
    return;
  }
  st(F, mu, g.V, n, X);
}

// long_mu(n) = naik W_mu(n) W_mu(n+mu) W_mu(n+2mu), written in host order [V][4][9]
__global__ void __launch_bounds__(kThreads) k_naik(Lat g, const double2* __restrict__ W, double naik,
                                                   double2* __restrict__ out) {
  const long n = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.V) return;
  const int mu = blockIdx.y;
  int c[4];
  coords(g, n, c);
  const M3 a = ld(W, mu, g.V, n);
  const M3 b = ld(W, mu, g.V, nb(g, c, mu, 1));
  const M3 d = ld(W, mu, g.V, nb(g, c, mu, 2));
  const M3 p = mm(mm(a, b), d);
  double2* o = out + ((size_t)n * 4 + mu) * 9;
#pragma unroll
  for (int e = 0; e < 9; ++e) o[e] = make_double2(naik * p.e[e].x, naik * p.e[e].y);
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

// one smearing level: U (fields) -> out (fields or host order)
int smear_level(const Lat& g, const double2* U, double2* S, double2* Z, const sqcg_smear_level& c, int aos,
                double2* out, cudaStream_t s) {
  const dim3 blk(kThreads);
  const unsigned gx = (unsigned)((g.V + kThreads - 1) / kThreads);
  const bool need_s = c.three_staple != 0.0 || c.five_staple != 0.0 || c.seven_staple != 0.0 || c.lepage != 0.0;
  const bool use_z = c.five_staple != 0.0 || c.seven_staple != 0.0;
  if (need_s) k_staple3<<<dim3(gx, 12), blk, 0, s>>>(g, U, S);
  if (use_z) k_staple57<<<dim3(gx, 12), blk, 0, s>>>(g, U, S, c.five_staple, c.seven_staple, Z);
  k_smear_links<<<dim3(gx, 4), blk, 0, s>>>(g, U, S, Z, c.one_link, c.three_staple, c.lepage, use_z ? 1 : 0, aos,
                                             out);
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
  double2* U = (double2*)workspace;
  double2* S = U + 4 * nf;
  double2* Z = S + kNumS * nf;
  double2* W = Z + 12 * nf;
  int* err = (int*)(W + 4 * nf);
  const unsigned gx = (unsigned)((g.V + kThreads - 1) / kThreads);
  SQCG_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
  k_links_to_fields<<<dim3(gx, 4), kThreads, 0, s>>>(g, (const double2*)thin, U);
  SQCG_CUDA_TRY(cudaGetLastError());
  SQCG_TRY(smear_level(g, U, S, Z, c.level1, 0, W, s));
  k_u3_project<<<dim3(gx, 4), kThreads, 0, s>>>(g, W, err);
  SQCG_CUDA_TRY(cudaGetLastError());
  SQCG_TRY(smear_level(g, W, S, Z, c.level2, 1, (double2*)fat, s));
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
