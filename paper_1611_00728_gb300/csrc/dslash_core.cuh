// Device core of the improved-staggered Dslash (arXiv:1611.00728 Sec. 3), shared by the
// one-pass kernels (dslash.cu) and the persistent single-reduction CG (cg_persistent.cu): colour
// algebra, link and vector loads, the kernel arguments and the 16-hop sum at one output site.
//
//   (D psi)(n) = sum_mu [ F_mu(n) psi(n+mu) - F_mu(n-mu)^+ psi(n-mu)
//                       + L_mu(n) psi(n+3mu) - L_mu(n-3mu)^+ psi(n-3mu) ]
//
// Links are [parity][mu][elem][Vh] (eta_mu and the boundary sign folded in), colour vectors [3][Vh].
#pragma once
#include "solver_device.cuh"
#include "sqcg_internal.cuh"

namespace dcore {

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

// NC: through the read-only (non-coherent) path. A kernel that reads a vector other blocks of the same
// launch have written (the persistent solver) must load it coherently (NC = false).
template <bool NC = true, typename R2>
__device__ __forceinline__ void load_vec(R2 (&v)[3], const R2* __restrict__ in, int Vh, int idx) {
#pragma unroll
  for (int c = 0; c < 3; ++c) v[c] = NC ? ldg2(in + (size_t)c * Vh + idx) : in[(size_t)c * Vh + idx];
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
// The input vector at a site: plain loads of a.in (the kernels), or another functor with
// operator()(R2 (&v)[3], int idx) (the persistent CG forms its input on the fly).
template <typename R2, bool NC>
struct PlainIn {
  const R2* in;
  int Vh;
  __device__ __forceinline__ void operator()(R2 (&v)[3], int idx) const { load_vec<NC>(v, in, Vh, idx); }
};

template <typename R, bool RECON, bool EIGHT, typename In>
__device__ __forceinline__ void dslash_site_in(const DArgs<R>& a, int i, typename V2<R>::T (&acc)[3], const In& in_at);

template <typename R, bool RECON, bool EIGHT, bool NC = true>
__device__ __forceinline__ void dslash_site(const DArgs<R>& a, int i, typename V2<R>::T (&acc)[3]) {
  dslash_site_in<R, RECON, EIGHT>(a, i, acc, PlainIn<typename V2<R>::T, NC>{a.in, a.g.Vh});
}

template <typename R, bool RECON, bool EIGHT, typename In>
__device__ __forceinline__ void dslash_site_in(const DArgs<R>& a, int i, typename V2<R>::T (&acc)[3], const In& in_at) {
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
        in_at(v, fwd);
        acc_mv<R>(acc, U, v);
        in_at(v, bwd);
        if (EIGHT) {
          load_link<R, R2, false>(U, a.fatb_p + (size_t)mu * 9 * Vh, Vh, i, R(1));
          acc_mv<R>(acc, U, v);
        } else {
          load_link<R, R2, false>(U, a.fat_q + (size_t)mu * 9 * Vh, Vh, bwd, R(1));
          sub_mdv<R>(acc, U, v);
        }
      } else {
        load_link<R, R2, RECON>(U, a.lng_p + (size_t)mu * a.nl * Vh, Vh, i, inv_s_f);
        in_at(v, fwd);
        acc_mv<R>(acc, U, v);
        in_at(v, bwd);
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

}  // namespace dcore
