/*
 * sqcg_oracle.c -- plain, slow FP64 CPU oracle for the improved-staggered CG.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file. It shares no code with the
 * CUDA library; the CUDA path must never call it.
 *
 * What it computes (MILC staggered CG, arXiv:1611.00728 Sec. 3-4; the paper
 * names the operator and the solvers but writes no formula, so the standard
 * improved-staggered definitions are spelled out here):
 *
 *   (D psi)(n) = sum_mu [  s_mu(n,1)      F_mu(n)        psi(n+mu)
 *                        - s_mu(n-mu,1)   F_mu(n-mu)^+   psi(n-mu)
 *                        + s_mu(n,3)      L_mu(n)        psi(n+3mu)
 *                        - s_mu(n-3mu,3)  L_mu(n-3mu)^+  psi(n-3mu) ]
 *
 * with F the fat (one-hop) and L the long (Naik, three-hop) links, and
 * s_mu(m,d) = eta_mu(m) * bc(m,mu,d) the sign of the forward hop of length d
 * that starts at m:  eta_x = 1, eta_y = (-1)^x, eta_z = (-1)^(x+y),
 * eta_t = (-1)^(x+y+z);  bc = -1 when the time direction is antiperiodic and
 * the hop crosses the last time slice (m_t + d >= Lt), else +1.
 *
 * Every hop has odd length, so D maps one parity onto the other. The CG
 * solves the even-site normal equation
 *     A x = (sigma - D_eo D_oe) x = b,   sigma = 4 m^2  (M = 2m + D),
 * by Hestenes-Stiefel CG; a multi-mass solve is the same system for each
 * shift sigma_s (Sec. 3: single- and multi-mass CG).
 *
 * Data layout (plain, lexicographic; nothing blocked or reordered):
 *   site  n = x + Lx*(y + Ly*(z + Lz*t))
 *   links double complex [V][4][3][3]  (forward links, row-major)
 *   field double complex [V][3]        (full lattice; only one parity used)
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static void coords(const int L[4], long n, int x[4]) {
  x[0] = (int)(n % L[0]); n /= L[0];
  x[1] = (int)(n % L[1]); n /= L[1];
  x[2] = (int)(n % L[2]);
  x[3] = (int)(n / L[2]);
}

static long site(const int L[4], const int x[4]) {
  return x[0] + (long)L[0] * (x[1] + (long)L[1] * (x[2] + (long)L[2] * x[3]));
}

/* coordinates of x + d * mu-hat with periodic wrap (d may be negative) */
static void hop(const int L[4], const int x[4], int mu, int d, int y[4]) {
  for (int nu = 0; nu < 4; ++nu) y[nu] = x[nu];
  y[mu] = ((x[mu] + d) % L[mu] + L[mu]) % L[mu];
}

/* staggered phase eta_mu(x) */
static double eta(int mu, const int x[4]) {
  int s = 0;
  for (int nu = 0; nu < mu; ++nu) s += x[nu];
  return (s & 1) ? -1.0 : 1.0;
}

/* sign of the forward hop of length d in direction mu starting at x */
static double hop_sign(const int L[4], int antiperiodic_t, const int x[4], int mu, int d) {
  double s = eta(mu, x);
  if (antiperiodic_t && mu == 3 && x[3] + d >= L[3]) s = -s;
  return s;
}

static const cplx* link(const cplx* U, long n, int mu) { return U + ((n * 4 + mu) * 9); }

/* out += c * U v */
static void add_mv(cplx out[3], double c, const cplx* U, const cplx* v) {
  for (int a = 0; a < 3; ++a) {
    cplx s = 0;
    for (int b = 0; b < 3; ++b) s += U[a * 3 + b] * v[b];
    out[a] += c * s;
  }
}

/* out += c * U^dagger v */
static void add_mdv(cplx out[3], double c, const cplx* U, const cplx* v) {
  for (int a = 0; a < 3; ++a) {
    cplx s = 0;
    for (int b = 0; b < 3; ++b) s += conj(U[b * 3 + a]) * v[b];
    out[a] += c * s;
  }
}

/* (D psi)(n) at one site, straight from the definition above */
static void dslash_at(const int L[4], int apbc, const cplx* fat, const cplx* lng,
                      const cplx* psi, long n, cplx out[3]) {
  int x[4], y[4];
  coords(L, n, x);
  out[0] = out[1] = out[2] = 0;
  for (int mu = 0; mu < 4; ++mu) {
    for (int k = 0; k < 2; ++k) {
      const int d = (k == 0) ? 1 : 3;
      const cplx* U = (k == 0) ? fat : lng;
      /* forward:  s(n,d) U_mu(n) psi(n + d mu) */
      hop(L, x, mu, d, y);
      add_mv(out, hop_sign(L, apbc, x, mu, d), link(U, n, mu), psi + site(L, y) * 3);
      /* backward: -s(n - d mu, d) U_mu(n - d mu)^dagger psi(n - d mu) */
      hop(L, x, mu, -d, y);
      long m = site(L, y);
      add_mdv(out, -hop_sign(L, apbc, y, mu, d), link(U, m, mu), psi + m * 3);
    }
  }
}

/* D applied at every site of parity out_parity; other sites of out untouched.
 * in and out must not alias. nthreads > 1 uses OpenMP over sites when built
 * with -fopenmp (same arithmetic per site). */
void oracle_dslash(const int L[4], int apbc, const cplx* fat, const cplx* lng,
                   const cplx* in, cplx* out, int out_parity, int nthreads) {
  const long V = (long)L[0] * L[1] * L[2] * L[3];
  (void)nthreads;
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
  for (long n = 0; n < V; ++n) {
    int x[4];
    coords(L, n, x);
    if (((x[0] + x[1] + x[2] + x[3]) & 1) != out_parity) continue;
    dslash_at(L, apbc, fat, lng, in, n, out + n * 3);
  }
}

/* D at a list of sites (any parity): out[i] = (D psi)(sites[i]), [nsites][3] */
void oracle_dslash_sites(const int L[4], int apbc, const cplx* fat, const cplx* lng,
                         const cplx* in, long nsites, const long* sites, cplx* out) {
  for (long i = 0; i < nsites; ++i) dslash_at(L, apbc, fat, lng, in, sites[i], out + i * 3);
}

/* A x = sigma x - D_eo D_oe x on the even sites; tmp is a full-lattice scratch
 * field whose odd sites receive D_oe x. Odd sites of y are set to zero. */
void oracle_normal_op(const int L[4], int apbc, const cplx* fat, const cplx* lng, double sigma,
                      const cplx* x, cplx* y, cplx* tmp, int nthreads) {
  const long V = (long)L[0] * L[1] * L[2] * L[3];
  oracle_dslash(L, apbc, fat, lng, x, tmp, 1, nthreads); /* tmp_o = D_oe x_e */
  oracle_dslash(L, apbc, fat, lng, tmp, y, 0, nthreads); /* y_e   = D_eo tmp_o */
  for (long n = 0; n < V; ++n) {
    int c[4];
    coords(L, n, c);
    const int even = ((c[0] + c[1] + c[2] + c[3]) & 1) == 0;
    for (int a = 0; a < 3; ++a)
      y[n * 3 + a] = even ? sigma * x[n * 3 + a] - y[n * 3 + a] : 0;
  }
}

/* <u, v> over the even sites */
static cplx dot_even(const int L[4], const cplx* u, const cplx* v) {
  const long V = (long)L[0] * L[1] * L[2] * L[3];
  cplx s = 0;
  for (long n = 0; n < V; ++n) {
    int c[4];
    coords(L, n, c);
    if ((c[0] + c[1] + c[2] + c[3]) & 1) continue;
    for (int a = 0; a < 3; ++a) s += conj(u[n * 3 + a]) * v[n * 3 + a];
  }
  return s;
}

/*
 * Conjugate gradient (Hestenes-Stiefel) for (sigma - D_eo D_oe) x = b on the
 * even sites. x holds the initial guess on entry and the solution on exit.
 * Stops when |r| / |b| <= tol (iterated residual) or after max_iter steps.
 * Returns the number of iterations; *true_rel_resid = |b - A x| / |b|
 * recomputed from the final x. Returns -1 if <p, A p> <= 0 (breakdown).
 */
int oracle_cg(const int L[4], int apbc, const cplx* fat, const cplx* lng, double sigma,
              const cplx* b, cplx* x, double tol, int max_iter, int nthreads,
              double* true_rel_resid) {
  const long V = (long)L[0] * L[1] * L[2] * L[3];
  const size_t bytes = (size_t)V * 3 * sizeof(cplx);
  cplx* r = calloc(1, bytes);
  cplx* p = calloc(1, bytes);
  cplx* Ap = calloc(1, bytes);
  cplx* tmp = calloc(1, bytes);
  int k = 0, status = 0;

  const double bb = creal(dot_even(L, b, b));
  oracle_normal_op(L, apbc, fat, lng, sigma, x, Ap, tmp, nthreads);
  for (long i = 0; i < V * 3; ++i) { r[i] = b[i] - Ap[i]; p[i] = r[i]; }
  /* odd sites of r and p are zero because b's odd sites are ignored: clear them */
  for (long n = 0; n < V; ++n) {
    int c[4];
    coords(L, n, c);
    if ((c[0] + c[1] + c[2] + c[3]) & 1)
      for (int a = 0; a < 3; ++a) r[n * 3 + a] = p[n * 3 + a] = 0;
  }
  double rr = creal(dot_even(L, r, r));
  while (k < max_iter && sqrt(rr / bb) > tol) {
    oracle_normal_op(L, apbc, fat, lng, sigma, p, Ap, tmp, nthreads);
    const double pAp = creal(dot_even(L, p, Ap));
    if (!(pAp > 0)) { status = -1; break; }
    const double alpha = rr / pAp;
    for (long i = 0; i < V * 3; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * Ap[i]; }
    const double rr_new = creal(dot_even(L, r, r));
    const double beta = rr_new / rr;
    for (long i = 0; i < V * 3; ++i) p[i] = r[i] + beta * p[i];
    rr = rr_new;
    ++k;
  }
  /* true residual from the final x */
  oracle_normal_op(L, apbc, fat, lng, sigma, x, Ap, tmp, nthreads);
  for (long i = 0; i < V * 3; ++i) r[i] = b[i] - Ap[i];
  for (long n = 0; n < V; ++n) {
    int c[4];
    coords(L, n, c);
    if ((c[0] + c[1] + c[2] + c[3]) & 1)
      for (int a = 0; a < 3; ++a) r[n * 3 + a] = 0;
  }
  if (true_rel_resid) *true_rel_resid = sqrt(creal(dot_even(L, r, r)) / bb);
  free(r); free(p); free(Ap); free(tmp);
  return status < 0 ? -1 : k;
}

/* number of OpenMP threads a parallel region gets (1 without OpenMP) */
int oracle_max_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
