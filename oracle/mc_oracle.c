/*
 * CPU oracle for the multilevel local-expansion Metropolis-Hastings method
 * of Saunders, Grant & Mueller, "A new algorithm for electrostatic
 * interactions in Monte Carlo simulations of charged particles"
 * (arXiv 2006.16622).
 *
 * TEST INFRASTRUCTURE ONLY: plain, slow, single threaded, FP64.  It follows
 * the paper's algorithms step by step in the paper's notation:
 *   - local expansion Eq. (2) and the level sum Eq. (1)        -> psi_level
 *   - Alg. L.1 (propose), Alg. 1 (direct part)                 -> orc_propose
 *   - Alg. L.2 (accept)                                        -> orc_accept
 *   - Alg. L.3 (initialise)                                    -> orc_setup
 *   - Sec. 3.4 periodic extensions: extended domain of 3^3 box copies, K/E
 *     initialise/accept/propose updates, image self-interaction correction
 * Readings where the paper is silent (normalisation of Y_n^m, the lattice
 * operator R, the energy factor 1/2, the dipole boundary term, the MH rule
 * and the random stream) are stated next to the code that takes them.
 *
 * Compile with -ffp-contract=off: proposal arithmetic must round exactly as
 * written so that replayed chains see bit-identical positions.
 */
#define _GNU_SOURCE
#include "mc_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define IDX(n, m) ((n) * (n) + (n) + (m))

/* ------------------------------------------------------------------------ */
/* factorials                                                                */
/* ------------------------------------------------------------------------ */
static double factorial(int k) {
  static double table[171];
  static int ready = 0;
  if (!ready) {
    table[0] = 1.0;
    for (int i = 1; i <= 170; i++) table[i] = table[i - 1] * (double)i;
    ready = 1;
  }
  return table[k];
}

/* ------------------------------------------------------------------------ */
/* Spherical harmonics.  The paper (Eq. 2-4) does not print the
 * normalisation; we take the one of its FMM references (Greengard):
 *   Y_n^m(theta, phi) = sqrt((n-|m|)!/(n+|m|)!) P_n^|m|(cos theta) e^{i m phi}
 * with P_n^m the associated Legendre function without the Condon-Shortley
 * phase.  With it, Eq. (2) with L_n^m = q r^-(n+1) Y_n^-m (Alg. L.2) is the
 * Legendre addition theorem for 1/|x - y|.                                   */
/* ------------------------------------------------------------------------ */
static void legendre_table(int p, double x, double *P /* [(p+1)*(p+1)] n-major */) {
  double s = sqrt(fmax(0.0, 1.0 - x * x));
  double pmm = 1.0;
  for (int m = 0; m <= p; m++) {
    if (m > 0) pmm *= (double)(2 * m - 1) * s;
    P[m * (p + 1) + m] = pmm;
    if (m + 1 <= p) P[(m + 1) * (p + 1) + m] = (double)(2 * m + 1) * x * pmm;
    for (int n = m + 2; n <= p; n++)
      P[n * (p + 1) + m] = ((double)(2 * n - 1) * x * P[(n - 1) * (p + 1) + m] -
                            (double)(n + m - 1) * P[(n - 2) * (p + 1) + m]) /
                           (double)(n - m);
  }
}

#define ORC_PMAX 64

/* sqrt((n-|m|)!/(n+|m|)!) for n <= ORC_PMAX, cached on first use */
static double ynorm(int n, int am) {
  static double table[(ORC_PMAX + 1) * (ORC_PMAX + 1)];
  static int ready = 0;
  if (!ready) {
    for (int nn = 0; nn <= ORC_PMAX; nn++)
      for (int mm = 0; mm <= nn; mm++)
        table[nn * (ORC_PMAX + 1) + mm] = sqrt(factorial(nn - mm) / factorial(nn + mm));
    ready = 1;
  }
  return table[n * (ORC_PMAX + 1) + am];
}

static void ylm_table(int p, double theta, double phi, cplx *Y) {
  double P[(ORC_PMAX + 1) * (ORC_PMAX + 1)];
  cplx eimp[ORC_PMAX + 1];
  legendre_table(p, cos(theta), P);
  /* e^{i m phi} for m = 0..p by repeated multiplication */
  const cplx e1 = cos(phi) + I * sin(phi);
  eimp[0] = 1.0;
  for (int m = 1; m <= p; m++) eimp[m] = eimp[m - 1] * e1;
  for (int n = 0; n <= p; n++) {
    for (int m = 0; m <= n; m++) {
      const double v = ynorm(n, m) * P[n * (p + 1) + m];
      Y[IDX(n, m)] = v * eimp[m];
      if (m) Y[IDX(n, -m)] = v * conj(eimp[m]);
    }
  }
}

/* spherical(x) of the paper: (r, theta, phi) */
static void spherical(const double x[3], double *r, double *theta, double *phi) {
  *r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  *theta = (*r > 0.0) ? acos(fmax(-1.0, fmin(1.0, x[2] / *r))) : 0.0;
  *phi = atan2(x[1], x[0]);
}

/* r^n Y_n^m */
static void regular_table(int p, const double x[3], cplx *out) {
  double r, th, ph;
  spherical(x, &r, &th, &ph);
  ylm_table(p, th, ph, out);
  double rn = 1.0;
  for (int n = 0; n <= p; n++) {
    for (int m = -n; m <= n; m++) out[IDX(n, m)] *= rn;
    rn *= r;
  }
}

/* r^-(n+1) Y_n^m */
static void irregular_table(int p, const double x[3], cplx *out) {
  double r, th, ph;
  spherical(x, &r, &th, &ph);
  ylm_table(p, th, ph, out);
  double rn = 1.0 / r;
  for (int n = 0; n <= p; n++) {
    for (int m = -n; m <= n; m++) out[IDX(n, m)] *= rn;
    rn /= r;
  }
}

static void to_interleaved(int p, const cplx *c, double *out) {
  for (int k = 0; k < (p + 1) * (p + 1); k++) {
    out[2 * k] = creal(c[k]);
    out[2 * k + 1] = cimag(c[k]);
  }
}

void orc_ylm(int p, double theta, double phi, double *out) {
  if (p < 0 || p > ORC_PMAX) return;
  cplx *Y = (cplx *)malloc(sizeof(cplx) * (p + 1) * (p + 1));
  ylm_table(p, theta, phi, Y);
  to_interleaved(p, Y, out);
  free(Y);
}

void orc_regular(int p, const double x[3], double *out) {
  if (p < 0 || p > ORC_PMAX) return;
  cplx *Y = (cplx *)malloc(sizeof(cplx) * (p + 1) * (p + 1));
  regular_table(p, x, Y);
  to_interleaved(p, Y, out);
  free(Y);
}

void orc_irregular(int p, const double x[3], double *out) {
  if (p < 0 || p > ORC_PMAX) return;
  cplx *Y = (cplx *)malloc(sizeof(cplx) * (p + 1) * (p + 1));
  irregular_table(p, x, Y);
  to_interleaved(p, Y, out);
  free(Y);
}

/* Eq. (4): M_n^m = sum_i q_i r_i^n Y_n^-m(theta_i, phi_i), about centre c */
void orc_multipole(int p, int n, const double *pos, const double *q, const double c[3],
                   double *out) {
  int C = (p + 1) * (p + 1);
  cplx *M = (cplx *)calloc(C, sizeof(cplx));
  cplx *R = (cplx *)malloc(sizeof(cplx) * C);
  for (int i = 0; i < n; i++) {
    double d[3] = {pos[3 * i] - c[0], pos[3 * i + 1] - c[1], pos[3 * i + 2] - c[2]};
    regular_table(p, d, R);
    for (int nn = 0; nn <= p; nn++)
      for (int m = -nn; m <= nn; m++) M[IDX(nn, m)] += q[i] * R[IDX(nn, -m)];
  }
  to_interleaved(p, M, out);
  free(M);
  free(R);
}

/* Eq. (2): Psi(x) = sum_{n,m} L_n^m r^n Y_n^m; the imaginary part vanishes
 * for the conjugate-symmetric coefficients of real charges. */
static double eval_local(int p, const cplx *Lc, const double x[3], cplx *work) {
  regular_table(p, x, work);
  cplx acc = 0.0;
  for (int n = 0; n <= p; n++)
    for (int m = -n; m <= n; m++) acc += Lc[IDX(n, m)] * work[IDX(n, m)];
  return creal(acc);
}

double orc_eval_local(int p, const double *Lc, const double x[3]) {
  int C = (p + 1) * (p + 1);
  cplx *Lz = (cplx *)malloc(sizeof(cplx) * C);
  cplx *w = (cplx *)malloc(sizeof(cplx) * C);
  for (int k = 0; k < C; k++) Lz[k] = Lc[2 * k] + I * Lc[2 * k + 1];
  double v = eval_local(p, Lz, x, w);
  free(Lz);
  free(w);
  return v;
}

/* ------------------------------------------------------------------------ */
/* Multipole-to-local translation.  The paper refers the periodic operator R
 * to the FMM literature; we use the translation theorem of Greengard and
 * Rokhlin for this normalisation: a multipole M about c = (rho, alpha, beta)
 * gives, about the origin,
 *   L_j^k = sum_{n,m} M_n^m i^{|k-m|-|k|-|m|} A_n^m A_j^k
 *           / ((-1)^n A_{j+n}^{m-k}) * Y_{j+n}^{m-k}(alpha, beta) / rho^{j+n+1}
 * with A_n^m = (-1)^n / sqrt((n-m)!(n+m)!).  The exponent |k-m|-|k|-|m| is
 * even and non-positive, so the i-power is a real sign.                     */
/* ------------------------------------------------------------------------ */
static double A_nm(int n, int m) {
  double s = (n % 2 == 0) ? 1.0 : -1.0;
  return s / sqrt(factorial(n - m) * factorial(n + m));
}

static double m2l_factor(int j, int k, int n, int m) {
  int e = abs(k - m) - abs(k) - abs(m); /* even, <= 0 */
  double ipow = ((-e / 2) % 2 == 0) ? 1.0 : -1.0;
  double sn = (n % 2 == 0) ? 1.0 : -1.0;
  return ipow * A_nm(n, m) * A_nm(j, k) / (sn * A_nm(j + n, m - k));
}

/* G[IDX(l, mu)] holds the translation kernel Y_l^mu / rho^(l+1) (or a
 * lattice sum of it), l <= 2p */
static void m2l_apply(int p, const cplx *M, const cplx *G, cplx *Lout) {
  for (int j = 0; j <= p; j++)
    for (int k = -j; k <= j; k++) {
      cplx acc = 0.0;
      for (int n = 0; n <= p; n++)
        for (int m = -n; m <= n; m++)
          acc += M[IDX(n, m)] * m2l_factor(j, k, n, m) * G[IDX(j + n, m - k)];
      Lout[IDX(j, k)] = acc;
    }
}

void orc_m2l(int p, const double *M, const double c[3], double *Lout) {
  int C = (p + 1) * (p + 1), C2 = (2 * p + 1) * (2 * p + 1);
  cplx *Mz = (cplx *)malloc(sizeof(cplx) * C);
  cplx *Lz = (cplx *)malloc(sizeof(cplx) * C);
  cplx *G = (cplx *)malloc(sizeof(cplx) * C2);
  for (int k = 0; k < C; k++) Mz[k] = M[2 * k] + I * M[2 * k + 1];
  irregular_table(2 * p, c, G);
  m2l_apply(p, Mz, G, Lz);
  to_interleaved(p, Lz, Lout);
  free(Mz);
  free(Lz);
  free(G);
}

/* ------------------------------------------------------------------------ */
/* Lattice sums for the far field outside the extended domain (Sec. 3.4):
 *   S_l^m = sum_{v in Z^3, max|v_i| >= 2} Y_l^m(v/|v|) / |v|^(l+1).
 * Reading (the operator R is only defined in the paper's reference
 * Saunders2019): images are summed in growing cubic shells.  Then l = 1 and
 * l = 2 vanish by the cube's symmetry, which is the vacuum ("spherical")
 * result; l = 0 multiplies the total charge, which must be zero.  For
 * 3 <= l < 16 the full sum over v != 0 converges absolutely and is taken by
 * an Ewald-type split (Poisson summation of the harmonic polynomial
 * |x|^l Y_l^m, split at t = 1):
 *   sum_{v!=0} Y(v)/|v|^(l+1) Q(l+1/2, pi |v|^2)
 *   + pi^(l-1/2)/Gamma(l+1/2) (-i)^l sum_{k!=0} |k|^(l-2) Y(k) e^{-pi |k|^2}
 * (Q the regularised upper incomplete gamma function) and the 26 shell-1
 * terms are subtracted.  For l >= 16 the shells are summed directly out to
 * max|v_i| = 24, where the tail is below 1e-18 relative.                    */
/* ------------------------------------------------------------------------ */
static double q_incgamma_half(int l, double x) {
  /* Q(l + 1/2, x) via Q(1/2,x) = erfc(sqrt x), Q(s+1,x) = Q(s,x) + x^s e^-x / Gamma(s+1) */
  double Q = erfc(sqrt(x));
  double s = 0.5, gam = sqrt(M_PI); /* Gamma(s) */
  for (int i = 0; i < l; i++) {
    double gs1 = s * gam; /* Gamma(s+1) */
    Q += exp(s * log(x) - x) / gs1;
    gam = gs1;
    s += 1.0;
  }
  return Q;
}

static void lattice_sums_compute(int lmax, double *out);

/* the unit-lattice sums depend only on lmax: computed once per process */
void orc_lattice_sums(int lmax, double *out) {
  static double *cache[ORC_PMAX + 1];
  if (lmax < 0 || lmax > ORC_PMAX) return;
  int C2 = (lmax + 1) * (lmax + 1);
  if (!cache[lmax]) {
    double *t = (double *)malloc(sizeof(double) * 2 * C2);
    lattice_sums_compute(lmax, t);
    cache[lmax] = t;
  }
  memcpy(out, cache[lmax], sizeof(double) * 2 * C2);
}

static void lattice_sums_compute(int lmax, double *out) {
  int C2 = (lmax + 1) * (lmax + 1);
  cplx *S = (cplx *)calloc(C2, sizeof(cplx));
  cplx *Y = (cplx *)malloc(sizeof(cplx) * C2);
  int lsplit = lmax < 15 ? lmax : 15;
  /* Ewald split for 3 <= l <= lsplit */
  if (lsplit >= 3) {
    const int R = 8;
    for (int x = -R; x <= R; x++)
      for (int y = -R; y <= R; y++)
        for (int z = -R; z <= R; z++) {
          if (x == 0 && y == 0 && z == 0) continue;
          double v[3] = {x, y, z}, r, th, ph;
          spherical(v, &r, &th, &ph);
          ylm_table(lsplit, th, ph, Y);
          int near = (abs(x) <= 1 && abs(y) <= 1 && abs(z) <= 1);
          double r2 = r * r;
          for (int l = 3; l <= lsplit; l++) {
            double rl1 = pow(r, -(double)(l + 1));
            double w = rl1 * q_incgamma_half(l, M_PI * r2);
            if (near) w -= rl1; /* remove the shell-1 terms */
            for (int m = -l; m <= l; m++) S[IDX(l, m)] += w * Y[IDX(l, m)];
            /* reciprocal part, same lattice point used as k */
            double gam = sqrt(M_PI);
            for (int i = 0; i < l; i++) gam *= (0.5 + i); /* Gamma(l+1/2) */
            double pref = pow(M_PI, l - 0.5) / gam;
            cplx mi = 1.0;
            for (int i = 0; i < l; i++) mi *= -I;
            double wk = pref * pow(r, (double)(l - 2)) * exp(-M_PI * r2);
            for (int m = -l; m <= l; m++) S[IDX(l, m)] += mi * wk * Y[IDX(l, m)];
          }
        }
  }
  /* direct shells for l >= 16 */
  if (lmax >= 16) {
    const int R = 24;
    for (int x = -R; x <= R; x++)
      for (int y = -R; y <= R; y++)
        for (int z = -R; z <= R; z++) {
          int mx = abs(x) > abs(y) ? abs(x) : abs(y);
          mx = mx > abs(z) ? mx : abs(z);
          if (mx < 2) continue;
          double v[3] = {x, y, z}, r, th, ph;
          spherical(v, &r, &th, &ph);
          ylm_table(lmax, th, ph, Y);
          for (int l = 16; l <= lmax; l++) {
            double rl1 = pow(r, -(double)(l + 1));
            for (int m = -l; m <= l; m++) S[IDX(l, m)] += rl1 * Y[IDX(l, m)];
          }
        }
  }
  to_interleaved(lmax, S, out);
  free(S);
  free(Y);
}

/* ------------------------------------------------------------------------ */
/* System state                                                              */
/* ------------------------------------------------------------------------ */
struct orc_sys {
  int64_t n;
  double a;
  int L, p, bc, dip, C;
  double *pos, *q;
  int nL;
  double inv_wL;
  /* finest-level cell lists (the paper's particle-to-cell indirection map) */
  int64_t **items;
  int *cnt, *cap;
  int *cell_of;
  /* per-level local coefficients L^Delta_{l,alpha}, index [l][cell*C + IDX] */
  cplx *Lx[16];
  /* multipole method (Sec. 3.3, alternative algorithm): per-level multipole
   * coefficients M_{l,alpha} of Eq. (4), same indexing; method 1 selects it */
  int method;
  cplx *Mx[16];
  /* short-range Lennard-Jones pair term (Sec. 5.3): 4 eps ((sig/r)^12 -
   * (sig/r)^6) for r < rc, off when eps = 0 */
  double lj_eps, lj_sig, lj_rc;
  /* periodic far field: box multipole K, its conjugate E, lattice sums */
  cplx *K, *E, *Slat;
  double D[3];
  double energy;
  double parts[4];
  cplx *w1, *w2, *w3, *w4;
  double *m2lf; /* m2l_factor(j,k,n,m), [IDX(j,k)][IDX(n,m)] */
};

static int ncell_axis(int l) { return 1 << (l - 1); }
static void setup_KE(orc_sys *s);
static void to_real_layout(int p, const cplx *X, double *out);
static double cell_width(const orc_sys *s, int l) { return s->a / (double)ncell_axis(l); }

/* finest-level cell coordinates: floor(x * nL / a), clamped to nL-1; a
 * coordinate on a face goes to the upper cell */
static void finest_cell(const orc_sys *s, const double x[3], int c[3]) {
  for (int d = 0; d < 3; d++) {
    int v = (int)floor(x[d] * s->inv_wL);
    if (v > s->nL - 1) v = s->nL - 1;
    if (v < 0) v = 0;
    c[d] = v;
  }
}

static int lin(int n, const int c[3]) { return (c[0] * n + c[1]) * n + c[2]; }

/* extended cell -> canonical cell and image shift (in box lengths) */
static int wrap_cell(const orc_sys *s, int n, const int e[3], int c[3], int sh[3]) {
  for (int d = 0; d < 3; d++) {
    if (s->bc == ORC_BC_FREE) {
      if (e[d] < 0 || e[d] >= n) return 0;
      c[d] = e[d];
      sh[d] = 0;
    } else {
      int v = ((e[d] % n) + n) % n;
      c[d] = v;
      sh[d] = (e[d] - v) / n;
    }
  }
  return 1;
}

static void cell_centre(const orc_sys *s, int l, const int e[3], double R[3]) {
  double w = cell_width(s, l);
  for (int d = 0; d < 3; d++) R[d] = ((double)e[d] + 0.5) * w;
}

/* Interaction list (Sec. 3.1): children of the parent's 27-cell
 * neighbourhood that are not the cell itself or one of its 26 neighbours.
 * Per axis the children span offsets [-2-b, 3-b] with b the cell's parity. */
static int il_offsets(const int c[3], int off[189][3]) {
  int k = 0;
  int lo[3], hi[3];
  for (int d = 0; d < 3; d++) {
    lo[d] = -2 - (c[d] & 1);
    hi[d] = 3 - (c[d] & 1);
  }
  for (int x = lo[0]; x <= hi[0]; x++)
    for (int y = lo[1]; y <= hi[1]; y++)
      for (int z = lo[2]; z <= hi[2]; z++) {
        if (abs(x) <= 1 && abs(y) <= 1 && abs(z) <= 1) continue;
        off[k][0] = x;
        off[k][1] = y;
        off[k][2] = z;
        k++;
      }
  return k;
}

/* interaction list of cell c on level l as (canonical cell, shift) pairs:
 * out[4*k .. 4*k+3] = linear canonical index, shift x, y, z */
int orc_interaction_list(const orc_sys *s, int level, const int c[3], int *out) {
  int off[189][3];
  int nl = ncell_axis(level), k = 0;
  int nIL = il_offsets(c, off);
  for (int t = 0; t < nIL; t++) {
    int e[3] = {c[0] + off[t][0], c[1] + off[t][1], c[2] + off[t][2]}, cc[3], sh[3];
    if (!wrap_cell(s, nl, e, cc, sh)) continue;
    out[4 * k] = lin(nl, cc);
    out[4 * k + 1] = sh[0];
    out[4 * k + 2] = sh[1];
    out[4 * k + 3] = sh[2];
    k++;
  }
  return k;
}

static void cell_list_add(orc_sys *s, int cell, int64_t i) {
  if (s->cnt[cell] == s->cap[cell]) {
    s->cap[cell] = s->cap[cell] ? 2 * s->cap[cell] : 8;
    s->items[cell] = (int64_t *)realloc(s->items[cell], sizeof(int64_t) * s->cap[cell]);
  }
  s->items[cell][s->cnt[cell]++] = i;
}

static void cell_list_remove(orc_sys *s, int cell, int64_t i) {
  for (int k = 0; k < s->cnt[cell]; k++)
    if (s->items[cell][k] == i) {
      s->items[cell][k] = s->items[cell][s->cnt[cell] - 1];
      s->cnt[cell]--;
      return;
    }
}

orc_sys *orc_create(int64_t n, const double *pos, const double *q, double a, int levels,
                    int p, int bc, int dipole_bc) {
  if (levels < 2 || levels > 9 || p < 0 || 2 * p > ORC_PMAX || n < 1) return NULL;
  orc_sys *s = (orc_sys *)calloc(1, sizeof(orc_sys));
  s->n = n;
  s->a = a;
  s->L = levels;
  s->p = p;
  s->bc = bc;
  s->dip = dipole_bc;
  s->C = (p + 1) * (p + 1);
  s->pos = (double *)malloc(sizeof(double) * 3 * n);
  s->q = (double *)malloc(sizeof(double) * n);
  memcpy(s->pos, pos, sizeof(double) * 3 * n);
  memcpy(s->q, q, sizeof(double) * n);
  s->nL = ncell_axis(levels);
  s->inv_wL = (double)s->nL / a;
  int ncell = s->nL * s->nL * s->nL;
  s->items = (int64_t **)calloc(ncell, sizeof(int64_t *));
  s->cnt = (int *)calloc(ncell, sizeof(int));
  s->cap = (int *)calloc(ncell, sizeof(int));
  s->cell_of = (int *)malloc(sizeof(int) * n);
  for (int64_t i = 0; i < n; i++) {
    int c[3];
    finest_cell(s, &s->pos[3 * i], c);
    s->cell_of[i] = lin(s->nL, c);
    cell_list_add(s, s->cell_of[i], i);
  }
  for (int l = 2; l <= levels; l++) {
    int nl = ncell_axis(l);
    s->Lx[l] = (cplx *)calloc((size_t)nl * nl * nl * s->C, sizeof(cplx));
  }
  s->K = (cplx *)calloc(s->C, sizeof(cplx));
  s->E = (cplx *)calloc(s->C, sizeof(cplx));
  int lmax = 2 * p;
  s->Slat = (cplx *)calloc((lmax + 1) * (lmax + 1), sizeof(cplx));
  if (bc == ORC_BC_PBC) {
    double *tmp = (double *)malloc(sizeof(double) * 2 * (lmax + 1) * (lmax + 1));
    orc_lattice_sums(lmax, tmp);
    for (int k = 0; k < (lmax + 1) * (lmax + 1); k++) s->Slat[k] = tmp[2 * k] + I * tmp[2 * k + 1];
    free(tmp);
  }
  {
    s->m2lf = (double *)malloc(sizeof(double) * s->C * s->C);
    for (int j = 0; j <= p; j++)
      for (int k = -j; k <= j; k++)
        for (int n = 0; n <= p; n++)
          for (int m = -n; m <= n; m++)
            s->m2lf[(size_t)IDX(j, k) * s->C + IDX(n, m)] = m2l_factor(j, k, n, m);
  }
  int Cw = (2 * p + 1) * (2 * p + 1);
  s->w1 = (cplx *)malloc(sizeof(cplx) * Cw);
  s->w2 = (cplx *)malloc(sizeof(cplx) * Cw);
  s->w3 = (cplx *)malloc(sizeof(cplx) * Cw);
  s->w4 = (cplx *)malloc(sizeof(cplx) * Cw);
  return s;
}

void orc_destroy(orc_sys *s) {
  if (!s) return;
  int ncell = s->nL * s->nL * s->nL;
  for (int c = 0; c < ncell; c++) free(s->items[c]);
  free(s->items);
  free(s->cnt);
  free(s->cap);
  free(s->cell_of);
  for (int l = 2; l <= s->L; l++) free(s->Lx[l]);
  for (int l = 2; l <= s->L; l++) free(s->Mx[l]);
  free(s->K);
  free(s->E);
  free(s->Slat);
  free(s->pos);
  free(s->q);
  free(s->w1);
  free(s->w2);
  free(s->w3);
  free(s->w4);
  free(s->m2lf);
  free(s);
}

/* R applied to a box multipole: H_j^k = sum K_n^m (M2L factor)
 * S_{j+n}^{m-k} a^-(j+n+1).  The lattice sums replace the single
 * translation kernel of one image by its sum over all images outside the
 * extended domain. */
static void apply_R(const orc_sys *s, const cplx *Kin, cplx *Hout) {
  int p = s->p, lmax = 2 * p, C = s->C;
  cplx *G = s->w4;
  for (int l = 0; l <= lmax; l++) {
    double sc = pow(s->a, -(double)(l + 1));
    for (int m = -l; m <= l; m++) G[IDX(l, m)] = s->Slat[IDX(l, m)] * sc;
  }
  /* same sum as m2l_apply, with the translation factors tabulated */
  for (int j = 0; j <= p; j++)
    for (int k = -j; k <= j; k++) {
      const double *f = s->m2lf + (size_t)IDX(j, k) * C;
      cplx acc = 0.0;
      for (int n = 0; n <= p; n++)
        for (int m = -n; m <= n; m++) acc += Kin[IDX(n, m)] * f[IDX(n, m)] * G[IDX(j + n, m - k)];
      Hout[IDX(j, k)] = acc;
    }
}

static const double *R1(const orc_sys *s, double c[3]) {
  c[0] = c[1] = c[2] = 0.5 * s->a;
  return c;
}

/* ---- Alg. L.3: initialise the local coefficients ---- */
static void setup_local(orc_sys *s) {
  int C = s->C;
  int off[189][3];
  cplx *irr = s->w1;
  for (int l = 2; l <= s->L; l++) {
    int nl = ncell_axis(l);
    memset(s->Lx[l], 0, sizeof(cplx) * (size_t)nl * nl * nl * C);
    for (int64_t i = 0; i < s->n; i++) {
      int cf[3], c[3];
      finest_cell(s, &s->pos[3 * i], cf);
      for (int d = 0; d < 3; d++) c[d] = cf[d] >> (s->L - l);
      int nIL = il_offsets(c, off);
      for (int k = 0; k < nIL; k++) {
        int e[3] = {c[0] + off[k][0], c[1] + off[k][1], c[2] + off[k][2]}, cc[3], sh[3];
        if (!wrap_cell(s, nl, e, cc, sh)) continue;
        double Rb[3], d[3];
        cell_centre(s, l, e, Rb);
        for (int t = 0; t < 3; t++) d[t] = s->pos[3 * i + t] - Rb[t];
        irregular_table(s->p, d, irr);
        cplx *Lb = s->Lx[l] + (size_t)lin(nl, cc) * C;
        for (int nn = 0; nn <= s->p; nn++)
          for (int m = -nn; m <= nn; m++) Lb[IDX(nn, m)] += s->q[i] * irr[IDX(nn, -m)];
      }
    }
  }
}

/* ---- FMM-variant initialisation (Sec. 3.2, last paragraph): multipole
 * expansions (Eq. 4) of every cell, then for every cell its local expansion
 * Psi^Delta as the sum of the multipole-to-local translations of the cells
 * of its interaction list (no local-to-local accumulation: the per-level
 * expansions are kept separate).  Multipoles are taken directly from the
 * particles on each level (the truncated upward translation is exact, so this
 * is the same multipole set). ---- */
/* sum over the interaction list of one target cell bc of level l of the
 * multipole-to-local translations; Mlev holds the level's multipoles, or is
 * NULL to take each source multipole directly from the particles */
static void fmm_target(orc_sys *s, int l, const int bc[3], const cplx *Mlev, cplx *Lb) {
  int C = s->C, p = s->p, C2 = (2 * p + 1) * (2 * p + 1);
  int nl = ncell_axis(l);
  double w = cell_width(s, l);
  int off[189][3];
  cplx *G = (cplx *)malloc(sizeof(cplx) * C2);
  cplx *T = (cplx *)malloc(sizeof(cplx) * C);
  cplx *Ms = (cplx *)malloc(sizeof(cplx) * C);
  cplx *R = (cplx *)malloc(sizeof(cplx) * C);
  memset(Lb, 0, sizeof(cplx) * C);
  int nIL = il_offsets(bc, off);
  for (int k = 0; k < nIL; k++) {
    int e[3] = {bc[0] + off[k][0], bc[1] + off[k][1], bc[2] + off[k][2]}, cc[3], sh[3];
    if (!wrap_cell(s, nl, e, cc, sh)) continue;
    const cplx *M;
    if (Mlev) {
      M = Mlev + (size_t)lin(nl, cc) * C;
    } else {
      /* Eq. (4) about the source cell's centre, from its charges */
      memset(Ms, 0, sizeof(cplx) * C);
      double Rc[3], d3[3];
      cell_centre(s, l, cc, Rc);
      for (int64_t i = 0; i < s->n; i++) {
        int cf[3];
        finest_cell(s, &s->pos[3 * i], cf);
        if ((cf[0] >> (s->L - l)) != cc[0] || (cf[1] >> (s->L - l)) != cc[1] ||
            (cf[2] >> (s->L - l)) != cc[2])
          continue;
        for (int t = 0; t < 3; t++) d3[t] = s->pos[3 * i + t] - Rc[t];
        regular_table(p, d3, R);
        for (int nn = 0; nn <= p; nn++)
          for (int m = -nn; m <= nn; m++) Ms[IDX(nn, m)] += s->q[i] * R[IDX(nn, -m)];
      }
      M = Ms;
    }
    /* source multipole centre relative to the target centre */
    double cvec[3] = {off[k][0] * w, off[k][1] * w, off[k][2] * w};
    irregular_table(2 * p, cvec, G);
    /* m2l_apply with the translation factors tabulated */
    for (int j = 0; j <= p; j++)
      for (int kk = -j; kk <= j; kk++) {
        const double *f = s->m2lf + (size_t)IDX(j, kk) * C;
        cplx acc = 0.0;
        for (int n = 0; n <= p; n++)
          for (int m = -n; m <= n; m++) acc += M[IDX(n, m)] * f[IDX(n, m)] * G[IDX(j + n, m - kk)];
        T[IDX(j, kk)] = acc;
      }
    for (int q = 0; q < C; q++) Lb[q] += T[q];
  }
  free(G);
  free(T);
  free(Ms);
  free(R);
}

/* Eq. (4) about each cell centre of level l, into M (zeroed here); the
 * loop of Alg. M.3 for one level */
static void multipoles_level(orc_sys *s, int l, cplx *M) {
  int C = s->C, p = s->p, nl = ncell_axis(l);
  cplx *R = (cplx *)malloc(sizeof(cplx) * C);
  memset(M, 0, sizeof(cplx) * (size_t)nl * nl * nl * C);
  for (int64_t i = 0; i < s->n; i++) {
    int cf[3], c[3];
    finest_cell(s, &s->pos[3 * i], cf);
    for (int d = 0; d < 3; d++) c[d] = cf[d] >> (s->L - l);
    double Rc[3], d3[3];
    cell_centre(s, l, c, Rc);
    for (int t = 0; t < 3; t++) d3[t] = s->pos[3 * i + t] - Rc[t];
    regular_table(p, d3, R);
    cplx *Mc = M + (size_t)lin(nl, c) * C;
    for (int nn = 0; nn <= p; nn++)
      for (int m = -nn; m <= nn; m++) Mc[IDX(nn, m)] += s->q[i] * R[IDX(nn, -m)];
  }
  free(R);
}

static void setup_local_fmm(orc_sys *s) {
  int C = s->C;
  for (int l = 2; l <= s->L; l++) {
    int nl = ncell_axis(l);
    size_t ncell = (size_t)nl * nl * nl;
    cplx *M = (cplx *)malloc(sizeof(cplx) * ncell * C);
    multipoles_level(s, l, M);
    for (size_t b = 0; b < ncell; b++) {
      int bc[3] = {(int)(b / ((size_t)nl * nl)), (int)((b / nl) % nl), (int)(b % nl)};
      fmm_target(s, l, bc, M, s->Lx[l] + b * C);
    }
    free(M);
  }
}

/* Alg. M.3 (the multipole method's initialisation) with the K/E of
 * Sec. 3.4 (ii); the system then proposes and accepts with Alg. M.1/M.2 */
void orc_setup_multipole(orc_sys *s) {
  s->method = 1;
  for (int l = 2; l <= s->L; l++) {
    int nl = ncell_axis(l);
    if (!s->Mx[l]) s->Mx[l] = (cplx *)malloc(sizeof(cplx) * (size_t)nl * nl * nl * s->C);
    multipoles_level(s, l, s->Mx[l]);
  }
  if (s->bc == ORC_BC_PBC) setup_KE(s);
  s->energy = orc_energy_fresh(s);
}

/* switch on the Lennard-Jones term; rc must not exceed the finest cell
 * width (every pair within rc is in the 27 near cells); -1 otherwise */
int orc_set_lj(orc_sys *s, double eps, double sig, double rc) {
  if (eps < 0.0 || sig <= 0.0 || rc <= 0.0 || rc > cell_width(s, s->L)) return -1;
  s->lj_eps = eps;
  s->lj_sig = sig;
  s->lj_rc = rc;
  return 0;
}

/* multipoles of level `level` (real layout of the unscaled M_n^m) */
int orc_get_multipole(const orc_sys *s, int level, double *out) {
  if (level < 2 || level > s->L || !s->Mx[level]) return -1;
  int nl = ncell_axis(level);
  for (int c = 0; c < nl * nl * nl; c++)
    to_real_layout(s->p, s->Mx[level] + (size_t)c * s->C, out + (size_t)c * s->C);
  return 0;
}

/* one cell's FMM-variant expansion (real layout), all from the particles:
 * for sampled checks at sizes where the whole pass is too slow */
/* Psi^Delta of one target cell c of level l by its definition (Alg. L.3,
 * Eq. 1): the sum over the entries f of IL(c) -- each the image of a
 * canonical cell shifted by sh boxes -- of the charges i of that cell,
 * q_i conj It(r_i + sh a - R_c).  By the symmetry of the interaction list
 * this is the value setup_local scatters into cell c; here it is gathered
 * for one cell (O(N) to find the charges), for sampled cells of systems too
 * large for the full setup. */
int orc_local_cell_direct(orc_sys *s, int l, const int c[3], double *out) {
  if (l < 2 || l > s->L) return -1;
  const int nl = ncell_axis(l), C = s->C;
  for (int d = 0; d < 3; d++)
    if (c[d] < 0 || c[d] >= nl) return -1;
  int off[189][3], src[189], shf[189][3];
  const int nIL = il_offsets(c, off);
  /* entries by canonical source cell: first[cell] -> entry, nxt[entry] */
  int *first = (int *)malloc(sizeof(int) * (size_t)nl * nl * nl);
  int nxt[189];
  for (int64_t k = 0; k < (int64_t)nl * nl * nl; k++) first[k] = -1;
  for (int k = 0; k < nIL; k++) {
    const int e[3] = {c[0] + off[k][0], c[1] + off[k][1], c[2] + off[k][2]};
    int cc[3];
    src[k] = -1;
    if (!wrap_cell(s, nl, e, cc, shf[k])) continue;
    src[k] = lin(nl, cc);
    nxt[k] = first[src[k]];
    first[src[k]] = k;
  }
  double Rc[3];
  cell_centre(s, l, c, Rc);
  cplx *Lb = (cplx *)calloc((size_t)C, sizeof(cplx));
  cplx *irr = (cplx *)malloc(sizeof(cplx) * C);
  for (int64_t i = 0; i < s->n; i++) {
    int cf[3], ci[3];
    finest_cell(s, &s->pos[3 * i], cf);
    for (int d = 0; d < 3; d++) ci[d] = cf[d] >> (s->L - l);
    for (int k = first[lin(nl, ci)]; k >= 0; k = nxt[k]) {
      double d3[3];
      for (int t = 0; t < 3; t++) d3[t] = s->pos[3 * i + t] + shf[k][t] * s->a - Rc[t];
      irregular_table(s->p, d3, irr);
      for (int nn = 0; nn <= s->p; nn++)
        for (int m = -nn; m <= nn; m++) Lb[IDX(nn, m)] += s->q[i] * irr[IDX(nn, -m)];
    }
  }
  to_real_layout(s->p, Lb, out);
  free(irr);
  free(Lb);
  free(first);
  return 0;
}

int orc_fmm_local_cell(orc_sys *s, int l, const int c[3], double *out) {
  if (l < 2 || l > s->L) return -1;
  cplx *Lb = (cplx *)malloc(sizeof(cplx) * s->C);
  fmm_target(s, l, c, NULL, Lb);
  to_real_layout(s->p, Lb, out);
  free(Lb);
  return 0;
}

void orc_setup_fmm(orc_sys *s) {
  s->method = 0;
  setup_local_fmm(s);
  if (s->bc == ORC_BC_PBC) setup_KE(s);
  s->energy = orc_energy_fresh(s);
}

/* ---- Sec. 3.4 (ii): K_n^m = sum q r^n Y_n^-m, E_n^m = sum q r^n Y_n^m ---- */
static void setup_KE(orc_sys *s) {
  memset(s->K, 0, sizeof(cplx) * s->C);
  memset(s->E, 0, sizeof(cplx) * s->C);
  s->D[0] = s->D[1] = s->D[2] = 0.0;
  double c1[3];
  R1(s, c1);
  for (int64_t i = 0; i < s->n; i++) {
    double d[3];
    for (int t = 0; t < 3; t++) d[t] = s->pos[3 * i + t] - c1[t];
    regular_table(s->p, d, s->w1);
    for (int nn = 0; nn <= s->p; nn++)
      for (int m = -nn; m <= nn; m++) {
        s->K[IDX(nn, m)] += s->q[i] * s->w1[IDX(nn, -m)];
        s->E[IDX(nn, m)] += s->q[i] * s->w1[IDX(nn, m)];
      }
    for (int t = 0; t < 3; t++) s->D[t] += s->q[i] * s->pos[3 * i + t];
  }
}

/* Psi^Delta_{l,alpha}(x - R_alpha) of Eq. (2) */
static double psi_level(orc_sys *s, int l, const int c[3], const double x[3]) {
  int nl = ncell_axis(l);
  double R[3], d[3];
  cell_centre(s, l, c, R);
  for (int t = 0; t < 3; t++) d[t] = x[t] - R[t];
  return eval_local(s->p, s->Lx[l] + (size_t)lin(nl, c) * s->C, d, s->w2);
}

/* the multipole method's level sum: sum over the interaction list of cell c
 * of level l of the multipole expansion (the paper's Phi) of each listed
 * cell (image-shifted centre) at x */
static double phi_mm_level(orc_sys *s, int l, const int c[3], const double x[3]) {
  int nl = ncell_axis(l), off[189][3];
  int nIL = il_offsets(c, off);
  double acc = 0.0;
  for (int k = 0; k < nIL; k++) {
    int e[3] = {c[0] + off[k][0], c[1] + off[k][1], c[2] + off[k][2]}, cc[3], sh[3];
    if (!wrap_cell(s, nl, e, cc, sh)) continue;
    double R[3], d[3];
    cell_centre(s, l, e, R);
    for (int t = 0; t < 3; t++) d[t] = x[t] - R[t];
    irregular_table(s->p, d, s->w2);
    const cplx *M = s->Mx[l] + (size_t)lin(nl, cc) * s->C;
    cplx v = 0.0;
    for (int n = 0; n <= s->p; n++)
      for (int m = -n; m <= n; m++) v += M[IDX(n, m)] * s->w2[IDX(n, m)];
    acc += creal(v);
  }
  return acc;
}

/* level-l contribution to the potential at x in cell c (either method) */
static double level_potential(orc_sys *s, int l, const int c[3], const double x[3]) {
  return s->method ? phi_mm_level(s, l, c, x) : psi_level(s, l, c, x);
}

/* U^inf = 1/2 sum E_n^m H_n^m.  The paper prints the sum without the 1/2;
 * the pair energy of the far images carries it, so we read the factor as
 * part of the definition (checked against Ewald summation). */
static double far_energy(orc_sys *s, const cplx *K, const cplx *E) {
  apply_R(s, K, s->w3);
  cplx acc = 0.0;
  for (int k = 0; k < s->C; k++) acc += E[k] * s->w3[k];
  return 0.5 * creal(acc);
}

/* tinfoil dipole term -2 pi |D|^2 / (3 V) (reading: the paper is silent on
 * the dipole boundary condition; cubic-shell summation gives the vacuum
 * result, conducting surroundings subtract this term as Ewald does) */
static double dipole_energy(const orc_sys *s, const double D[3]) {
  if (s->bc != ORC_BC_PBC || s->dip != ORC_TINFOIL) return 0.0;
  double V = s->a * s->a * s->a;
  return -2.0 * M_PI / (3.0 * V) * (D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
}

/* Lennard-Jones pair energy, truncated at rc (0 beyond) */
static double lj_pair(const orc_sys *s, double r) {
  if (s->lj_eps == 0.0 || r >= s->lj_rc) return 0.0;
  double sr6 = pow(s->lj_sig / r, 6.0);
  return 4.0 * s->lj_eps * (sr6 * sr6 - sr6);
}

/* Lennard-Jones energy of particle at x (id i, excluded with all its
 * images: they lie beyond rc) with the charges of the 27 near cells */
static double lj_particle(orc_sys *s, int64_t i, const double x[3]) {
  if (s->lj_eps == 0.0) return 0.0;
  int cf[3];
  finest_cell(s, x, cf);
  double u = 0.0;
  for (int dx = -1; dx <= 1; dx++)
    for (int dy = -1; dy <= 1; dy++)
      for (int dz = -1; dz <= 1; dz++) {
        int e[3] = {cf[0] + dx, cf[1] + dy, cf[2] + dz}, cc[3], sh[3];
        if (!wrap_cell(s, s->nL, e, cc, sh)) continue;
        int cell = lin(s->nL, cc);
        for (int k = 0; k < s->cnt[cell]; k++) {
          int64_t t = s->items[cell][k];
          if (t == i) continue;
          double d[3];
          for (int w = 0; w < 3; w++) d[w] = x[w] - (s->pos[3 * t + w] + sh[w] * s->a);
          u += lj_pair(s, sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]));
        }
      }
  return u;
}

/* potential at particle i from everything except itself at its own
 * position: level expansions plus direct near cells */
static double phi_particle(orc_sys *s, int64_t i) {
  const double *x = &s->pos[3 * i];
  int cf[3];
  finest_cell(s, x, cf);
  double phi = 0.0;
  for (int l = s->L; l >= 2; l--) {
    int c[3] = {cf[0] >> (s->L - l), cf[1] >> (s->L - l), cf[2] >> (s->L - l)};
    phi += level_potential(s, l, c, x);
  }
  for (int dx = -1; dx <= 1; dx++)
    for (int dy = -1; dy <= 1; dy++)
      for (int dz = -1; dz <= 1; dz++) {
        int e[3] = {cf[0] + dx, cf[1] + dy, cf[2] + dz}, cc[3], sh[3];
        if (!wrap_cell(s, s->nL, e, cc, sh)) continue;
        int cell = lin(s->nL, cc);
        for (int k = 0; k < s->cnt[cell]; k++) {
          int64_t t = s->items[cell][k];
          if (t == i && sh[0] == 0 && sh[1] == 0 && sh[2] == 0) continue;
          double d[3];
          for (int u = 0; u < 3; u++) d[u] = x[u] - (s->pos[3 * t + u] + sh[u] * s->a);
          phi += s->q[t] / sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        }
      }
  return phi;
}

double orc_energy_fresh(orc_sys *s) {
  double U = 0.0;
  for (int64_t i = 0; i < s->n; i++)
    U += 0.5 * s->q[i] * phi_particle(s, i) + 0.5 * lj_particle(s, i, &s->pos[3 * i]);
  if (s->bc == ORC_BC_PBC) {
    U += far_energy(s, s->K, s->E);
    U += dipole_energy(s, s->D);
  }
  return U;
}

void orc_setup(orc_sys *s) {
  s->method = 0;
  setup_local(s);
  if (s->bc == ORC_BC_PBC) setup_KE(s);
  s->energy = orc_energy_fresh(s);
}

/* ---- Alg. L.1 with Alg. 1 and the periodic extensions ---- */
double orc_propose(orc_sys *s, int64_t j, const double rnew[3]) {
  const double *r = &s->pos[3 * j];
  double q = s->q[j];
  s->parts[0] = s->parts[1] = s->parts[2] = s->parts[3] = 0.0;
  if (r[0] == rnew[0] && r[1] == rnew[1] && r[2] == rnew[2]) return 0.0;
  if (s->bc == ORC_BC_FREE)
    for (int t = 0; t < 3; t++)
      if (!(rnew[t] >= 0.0 && rnew[t] < s->a)) return INFINITY;
  int cf[3], cfn[3];
  finest_cell(s, r, cf);
  finest_cell(s, rnew, cfn);

  /* expansions on levels L..2 (level 1 holds no interactions: with
   * periodic boundaries everything outside the extended domain is in K/E) */
  double dU_exp = 0.0;
  for (int l = s->L; l >= 2; l--) {
    int c[3], cn[3];
    for (int t = 0; t < 3; t++) {
      c[t] = cf[t] >> (s->L - l);
      cn[t] = cfn[t] >> (s->L - l);
    }
    dU_exp += q * (level_potential(s, l, cn, rnew) - level_potential(s, l, c, r));
  }

  /* Alg. 1: direct interactions with the 27 near cells (cells of the
   * extended domain with periodic boundaries).  Old side: everything but
   * the moving particle itself.  New side: the current particle data, which
   * still holds the moving particle at its old position. */
  double dU_dir = 0.0;
  int overlap = 0;
  for (int side = 0; side < 2; side++) {
    const int *cc0 = side ? cfn : cf;
    const double *x = side ? rnew : r;
    for (int dx = -1; dx <= 1; dx++)
      for (int dy = -1; dy <= 1; dy++)
        for (int dz = -1; dz <= 1; dz++) {
          int e[3] = {cc0[0] + dx, cc0[1] + dy, cc0[2] + dz}, cc[3], sh[3];
          if (!wrap_cell(s, s->nL, e, cc, sh)) continue;
          int cell = lin(s->nL, cc);
          for (int k = 0; k < s->cnt[cell]; k++) {
            int64_t i = s->items[cell][k];
            if (side == 0 && i == j && sh[0] == 0 && sh[1] == 0 && sh[2] == 0) continue;
            double d[3];
            for (int u = 0; u < 3; u++) d[u] = x[u] - (s->pos[3 * i + u] + sh[u] * s->a);
            double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (side == 1 && dist == 0.0) overlap = 1;
            if (side == 0)
              dU_dir -= q * s->q[i] / dist;
            else
              dU_dir += q * s->q[i] / dist;
          }
        }
  }
  /* self-interaction removal of Alg. 1, replaced with periodic
   * boundaries by the sum over the 27 images plus the constant for the 26
   * image copies counted on the old side */
  if (s->bc == ORC_BC_PBC) {
    for (int nx = -1; nx <= 1; nx++)
      for (int ny = -1; ny <= 1; ny++)
        for (int nz = -1; nz <= 1; nz++) {
          double d[3] = {rnew[0] - (r[0] + nx * s->a), rnew[1] - (r[1] + ny * s->a),
                         rnew[2] - (r[2] + nz * s->a)};
          dU_dir -= q * q / sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        }
    dU_dir += q * q / s->a * (6.0 + 8.0 / sqrt(3.0) + 12.0 / sqrt(2.0));
  } else {
    double d[3] = {rnew[0] - r[0], rnew[1] - r[1], rnew[2] - r[2]};
    dU_dir -= q * q / sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  }

  /* short-range Lennard-Jones change (the moving particle's own copy and
   * images excluded on both sides) */
  dU_dir += lj_particle(s, j, rnew) - lj_particle(s, j, r);

  double dU_far = 0.0, dU_dip = 0.0;
  if (s->bc == ORC_BC_PBC) {
    /* Sec. 3.4 (iv), literal: H = R(K), U = E.H, post-move dK, dE,
     * dH = R(dK), dU = dE.dH - U (with the factor 1/2, see far_energy) */
    double U_inf = far_energy(s, s->K, s->E);
    double c1[3], d0[3], d1[3];
    R1(s, c1);
    for (int t = 0; t < 3; t++) {
      d0[t] = r[t] - c1[t];
      d1[t] = rnew[t] - c1[t];
    }
    cplx *Sa = s->w1, *Sb = s->w2;
    regular_table(s->p, d0, Sa);
    regular_table(s->p, d1, Sb);
    cplx *dK = (cplx *)malloc(sizeof(cplx) * s->C);
    cplx *dE = (cplx *)malloc(sizeof(cplx) * s->C);
    for (int nn = 0; nn <= s->p; nn++)
      for (int m = -nn; m <= nn; m++) {
        dK[IDX(nn, m)] = s->K[IDX(nn, m)] + q * (Sb[IDX(nn, -m)] - Sa[IDX(nn, -m)]);
        dE[IDX(nn, m)] = s->E[IDX(nn, m)] + q * (Sb[IDX(nn, m)] - Sa[IDX(nn, m)]);
      }
    dU_far = far_energy(s, dK, dE) - U_inf;
    free(dK);
    free(dE);
    double Dn[3];
    for (int t = 0; t < 3; t++) Dn[t] = s->D[t] + q * (rnew[t] - r[t]);
    dU_dip = dipole_energy(s, Dn) - dipole_energy(s, s->D);
  }
  s->parts[0] = dU_exp;
  s->parts[1] = dU_dir;
  s->parts[2] = dU_far;
  s->parts[3] = dU_dip;
  if (overlap) return INFINITY;
  return dU_exp + dU_dir + dU_far + dU_dip;
}

void orc_last_parts(const orc_sys *s, double parts[4]) {
  for (int k = 0; k < 4; k++) parts[k] = s->parts[k];
}

/* the same far-field change written as Re(d^H H) + 1/2 d^H R d with
 * d the change of K; equal to the literal form when R is Hermitian */
double orc_far_delta_factored(orc_sys *s, int64_t j, const double rnew[3]) {
  if (s->bc != ORC_BC_PBC) return 0.0;
  const double *r = &s->pos[3 * j];
  double q = s->q[j], c1[3], d0[3], d1[3];
  R1(s, c1);
  for (int t = 0; t < 3; t++) {
    d0[t] = r[t] - c1[t];
    d1[t] = rnew[t] - c1[t];
  }
  cplx *Sa = s->w1, *Sb = s->w2;
  regular_table(s->p, d0, Sa);
  regular_table(s->p, d1, Sb);
  cplx *dK = (cplx *)malloc(sizeof(cplx) * s->C);
  cplx *H = (cplx *)malloc(sizeof(cplx) * s->C);
  cplx *RdK = (cplx *)malloc(sizeof(cplx) * s->C);
  for (int nn = 0; nn <= s->p; nn++)
    for (int m = -nn; m <= nn; m++) dK[IDX(nn, m)] = q * (Sb[IDX(nn, -m)] - Sa[IDX(nn, -m)]);
  apply_R(s, s->K, H);
  apply_R(s, dK, RdK);
  cplx a1 = 0.0, a2 = 0.0;
  for (int k = 0; k < s->C; k++) {
    a1 += conj(dK[k]) * H[k];
    a2 += conj(dK[k]) * RdK[k];
  }
  free(dK);
  free(H);
  free(RdK);
  return creal(a1) + 0.5 * creal(a2);
}

/* ---- Alg. L.2 with the K/E update of Sec. 3.4 (iii) ---- */
void orc_accept(orc_sys *s, int64_t j, const double rnew[3], double dE) {
  double *r = &s->pos[3 * j];
  double q = s->q[j];
  if (r[0] == rnew[0] && r[1] == rnew[1] && r[2] == rnew[2]) return;
  int cf[3], cfn[3], off[189][3];
  finest_cell(s, r, cf);
  finest_cell(s, rnew, cfn);
  int C = s->C;
  cplx *irr = s->w1;
  /* Alg. M.2: remove the charge from the multipoles of its old cells and
   * add it to those of its new cells on every level */
  for (int l = s->L; s->method && l >= 2; l--) {
    int nl = ncell_axis(l);
    for (int side = 0; side < 2; side++) {
      const int *cfs = side ? cfn : cf;
      const double *x = side ? rnew : r;
      double sg = side ? q : -q;
      int c[3] = {cfs[0] >> (s->L - l), cfs[1] >> (s->L - l), cfs[2] >> (s->L - l)};
      double Rc[3], d[3];
      cell_centre(s, l, c, Rc);
      for (int t = 0; t < 3; t++) d[t] = x[t] - Rc[t];
      regular_table(s->p, d, irr);
      cplx *Mc = s->Mx[l] + (size_t)lin(nl, c) * C;
      for (int nn = 0; nn <= s->p; nn++)
        for (int m = -nn; m <= nn; m++) Mc[IDX(nn, m)] += sg * irr[IDX(nn, -m)];
    }
  }
  for (int l = s->L; !s->method && l >= 2; l--) {
    int nl = ncell_axis(l);
    for (int side = 0; side < 2; side++) {
      const int *cfs = side ? cfn : cf;
      const double *x = side ? rnew : r;
      double sg = side ? q : -q;
      int c[3] = {cfs[0] >> (s->L - l), cfs[1] >> (s->L - l), cfs[2] >> (s->L - l)};
      int nIL = il_offsets(c, off);
      for (int k = 0; k < nIL; k++) {
        int e[3] = {c[0] + off[k][0], c[1] + off[k][1], c[2] + off[k][2]}, cc[3], sh[3];
        if (!wrap_cell(s, nl, e, cc, sh)) continue;
        double Rb[3], d[3];
        cell_centre(s, l, e, Rb);
        for (int t = 0; t < 3; t++) d[t] = x[t] - Rb[t];
        irregular_table(s->p, d, irr);
        cplx *Lb = s->Lx[l] + (size_t)lin(nl, cc) * C;
        for (int nn = 0; nn <= s->p; nn++)
          for (int m = -nn; m <= nn; m++) Lb[IDX(nn, m)] += sg * irr[IDX(nn, -m)];
      }
    }
  }
  if (s->bc == ORC_BC_PBC) {
    double c1[3], d0[3], d1[3];
    R1(s, c1);
    for (int t = 0; t < 3; t++) {
      d0[t] = r[t] - c1[t];
      d1[t] = rnew[t] - c1[t];
    }
    regular_table(s->p, d0, s->w1);
    regular_table(s->p, d1, s->w2);
    for (int nn = 0; nn <= s->p; nn++)
      for (int m = -nn; m <= nn; m++) {
        s->K[IDX(nn, m)] += q * (s->w2[IDX(nn, -m)] - s->w1[IDX(nn, -m)]);
        s->E[IDX(nn, m)] += q * (s->w2[IDX(nn, m)] - s->w1[IDX(nn, m)]);
      }
    for (int t = 0; t < 3; t++) s->D[t] += q * (rnew[t] - r[t]);
  }
  int oldc = s->cell_of[j], newc = lin(s->nL, cfn);
  if (oldc != newc) {
    cell_list_remove(s, oldc, j);
    cell_list_add(s, newc, j);
    s->cell_of[j] = newc;
  }
  for (int t = 0; t < 3; t++) r[t] = rnew[t];
  s->energy += dE;
}

double orc_energy(const orc_sys *s) { return s->energy; }

void orc_get_positions(const orc_sys *s, double *out) {
  memcpy(out, s->pos, sizeof(double) * 3 * s->n);
}

/* real layout: per n, Re X_n^0 then (Re X_n^m, Im X_n^m) for m = 1..n */
static void to_real_layout(int p, const cplx *X, double *out) {
  for (int n = 0; n <= p; n++) {
    out[n * n] = creal(X[IDX(n, 0)]);
    for (int m = 1; m <= n; m++) {
      out[n * n + 2 * m - 1] = creal(X[IDX(n, m)]);
      out[n * n + 2 * m] = cimag(X[IDX(n, m)]);
    }
  }
}

int orc_get_local(const orc_sys *s, int level, double *out) {
  if (level < 2 || level > s->L) return -1;
  int nl = ncell_axis(level);
  for (int c = 0; c < nl * nl * nl; c++)
    to_real_layout(s->p, s->Lx[level] + (size_t)c * s->C, out + (size_t)c * s->C);
  return 0;
}

void orc_get_KH(orc_sys *s, double *K, double *H) {
  cplx *Hc = (cplx *)malloc(sizeof(cplx) * s->C);
  apply_R(s, s->K, Hc);
  to_real_layout(s->p, s->K, K);
  to_real_layout(s->p, Hc, H);
  free(Hc);
}

double orc_dipole_energy_coeff(const orc_sys *s) {
  return (s->bc == ORC_BC_PBC && s->dip == ORC_TINFOIL) ? -2.0 * M_PI / (3.0 * s->a * s->a * s->a)
                                                        : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
 * two 32x32->64 multiplies with constants 0xD2511F53, 0xCD9E8D57; the key
 * is bumped by the Weyl constants 0x9E3779B9, 0xBB67AE85 between rounds.    */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; round++) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* Proposal stream (reading; the paper leaves the MC driver to the user):
 * key = (seed_lo, seed_hi); block A from counter (step_lo, step_hi, chain, 0),
 * block B from (step_lo, step_hi, chain, 1).  j = floor(A0 * n / 2^32);
 * delta_k = h (2 u_k - 1) with u_k = (A_k + 1/2) 2^-32 for k = 1..3;
 * acceptance uniform u = ((B0 >> 5) 2^26 + (B1 >> 6)) 2^-53.              */
void orc_proposal(int64_t n, double half_width, uint64_t seed, uint64_t step, uint32_t chain,
                  int64_t *j, double delta[3], double *u) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t ca[4] = {(uint32_t)step, (uint32_t)(step >> 32), chain, 0u};
  uint32_t cb[4] = {(uint32_t)step, (uint32_t)(step >> 32), chain, 1u};
  uint32_t A[4], B[4];
  orc_philox4x32_10(ca, key, A);
  orc_philox4x32_10(cb, key, B);
  *j = (int64_t)(((uint64_t)A[0] * (uint64_t)n) >> 32);
  for (int k = 0; k < 3; k++) {
    double uk = ((double)A[k + 1] + 0.5) * (1.0 / 4294967296.0);
    delta[k] = half_width * (2.0 * uk - 1.0);
  }
  *u = ((double)(B[0] >> 5) * 67108864.0 + (double)(B[1] >> 6)) * (1.0 / 9007199254740992.0);
}

/* Metropolis-Hastings: accept iff dE <= 0 or log(u) < -beta dE.  A decision
 * within 1e-9 (relative) of the threshold is counted as borderline.  With
 * `follow` (a driver option for checking a chain whose energy changes carry
 * a known rounding error, the paper has no counterpart), step t is accepted
 * iff follow[t] != 0 whatever the rule says, and log_acc still records the
 * rule's own decision. */
static int64_t run_chain(orc_sys *s, int64_t n_steps, uint64_t seed, uint64_t step0,
                         uint32_t chain, double beta, double half_width, const uint8_t *follow,
                         int64_t *log_j, double *log_dE, uint8_t *log_acc,
                         int64_t *n_borderline) {
  int64_t n_acc = 0, nb = 0;
  for (int64_t t = 0; t < n_steps; t++) {
    int64_t j;
    double delta[3], u, rnew[3];
    orc_proposal(s->n, half_width, seed, step0 + (uint64_t)t, chain, &j, delta, &u);
    for (int k = 0; k < 3; k++) {
      double x = s->pos[3 * j + k] + delta[k];
      if (s->bc == ORC_BC_PBC) {
        if (x < 0.0) x += s->a;
        if (x >= s->a) x -= s->a;
      }
      rnew[k] = x;
    }
    double dE = orc_propose(s, j, rnew);
    int acc;
    if (dE <= 0.0) {
      acc = 1;
    } else {
      double lu = log(u), t2 = -beta * dE;
      acc = lu < t2;
      if (fabs(lu - t2) < 1e-9 * fmax(1.0, fabs(t2))) nb++;
    }
    if (log_j) log_j[t] = j;
    if (log_dE) log_dE[t] = dE;
    if (log_acc) log_acc[t] = (uint8_t)acc;
    if (follow) acc = follow[t] != 0;
    if (acc) {
      orc_accept(s, j, rnew, dE);
      n_acc++;
    }
  }
  if (n_borderline) *n_borderline = nb;
  return n_acc;
}

int64_t orc_run(orc_sys *s, int64_t n_steps, uint64_t seed, uint64_t step0, uint32_t chain,
                double beta, double half_width, int64_t *log_j, double *log_dE,
                uint8_t *log_acc, int64_t *n_borderline) {
  return run_chain(s, n_steps, seed, step0, chain, beta, half_width, NULL, log_j, log_dE, log_acc,
                   n_borderline);
}

int64_t orc_run_follow(orc_sys *s, int64_t n_steps, uint64_t seed, uint64_t step0,
                       uint32_t chain, double beta, double half_width, const uint8_t *follow,
                       int64_t *log_j, double *log_dE, uint8_t *log_acc, int64_t *n_borderline) {
  return run_chain(s, n_steps, seed, step0, chain, beta, half_width, follow, log_j, log_dE,
                   log_acc, n_borderline);
}

/* ------------------------------------------------------------------------ */
/* Ewald summation with conducting (tinfoil) boundary:
 *   U = 1/2 sum_{i,j} sum'_n q_i q_j erfc(kappa |r_ij + n a|) / |r_ij + n a|
 *     + (2 pi / V) sum_{k != 0} exp(-k^2 / 4 kappa^2) / k^2 |sum_j q_j e^{i k.r_j}|^2
 *     - kappa / sqrt(pi) sum_i q_i^2                (neutral systems)       */
/* ------------------------------------------------------------------------ */
double orc_ewald_energy(int64_t n, const double *pos, const double *q, double a, double kappa,
                        int nreal, int nrecip) {
  double Ur = 0.0;
  for (int64_t i = 0; i < n; i++)
    for (int64_t j = 0; j < n; j++)
      for (int x = -nreal; x <= nreal; x++)
        for (int y = -nreal; y <= nreal; y++)
          for (int z = -nreal; z <= nreal; z++) {
            if (i == j && x == 0 && y == 0 && z == 0) continue;
            double d[3] = {pos[3 * i] - pos[3 * j] + x * a, pos[3 * i + 1] - pos[3 * j + 1] + y * a,
                           pos[3 * i + 2] - pos[3 * j + 2] + z * a};
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            Ur += 0.5 * q[i] * q[j] * erfc(kappa * r) / r;
          }
  double Uk = 0.0, V = a * a * a;
  for (int x = -nrecip; x <= nrecip; x++)
    for (int y = -nrecip; y <= nrecip; y++)
      for (int z = -nrecip; z <= nrecip; z++) {
        if (x == 0 && y == 0 && z == 0) continue;
        double k[3] = {2.0 * M_PI * x / a, 2.0 * M_PI * y / a, 2.0 * M_PI * z / a};
        double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        double sr = 0.0, si = 0.0;
        for (int64_t j = 0; j < n; j++) {
          double ph = k[0] * pos[3 * j] + k[1] * pos[3 * j + 1] + k[2] * pos[3 * j + 2];
          sr += q[j] * cos(ph);
          si += q[j] * sin(ph);
        }
        Uk += 2.0 * M_PI / V * exp(-k2 / (4.0 * kappa * kappa)) / k2 * (sr * sr + si * si);
      }
  double Us = 0.0;
  for (int64_t i = 0; i < n; i++) Us -= kappa / sqrt(M_PI) * q[i] * q[i];
  return Ur + Uk + Us;
}

double orc_direct_energy(int64_t n, const double *pos, const double *q) {
  double U = 0.0;
  for (int64_t i = 0; i < n; i++)
    for (int64_t j = i + 1; j < n; j++) {
      double d[3] = {pos[3 * i] - pos[3 * j], pos[3 * i + 1] - pos[3 * j + 1],
                     pos[3 * i + 2] - pos[3 * j + 2]};
      U += q[i] * q[j] / sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    }
  return U;
}
