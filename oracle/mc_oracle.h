/*
 * CPU oracle for the multilevel local-expansion Metropolis-Hastings
 * electrostatics method (Saunders, Grant, Mueller, arXiv 2006.16622).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, single-threaded,
 * obviously-correct reference that the CUDA path is checked against.  Only
 * the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load it.  It shares no code, header, table or constant generator with the
 * CUDA library; the two meet only through seeded inputs.
 *
 * Notation (paper Sec. 3): p = expansion order (largest n), C = (p+1)^2
 * complex coefficients per expansion stored as full (n, m = -n..n) arrays
 * indexed n*n + n + m; L = number of octree levels, level l has 2^(l-1)
 * cells per axis; a = cubic box side.
 */
#ifndef MC_ORACLE_H
#define MC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_BC_PBC 0
#define ORC_BC_FREE 1
#define ORC_TINFOIL 0
#define ORC_VACUUM 1

typedef struct orc_sys orc_sys;

/* ---- special functions (Eq. 2-4 normalisation) ---- */
/* Y_n^m(theta, phi) for all n <= p, m = -n..n; out is complex interleaved
 * (re, im) of length 2*(p+1)^2. */
void orc_ylm(int p, double theta, double phi, double *out);
/* r^n Y_n^m(x/|x|) (regular) and r^-(n+1) Y_n^m (irregular). */
void orc_regular(int p, const double x[3], double *out);
void orc_irregular(int p, const double x[3], double *out);
/* multipole coefficients (Eq. 4) of charges about centre c */
void orc_multipole(int p, int n, const double *pos, const double *q,
                   const double c[3], double *out);
/* M2L: local coefficients about the origin from a multipole about c */
void orc_m2l(int p, const double *M, const double c[3], double *Lout);
/* evaluate a local expansion (Eq. 2) at displacement x; real part */
double orc_eval_local(int p, const double *Lc, const double x[3]);

/* ---- lattice sums for the periodic far field ---- */
/* S_l^m = sum over integer vectors v with max|v_i| >= 2 of
 * Y_l^m(v/|v|) / |v|^(l+1); complex interleaved, l <= lmax. */
void orc_lattice_sums(int lmax, double *out);

/* ---- system ---- */
orc_sys *orc_create(int64_t n, const double *pos, const double *q, double a,
                    int levels, int p, int bc, int dipole_bc);
void orc_destroy(orc_sys *s);
void orc_setup(orc_sys *s);                       /* Alg. L.3 + K/E + U0 */
/* FMM-variant initialisation: per-level multipoles + M2L over interaction lists */
void orc_setup_fmm(orc_sys *s);
/* one cell's FMM-variant expansion (real layout), source multipoles taken
 * directly from the charges; -1 for a bad level */
int orc_fmm_local_cell(orc_sys *s, int level, const int c[3], double *out);
/* one cell's Alg. L.3 expansion (real layout) by its definition, gathered
 * from the charges of its interaction list; needs no setup; -1 for a bad
 * level or cell */
int orc_local_cell_direct(orc_sys *s, int level, const int c[3], double *out);
/* the multipole method (Sec. 3.3, alternative algorithm): Alg. M.3 + K/E +
 * U0; afterwards propose/accept/run/energy follow Alg. M.1/M.2.  orc_setup
 * or orc_setup_fmm switch back to the local method. */
void orc_setup_multipole(orc_sys *s);
/* short-range Lennard-Jones term 4 eps((sig/r)^12 - (sig/r)^6), r < rc
 * (Sec. 5.3; call before a setup); rc <= finest cell width, else -1 */
int orc_set_lj(orc_sys *s, double eps, double sig, double rc);
/* level multipoles M_n^m (real layout), -1 for a bad level or before setup */
int orc_get_multipole(const orc_sys *s, int level, double *out);
double orc_propose(orc_sys *s, int64_t j, const double rnew[3]);  /* Alg. L.1 */
/* split of the last proposal: [0] expansions, [1] direct (Alg. 1 incl.
 * image correction), [2] far lattice, [3] dipole (tinfoil) term */
void orc_last_parts(const orc_sys *s, double parts[4]);
/* far-lattice change in the factored form Re(d^H H) + 1/2 d^H R d */
double orc_far_delta_factored(orc_sys *s, int64_t j, const double rnew[3]);
void orc_accept(orc_sys *s, int64_t j, const double rnew[3], double dE); /* Alg. L.2 */
double orc_energy(const orc_sys *s);              /* running total energy */
double orc_energy_fresh(orc_sys *s);              /* U from current state */
void orc_get_positions(const orc_sys *s, double *out);
/* local coefficients of level l (2..L) in the real layout: per cell, per n:
 * Re L_n^0, then (Re L_n^m, Im L_n^m) for m = 1..n */
int orc_get_local(const orc_sys *s, int level, double *out);
void orc_get_KH(orc_sys *s, double *K, double *H);  /* real layout, H = R(K) */
double orc_dipole_energy_coeff(const orc_sys *s);
/* interaction list of cell c (level coordinates) as (canonical linear index,
 * shift x, y, z) quadruples; returns the count */
int orc_interaction_list(const orc_sys *s, int level, const int c[3], int *out);

/* ---- Metropolis-Hastings driver with Philox4x32-10 proposals ---- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_proposal(int64_t n, double half_width, uint64_t seed, uint64_t step,
                  uint32_t chain, int64_t *j, double delta[3], double *u);
/* runs steps [step0, step0+n_steps); per-step logs may be NULL */
int64_t orc_run(orc_sys *s, int64_t n_steps, uint64_t seed, uint64_t step0,
                uint32_t chain, double beta, double half_width,
                int64_t *log_j, double *log_dE, uint8_t *log_acc,
                int64_t *n_borderline);
/* as orc_run, but step t is accepted iff follow[t] != 0 (log_acc keeps the
 * rule's own decision): replays the states of a chain whose decisions were
 * taken elsewhere */
int64_t orc_run_follow(orc_sys *s, int64_t n_steps, uint64_t seed, uint64_t step0,
                       uint32_t chain, double beta, double half_width, const uint8_t *follow,
                       int64_t *log_j, double *log_dE, uint8_t *log_acc,
                       int64_t *n_borderline);

/* ---- exact periodic Coulomb energy by Ewald summation (tinfoil) ---- */
double orc_ewald_energy(int64_t n, const double *pos, const double *q, double a,
                        double kappa, int nreal, int nrecip);
/* free-space direct pair energy */
double orc_direct_energy(int64_t n, const double *pos, const double *q);

#ifdef __cplusplus
}
#endif
#endif
