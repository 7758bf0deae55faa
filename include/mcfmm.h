/*
 * mcfmm: GB300 (sm_103a) library for the multilevel local-expansion
 * Metropolis-Hastings electrostatics method of Saunders, Grant & Mueller,
 * "A new algorithm for electrostatic interactions in Monte Carlo simulations
 * of charged particles" (arXiv 2006.16622).
 *
 * C ABI: plain pointers and sizes only.  Every call returns MC_OK (0) or a
 * negative MC_ERR_* status; mc_strerror() names it.  The library owns all
 * device memory of a context; inputs are copied, the caller keeps ownership
 * of its arrays.  Calls on one context are not thread safe.
 *
 * Conventions
 *   - the box is the cube [0, a)^3; positions are (n, 3) row-major doubles;
 *   - p is the expansion order (largest n of Eq. 2), 0 <= p <= 15; an
 *     expansion has (p+1)^2 real numbers in the "real layout": for each n,
 *     Re X_n^0 then (Re X_n^m, Im X_n^m) for m = 1..n (X_n^-m = conj X_n^m);
 *   - level l (1 = whole box) has 2^(l-1) cells per axis; cell (i, j, k) of a
 *     level has linear index (i * n_l + j) * n_l + k;
 *   - coefficients use the normalisation Y_n^m = sqrt((n-|m|)!/(n+|m|)!)
 *     P_n^|m|(cos t) e^{i m phi} (no Condon-Shortley phase);
 *   - energies are in units of q^2 / length (Gaussian units, unit charges).
 */
#ifndef MCFMM_H
#define MCFMM_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MC_OK 0
#define MC_ERR_ARG (-1)        /* invalid argument (null pointer, size, index) */
#define MC_ERR_NONNEUTRAL (-2) /* periodic boundaries need sum q = 0 */
#define MC_ERR_LEVELS (-4)     /* levels outside 2..8 */
#define MC_ERR_OUTSIDE (-5)    /* a position outside [0, a)^3 */
#define MC_ERR_CUDA (-6)       /* a CUDA runtime call failed */
#define MC_ERR_TIMEOUT (-7)    /* a device-side wait gave up (bounded spin) */
#define MC_ERR_CAPACITY (-8)   /* a finest cell overflowed its slot capacity */
#define MC_ERR_ORDER (-9)      /* expansion order p outside 0..15 */
#define MC_ERR_STATE (-10)     /* call out of order (e.g. propose before setup) */
#define MC_ERR_NOMEM (-11)     /* device allocation failed */
#define MC_ERR_SCRATCH (-12)   /* request larger than the fixed no-allocation scratch */
#define MC_ERR_PENDING (-13)   /* a CUDA error of earlier work was pending at the call */

#define MC_BC_PBC 0   /* periodic cube (paper Sec. 3.4) */
#define MC_BC_FREE 1  /* free space (paper Sec. 3.4, first paragraph) */
#define MC_TINFOIL 0  /* conducting surroundings: dipole term removed */
#define MC_VACUUM 1   /* cubic-shell (vacuum) summation of the images */
#define MC_FP64 0     /* every step in FP64 */
#define MC_FP32_EVAL 1 /* harmonics and near field in FP32; FP64 accumulators,
                          energy and periodic lattice term */
#define MC_SETUP_P2L 0 /* Alg. L.3 as a per-target gather */
#define MC_SETUP_FMM 1 /* FMM variant (Sec. 3.2, last paragraph): per-level
                          multipoles, then multipole-to-local over the
                          interaction lists; equal to MC_SETUP_P2L up to the
                          multipole truncation */
#define MC_SETUP_MULTIPOLE 2 /* the multipole method (Sec. 3.3, alternative
                          algorithm): Alg. M.3; the context then proposes and
                          accepts with Alg. M.1/M.2 (a later MC_SETUP_P2L or
                          MC_SETUP_FMM switches back to the local method) */

typedef struct mc_ctx mc_ctx;

typedef struct {
  int64_t steps;      /* proposals made by the last mc_run */
  int64_t accepted;   /* accepted proposals */
  int64_t borderline; /* decisions within 1e-9 (relative) of the threshold */
  int64_t resetups;   /* full re-setups done by the last mc_run */
  double energy;      /* running total energy after the run */
  double max_drift;   /* max |running - fresh| energy seen at a re-setup */
  double sum_drift;   /* sum of (running - fresh) over the re-setups */
  double sum_abs_drift; /* sum of |running - fresh| over the re-setups */
} mc_stats;

/* Create a context (paper Sec. 4, the MCFMM_LM constructor).
 *   n            number of charges (>= 1)
 *   pos, q       host arrays, (n, 3) positions in [0, box)^3 and n charges
 *   box          cube side a > 0
 *   levels       octree levels L, 2..8 (finest level has 8^(L-1) cells)
 *   p            expansion order 0..15
 *   bc           MC_BC_PBC or MC_BC_FREE; PBC needs sum q = 0 (|sum| < 1e-9)
 *   dipole_bc    MC_TINFOIL or MC_VACUUM (ignored for MC_BC_FREE)
 *   precision    MC_FP64 or MC_FP32_EVAL
 *   cuda_stream  cudaStream_t the context launches on, NULL = legacy stream
 * Allocates device memory; the expansions are undefined until mc_setup. */
int mc_init(mc_ctx **out, int64_t n, const double *pos, const double *q, double box,
            int levels, int p, int bc, int dipole_bc, int precision, void *cuda_stream);

/* Alg. L.3 (initialise local expansions), the box multipole K/E of
 * Sec. 3.4 (ii), the lattice local expansion H = R(K) and the total energy.
 * mode: MC_SETUP_P2L (exact P2L of every charge) or MC_SETUP_FMM (the
 * O(p^4 N) FMM variant; allocates its multipole and offset tables on first
 * use).  Synchronous. */
int mc_setup(mc_ctx *ctx, int mode);

/* Alg. L.1 with Alg. 1 and the periodic terms of Sec. 3.4: the energy change
 * of moving charge j (0 <= j < n) to r_new in [0, a)^3.  Writes +inf when
 * r_new coincides with another charge.  Synchronous. */
int mc_propose(mc_ctx *ctx, int64_t j, const double r_new[3], double *dE_out);

/* Alg. L.2 with the K/E update of Sec. 3.4 (iii): accept the move of j to
 * r_new.  dE_or_null: the energy change to add to the running energy; NULL
 * recomputes it with Alg. L.1 first (as the paper's accept() does). */
int mc_accept(mc_ctx *ctx, int64_t j, const double r_new[3], const double *dE_or_null);

/* Metropolis-Hastings chain of n_steps proposals in one persistent launch:
 * the user loop of Sec. 4.1 (propose(), then accept() when the move is
 * taken) run on the device, each proposal by Alg. L.1 and each accept by
 * Alg. L.2.  Proposal t (global step counter s, which continues across calls) draws
 * j, a displacement uniform in [-h, h]^3 and u uniform in [0, 1) from
 * Philox4x32-10 keyed by seed; the move is accepted iff dE <= 0 or
 * log(u) < -beta dE.  resetup_every_accepts > 0 re-runs mc_setup after that
 * many accepts and records the running-minus-fresh energy drift.
 * stats/log arrays may be NULL; when all are NULL and resetup is 0 the call
 * only enqueues the launch on the context stream and returns.  The log
 * arrays are host arrays of n_steps entries (moved charge, dE, accepted). */
int mc_run(mc_ctx *ctx, int64_t n_steps, uint64_t seed, double beta, double half_width,
           int64_t resetup_every_accepts, mc_stats *stats, int64_t *log_j, double *log_dE,
           uint8_t *log_acc);

/* The chain's global step counter s: proposals made so far by mc_run and
 * mc_batch_run (autotuning runs included) on this context; the next proposal
 * draws Philox counter s.  Lets a caller resume or re-draw the chain
 * elsewhere (Sec. 4.1 leaves the driver loop, and so its random stream, to
 * the user). */
int mc_step_counter(mc_ctx *ctx, int64_t *out);
/* Running total energy (setup energy plus accepted changes): the energy
 * the Sec. 4.1 interface tracks through the dE of each accept(). */
int mc_energy(mc_ctx *ctx, double *e_out);
/* Total energy recomputed from the current expansions and positions. */
int mc_energy_fresh(mc_ctx *ctx, double *e_out);
/* Current positions (n, 3) into a host array: the PositionDat r that
 * accept() updates in Sec. 4.1. */
int mc_get_positions(mc_ctx *ctx, double *pos_out);
/* Local coefficients L^Delta of level l (2..L), all cells, real layout,
 * paper normalisation; host array of 8^(l-1) * (p+1)^2 doubles. */
int mc_get_local(mc_ctx *ctx, int level, double *out);
/* Box multipole K and lattice local expansion H = R(K), real layout, paper
 * normalisation; host arrays of (p+1)^2 doubles (zeros for MC_BC_FREE). */
int mc_get_far(mc_ctx *ctx, double *K_out, double *H_out);
/* Short-range Lennard-Jones pair term 4 eps((sigma/r)^12 - (sigma/r)^6) for
 * r < cutoff between different particles (Sec. 5.3: the paper adds a
 * repulsive Lennard-Jones potential with a 12 Angstrom cutoff to its full
 * MC runs and gives no parameters); eps = 0 switches it off.  The cutoff may
 * not exceed the finest cell width (every pair in range is then a near-cell
 * pair of Alg. 1), else MC_ERR_ARG.  Call mc_setup again afterwards
 * (MC_ERR_STATE until then). */
int mc_set_lj(mc_ctx *ctx, double eps, double sigma, double cutoff);
/* Work split of the near-field sum (Alg. 1) in the chain kernels: each of
 * the 27 near cells is summed by `parts` items per side (2 parts items when
 * r and r' share their finest cell), each taking every parts-th block of 32
 * of the cell's charges.  parts = 0 restores the automatic choice made by
 * mc_init (one item per 48 charges of mean finest-cell occupancy, at most
 * 4); 1..4 forces it.  The result is the same sum in another order (dE
 * changes at rounding level only).  MC_ERR_ARG when parts is out of range or
 * the step's item slots (384) cannot hold 54 parts near items beside the
 * far-field and expansion items of this (p, L).  used_out (optional, host)
 * receives the split in force. */
int mc_set_near_parts(mc_ctx *ctx, int parts, int *used_out);
/* Multipoles M_n^m of Eq. (4) of every cell of `level` (multipole method
 * only, else MC_ERR_STATE), layout as mc_get_local. */
int mc_get_multipole(mc_ctx *ctx, int level, double *out);
/* Lattice sums S_l^m = sum over integer v with max|v_i| >= 2 of
 * Y_l^m(v/|v|)/|v|^(l+1), l <= lmax <= 30, as computed on the device;
 * complex interleaved, index 2*(l*l + l + m). */
int mc_lattice_sums(int lmax, double *out);
/* Schedule of mc_run / mc_batch_run chains.
 *   MC_SCHEDULE_PHASED     (default for FP32-eval contexts) propose items, grid barrier,
 *                          decision, accept items, grid barrier: two barriers
 *                          per accepted step.  The Alg. L.2 contributions of
 *                          the proposed move are computed during the
 *                          proposal phase, on the warps the proposal leaves
 *                          idle, and only added after the decision;
 *   MC_SCHEDULE_PIPELINED  withdrawn (slower than MC_SCHEDULE_PHASED in every
 *                          measurement on GB300); its value is refused with
 *                          MC_ERR_ARG;
 *   MC_SCHEDULE_PLAIN      (default for FP32-eval batches) as PHASED, with
 *                          the Alg. L.2 contributions computed after the
 *                          decision (no work on rejected moves);
 *   MC_SCHEDULE_ASYNC      (default for FP64 contexts) no barrier inside the
 *                          step loop: warps meet through per-step partial
 *                          slots and counters; the geometry of step k+1 is
 *                          published before the decision of step k (unless
 *                          both draw the same particle), so its speculative
 *                          Alg. L.2 contributions and far-field change run
 *                          while step k is decided and applied.  Same results
 *                          to roundoff.  mc_run chains of the local method
 *                          only; single proposals (mc_propose, mc_accept) and
 *                          the multipole method run phased. */
#define MC_SCHEDULE_PHASED 0
#define MC_SCHEDULE_PIPELINED 1
#define MC_SCHEDULE_PLAIN 2
#define MC_SCHEDULE_ASYNC 3
int mc_set_schedule(mc_ctx *ctx, int schedule);
/* CTAs of the persistent chain launches of ctx (mc_run, mc_propose,
 * mc_accept): 1 <= n_cta <= the multiprocessor count, one CTA per SM; 0
 * restores the default: every SM, except 5/7 of them for the phased chain of
 * an FP32-eval context (measured faster).  The work items of a step are dealt over
 * the warps of the grid and their partial results are combined in one fixed
 * order, so the results do not depend on n_cta.  MC_ERR_ARG outside that
 * range; takes effect at the next launch. */
int mc_set_ctas(mc_ctx *ctx, int n_cta);
/* Status of the last asynchronous launch (MC_OK, MC_ERR_TIMEOUT, ...). */
int mc_status(mc_ctx *ctx);
/* Wait-limit of the device-side grid barrier in nanoseconds (default 2e9);
 * a wait that runs out sets MC_ERR_TIMEOUT and the launch returns. */
int mc_set_wait_limit(mc_ctx *ctx, int64_t ns);
/* Failure-path testing (the paper has no counterpart): the grid barriers of
 * the following mc_run calls on ctx also wait for missing_arrivals CTAs that
 * never arrive, so the first wait runs out after the wait limit, the launch
 * ends with MC_ERR_TIMEOUT before any accepted move is applied, and the
 * context stays usable.  0 (the default) restores normal runs; 0..1024,
 * else MC_ERR_ARG. */
int mc_inject_wait_fault(mc_ctx *ctx, int missing_arrivals);
/* Diagnostics: with profiling on, mc_run accumulates MC_PROF_COUNTERS device
 * timers (globaltimer nanoseconds) of its persistent launch: [0..4] CTA 0's
 * own propose items, first barrier wait, decision, own accept items, second
 * barrier wait (MC_SCHEDULE_ASYNC: [0] publication of a step's geometry to
 * its decision, [1] publication to the start of the decision's poll);
 * [5] proposals, [6] accepts; [8+t], [24+t], [40+t] summed
 * duration, count and maximum of work items of type t (0 expansion
 * evaluation, 1 near cell, 2 far lattice block, 3 image/dipole term,
 * 4 small-level accept entry or apply, 5 accept target cell or apply,
 * 6 bookkeeping and K/H, 7 speculative small-level contribution,
 * 8 speculative large-level contribution; MC_SCHEDULE_ASYNC also, as times
 * from the publication of the item's step: 9 expansion item's state ready,
 * 10 expansion item done, 11 decision seen by an apply item, 12 its
 * operands loaded, 13 apply item done, 14 near item's state ready, 15 far /
 * near / image item done).  mc_profile_read copies them (out:
 * MC_PROF_COUNTERS uint64) and clears them. */
#define MC_PROF_COUNTERS 56
int mc_profile(mc_ctx *ctx, int on);
int mc_profile_read(mc_ctx *ctx, uint64_t *out);
void mc_destroy(mc_ctx *ctx);
const char *mc_strerror(int status);

/* ---- batched form: many independent chains in one persistent launch ----
 * The contexts (created and set up with mc_init/mc_setup on the same device
 * and with the same precision) keep ownership of their systems; a batch runs
 * their chains concurrently, each on its own group of CTAs with its own grid
 * barrier, in one cooperative launch replayed from a CUDA graph. */
typedef struct mc_batch mc_batch;
/* ctxs: n_chains context pointers (the batch does not own them; destroy the
 * batch before its contexts).  The initial CTA split gives every chain at
 * least one CTA, the rest in proportion to its number of levels. */
int mc_batch_create(mc_batch **out, int n_chains, mc_ctx *const *ctxs);
/* Autotuner: times short runs (trial_steps proposals per chain, which
 * advance the chains) at one and two CTAs per chain, fits each chain's time
 * per proposal t(g) = a + b/g, assigns the SMs greedily to minimise the
 * slowest chain's time, then picks the far-field tile count (column blocks
 * per row block, 1..16) with the shortest slowest-chain time. */
int mc_batch_tune(mc_batch *b, int64_t trial_steps, double beta, double half_width);
/* Runs n_steps proposals on every chain (seeds[i] keys chain i, Philox
 * counter word 2 = i; step counters continue across calls).  The launch is
 * captured once per (n_steps, beta, h, split, tiles) into a CUDA graph and
 * replayed.  stats: n_chains entries or NULL (NULL and no logs = enqueue
 * only).  Logs: host arrays of n_chains * n_steps entries or NULL (logged
 * runs are not graphed). */
int mc_batch_run(mc_batch *b, int64_t n_steps, const uint64_t *seeds, double beta,
                 double half_width, mc_stats *stats, int64_t *log_j, double *log_dE,
                 uint8_t *log_acc);
/* CTAs given to each chain (n_chains ints) and the far-field tile count. */
int mc_batch_info(mc_batch *b, int *ctas_out, int *nf_cols_out);
/* Schedule of the batch's chains (MC_SCHEDULE_*; default phased for FP64,
 * plain for FP32-eval batches). */
int mc_batch_set_schedule(mc_batch *b, int schedule);
void mc_batch_destroy(mc_batch *b);

/* Measured peak rate of the fused multiply-add pipe of the current device
 * (fp64 != 0: FP64, else FP32), in flop/s (2 per FMA): independent FMA
 * chains on every SM, timed with CUDA events, the loop grown until one
 * launch lasts about target_seconds (0 < target_seconds <= 10), best of three.
 * The denominator of the roofline of the ALU-bound chain kernels.  A
 * measurement helper; the paper has no counterpart.  Synchronous; allocates
 * and frees a small output buffer. */
int mc_probe_fma_rate(int fp64, double target_seconds, double *flops_out);

/* Size of the fixed device scratch of mc_p2l_level_noalloc, in doubles
 * (8 MiB), held by every GPU that loads the library until the process exits. */
#define MC_NOALLOC_SCRATCH_DOUBLES (1 << 20)

/* Local expansions of one level, computed without any allocation.
 *
 * The paper has no counterpart: this is a service for callers that cannot
 * let a library call cudaMalloc or cudaFree -- code that hands out every
 * byte of device memory from its own pool, code running where an allocation
 * would synchronise the device or is forbidden, embedders that audit hidden
 * allocations.  It computes the same coefficients as mc_setup + mc_get_local
 * give for one level, from buffers the caller owns:
 *   d_part        device, n rows of (x, y, z, q) doubles, grouped by finest
 *                 cell (levels L: 2^(L-1) cells per axis, cell of a point =
 *                 floor(x 2^(L-1) / box) clamped, linear index (i n + j) n + k);
 *   d_cell_start  device, 8^(L-1) + 1 ints: the charges of finest cell c are
 *                 rows [d_cell_start[c], d_cell_start[c+1]) of d_part;
 *   n             rows of d_part (>= 0); informational: only checked for
 *                 sign, the cell offsets alone decide which rows are read;
 *   box, levels, p, bc  as for mc_init; 2 <= level <= levels;
 *   d_out         device, 8^(level-1) * (p+1)^2 doubles, written in the real
 *                 layout and paper normalisation of mc_get_local;
 *   cuda_stream   stream to launch on (NULL = legacy stream); the call only
 *                 enqueues work and returns.
 * Intermediate sums live in one file-scope device array of
 * MC_NOALLOC_SCRATCH_DOUBLES doubles.  A level whose 8^(level-1) (p+1)^2
 * coefficients exceed it is refused with MC_ERR_SCRATCH before any launch.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the rest
 * of the process; make that first call before any stream capture, and make
 * no call after a cudaDeviceReset of that device (the kept address is then
 * stale).  Every call shares the one array: each call writes every scratch
 * value it reads before reading it, so nothing needs clearing, but calls
 * whose work overlaps on the GPU (other streams, other host threads) race on
 * it and must be serialised by the caller.  A CUDA error left pending by
 * earlier, unrelated work is neither cleared nor reported as this call's own:
 * the call then launches nothing and returns MC_ERR_PENDING. */
int mc_p2l_level_noalloc(const double *d_part, const int *d_cell_start, int64_t n, double box,
                         int levels, int level, int p, int bc, double *d_out, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
