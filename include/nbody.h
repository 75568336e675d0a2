/*
 * nbody.h -- C ABI of the GB300 direct-summation N-body library (libnbody.so).
 *
 * The library evaluates the Plummer-softened Newtonian acceleration
 *   a_i = G sum_{j != i} m_j d_ij / (|d_ij|^2 + eps^2)^(3/2),  d_ij = x_j - x_i
 * (paper eq. 1, Sec. 2, with the softening of Sec. 3) and its time
 * derivative, the jerk
 *   j_i = G sum_{j != i} m_j [ w_ij / s^3 - 3 (d_ij . w_ij) d_ij / s^5 ],
 *   w_ij = v_j - v_i, s^2 = |d_ij|^2 + eps^2
 * for a list of active i-particles against all j-particles, on one GPU, and
 * advances the system with the 4th-order Hermite predictor-corrector and
 * power-of-two block time steps (the paper's individual per-particle time
 * steps, Sec. 2, strategy (ii); the Hermite scheme itself is Makino &
 * Aarseth 1992 and is not printed in the paper), or with the paper's own
 * fixed-step symplectic integrators (Sec. 2.2: the leapfrog and a
 * sixth-order composition) and, optionally, its external Galactic field
 * (Sec. 2.1).
 *
 * Conventions (every entry point):
 *  - Every call returns nb_status; NB_OK is 0.  On error a message is kept
 *    per host thread and returned by nb_last_error().  No C++ exception
 *    crosses this interface.
 *  - Host pointers are owned by the caller and are only read or written
 *    during the call.  Device pointers (the *_dev entry points) are owned by
 *    the caller; the library never frees memory it did not allocate.
 *  - Vectors are (n, 3) row-major float64 arrays: x[3*i + c].
 *  - Time is kept as integer ticks of 2^-20; time arguments given as double
 *    must be exact multiples of 2^-20.
 *  - Work is queued on the stream given in nb_config.stream (NULL = the
 *    legacy default stream).  Calls that return host data synchronise that
 *    stream (with a host watchdog, see nb_config.sync_timeout_ms).
 *  - A context is not thread-safe: one host thread at a time.
 */
#ifndef NBODY_GB300_H
#define NBODY_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nb_ctx nb_ctx; /* opaque, library-owned */

typedef enum {
  NB_OK = 0,
  NB_ERR_INVALID_ARG = 1, /* bad size, NULL pointer, non-finite input, bad time */
  NB_ERR_STATE = 2,       /* call out of order (e.g. correct before force) */
  NB_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed */
  NB_ERR_OOM = 4,         /* device allocation failed (or the test cap hit) */
  NB_ERR_NUMERIC = 5,     /* a result was not finite */
  NB_ERR_TIMEOUT = 6,     /* the host watchdog gave up waiting for the GPU */
  NB_ERR_DEVICE = 7       /* a kernel's bounded wait ran out; see message */
} nb_status;

typedef enum { NB_FP32 = 0, NB_DS = 1 } nb_precision;

/* Integration and arithmetic settings.  Fill with nb_default_config(). */
typedef struct {
  double G;          /* gravitational constant (paper: G = 1, Sec. 3) */
  double eps;        /* Plummer softening length, >= 0 (paper Sec. 3).  With
                        eps == 0 the kernels mask the i == j term. */
  double eta;        /* Aarseth accuracy parameter for block steps */
  double eta_start;  /* initial step: dt0 = eta_start |a| / |j| */
  int32_t lev_min;   /* largest step 2^-lev_min; 0 <= lev_min <= lev_max */
  int32_t lev_max;   /* smallest step 2^-lev_max; lev_max <= 20 */
  int32_t precision; /* nb_precision: pair arithmetic and accumulation */
  int32_t block_steps; /* 1: Aarseth block steps; 0: shared dt = 2^-lev_shared */
  int32_t lev_shared;  /* shared step level when block_steps == 0 */
  int32_t sync_timeout_ms; /* host watchdog per synchronisation; <= 0: 600 s */
  void *stream;      /* cudaStream_t to queue work on; NULL = default stream */
} nb_config;

/* Defaults: G = 1, eps = 1e-3, eta = 0.01, eta_start = 0.01, lev 3..20,
 * NB_DS, block steps on, lev_shared = 8, watchdog 600 s, default stream. */
void nb_default_config(nb_config *cfg);

/* Create a context holding n particles (1 <= n <= 2^30).  m (n), x and v
 * ((n,3)) are host arrays copied to the device.  Evaluates a and j at t = 0
 * for every particle and sets the initial step levels (block steps:
 * dt0 = eta_start |a|/|j| quantised down to a power of two; shared: lev_shared).
 * Errors: NB_ERR_INVALID_ARG (n out of range, NULL, non-finite, bad config),
 * NB_ERR_OOM, NB_ERR_CUDA.  On error *out is set to NULL. */
nb_status nb_init(nb_ctx **out, int64_t n, const double *m, const double *x,
                  const double *v, const nb_config *cfg);

/* Release every device and host resource of the context.  NULL is a no-op. */
void nb_destroy(nb_ctx *ctx);

/* Block scheduling (paper Sec. 2, individual time steps): t_next =
 * min_i (t_i + dt_i); the active list becomes every i with t_i + dt_i ==
 * t_next, in ascending index order (deterministic).  Returns t_next (time
 * units) and the number of active particles; synchronises the stream. */
nb_status nb_next_block(nb_ctx *ctx, double *t_next, int64_t *n_active);

/* Predict every particle to time t (Hermite predictor, FP64):
 *   x_p = x + v dt + a dt^2/2 + j dt^3/6, v_p = v + a dt + j dt^2/2,
 *   dt = t - t_i, and write the j-records the force kernels read (FP32 or
 * double-single split positions).  Asynchronous.  t must be a tick multiple
 * and not earlier than any t_i (NB_ERR_INVALID_ARG). */
nb_status nb_predict(nb_ctx *ctx, double t);

/* Acceleration and jerk (eq. 1 and its time derivative) on the particles
 * idx[0..n_idx) from all n particles at the last predicted state.
 * idx == NULL: the current active list (n_idx must equal its length, or be
 * negative to take it); the result is then also kept for nb_correct.
 * acc/jerk: host (n_idx,3) outputs, either may be NULL.  Synchronises.
 * Errors: NB_ERR_INVALID_ARG (index out of range, n_idx mismatch),
 * NB_ERR_STATE (no prediction yet), NB_ERR_NUMERIC (non-finite result). */
nb_status nb_force_jerk(nb_ctx *ctx, const int32_t *idx, int64_t n_idx,
                        double *acc, double *jerk);

/* Same on device pointers, asynchronous on the context stream: d_idx
 * (int32, n_idx entries, each in [0, n); NULL = the active list as above),
 * d_acc / d_jerk (float64, (n_idx,3); may be NULL when idx == NULL, in
 * which case the result is kept only for nb_correct).  Indices are not
 * range-checked on the device: an out-of-range index is undefined behaviour. */
nb_status nb_force_jerk_dev(nb_ctx *ctx, const int32_t *d_idx, int64_t n_idx,
                            double *d_acc, double *d_jerk);

/* Hermite corrector (Makino & Aarseth 1992) for the active list at time t
 * (must equal the t_next of the current block and follow a force
 * evaluation of the active list at that time), then the Aarseth step
 * criterion and its power-of-two quantisation (block steps: shrink freely,
 * grow by one level only on a multiple of the doubled step).  Asynchronous. */
nb_status nb_correct(nb_ctx *ctx, double t);

/* One full block step: nb_next_block, nb_predict, nb_force_jerk_dev on the
 * active list, nb_correct.  Returns t_next and the active count. */
nb_status nb_step(nb_ctx *ctx, double *t_next, int64_t *n_active);

/* Block steps without a host round trip per step: the active count, the
 * force shape and the stream-K split are taken on the device, and a CUDA
 * graph of 32 block steps (scheduling, predictor, force + jerk, corrector)
 * is replayed until the next block would pass t_end or max_blocks steps
 * (0 = no limit) have run; the host synchronises once per replay.  The
 * steps are the ones nb_step takes with the built-in force shapes (an
 * installed tuning table or a forced variant is not used here), so the
 * results are bit-identical to an nb_step loop under the built-in choice.
 *
 * Two forms of the same steps.  When every particle's next time is the
 * first multiple of its step 2^-lev after the latest particle time (always
 * true of states this library integrates from nb_init; block scheduling of
 * the paper's Sec. 2, strategy (ii)), a fused form runs: the next block
 * time comes from per-level particle counts kept on the device and the
 * active list from the levels alone, so a step is three kinds of kernel
 * (scheduling + predictor, force, fix-up + corrector).  Otherwise (a state
 * set with nb_set_state that lacks the property) the general scheduler
 * runs (minimum of t_i + dt_i over all particles).  A check kernel decides
 * at the start of each call.  NB_ERR_DEVICE if a bounded device-side wait
 * ran out.
 * Returns the number of block steps taken and the time of the last one.
 * t_end must be a tick multiple; particles due later stay where they are. */
nb_status nb_run_blocks(nb_ctx *ctx, double t_end, int64_t max_blocks,
                        int64_t *blocks_done, double *t_last);

/* Block-step form of nb_run_blocks: NB_BLOCKS_AUTO (default: fused when
 * the schedule allows it) or NB_BLOCKS_GENERAL (always the general
 * scheduler; for comparison).  No counterpart in the paper.
 * NB_ERR_INVALID_ARG for another value. */
enum { NB_BLOCKS_AUTO = 0, NB_BLOCKS_GENERAL = 1 };
nb_status nb_set_block_mode(nb_ctx *ctx, int32_t mode);

/* *fused = 1 if the last nb_run_blocks call ran the fused form, else 0. */
nb_status nb_last_block_path(nb_ctx *ctx, int32_t *fused);

/* Fixed-step symplectic integration of every particle (paper Sec. 2.2):
 * nsteps steps of length dt (any finite value; a negative dt integrates
 * backwards) of the scheme of the given order, on the context's FP64
 * state with forces in its precision (FP32 or split precision, softening
 * eps, no jerk; the built-in force shapes, not a forced variant or an
 * installed tuning table).
 *   order 2: kick-drift-kick leapfrog, one force evaluation per step;
 *   order 6: the symmetric composition of seven leapfrog steps of lengths
 *            w_k dt with the sixth-order weights of Kinoshita, Yoshida &
 *            Nakai (1991), Table 1, first column (Yoshida's 1990 solution
 *            A: w1 = -1.17767998417887, w2 = 0.235573213359358,
 *            w3 = 0.784513610477557, w0 = 1 - 2 (w1 + w2 + w3), stages
 *            w3 w2 w1 w0 w1 w2 w3), seven force evaluations per step.
 * The call first evaluates the acceleration at the current positions (so
 * nsteps = 0 only refreshes it); the kicks between two drifts of a step
 * are merged, and each step ends with its closing half kick, so x and v
 * are synchronous after every step.  One step is captured as a CUDA graph
 * (cached for the last order and dt) and replayed.  On return x, v hold
 * the new state and a the acceleration at x (nb_get_state); t_tick, lev
 * and jerk are not advanced, so Hermite calls (nb_next_block, nb_predict,
 * nb_step, nb_run_blocks) answer NB_ERR_STATE until nb_set_state gives a
 * Hermite state.  Synchronises.  NB_ERR_INVALID_ARG: order not 2 or 6,
 * non-finite dt, nsteps < 0.  In split precision, particles in a spatial
 * order let the force kernel take its tile-relative far field for distant
 * tiles (10 % faster at N = 65,536 and 26 % at 262,144 on a uniform sphere
 * than in a random order); see nb_set_symplectic_layout. */
nb_status nb_symplectic(nb_ctx *ctx, int32_t order, double dt, int64_t nsteps);

/* Particle layout of nb_symplectic runs.  NB_LAYOUT_SPATIAL: each run with
 * nsteps > 0 orders the particles by a balanced bisection of their current
 * positions (nb_spatial_order with 256-particle leaves, on the host cores),
 * gathers x, v, m into that order on the device, steps them there and
 * scatters x, v, a back, so the caller sees its own order; the force sums
 * then run in another order, which changes results only by rounding.
 * NB_LAYOUT_AS_GIVEN: the particles' own order.  NB_LAYOUT_AUTO (default):
 * spatial in split precision for N >= 131,072 when the run's estimated
 * force time is large against the ordering's cost, else as given.
 * NB_ERR_INVALID_ARG for another value. */
enum { NB_LAYOUT_AUTO = 0, NB_LAYOUT_AS_GIVEN = 1, NB_LAYOUT_SPATIAL = 2 };
nb_status nb_set_symplectic_layout(nb_ctx *ctx, int32_t mode);

/* *spatial = 1 if the last nb_symplectic call ran in the spatial layout. */
nb_status nb_last_symplectic_layout(nb_ctx *ctx, int32_t *spatial);

/* External Galactic field (paper Sec. 2.1: the pair forces are summed with
 * the field of Allen & Santillan 1991, a spherical bulge and halo and an
 * axisymmetric disk).  With d = x - center, r = |d|, R^2 = d_x^2 + d_y^2,
 * z = d_z:
 *   bulge (Plummer)        Phi = -G m_bulge / sqrt(r^2 + b_bulge^2)
 *   disk (Miyamoto-Nagai)  Phi = -G m_disk / sqrt(R^2 + (a_disk
 *                                + sqrt(z^2 + b_disk^2))^2)
 *   halo                   enclosed mass M(r) = m_halo q^g / (1 + q^(g-1)),
 *                          q = r / a_halo, g = gamma_halo, constant beyond
 *                          r_cut; force -G M(r) d / r^3; potential
 *                          -G M(r)/r - G m_halo / ((g-1) a_halo)
 *                          [F(q_cut) - F(q)], F(q) = ln(1 + q^(g-1))
 *                          - (g-1) / (1 + q^(g-1)), inside the cut and
 *                          -G M(r_cut) / r beyond.
 * All parameters are in the context's units (G is the field's own
 * gravitational constant). */
typedef struct nb_external {
  double G;
  double center[3];
  double m_bulge, b_bulge;
  double m_disk, a_disk, b_disk;
  double m_halo, a_halo, gamma_halo, r_cut;
} nb_external;

/* Fill e with Allen & Santillan's (1991) parameters in their units (length
 * 1 kpc, mass 2.32e7 solar masses, velocity 10 km/s, G = 1): m_bulge = 606,
 * b_bulge = 0.3873, m_disk = 3690, a_disk = 5.3178, b_disk = 0.25,
 * m_halo = 4615, a_halo = 12, gamma_halo = 2.02, r_cut = 100, centre at
 * the origin.  The model's circular speed at 8.5 kpc is 220 km/s. */
void nb_external_allen_santillan(nb_external *e);

/* Set (e non-NULL, copied) or remove (NULL) the context's external field.
 * While set, everything is FP64 at each particle's own position:
 *  - nb_symplectic adds the field's acceleration to the pair sum in every
 *    kick and leaves the total in a;
 *  - the Hermite corrector (nb_correct, nb_step, nb_run_blocks) adds the
 *    field's acceleration and jerk (the time derivative of the
 *    acceleration along the velocity) at each active particle's predicted
 *    position and velocity to its pair sums, so a and jerk in the state
 *    are totals and the predictor and step criterion use them;
 *  - nb_energy adds sum_i m_i Phi(x_i) to the potential energy.
 * The call itself moves the field into (or the previous one out of) every
 * particle's stored a and jerk at its own stored x, v; on a context where
 * no step has been taken since nb_init it also recomputes the initial
 * levels from the totals.  With a field set, a and jerk given to
 * nb_set_state must include it (as nb_get_state returns them).
 * Synchronises.  NB_ERR_INVALID_ARG: a non-finite parameter, a negative G,
 * mass or a_disk, b_bulge, b_disk, a_halo or r_cut not positive, or
 * gamma_halo <= 1. */
nb_status nb_set_external(nb_ctx *ctx, const nb_external *e);

/* Energy of the current (synchronised) state in FP64 on the GPU:
 * K = 1/2 sum m v^2, W = -G sum_{i<j} m_i m_j / sqrt(r_ij^2 + eps^2)
 * (the softened pair potential consistent with the force), plus
 * sum_i m_i Phi_ext(x_i) when an external field is set.  Uses the
 * particles' own stored x, v (not predicted).  Synchronises. */
nb_status nb_energy(nb_ctx *ctx, double *kin, double *pot, double *tot);

/* Copy the integrator state to host arrays (any may be NULL):
 * x, v, a, jerk (n,3); t_tick (n) int64 ticks of 2^-20; lev (n) int32.
 * Synchronises.  Together with nb_set_state this is checkpoint/resume:
 * a run continued from a copied state is bitwise identical. */
nb_status nb_get_state(nb_ctx *ctx, double *x, double *v, double *a,
                       double *jerk, int64_t *t_tick, int32_t *lev);

/* Overwrite the state (all six arrays required; masses are kept).
 * Validates finiteness, 0 <= lev <= 20 and t_tick a multiple of 2^(20-lev).
 * The next call must be nb_next_block or nb_predict. */
nb_status nb_set_state(nb_ctx *ctx, const double *x, const double *v,
                       const double *a, const double *jerk,
                       const int64_t *t_tick, const int32_t *lev);

/* Copy the current active list (int32 indices) into idx, which holds cap
 * entries; *n_active receives its length.  The list is in storage order:
 * ascending indices until nb_relayout re-stores the particles, afterwards
 * ascending storage slots given as the caller's indices (the order of the
 * rows of nb_force_jerk's result for idx == NULL).  Synchronises. */
nb_status nb_get_active(nb_ctx *ctx, int32_t *idx, int64_t cap,
                        int64_t *n_active);

/* Storage order (no counterpart in the paper; it keeps the force kernel's
 * tile-relative far field, a layout optimisation, effective over a long
 * run).  The split-precision force kernel walks a 256-record tile with
 * plain FP32 differences when the tile is far from the i-block (box
 * distance at least the tile's radius), which needs tiles and i-blocks
 * compact in space: particles given in nb_spatial_order are, but as they
 * move the tiles spread and more of them take the slower split path (a
 * King W0 = 7 cluster of 2^20 particles: 97 % of tile pairs far at t = 0,
 * about 78 % at t = 0.1 and 15 % at t = 0.5).
 * nb_relayout re-stores every per-particle array of the context in a
 * balanced-bisection order of the current positions (256-particle leaves,
 * computed on the host cores, as nb_spatial_order): the caller's view does
 * not change.  nb_get_state, nb_set_state and the index lists of
 * nb_force_jerk / nb_force_jerk_dev keep the caller's (nb_init) order,
 * nb_get_active returns the caller's indices; what changes is the order of
 * the force sums (results differ by rounding only) and the order of the
 * active list.  The j-records and the active list of the old order are
 * dropped: the next call must be nb_next_block, nb_run_blocks or
 * nb_symplectic.  Synchronises; costs a copy of the positions to the host,
 * the bisection on the host cores and a gather of the state on the device
 * (about 30 ms for 2^20 particles with 16 host cores).  NB_ERR_STATE on a shard (nb_shard_set with nranks > 1),
 * NB_ERR_NUMERIC for a non-finite position. */
nb_status nb_relayout(nb_ctx *ctx);

/* Automatic relayout: nb_next_block and nb_run_blocks re-store the
 * particles first when at least block_steps block steps have been taken
 * since the last relayout (nb_run_blocks checks at the start of each call
 * only).  0 (the default) turns it off; NB_ERR_INVALID_ARG if negative. */
nb_status nb_set_relayout_every(nb_ctx *ctx, int64_t block_steps);

/* perm (n entries, may be NULL): perm[s] is the caller's index of the
 * particle stored in slot s (the identity before the first relayout);
 * *relayouts (may be NULL): relayouts so far. */
nb_status nb_get_storage_order(nb_ctx *ctx, int32_t *perm, int64_t *relayouts);

/* Counters: block steps taken, interactions evaluated (n_act * n summed
 * over force evaluations), and particles whose step criterion fell below
 * 2^-lev_max and were clamped.  Synchronises. */
nb_status nb_get_counters(nb_ctx *ctx, int64_t *n_blocks,
                          int64_t *n_interactions, int64_t *n_clamped);

/* Wait for all queued work (host watchdog) and report device-side errors. */
nb_status nb_sync(nb_ctx *ctx);

/* Number of kernel launches the library has queued on this context. */
int64_t nb_launch_count(const nb_ctx *ctx);

/* Force-kernel shape for the next force evaluations (autotuning):
 * variant indexes the compiled shape table (see nb_variant_info); -1
 * restores the built-in choice by active-list length.  grid_ctas > 0 caps
 * the persistent grid.  Errors: NB_ERR_INVALID_ARG for an unknown variant or
 * one whose precision differs from the context's. */
nb_status nb_set_force_variant(nb_ctx *ctx, int32_t variant, int32_t grid_ctas);

/* Data layout helper (host only): a permutation that lists the n particles
 * (x: (n,3) host array) leaf by leaf of a balanced bisection tree whose
 * leaves hold `leaf` particles (256 matches the force kernels' tiles):
 * perm[k] is the particle to store at position k.  Storing particles in
 * this order makes the kernels' 256-record tiles and i-blocks spatially
 * compact, which lets the split-precision kernel take its tile-relative
 * far-field path for most tiles; it changes no result beyond rounding
 * order.  Deterministic (ties broken by index). */
nb_status nb_spatial_order(int64_t n, const double *x, int64_t leaf,
                           int64_t *perm);

/* Install a tuning table for the built-in variant choice: for an active
 * list of n_i particles the first entry k (in order) with n_i >= min_n[k]
 * gives the variant and, when grid_ctas is non-NULL and grid_ctas[k] > 0,
 * a cap on its persistent grid (fewer CTAs split each i-block's j-range
 * into fewer stream-K segments); lists shorter than every min_n fall back
 * to the built-in choice.  count == 0 removes the table.  Variants must
 * match the context's precision and eps masking (NB_ERR_INVALID_ARG), grid
 * caps must be >= 0; at most 32 entries.  An explicit nb_set_force_variant
 * still takes precedence. */
nb_status nb_set_force_table(nb_ctx *ctx, int32_t count, const int64_t *min_n,
                             const int32_t *variant, const int32_t *grid_ctas);

/* Describe compiled force-kernel variant v: precision, i-particles per
 * thread, threads per i-particle, threads per CTA, and whether it packs two
 * i-particles into each FP32x2 instruction (results are bit-identical to
 * the unpacked variant of the same shape).  Any output may be NULL.
 * NB_ERR_INVALID_ARG past the end of the table. */
nb_status nb_variant_info(int32_t v, int32_t *precision, int32_t *ipt,
                          int32_t *tpi, int32_t *threads, int32_t *packed);

/* Fault injection for tests: kind 1 makes the next device allocation of
 * nb_init fail with NB_ERR_OOM (process-wide, one shot); kind 2 makes the
 * next synchronisation of ctx report NB_ERR_TIMEOUT (ctx required); kind 3
 * makes every bounded wait of the fused block steps' look-back (the
 * ordered compaction of the active list in nb_run_blocks) wait a few polls
 * for a word that no CTA publishes, so each runs out and nb_run_blocks
 * returns NB_ERR_DEVICE (ctx required; in force until kind 0); kind 0
 * clears the context's injections.  No GPU fault is ever caused.
 *
 * Device-side errors (NB_ERR_DEVICE) are reported once: the device error
 * word is cleared when it is read.  The particle state after the failed
 * call is unspecified; nb_set_state restores a saved one. */
nb_status nb_debug_inject(nb_ctx *ctx, int32_t kind);

/* ------------------------------------------------------------------------
 * Batched form: many independent clusters, shared step dt = 2^-lev_shared,
 * advanced by one persistent kernel per S steps (a CUDA graph of those
 * launches is captured once and replayed).  Same force law, jerk and
 * Hermite-4 corrector as above; cluster c holds particles
 * [offsets[c], offsets[c+1]) of the concatenated arrays and interacts only
 * with itself.  Cluster sizes 1..4096.
 * ---------------------------------------------------------------------- */
typedef struct nb_batch nb_batch; /* opaque, library-owned */

/* Copy the clusters to the device and evaluate a, j at t = 0.  cfg must have
 * block_steps == 0; cfg->lev_shared sets dt; cfg->precision and cfg->eps as
 * for nb_init.  Errors: NB_ERR_INVALID_ARG, NB_ERR_OOM, NB_ERR_CUDA. */
nb_status nb_batched_init(nb_batch **out, int32_t n_clusters,
                          const int64_t *offsets, const double *m,
                          const double *x, const double *v,
                          const nb_config *cfg);
void nb_batched_destroy(nb_batch *b);

/* Advance every cluster nsteps shared steps: ceil(nsteps / S) persistent
 * launches (S = steps per launch, see nb_batched_set_tuning), each a queue
 * of all clusters largest first; captured once into a CUDA graph per
 * (nsteps, tuning) and replayed.  Asynchronous. */
nb_status nb_batched_run(nb_batch *b, int64_t nsteps);

/* The same steps with one single-CTA launch per cluster per S steps (the
 * per-cluster-launch baseline).  Results are bitwise equal to
 * nb_batched_run's.  Asynchronous. */
nb_status nb_batched_run_per_cluster(nb_batch *b, int64_t nsteps);

/* Kernel shape (variant of nb_batched_variant_info, -1 = built-in), steps
 * per launch S >= 1, persistent grid cap (0 = #SMs x resident CTAs) and
 * graph use (0 = plain launches).  Used by the autotuner. */
nb_status nb_batched_set_tuning(nb_batch *b, int32_t variant,
                                int32_t steps_per_launch, int32_t grid_ctas,
                                int32_t use_graph);
/* Shape of batched variant v: precision, i-particles per thread, threads
 * per CTA, and 1 if two i-particles share each packed FP32x2 instruction.
 * Any output may be NULL; NB_ERR_INVALID_ARG past the last variant. */
nb_status nb_batched_variant_info(int32_t v, int32_t *precision, int32_t *ipt,
                                  int32_t *threads, int32_t *packed);

/* Per-cluster FP64 kinetic and softened potential energy into host arrays
 * of n_clusters entries (either may be NULL).  Synchronises. */
nb_status nb_batched_energy(nb_batch *b, double *kin, double *pot);

/* Copy the concatenated state to host (N,3) arrays (any may be NULL). */
nb_status nb_batched_get_state(nb_batch *b, double *x, double *v, double *a,
                               double *jerk);
nb_status nb_batched_sync(nb_batch *b);
int64_t nb_batched_launch_count(const nb_batch *b);

/* ------------------------------------------------------------------------
 * Differentiable leapfrog (paper Sec. 3.1, the classic second-order
 * symplectic scheme, kick-drift-kick form) in FP32, with the adjoint of the
 * force sum.  All pointers are caller-owned device arrays (float32):
 * x, v (n,3) row-major, m (n).  Work is queued on `stream` (NULL = default
 * stream); nothing is allocated.  Errors: NB_ERR_INVALID_ARG for n outside
 * [1, 2^30], eps < 0, G <= 0, a NULL pointer or a bad step count;
 * NB_ERR_CUDA for a failed launch.
 * ---------------------------------------------------------------------- */

/* acc = a(x): G sum_{j != i} m_j d / (|d|^2 + eps^2)^(3/2) (eq. 1,
 * softened).  acc is (n,3). */
nb_status nb_lf_acc(int64_t n, const float *d_x, const float *d_m, float eps,
                    float G, float *d_acc, void *stream);

/* Vector-Jacobian product of the acceleration map for a cotangent g
 * ((n,3), g_i = dL/da_i): gx_k = G sum_{j != k} T(x_j - x_k)(m_k g_j -
 * m_j g_k) with T(d) = I/s^3 - 3 d d^T/s^5, and gm_k = G sum_{i != k}
 * g_i . (x_k - x_i)/s^3.  gx (n,3) and gm (n) are overwritten. */
nb_status nb_lf_acc_vjp(int64_t n, const float *d_x, const float *d_m,
                        const float *d_g, float eps, float G, float *d_gx,
                        float *d_gm, void *stream);

/* Floats of the checkpoint buffer (ceil(nsteps/ckpt_every) slots of (x, v))
 * and of the reverse pass's work buffer; -1 for bad arguments. */
int64_t nb_lf_ckpt_floats(int64_t n, int64_t nsteps, int32_t ckpt_every);
int64_t nb_lf_work_floats(int64_t n, int32_t ckpt_every);

/* nsteps KDK steps of dt in place on d_x, d_v (d_acc (n,3) receives the
 * final acceleration).  If d_ckpt is not NULL, (x, v) at every step that is
 * a multiple of ckpt_every is stored in it (nb_lf_ckpt_floats floats). */
nb_status nb_lf_forward(int64_t n, const float *d_m, float *d_x, float *d_v,
                        float *d_acc, int64_t nsteps, float dt, float eps,
                        float G, int32_t ckpt_every, float *d_ckpt,
                        void *stream);

/* Reverse pass of nb_lf_forward from its checkpoints: on entry d_lx, d_lv
 * hold dL/dx(T), dL/dv(T); on exit dL/dx(0), dL/dv(0), and d_lm (n) holds
 * dL/dm.  Each segment of ckpt_every steps is re-run from its checkpoint
 * into d_work (nb_lf_work_floats floats) and walked backwards. */
nb_status nb_lf_backward(int64_t n, const float *d_m, const float *d_ckpt,
                         int64_t nsteps, float dt, float eps, float G,
                         int32_t ckpt_every, float *d_lx, float *d_lv,
                         float *d_lm, float *d_work, void *stream);

/* ------------------------------------------------------------------------
 * i-split shards (the paper's two-GPU version of its code, Sec. 4, splits
 * the particles whose forces are computed among the GPUs; every GPU keeps
 * all particles as sources).  A context becomes shard `rank` of `nranks`
 * (<= 64): it owns particles [bounds[rank], bounds[rank+1]) of a contiguous
 * partition (bounds[0] = 0 <= ... <= bounds[nranks] = n, nranks + 1 host
 * entries), keeps the whole state, and in the host-driven block step
 *   nb_next_block  finds the whole active list and every rank's slice of
 *                  it (ascending indices, so the slices are consecutive);
 *   nb_predict     predicts every particle;
 *   nb_force_jerk[_dev] (index list NULL) evaluates the own slice only
 *                  (outputs, when given, hold the slice's rows);
 *   nb_correct     corrects the own slice only;
 *   nb_shard_export writes the slice's corrected records (count through
 *                  *count) to d_rec, device memory of NB_SHARD_RECORD_DOUBLES
 *                  doubles each: x, v, a, jerk (3 each), then the bit
 *                  patterns of t_tick (int64) and lev (as an int64);
 *   (the caller concatenates all ranks' records in rank order, e.g. by an
 *    all-gather, or by letting every shard export at its slice's offset of
 *    one buffer when all shards live on one device)
 *   nb_shard_import takes that concatenation (n_rec = the block's active
 *                  count, list order) and stores the other ranks' records.
 * After the import every shard holds the same state.  nranks == 1 undoes
 * the sharding.  Call between block steps (NB_ERR_STATE otherwise); shards
 * run host-driven steps only (nb_run_blocks and nb_symplectic return
 * NB_ERR_STATE), and nb_next_block returns NB_ERR_STATE until the last
 * block's import is done; a context re-stored by nb_relayout cannot
 * become a shard (NB_ERR_STATE).  nb_shard_offsets gives the nranks + 1 slice
 * offsets of the block last found by nb_next_block (host array; for an
 * unsharded context 0 and the active count). */
#define NB_SHARD_RECORD_DOUBLES 14
nb_status nb_shard_set(nb_ctx *ctx, int32_t nranks, int32_t rank, const int64_t *bounds);
nb_status nb_shard_offsets(nb_ctx *ctx, int64_t *offsets);
nb_status nb_shard_export(nb_ctx *ctx, double *d_rec, int64_t *count);
nb_status nb_shard_import(nb_ctx *ctx, const double *d_rec, int64_t n_rec);

/* ------------------------------------------------------------------------
 * Allocation-free force + jerk.  The paper has no counterpart: this entry
 * point exists for callers that cannot let the library allocate device
 * memory -- programs whose device memory all belongs to another allocator
 * (a framework's caching allocator, a pool sized once at start-up), code
 * that must not risk the device-wide synchronisation cudaMalloc/cudaFree can
 * cause, and hosts that forbid allocation after initialisation.  It needs
 * no context and calls no cudaMalloc, cudaFree or allocating library
 * routine.
 *
 * Computes, on the caller's stream, the softened acceleration
 * a_i = G sum_j m_j d / (|d|^2 + eps^2)^(3/2), d = x_j - x_i, and its time
 * derivative (the jerk) on the particles d_idx[0..n_idx) (NULL:
 * 0..n_idx-1, n_idx <= n; an index list may repeat indices and be longer
 * than n) from all n particles.  When eps^2 is not a normal FP32 number
 * (eps == 0 included) the i == j term is zeroed explicitly.
 * Inputs: d_m (n), d_x and d_v ((n,3) row-major), all float64 device
 * arrays; outputs d_acc and d_jerk, float64 (n_idx,3), device.  precision:
 * NB_FP32 or NB_DS.  Indices must lie in [0, n) (not checked on the device).
 *
 * Scratch: the partial sums of i-blocks split across CTAs live in one
 * static device array of 2^20 doubles (8 MiB) that every GPU loading the
 * library holds until the process exits; a launch uses at most 341 CTAs so
 * that they fit, whatever n and n_idx are.  Every call shares that array
 * and it keeps the last call's contents; each call writes every partial it
 * later reads, so nothing needs clearing, but calls whose work overlaps on
 * the GPU (other streams, or other host threads on the same device) race on
 * it and must be serialised by the caller.
 *
 * The first call on each device resolves the array's device address
 * (cudaGetSymbolAddress, with that device current) and the kernel's
 * occupancy; make that first call before any stream capture begins.
 * Errors: NB_ERR_INVALID_ARG for n outside [1, 2^31-1], n_idx outside
 * [0, 2^31-1] (or above n without an index list), a NULL pointer, eps < 0,
 * G <= 0 or an unknown precision; NB_ERR_CUDA for a failed launch or set-up,
 * and, without launching anything, when a CUDA error from earlier work is
 * already pending on the calling thread (that error is left set).
 * Asynchronous; n_idx == 0 is a no-op.
 * ---------------------------------------------------------------------- */
nb_status nb_force_jerk_noalloc(int64_t n, const double *d_m,
                                const double *d_x, const double *d_v,
                                const int32_t *d_idx, int64_t n_idx,
                                double eps, double G, int32_t precision,
                                double *d_acc, double *d_jerk, void *stream);

const char *nb_status_string(nb_status s);
const char *nb_last_error(void); /* message of the last error on this thread */

#ifdef __cplusplus
}
#endif
#endif /* NBODY_GB300_H */
