/*
 * eik.h -- C ABI of the GB300 (sm_103a) exactly monotone Eikonal solver.
 *
 * What it computes (arXiv 2103.05694, Henriksen, You, Pingali):
 *   the arrival times t of the Dirichlet problem ||grad t|| = 1/v (Eq.
 *   eikonal_bvp) discretised by the first-order upwind scheme (Eq.
 *   finite_difference), i.e. the unique fixed point of the local update
 *   operator (Theorem 1), where the operator is evaluated with the paper's
 *   exactly monotone rounding d-bar (section "Achieving Exact Monotonicity
 *   with Finite Precision Arithmetic"):
 *
 *     for a non-source cell n with axis minima a_k = min(t[n - e_k], t[n + e_k])
 *     (off-grid neighbours count as +inf), r = fl(h / v_n), c = fl(r * r):
 *       G(tau) = fl(fl(q_x + q_y) + q_z),  q_k = fl(m_k * m_k),
 *       m_k = max(fl(tau - a_k), +0),
 *       t[n] = the smallest binary64 tau with G(tau) >= c  (+inf if all a_k = +inf).
 *   Source cells keep their given time t0 (duplicates: the smallest).
 *
 * The fixed point is reached by asynchronous relaxed-priority scheduling
 * (Algorithm 6, "Asynchronous Marching Method"): a persistent CUDA kernel pops
 * tiles of cells from integer buckets floor(t / delta) and relaxes them.
 * Because d-bar is exactly monotone and causal, every schedule gives the same
 * bits (Theorem 1); the result equals a single-threaded fast marching method
 * (Algorithm 2) with the same d-bar bit for bit.
 *
 * Layout: every grid is C-order with x (the last dimension) contiguous;
 * dims = {ny, nx} for ndim = 2 and {nz, ny, nx} for ndim = 3.  Terms of G are
 * summed in axis order x, y, z.  Sources are flat C-order cell indices.
 *
 * Memory: pointer arguments may be device pointers (cudaMalloc, torch CUDA
 * tensors) or host pointers (pageable or pinned); each is classified with
 * cudaPointerGetAttributes.  Pinned host memory is mapped into the device's
 * address space, so the library's kernels read and write it in place over the
 * chip-to-chip link inside the call.  Speeds are read by the kernel that forms
 * c; outputs are written by one copy kernel after the solve.  Other host
 * buffers are copied with cudaMemcpyAsync.  The caller owns every buffer it
 * passes; the library owns its workspace (device scratch sized to the largest
 * problem seen, kept per device until eik_release()).
 *
 * Streams: work is enqueued on `stream` (a cudaStream_t, NULL = legacy default
 * stream).  Calls return after the stream has reached the end of the call's
 * work (the status is read back from the device); they are not thread-safe
 * against each other (a process-wide lock serialises them).
 *
 * Errors: inputs are checked on the host before launch where the data is
 * host-visible (EIK_EINVAL, nothing launched), and on the device otherwise
 * (speed <= 0, non-finite speed or h/v, source index out of range, negative or
 * NaN source time: EIK_EINVAL, out_t contents unspecified).  A device wait
 * that exceeds its limit ends the kernel with EIK_ETIMEOUT; it never traps.
 * A frontier overflow is retried internally with a larger capacity; it is
 * reported (EIK_ECAPACITY) only when the capacity limit is reached.
 */
#ifndef EIK_H
#define EIK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EIK_OK = 0,
    EIK_EINVAL = 1,     /* bad argument (host check) or bad input data (device check) */
    EIK_ENOMEM = 2,     /* device or pinned-host allocation failed */
    EIK_ECAPACITY = 3,  /* frontier overflow at the largest allowed capacity */
    EIK_ETIMEOUT = 4,   /* a device wait reached its limit; the kernel returned */
    EIK_ECUDA = 5       /* a CUDA runtime call failed (message: eik_last_error()) */
} eik_status;

/* Tuning knobs.  Zero (or a NULL pointer) selects the default; eik_autotune picks
 * them for a given batch.  Defaults depend on how many independent wavefronts the
 * batch has:
 *   2D, fewer than 8 sources in the batch: 16x16 tiles, k_delta 16, window 16,
 *     band 16, 1 CTA per SM (latency-bound: one front);
 *   2D, 8 or more sources: 16x8 tiles, k_delta 4, window 16, band 8, 8 CTAs of
 *     128 threads per SM;
 *   3D, fewer than 8 sources: 4x4x4 tiles, k_delta 0.75, window 31, band 6, 14 CTAs
 *     of 64 threads per SM;
 *   3D, 8 or more sources: 4x4x4 tiles, k_delta 0.375, window 31, band 6, 20 CTAs
 *     of 64 threads per SM (a lean build compiled for 20 CTAs; a solve that needs the
 *     full build runs 16: counters, a trace, the update forms, change tracking, or
 *     fewer than 8 tiles per CTA, where lists use lane groups).
 * (The per-CTA work is latency-bound, so the kernel is compiled for as many
 * resident CTAs as registers allow: 2 per SM for 256-cell tiles, 8 for 128-cell
 * tiles, 16 for 64-cell tiles, 20 for the wide lean build of 4x4x4 tiles.)
 * With arith = 2 the first shape (16x16, 8x8x4) and k_delta 16 (2D) / 2 (3D). */
typedef struct {
    double delta;          /* bucket width in time units; <= 0: auto (k_delta * mean h/v) */
    double k_delta;        /* auto bucket width in cell travel times; <= 0: default (above) */
    int64_t capacity;      /* initial frontier ring capacity per bucket slot; 0: auto */
    int64_t timeout_ms;    /* limit of any single device wait; 0: 60000 */
    int ctas_per_sm;       /* persistent CTAs per SM, capped by what the launched build holds
                              resident (above; above 16, 4x4x4 3D tiles take the wide lean
                              build when the solve is lean); 0: default */
    int counters;          /* nonzero: collect eik_stats counters (small cost) */
    int test_stall;        /* testing aid, keep 0: the solve first waits on a device flag
                              that nothing sets, so the wait reaches timeout_ms and the
                              call returns EIK_ETIMEOUT (exercises the bounded waits) */
    int window;            /* buckets above the lowest active bucket that may be worked on
                              (look-ahead of the relaxed priority order; values above 31
                              act as 31); 0: default */
    double band;           /* in-tile acceptance band in units of (smallest h/v of the tile)
                              / sqrt(ndim), i.e. one cell's travel time; <= 0: default */
    int arith;             /* arithmetic of d-bar: 1 = FP64 unit, 2 = exact emulation on the
                              integer pipes (same results bit for bit); 0: default */
    int sched_flags;       /* bit 0: the look-ahead window follows the lowest bucket holding
                              queued entries only (tiles still running do not hold it);
                              bits 1-2: lane-group d-bar, 0 = automatic (when the batch has
                              fewer than 8 tiles per persistent CTA), 1 = never, 2 = for
                              lists of up to a quarter of the tile, 3 = an eighth;
                              bits 3-4 (eik_adjoint only): schedule, 0 = default (tiles when
                              every problem has the same ndim, else levels), 1 = levels,
                              2 = tiles;
                              bit 5 (update 1-3 only, EIK_EINVAL otherwise): change tracking,
                              the conservative work tracking of the Mitigation Strategies
                              section: a recomputed value that differs from the cell's, up or
                              down, replaces it and re-activates the neighbours (termination
                              is no longer guaranteed: after 256 tile visits per tile the
                              solve stops with EIK_ETIMEOUT);
                              bit 6 (eik_solve, eik_solve_batched, eik_solve_noalloc, plans,
                              eik_autotune, eik_adjoint): the `speed` arrays hold slowness s
                              instead, and the speed used is v = fl(1/s), correctly rounded, on
                              the device (the traveltime-tomography parameterisation);
                              bit 7 (eik_adjoint only): problems whose dL_dslowness pointers
                              are equal form a group, and that array receives the sum of their
                              gradients, +0 + g_first + ... + g_last in problem order, each
                              addition rounded to nearest (deterministic; the per-problem
                              gradients go to library workspace, 8 bytes per cell of the
                              batch) */
    void *trace;           /* optional device buffer of trace_cap 32-byte visit records
                              {int64 t_claim_ns, t_end_ns; uint32 tile, lowest bucket,
                              rounds, flags}; NULL: no trace */
    int64_t trace_cap;
    int tile;              /* tile shape, cells x*y(*z), one CTA thread per cell; 0: default
                              (above).  2D: 1 = 16x16, 2 = 32x8, 3 = 32x4, 4 = 16x8,
                              5 = 16x4; 3D: 1 = 8x8x4, 2 = 16x4x4, 3 = 32x4x2, 4 = 8x4x4,
                              5 = 4x4x4.  Shapes 2-5 need arith 0/1 (EIK_EINVAL otherwise). */
    int update;            /* the local update: 0 = d-bar, exactly monotone (section "Achieving
                              Exact Monotonicity"), the default; for the ablation of the
                              Mitigation Strategies section, 2D only: 1 = Algorithm 1 with the
                              classical explicit root d-tilde, 2 = with the rearranged root
                              d-hat, 3 = d-hat refined by Newton's method on the root problem
                              (the variant of the Achieving Exact Monotonicity section; stops
                              when an iterate repeats or after 4 steps).  1-3 are not proven
                              monotone: results may depend on the schedule and need not be a
                              fixed point (Table 3). */
    int schedule;          /* 0 = asynchronous bucketed tiles (Algorithm 6), the default;
                              single problems only, device pointers, for comparison:
                              1 = fast iterative method (Algorithm 3, epsilon = 0, rounds),
                              2 = topology-driven (Algorithm 4, every cell every iteration),
                              3 = fast sweeping method (Algorithm 5, 2^ndim sweep directions,
                              each sweep in hyperplane order).  Same bits (Theorem 1),
                              different work and time.  Options other than timeout_ms and
                              counters do not apply to 1-3. */
    int reserved;          /* keep 0 */
} eik_opts;

/* Work accounting (the paper's good/empty/bad updates, Results section). */
typedef struct {
    int64_t evals;         /* operator applications (cells flagged for update) */
    int64_t decreases;     /* applications that lowered a value (good + bad) */
    int64_t good;          /* reached non-source cells (one final-setting update each) */
    int64_t visits;        /* tile visits by the persistent kernel */
    int64_t pushes;        /* frontier entries pushed */
    int64_t stale_pops;    /* frontier entries dropped as stale */
    int64_t rounds;        /* relaxation rounds summed over tile visits */
    int64_t retries;       /* capacity retries performed */
    int64_t max_queue;     /* deepest bucket slot seen at a push (entries) */
    int64_t visit_ns;      /* tile-visit time summed over CTAs (counters only) */
    int64_t idle_ns;       /* time CTAs spent looking for work (counters only) */
    int64_t ctas;          /* persistent CTAs launched */
    int64_t trace_n;       /* visit records produced (only the first trace_cap are stored) */
    int64_t detail[9];     /* counters >= 2 only: SM cycles of one thread per CTA spent in
                              [0] tile load, [1] round phase A (acceptance of the previous
                              round's candidates and evaluation), [2] phase B (d-bar),
                              [3] 0 (no separate acceptance phase), [4] commit and
                              activation; [5] Newton steps, [6] ulp-walk steps,
                              [7] bisection fallbacks, [8] d-bar evaluations */
    double solve_ms;       /* device time of the persistent solve kernel(s), CUDA events
                              recorded on `stream` around each launch */
} eik_stats;

/* Solve one grid (Algorithm 6 with d-bar, result identical to Algorithm 2).
 *   speed   [N] float64, v > 0 finite (device or host)
 *   h       grid spacing, > 0 finite
 *   ndim    2 or 3; dims[ndim] C-order extents, each >= 1, product N < 2^40
 *   src_idx [nsrc] int64 flat indices in [0, N); src_t [nsrc] float64 >= 0
 *           (NULL: all 0); nsrc >= 0 (0 leaves every cell at +inf)
 *   out_t   [N] float64 arrival times (written; +inf where unreachable)
 *   opts    NULL for defaults; stats NULL if not wanted.
 */
eik_status eik_solve(const double *speed, double h, int ndim, const int64_t *dims,
                     const int64_t *src_idx, const double *src_t, int64_t nsrc,
                     double *out_t, const eik_opts *opts, eik_stats *stats, void *stream);

/* One problem of a batch.  Each pointer may be a device or a host pointer
 * (see Memory above).  Problems may share a speed array. */
typedef struct {
    const double *speed;
    double h;
    int ndim;
    int64_t dims[3];
    const int64_t *src_idx;
    const double *src_t;   /* NULL: all sources at 0 */
    int64_t nsrc;
    double *out_t;
} eik_problem;

/* Solve nprob independent problems in ONE persistent launch: tiles of every
 * problem share the bucket scheduler (batching of sources and uneven grids).
 * stats (optional) accumulates over the batch. */
eik_status eik_solve_batched(const eik_problem *probs, int nprob, const eik_opts *opts,
                             eik_stats *stats, void *stream);

/* Self-test of the exact arithmetic.  d-bar can be evaluated with exact
 * round-to-nearest binary64 operations emulated on the integer pipes (FP64 is
 * scarce on GB300, opts.arith = 2) or on the FP64 unit (the default, with a
 * float-float starting point and an exact test); this runs n random and
 * tie-heavy trials on the current device, comparing each emulated operation
 * with the hardware FP64 unit, and each d-bar with a plain bisection over G
 * built from the hardware operations, bit for bit.  mismatches[32] receives:
 * [0] x-y, [1] m*m, [2] x+y, [3] G 2D, [4] G 3D, [5] integer d-bar 2D,
 * [6] integer d-bar 3D, [7] lane-group update 2D x8, [8] 3D x8, [9] 2D x4,
 * [10] FP64-unit d-bar 2D, [11] FP64-unit d-bar 3D mismatch counts,
 * [15] trials run, [16 + k] the first failing trial of check k (-1 if none).
 * Allocates and frees a small device buffer; synchronises `stream`. */
eik_status eik_selftest(int64_t n, uint64_t seed, int64_t *mismatches, void *stream);

/* Instrument for the FP64 roofline (the paper has no counterpart): the
 * current device's throughput of FP64 additions, in thread instructions per
 * second (*inst_per_s), timed with CUDA events over one launch of eight
 * independent __dadd_rn chains per thread, `iters` steps each, on 8 CTAs of
 * 256 threads per SM (after one shorter warm-up launch).  GB300's FP64 unit
 * runs DADD, DMUL and DFMA at one rate.  Allocates and frees a small device
 * buffer; synchronises `stream`.  EIK_EINVAL for iters <= 0. */
eik_status eik_fp64_rate(int64_t iters, double *inst_per_s, void *stream);

/* The single-grid solve of eik_solve without allocating any memory.  (The
 * paper has no counterpart: this serves callers that cannot allocate device
 * memory, e.g. code whose device memory belongs to an arena allocator that
 * forbids outside cudaMalloc calls, or latency-sensitive loops where
 * cudaMalloc / cudaFree would synchronise the device.)
 *   Arguments and results as eik_solve, with these limits:
 *   - speed, src_idx, src_t (if not NULL) and out_t must be device pointers;
 *   - at most 2^20 cells, 2^15 tiles (2D tiles 16x16, 3D tiles 8x8x4) and
 *     2048 sources; larger inputs return EIK_EINVAL before anything runs;
 *   - no capacity retry: a frontier overflow returns EIK_ECAPACITY;
 *   - stats->solve_ms, max_queue and the timing details stay 0;
 *     opts->trace and opts->test_stall are ignored;
 *   - the first tile shape (16x16, 8x8x4) whatever the dimension, k_delta 16 (2D) /
 *     2 (3D) unless opts->k_delta is set; opts->tile must be 0.
 * Scratch memory is one fixed file-scope device array of about 21 MB, present
 * on every GPU that loads the library until the process exits.  Each call
 * looks up that array's device address on the current device
 * (cudaGetSymbolAddress, which allocates nothing).  Every call shares the
 * array and clears what must start at zero; calls whose GPU work overlaps
 * (other streams, other host threads) race on it and must be serialised by
 * the caller.  Every failure leaves its reason for eik_last_error().
 * Synchronises `stream` to read the status. */
eik_status eik_solve_noalloc(const double *speed, double h, int ndim, const int64_t *dims,
                             const int64_t *src_idx, const double *src_t, int64_t nsrc,
                             double *out_t, const eik_opts *opts, eik_stats *stats,
                             void *stream);

/* Adjoint for traveltime tomography (not in the paper: implicit
 * differentiation of the real-arithmetic local equations at the computed
 * fixed point).  For each problem i, probs[i].out_t must hold the arrival
 * times solved for exactly that problem (speed, h, sources); dL_dt[i] (NULL,
 * or dL_dt == NULL: zero) is d(loss)/d(t) per cell; dL_dslowness[i] receives
 * d(loss)/d(s) with slowness s = 1/v per cell (written, not accumulated; 0 at
 * sources and unreachable cells; with opts->sched_flags bit 7, problems that
 * share an output array receive their gradients' sum in problem order; with
 * bit 6, probs[i].speed holds slowness and v = fl(1/s)).  For a reached
 * non-source cell n with axis
 * minima a_k and active axes A = {k : a_k < t_n}, S_n = sum_A (t_n - a_k):
 *   lambda_n = dL_dt_n + sum_{downwind m} lambda_m (t_m - t_n) / S_m
 *   (halved where m's two neighbours on that axis tie), downwind neighbours in
 *   the order x-, x+, y-, y+, z-, z+;  dL/ds_n = lambda_n (h^2 s_n) / S_n.
 * Every operation is separately rounded in that order, so results are
 * reproducible bit for bit.  Device pointers only.  A parallel set-up pass
 * evaluates every weight; then the cells are processed in dependency order by
 * one of two schedules (opts->sched_flags bits 3-4), with the same results:
 *   tiles (default): persistent CTAs take tiles of 16x8 (2D) or 8x8x4 (3D)
 *     cells from a queue and run the dependency order inside a tile in shared
 *     memory; a tile is queued when a cell of it may have become ready;
 *   levels: one cooperative launch processes the cells level by level, its
 *     blocks meeting at a grid barrier between levels.
 * Every device wait is bounded by opts->timeout_ms (EIK_ETIMEOUT); opts->
 * ctas_per_sm caps the CTAs of the tile schedule.  Workspace: about 34 (tiles)
 * or 53 (levels) bytes per cell of the batch, kept for the next call
 * (eik_release frees it).
 * Synchronises `stream`.  stats (optional): good = cells processed, evals =
 * reached cells, solve_ms = device time of the adjoint launches; tiles: visits
 * = tile visits, rounds = in-tile rounds summed over visits, ctas; with
 * opts->counters also visit_ns / idle_ns = CTA time in visits / waiting for a
 * tile and detail[0..3] = SM cycles (thread 0 of each CTA, summed) waiting,
 * loading, in rounds, storing (a build of the kernel with these clocks);
 * levels: rounds = levels. */
eik_status eik_adjoint(const eik_problem *probs, int nprob, const double *const *dL_dt,
                       double *const *dL_dslowness, const eik_opts *opts, eik_stats *stats,
                       void *stream);

/* Slab decomposition of one grid (the domain decomposition that the paper
 * leaves to future work, Introduction).  Solves the same problem as eik_solve,
 * with the same result bit for bit: the outermost axis (z in 3D, y in 2D) is
 * split into nslabs slabs of near-equal thickness; each slab, extended by one
 * ghost row on each side it shares with a neighbour, is one problem of a batch
 * (one persistent launch for all slabs).  A ghost row holds the neighbour's
 * values of those cells from the previous epoch as fixed sources (cells the
 * neighbour has not reached yet stay free).  Between epochs the rows next to
 * each slab boundary are copied, device to device, into an exchange buffer;
 * the epochs repeat until no exchanged value changes (a global AND over the
 * boundaries).  Ghost values only decrease from epoch to epoch, so the loop
 * ends, and then every cell satisfies the update with its neighbours' final
 * values: the union is the unique fixed point (Theorem 1).  Every epoch
 * solves the slabs from +inf; all slabs run on the calling device (with one
 * slab per GPU, the exchange is a peer copy of one row into the neighbour's
 * memory).
 *   speed, out_t: device pointers; src_idx / src_t: host or device; other
 *   arguments as eik_solve.  1 <= nslabs <= outermost extent (EIK_EINVAL
 *   otherwise); opts->update, schedule, test_stall and sched_flags bit 5 must
 *   be 0.  *epochs (optional) receives the number of epochs; stats accumulate
 *   over them (good: reached non-source cells, with opts->counters).  More than
 *   64 + 8 nslabs epochs give EIK_ETIMEOUT.  Workspace: one field per slab (the
 *   grid plus 2 (nslabs - 1) rows) and 2 (nslabs - 1) exchanged rows.
 *   Synchronises `stream`. */
eik_status eik_solve_slabs(const double *speed, double h, int ndim, const int64_t *dims,
                           const int64_t *src_idx, const double *src_t, int64_t nsrc,
                           double *out_t, int nslabs, const eik_opts *opts, eik_stats *stats,
                           int *epochs, void *stream);

/* Fixed-order sum of k arrays of n doubles: dst[i] = (((+0 + src[0][i]) +
 * src[1][i]) + ...) + src[k-1][i], each addition rounded to nearest in that
 * order (k = 0 writes +0).  src is a host array of k device pointers; dst a
 * device pointer (it may alias none of the inputs).  This is the cross-source
 * gradient sum of eik_adjoint's sched_flags bit 7, exposed for sharded
 * tomography: ranks that solved different sources gather their per-source
 * gradients on one device and sum them here in source order, which gives the
 * bits of the single-device step.  (Not in the paper.)  EIK_EINVAL for
 * non-device pointers.  Synchronises `stream`. */
eik_status eik_sum_ordered(const double *const *src, int k, double *dst, int64_t n, void *stream);

/* Update-form ablation (Mitigation Strategies section, Tables 1 and 2): for
 * i < n, out[i] = one application of Algorithm 1 at a cell of speed v = speed[i]
 * with axis minima t_h[i], t_v[i] (2D): form 1 = classical root d-tilde,
 * form 2 = rearranged root d-hat, form 3 = d-hat then Newton (as eik_opts.update;
 * all three one-sided min + h/v when |t_h - t_v| >= h/v or one minimum is +inf),
 * form 0 = d-bar.  +inf when both minima are +inf.
 * Device pointers only; EIK_EINVAL otherwise.  Synchronises `stream`.  The
 * paper has no interface of this kind: it exposes the update for testing. */
eik_status eik_eval_update(int form, const double *speed, double h, const double *t_h,
                           const double *t_v, int64_t n, double *out, void *stream);

/* The fixed-point residual of Table 3: re-applies the update (form as in
 * eik_eval_update; 1-3: 2D only) at every cell of prob->out_t using the
 * final values of its neighbours.  *bad = cells whose value changes (sources:
 * value != their smallest t0), *max_rel = the largest |t - tau| / t over cells
 * where both are finite and t > 0 (+inf if a changing cell is not), 0 for a
 * fixed point.  prob: device pointers only.  Synchronises `stream`. */
eik_status eik_residual(const eik_problem *prob, int form, int64_t *bad, double *max_rel,
                        void *stream);

/* One configuration tried by eik_autotune. */
typedef struct {
    eik_opts opts;         /* the configuration, with explicit values */
    double ms;             /* fastest device time of the solve over the repeats; -1 on failure */
    int status;            /* eik_status of the trial */
    int reserved;
} eik_tune_trial;

/* Autotuner (the paper leaves the bucket width Delta open; tile shape,
 * look-ahead window, acceptance band, CTAs per SM and frontier capacity are
 * this implementation's).  Solves the batch (device pointers only, as
 * eik_solve_batched) `repeats` times per configuration (<= 0: 2) and does
 * coordinate descent from `base` (NULL: defaults) over tile, k_delta (unless
 * base->delta > 0), window, band and ctas_per_sm, at most two passes; a change
 * is kept when it saves more than 1 % of the fastest device time.  Then sets
 * capacity (unless base->capacity > 0) to 16x the deepest bucket slot seen (at
 * least 1024).
 * Every trial's output must equal the first trial's bit for bit (a digest of
 * all outputs is compared; the fixed point does not depend on the schedule,
 * Theorem 1): otherwise EIK_ECUDA.  The outputs hold the solution on return.
 * best receives the chosen options; trials[0..*ntrials) (optional, up to
 * max_trials) the configurations tried, in order.  base->update must be 0 (the
 * explicit forms give schedule-dependent bits): EIK_EINVAL.  Synchronous. */
eik_status eik_autotune(const eik_problem *probs, int nprob, const eik_opts *base, int repeats,
                        eik_opts *best, eik_tune_trial *trials, int max_trials, int *ntrials,
                        void *stream);

/* Plans: a batch prepared once and solved many times.
 * eik_plan_create checks the problems (device pointers, or pinned host pointers
 * that each solve reads and writes in place; all of one ndim),
 * copies and de-duplicates their sources, and allocates the plan's own device
 * workspace (synchronous).  eik_plan_enqueue enqueues one complete solve of
 * every problem on `stream` -- constants, initial field, seeds and ONE
 * persistent launch over the tiles of all problems -- without allocating and
 * without waiting for the device, so a CUDA graph can capture it and replay it.
 * The speed arrays are read and out_t written by each solve; keep them alive
 * while the plan is used.  eik_plan_status synchronises `stream` and returns
 * the status of the last completed solve (and its counters when the plan was
 * created with opts->counters); a frontier overflow is reported as
 * EIK_ECAPACITY (no retry inside a plan: create it with a larger capacity).
 * eik_plan_destroy frees the plan (after its work has completed). */
typedef struct eik_plan eik_plan;
eik_status eik_plan_create(const eik_problem *probs, int nprob, const eik_opts *opts,
                           eik_plan **plan);
eik_status eik_plan_enqueue(eik_plan *plan, void *stream);
eik_status eik_plan_status(eik_plan *plan, eik_stats *stats, void *stream);
void eik_plan_destroy(eik_plan *plan);

/* Release the library's device workspace on the current device. */
void eik_release(void);

/* Human-readable name of a status code (static string). */
const char *eik_status_str(eik_status s);

/* Message of the last EIK_ECUDA / EIK_EINVAL of this process (static buffer). */
const char *eik_last_error(void);

/* Version of the ABI (major * 100 + minor). */
int eik_abi_version(void);

/* Number of CUDA kernels this library has launched, or enqueued into a stream
 * capture, since it was loaded (all devices, all threads).  A caller that
 * replays a captured graph counts the kernels captured per enqueue itself.
 * The paper has no counterpart: it is an instrument for counting device work. */
uint64_t eik_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* EIK_H */
