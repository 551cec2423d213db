/*
 * vmc.h -- C ABI of the GB300 sparse determinant-ratio engine.
 *
 * The engine computes, for single-electron variational Monte Carlo moves, the
 * determinant ratio of successive Slater matrices
 *     det(A') / det(A) = 1 + u^T A^{-1} e_i ,   u = a' - a_i
 * (Ahuja, Clark, de Sturler, Ceperley, Kim, "Improved Scaling for Quantum Monte
 * Carlo on Insulators": Sec. 1 Eq. 2; Sec. 3 Eqs. 11-13) by solving A z = e_i with
 * right-preconditioned GMRES (Sec. 3.2 Eq. 15), the preconditioner being ILUTP
 * (Sec. 3.2 Eq. 14; Sec. 4) of a geometrically reordered matrix (Sec. 3.1, the
 * greedy particle/orbital algorithm), cheaply updated after every accepted move
 * (Sec. 3.2 Eqs. 16-18), with the effective-stability monitor N of Sec. 3.1 Eq. 10
 * deciding when to reorder and refactor (Sec. 4).
 *
 * Conventions for every call:
 *   - Pointers are plain host pointers unless the name says "_dev" (device).
 *   - Host inputs are copied before the call returns; host outputs are written
 *     before it returns (the call synchronises its stream when it copies to host).
 *   - The context owns all device memory it allocates; vmc_destroy frees it.
 *   - Errors are returned as vmc_status; nothing aborts, throws or traps across
 *     the ABI.  vmc_last_error() describes the most recent failure.
 *   - Particle ids k and walker ids are the caller's (original) labels; the
 *     reorderings are internal.
 *   - A context is not thread-safe; calls on one context must be serialised.
 */
#ifndef VMC_H
#define VMC_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vmc_ctx vmc_ctx; /* opaque */

typedef enum {
  VMC_OK = 0,
  VMC_ERR_INVALID = 1,   /* bad argument or size                                  */
  VMC_ERR_CUDA = 2,      /* a CUDA runtime call failed                             */
  VMC_ERR_OOM = 3,       /* device allocation failed                               */
  VMC_ERR_NOCONV = 4,    /* GMRES did not converge after reorder + restarts        */
  VMC_ERR_BREAKDOWN = 5, /* singular Slater matrix or unusable factorisation       */
  VMC_ERR_TIMEOUT = 6,   /* a bounded device wait ran out                          */
  VMC_ERR_STATE = 7,     /* call out of order (e.g. vmc_accept without vmc_ratio)  */
  VMC_ERR_CAPACITY = 8   /* a fixed device capacity was exceeded                   */
} vmc_status;

/* One walker's physical system (Sec. 2.1 Eq. 3; Sec. 4).
 * Sites: simple cubic Z = a (x, y, z), x, y, z in [0, K), numbered
 * j = x + K (y + K z); body-centred cubic adds a (x+1/2, y+1/2, z+1/2) as j = 2 cell + 1
 * (corner j = 2 cell).  Orbitals phi_j(r) = exp(-kappa |r - Z_j|^2) when the
 * minimum-image distance is <= r_c, else 0.  Box side L = K a, periodic.
 * Requires r_c < L/2 and r_c larger than the lattice's covering radius. */
typedef struct {
  int K;          /* cells per side (>= 2)                     */
  int lattice;    /* 0 = simple cubic (n = K^3), 1 = bcc (2K^3) */
  double a;       /* lattice constant                          */
  double kappa;   /* Gaussian decay rate                       */
  double r_c;     /* orbital cutoff radius                     */
} vmc_system;

/* Precision (the precision split of Sec. 3.2 on GB300):
 *   FP64        : everything in FP64.
 *   MIXED       : ILUTP factorisation (pivot selection, elimination, dropping) in FP64,
 *                 factors stored and applied in FP32, inner GMRES in FP32; FP64 outer
 *                 refinement residual e_i - A x, ratio 1 + u^T x and stability monitor.
 *   MIXED_F32ILU: as MIXED but the ILUTP working row is FP32 too (faster refactoring;
 *                 the stored factors are FP32 in both mixed modes). */
enum { VMC_PREC_FP64 = 0, VMC_PREC_MIXED = 1, VMC_PREC_MIXED_F32ILU = 2 };
enum {
  VMC_ENGINE_PLAIN = 0,      /* one walker per launch, one launch per move step      */
  VMC_ENGINE_STEP = 1,       /* one launch per move step advancing every walker      */
  VMC_ENGINE_PERSISTENT = 2, /* one launch per sweep, every walker (a CTA per walker,
                                or a CTA pair with background refactorisation)      */
  VMC_ENGINE_DENSE_SM = 3    /* explicit inverse + Sherman-Morrison (Sec. 1), FP64;
                                vmc_sweep only (single-move and inspection calls return
                                VMC_ERR_INVALID); a fresh inverse every sm_refresh sweeps */
};

/* Solver parameters.  vmc_default_params() fills the defaults noted here. */
typedef struct {
  double drop_tol;     /* ILUTP drop tolerance tau, relative to ||a_i||_2 (1e-4)         */
  double permtol;      /* ILUTP column-pivot tolerance: swap when permtol|w_j| > |w_i| (0.5) */
  int lfil_extra;      /* extra entries kept per L and per U row; < 0: ceil(avg nnz/row / 2) (-1) */
  int gmres_m;         /* Krylov dimension per inner solve, <= 40 (30)                   */
  int max_restarts;    /* GMRES cycles of a solve beyond the first two (10); a solve still short
                          of its goal then reorders, refactors and solves again from scratch with
                          four times as many cycles, and reports VMC_ERR_NOCONV if that fails */
  double inner_rtol;   /* inner GMRES relative tolerance; <= 0: 1e-10 FP64, 1e-5 mixed (0) */
  double ratio_tol;    /* goal: predicted relative ratio error (1e-12)                   */
  double N_max;        /* reorder + refactor when the stability monitor N exceeds it (100) */
  double slow_factor;  /* ... or when the iterations reach slow_factor x the average (4)  */
  int max_updates;     /* refactor after this many rank-one preconditioner updates; -1 =
                          auto: 64 with background refactorisation, 128 without (-1)    */
  int precision;       /* VMC_PREC_* (MIXED)                                               */
  int engine;          /* VMC_ENGINE_* (PERSISTENT)                                        */
  int block_threads;   /* threads per walker CTA: 64..256, multiple of 32; 0 = auto (0)  */
  int sm_refresh;      /* dense engine: fresh inverse every sm_refresh sweeps; 0: never (1) */
  int refactor_lag;    /* PERSISTENT engine: background refactorisation.  A second CTA per
                          walker (a cluster of two) factors a snapshot of A taken once the
                          update chain holds refactor_lag updates past its root; the solver
                          adopts those factors exactly refactor_lag accepts later (waiting for
                          them if need be) and keeps only the newer chain entries (Sec. 3.2
                          Eqs. 16-18 hold for any root), so results do not depend on timing.
                          0: off (refactor in line when the chain is full); > 0: on, clamped
                          to max_updates / 2; -1: auto -- on with max_updates / 2 when every
                          walker pair fits on the GPU at once (2 x walkers <= SMs) and no
                          system exceeds n = 8192 (beyond that one factorisation outlasts
                          the accepts between adoptions and in-line refactoring is faster;
                          at n = 32768 it takes about 28 s, near the 30 s bound on the
                          solver's wait, past which the walker reports VMC_ERR_TIMEOUT) (-1) */
  int refactor_reorder; /* background refactorisations first re-pair particles and orbitals
                          (the greedy reordering of Sec. 3.1) on the snapshot positions; the
                          solver adopts the new row order with the factors (0) */
  int trisolve;        /* triangular solves: 0 = level-synchronous (a barrier among the
                          solving warps per level); 1 = synchronisation-free
                          when both solve vectors fit in shared memory (a warp waits only for
                          the entries its rows read), else level-synchronous (0) */
  int graphs;          /* STEP and PLAIN engines: capture one sweep's launches as a CUDA graph
                          (with the sweep index kept on the device) and replay it once per
                          sweep (1), or launch them one by one (0).  Used when the call makes
                          one sweep or keeps no logs (1) */
  double trigger_rtol; /* the controller's convergence test (Sec. 4: reorder when the iterative
                          solver does not reach the required tolerance within the maximum number
                          of iterations): the solve of a move counts as converged when its
                          residual reaches trigger_rtol x ||e_i|| within trigger_its GMRES
                          iterations, counted over all cycles (restarts and refinement passes).
                          The solve itself always runs on to inner_rtol and the ratio goal;
                          a failed test reorders and refactors for the moves that follow.
                          <= 0: 1e-6, the paper's GMRES tolerance (1e-6) */
  int trigger_its;     /* ... and its maximum iteration count; <= 0: 40, the paper's (40) */
  int sweep_moves;     /* moves per sweep: 0 = every particle (a full sweep); m > 0 = only
                          particles 0 .. m-1 of each walker (bounded partial sweeps for tests,
                          diagnostics and autotuner trials; the log entries of particles not
                          moved are left unwritten) (0) */
  int ilutp_variant;   /* ILUTP implementation (same factors, bit for bit): 0 = auto: the
                          working row in shared memory as a hash map keyed by label when the dense
                          working row of n entries does not fit the walker CTA's shared memory
                          (and n <= 65535), else the dense row; 1 = always the dense row; 2 =
                          always the hash map where it fits (0) */
  int trisolve_warp_rows; /* level-synchronous triangular solves: a level of at most this many
                          rows, <= 32, is solved by one warp alone, with no barrier among the
                          solving warps after it (the other warps meet it before the next larger
                          level); 0 = every level by all solving warps (0) */
  int trisolve_group;  /* grouped triangular solves (a partitioned inverse of each factor): at
                          every factorisation, consecutive levels are merged into groups of at
                          most this many levels and each row of a group is expanded, by
                          substitution of the group's earlier rows, into a row that reads only
                          the input vector and the solution of earlier groups; the solve then
                          synchronises once per group instead of once per level.  The same
                          operator as level-by-level substitution in exact arithmetic.  A level
                          whose expanded rows would exceed the expanded-row capacity
                          (trisolve_row_cap) starts a new group.  0 or 1: level by level;
                          ignored with trisolve = 1 (8) */
  int trisolve_row_cap; /* expanded-row capacity of the grouped solves, in entries: 0 = max(c + 4,
                          min(2 c, 160)) with c the factor-row capacity; otherwise max(c + 4,
                          this), at most 480 (0) */
  int trisolve_lane_entries; /* triangular solves: each row is summed by a group of lanes sized
                          for at most this many entries a lane on the level's (group's)
                          longest row, <= 64; 0 = 2 in FP32, 8 in FP64 (0) */
} vmc_solver_params;

/* Per-walker statistics (Sec. 4 Tables 2 and 3 analogues). */
typedef struct {
  int64_t proposals, accepts;
  int64_t solves;            /* linear solves started (one per ratio, plus re-solves)      */
  int64_t inner_iterations;  /* GMRES iterations over all passes                           */
  int64_t first_pass_iterations; /* iterations of the first pass (the paper's k1 count)    */
  int64_t outer_passes;      /* FP64 refinement passes                                      */
  int64_t reorders;          /* reorder + refactor events (all causes)                      */
  int64_t reorder_monitor, reorder_noconv, reorder_slow, reorder_breakdown;
  int64_t refactors_updates; /* refactorisations because max_updates was reached           */
  int64_t factorizations;    /* all ILUTP factorisations                                   */
  int64_t pivots;            /* ILUTP column swaps in the last factorisation               */
  double N_max_seen, N_sum;  /* stability monitor: max and sum over solves                 */
  double nnz_A, nnz_LU;      /* nonzeros of A and of L+U at the last factorisation         */
  int levels_L, levels_U;    /* triangular-solve level counts at the last factorisation    */
  int n_updates;             /* current length of the update chain                         */
  int status;                /* vmc_status of this walker (sticky)                          */
  int64_t its_hist[64];      /* histogram of first-pass iterations (last bin: >= 63)       */
  int64_t phase_cycles[16];  /* SM clock cycles by phase (thread 0 of the walker's CTA):
                                0 row build, 1 first solve pass, 2 refinement passes,
                                3 factorisation incl. reorder, 4 reordering, 5 commit + update,
                                6 whole steps, 7 triangular solves, 8 update-chain apply,
                                9 SpMV, 10 orthogonalisation + Givens, 11 FP64 residuals,
                                12 ILUTP rows, 13 level sets + streams, 14 producer waits
                                for a free ring slot (inside 7), 15 consumer waits for
                                triangular-factor chunks to land (inside 7) */
  double alg_bytes;          /* algorithmic (compulsory) bytes of the solves: per phase the
                                matrix/factor values and indices, the vectors read and written */
  int64_t ilu_rows, ilu_elims, ilu_cand; /* ILUTP rows factored, eliminations performed, and
                                working-row entries before dropping (summed over rows) */
  int chunks_L, chunks_U;    /* stream chunks of the triangular solves (>= levels)         */
  int64_t refactors_async;   /* factorisations adopted from the background factor CTA      */
  int64_t async_wait_cycles; /* solver cycles spent waiting for / adopting them            */
  int64_t async_factor_cycles; /* factor-CTA cycles spent factoring (off the solver's path) */
  int factor_set;            /* factor set in use (0 or 1)                                  */
  int async_lag;             /* the refactor_lag in effect (0: in-line refactorisation)     */
  int max_updates;           /* the max_updates in effect                                   */
  int groups_L, groups_U;    /* synchronisation steps of the triangular solves at the last
                                factorisation (groups of levels; = the level counts when the
                                solves are not grouped)                                       */
  int64_t trigger_iterations; /* GMRES iterations until the residual reached trigger_rtol, summed
                                over solves (the paper's iteration count k1 at its tolerance 1e-6) */
  int64_t reorders_skipped;  /* triggers (monitor, non-convergence, slow) that fired while the
                                factors were those of a reorder + refactorisation of the very
                                same matrix (no move accepted since): refactoring it again
                                would reproduce them, so the solve only restarts           */
  int64_t stream_bytes;      /* bytes of the L and U chunk streams at the last factorisation:
                                what one preconditioner apply reads (grouped rows expanded)  */
} vmc_stats;

/* Fill p (host) with the defaults above; VMC_ERR_INVALID for NULL. */
vmc_status vmc_default_params(vmc_solver_params* p);

/* One autotuner trial (see vmc_autotune). */
typedef struct {
  int engine;          /* VMC_ENGINE_PERSISTENT or VMC_ENGINE_STEP                        */
  int block_threads;   /* threads per walker CTA                                          */
  int max_updates;     /* update-chain length before a refactorisation                    */
  int refactor_lag;    /* the lag in effect: > 0 background refactorisation (walker pairs) */
  double ratios_per_s; /* measured determinant ratios per second (0 when the trial failed) */
  int status;          /* vmc_status of the trial                                        */
  int lfil_extra;      /* ILUTP fill limit of the trial (-1: half the average row count)   */
  int trisolve_group;  /* triangular-solve grouping of the trial (1: level by level)       */
} vmc_tune_trial;

/* Autotuner: picks the launch mapping and solver layout for these walkers by timing
 * short trials on the device.  First the ILUTP fill limit lfil_extra: -1 (half the
 * average row count, the paper's), 16, 32 or 48, with the default mapping; then, at the
 * best of those, the mapping: a CTA pair per walker with background refactorisation
 * (when the pairs fit), a CTA per walker (persistent), one launch per step (STEP engine),
 * with 128 or 256 threads per CTA; then max_updates of 32, 64 or 128 for the best of
 * those; then grouped (8 levels) against level-by-level triangular solves (trisolve_group).
 * Each trial creates a context
 * from `params` with the candidate's fields, starts the walkers from `seeds` and
 * `jitter`, makes n_walkers x `steps` moves twice, untimed then timed (proposal width
 * sigma) -- as a budgeted advance with the persistent engine (the batch's throughput),
 * as a partial sweep of `steps` moves per walker with the STEP engine -- and destroys the
 * context.  The mapping and the fill limit do
 * not change the method's results -- only its cost, and the rounding.
 * params (in/out): the base parameters; on return engine, block_threads, max_updates,
 * refactor_lag, lfil_extra and trisolve_group hold the fastest trial's.  trials (nullable): receives up to
 * max_trials trial records, *n_trials (nullable) their number.  stream as in vmc_create.
 * Returns VMC_ERR_INVALID on bad arguments or a DENSE_SM engine, the first failure if
 * every trial fails, else VMC_OK. */
vmc_status vmc_autotune(const vmc_system* systems, int n_walkers, vmc_solver_params* params, const uint64_t* seeds,
                        double jitter, double sigma, int steps, vmc_tune_trial* trials, int max_trials,
                        int* n_trials, void* stream);
/* vmc_autotune from a given state (e.g. an equilibrated one, where the solves are far
 * harder than at the start): xyz (host, walker-major, as vmc_set_positions_all) and the
 * sweep index sweep0; both the untimed and the timed trial sweep start from that state.
 * xyz = NULL: as vmc_autotune (start from seeds and jitter). */
vmc_status vmc_autotune_state(const vmc_system* systems, int n_walkers, vmc_solver_params* params,
                              const uint64_t* seeds, double jitter, const double* xyz, int64_t sweep0, double sigma,
                              int steps, vmc_tune_trial* trials, int max_trials, int* n_trials, void* stream);

/* Create a context for n_walkers walkers; systems[w] is walker w's system
 * (walkers may differ in size: an uneven batch).  systems: host, n_walkers entries,
 * copied.  params: host, copied; NULL means the defaults.  stream: a cudaStream_t (or
 * NULL for the default stream) on which every device operation of the context runs.
 * Allocates all device memory up front.  Positions must be set next
 * (vmc_init_positions or vmc_set_positions).
 * Errors: VMC_ERR_INVALID for a NULL out or systems or n_walkers outside [1, 65535]
 * (then *out is NULL), and for a parameter or a system out of range (the message names
 * it); VMC_ERR_OOM / VMC_ERR_CUDA when device allocation or set-up fails or no usable
 * device is current.  In every case but the first *out still receives the context so
 * that vmc_last_error can describe the failure: release it with vmc_destroy. */
vmc_status vmc_create(const vmc_system* systems, int n_walkers, const vmc_solver_params* params,
                      void* stream, vmc_ctx** out);
/* Free every device allocation of the context and the context itself (device work
 * still queued on its stream completes first).  VMC_ERR_INVALID for NULL. */
vmc_status vmc_destroy(vmc_ctx* ctx);

/* Start walker w at r_i = wrap(Z_i + jitter N(0,1)^3) with normals from
 * Philox4x32-10(key = seeds[w], counter = (0, i, 0, j)), for every walker; then build
 * the Slater matrices, reorder (Sec. 3.1) and factor (Sec. 3.2).  seeds: host,
 * n_walkers entries.  Resets every walker's statistics and status and drops pending
 * ratios.  Errors: VMC_ERR_INVALID (NULL seeds, negative or NaN jitter), VMC_ERR_CUDA,
 * or the first failing walker's status (e.g. VMC_ERR_CAPACITY). */
vmc_status vmc_init_positions(vmc_ctx* ctx, const uint64_t* seeds, double jitter);
/* Set walker w's positions (host, n*3 doubles, particle order; wrapped into the box)
 * and rebuild its matrix, ordering and factorisation; resets that walker's statistics
 * and status.  Errors: VMC_ERR_INVALID (NULL xyz, walker out of range, a non-finite
 * coordinate), VMC_ERR_CUDA, or the walker's failure status. */
vmc_status vmc_set_positions(vmc_ctx* ctx, int walker, const double* xyz);
/* vmc_set_positions for every walker at once (one set-up launch for the batch): xyz is
 * host, walker-major, sum_w n_w*3 doubles (walker w's block starts at 3 (n_0 + ... +
 * n_{w-1})), particle order within a block; wrapped into each walker's box.  Restores a
 * saved batch state (with vmc_set_sweep_count) or starts every walker from given
 * positions.  Resets every walker's statistics and status and drops pending ratios.
 * Errors: VMC_ERR_INVALID (NULL xyz, a non-finite coordinate), VMC_ERR_CUDA, or the
 * first failing walker's status. */
vmc_status vmc_set_positions_all(vmc_ctx* ctx, const double* xyz);
/* Copy walker w's current positions (particle order, in [0, L)) to xyz (host, n*3
 * doubles); synchronises the stream.  VMC_ERR_INVALID for bad arguments. */
vmc_status vmc_get_positions(vmc_ctx* ctx, int walker, double* xyz);
/* Walker w's particle count n (K^3 or 2K^3), or -1 for bad arguments. */
int vmc_walker_n(const vmc_ctx* ctx, int walker);

/* Single move: det(A')/det(A) for moving particle k of walker w to r_new (host, 3
 * doubles; wrapped into the box).  Nothing is committed; the solve is kept so that
 * vmc_accept can commit it.  Sec. 3 Eq. 13.  ratio: host, written on success.
 * Errors: VMC_ERR_INVALID (dense engine, NULL pointers, walker or k out of range, a
 * non-finite coordinate), VMC_ERR_STATE (positions not set), VMC_ERR_NOCONV (the solve
 * did not converge after reorder + restarts; nothing is pending), or the walker's
 * failure status. */
vmc_status vmc_ratio(vmc_ctx* ctx, int walker, int k, const double r_new[3], double* ratio);
/* vmc_ratio plus the quantities of a drift-diffusion step at the proposed position
 * (Sec. 2.2; the same solve: column k of A'^{-1} is A^{-1} e_k / ratio):
 *   grad = grad_{r'} ln|det A'|   (host, 3 doubles; nullable)
 *   lap  = lap_{r'} det A' / det A'   (host; nullable)
 * with grad phi = -2 kappa (r' - Z) phi and lap phi = (4 kappa^2 |r' - Z|^2 - 6 kappa) phi
 * (minimum image).  Accurate to the solve's tolerance; the refinement targets the ratio.
 * The move stays pending for vmc_accept as with vmc_ratio. */
vmc_status vmc_ratio_grad(vmc_ctx* ctx, int walker, int k, const double r_new[3], double* ratio, double grad[3],
                          double* lap);
/* Commit the move of the last vmc_ratio on walker w: replace the Slater row and
 * apply the rank-one preconditioner update (Sec. 3.2 Eq. 17).  VMC_ERR_STATE if
 * no ratio is pending. */
vmc_status vmc_accept(vmc_ctx* ctx, int walker);

/* Metropolis sweeps (Sec. 2.2): every walker moves particles 0..n-1 in order,
 * r' = wrap(r + sigma N(0,1)^3) (counter (sweep, i, 1, j)), accepted iff
 * ratio^2 > U with U from counter (sweep, i, 2, 0), key seeds[w].  Sweep indices
 * continue from the context's sweep counter.  seeds: host, n_walkers entries.  Logs
 * (host, nullable): walker-major, sum_w n_sweeps * n_w entries, walker w's block starting
 * at n_sweeps * (n_0 + ... + n_{w-1}); the device buffers behind them are grown as needed
 * and owned by the context.  Pending ratios are dropped.  Returns after the logs are
 * written.  Errors: VMC_ERR_INVALID (NULL seeds, n_sweeps < 0, negative or NaN sigma),
 * VMC_ERR_STATE (positions not set), VMC_ERR_OOM (log buffers), VMC_ERR_CUDA, or the
 * first failing walker's status. */
vmc_status vmc_sweep(vmc_ctx* ctx, int n_sweeps, double sigma, const uint64_t* seeds,
                     uint8_t* accept_log, double* ratio_log);
/* Same, with device-resident logs (nullable) and no host synchronisation: the call
 * only enqueues work on the context's stream.  seeds_dev and the logs (device, owned by
 * the caller) must stay valid until that work completes; walker failures surface at
 * vmc_synchronize.  Errors at enqueue: VMC_ERR_INVALID, VMC_ERR_STATE, VMC_ERR_OOM (the
 * sweep graph's state), VMC_ERR_CUDA. */
vmc_status vmc_sweep_async(vmc_ctx* ctx, int n_sweeps, double sigma, const uint64_t* seeds_dev,
                           uint8_t* accept_log_dev, double* ratio_log_dev);
/* Budgeted advance (PERSISTENT engine only): the batch makes total_moves Metropolis
 * moves in all, claimed one at a time by the walkers, so that walkers whose solves are
 * cheaper make more of them and no SM idles while the slowest walker finishes a fixed
 * share (the walkers' solve costs differ several-fold).  Every walker continues its own
 * chain from where it stands -- the particle after its last move, or particle 0 of the
 * context's sweep counter after vmc_create / vmc_set_positions(_all) / vmc_sweep --
 * through the particles in order and on into the following sweeps; its moves are the
 * ones full sweeps make (the same proposals, uniforms and factor adoption points), only
 * how many a walker makes in one call depends on timing.  The context's sweep counter is
 * not advanced; vmc_sweep starts every walker at particle 0 of that counter again.  No
 * logs.  seeds_dev: device, n_walkers seeds, valid until the work completes.  Enqueues
 * only; failures surface at vmc_synchronize.  VMC_ERR_INVALID for another engine or bad
 * arguments, VMC_ERR_STATE before positions are set. */
vmc_status vmc_advance_async(vmc_ctx* ctx, int64_t total_moves, double sigma, const uint64_t* seeds_dev);
/* vmc_advance_async with host seeds (copied), waiting for completion; accepts_out (host,
 * n_walkers, nullable) receives every walker's accepted-move count (the statistic). */
vmc_status vmc_advance(vmc_ctx* ctx, int64_t total_moves, double sigma, const uint64_t* seeds,
                       int64_t* accepts_out);
/* Where walker w's chain stands: the next move is particle *particle of sweep *sweep
 * (host outputs; synchronises the stream).  VMC_ERR_INVALID for bad arguments. */
vmc_status vmc_get_progress(vmc_ctx* ctx, int walker, int64_t* sweep, int* particle);
/* Device status check after vmc_sweep_async: synchronises and returns the first
 * walker error. */
vmc_status vmc_synchronize(vmc_ctx* ctx);

/* Kinetic energy of every walker's current configuration (Sec. 4 Eq. 21, read as
 *   E = (1/2n) sum_{p,o} (6 kappa - 4 kappa^2 |r_p - Z_o|^2) A_po (A^{-1})_op ,
 * min-image distances): for each particle p one solve A z = e_p by the engine's
 * preconditioned GMRES (z = column p of A^{-1}), contracted with p's Slater row
 * weighted by the Laplacian factor of each Gaussian, refined in FP64 to the solver's
 * ratio_tol.  energy: host, n_walkers doubles, written before return.  Counts as n
 * solves per walker in the statistics.  VMC_ERR_INVALID with the dense engine,
 * VMC_ERR_STATE before positions are set. */
vmc_status vmc_kinetic_energy(vmc_ctx* ctx, double* energy);

/* Walker w's statistics (host struct, written before return; synchronises the stream).
 * VMC_ERR_INVALID for bad arguments. */
vmc_status vmc_get_stats(vmc_ctx* ctx, int walker, vmc_stats* out);
/* Zero every walker's event counters (proposals, accepts, solves, iterations, reorders,
 * refactorisations), the monitor's max and sum, the histogram, the cycle counts and the
 * algorithmic bytes; the status and the description of the current state (nonzeros,
 * level counts, chain length, factor set) are kept.  Synchronises the stream. */
vmc_status vmc_reset_stats(vmc_ctx* ctx);
/* Text of the most recent failure on ctx (owned by ctx, valid until its next call);
 * "null context" for NULL. */
const char* vmc_last_error(const vmc_ctx* ctx);
/* Sweeps done so far (the sweep counter used for the proposals); -1 for NULL. */
int64_t vmc_sweep_count(const vmc_ctx* ctx);
/* Set the sweep counter (to replay a stretch of a chain); VMC_ERR_INVALID if negative. */
vmc_status vmc_set_sweep_count(vmc_ctx* ctx, int64_t sweeps);

/* ---- inspection (tests) -------------------------------------------------------- */
/* Walker w's reordered Slater matrix A_p = P A Q_0 as dense row-major n*n (host),
 * and the permutations: part_of_row[r] = particle in row r, orb_of_col[c] = orbital
 * in column c. Any pointer may be NULL. */
vmc_status vmc_get_matrix(vmc_ctx* ctx, int walker, double* A_dense, int* part_of_row,
                          int* orb_of_col);
/* Walker w's ILUTP factors of A_p Q = L U as dense row-major n*n (host): L unit lower
 * (diagonal stored as 1), U upper, perm[t] = column of A_p in factor column t. */
vmc_status vmc_get_factors(vmc_ctx* ctx, int walker, double* L_dense, double* U_dense, int* perm);
/* Apply the current preconditioner M (Sec. 3.2 Eq. 18) of walker w to v (host, n,
 * indexed by rows of A_p) giving z (host, n, indexed by columns of A_p). */
vmc_status vmc_apply_preconditioner(vmc_ctx* ctx, int walker, const double* v, double* z);
/* Force a reorder + refactorisation of walker w now (tests). */
vmc_status vmc_refactor(vmc_ctx* ctx, int walker, int reorder);
/* Kernel microbenchmark over all walkers (no synchronisation; the caller times the
 * launch on the context's stream): `reps` back-to-back applications of one hot-path
 * kernel per walker -- which = 0: the L and U level-scheduled triangular solves
 * (Sec. 3.2 Eq. 18 without the update chain), 1: the SpMV y = A_p x in the working
 * precision, 2: the whole preconditioner apply -- on a fixed vector.  The walkers'
 * alg_bytes statistic grows by the algorithmic bytes moved.  Clobbers the walkers'
 * Krylov work vectors (any pending vmc_ratio is dropped). */
vmc_status vmc_kernel_bench(vmc_ctx* ctx, int which, int reps);
/* Failure detection check (tests): launches a kernel that waits on a device barrier
 * phase nothing completes, with the solver's bounded wait (~1 s); returns
 * VMC_ERR_TIMEOUT when the wait gave up and reported it, as every bounded wait in the
 * engine does.  The context stays usable. */
vmc_status vmc_check_wait_timeout(vmc_ctx* ctx);
/* Philox4x32-10 on the device for n counters (host arrays ctr: 4n words, key: 2
 * words, out: 4n words): checks the device generator against its definition. */
vmc_status vmc_philox_device(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n);

/* ---- determinant ratio without device allocation ------------------------------- */
/* The paper has no counterpart to this entry point; it serves callers that cannot
 * call cudaMalloc (a framework that owns all device memory through its own pool,
 * latency-critical code where an allocation's implicit synchronisation is not
 * acceptable, or a process that has already reserved the free memory).
 * vmc_ratio_noalloc computes det(A')/det(A) for moving particle k of ONE walker to
 * r_new, like vmc_create + vmc_set_positions + vmc_ratio with the same parameters,
 * but allocates nothing: the whole walker workspace lives in a fixed device array of
 * vmc_noalloc_capacity() bytes (16 MiB) that every GPU loading this library holds
 * until the process exits.
 *   sys, params : host; params may be NULL (defaults); engine is ignored.
 *   xyz_dev     : device, n*3 doubles, positions in [0, K a) in particle order.
 *   k, r_new    : particle index and its proposed position (host, 3 doubles).
 *   ratio_dev   : device, one double, receives the ratio.
 *   stream      : cudaStream_t or NULL; the call synchronises it before returning.
 * Returns VMC_ERR_CAPACITY when the system's workspace exceeds the fixed array,
 * VMC_ERR_INVALID for bad arguments, other codes as vmc_ratio; the message is in
 * vmc_noalloc_last_error() (per host thread).
 * The array's device address is looked up on the first call made with each device
 * current; make that first call before any stream capture.  Every call reuses and
 * overwrites the same array, so calls that overlap on the GPU (other streams,
 * other host threads) race: serialise them. */
vmc_status vmc_ratio_noalloc(const vmc_system* sys, const vmc_solver_params* params, const double* xyz_dev,
                             int k, const double r_new[3], double* ratio_dev, void* stream);
size_t vmc_noalloc_capacity(void);
const char* vmc_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
