/*
 * mc.h -- C ABI of libmc, a GB300 (sm_103a) library for history-based Monte
 * Carlo particle transport in which every particle history owns one LCG
 * stream, seeded either by hashing (the method of Cuneo & Variansyah, "An
 * Alternative to Stride-Based RNG for Monte Carlo Transport", arXiv
 * 2403.06362) or by striding with Brown's skip-ahead (the baseline the
 * paper compares against).
 *
 * Conventions shared by every entry point
 *   - Pointers named d_* are DEVICE pointers owned by the caller; h_* are
 *     host pointers owned by the caller.  The library never frees caller
 *     memory and never keeps a caller pointer after a call returns.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device work is enqueued on it and the call returns without
 *     waiting, except where a call says it synchronises.
 *   - Every call returns an int status: MC_OK (0) or a negative MC_ERR_*.
 *     mc_last_error() gives a message for the calling thread's last error.
 *     Argument errors are detected on the host before anything is enqueued.
 *   - LCG states are m-bit integers stored in uint64_t (high bits zero).
 *   - A "uniform" is u = floor(X / 2^(m-53)) * 2^-53 in [0,1) as an IEEE
 *     double (for m < 53: X * 2^-m), taken from the state AFTER each step:
 *     the seed itself is never an output (Section 2, Eq. 1: the next state
 *     "also serves as the output").
 *   - Every call is bit-reproducible: results depend on the inputs only,
 *     never on launch shape, schedule or timing.
 */
#ifndef MC_H
#define MC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define MC_API __attribute__((visibility("default")))
#else
#define MC_API
#endif

/* ------------------------------------------------------------------ status */
enum {
    MC_OK = 0,
    MC_ERR_ARG = -1,       /* invalid argument (checked on the host)          */
    MC_ERR_CUDA = -2,      /* a CUDA runtime call failed                      */
    MC_ERR_OVERFLOW = -3,  /* a tally bin left the int64 headroom (2^62)      */
    MC_ERR_EVENT_CAP = -4, /* some history hit the per-history event cap      */
    MC_ERR_TIMEOUT = -5,   /* a bounded device wait gave up                   */
    MC_ERR_CAPACITY = -6,  /* a bounded device buffer (secondary bank) filled */
    MC_ERR_STATE = -7      /* call out of order (e.g. no context)             */
};

/* Thread-local message describing the last failing call of this thread. */
MC_API const char* mc_last_error(void);

/* ------------------------------------------------------------- LCG (Eq. 1)
 * X_{n+1} = (g X_n + c) mod 2^m, 1 <= m <= 64.  g must be odd (an even g
 * has no skip-ahead inverse and no full period).  The workload parameters
 * are m = 63, g = 2806196910506780709, c = 1 (MCNP5's 63-bit generator,
 * full period since c is odd and g = 1 mod 4). */
typedef struct {
    uint32_t m;
    uint32_t reserved; /* must be 0 */
    uint64_t g;
    uint64_t c;
} mc_lcg;

/* --------------------------------------------------------------- context
 * A context owns the library's scratch memory on one device: work-queue
 * tickets, the status word, the device copy of the problem list and the
 * particle banks of the event-based schedule.  Create it once, outside any
 * timed or captured region; it allocates device memory.  A context may be
 * used from one host thread at a time. */
typedef struct mc_ctx mc_ctx;

/* Creates a context on `device` (the device is made current).  *out is set
 * on success.  Errors: MC_ERR_ARG (out NULL), MC_ERR_CUDA. */
MC_API int mc_ctx_create(mc_ctx** out, int device);
/* Frees the context and its device memory (synchronises the device). */
MC_API void mc_ctx_destroy(mc_ctx* ctx);

/* Bounds on the waits of mc_transport_run under this context (failure
 * detection; the paper has no counterpart).  Each bound turns a wait that
 * would not end into an error status instead of a hang; the defaults are
 * far above anything a valid run needs, and lowering them exists to test
 * the give-up paths.  Every field is taken literally (0 is a bound of 0).
 *   pool_lock_attempts  slab history kernel: attempts a warp makes at its
 *                       block's compaction-pool lock before it gives up
 *                       (default 2^20).  A warp that gives up skips the
 *                       hand-over; one that is leaving counts what the pool
 *                       may still hold in MC_C_DROPPED, which mc_tally_read
 *                       reports as MC_ERR_CAPACITY.  0: no warp ever takes
 *                       the lock, so no particle moves (tallies unchanged).
 *   box_generations     generations of weight-window children the host
 *                       follows before MC_ERR_TIMEOUT (default 10000).
 *   pulse_generations   generations of overflowed pulse secondaries (hash
 *                       modes) before MC_ERR_TIMEOUT (default 100000).
 *   event_iterations    iterations of the event-based schedules (slab, and
 *                       box per generation) before MC_ERR_TIMEOUT; rounded
 *                       up to whole batches of iterations.  UINT64_MAX (the
 *                       default) derives the bound from the event cap and
 *                       the history count.
 * A run that gave up leaves the tally partial; the context stays usable. */
typedef struct {
    uint32_t pool_lock_attempts;
    uint32_t box_generations;
    uint32_t pulse_generations;
    uint32_t reserved; /* must be 0 */
    uint64_t event_iterations;
} mc_limits;

/* Sets the context's bounds (NULL restores the defaults) or reads them.
 * Errors: MC_ERR_ARG (ctx NULL, reserved != 0, out NULL). */
MC_API int mc_ctx_set_limits(mc_ctx* ctx, const mc_limits* limits);
MC_API int mc_ctx_get_limits(const mc_ctx* ctx, mc_limits* out);

/* ---------------------------------------------------------- hash seeding
 * Section 4, Listing 1 and Eq. (3): d_states[i] = hash(key_begin + i,
 * parent_seed) mod 2^m, where hash is the modified murmur_hash64a of
 * Listing 1 (64-bit key and seed, wrapping 64-bit products).  For the
 * hierarchical seeds of Eq. (4) pass parent_seed = hash(i, s) (see
 * mc_hash64).  d_states: uint64_t[count], any alignment of 8 bytes; written
 * with coalesced 16-byte stores where aligned.  count = 0 is a no-op.
 * Errors: MC_ERR_ARG (ctx/lcg/d_states NULL with count > 0, bad lcg). */
MC_API int mc_seed_hash(mc_ctx* ctx, const mc_lcg* lcg, uint64_t parent_seed, uint64_t key_begin,
                        uint64_t count, uint64_t* d_states, void* stream);

/* -------------------------------------------------------- stride seeding
 * Section 3, Eq. (2): d_states[i] = X_{Q*(id_begin+i)}, the state reached
 * from X_0 = x0 after Q*(id_begin+i) LCG steps (unit k gets X_{Qk}; unit 0
 * gets x0 itself).  Computed by Brown's binary skip-ahead, evaluated on the
 * device; the step count is taken mod 2^64, which is exact because the
 * affine map of 2^64 steps is the identity mod 2^64 for odd g.
 * Errors: as mc_seed_hash; stride_q = 0 is allowed (all states = x0). */
MC_API int mc_seed_stride(mc_ctx* ctx, const mc_lcg* lcg, uint64_t x0, uint64_t stride_q,
                          uint64_t id_begin, uint64_t count, uint64_t* d_states, void* stream);

/* ----------------------------------------------------------------- draws
 * Advances n_streams streams by `draws` steps each (Eq. 1) and reports the
 * uniforms.  Draw j of stream i is the uniform of the stream's (j+1)-th
 * state.
 *   seed      NULL: d_states holds the n_streams input states and is
 *             overwritten with the final states.
 *             non-NULL: the streams are seeded in the kernel, stream i with
 *             the seed of unit id_begin + i (fused seeding + draws); d_states
 *             (nullable) receives the final states.
 *   d_u       nullable; double[draws][n_streams] (draw-major: d_u[j*n+i]).
 *   d_digest  nullable; uint64_t[n_streams]; the wrapping 64-bit sum of the
 *             IEEE-754 bit patterns of the stream's draws (lets a caller
 *             consume every draw without storing it).
 * Errors: MC_ERR_ARG (bad lcg or seed spec, d_states NULL without seed). */
typedef struct {
    uint32_t mode;     /* MC_SEED_HASH, MC_SEED_STRIDE or MC_SEED_HASH_HIER */
    uint32_t reserved; /* must be 0 */
    uint64_t seed;     /* hash: global seed s; stride: X_0 */
    uint64_t stride_q; /* stride: Q */
    uint64_t key;      /* hierarchical hash: key i of hash(j, hash(i, s)) */
} mc_seed_spec;

MC_API int mc_lcg_draw(mc_ctx* ctx, const mc_lcg* lcg, const mc_seed_spec* seed, uint64_t id_begin,
                       uint64_t* d_states, uint64_t n_streams, uint32_t draws, double* d_u,
                       uint64_t* d_digest, void* stream);

/* mc_lcg_draw on HOST buffers (Section 2, Eq. 1; seeds by Eqs. 2-4): the
 * same streams, draws, final states and digests, for a caller that holds
 * its inputs and wants its results in host memory.
 *   seed      as for mc_lcg_draw; NULL: h_states holds the input states.
 *   h_states  nullable with a seed (then no final states are returned);
 *             host uint64_t[n_streams], in/out without a seed.
 *   h_digest  nullable host uint64_t[n_streams].  At least one of h_states
 *             and h_digest is required.
 * The range is processed in slices of 2^22 streams through two device slots
 * owned by the context (128 MiB, allocated on the first call): the draw
 * kernel of one slice runs on `stream` while a private copy stream returns
 * the previous slice.  Page-locked host buffers (cudaHostAlloc) let the
 * copies overlap the kernels; pageable ones work, serialised.  The call
 * returns when every result is in host memory.  Not for use inside stream
 * capture.  Errors: as mc_lcg_draw, MC_ERR_ARG without an output. */
MC_API int mc_lcg_draw_host(mc_ctx* ctx, const mc_lcg* lcg, const mc_seed_spec* seed, uint64_t id_begin,
                            uint64_t* h_states, uint64_t n_streams, uint32_t draws, uint64_t* h_digest,
                            void* stream);

/* --------------------------------------------------------------- transport
 * History-based (or event-based) one-speed transport in a slab, or
 * multigroup transport in a two-region box; every source history owns one
 * LCG stream seeded by hash or stride, and secondaries created by splitting
 * are seeded on demand by S_c = hash(k, S_p) (Section 4, Eq. 5).
 * Flux tallies are track-length estimates accumulated as int64 fixed point
 * (scale 2^32, one llrint per contribution), so totals are independent of
 * scheduling and bit-identical across launch shapes and schedules. */
enum { MC_SEED_HASH = 0, MC_SEED_STRIDE = 1, MC_SEED_HASH_HIER = 2 };
enum { MC_SRC_ISOTROPIC = 0, MC_SRC_BEAM = 1 };
enum { MC_GEOM_SLAB = 0, MC_GEOM_BOX = 1, MC_GEOM_PULSE = 2 };
enum { MC_FP64 = 0, MC_FP32_GUARDED = 1 };
enum { MC_SCHED_HISTORY = 0, MC_SCHED_EVENT = 1, MC_SCHED_AUTO = 2 };

/* Box problem data (geometry MC_GEOM_BOX); host memory, read during the call. */
#define MC_BOX_MAX_GROUPS 8
#define MC_BOX_MAX_MESH 1024
typedef struct {
    double side;                      /* cube [0,side]^3                           */
    double inner_lo, inner_hi;        /* inner region [inner_lo,inner_hi]^3        */
    double sigma_t[2];                /* per region: 0 = outer, 1 = inner          */
    double c[2];                      /* scattering ratio per region               */
    double ww_low[2], ww_high[2], ww_survive[2]; /* weight window per region       */
    double scatter_cdf[2][MC_BOX_MAX_GROUPS][MC_BOX_MAX_GROUPS]; /* [r][g][g'] CDF */
    uint32_t n_groups;
    uint32_t mesh;                    /* cells per axis (<= MC_BOX_MAX_MESH)        */
    uint32_t max_split;               /* cap on n of one split                     */
    uint32_t reserved;
} mc_box_spec;

/* Pulse problem data (geometry MC_GEOM_PULSE; Section 5's supercritical,
 * time-dependent test): a pulse at t = x = 0 in an infinite homogeneous
 * medium (speed 1), collisions scatter with probability c into
 * floor(nu + u) outgoing particles (k = c * nu), census at t_end; the
 * collision-estimator flux over [-x_half, x_half] is tallied in unit time
 * bins [j, j+1), j < n_time_bins, per (repetition, batch).  Secondaries get
 * hash seeds S_c = hash(k, S_p) (Eq. 5) unless seeding is MC_SEED_STRIDE, in
 * which case a history's secondaries draw from its one stream, depth-first.
 * Histories: n_reps * n_batches * per_batch; history g belongs to rep
 * g / (n_batches * per_batch) and batch (g / per_batch) % n_batches;
 * MC_SEED_HASH_HIER seeds it with hash(particle, hash(batch, hash(rep, s))).
 *
 * Census phases (n_census >= 2; hash seeding only): time is cut into
 * n_census equal phases, T_p = t_end p / n_census.  A particle reaching
 * T_p < t_end is banked with its stream, direction and weight; at the end
 * of each phase every (rep, batch) group's bank is population-controlled
 * back toward pc_target particles (0 = per_batch): with W the exact sum of
 * llrint(w 2^32) over the group's bank, particle i gets
 * n_i = floor(w_i pc_target / (W 2^-32) + xi_i) copies of weight
 * W 2^-32 / pc_target, where xi_i = (hash(2^63 + p, S_i) >> 11) 2^-53 is a
 * one-off hashed value of the particle's state S_i (Section 4).  Copy 0
 * continues the particle's stream, copy c >= 1 gets hash(c - 1, S_i) (Eq. 5).
 * No decision depends on the order of the bank, so results are bit-identical
 * in any schedule.  The history range must cover whole groups; per-history
 * outputs and stride exceedance are not produced in this mode; counters add
 * MC_C_BANKED (banked particles), MC_C_SPLITS (copies beyond the first) and
 * MC_C_ROULETTE_KILLS (banked particles given no copy).  The two particle
 * banks (48 bytes per particle, sized from the expected population) belong
 * to the context; a full bank is reported as MC_ERR_CAPACITY by
 * mc_tally_read. */
typedef struct {
    double c, nu, t_end, x_half, sigma_t;
    uint32_t n_reps, n_batches, per_batch, n_time_bins;
    uint32_t n_census;  /* phases; 0 or 1 = none                             */
    uint32_t pc_target; /* population per group after a control; 0 = per_batch */
} mc_pulse_spec;

typedef struct {
    uint32_t geometry;    /* MC_GEOM_SLAB, MC_GEOM_BOX or MC_GEOM_PULSE            */
    uint32_t source;      /* MC_SRC_ISOTROPIC (uniform in the slab/box) or BEAM   */
    uint32_t seeding;     /* MC_SEED_HASH, MC_SEED_STRIDE, MC_SEED_HASH_HIER       */
    uint32_t n_bins;      /* slab: equal-width bins over [0,L]; box: mesh^3        */
    uint32_t n_batches;   /* contiguous history-id batches (>= 1)                  */
    uint32_t reserved;
    double L;             /* slab thickness                                        */
    double sigma_t;       /* slab total cross section                              */
    double c;             /* slab scattering ratio                                 */
    uint64_t n_histories; /* source histories, local ids 0..n-1                    */
    uint64_t seed;        /* hash: global seed s; stride: X_0                      */
    uint64_t stride_q;    /* stride Q (also the nominal stride for exceedance)     */
    uint64_t id_offset;   /* stride: unit index of local history 0                 */
    uint64_t key;         /* hierarchical hash key i                               */
    uint64_t tally_offset;/* first int64 slot of this problem: [batch][bin]        */
    const mc_box_spec* box; /* geometry MC_GEOM_BOX only                           */
    const mc_pulse_spec* pulse; /* geometry MC_GEOM_PULSE only: n_bins = n_time_bins, */
                            /* n_batches = n_reps * n_batches (one call, one problem) */
} mc_problem;

typedef struct {
    uint32_t schedule;      /* MC_SCHED_HISTORY, MC_SCHED_EVENT, MC_SCHED_AUTO     */
                            /* (AUTO: the mc_autotune choice, cached per shape)   */
    uint32_t precision;     /* MC_FP64 or MC_FP32_GUARDED (flight and geometry)   */
    uint32_t block;         /* threads per block; 0 = library default             */
    uint32_t chunk;         /* histories a warp takes per ticket grab; 0 = default */
    uint32_t blocks_per_sm; /* 0 = from the occupancy calculator                  */
    uint32_t use_graph;     /* 1 = capture the launch sequence once and replay    */
    uint32_t accumulate;    /* 0 = zero tallies and counts first; 1 = add to them */
    uint32_t tally_mode;    /* 0 = auto, 1 = stage all slots in shared memory,    */
                            /* 2 = global atomics only (results are identical)    */
    uint64_t event_cap;     /* per-history flight cap; 0 = 2^40                   */
    uint64_t range_begin;   /* run only global histories [begin,end) of the       */
    uint64_t range_end;     /* concatenated problems; end 0 = all                 */
    uint32_t stack_depth;   /* pulse problem: pending secondaries a lane keeps    */
                            /* (1..256, 0 = 256); in hash modes the rest wait in  */
                            /* a device overflow bank processed after the launch  */
                            /* (their streams depend only on their seeds, Eq. 5); */
                            /* stride mode counts them in MC_C_DROPPED            */
    uint32_t tally_atomics; /* history-schedule kernels (slab, box, pulse, census  */
                            /* phases): 0 = library default (1), 1 = one atomic   */
                            /* per lane and contribution, 2 = warp-aggregated:    */
                            /* the lanes adding to one slot together combine      */
                            /* their values and one lane adds the sum.  The bits  */
                            /* are the same either way; event schedules use 1.    */
} mc_run_config;

/* Counter block per problem: uint64_t[MC_NCOUNT], exact integers. */
enum {
    MC_C_SOURCE = 0, MC_C_FLIGHTS, MC_C_COLLISIONS, MC_C_ABSORPTIONS, MC_C_SCATTERS,
    MC_C_LEAK_LO, MC_C_LEAK_HI, MC_C_DRAWS, MC_C_EXCEED_HIST, MC_C_EXCEED_DRAWS,
    MC_C_SPLITS, MC_C_ROULETTE_KILLS, MC_C_CAPPED, MC_C_MAX_DRAWS, MC_C_CHILDREN,
    MC_C_DROPPED, /* secondaries lost to a full bounded stack (MC_ERR_CAPACITY) */
    MC_C_BANKED,  /* pulse census phases: particles banked at an intermediate census */
    MC_NCOUNT
};

typedef struct {
    int64_t* d_bins;        /* device int64[n_slots], fixed point 2^-32         */
    uint64_t n_slots;
    uint64_t* d_counts;     /* device uint64[n_problems][MC_NCOUNT]             */
    uint64_t* d_hist_state; /* nullable device uint64[total histories]: final   */
    uint64_t* d_hist_draws; /* state / draw count per source history, indexed   */
                            /* by global history index (problem prefix + id)    */
} mc_tally;

/* Runs every history of the n_problems problems (or config->range) and
 * accumulates track-length tallies and counters.  Problems and the box
 * spec are host memory read during the call (copied to the context).
 * The call enqueues work on `stream` and returns; the device status word
 * is checked by mc_tally_read.  Errors: MC_ERR_ARG (bad problem: L, sigma_t
 * <= 0, c outside [0,1], n_bins or n_batches 0, slots outside the tally),
 * MC_ERR_CUDA. */
MC_API int mc_transport_run(mc_ctx* ctx, const mc_lcg* lcg, const mc_problem* problems,
                            uint32_t n_problems, const mc_run_config* config, const mc_tally* tally,
                            void* stream);

/* Launch-shape autotuner for mc_transport_run (schedule MC_SCHED_AUTO calls
 * it on the first run of each workload shape and caches the answer in the
 * context).  Times every candidate -- history schedule with block 128/256/512
 * and chunks of 1/4, 1 and 4 times the default, and the event schedule as a
 * captured graph -- on a sample of the histories (all of them up to 2^17,
 * else max(2^17, 1/4) from the middle of the list), writing only into a
 * context-owned scratch tally;
 * the caller's tally is not touched.  *best receives `base` with schedule,
 * block, chunk and use_graph replaced by the fastest candidate; *best_ms
 * (nullable) its time on the sample.  Results never depend on the choice:
 * tallies are bit-identical across all candidates.  Synchronises `stream`.
 * Errors: as mc_transport_run. */
MC_API int mc_autotune(mc_ctx* ctx, const mc_lcg* lcg, const mc_problem* problems, uint32_t n_problems,
                       const mc_run_config* base, const mc_tally* tally, mc_run_config* best, float* best_ms,
                       void* stream);

/* The slab transport of mc_transport_run for callers that cannot allocate
 * device memory (the paper has no counterpart; this is a deployment aid).
 * mc_transport_run needs an mc_ctx, and creating one calls cudaMalloc.  Code
 * whose device memory belongs to another allocator (a framework's caching
 * allocator, a fixed pool that accounts for every byte) and code that must
 * not grow its footprint or take cudaMalloc's implicit synchronisation after
 * start-up cannot make that call.  This entry point allocates nothing: its
 * scratch (work ticket and device problem list) is one fixed __device__
 * array inside libmc, about 41 KiB, present on every device that loads the
 * library until the process exits.
 *   - Slab problems only, at most 256 per call, the history-based schedule
 *     only (box or pulse problems, more problems and MC_SCHED_EVENT are
 *     MC_ERR_ARG, each with its own message); every other argument is
 *     checked as by mc_transport_run, with the same errors.
 *   - The caller still owns and passes the tally buffers; the results are
 *     the same bits as mc_transport_run's.  Launch shape: the same default
 *     block and chunk; launches of several problems compute bin edges on the
 *     fly instead of reading per-problem edge tables (which would need
 *     scratch growing with the bin count), so they can run slower.
 *   - The first call on a device looks up the array's device address (with
 *     that device current); make it before any stream capture starts.  The
 *     address is kept for the life of the process: resetting the device
 *     after the first call is not supported.
 *   - All calls share the array, which keeps the last call's contents (each
 *     call rewrites the problem list and zeroes the ticket first): calls
 *     whose GPU work overlaps (other streams, other host threads) race and
 *     must be serialised. */
MC_API int mc_transport_run_static(const mc_lcg* lcg, const mc_problem* problems, uint32_t n_problems,
                                   const mc_run_config* config, const mc_tally* tally, void* stream);

/* Reads problem `problem`'s tally back (synchronises `stream`).
 *   h_flux      double[n_bins]: flux per source history and unit volume,
 *               phi_b = sum_b * 2^-32 / (N * V_b), over all batches.
 *   h_rel_err   nullable double[n_bins]: relative standard error of phi_b
 *               from the batch means (0 when n_batches < 2).
 *   h_batch     nullable double[n_batches][n_bins]: phi per batch.
 *   h_raw       nullable int64_t[n_batches][n_bins]: raw fixed point.
 *   h_counts    nullable uint64_t[MC_NCOUNT].
 * Errors: MC_ERR_ARG, MC_ERR_CUDA, MC_ERR_OVERFLOW (|bin| >= 2^62),
 * MC_ERR_EVENT_CAP (a history was capped), MC_ERR_CAPACITY. */
MC_API int mc_tally_read(mc_ctx* ctx, const mc_problem* problems, uint32_t problem,
                         const mc_tally* tally, double* h_flux, double* h_rel_err, double* h_batch,
                         int64_t* h_raw, uint64_t* h_counts, void* stream);

/* ---------------------------------------------------------- host helpers */

/* Listing 1 on the host: hash(k, s) as a full 64-bit value (e.g. the parent
 * seed hash(i, s) of Eq. 4). */
MC_API uint64_t mc_hash64(uint64_t k, uint64_t s);

/* Diagnostics of the fp64 flight logarithm (no counterpart in the paper):
 * the fp64 transport samples d = -ln(1 - u) / Sigma_t with a table-driven
 * logarithm (Tang's method) that costs half the fp64 instructions of the
 * CUDA library's.  mc_log1m evaluates it on the host (same code, same bits as
 * the device); mc_log1m_device writes d_out[i] = ln(1 - d_u[i]) on the device
 * with that logarithm (which = 0) or with the CUDA library's log (which = 1).
 * u in [0, 1), a multiple of 2^-53.  Errors: MC_ERR_ARG, MC_ERR_CUDA. */
MC_API double mc_log1m(double u);
MC_API int mc_log1m_device(const double* d_u, double* d_out, uint64_t n, int which, void* stream);

/* Diagnostics of the fp64 steps the transport computes on the integer pipes
 * (no counterpart in the paper): mc_recip_rn(y) is 1/y rounded to nearest
 * even, exactly as IEEE division: a table of 2^63/F (F the left end of the
 * mantissa's cell among 1024, the flight logarithm's table), 1/(1 + r)
 * through r^5 by Horner's rule on non-negative fixed point, an exact
 * remainder check and the rounding; IEEE division for zero, subnormal or
 * huge operands (host evaluation of the device code);
 * mc_recip_rn_device writes d_out[i] = 1/d_y[i] with it (which = 0) or with
 * the CUDA division (which = 1); mc_two_u_minus_1(n) is 2u - 1 for the
 * uniform u = n 2^-53 (n < 2^53; 0 otherwise).  Errors: MC_ERR_ARG,
 * MC_ERR_CUDA. */
MC_API double mc_recip_rn(double y);
MC_API double mc_two_u_minus_1(uint64_t n);
/* llrint(v) for 0 <= v < 2^62; a < b for non-NaN doubles (1 or 0); RN(j h)
 * for 0 <= j < 2^11 and a normal h > 0 with a normal product. */
MC_API long long mc_llrint_nonneg(double v);
MC_API int mc_d_lt(double a, double b);
MC_API double mc_mul_small(uint32_t j, double h);
MC_API int mc_recip_rn_device(const double* d_y, double* d_out, uint64_t n, int which, void* stream);

/* Section 5 normality procedure on host data x[n_batches][n_points]: the
 * normalised deviations z = (x - mean)/sd per point (sd with n-1) and the
 * Shapiro-Wilk W and p-value of each point's batch values (Royston's
 * approximation, 3 <= n_batches <= 5000).  z, w, p nullable.
 * Errors: MC_ERR_ARG (n_batches outside [3,5000]; a point with zero spread
 * gets W = p = NaN and the call returns MC_ERR_ARG after filling the rest). */
MC_API int mc_normality(const double* h_x, uint32_t n_batches, uint32_t n_points, double* h_z,
                        double* h_w, double* h_p);

#ifdef __cplusplus
}
#endif
#endif /* MC_H */
