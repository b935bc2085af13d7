/*
 * nbody.h -- C ABI of the GB300 direct-summation gravity library (libnbody.so).
 *
 * The library computes, for every particle i of one system or of each
 * independent cluster of an ensemble, the softened gravitational acceleration
 * and potential
 *
 *     a_i   =  G sum_{j != i} m_j (r_j - r_i) / (|r_j - r_i|^2 + eps^2)^(3/2)
 *     phi_i = -G sum_{j != i} m_j           / (|r_j - r_i|^2 + eps^2)^(1/2)
 *
 * (the force sum of Almerol et al., SC'25 workshops, Sec. 3, divided by m_i,
 * with Plummer softening eps), and advances the system with kick-drift-kick
 * leapfrog in FP64 (the paper keeps all integration in double precision,
 * Sec. 3, mixed-precision paragraph).
 *
 * Two arithmetic modes (chosen per context):
 *   NBODY_F64  -- every pairwise operation in IEEE double.
 *   NBODY_F32C -- positions stay FP64; each tile of particles is re-expressed
 *                 as FP32 offsets from its own centre (the FP32 mean of its
 *                 FP32-rounded positions, held as a float pair whose low part
 *                 is 0: each offset is the FP64 difference from that centre,
 *                 rounded once), pairwise terms run in FP32 (hardware rsqrt)
 *                 with tile-centre differences formed exactly as float pairs,
 *                 the self pair (j == i) is left out before any FP32 sum, each
 *                 particle's per-tile partial sum is folded into a
 *                 Kahan-compensated FP32 accumulator, and the cross-CTA
 *                 reduction, the final scaling by G and the leapfrog run in
 *                 FP64.  This is the paper's mixed-precision split (FP32
 *                 forces, FP64 everything else, Sec. 3).
 *
 * Conventions for every entry point:
 *   * Array layout: positions, velocities and accelerations are
 *     structure-of-arrays double[3][n] (all x, then all y, then all z);
 *     masses and potentials are double[n].  n is the context's n_total and
 *     particle k of cluster c is row cluster_offsets[c] + k.
 *   * Pointers may be device memory (cudaMalloc, torch CUDA tensors) or host
 *     memory (pageable or pinned).  Host arrays are staged through device
 *     buffers owned by the context; when any OUTPUT array is host memory the
 *     call synchronises the stream before it returns, so the values are ready.
 *     All pointers must be 8-byte aligned.
 *   * Ownership: the caller owns every array it passes; the library never
 *     frees or keeps them past the call, except that nbody_step caches a CUDA
 *     graph keyed by the pointer values (a later call with other pointers
 *     captures a new graph).  The context owns its scratch (packed tiles,
 *     partial sums, permutation, work queue, graphs, staging buffers).
 *   * Streams: `stream` is a cudaStream_t (NULL = the legacy default stream).
 *     Work is enqueued on it; only nbody_energy and calls with host outputs
 *     synchronise.
 *   * Errors: every int-returning call returns NBODY_OK (0) or a negative
 *     NBODY_E* code.  An error inside a call leaves the context in a sticky
 *     error state: later calls return NBODY_ESTATE until nbody_destroy.
 *     nbody_last_error_message gives a one-line description.
 *   * A context may be used from one host thread at a time.
 *   * Empty systems (n_total == 0) and empty clusters are valid; calls on them
 *     do nothing and succeed.
 */
#ifndef NBODY_H
#define NBODY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define NBODY_OK 0
#define NBODY_EINVAL (-1)       /* invalid argument or configuration */
#define NBODY_ENOMEM (-2)       /* a device or host allocation failed */
#define NBODY_ECUDA (-3)        /* a CUDA runtime call failed */
#define NBODY_ENONFINITE (-4)   /* NBODY_FLAG_CHECK_FINITE found a NaN/Inf output */
#define NBODY_ETIMEOUT (-5)     /* a bounded device-side wait gave up */
#define NBODY_ESTATE (-6)       /* the context holds an earlier error */
#define NBODY_EUNSUPPORTED (-7) /* no kernel instantiation for the requested tiles */
#define NBODY_ETOOBIG (-8)      /* n exceeds the fixed scratch of nbody_forces_noalloc */

/* arithmetic modes */
#define NBODY_F64 0
#define NBODY_F32C 1

/* configuration flags */
#define NBODY_FLAG_AUTOTUNE 1     /* choose the tile shape at init by timing candidates */
#define NBODY_FLAG_PROFILE 2      /* time every force-kernel launch with CUDA events */
#define NBODY_FLAG_CHECK_FINITE 4 /* verify outputs are finite after each call (syncs) */
#define NBODY_FLAG_NO_GRAPH 8     /* nbody_step launches eagerly instead of graph replay */
#define NBODY_FLAG_TRACE 16       /* F32C block steps: record each step's start and size (nbody_block_trace) */

/*
 * Tile shape of the F32C force kernel.  block = threads per CTA, p = i-particles
 * held in registers by each thread (one CTA owns block*p consecutive packed
 * particles, which also form one tile with its own centre), tj = j-particles
 * staged in shared memory per step, split = number of CTAs that share one
 * i-tile's j-range (their FP64 partial sums are reduced in a fixed order),
 * ctas_per_sm = the resident-CTA target the kernel variant was compiled for
 * (it caps registers per thread).  All zero = choose automatically; zero in
 * split or ctas_per_sm alone = choose that field.  nbody_tiles_supported()
 * lists the compiled (block, p, tj, ctas_per_sm).
 */
typedef struct nbody_tiles {
    int32_t block;
    int32_t p;
    int32_t tj;
    int32_t split;
    int32_t ctas_per_sm;
} nbody_tiles;

typedef struct nbody_config {
    int64_t n_total;                 /* particles over all clusters, 0 <= n_total <= 2^30 */
    int32_t n_clusters;              /* >= 1; clusters never interact */
    int32_t mode;                    /* NBODY_F64 or NBODY_F32C */
    const int64_t *cluster_offsets;  /* host, n_clusters + 1 nondecreasing entries from 0 to
                                        n_total; may be NULL when n_clusters == 1 */
    const double *eps;               /* host, n_clusters softening lengths, each finite, >= 0 */
    double G;                        /* gravitational constant, finite */
    int32_t reorder_every;           /* F32C: re-sort particles along a Morton curve every k
                                        force evaluations (0 = keep the caller's order); in
                                        block steps every k * dt_max of simulated time */
    int32_t flags;                   /* NBODY_FLAG_* */
    nbody_tiles tiles;               /* F32C tile shape; zeros = default or autotuned */
    int64_t max_device_bytes;        /* cap on the device memory the context may hold (its
                                        scratch, staging buffers, tuner and jerk/block-step
                                        state); 0 = no cap.  An allocation that would pass
                                        it is refused before cudaMalloc is called and fails
                                        the call with NBODY_ENOMEM, exactly like a failed
                                        cudaMalloc (sticky in the context) */
} nbody_config;

typedef struct nbody_ctx nbody_ctx;

/*
 * Create a context: validates cfg, allocates the scratch for n_total particles
 * on the current CUDA device, builds the work queue and, with
 * NBODY_FLAG_AUTOTUNE, times the candidate tile shapes (results are cached in
 * the file named by the NBODY_TUNE_CACHE environment variable, if set).
 * `stream` carries the set-up work; the call synchronises it before returning.
 * On failure *out is NULL.
 */
int nbody_init(nbody_ctx **out, const nbody_config *cfg, void *stream);

/* Release everything the context owns (NULL is a no-op).  Synchronises the device. */
void nbody_destroy(nbody_ctx *ctx);

/*
 * Acceleration and potential of every particle (Sec. 3 force sum, softened).
 *   pos  in : double[3][n]   mass in : double[n]
 *   acc  out: double[3][n]   pot  out: double[n], or NULL to skip it
 * pos/mass are only read; acc/pot must not alias them.
 */
int nbody_forces(nbody_ctx *ctx, const double *pos, const double *mass, double *acc, double *pot,
                 void *stream);

/*
 * nsteps >= 0 kick-drift-kick leapfrog steps of size dt (finite, any sign):
 *   v += dt/2 a(x);  x += dt v;  a, phi <- forces(x);  v += dt/2 a(x)
 *   pos, vel in/out: double[3][n]     mass in: double[n]
 *   acc, pot in/out: on entry a(x) and phi(x) at the current positions (from
 *                    nbody_forces or an earlier step); on exit at the final ones
 *   diag out (may be NULL): double[nsteps][n_clusters][9], after each step the
 *                    nbody_energy values of every cluster
 * Steps are replayed from a captured CUDA graph unless NBODY_FLAG_NO_GRAPH.
 */
int nbody_step(nbody_ctx *ctx, double *pos, double *vel, const double *mass, double *acc,
               double *pot, double dt, int32_t nsteps, double *diag, void *stream);

/*
 * Acceleration, jerk (its time derivative) and potential of every particle.
 * The paper's device kernel computes the acceleration together with the jerk
 * (Sec. 3); with r = r_j - r_i, u = v_j - v_i and d2 = |r|^2 + eps^2:
 *     jerk_i = G sum_{j != i} m_j [ u / d2^(3/2) - 3 (r . u) r / d2^(5/2) ]
 *   pos, vel in : double[3][n]     mass in : double[n]
 *   acc, jerk out: double[3][n]    pot  out: double[n], or NULL
 * In NBODY_F32C mode velocities, like positions, are FP32 offsets from a
 * per-tile centre (the FP32 mean of the tile's FP32-rounded values, low part
 * 0); the call uses its own tile geometry (built on first use, shape set by
 * nbody_set_jerk_tiles or chosen from n).
 */
int nbody_forces_jerk(nbody_ctx *ctx, const double *pos, const double *vel, const double *mass,
                      double *acc, double *jerk, double *pot, void *stream);

/*
 * nsteps >= 0 fourth-order Hermite predictor-corrector steps of size dt, one
 * shared step for all particles:
 *   x_p = x + v dt + a dt^2/2 + j dt^3/6,  v_p = v + a dt + j dt^2/2
 *   a1, j1, phi <- nbody_forces_jerk(x_p, v_p)
 *   v <- v + (a + a1) dt/2 + (j - j1) dt^2/12,  x <- x + (v_old + v) dt/2 + (a - a1) dt^2/12
 *   pos, vel, acc, jerk in/out (acc, jerk on entry at the current state, e.g.
 *   from nbody_forces_jerk); pot out (at the predicted positions of the last
 *   step); diag as in nbody_step (W from that pot).  Graph-replayed unless
 *   NBODY_FLAG_NO_GRAPH.
 */
int nbody_step_hermite(nbody_ctx *ctx, double *pos, double *vel, const double *mass, double *acc,
                       double *jerk, double *pot, double dt, int32_t nsteps, double *diag,
                       void *stream);

/*
 * Individual (block) time steps around the Hermite scheme -- the usual partner
 * of a jerk-based integrator (Makino & Aarseth 1992; the paper computes the
 * jerk, Sec. 3, but does not describe its stepping).  Every particle keeps its
 * own time and a power-of-two step; one block step predicts all particles to
 * t_next = min(t_i + dt_i), evaluates acceleration and jerk of the active
 * particles (t_i + dt_i == t_next) against all predicted ones, corrects those
 * and picks their next step by Aarseth's criterion
 *     dt = sqrt(eta (|a| |a''| + |a'|^2) / (|a'| |a'''| + |a''|^2)),
 * halving it until below that value (not below dt_min) or doubling it when
 * allowed (<= dt_max, t_next a multiple of the doubled step).  The schedule
 * (the next block time -- the next multiple of the smallest occupied step --,
 * compaction of the active set, work queue) runs on the device, so block steps
 * are replayed CUDA graphs (eight steps to a graph unless NBODY_FLAG_PROFILE
 * records per-step events); the host checks progress every 16-256 steps.
 * With NBODY_F32C the predicted j-set is packed as FP32 offsets from a frame
 * per centre tile that moves at the tile's mean velocity: each particle's
 * offset from its frame is kept between steps as a float pair and predicted
 * by a short FP32 polynomial; the frames are set again from the FP64 state
 * after every re-sort and at the start of every nbody_block_advance call (the
 * arrays are the caller's and may have changed).  Steps with at most 32 active
 * particles difference close pairs exactly (position offsets as float pairs):
 * FP32-rounded offsets would make a close pair's forces noisy enough for the
 * criterion (its third-derivative term scales as 1/h^3) to shrink its step
 * towards dt_min.  The F32C corrector keeps x, v and the derivative
 * estimates in FP64 and evaluates the criterion in FP32 (it only selects a
 * power of two, from inputs that carry the FP32 pair sums' error), so a
 * decision can differ from the FP64 one where the criterion lies within that
 * error of a power-of-two boundary.  With NBODY_F64 every pair is FP64 and the
 * step decisions equal the FP64 oracle's.
 *
 * nbody_block_start: computes a, jerk, pot at the current state (t = 0) and the
 *   initial steps, the largest power of two <= min(dt_max, eta_s |a|/|a'|),
 *   not below dt_min.  dt_max and dt_min are powers of two with
 *   dt_max / dt_min <= 2^40, and t_end / dt_min <= 2^60 (times are counted in
 *   units of dt_min), and with NBODY_F32C dt_min >= 2^-126 (NBODY_EINVAL
 *   otherwise).  Unless jerk tiles
 *   were set (nbody_set_jerk_tiles) or built by an earlier jerk call, it picks
 *   a tile shape suited to block steps (narrower j-tiles for large N).
 * nbody_block_advance: block steps until every particle reaches t_end (a
 *   multiple of dt_max, so all particles are synchronised there; a batch may
 *   run a few steps past it, which find no active particle and change
 *   nothing); *blocks and
 *   *evals (may be NULL) receive the totals since nbody_block_start.  Pass the
 *   same arrays as to nbody_block_start; acc/jerk/pot hold each particle's last
 *   corrector values (taken at its last predicted state).
 * nbody_block_state: copies every particle's time and step to host arrays.
 * All arrays must be device memory (NBODY_EINVAL otherwise).
 */
int nbody_block_start(nbody_ctx *ctx, const double *pos, const double *vel, const double *mass,
                      double *acc, double *jerk, double *pot, double dt_max, double dt_min,
                      double eta, double eta_s, void *stream);
int nbody_block_advance(nbody_ctx *ctx, double *pos, double *vel, const double *mass, double *acc,
                        double *jerk, double *pot, double t_end, int64_t *blocks, int64_t *evals,
                        void *stream);
int nbody_block_state(nbody_ctx *ctx, double *t_host, double *dt_host, void *stream);

/*
 * With NBODY_FLAG_TRACE (NBODY_F32C block steps): the device records, as each
 * block step's pack starts, the global timer (ns) and the number of particles
 * the previous step moved, in a ring of NBODY_TRACE_CAP records indexed by the
 * step count.  nbody_block_trace copies records first .. first + count - 1 to
 * out (host, 2 * count values: time, count): record k holds the start of step
 * k + 1 (steps counted from 1 as *blocks counts them) and the size of step k,
 * so step k took record k's time minus record k - 1's.  The record after an
 * advance call's last step is its end (the next pack's start, or the call's
 * end); the next call's first step starts from its own record, which replaces
 * it, so read a call's records before the next call.  Requires
 * first + count <= blocks + 1 and count <= NBODY_TRACE_CAP, with the records
 * not yet overwritten (blocks + 1 - first <= NBODY_TRACE_CAP); NBODY_EINVAL
 * otherwise, NBODY_ESTATE without the flag.  Synchronises `stream`.
 */
#define NBODY_TRACE_CAP 65536
int nbody_block_trace(nbody_ctx *ctx, uint64_t *out, int64_t first, int64_t count, void *stream);

/* Tile shape of the acceleration + jerk kernel in use (zeros before its first use or in F64). */
int nbody_get_jerk_tiles(const nbody_ctx *ctx, nbody_tiles *out);

/* Choose the acceleration + jerk kernel's tile shape (rebuilds its geometry). */
int nbody_set_jerk_tiles(nbody_ctx *ctx, const nbody_tiles *tiles);

/*
 * Per-cluster diagnostics, FP64, fixed summation order (bitwise reproducible):
 *   out_host[c*9 + 0..8] = K, W, E, Px, Py, Pz, Lx, Ly, Lz with
 *   K = 1/2 sum m|v|^2, W = 1/2 sum m phi, E = K + W, P = sum m v, L = sum m x cross v.
 * out_host is host memory of n_clusters*9 doubles; the call synchronises `stream`.
 */
int nbody_energy(nbody_ctx *ctx, const double *pos, const double *vel, const double *mass,
                 const double *pot, double *out_host, void *stream);

/* Time the candidate tile shapes now and keep the fastest (see NBODY_FLAG_AUTOTUNE). */
int nbody_tune(nbody_ctx *ctx, void *stream);

/* The tile shape in use (F32C), or zeros in F64 mode. */
int nbody_get_tiles(const nbody_ctx *ctx, nbody_tiles *out);

/*
 * Compiled (block, p, tj, ctas_per_sm) shapes of the F32C kernel.  Writes up to
 * `cap` entries (split = 0) and returns how many exist.
 */
int nbody_tiles_supported(nbody_tiles *out, int cap);

/*
 * With NBODY_FLAG_PROFILE: total device time (ms) of the force-kernel launches
 * since the last reset and their count.  Waits for launches still in flight.
 * reset != 0 clears the totals afterwards.
 */
int nbody_profile_read(nbody_ctx *ctx, double *ms_total, int64_t *launches, int reset);

/* Number of kernels the library has launched on this context (eager and graph nodes). */
int64_t nbody_kernel_launches(const nbody_ctx *ctx);

/*
 * nbody_forces_noalloc -- the F32C force evaluation of ONE system with no
 * memory allocation at all.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory when they need forces
 * (code running inside a memory pool or arena it does not own, loops that must
 * not pay allocation latency, plug-ins in a host process that has already
 * reserved the GPU's memory).  nbody_init allocates a context's scratch with
 * cudaMalloc, so those callers cannot use the other entry points.
 *
 * Instead, the scratch (packed tiles, permutation, work queue, partial sums) is
 * a fixed array of NBODY_NOALLOC_SCRATCH_BYTES compiled into libnbody.so; every
 * GPU that loads the library holds it until the process exits.  The call makes
 * no cudaMalloc, cudaFree or other allocating call.
 *
 *   n          particles, 0 <= n <= NBODY_NOALLOC_MAX_N (larger n: NBODY_ETOOBIG)
 *   pos  in  : device double[3][n]      mass in : device double[n]
 *   acc  out : device double[3][n]      pot  out: device double[n] or NULL
 *   eps, G   : softening length (finite, >= 0) and gravitational constant
 * Host pointers are rejected (NBODY_EINVAL): staging them would need buffers.
 *
 * The result equals nbody_forces on a single-cluster NBODY_F32C context without
 * reordering, using tile shape (128, 2, 256) and a split chosen from n.
 * The work is enqueued on `stream`; the call does not synchronise.
 *
 * The first call on a device looks up the array's device address (once per
 * device, with that device current), so make the first call before any stream
 * capture.  All calls share the one array and it keeps the last call's
 * contents (each call re-initialises what must start from zero): two calls
 * whose work overlaps on the GPU -- e.g. on different streams without ordering
 * -- race and corrupt each other's results.  Serialise them.
 */
#define NBODY_NOALLOC_MAX_N 262144
#define NBODY_NOALLOC_SCRATCH_BYTES 10297856
int nbody_forces_noalloc(int64_t n, const double *pos, const double *mass, double eps, double G,
                         double *acc, double *pot, void *stream);

/* Static description of a status code. */
const char *nbody_strerror(int status);

/* One-line description of the context's last error ("" if none). */
const char *nbody_last_error_message(const nbody_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* NBODY_H */
