/*
 * tr.h -- C ABI of the GB300-native event-based Monte Carlo transport library.
 *
 * The library advances neutron histories event by event on one GPU and
 * regroups ("remaps") particles between events so that every warp executes a
 * single event type: thread-data remapping, the event-based approach of
 * Cuneo, Morgan, Variansyah, Niemeyer (M&C 2025), Sec. 2.  Two remapping
 * schemes are provided: stack-based (Sec. 3.1) and asynchronous (Sec. 3.2),
 * each with the monolithic ("step" = one history-loop iteration) or the
 * decomposed (step / collision / surface crossing) task scheme of Sec. 4.
 *
 * Conventions shared by every entry point:
 *  - All arguments are plain C types.  Host pointers are read during the call
 *    only and never retained; the library copies what it needs.
 *  - Every function returns a tr_status.  No C++ exception crosses this
 *    boundary, the library never aborts and no device code traps.  On any
 *    status other than TR_OK, tr_last_error() returns a one-line message for
 *    the calling thread.
 *  - Device memory comes from the allocator callbacks of tr_device_ctx (or
 *    cudaMallocAsync/cudaFreeAsync on the context stream when they are NULL)
 *    and all work is enqueued on the context stream.  Functions that return
 *    results on the host synchronise that stream before returning.
 *  - Floating point: IEEE binary64 everywhere; no implicit FMA contraction,
 *    fused multiply-adds only where the arithmetic contract writes them.
 */
#ifndef TR_H
#define TR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TR_OK = 0,
    TR_ERR_INVALID = 1,   /* malformed description or options */
    TR_ERR_NOMEM = 2,     /* allocation failed */
    TR_ERR_CAPACITY = 3,  /* a particle queue, link arena or fission bank overflowed */
    TR_ERR_TIMEOUT = 4,   /* a bounded device spin-wait gave up (max_spin) */
    TR_ERR_CUDA = 5,      /* a CUDA runtime call failed */
    TR_ERR_STATE = 6      /* call order violated (e.g. no prior forward run) */
} tr_status;

/* Event / final-state codes, the event vocabulary of Sec. 4. */
enum {
    TR_EV_SOURCE = 0, TR_EV_SCATTER = 1, TR_EV_ABSORB = 2, TR_EV_SURF_INTERNAL = 3,
    TR_EV_SURF_REFLECT = 4, TR_EV_LEAK = 5, TR_EV_CUTOFF = 6, TR_EV_MAXEV = 7
};

enum { TR_BC_VACUUM = 0, TR_BC_REFLECT = 1 };
enum { TR_XS_MG = 0, TR_XS_CE = 1 };
enum { TR_SRC_POINT = 0, TR_SRC_BOX = 1, TR_SRC_PINS = 2 };
/* Remapping scheme: stack-based (Sec. 3.1) or asynchronous (Sec. 3.2). */
enum { TR_SCHEME_STACK = 0, TR_SCHEME_ASYNC = 1 };
/* Task decomposition (Sec. 4): one "step" event; step / collision / surface;
 * or those three plus a cross-section lookup event of its own (one of the
 * alternate decompositions Sec. 5.2 points to), whose values travel with the
 * particle to the step and collision that follow.  STREAM (asynchronous
 * scheme only) is another alternate decomposition: steps and surface
 * crossings run inline, up to remap_every steps, and only collisions are
 * deferred to a queue of their own.  The lookup event does not count as an
 * event: all four give the same histories. */
enum { TR_DECOMP_MONO = 0, TR_DECOMP_SPLIT = 1, TR_DECOMP_SPLIT_LOOKUP = 2, TR_DECOMP_STREAM = 3 };

/* Rectilinear grid of cells; each cell may hold one z-aligned cylinder
 * ("pin") of radius pin_radius centred in its x-y box.  Planes are ascending;
 * the outermost z planes may be -inf/+inf (unbounded).  Arrays are row-major
 * [nz][ny][nx].  pin_material < 0 (or a NULL array) means no pin. */
typedef struct {
    int32_t nx, ny, nz;                 /* 1 .. 1023 each */
    const double *x_planes;             /* nx + 1 */
    const double *y_planes;             /* ny + 1 */
    const double *z_planes;             /* nz + 1 */
    int32_t bc[6];                      /* faces x-, x+, y-, y+, z-, z+ */
    const int32_t *cell_material;       /* [nz][ny][nx] */
    const int32_t *pin_material;        /* [nz][ny][nx] or NULL */
    double pin_radius;
} tr_geometry_desc;

/* Cross sections.  Multigroup: sigma_t[m][g], sigma_s[m][g][g'] (from g to
 * g'), nu_sigma_f[m][g], chi[m][g].  Continuous energy: per nuclide an
 * ascending energy grid (eV) with elastic, capture and fission cross sections
 * (barn) per point, rows concatenated over nuclides (nuc_offset[n]..
 * nuc_offset[n+1]); target mass ratio A per nuclide; number densities
 * density[m][n] (atoms / barn cm).  Histories below energy_cutoff end. */
typedef struct {
    int32_t kind;                       /* TR_XS_MG or TR_XS_CE */
    int32_t n_materials;                /* 1 .. 256 */
    int32_t n_groups;                   /* MG: 1 .. 128 */
    const double *sigma_t, *sigma_s, *nu_sigma_f, *chi;
    int32_t n_nuclides;                 /* CE: 1 .. 16 */
    const int64_t *nuc_offset;          /* n_nuclides + 1 */
    const double *nuc_energy;           /* nuc_offset[n_nuclides] */
    const double *nuc_sigma;            /* [row][3] elastic, capture, fission */
    const double *nuc_awr;              /* n_nuclides */
    const double *density;              /* [n_materials][n_nuclides] */
    double energy_cutoff;
    const double *inv_velocity;         /* MG: [n_groups] inverse speeds (s/cm), needed by timed problems */
} tr_xs_desc;

/* Source (the make_work entry point of Sec. 3).  POINT: fixed position,
 * isotropic unless `isotropic` is 0 (then `direction`).  BOX: uniform in
 * [lo, hi].  PINS: uniform in [lo, hi] restricted by rejection to pins whose
 * material has source_material[m] != 0.  Multigroup group: `group`, or chi of
 * the birth material when group < 0.  CE energy: tabulated inverse CDF
 * (cdf_energy, cdf_prob with n_cdf points) or `energy` when n_cdf == 0. */
typedef struct {
    int32_t kind;
    int32_t isotropic;
    int32_t group;
    int32_t n_cdf;
    double point[3], direction[3], lo[3], hi[3];
    double energy;
    const uint8_t *source_material;     /* [n_materials] (PINS) */
    const double *cdf_energy, *cdf_prob;
} tr_source_desc;

/* Tallies: an optional track-length flux mesh over [lo, hi] with n cells per
 * axis (per group when by_group != 0, multigroup only), and an optional
 * continuous-energy flux tally per material over n_energy_bins bins with
 * ascending, non-negative edges (eV; TR_ERR_INVALID otherwise).  The flux,
 * absorption-rate and production-rate totals are always scored.
 * Time (the paper's temporal tally resolution, Sec. 4; the formulas are our
 * reading): t_census > 0 makes the problem timed.  Histories start at t = 0
 * and move at speed 1/inv_velocity[g] (multigroup) or c sqrt(2E / m_n c^2)
 * (continuous energy); a history whose time would pass t_census first ends
 * there with the event TR_EV_CUTOFF.  n_time_bins > 0 (at most 4096) adds a
 * flux tally over that many uniform bins of [0, t_census).  Timed problems
 * run fixed source only.
 * Weight windows (the closeout event of the paper's decomposed scheme,
 * Sec. 4, "weights and weight windows for the particle's next loop
 * iteration"; the rules are our reading): ww_lower != NULL gives a lower
 * bound L per mesh voxel and group ([voxel][g], G = 1 for continuous energy;
 * 0 = no window).  Particles carry a weight (1 at birth) and every score is
 * weight x track length.  After each event a particle survives, in the voxel
 * holding its position: below L, Russian roulette to weight ww_survival x L
 * (the history otherwise ends as TR_EV_CUTOFF); above ww_upper x L, a split
 * into k = min(ceil(w / (ww_upper L)), ww_max_split) copies of weight w / k,
 * each copy with its own random stream.  Needs the mesh; requires
 * ww_upper > 1, 0 < ww_survival <= ww_upper, 2 <= ww_max_split <= 64.
 * Offered for fixed-source runs with the monolithic scheme (both
 * schedulers); copies go to the block's stash (asynchronous scheme: a full
 * stash gives TR_ERR_CAPACITY; raise stash_slots) or to the output stack
 * (stack scheme: TR_ERR_CAPACITY beyond queue_capacity). */
typedef struct {
    int32_t has_mesh;
    int32_t mesh_n[3];
    int32_t by_group;
    int32_t n_energy_bins;
    double mesh_lo[3], mesh_hi[3];
    const double *energy_edges;         /* n_energy_bins + 1 */
    int32_t n_time_bins;                /* 0 .. 4096 (needs t_census > 0) */
    double t_census;                    /* s; 0 = untimed */
    const double *ww_lower;             /* [mesh voxel][g] weight-window lower bounds, or NULL */
    double ww_upper, ww_survival;       /* upper bound and survival weight, as multiples of the lower bound */
    int32_t ww_max_split;               /* most copies per split */
} tr_tally_desc;

/* Device context.  alloc/free (optional) receive the byte size or pointer,
 * the stream and `user`; they must return 256-byte aligned device memory
 * usable on `stream`.  When both are NULL the library uses
 * cudaMallocAsync / cudaFreeAsync on `stream`. */
typedef struct {
    int32_t device;
    void *stream;                       /* cudaStream_t; NULL = legacy default stream */
    void *(*alloc)(size_t bytes, void *stream, void *user);
    void (*free)(void *ptr, void *stream, void *user);
    void *user;
} tr_device_ctx;

typedef struct tr_problem tr_problem;

/* Run options.  Zero-valued tuning fields take the library's defaults. */
typedef struct {
    uint64_t n_histories;
    uint64_t seed;
    int32_t scheme;                     /* TR_SCHEME_STACK / TR_SCHEME_ASYNC */
    int32_t decomposition;              /* TR_DECOMP_MONO / TR_DECOMP_SPLIT */
    uint64_t queue_capacity;            /* stack: particles per event stack; async: global links */
    int32_t blocks_per_sm;              /* resident blocks per SM */
    int32_t remap_every;                /* events a particle advances between remaps (>= 1) */
    int32_t stash_slots;                /* async: particle slots per block stash (0: 288 monolithic, 512 otherwise) */
    int64_t max_spin;                   /* async: iterations before a spin-wait gives up */
    uint32_t max_events;                /* per-history event cap (default 1e7) */
    int32_t want_event_log;             /* keep per-history (events, cell, type) for tr_event_log */
    int32_t spill_threshold;            /* async: spill a full link once a queue exceeds this (0 = default) */
    uint32_t problem_tag;               /* random stream tag (batched runs: problem index) */
    uint64_t first_history;             /* fixed source: run histories first .. first + n - 1 (a shard) */
    uint32_t max_wait_ms;               /* async: wall-clock limit of one spin-wait (0 = 60000) */
    uint32_t reserved;
} tr_run_opts;

typedef struct {
    uint64_t histories;
    uint64_t events;                    /* processed transport events (source events excluded) */
    uint64_t events_by_type[8];         /* TR_EV_* counts, source included */
    uint64_t final_by_type[8];          /* histories by final event type */
    uint64_t launches;                  /* kernel launches of the transport loop */
    uint64_t spills, refills;           /* async: links moved to / from global memory */
    double seconds;                     /* device time of the whole run */
    double transport_seconds;           /* device time of the transport-loop kernels alone */
    int32_t used_blocks_per_sm;         /* tr_run_batched: tuning the run used (autotuned where */
    int32_t used_stash_slots;           /*   opts left it 0); 0 after single runs */
    int32_t used_remap_every;
    int32_t reserved;
} tr_run_stats;

/* Create a problem on the device.  Copies every array (the caller keeps
 * ownership of its buffers).  n_tallies is 0 or 1.  Errors: TR_ERR_INVALID
 * for malformed descriptions (sizes, non-ascending planes, material ids out
 * of range), TR_ERR_NOMEM, TR_ERR_CUDA.  *out is NULL on failure. */
tr_status tr_problem_create(const tr_geometry_desc *geometry, const tr_xs_desc *xs,
                            const tr_source_desc *source, const tr_tally_desc *tallies, int32_t n_tallies,
                            const tr_device_ctx *ctx, tr_problem **out);

/* Replace the multigroup cross sections of a problem in place (the paper has
 * no counterpart: it serves the derivative workflow, where the cross
 * sections are the parameters being optimised).  sigma_t [m][g],
 * sigma_s [m][g][g'] and nu_sigma_f [m][g], n_materials x n_groups as at
 * creation, row-major doubles; device memory of the problem's device when
 * on_device != 0 (no host copy), else host memory.  The derived tables
 * (1/sigma_t, the cumulative scattering rows, sigma_a) are rebuilt on the
 * device with the operations problem creation uses, so runs equal those of
 * a problem created with these values.  chi is unchanged.  Results and a
 * kept power-iteration state of earlier runs are dropped (TR_ERR_STATE until
 * the next run), and checkpoints taken before no longer match.  Synchronises
 * the problem's stream.  Errors: TR_ERR_INVALID for NULL arrays, a
 * continuous-energy problem, a sigma_t that is not positive and finite or a
 * sigma_s that is negative or not finite (the problem keeps its previous
 * values); TR_ERR_NOMEM; TR_ERR_CUDA. */
tr_status tr_problem_set_xs(tr_problem *problem, const double *sigma_t, const double *sigma_s,
                            const double *nu_sigma_f, int32_t on_device);

/* Destroy a problem (NULL-safe); frees through the context's callbacks on its stream. */
void tr_problem_destroy(tr_problem *problem);

/* Fixed-source run (Sec. 4: source, step, collision, surface-crossing events
 * until every history ends).  Zeroes the tallies first; tallies become means
 * per source particle.  Synchronises the context stream before filling
 * `stats` (may be NULL).  TR_ERR_CAPACITY / TR_ERR_TIMEOUT leave the problem
 * usable with undefined tallies. */
tr_status tr_run_fixed_source(tr_problem *problem, const tr_run_opts *opts, tr_run_stats *stats);

/* Batched fixed-source run: n independent multigroup problems transported in
 * one persistent launch of the asynchronous scheme (Sec. 3.2), the source
 * cursor running over all problems' histories and each particle carrying its
 * problem index, so that work from every problem fills the same warps.
 * probs[0..n-1]: problems created on one device (probs[0], the leader, owns
 * the launch's workspace and stream; a problem may appear in one batch only
 * once).  n_histories[i] (< 2^32): histories of problem i.  opts: as for
 * tr_run_fixed_source with scheme TR_SCHEME_ASYNC and first_history 0;
 * problem i uses the random-stream tag problem_tag ^ i (problem_tag < 2^31),
 * so each problem's tallies, counts and event log equal those of
 * tr_run_fixed_source on that problem alone with that tag.  Fields
 * blocks_per_sm, stash_slots and remap_every left at 0 are autotuned: the
 * first call with a given batch times the candidate settings on 1/16 of each
 * problem's histories and keeps the fastest for later calls.  The whole run
 * (zeroing, transport, normalisation) is captured once as a CUDA graph and
 * replayed while the batch, the options and the leader's buffers stay the
 * same.  stats (may be NULL): n entries, per problem (spills, refills and
 * times are the batch's).  Errors: TR_ERR_INVALID (NULL, n < 1, continuous
 * energy, mixed devices, stack scheme, first_history != 0), TR_ERR_NOMEM,
 * TR_ERR_CAPACITY, TR_ERR_TIMEOUT, TR_ERR_CUDA.  Synchronises the leader's
 * stream (and each member's stream before the launch). */
tr_status tr_run_batched(tr_problem *const *probs, int32_t n, const uint64_t *n_histories, const tr_run_opts *opts,
                         tr_run_stats *stats);

typedef struct {
    uint64_t n_per_batch;
    uint32_t n_inactive, n_active;
    double k0;                          /* initial eigenvalue guess (default 1) */
    double bank_capacity_factor;        /* fission bank = factor * n_per_batch (default 4) */
    tr_run_opts run;                    /* seed, scheme, decomposition, tuning */
    uint32_t stop_after;                /* end after this many batches in all, keeping the state for
                                           tr_eig_checkpoint (0 or >= n_inactive + n_active: run to the end) */
    const void *resume_from;            /* host buffer from tr_eig_checkpoint (NULL: start afresh) */
    size_t resume_bytes;
} tr_eig_opts;

typedef struct {
    double k_mean, k_std;               /* over active batches; std of the mean */
    double *k_batch;                    /* caller buffer, n_inactive + n_active (may be NULL) */
    double *ktl_batch;                  /* caller buffer, track-length k per batch (may be NULL) */
    uint64_t *n_source;                 /* caller buffer, source size per batch (may be NULL) */
    uint64_t histories, events;
    uint64_t final_by_type[8];
    double seconds;                     /* device time of all batches */
    double transport_seconds;           /* device time of the transport-loop kernels alone */
    uint64_t transport_launches;        /* launches of the transport-loop kernels */
    uint32_t batches_done;              /* batches completed, counting those before a resume */
} tr_eig_result;

/* k-eigenvalue power iteration (Sec. 4: inactive then active cycles with
 * splitting-roulette population control).  Each batch banks fission sites,
 * orders the bank by (parent history, site sequence), and resamples it to
 * n_per_batch by splitting roulette.  Tallies become the mean over active
 * batches of the per-batch means per source particle; tr_tally_stddev gives
 * the standard deviation of that mean.  Multigroup only (TR_ERR_INVALID
 * otherwise).  The event log holds the last batch. */
tr_status tr_run_power_iteration(tr_problem *problem, const tr_eig_opts *opts, tr_eig_result *out);

/* Checkpoint of a power iteration that ended early (opts.stop_after): the
 * state before the next batch, namely the opts it ran with, the batch index,
 * the eigenvalue, the resampled source bank, the running eigenvalue sums, the
 * active-batch tally sums, the event counters and the per-batch eigenvalue,
 * track-length eigenvalue and source size so far.  Passing it back as
 * opts.resume_from (same problem description and opts apart from stop_after
 * and the resume fields, else TR_ERR_STATE) continues with the same histories
 * and eigenvalues as an uninterrupted run; the tallies agree to rounding
 * (summation order).  buf == NULL: *bytes receives the size.  Otherwise the
 * state is written to buf (cap bytes, TR_ERR_INVALID if too small).  The
 * buffer is plain host memory and may be stored in a file; it is not portable
 * across library versions.  TR_ERR_STATE when the last power iteration ran to
 * the end (or none ran). */
tr_status tr_eig_checkpoint(const tr_problem *problem, void *buf, size_t cap, size_t *bytes);

/* Derivatives of L = sum_b g_b T_b with respect to the multigroup cross
 * sections, where T are the fixed-source tallies of the preceding
 * tr_run_fixed_source (same opts: histories, seed, tag, first history and
 * event cap, else TR_ERR_STATE) and g the upstream gradients.  The estimator
 * is the score-function (likelihood-ratio) sum in causal form over the
 * random decisions of each history (flight lengths, reaction outcomes) plus
 * the explicit dependence of the absorption and production tallies; the
 * histories are recomputed from their random-number keys, never stored.
 * Inputs (device memory): d_grad_mesh [mesh size] (NULL = 0) and
 * d_grad_scalars [3] = gradients of (flux, absorption rate, production rate)
 * (NULL = 0).  Outputs (device memory, overwritten): d_sigt [m][g],
 * d_sigs [m][g][g'] and d_nusigf [m][g], means per source particle.
 * Derivatives with respect to a zero scattering cross section are not
 * estimated (the transfer never occurs).  Multigroup only (TR_ERR_INVALID
 * otherwise).  Synchronises the problem's stream. */
tr_status tr_sensitivities(tr_problem *problem, const tr_run_opts *opts, const double *d_grad_mesh,
                           const double *d_grad_scalars, double *d_sigt, double *d_sigs, double *d_nusigf);

/* Tally ids for tr_tallies / tr_tally_stddev. */
enum { TR_TALLY_MESH = 0, TR_TALLY_ENERGY = 1, TR_TALLY_SCALARS = 2, TR_TALLY_TIME = 3 };

/* Copy a tally (mesh: [group][z][y][x]; energy: [material][bin]; scalars:
 * flux, absorption rate, production rate; time: [bin]) into `out`, host memory unless
 * out_on_device != 0.  n_out must equal the tally size (TR_ERR_INVALID
 * otherwise).  Synchronises the context stream. */
tr_status tr_tallies(const tr_problem *problem, int32_t tally_id, double *out, size_t n_out, int32_t out_on_device);

/* Standard deviation of the mean of a tally over the active batches of the
 * last power iteration (TR_ERR_STATE after a fixed-source run); same
 * arguments, layout and errors as tr_tallies. */
tr_status tr_tally_stddev(const tr_problem *problem, int32_t tally_id, double *out, size_t n_out,
                          int32_t out_on_device);
/* Number of doubles of a tally (0 if absent). */
size_t tr_tally_size(const tr_problem *problem, int32_t tally_id);

/* Per-history log of the last run (requires want_event_log): final event
 * count, final cell id ((k ny + j) nx + i) * 2 + inside_pin, final type.
 * n must equal the number of histories of that run.  Host buffers. */
tr_status tr_event_log(const tr_problem *problem, uint32_t *n_events, int32_t *final_cell, uint8_t *final_type,
                       size_t n);

/* Size of the static scratch of tr_run_fixed_source_noalloc (bytes held on
 * every GPU that loads the library), the largest queue_capacity (particles
 * of spill space) it accepts, and the most tally bins (mesh + energy + the 3
 * scalars) a problem run through it may have. */
#define TR_NOALLOC_SCRATCH_BYTES (1024u * 1024u)
#define TR_NOALLOC_MAX_QUEUE_CAPACITY 4096u
#define TR_NOALLOC_MAX_TALLY_BINS 24576u

/* Fixed-source run that allocates nothing (the paper has no counterpart; it
 * exists for callers of this library that cannot allocate device memory
 * while they run, such as an application that reserves the GPU's memory for
 * its own pool at start-up, or a latency-sensitive loop that cannot accept
 * the device synchronisation of cudaMalloc/cudaFree).  It runs the
 * asynchronous scheme (opts->scheme must be TR_SCHEME_ASYNC, either
 * decomposition) and gives the same results as tr_run_fixed_source.
 *  - Scratch (error word, counters, scheduler control block, a link arena of
 *    TR_NOALLOC_MAX_QUEUE_CAPACITY particles for spills, and the tally
 *    accumulators of up to TR_NOALLOC_MAX_TALLY_BINS bins) is a file-scope
 *    __device__ array of TR_NOALLOC_SCRATCH_BYTES that each GPU loading the
 *    library holds until exit.  No cudaMalloc, cudaFree, event or stream
 *    creation happens in this call.
 *  - The first call on each device looks the array's device address up
 *    (cudaGetSymbolAddress, with that device current); make that first call
 *    before any stream capture.  With CUDA's lazy module loading, the first
 *    call that runs a given kernel variant (scheme, decomposition, remap
 *    frequency) also loads that kernel, which the driver may back with
 *    device memory: make one call with the options you will use at set-up,
 *    before the memory is reserved elsewhere; later calls with those options
 *    take no device memory.
 *  - Every call on a device shares the array; each call clears what must
 *    start at zero.  Calls whose work overlaps on the GPU (other streams or
 *    threads) race on the array and must not be issued concurrently.
 *  - Inputs: `problem` from tr_problem_create; `opts` as for
 *    tr_run_fixed_source (queue_capacity counts spill particles, at most
 *    TR_NOALLOC_MAX_QUEUE_CAPACITY, 0 = the maximum; want_event_log must be
 *    0).  Outputs: device arrays of tr_tally_size() doubles for the mesh and
 *    energy tallies (NULL allowed when the tally is absent) and 3 doubles of
 *    scalar tallies, all means per source particle; `stats` (may be NULL)
 *    has no timing (seconds are 0).  The problem's own tallies are left
 *    untouched.  Synchronises the problem's stream before returning.
 *  - Errors: TR_ERR_INVALID for a non-async scheme, an event log request, a
 *    queue_capacity above the maximum, more tally bins than the maximum or
 *    NULL outputs; TR_ERR_CUDA,
 *    TR_ERR_TIMEOUT, TR_ERR_CAPACITY as for tr_run_fixed_source. */
tr_status tr_run_fixed_source_noalloc(tr_problem *problem, const tr_run_opts *opts, double *mesh_out,
                                      double *energy_out, double *scalars_out, tr_run_stats *stats);

/* Device-side check of the random numbers, for the test suite (Philox-4x32-10,
 * Salmon et al., SC'11; the generator is our reading of the paper's
 * hash-based generator, Sec. 3): for i < n, the library's device Philox on
 * counter ctr[4i..4i+3] and key key[2i..2i+1], and a call of CUDA's own
 * curand_Philox4x32_10 on the same words.  All arrays are host memory: ctr
 * 4n and key 2n words in, ours and curand_out 4n words out each.  Uses the
 * current device and device scratch it allocates; synchronous.  Errors:
 * TR_ERR_INVALID for NULL arrays or n > 2^26, TR_ERR_CUDA. */
tr_status tr_selftest_philox(const uint32_t *ctr, const uint32_t *key, size_t n, uint32_t *ours,
                             uint32_t *curand_out);

/* Device-side check of the logarithm the transport kernels evaluate (Tang's
 * table-driven method with the problem's table): out[i] = log(x[i]) for the
 * n host values x (positive, finite, normal; others give TR_ERR_INVALID),
 * computed on the problem's device, written to the host array out.  Device
 * scratch is allocated; synchronous on the problem's stream.  n <= 2^26. */
tr_status tr_selftest_log(const tr_problem *problem, const double *x, size_t n, double *out);

/* The exponential ziggurat table the transport kernels of this problem read
 * (built on the device at problem creation): 1024 doubles to the host array
 * out, {W_i, C_i} for the 256 layers, then {f_i, f_i+1 - f_i}.  Synchronous. */
tr_status tr_selftest_zig_table(const tr_problem *problem, double *out);

/* Issue-rate probe of the arithmetic pipes (the roofline's denominators; the
 * paper has no counterpart): eight independent dependency chains per thread,
 * eight blocks of 256 threads per SM on the current device.  op 0..4: FP64
 * add, multiply, fma, division and square root (correctly rounded); 5: FP32
 * fma; 6: INT32 multiply-add (thread-operations per second to *per_second);
 * 7: FP64 fma executed by only the first `lanes` (1..32) lanes of each warp
 * (FP64 warp instructions per second: constant in `lanes` when a warp
 * instruction costs the same pipe time however few lanes are active);
 * 8 / 9: reciprocal by the IEEE sequence / by tr_selftest_softfp's integer
 * method; 10 / 11: square root, the same pair.
 * Allocates device scratch; synchronous.  TR_ERR_INVALID for a bad op. */
tr_status tr_selftest_issue_rate(int32_t op, int32_t lanes, double *per_second);

/* The transport kernels' correctly rounded reciprocal and square root
 * computed on the integer and FP32 pipes (paper has no counterpart: a GB300
 * economy of the FP64 pipe), beside the IEEE hardware sequences, for n host
 * doubles x[] into out[]: op 0: sf_rcp(x), 1: 1.0 / x, 2: sf_sqrt(x),
 * 3: sqrt(x); op 4: sf_div(x[2i], x[2i+1]), 5: x[2i] / x[2i+1] into
 * out[i] for i < n/2 (n even).  Ops 0 and 1 (2 and 3, 4 and 5) must agree
 * bit for bit on every input.  Allocates device scratch; synchronous.
 * n <= 2^26. */
tr_status tr_selftest_softfp(int32_t op, const double *x, size_t n, double *out);

/* Diagnostics: number of kernels this library has launched in this process
 * (all kernels, all problems).  Read it before and after a call to count the
 * launches the call made. */
uint64_t tr_kernel_launch_count(void);

/* Thread-local message for the last non-OK status of this thread. */
const char *tr_last_error(void);

/* Library version string. */
const char *tr_version(void);

#ifdef __cplusplus
}
#endif
#endif
