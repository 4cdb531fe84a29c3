/*
 * oracle.h -- CPU oracle for event-based Monte Carlo neutron transport.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded FP64
 * history-based tracker that defines the expected results of the GPU library.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load it.  It shares no source with the CUDA library; both implement the
 * same arithmetic contract independently.
 *
 * The paper (Cuneo et al., M&C 2025) describes the transport loop only by its
 * events (Sec. 4: source / make_work, step = move + tally, collision, surface
 * crossing, closeout) and states that the C5G7 runs are analog with
 * splitting-roulette population control (Sec. 4, Sec. 5.1).  Every physics
 * formula below is therefore a reading, written out once in the arithmetic
 * contract and cited in each function.
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Event / final-state codes (the event vocabulary of Sec. 4). */
enum { ORC_SOURCE = 0, ORC_SCATTER = 1, ORC_ABSORB = 2, ORC_SURF_INTERNAL = 3,
       ORC_SURF_REFLECT = 4, ORC_LEAK = 5, ORC_CUTOFF = 6, ORC_MAXEV = 7 };

typedef struct {
    /* geometry: rectilinear grid of cells, optional centred z-cylinder per cell */
    int32_t nx, ny, nz;
    const double *xp, *yp, *zp;          /* nx+1, ny+1, nz+1 ascending planes */
    int32_t bc[6];                       /* x-,x+,y-,y+,z-,z+ : 0 vacuum, 1 reflect */
    const int32_t *cell_mat;             /* [nz][ny][nx] */
    const int32_t *pin_mat;              /* [nz][ny][nx], <0 none */
    double pin_r;
    /* cross sections */
    int32_t xs_kind;                     /* 0 multigroup, 1 continuous energy */
    int32_t n_mat, n_grp;
    const double *sigt, *sigs, *nusigf, *chi;  /* [m][g], [m][g][g'], [m][g], [m][g] */
    int32_t n_nuc;
    const int64_t *nuc_off;              /* n_nuc+1 row offsets */
    const double *nuc_e;                 /* energies (eV), concatenated */
    const double *nuc_sig;               /* [row][3]: elastic, capture, fission (barn) */
    const double *nuc_awr;               /* A per nuclide */
    const double *mat_dens;              /* [m][n_nuc] atoms/(barn cm) */
    double e_cut;
    /* source */
    int32_t src_kind, src_iso, src_group, n_cdf;
    double src_pt[3], src_dir[3], src_lo[3], src_hi[3], src_energy;
    const uint8_t *src_mat;              /* [n_mat] */
    const double *cdf_e, *cdf_p;         /* n_cdf points */
    /* tallies */
    int32_t has_mesh, mesh_n[3], mesh_by_group, n_ebins;
    double mesh_lo[3], mesh_hi[3];
    const double *e_edges;               /* n_ebins + 1 */
    /* time (0 = untimed): particles start at t = 0 and end at the census time
     * t_cen; speeds from inv_vel[g] (multigroup, s/cm) or from the energy
     * (continuous energy); n_tbins uniform time bins over [0, t_cen) */
    const double *inv_vel;
    int32_t n_tbins;
    double t_cen;
    /* weight windows (NULL = none; fixed source only): the lower bound per
     * tally-mesh voxel and group, [voxel][g] (0: no window there); upper bound
     * ww_upper x lower, roulette survival weight ww_survival x lower, at most
     * ww_max_split copies per split */
    const double *ww_lo;
    double ww_upper, ww_survival;
    int32_t ww_max_split;
} orc_problem;

typedef struct {
    /* inputs */
    uint64_t n_hist, seed;
    uint32_t tag, max_events;
    uint64_t id_offset;                  /* histories id_offset .. id_offset + n_hist - 1 */
    /* outputs: caller-allocated arrays, any may be NULL */
    double *mesh;                        /* mesh tally, mean per source particle */
    double *energy;                      /* energy tally [m][bin], mean per source particle */
    uint32_t *log_n;                     /* per-history final event count */
    int32_t *log_cell;                   /* per-history final cell id */
    uint8_t *log_type;                   /* per-history final event type */
    double *hist_track;                  /* per-history total track length */
    uint32_t *hist_coll;                 /* per-history collision count */
    /* outputs: scalars */
    double scalars[3];                   /* flux, absorption rate, production rate per source particle */
    uint64_t events_by_type[8];          /* processed events by type (SOURCE counted) */
    uint64_t final_by_type[8];           /* histories by final type */
    double *time_tally;                  /* [n_tbins] flux per time bin, mean per source particle (may be NULL) */
} orc_fixed;

typedef struct {
    /* inputs */
    uint64_t n_per_batch, seed, bank_capacity;
    uint32_t n_inactive, n_active, max_events;
    double k0;
    /* outputs (caller arrays of length n_inactive + n_active, may be NULL) */
    double *k_batch, *ktl_batch;
    uint64_t *n_source, *n_sites;
    /* active-batch mean and standard deviation of each tally (may be NULL) */
    double *mesh_mean, *mesh_std, *energy_mean, *energy_std;
    double scalars_mean[3], scalars_std[3];
    double k_mean, k_std;
    /* per-history log of batch `log_batch` (arrays of bank_capacity entries) */
    uint32_t log_batch;
    uint32_t *log_n; int32_t *log_cell; uint8_t *log_type;
    uint64_t log_count;
    uint64_t events_by_type[8], final_by_type[8];
} orc_eig;

/* status codes (same meaning as the library's, numbered independently) */
enum { ORC_OK = 0, ORC_ERR_INVALID = 1, ORC_ERR_NOMEM = 2, ORC_ERR_CAPACITY = 3, ORC_ERR_STATE = 6 };

/* Derivatives of L = sum_b g_b T_b (T = fixed-source tallies per source
 * particle, g = upstream gradients) with respect to the multigroup data, by
 * the score-function (likelihood-ratio) estimator in causal form plus the
 * pathwise terms of the reaction-rate tallies.  Multigroup, fixed source. */
typedef struct {
    uint64_t n_hist, seed;
    uint32_t tag, max_events;
    const double *g_mesh;                /* mesh_size upstream gradients (NULL = 0) */
    const double *g_scal;                /* 3: flux, absorption, production (NULL = 0) */
    double *d_sigt;                      /* out [m][g] */
    double *d_sigs;                      /* out [m][g][g'] */
    double *d_nusigf;                    /* out [m][g] */
    double value;                        /* out: L itself (mean per source particle) */
    uint64_t id_offset;                  /* first history index (histories id_offset .. id_offset + n_hist - 1) */
} orc_sens;

int orc_fixed_source(const orc_problem *P, orc_fixed *o);
int orc_sensitivities(const orc_problem *P, orc_sens *o);
int orc_power_iteration(const orc_problem *P, orc_eig *o);

/* unit-level entry points used by the pin tests */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_uniform(uint32_t lo, uint32_t hi);
double orc_log(double x);
void orc_iso_dir(uint64_t seed, uint32_t tag, uint64_t id, uint32_t n, double dir[3]);
double orc_exp_event(uint64_t seed, uint32_t tag, uint64_t id, uint32_t n);
int orc_ce_macro(const orc_problem *P, int m, double E, double out[2]);
void orc_zig_table(double out[1024]);
void orc_elastic(double A, double E, double mu_cm, double *E_out, double *mu_lab);
void orc_rotate(const double dir[3], double mu, double cphi, double sphi, double out[3]);
void orc_azimuth(uint64_t seed, uint32_t tag, uint64_t id, uint32_t n, double out[2]);
void orc_elastic_scatter(uint64_t seed, uint32_t tag, uint64_t id, uint32_t n, double A, double E, const double d[3],
                         double d_out[3], double *E_out);
double orc_cdf_sample(const double *e, const double *p, int32_t n, double xi);
double orc_mesh_segment(const orc_problem *P, const double p0[3], const double dir[3], double len, double *mesh);
int64_t orc_nuclide_index(const double *e, int64_t n, double E);

#ifdef __cplusplus
}
#endif
#endif
