/*
 * oracle.c -- CPU oracle for event-based Monte Carlo neutron transport.
 *
 * TEST INFRASTRUCTURE ONLY: only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load or run this code.  It is a plain,
 * slow, single-threaded FP64 history-based tracker.  It shares no source with
 * the CUDA library.
 *
 * Build with contraction off (gcc -O2 -ffp-contract=off): every floating-
 * point operation below is one IEEE-754 binary64 operation, evaluated in the
 * order written, so that the GPU library (which implements the same contract
 * independently, also without implicit contraction) takes every branch the
 * same way.  Where the contract fuses a product with a sum, the code says so
 * with an explicit fma() (one correctly rounded operation, the same on every
 * machine): the log polynomial and its exponent term, the move, the pin
 * terms, the squared transverse direction, the cylinder discriminant, and
 * 1 - mu^2 in the direction formulas.
 *
 * What the paper fixes, and what is a reading:
 *  - The transport loop is split into events: a source event (make_work),
 *    the "step" (move to the next event site and score the path), collision,
 *    surface crossing, and closeout (Sec. 4).  A history is processed event
 *    by event below; the event counter n counts every processed event,
 *    including the source event.
 *  - Particles are created through atomic counters and a hash-based RNG
 *    (Sec. 3): here every random number is Philox-4x32-10 (Salmon et al.,
 *    SC'11) keyed by (seed, stream tag) with counter (n, block j, id).
 *  - The C5G7 runs are analog, without implicit capture, with splitting-
 *    roulette population control (Sec. 4, Sec. 5.1).
 *  - Everything else (sampling formulas, geometry tie-breaks, estimators) is
 *    our reading; each function names the reading it implements.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11): 10 rounds of two 32x32->64 multiplications by  */
/* the round multipliers, with the key bumped by the Weyl increments.        */
/* ------------------------------------------------------------------------ */
#define PH_M0 0xD2511F53u
#define PH_M1 0xCD9E8D57u
#define PH_W0 0x9E3779B9u
#define PH_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PH_W0;
            k1 += PH_W1;
        }
        uint64_t p0 = (uint64_t)PH_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)PH_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Uniform in (0,1): the top 52 bits of the 64-bit word (hi:lo), plus one half,
 * times 2^-52.  Exact in binary64; never 0 or 1. */
double orc_uniform(uint32_t lo, uint32_t hi)
{
    uint64_t w = ((uint64_t)hi << 32) | (uint64_t)lo;
    return ((double)(w >> 12) + 0.5) * 0x1p-52;
}

/* One Philox block for stream (seed, tag), counter (n, j, id_lo, id_hi):   */
/* its four words, and its two uniforms (words 0-1 and 2-3).                 */
static void rng_words(uint64_t seed, uint32_t tag, uint64_t id, uint32_t n, uint32_t j, uint32_t r[4])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ tag};
    uint32_t ctr[4] = {n, j, (uint32_t)id, (uint32_t)(id >> 32)};
    orc_philox4x32_10(ctr, key, r);
}

static void rng_block(uint64_t seed, uint32_t tag, uint64_t id, uint32_t n, uint32_t j, double xi[2])
{
    uint32_t r[4];
    rng_words(seed, tag, id, n, j, r);
    xi[0] = orc_uniform(r[0], r[1]);
    xi[1] = orc_uniform(r[2], r[3]);
}

/* Block indices within one event (the contract's fixed assignment). */
#define BLK_MAIN 0u      /* (distance / source mu, reaction / source energy) */
#define BLK_ANGLE 1u     /* (CM cosine of an elastic scatter, unused) */
#define BLK_FISSION 2u   /* (number of fission sites, unused) */
#define BLK_AZIMUTH 3u   /* 3 + t: azimuth rejection try t, t < 64 */
#define BLK_CLOSE 4000u  /* (closeout roulette, unused) */
#define BLK_SPLIT 4001u  /* 4001 + c: stream tag of split copy c (word 0), c < 64 */
#define MAX_SPLIT 64
#define N_AZIMUTH_TRIES 64u
#define BLK_SITE 100u    /* 100 + c: fission site c (chi sample, unused) */
#define BLK_POS 200u     /* 200 + 2t, 201 + 2t: source position trial t */
#define N_POS_TRIES 1024u
#define BLK_ZIG 3000u    /* 3000 + t: exponential ziggurat, try t's wedge/tail uniform (words 2-3) */
#define N_ZIG_TRIES 64u  /*   and try t+1's layer and uniform (words 0-1)                        */
#define TAG_POPULATION 0x80000000u

/* ------------------------------------------------------------------------ */
/* Natural logarithm of a positive normal double (the contract's own), by    */
/* Tang's table-driven method (ACM TOMS 16 (1990) 378):                      */
/*   x = 2^e m, m in [sqrt(1/2), sqrt(2)]; k = the integer nearest            */
/*   128 (m - 1), c_k = 1 + k/128, i_k = 1/c_k (rounded);                     */
/*   r = fma(m, i_k, -1); log1p(r) = r + r^2 (-1/2 + r (1/3 + ... + r/7))     */
/*   (Horner from 1/7, one fma a step; |r| < 2^-7.4);                          */
/*   log x = fma(e, LN2_HI, fma(e, LN2_LO, T_k + log1p(r))), T_k = -log(i_k).  */
/* The table values T_k come from the atanh series:                          */
/*   s = (m-1)/(m+1); log m = 2 s sum_{j=0..9} s^(2j)/(2j+1) (Horner in s^2,  */
/*   each step one fma); log x = fma(e, LN2_HI, fma(e, LN2_LO, log m)).        */
/* ln 2 is split at 40 bits (e*LN2_HI is exact).                               */
/* ------------------------------------------------------------------------ */
static double bits_to_double(uint64_t b) { double d; memcpy(&d, &b, 8); return d; }
static uint64_t double_to_bits(double d) { uint64_t b; memcpy(&b, &d, 8); return b; }

static double log_atanh(double x)
{
    const double SQRT2 = bits_to_double(0x3FF6A09E667F3BCDull);
    const double LN2_HI = bits_to_double(0x3FE62E42FEFA4000ull);
    const double LN2_LO = bits_to_double(0xBD48432A1B0E2634ull);
    uint64_t b = double_to_bits(x);
    int e = (int)((b >> 52) & 0x7FF) - 1023;
    double m = bits_to_double((b & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull);
    if (m > SQRT2) {
        m = m * 0.5;
        e = e + 1;
    }
    double s = (m - 1.0) / (m + 1.0);
    double z = s * s;
    double p = 1.0 / 19.0;
    p = fma(p, z, 1.0 / 17.0);
    p = fma(p, z, 1.0 / 15.0);
    p = fma(p, z, 1.0 / 13.0);
    p = fma(p, z, 1.0 / 11.0);
    p = fma(p, z, 1.0 / 9.0);
    p = fma(p, z, 1.0 / 7.0);
    p = fma(p, z, 1.0 / 5.0);
    p = fma(p, z, 1.0 / 3.0);
    p = fma(p, z, 1.0);
    double r = (s + s) * p;
    double de = (double)e;
    return fma(de, LN2_HI, fma(de, LN2_LO, r));
}

#define LOG_K_LO (-38)
#define LOG_K_HI 54
static double log_inv_c[LOG_K_HI - LOG_K_LO + 1];
static double log_t[LOG_K_HI - LOG_K_LO + 1];
static int log_ready = 0;

static void log_make_table(void)
{
    for (int k = LOG_K_LO; k <= LOG_K_HI; ++k) {
        double c = (double)(128 + k) / 128.0;
        double ic = 1.0 / c;
        log_inv_c[k - LOG_K_LO] = ic;
        log_t[k - LOG_K_LO] = -log_atanh(ic);
    }
    log_ready = 1;
}

double orc_log(double x)
{
    const double SQRT2 = bits_to_double(0x3FF6A09E667F3BCDull);
    const double LN2_HI = bits_to_double(0x3FE62E42FEFA4000ull);
    const double LN2_LO = bits_to_double(0xBD48432A1B0E2634ull);
    if (!log_ready) log_make_table();
    uint64_t b = double_to_bits(x);
    int e = (int)((b >> 52) & 0x7FF) - 1023;
    double m = bits_to_double((b & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull);
    if (m > SQRT2) {
        m = m * 0.5;
        e = e + 1;
    }
    /* nearest table point: m - 1 is exact here, and so is its scaling by 128 */
    int k = (int)floor((m - 1.0) * 128.0 + 0.5);
    double ic = log_inv_c[k - LOG_K_LO];
    double r = fma(m, ic, -1.0);
    double q = 1.0 / 7.0;
    q = fma(q, r, -1.0 / 6.0);
    q = fma(q, r, 1.0 / 5.0);
    q = fma(q, r, -1.0 / 4.0);
    q = fma(q, r, 1.0 / 3.0);
    q = fma(q, r, -1.0 / 2.0);
    double p = fma(q, r * r, r);
    double de = (double)e;
    return fma(de, LN2_HI, fma(de, LN2_LO, log_t[k - LOG_K_LO] + p));
}

/* ------------------------------------------------------------------------ */
/* Exponential variate (the distance to collision in mean free paths) by the */
/* ziggurat method of Marsaglia and Tsang (J. Stat. Softw. 5, 2000), with    */
/* 256 layers of equal area v under f(x) = e^-x and their r and v:           */
/*   layer 0: the base [0, v/f(r)] x [0, f(r)] with the tail beyond r;        */
/*   layer i >= 1: [0, X_i] x [f(X_i), f(X_i+1)], X_1 = r, X_256 = 0.         */
/* Table: f(X_1) = v/(r+1) (the base area v = (r+1) e^-r), then               */
/* f(X_i+1) = f(X_i) + v/X_i and X_i+1 = -log f(X_i+1) with the contract's    */
/* log; f(X_256) = 1.                                                        */
/* A try takes layer i (the low 8 bits of its word pair) and the uniform U   */
/* of that pair: x = U W_i (W_0 = v/f(r), W_i = X_i) is accepted when below   */
/* the inner width C_i (C_0 = r, C_i = X_i+1).  Otherwise, with the uniform   */
/* U2 of words 2-3 of block BLK_ZIG + t: layer 0 returns r - log U2 (the      */
/* tail, memoryless); layer i accepts x if x < -log(fma(U2, f_i+1 - f_i,     */
/* f_i)), else try t+1 takes words 0-1 of the same block.                     */
/* ------------------------------------------------------------------------ */
#define ZIG_N 256
static double zig_w[ZIG_N], zig_c[ZIG_N], zig_f[ZIG_N], zig_df[ZIG_N];
static int zig_ready = 0;

static void zig_make_table(void)
{
    const double r = 7.69711747013104972;
    const double v = 0.0039496598225815571993;
    double X[ZIG_N + 1], F[ZIG_N + 1];
    X[1] = r;
    F[1] = v / (r + 1.0);
    for (int i = 1; i < ZIG_N - 1; ++i) {
        F[i + 1] = F[i] + v / X[i];
        X[i + 1] = -orc_log(F[i + 1]);
    }
    X[ZIG_N] = 0.0;
    F[ZIG_N] = 1.0;
    zig_w[0] = v / F[1];
    zig_c[0] = r;
    zig_f[0] = 0.0;
    zig_df[0] = 0.0;
    for (int i = 1; i < ZIG_N; ++i) {
        zig_w[i] = X[i];
        zig_c[i] = X[i + 1];
        zig_f[i] = F[i];
        zig_df[i] = F[i + 1] - F[i];
    }
    zig_ready = 1;
}

void orc_zig_table(double out[4 * ZIG_N])
{
    if (!zig_ready) zig_make_table();
    for (int i = 0; i < ZIG_N; ++i) {
        out[i] = zig_w[i];
        out[ZIG_N + i] = zig_c[i];
        out[2 * ZIG_N + i] = zig_f[i];
        out[3 * ZIG_N + i] = zig_df[i];
    }
}

/* words lo, hi: the pair for try 0 (words 0-1 of the event's main block) */
static double exp_sample(uint64_t seed, uint32_t tag, uint64_t id, uint32_t n, uint32_t lo, uint32_t hi)
{
    if (!zig_ready) zig_make_table();
    int i = (int)(lo & 0xFFu);
    double U = orc_uniform(lo, hi);
    double x = U * zig_w[i];
    if (x < zig_c[i]) return x;
    for (uint32_t t = 0; t < N_ZIG_TRIES; ++t) {
        uint32_t w[4];
        rng_words(seed, tag, id, n, BLK_ZIG + t, w);
        double U2 = orc_uniform(w[2], w[3]);
        if (i == 0) return zig_c[0] - orc_log(U2);
        double y = fma(U2, zig_df[i], zig_f[i]);
        if (x < -orc_log(y)) return x;
        i = (int)(w[0] & 0xFFu);
        U = orc_uniform(w[0], w[1]);
        x = U * zig_w[i];
        if (x < zig_c[i]) return x;
    }
    return -orc_log(U);   /* after N_ZIG_TRIES rejected tries (probability below 1e-100) */
}

/* the exponential variate of event n of history id (pin tests) */
double orc_exp_event(uint64_t seed, uint32_t tag, uint64_t id, uint32_t n)
{
    uint32_t w[4];
    rng_words(seed, tag, id, n, BLK_MAIN, w);
    return exp_sample(seed, tag, id, n, w[0], w[1]);
}

/* ------------------------------------------------------------------------ */
/* Directions.  A point of the unit disk by rejection in the unit square     */
/* (von Neumann): a = 2 xi - 1, b = 2 xi' - 1, accept 0 < s <= 1 with         */
/* s = a^2 + b^2.  Azimuth: cos phi = (a^2 - b^2)/s, sin phi = 2ab/s (no      */
/* trig).  Isotropic direction (Marsaglia 1972): (1 - 2s, 2a sqrt(1 - s),     */
/* 2b sqrt(1 - s)).                                                           */
/* ------------------------------------------------------------------------ */
static void disk_point(uint64_t seed, uint32_t tag, uint64_t id, uint32_t n, double *pa, double *pb, double *pa2,
                       double *pb2, double *ps)
{
    double a = 1.0, b = 0.0, a2 = 1.0, b2 = 0.0, s = 1.0;
    for (uint32_t t = 0; t < N_AZIMUTH_TRIES; ++t) {
        double xi[2];
        rng_block(seed, tag, id, n, BLK_AZIMUTH + t, xi);
        double ta = 2.0 * xi[0] - 1.0;
        double tb = 2.0 * xi[1] - 1.0;
        double ta2 = ta * ta, tb2 = tb * tb;
        double ts = ta2 + tb2;
        if (ts <= 1.0 && ts > 0.0) {
            a = ta; b = tb; a2 = ta2; b2 = tb2; s = ts;
            break;
        }
    }
    *pa = a; *pb = b; *pa2 = a2; *pb2 = b2; *ps = s;
}

static void azimuth(uint64_t seed, uint32_t tag, uint64_t id, uint32_t n, double *cphi, double *sphi)
{
    double a, b, a2, b2, s;
    disk_point(seed, tag, id, n, &a, &b, &a2, &b2, &s);
    double inv_s = 1.0 / s;
    *cphi = (a2 - b2) * inv_s;
    *sphi = (2.0 * (a * b)) * inv_s;
}

/* The azimuth of event n of history id: out = (cos phi, sin phi). */
void orc_azimuth(uint64_t seed, uint32_t tag, uint64_t id, uint32_t n, double out[2])
{
    azimuth(seed, tag, id, n, &out[0], &out[1]);
}

void orc_iso_dir(uint64_t seed, uint32_t tag, uint64_t id, uint32_t n, double dir[3])
{
    double a, b, a2, b2, s;
    disk_point(seed, tag, id, n, &a, &b, &a2, &b2, &s);
    double t = 2.0 * sqrt(1.0 - s);
    dir[0] = 1.0 - 2.0 * s;
    dir[1] = a * t;
    dir[2] = b * t;
}

/* Rotate direction `d` by polar cosine mu and azimuth (cphi, sphi): the
 * standard lab-frame rotation; near the poles (|w| > 1 - 1e-10) the new
 * direction is taken about the z axis. */
void orc_rotate(const double d[3], double mu, double cphi, double sphi, double out[3])
{
    double t = fma(-mu, mu, 1.0);
    if (t < 0.0) t = 0.0;
    double st = sqrt(t);
    double u = d[0], v = d[1], w = d[2];
    if (fabs(w) > 0.9999999999) {
        out[0] = st * cphi;
        out[1] = st * sphi;
        out[2] = (w > 0.0) ? mu : -mu;
        return;
    }
    double sq = sqrt(fma(-w, w, 1.0));
    double a1 = st / sq;
    out[0] = mu * u + a1 * ((u * w) * cphi - v * sphi);
    out[1] = mu * v + a1 * ((v * w) * cphi + u * sphi);
    out[2] = mu * w - (st * sq) * cphi;
}

/* Elastic scatter off a target of mass ratio A at rest, isotropic in the
 * centre-of-mass frame: E' = E (A^2 + 2 A mu + 1)/(A + 1)^2,
 * mu_lab = (1 + A mu)/sqrt(A^2 + 2 A mu + 1). */
void orc_elastic(double A, double E, double mu_cm, double *E_out, double *mu_lab)
{
    double q = (A * A + (2.0 * A) * mu_cm) + 1.0;
    double inv_ap1sq = 1.0 / ((A + 1.0) * (A + 1.0));
    *E_out = (E * q) * inv_ap1sq;
    *mu_lab = (1.0 + A * mu_cm) / sqrt(q);
}

/* The elastic scatter of event n of history id off a target of mass ratio A:
 * the CM cosine from block BLK_ANGLE, the lab energy and cosine, the azimuth,
 * and the incoming direction d rotated into d_out.  The continuous-energy
 * collision runs exactly this. */
void orc_elastic_scatter(uint64_t seed, uint32_t tag, uint64_t id, uint32_t n, double A, double E, const double d[3],
                         double d_out[3], double *E_out)
{
    double xa[2];
    rng_block(seed, tag, id, n, BLK_ANGLE, xa);
    double mu_cm = 2.0 * xa[0] - 1.0;
    double mu;
    orc_elastic(A, E, mu_cm, E_out, &mu);
    double cphi, sphi;
    azimuth(seed, tag, id, n, &cphi, &sphi);
    orc_rotate(d, mu, cphi, sphi, d_out);
}

/* Inverse-CDF sample from a tabulated CDF (e[k], p[k]), k < n: the largest k
 * with p[k] <= xi (k <= n-2), then linear interpolation. */
double orc_cdf_sample(const double *e, const double *p, int32_t n, double xi)
{
    int32_t k = 0;
    for (int32_t i = 0; i < n - 1; ++i)
        if (p[i] <= xi) k = i;
    return e[k] + (xi - p[k]) * (e[k + 1] - e[k]) / (p[k + 1] - p[k]);
}

/* Largest i in [0, n-2] with e[i] <= E (binary search over a sorted grid). */
int64_t orc_nuclide_index(const double *e, int64_t n, double E)
{
    if (E >= e[n - 1]) return n - 2;
    if (E <= e[0]) return 0;
    int64_t lo = 0, hi = n - 1;           /* e[lo] <= E < e[hi] */
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        if (e[mid] <= E) lo = mid; else hi = mid;
    }
    return lo;
}

/* ------------------------------------------------------------------------ */
/* Tally accumulation: Neumaier compensated sums in history order.            */
/* ------------------------------------------------------------------------ */
typedef struct { double s, c; } nsum;

static void nadd(nsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static double nval(const nsum *a) { return a->s + a->c; }

/* ------------------------------------------------------------------------ */
/* Problem set-up: derived tables every event uses.                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    const orc_problem *P;
    int G;
    double *inv_sigt;    /* [m][g] = 1/sigma_t */
    double *cum_s;       /* [m][g][g'] running sum of sigma_s over g' */
    double *sig_a;       /* [m][g] = sigma_t - total scatter */
    double *cum_chi;     /* [m][g] running sum of chi */
    double *slope;       /* CE: per grid row and reaction (s[i+1]-s[i])/(E[i+1]-E[i]) */
    int64_t n_rows;
    int64_t mesh_vox;
    /* tallies */
    nsum *mesh, *energy, scal[3], *time;
    double v_c;          /* CE speed per sqrt(eV): v = v_c sqrt(E) cm/s */
    /* run */
    uint64_t seed;
    uint32_t tag, max_events;
    int eig;
    double inv_k;
    /* fission bank */
    double *bank_pos; int32_t *bank_g, *bank_cell; double *bank_E;
    uint64_t bank_n, bank_cap;
    int bank_overflow;
    uint64_t events_by_type[8];
    /* adjoint: per-event record of the current history */
    struct orc_rec { int m, g, collided, react, h; double len, f; } *rec;
    int rec_n, rec_cap, recording;
    const double *gw_mesh, *gw_scal;
    /* weight windows: the current family's split copies waiting to run */
    struct particle_s *split;
    int split_n, split_cap;
} ctx;

static int setup(ctx *C, const orc_problem *P)
{
    memset(C, 0, sizeof(*C));
    C->P = P;
    if (P->nx < 1 || P->ny < 1 || P->nz < 1 || P->n_mat < 1) return ORC_ERR_INVALID;
    if (P->xs_kind == 0) {
        int M = P->n_mat, G = P->n_grp;
        C->G = G;
        C->inv_sigt = malloc(sizeof(double) * M * G);
        C->cum_s = malloc(sizeof(double) * M * G * G);
        C->sig_a = malloc(sizeof(double) * M * G);
        C->cum_chi = malloc(sizeof(double) * M * G);
        for (int m = 0; m < M; ++m) {
            double c = 0.0;
            for (int g = 0; g < G; ++g) {
                c = c + P->chi[m * G + g];
                C->cum_chi[m * G + g] = c;
            }
            for (int g = 0; g < G; ++g) {
                double st = P->sigt[m * G + g];
                C->inv_sigt[m * G + g] = 1.0 / st;
                double cs = 0.0;
                for (int h = 0; h < G; ++h) {
                    cs = cs + P->sigs[(m * G + g) * G + h];
                    C->cum_s[(m * G + g) * G + h] = cs;
                }
                C->sig_a[m * G + g] = st - cs;
            }
        }
    } else {
        if (P->n_nuc < 1 || P->n_nuc * 3 > 64) return ORC_ERR_INVALID;
        C->G = 1;
        C->n_rows = P->nuc_off[P->n_nuc];
        C->slope = malloc(sizeof(double) * 3 * (size_t)C->n_rows);
        for (int n = 0; n < P->n_nuc; ++n)
            for (int64_t r = P->nuc_off[n]; r < P->nuc_off[n + 1]; ++r)
                for (int k = 0; k < 3; ++k)
                    C->slope[3 * r + k] = (r + 1 < P->nuc_off[n + 1])
                                              ? (P->nuc_sig[3 * (r + 1) + k] - P->nuc_sig[3 * r + k]) /
                                                    (P->nuc_e[r + 1] - P->nuc_e[r])
                                              : 0.0;
    }
    C->mesh_vox = P->has_mesh ? (int64_t)P->mesh_n[0] * P->mesh_n[1] * P->mesh_n[2] : 0;
    int64_t msize = C->mesh_vox * ((P->mesh_by_group && P->xs_kind == 0) ? C->G : 1);
    C->mesh = calloc((size_t)(msize > 0 ? msize : 1), sizeof(nsum));
    int64_t esize = (int64_t)P->n_ebins * P->n_mat;
    C->energy = calloc((size_t)(esize > 0 ? esize : 1), sizeof(nsum));
    if (P->t_cen < 0.0 || P->n_tbins < 0 || (P->n_tbins > 0 && !(P->t_cen > 0.0))) return ORC_ERR_INVALID;
    if (P->t_cen > 0.0 && P->xs_kind == 0) {
        if (!P->inv_vel) return ORC_ERR_INVALID;
        for (int g = 0; g < C->G; ++g)
            if (!(P->inv_vel[g] > 0.0)) return ORC_ERR_INVALID;
    }
    C->time = calloc((size_t)(P->n_tbins > 0 ? P->n_tbins : 1), sizeof(nsum));
    /* neutron speed from kinetic energy: v = c sqrt(2 E / (m_n c^2)) */
    C->v_c = 2.99792458e10 * sqrt(2.0 / 939.56542052e6);
    return ORC_OK;
}

static void teardown(ctx *C)
{
    free(C->rec);
    free(C->split);
    free(C->inv_sigt); free(C->cum_s); free(C->sig_a); free(C->cum_chi); free(C->slope);
    free(C->mesh); free(C->energy); free(C->time);
    free(C->bank_pos); free(C->bank_g); free(C->bank_cell); free(C->bank_E);
}

static void clear_tallies(ctx *C)
{
    const orc_problem *P = C->P;
    int64_t msize = C->mesh_vox * ((P->mesh_by_group && P->xs_kind == 0) ? C->G : 1);
    if (msize > 0) memset(C->mesh, 0, sizeof(nsum) * (size_t)msize);
    int64_t esize = (int64_t)P->n_ebins * P->n_mat;
    if (esize > 0) memset(C->energy, 0, sizeof(nsum) * (size_t)esize);
    if (P->n_tbins > 0) memset(C->time, 0, sizeof(nsum) * (size_t)P->n_tbins);
    memset(C->scal, 0, sizeof(C->scal));
}

/* ------------------------------------------------------------------------ */
/* Particle state                                                            */
/* ------------------------------------------------------------------------ */
typedef struct particle_s {
    double x[3], d[3], E;
    double t;                            /* time since the source (timed problems) */
    int32_t g, ci[3], in;
    uint32_t n;
    uint64_t id;                         /* random-stream id: batch << 32 | index, a split copy's tag xored into the high word */
    int alive, final_type;
    double track;
    uint32_t coll;
    double w;                            /* statistical weight (1 at birth; the closeout changes it) */
} particle;

static int64_t cell_lin(const orc_problem *P, const particle *p)
{
    return ((int64_t)p->ci[2] * P->ny + p->ci[1]) * P->nx + p->ci[0];
}
static int32_t cell_id(const orc_problem *P, const particle *p) { return (int32_t)(cell_lin(P, p) * 2 + p->in); }

static int material(const orc_problem *P, const particle *p)
{
    int64_t c = cell_lin(P, p);
    return p->in ? P->pin_mat[c] : P->cell_mat[c];
}

static const double *planes(const orc_problem *P, int a)
{
    return a == 0 ? P->xp : (a == 1 ? P->yp : P->zp);
}
static int nplanes(const orc_problem *P, int a) { return a == 0 ? P->nx : (a == 1 ? P->ny : P->nz); }

/* Pin relation of point (x, y) in cell (i, j): c = dx^2 + dy^2 - r^2 and
 * k = dx u + dy v with the centre at the midpoint of the cell's x-y box. */
static void pin_terms(const orc_problem *P, const particle *p, double *c, double *k, double *dx, double *dy)
{
    double xc = 0.5 * (P->xp[p->ci[0]] + P->xp[p->ci[0] + 1]);
    double yc = 0.5 * (P->yp[p->ci[1]] + P->yp[p->ci[1] + 1]);
    *dx = p->x[0] - xc;
    *dy = p->x[1] - yc;
    *c = fma(*dx, *dx, (*dy) * (*dy)) - P->pin_r * P->pin_r;
    *k = fma(*dx, p->d[0], (*dy) * p->d[1]);
}

static int has_pin(const orc_problem *P, const particle *p) { return P->pin_mat[cell_lin(P, p)] >= 0; }

/* Locate a point: on each axis the largest i in [0, n-1] with plane[i] <= x,
 * stepping down one cell when x sits exactly on an interior plane and the
 * direction component is negative.  Inside a pin iff c < 0. */
static void locate(const orc_problem *P, particle *p)
{
    for (int a = 0; a < 3; ++a) {
        const double *pl = planes(P, a);
        int n = nplanes(P, a);
        int i = 0;
        for (int t = 0; t < n; ++t)
            if (pl[t] <= p->x[a]) i = t;
        if (i > 0 && p->x[a] == pl[i] && p->d[a] < 0.0) i = i - 1;
        p->ci[a] = i;
    }
    p->in = 0;
    if (has_pin(P, p)) {
        double c, k, dx, dy;
        pin_terms(P, p, &c, &k, &dx, &dy);
        p->in = (c < 0.0) ? 1 : 0;
    }
}

/* ------------------------------------------------------------------------ */
/* Cross sections                                                            */
/* ------------------------------------------------------------------------ */
typedef struct {
    double st, inv_st, sa, nsf;
    /* CE reaction table: cumulative macroscopic values in (nuclide, reaction) order */
    int nterm;
    double cum[64];
    int term_nuc[64], term_r[64];
    double term_val[64];
} xsval;

static void xs_lookup(const ctx *C, int m, const particle *p, xsval *X)
{
    const orc_problem *P = C->P;
    if (P->xs_kind == 0) {
        int G = C->G;
        X->st = P->sigt[m * G + p->g];
        X->inv_st = C->inv_sigt[m * G + p->g];
        X->sa = C->sig_a[m * G + p->g];
        X->nsf = P->nusigf[m * G + p->g];
        X->nterm = 0;
        return;
    }
    /* CE: per nuclide present, interpolate each reaction on the nuclide's own
     * grid at the largest point E_i <= E: sigma = fma(E - E_i, slope_i, s_i)
     * with slope_i = (s_i+1 - s_i)/(E_i+1 - E_i); macroscopic terms N*sigma
     * accumulated in (nuclide, elastic/capture/fission) order; sigma_t is the
     * running total. */
    double cum = 0.0, sa = 0.0;
    int t = 0;
    for (int n = 0; n < P->n_nuc; ++n) {
        double N = P->mat_dens[m * P->n_nuc + n];
        if (!(N > 0.0)) continue;
        int64_t off = P->nuc_off[n], cnt = P->nuc_off[n + 1] - off;
        int64_t i = orc_nuclide_index(P->nuc_e + off, cnt, p->E);
        int64_t r0 = off + i;
        double dE = p->E - P->nuc_e[r0];
        for (int r = 0; r < 3; ++r) {
            double sig = fma(dE, C->slope[r0 * 3 + r], P->nuc_sig[r0 * 3 + r]);
            double mac = N * sig;
            cum = cum + mac;
            if (r > 0) sa = sa + mac;
            X->cum[t] = cum;
            X->term_nuc[t] = n;
            X->term_r[t] = r;
            X->term_val[t] = mac;
            ++t;
        }
    }
    X->nterm = t;
    X->st = cum;
    X->inv_st = 1.0 / cum;
    X->sa = sa;
    X->nsf = 0.0;
}

/* Macroscopic sigma_t and sigma_a of material m at energy E (continuous
 * energy; pin tests).  Returns ORC_OK or an error. */
int orc_ce_macro(const orc_problem *P, int m, double E, double out[2])
{
    if (P->xs_kind != 1 || m < 0 || m >= P->n_mat) return ORC_ERR_INVALID;
    ctx C;
    int s = setup(&C, P);
    if (s == ORC_OK) {
        particle p;
        memset(&p, 0, sizeof(p));
        p.E = E;
        xsval X;
        xs_lookup(&C, m, &p, &X);
        out[0] = X.st;
        out[1] = X.sa;
    }
    teardown(&C);
    return s;
}


/* ------------------------------------------------------------------------ */
/* Tallies for one straight segment (p0, d, len).                            */
/* Mesh: clip the segment against every voxel slab-wise (Kay-Kajiya slabs)   */
/* over the index box that the segment's end points span, widened by one.    */
/* ------------------------------------------------------------------------ */
static double mesh_plane(const orc_problem *P, int a, int i)
{
    return P->mesh_lo[a] + (P->mesh_hi[a] - P->mesh_lo[a]) * ((double)i / (double)P->mesh_n[a]);
}

static double clip_voxel(const orc_problem *P, const double p0[3], const double d[3], double len, const int idx[3])
{
    double tlo = 0.0, thi = len;
    for (int a = 0; a < 3; ++a) {
        double lo = mesh_plane(P, a, idx[a]), hi = mesh_plane(P, a, idx[a] + 1);
        if (d[a] == 0.0) {
            if (p0[a] < lo || p0[a] >= hi) return 0.0;
            continue;
        }
        double t1 = (lo - p0[a]) / d[a], t2 = (hi - p0[a]) / d[a];
        double tmin = t1 < t2 ? t1 : t2, tmax = t1 < t2 ? t2 : t1;
        if (tmin > tlo) tlo = tmin;
        if (tmax < thi) thi = tmax;
    }
    return thi > tlo ? thi - tlo : 0.0;
}

static void mesh_range(const orc_problem *P, int a, double x0, double x1, int *i0, int *i1)
{
    double lo = x0 < x1 ? x0 : x1, hi = x0 < x1 ? x1 : x0;
    double w = (P->mesh_hi[a] - P->mesh_lo[a]) / (double)P->mesh_n[a];
    double f0 = floor((lo - P->mesh_lo[a]) / w) - 1.0, f1 = floor((hi - P->mesh_lo[a]) / w) + 1.0;
    if (f0 < 0.0) f0 = 0.0;
    if (f1 > (double)(P->mesh_n[a] - 1)) f1 = (double)(P->mesh_n[a] - 1);
    *i0 = (int)f0;
    *i1 = (int)f1;
}

/* Track length of the segment in each mesh cell it crosses, times the
 * weight w, added to the mesh tally (or to out). */
static void score_mesh(ctx *C, const double p0[3], const double d[3], double len, int g, double *out, double w)
{
    const orc_problem *P = C->P;
    if (!P->has_mesh || !(len > 0.0)) return;
    int r0[3], r1[3];
    for (int a = 0; a < 3; ++a) {
        double x1 = p0[a] + len * d[a];
        if ((p0[a] < P->mesh_lo[a] && x1 < P->mesh_lo[a]) || (p0[a] > P->mesh_hi[a] && x1 > P->mesh_hi[a])) return;
        mesh_range(P, a, p0[a], x1, &r0[a], &r1[a]);
        if (r0[a] > r1[a]) return;
    }
    int64_t goff = (P->mesh_by_group && P->xs_kind == 0) ? (int64_t)g * C->mesh_vox : 0;
    int idx[3];
    for (idx[2] = r0[2]; idx[2] <= r1[2]; ++idx[2])
        for (idx[1] = r0[1]; idx[1] <= r1[1]; ++idx[1])
            for (idx[0] = r0[0]; idx[0] <= r1[0]; ++idx[0]) {
                double l = clip_voxel(P, p0, d, len, idx);
                if (l > 0.0) {
                    int64_t v = ((int64_t)idx[2] * P->mesh_n[1] + idx[1]) * P->mesh_n[0] + idx[0];
                    if (out) out[goff + v] += l;
                    else nadd(&C->mesh[goff + v], w * l);
                }
            }
}

double orc_mesh_segment(const orc_problem *P, const double p0[3], const double dir[3], double len, double *mesh)
{
    ctx C;
    memset(&C, 0, sizeof(C));
    C.P = P;
    C.G = P->n_grp;
    C.mesh_vox = (int64_t)P->mesh_n[0] * P->mesh_n[1] * P->mesh_n[2];
    score_mesh(&C, p0, dir, len, 0, mesh, 1.0);
    return len;
}

/* The segment's scores: its track length times the particle's weight (1 in
 * analog runs, so the weighted scores are the plain track lengths). */
static void score_segment(ctx *C, const particle *p, const double p0[3], double len, int m, const xsval *X)
{
    const orc_problem *P = C->P;
    const double wl = p->w * len;
    score_mesh(C, p0, p->d, len, p->g, NULL, p->w);
    nadd(&C->scal[0], wl);
    nadd(&C->scal[1], wl * X->sa);
    nadd(&C->scal[2], wl * X->nsf);
    if (P->n_ebins > 0 && P->xs_kind == 1) {
        const double *e = P->e_edges;
        int nb = P->n_ebins;
        if (p->E >= e[0] && p->E < e[nb]) {
            int lo = 0, hi = nb;          /* e[lo] <= E < e[hi] */
            while (hi - lo > 1) {
                int mid = lo + (hi - lo) / 2;
                if (e[mid] <= p->E) lo = mid; else hi = mid;
            }
            nadd(&C->energy[(int64_t)m * nb + lo], wl);
        }
    }
}

/* Upstream-gradient-weighted contribution of one segment to L:
 * sum over mesh cells of g_mesh * length in the cell (same slab clipping as
 * the mesh tally) + g_flux*len + g_abs*len*sigma_a + g_prod*len*nu_sigma_f. */
static double weighted_segment(const ctx *C, const particle *p, const double p0[3], double len, const xsval *X)
{
    const orc_problem *P = C->P;
    nsum f;
    memset(&f, 0, sizeof(f));
    if (C->gw_mesh && P->has_mesh && len > 0.0) {
        int r0[3], r1[3], ok = 1;
        for (int a = 0; a < 3 && ok; ++a) {
            double x1 = p0[a] + len * p->d[a];
            if ((p0[a] < P->mesh_lo[a] && x1 < P->mesh_lo[a]) || (p0[a] > P->mesh_hi[a] && x1 > P->mesh_hi[a])) ok = 0;
            else {
                mesh_range(P, a, p0[a], x1, &r0[a], &r1[a]);
                if (r0[a] > r1[a]) ok = 0;
            }
        }
        int64_t goff = (P->mesh_by_group && P->xs_kind == 0) ? (int64_t)p->g * C->mesh_vox : 0;
        int idx[3];
        if (ok)
            for (idx[2] = r0[2]; idx[2] <= r1[2]; ++idx[2])
                for (idx[1] = r0[1]; idx[1] <= r1[1]; ++idx[1])
                    for (idx[0] = r0[0]; idx[0] <= r1[0]; ++idx[0]) {
                        double l = clip_voxel(P, p0, p->d, len, idx);
                        if (l > 0.0) {
                            int64_t v = ((int64_t)idx[2] * P->mesh_n[1] + idx[1]) * P->mesh_n[0] + idx[0];
                            nadd(&f, C->gw_mesh[goff + v] * l);
                        }
                    }
    }
    if (C->gw_scal) {
        nadd(&f, C->gw_scal[0] * len);
        nadd(&f, C->gw_scal[1] * (len * X->sa));
        nadd(&f, C->gw_scal[2] * (len * X->nsf));
    }
    return nval(&f);
}

static void record_event(ctx *C, const particle *p, int m, int collided, double len, double f)
{
    if (C->rec_n == C->rec_cap) {
        C->rec_cap = C->rec_cap ? 2 * C->rec_cap : 256;
        C->rec = realloc(C->rec, sizeof(*C->rec) * (size_t)C->rec_cap);
    }
    struct orc_rec *r = &C->rec[C->rec_n++];
    r->m = m; r->g = p->g; r->collided = collided; r->react = 0; r->h = -1; r->len = len; r->f = f;
}

/* ------------------------------------------------------------------------ */
/* Source event (make_work, Sec. 3): n = 0 draws.                            */
/* ------------------------------------------------------------------------ */
static int sample_chi(const ctx *C, int m, double xi)
{
    int G = C->G;
    const double *cc = C->cum_chi + (size_t)m * G;
    double t = xi * cc[G - 1];
    for (int g = 0; g < G; ++g)
        if (t < cc[g]) return g;
    for (int g = G - 1; g >= 0; --g)
        if (C->P->chi[m * G + g] > 0.0) return g;
    return G - 1;
}

static int source_particle(ctx *C, particle *p, uint64_t id, const double *site_pos, int site_g, int site_cell,
                           double site_E)
{
    const orc_problem *P = C->P;
    memset(p, 0, sizeof(*p));
    p->id = id;
    p->alive = 1;
    double xi0[2];
    rng_block(C->seed, C->tag, id, 0, BLK_MAIN, xi0);
    /* direction first (location ties on faces use its sign) */
    if (site_pos || P->src_kind != 0 || P->src_iso) {
        orc_iso_dir(C->seed, C->tag, id, 0, p->d);
    } else {
        p->d[0] = P->src_dir[0]; p->d[1] = P->src_dir[1]; p->d[2] = P->src_dir[2];
    }
    if (site_pos) {
        p->x[0] = site_pos[0]; p->x[1] = site_pos[1]; p->x[2] = site_pos[2];
        int64_t c = site_cell >> 1;
        p->in = site_cell & 1;
        p->ci[0] = (int32_t)(c % P->nx);
        p->ci[1] = (int32_t)((c / P->nx) % P->ny);
        p->ci[2] = (int32_t)(c / ((int64_t)P->nx * P->ny));
        p->g = site_g;
        p->E = site_E;
    } else if (P->src_kind == 0) {
        p->x[0] = P->src_pt[0]; p->x[1] = P->src_pt[1]; p->x[2] = P->src_pt[2];
        locate(P, p);
    } else {
        uint32_t t;
        for (t = 0; t < N_POS_TRIES; ++t) {
            double a[2], b[2];
            rng_block(C->seed, C->tag, id, 0, BLK_POS + 2 * t, a);
            rng_block(C->seed, C->tag, id, 0, BLK_POS + 2 * t + 1, b);
            p->x[0] = P->src_lo[0] + a[0] * (P->src_hi[0] - P->src_lo[0]);
            p->x[1] = P->src_lo[1] + a[1] * (P->src_hi[1] - P->src_lo[1]);
            p->x[2] = P->src_lo[2] + b[0] * (P->src_hi[2] - P->src_lo[2]);
            locate(P, p);
            if (P->src_kind == 1) break;
            if (p->in && P->src_mat[P->pin_mat[cell_lin(P, p)]]) break;
        }
        if (t == N_POS_TRIES) return ORC_ERR_INVALID;
    }
    if (!site_pos) {
        int m = material(P, p);
        if (P->xs_kind == 0) {
            p->g = (P->src_group >= 0) ? P->src_group : sample_chi(C, m, xi0[1]);
        } else {
            p->E = (P->n_cdf > 1) ? orc_cdf_sample(P->cdf_e, P->cdf_p, P->n_cdf, xi0[1]) : P->src_energy;
        }
    }
    p->n = 1;
    p->w = 1.0;
    C->events_by_type[ORC_SOURCE]++;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* One transport event (Sec. 4): distance to collision vs. distance to       */
/* surface, move and score the path, then collide or cross the surface.     */
/* ------------------------------------------------------------------------ */
static void kill(particle *p, int type)
{
    p->alive = 0;
    p->final_type = type;
}

static void bank_site(ctx *C, const particle *p, int g)
{
    if (C->bank_n >= C->bank_cap) {
        C->bank_overflow = 1;
        return;
    }
    uint64_t b = C->bank_n++;
    C->bank_pos[3 * b + 0] = p->x[0];
    C->bank_pos[3 * b + 1] = p->x[1];
    C->bank_pos[3 * b + 2] = p->x[2];
    C->bank_g[b] = g;
    C->bank_cell[b] = cell_id(C->P, p);
    C->bank_E[b] = p->E;
}

static void collide(ctx *C, particle *p, int m, const xsval *X, double xi_react)
{
    const orc_problem *P = C->P;
    p->coll++;
    if (P->xs_kind == 0) {
        int G = C->G;
        /* k-eigenvalue: bank floor(nu_sigma_f/sigma_t/k + xi) sites before the reaction */
        if (C->eig && X->nsf > 0.0) {
            double xf[2];
            rng_block(C->seed, C->tag, p->id, p->n, BLK_FISSION, xf);
            double t = ((X->nsf * X->inv_st) * C->inv_k) + xf[0];
            int nf = (int)floor(t);
            for (int c = 0; c < nf; ++c) {
                double xs[2];
                rng_block(C->seed, C->tag, p->id, p->n, BLK_SITE + (uint32_t)c, xs);
                bank_site(C, p, sample_chi(C, m, xs[0]));
            }
        }
        /* reaction: first g' with xi*sigma_t < running scatter sum, else absorb */
        double t = xi_react * X->st;
        const double *cs = C->cum_s + ((size_t)m * G + p->g) * G;
        int gp = -1;
        for (int h = 0; h < G; ++h)
            if (t < cs[h]) { gp = h; break; }
        if (gp < 0) {
            if (C->recording) C->rec[C->rec_n - 1].react = 2;
            kill(p, ORC_ABSORB);
            C->events_by_type[ORC_ABSORB]++;
            return;
        }
        if (C->recording) {
            C->rec[C->rec_n - 1].react = 1;
            C->rec[C->rec_n - 1].h = gp;
        }
        p->g = gp;
        orc_iso_dir(C->seed, C->tag, p->id, p->n, p->d);
        C->events_by_type[ORC_SCATTER]++;
        return;
    }
    /* continuous energy: first (nuclide, reaction) term with xi*sigma_t below
     * the running sum; if none (rounding), the last term with a positive value */
    double t = xi_react * X->st;
    int sel = -1;
    for (int i = 0; i < X->nterm; ++i)
        if (t < X->cum[i]) { sel = i; break; }
    if (sel < 0)
        for (int i = X->nterm - 1; i >= 0; --i)
            if (X->term_val[i] > 0.0) { sel = i; break; }
    if (sel < 0 || X->term_r[sel] != 0) {
        kill(p, ORC_ABSORB);
        C->events_by_type[ORC_ABSORB]++;
        return;
    }
    double A = P->nuc_awr[X->term_nuc[sel]];
    double E1, nd[3];
    orc_elastic_scatter(C->seed, C->tag, p->id, p->n, A, p->E, p->d, nd, &E1);
    p->d[0] = nd[0]; p->d[1] = nd[1]; p->d[2] = nd[2];
    p->E = E1;
    C->events_by_type[ORC_SCATTER]++;
    if (p->E < P->e_cut) kill(p, ORC_CUTOFF);
}

/* Time tally (our reading of the paper's temporal tally resolution, Sec. 4):
 * the segment occupies [t0, t1] in time; each uniform bin b of width
 * w = t_cen / n_tbins gets the track length spent in it, (hi - lo) / inv_v
 * with [lo, hi] = [t0, t1] clipped to [b w, (b + 1) w]. */
static void score_time(ctx *C, double t0, double t1, double inv_v, double wt)
{
    const orc_problem *P = C->P;
    if (P->n_tbins <= 0 || !(t1 > t0)) return;
    const int nb = P->n_tbins;
    const double w = P->t_cen / (double)nb;
    int b = (int)floor(t0 / w);
    if (b < 0) b = 0;
    for (; b < nb; ++b) {
        double lo = (double)b * w, hi = (double)(b + 1) * w;
        if (lo >= t1) break;
        if (t0 > lo) lo = t0;
        if (t1 < hi) hi = t1;
        if (hi > lo) nadd(&C->time[b], wt * ((hi - lo) / inv_v));
    }
}

/* ------------------------------------------------------------------------ */
/* Closeout (Sec. 4: weights and weight windows for the particle's next loop */
/* iteration).  Our reading: the window of the particle's tally-mesh voxel   */
/* (i_a = floor((x_a - lo_a) (1 / ((hi_a - lo_a) / n_a))), outside the mesh: */
/* none) and group has lower bound L (0: none), upper bound ww_upper L and   */
/* survival weight S = ww_survival L.  Below L: Russian roulette, survive    */
/* with probability w / S (xi S < w, xi the first uniform of block BLK_CLOSE */
/* at the particle's event count n) at weight S, else the history ends as    */
/* CUTOFF.  Above the upper bound: k = min(ceil(w / U), ww_max_split) copies */
/* of weight w / k; the particle continues as copy 0 and copy c = 1..k-1     */
/* takes the stream tag t_c = word 0 of block BLK_SPLIT + c, with bit 31 set,*/
/* xored into the high word of its stream id.  Copies are pushed on the     */
/* family's stack and run after the particle.                                */
/* ------------------------------------------------------------------------ */
static int ww_voxel(const orc_problem *P, const particle *p)
{
    if (!P->has_mesh) return -1;
    int idx[3];
    for (int a = 0; a < 3; ++a) {
        const double w = (P->mesh_hi[a] - P->mesh_lo[a]) / (double)P->mesh_n[a];
        const double t = floor((p->x[a] - P->mesh_lo[a]) * (1.0 / w));
        if (!(t >= 0.0) || !(t < (double)P->mesh_n[a])) return -1;
        idx[a] = (int)t;
    }
    return (idx[2] * P->mesh_n[1] + idx[1]) * P->mesh_n[0] + idx[0];
}

static void closeout(ctx *C, particle *p)
{
    const orc_problem *P = C->P;
    const int v = ww_voxel(P, p);
    if (v < 0) return;
    const int g = P->xs_kind == 0 ? p->g : 0;
    const int G = P->xs_kind == 0 ? C->G : 1;
    const double L = P->ww_lo[(int64_t)v * G + g];
    if (!(L > 0.0)) return;
    if (p->w < L) {
        const double S = P->ww_survival * L;
        double xi[2];
        rng_block(C->seed, C->tag, p->id, p->n, BLK_CLOSE, xi);
        if (xi[0] * S < p->w) {
            p->w = S;
        } else {
            kill(p, ORC_CUTOFF);
        }
        return;
    }
    const double U = P->ww_upper * L;
    if (!(p->w > U)) return;
    int k = (int)ceil(p->w / U);
    if (k > P->ww_max_split) k = P->ww_max_split;
    if (k < 2) return;
    p->w = p->w / (double)k;
    for (int c = 1; c < k; ++c) {
        uint32_t r[4];
        rng_words(C->seed, C->tag, p->id, p->n, BLK_SPLIT + (uint32_t)c, r);
        const uint64_t tag = (uint64_t)(r[0] | 0x80000000u);
        if (C->split_n == C->split_cap) {
            C->split_cap = C->split_cap ? 2 * C->split_cap : 64;
            C->split = realloc(C->split, sizeof(particle) * (size_t)C->split_cap);
        }
        particle q = *p;
        q.id = p->id ^ (tag << 32);
        q.track = 0.0;
        q.coll = 0;
        C->split[C->split_n++] = q;
    }
}

static void event(ctx *C, particle *p)
{
    const orc_problem *P = C->P;
    int m = material(P, p);
    xsval X;
    xs_lookup(C, m, p, &X);
    uint32_t w0[4];
    rng_words(C->seed, C->tag, p->id, p->n, BLK_MAIN, w0);
    double xi[2] = {orc_uniform(w0[0], w0[1]), orc_uniform(w0[2], w0[3])};
    double dcol = exp_sample(C->seed, C->tag, p->id, p->n, w0[0], w0[1]) * X.inv_st;

    /* plane distances along each axis to the exit face in the direction of travel */
    double dp[3];
    for (int a = 0; a < 3; ++a) {
        const double *pl = planes(P, a);
        double dir = p->d[a];
        if (dir > 0.0) dp[a] = (pl[p->ci[a] + 1] - p->x[a]) * (1.0 / dir);
        else if (dir < 0.0) dp[a] = (pl[p->ci[a]] - p->x[a]) * (1.0 / dir);
        else dp[a] = INFINITY;
        if (!(dp[a] > 0.0)) dp[a] = 0.0;   /* clamp; -0.0 becomes +0.0 */
    }
    /* cylinder distance */
    int pin = has_pin(P, p);
    double dcyl = INFINITY;
    if (pin) {
        double c, k, dx, dy;
        pin_terms(P, p, &c, &k, &dx, &dy);
        double a = fma(p->d[0], p->d[0], p->d[1] * p->d[1]);
        if (a > 0.0) {
            double inv_a = 1.0 / a;
            if (p->in) {
                double disc = fma(k, k, -(a * c));
                if (disc < 0.0) disc = 0.0;
                dcyl = (sqrt(disc) - k) * inv_a;
            } else if (k < 0.0) {
                double disc = fma(k, k, -(a * c));
                if (disc >= 0.0) dcyl = ((-k) - sqrt(disc)) * inv_a;
            }
        }
        if (!(dcyl > 0.0)) dcyl = 0.0;
    }
    /* surface selection */
    int cyl_hit;
    double ds;
    if (p->in) {
        cyl_hit = dcyl < dp[2];
        ds = cyl_hit ? dcyl : dp[2];
    } else {
        double dmin = dp[0];
        if (dp[1] < dmin) dmin = dp[1];
        if (dp[2] < dmin) dmin = dp[2];
        cyl_hit = pin && dcyl < dmin;
        ds = cyl_hit ? dcyl : dmin;
    }
    int collided = dcol < ds;
    double dist = collided ? dcol : ds;
    /* timed problems: the census ends the history when it comes strictly
     * before the collision or surface (speed from the group or the energy) */
    int census = 0;
    double inv_v = 0.0;
    if (P->t_cen > 0.0) {
        inv_v = (P->xs_kind == 1) ? 1.0 / (C->v_c * sqrt(p->E)) : P->inv_vel[p->g];
        double left = P->t_cen - p->t;
        double dcen = left > 0.0 ? left / inv_v : 0.0;
        if (dcen < dist) {
            census = 1;
            dist = dcen;
        }
    }

    /* move and score the path */
    double p0[3] = {p->x[0], p->x[1], p->x[2]};
    if (!census && !collided && ds == INFINITY) {
        /* no surface ahead and no collision: the particle escapes */
        kill(p, ORC_LEAK);
        C->events_by_type[ORC_LEAK]++;
        p->n++;
        return;
    }
    p->x[0] = fma(dist, p->d[0], p->x[0]);
    p->x[1] = fma(dist, p->d[1], p->x[1]);
    p->x[2] = fma(dist, p->d[2], p->x[2]);
    score_segment(C, p, p0, dist, m, &X);
    if (P->t_cen > 0.0) {
        double t0 = p->t;
        p->t = census ? P->t_cen : fma(dist, inv_v, p->t);
        score_time(C, t0, p->t, inv_v, p->w);
    }
    p->track += dist;
    if (C->recording) record_event(C, p, m, collided, dist, weighted_segment(C, p, p0, dist, &X));

    if (census) {
        kill(p, ORC_CUTOFF);
        C->events_by_type[ORC_CUTOFF]++;
    } else if (collided) {
        collide(C, p, m, &X, xi[1]);
    } else if (cyl_hit) {
        p->in = !p->in;
        C->events_by_type[ORC_SURF_INTERNAL]++;
    } else {
        int leak = 0, refl = 0, moved_xy = 0, moved_z = 0;
        for (int a = 0; a < 3; ++a) {
            if (p->in && a < 2) continue;   /* inside a pin only the z planes bound the cell */
            if (!(dp[a] == ds)) continue;
            int hi_side = p->d[a] > 0.0;
            int n = nplanes(P, a);
            int boundary = hi_side ? (p->ci[a] == n - 1) : (p->ci[a] == 0);
            if (boundary) {
                int bc = P->bc[2 * a + hi_side];
                if (bc == 1) { p->d[a] = -p->d[a]; refl = 1; }
                else leak = 1;
            } else {
                p->ci[a] += hi_side ? 1 : -1;
                if (a < 2) moved_xy = 1; else moved_z = 1;
            }
        }
        if (leak) {
            kill(p, ORC_LEAK);
            C->events_by_type[ORC_LEAK]++;
        } else {
            if (moved_xy || moved_z) {
                if (!has_pin(P, p) || moved_xy) {
                    p->in = 0;
                } else if (!p->in) {
                    double c, k, dx, dy;
                    pin_terms(P, p, &c, &k, &dx, &dy);
                    p->in = (c < 0.0 || (c == 0.0 && k < 0.0)) ? 1 : 0;
                }
            }
            C->events_by_type[refl ? ORC_SURF_REFLECT : ORC_SURF_INTERNAL]++;
        }
    }
    p->n++;
    if (p->alive && p->n >= C->max_events) kill(p, ORC_MAXEV);
    if (p->alive && P->ww_lo) closeout(C, p);
}

/* ------------------------------------------------------------------------ */
/* Fixed-source driver                                                       */
/* ------------------------------------------------------------------------ */
static void finish_tallies(ctx *C, double norm, double *mesh, double *energy, double scal[3])
{
    const orc_problem *P = C->P;
    int64_t msize = C->mesh_vox * ((P->mesh_by_group && P->xs_kind == 0) ? C->G : 1);
    if (mesh)
        for (int64_t i = 0; i < msize; ++i) mesh[i] = nval(&C->mesh[i]) / norm;
    int64_t esize = (int64_t)P->n_ebins * P->n_mat;
    if (energy)
        for (int64_t i = 0; i < esize; ++i) energy[i] = nval(&C->energy[i]) / norm;
    for (int i = 0; i < 3; ++i) scal[i] = nval(&C->scal[i]) / norm;
}

static void finish_time(ctx *C, double norm, double *out)
{
    if (out)
        for (int b = 0; b < C->P->n_tbins; ++b) out[b] = nval(&C->time[b]) / norm;
}

int orc_fixed_source(const orc_problem *P, orc_fixed *o)
{
    ctx C;
    int st = setup(&C, P);
    if (st) { teardown(&C); return st; }
    C.seed = o->seed;
    C.tag = o->tag;
    C.max_events = o->max_events ? o->max_events : 10000000u;
    memset(o->final_by_type, 0, sizeof(o->final_by_type));
    for (uint64_t i = 0; i < o->n_hist; ++i) {
        const uint64_t id = o->id_offset + i;
        particle p;
        st = source_particle(&C, &p, id, NULL, 0, 0, 0.0);
        if (st) break;
        C.split_n = 0;
        while (p.alive) event(&C, &p);
        o->final_by_type[p.final_type]++;
        if (o->log_n) o->log_n[i] = p.n;
        if (o->log_cell) o->log_cell[i] = cell_id(P, &p);
        if (o->log_type) o->log_type[i] = (uint8_t)p.final_type;
        if (o->hist_track) o->hist_track[i] = p.track;
        if (o->hist_coll) o->hist_coll[i] = p.coll;
        /* split copies of this history (weight windows), depth first */
        while (C.split_n > 0) {
            particle q = C.split[--C.split_n];
            while (q.alive) event(&C, &q);
            o->final_by_type[q.final_type]++;
        }
    }
    finish_tallies(&C, (double)o->n_hist, o->mesh, o->energy, o->scalars);
    finish_time(&C, (double)o->n_hist, o->time_tally);
    memcpy(o->events_by_type, C.events_by_type, sizeof(C.events_by_type));
    teardown(&C);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Sensitivities.  Per history the events are recorded, F = sum_k f_k is the  */
/* history's weighted score, and every random decision d contributes          */
/* s_d * (F - F_before_d), where F_before_d sums the segments completed before */
/* d (a flight decision owns the segment it creates; a reaction decision comes */
/* after it).  Scores:                                                         */
/*   flight ending in a collision   d/dSt = 1/St - len                         */
/*   flight ending at a surface     d/dSt = -len                               */
/*   scatter g -> h                 d/dSs[g->h] = 1/Ss[g->h], d/dSt = -1/St     */
/*   absorption (prob. Sa/St)       d/dSt = 1/Sa - 1/St, d/dSs[g->*] = -1/Sa    */
/* Pathwise terms of f_k: g_abs*len on St and -g_abs*len on every Ss[g->*]   */
/* (Sa = St - sum Ss), g_prod*len on nuSf.  Directions and the source do not   */
/* depend on the cross sections.                                               */
/* ------------------------------------------------------------------------ */
int orc_sensitivities(const orc_problem *P, orc_sens *o)
{
    if (P->xs_kind != 0 || P->t_cen > 0.0 || P->ww_lo) return ORC_ERR_INVALID;   /* untimed analog multigroup only */
    ctx C;
    int st = setup(&C, P);
    if (st) { teardown(&C); return st; }
    C.seed = o->seed;
    C.tag = o->tag;
    C.max_events = o->max_events ? o->max_events : 10000000u;
    C.recording = 1;
    C.gw_mesh = o->g_mesh;
    C.gw_scal = o->g_scal;
    const int M = P->n_mat, G = C.G;
    nsum *dst = calloc((size_t)M * G, sizeof(nsum)), *dss = calloc((size_t)M * G * G, sizeof(nsum));
    nsum *dnf = calloc((size_t)M * G, sizeof(nsum)), val;
    memset(&val, 0, sizeof(val));
    for (uint64_t k = 0; k < o->n_hist && st == ORC_OK; ++k) {
        const uint64_t id = o->id_offset + k;
        particle p;
        C.rec_n = 0;
        st = source_particle(&C, &p, id, NULL, 0, 0, 0.0);
        if (st) break;
        while (p.alive) event(&C, &p);
        nsum Fs;
        memset(&Fs, 0, sizeof(Fs));
        for (int k = 0; k < C.rec_n; ++k) nadd(&Fs, C.rec[k].f);
        const double F = nval(&Fs);
        nadd(&val, F);
        double before = 0.0;
        for (int k = 0; k < C.rec_n; ++k) {
            const struct orc_rec *r = &C.rec[k];
            const int mg = r->m * G + r->g;
            const double inv_st = C.inv_sigt[mg];
            const double after_flight = F - before;
            /* flight decision */
            const double sf = r->collided ? inv_st - r->len : -r->len;
            nadd(&dst[mg], sf * after_flight);
            /* pathwise terms of this segment */
            if (o->g_scal) {
                const double ga = o->g_scal[1] * r->len;
                nadd(&dst[mg], ga);
                for (int h = 0; h < G; ++h) nadd(&dss[(size_t)mg * G + h], -ga);
                nadd(&dnf[mg], o->g_scal[2] * r->len);
            }
            before = before + r->f;
            if (!r->collided) continue;
            const double after = F - before;
            if (r->react == 1) {
                const double ss = P->sigs[(size_t)mg * G + r->h];
                nadd(&dss[(size_t)mg * G + r->h], (1.0 / ss) * after);
                nadd(&dst[mg], (-inv_st) * after);
            } else if (r->react == 2) {
                const double inv_sa = 1.0 / C.sig_a[mg];
                nadd(&dst[mg], (inv_sa - inv_st) * after);
                for (int h = 0; h < G; ++h) nadd(&dss[(size_t)mg * G + h], (-inv_sa) * after);
            }
        }
    }
    const double n = (double)o->n_hist;
    for (int i = 0; i < M * G; ++i) {
        if (o->d_sigt) o->d_sigt[i] = nval(&dst[i]) / n;
        if (o->d_nusigf) o->d_nusigf[i] = nval(&dnf[i]) / n;
    }
    for (int i = 0; i < M * G * G; ++i)
        if (o->d_sigs) o->d_sigs[i] = nval(&dss[i]) / n;
    o->value = nval(&val) / n;
    free(dst); free(dss); free(dnf);
    teardown(&C);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Power iteration (Sec. 4): batches with a fission bank; the bank is kept   */
/* in (parent id, parent event, child) order, which a history-ordered loop   */
/* produces directly; splitting-roulette population control restores the     */
/* batch size: with r = N/M each site gets floor(r) copies plus one more     */
/* with probability r - floor(r).                                            */
/* ------------------------------------------------------------------------ */
int orc_power_iteration(const orc_problem *P, orc_eig *o)
{
    if (P->xs_kind != 0 || P->t_cen > 0.0 || P->ww_lo) return ORC_ERR_INVALID;   /* untimed analog multigroup only */
    ctx C;
    int st = setup(&C, P);
    if (st) { teardown(&C); return st; }
    C.seed = o->seed;
    C.tag = 0;
    C.max_events = o->max_events ? o->max_events : 10000000u;
    C.eig = 1;
    uint64_t cap = o->bank_capacity ? o->bank_capacity : 4 * o->n_per_batch + 64;
    C.bank_cap = cap;
    C.bank_pos = malloc(sizeof(double) * 3 * cap);
    C.bank_g = malloc(sizeof(int32_t) * cap);
    C.bank_cell = malloc(sizeof(int32_t) * cap);
    C.bank_E = malloc(sizeof(double) * cap);
    double *src_pos = malloc(sizeof(double) * 3 * cap);
    int32_t *src_g = malloc(sizeof(int32_t) * cap), *src_cell = malloc(sizeof(int32_t) * cap);
    double *src_E = malloc(sizeof(double) * cap);
    uint32_t nb = o->n_inactive + o->n_active;
    int64_t msize = C.mesh_vox * (P->mesh_by_group ? C.G : 1);
    double *mb = calloc((size_t)(msize > 0 ? msize : 1), sizeof(double));
    nsum *msum = calloc((size_t)(msize > 0 ? msize : 1), sizeof(nsum));
    nsum *msq = calloc((size_t)(msize > 0 ? msize : 1), sizeof(nsum));
    nsum ssum[3], ssq[3], ksum, ksq;
    memset(ssum, 0, sizeof(ssum)); memset(ssq, 0, sizeof(ssq));
    memset(&ksum, 0, sizeof(ksum)); memset(&ksq, 0, sizeof(ksq));
    memset(o->final_by_type, 0, sizeof(o->final_by_type));
    o->log_count = 0;

    double k = o->k0 > 0.0 ? o->k0 : 1.0;
    uint64_t N = o->n_per_batch;
    int have_bank = 0;
    for (uint32_t b = 0; b < nb && st == ORC_OK; ++b) {
        clear_tallies(&C);
        C.bank_n = 0;
        C.bank_overflow = 0;
        C.inv_k = 1.0 / k;
        for (uint64_t i = 0; i < N; ++i) {
            particle p;
            uint64_t id = ((uint64_t)b << 32) | i;
            if (have_bank)
                st = source_particle(&C, &p, id, src_pos + 3 * i, src_g[i], src_cell[i], src_E[i]);
            else
                st = source_particle(&C, &p, id, NULL, 0, 0, 0.0);
            if (st) break;
            while (p.alive) event(&C, &p);
            o->final_by_type[p.final_type]++;
            if (b == o->log_batch && i < cap) {
                if (o->log_n) o->log_n[i] = p.n;
                if (o->log_cell) o->log_cell[i] = cell_id(P, &p);
                if (o->log_type) o->log_type[i] = (uint8_t)p.final_type;
                o->log_count = i + 1;
            }
        }
        if (st) break;
        if (C.bank_overflow) { st = ORC_ERR_CAPACITY; break; }
        uint64_t M = C.bank_n;
        double kb = k * ((double)M / (double)N);
        double scal[3];
        finish_tallies(&C, (double)N, mb, NULL, scal);
        if (o->k_batch) o->k_batch[b] = kb;
        if (o->ktl_batch) o->ktl_batch[b] = scal[2];
        if (o->n_source) o->n_source[b] = N;
        if (o->n_sites) o->n_sites[b] = M;
        if (b >= o->n_inactive) {
            for (int64_t v = 0; v < msize; ++v) { nadd(&msum[v], mb[v]); nadd(&msq[v], mb[v] * mb[v]); }
            for (int i = 0; i < 3; ++i) { nadd(&ssum[i], scal[i]); nadd(&ssq[i], scal[i] * scal[i]); }
            nadd(&ksum, kb); nadd(&ksq, kb * kb);
        }
        k = kb;
        if (M == 0) { st = ORC_ERR_STATE; break; }
        /* splitting roulette to n_per_batch */
        double r = (double)o->n_per_batch / (double)M;
        double fl = floor(r), fr = r - fl;
        uint64_t nn = 0;
        for (uint64_t s = 0; s < M; ++s) {
            uint32_t key[2] = {(uint32_t)o->seed, (uint32_t)(o->seed >> 32) ^ TAG_POPULATION};
            uint32_t ctr[4] = {b, 0u, (uint32_t)s, (uint32_t)(s >> 32)};
            uint32_t rr[4];
            orc_philox4x32_10(ctr, key, rr);
            double xi = orc_uniform(rr[0], rr[1]);
            uint64_t copies = (uint64_t)fl + (xi < fr ? 1u : 0u);
            for (uint64_t c = 0; c < copies; ++c) {
                if (nn >= cap) { st = ORC_ERR_CAPACITY; break; }
                src_pos[3 * nn + 0] = C.bank_pos[3 * s + 0];
                src_pos[3 * nn + 1] = C.bank_pos[3 * s + 1];
                src_pos[3 * nn + 2] = C.bank_pos[3 * s + 2];
                src_g[nn] = C.bank_g[s];
                src_cell[nn] = C.bank_cell[s];
                src_E[nn] = C.bank_E[s];
                ++nn;
            }
            if (st) break;
        }
        N = nn;
        have_bank = 1;
    }
    /* active-batch statistics: mean and standard deviation of the mean */
    double na = (double)o->n_active;
    for (int64_t v = 0; v < msize && st == ORC_OK; ++v) {
        double mean = nval(&msum[v]) / na;
        if (o->mesh_mean) o->mesh_mean[v] = mean;
        if (o->mesh_std) {
            double var = (nval(&msq[v]) / na - mean * mean) / (na - 1.0);
            o->mesh_std[v] = var > 0.0 ? sqrt(var) : 0.0;
        }
    }
    for (int i = 0; i < 3; ++i) {
        double mean = nval(&ssum[i]) / na;
        double var = (nval(&ssq[i]) / na - mean * mean) / (na - 1.0);
        o->scalars_mean[i] = mean;
        o->scalars_std[i] = var > 0.0 ? sqrt(var) : 0.0;
    }
    {
        double mean = nval(&ksum) / na;
        double var = (nval(&ksq) / na - mean * mean) / (na - 1.0);
        o->k_mean = mean;
        o->k_std = var > 0.0 ? sqrt(var) : 0.0;
    }
    memcpy(o->events_by_type, C.events_by_type, sizeof(C.events_by_type));
    free(src_pos); free(src_g); free(src_cell); free(src_E); free(mb); free(msum); free(msq);
    teardown(&C);
    return st;
}
