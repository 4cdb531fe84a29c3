// tr_device.cuh -- device-side problem data, particle state and per-event physics.
//
// Every floating-point operation that decides a branch follows the library's
// arithmetic contract: IEEE binary64, evaluated in the written order, with no
// implicit contraction (-fmad=false); where the contract fuses a product with
// a sum the code calls __fma_rn (one correctly rounded operation): the log
// polynomial and its exponent term, the move, the pin terms, the squared
// transverse direction, the cylinder discriminant and 1 - mu^2 in the
// direction formulas.  Each fused operation also saves an FP64 instruction.
// Where a result is produced with integer
// bit manipulation instead of a double instruction (uniforms, exponent
// extraction, comparisons of non-negative doubles), the integer form yields
// exactly the value the double form would; GB300 issues FP64 at a small
// fraction of its integer rate, so every FP64 instruction saved counts.
//
// Paper context (Cuneo et al., M&C 2025): the transport loop is split into
// events (Sec. 4): source (make_work, Sec. 3), step (move to the next site and
// score the path), collision, surface crossing.  Particles are created through
// an atomic counter and a counter-based random number generator (Sec. 3).
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

#include "tr_fixed.cuh"
#include "tr_softfp.cuh"

namespace tr {

// The transport's correctly rounded reciprocal and square root: the same
// bits as 1.0 / x and sqrt(x).  TR_SOFTFP bit 0 (reciprocal) and bit 1
// (square root) select the integer-pipe versions of tr_softfp.cuh instead
// of the IEEE sequences on the FP64 pipe.  Alone they run 2.1x (reciprocal)
// and 3.0x (square root) the IEEE rate, but inside the transport kernels
// they measured slower (lattice 2.77e9 -> 2.61e9 events/s with both: the
// kernels are not bound by FP64 issue alone), so the default is 0.
#ifndef TR_SOFTFP
#define TR_SOFTFP 0
#endif
__device__ __forceinline__ double tr_rcp(double x) { return (TR_SOFTFP & 1) ? sf_rcp(x) : __drcp_rn(x); }
__device__ __forceinline__ double tr_sqrt(double x) { return (TR_SOFTFP & 2) ? sf_sqrt(x) : __dsqrt_rn(x); }

constexpr int EV_SOURCE = 0, EV_SCATTER = 1, EV_ABSORB = 2, EV_SURF_INTERNAL = 3, EV_SURF_REFLECT = 4,
              EV_LEAK = 5, EV_CUTOFF = 6, EV_MAXEV = 7;
// Outcome of a collision whose scatter leaves the energy below the cutoff:
// the event counts as a scatter and the history ends with final type CUTOFF
// (as an event that reaches the event cap counts as its own type and ends
// with MAXEV).  Never stored: finish_event maps it.
constexpr int EV_SCATTER_CUTOFF = 8;
constexpr int ERR_NONE = 0, ERR_CAPACITY = 3, ERR_TIMEOUT = 4, ERR_INVALID = 1, ERR_RANGE = 5;

// Optional lane-occupancy counters (diagnostic builds with -DTR_PROFILE_LANES
// only): per site, the number of warp arrivals and the active lanes summed.
#ifdef TR_PROFILE_LANES
static __device__ unsigned long long g_lane_prof[64];
// Branch-free: every active lane adds (1 for the group's first lane, else 0)
// and 1, so the counters themselves split no warp.
#define TR_LANES(site)                                                                          \
    do {                                                                                        \
        const unsigned m_ = __activemask();                                                     \
        const unsigned long long lead_ = (int)(threadIdx.x & 31) == __ffs(m_) - 1 ? 1ull : 0ull; \
        atomicAdd(&g_lane_prof[2 * (site)], lead_);                                             \
        atomicAdd(&g_lane_prof[2 * (site) + 1], 1ull);                                          \
    } while (0)
#else
#define TR_LANES(site) \
    do {               \
    } while (0)
#endif

// Random-block assignment within one event (counter word 1).
constexpr uint32_t BLK_MAIN = 0u;      // (distance | source cosine, reaction | source group/energy)
constexpr uint32_t BLK_ANGLE = 1u;     // (CM cosine of an elastic scatter, -)
constexpr uint32_t BLK_FISSION = 2u;   // (fission-site count, -)
constexpr uint32_t BLK_AZIMUTH = 3u;   // 3 + t, t < 64: azimuth rejection tries
constexpr uint32_t N_AZIMUTH = 64u;
constexpr uint32_t BLK_SITE = 100u;    // 100 + c: fission site c
constexpr uint32_t BLK_POS = 200u;     // 200 + 2t, 201 + 2t: source position trial t
constexpr uint32_t N_POS = 1024u;
constexpr uint32_t BLK_ZIG = 3000u;    // 3000 + t: exponential ziggurat, try t's wedge or tail
                                       // uniform (words 2-3) and try t+1's layer and uniform (words 0-1)
constexpr uint32_t N_ZIG = 64u;
constexpr uint32_t BLK_CLOSE = 4000u;  // (closeout roulette, -)
constexpr uint32_t BLK_SPLIT = 4001u;  // 4001 + c: stream tag of split copy c (word 0), c < 64
constexpr int WW_MAX_SPLIT = 64;
constexpr int ZIG_N = 256;             // ziggurat layers
constexpr uint32_t TAG_POP = 0x80000000u;

// next event types of the decomposed schemes (queue ids); DEAD ends the history
constexpr int Q_STEP = 0, Q_COLLIDE = 1, Q_SURFACE = 2, Q_LOOKUP = 3, N_QUEUES = 4, Q_DEAD = 4;
// task decompositions: monolithic (one event per step), decomposed (step,
// collision, surface crossing), decomposed with the cross-section lookup as
// an event of its own (the lookup's values travel with the particle), or
// streaming: steps and surface crossings run inline, up to remap_every steps,
// and only collisions are deferred to a queue of their own
constexpr int DEC_MONO = 0, DEC_SPLIT = 1, DEC_LOOKUP = 2, DEC_STREAM = 3;
__host__ __device__ constexpr int dec_queues(int dec)
{
    return dec == DEC_MONO ? 1 : (dec == DEC_SPLIT ? 3 : (dec == DEC_LOOKUP ? 4 : 2));
}

struct DevProblem {
    // geometry
    int nx, ny, nz;
    const double *xp, *yp, *zp;        // planes
    const double *xc, *yc;             // pin centres per column / row: 0.5 (p[i] + p[i+1])
    const int *cellinfo;               // [nz][ny][nx]: cell material | (pin material + 1) << 16
    int bc[6];
    double r2;                         // pin radius squared
    // cross sections
    int kind, n_mat, G;
    const double *sigt, *inv_sigt, *sig_a, *nusigf, *cum_s, *cum_chi, *chi, *sigs;
    int n_nuc;
    const double *nuc_e, *nuc_sig, *nuc_slope;    // CE rows: energy, 3 cross sections, 3 slopes to the next row
    const double *dens;                // [m][n]
    const double *awr, *inv_ap1sq;     // per nuclide
    double e_cut;
    int n_union;
    const double *ue;                  // union grid energies
    const int *uptr;                   // [u][n] absolute nuclide row of the largest point <= ue[u]
    int n_hash;                        // buckets over the double bit pattern of E
    int hash_shift;
    long long hash_base;
    const int *hash;                   // n_hash + 1: first union index whose bucket >= b
    int hash_smem_off;                 // > 0: this launch's blocks hold hash[] at this byte offset of
                                       // their dynamic shared memory (0: read it from global memory)
    // source
    int src_kind, src_iso, src_group, n_cdf;
    double src_pt[3], src_dir[3], src_lo[3], src_hi[3], src_energy;
    const unsigned char *src_mat;
    const double *cdf_e, *cdf_p;
    // tallies
    int has_mesh, mesh_n[3], by_group, n_ebins, mesh_vox;
    double mesh_lo[3], mesh_hi[3], mesh_w[3], mesh_iw[3];
    const int *cell2vox;               // [nx | ny | nz]: mesh voxel holding geometry cell i on that axis, or -1
    int mesh_walk;                     // some cell lies in no single mesh voxel: its segments take the mesh walk
    int walk_smem_off;                 // > 0: this launch's warps queue those segments (WalkQ) at this byte
                                       // offset of their dynamic shared memory (the monolithic asynchronous kernel)
    const double *e_edges;
    int mesh_size, energy_size;
    // time: histories start at t = 0 and end at the census time t_cen (timed
    // problems only); speeds from inv_vel[g] (MG, s/cm) or v_c sqrt(E) (CE);
    // n_tbins uniform flux bins of width tb_w over [0, t_cen)
    int timed, n_tbins;
    double t_cen, tb_w, v_c;
    const double *inv_vel;
    // logarithm table: {1/c_k, -log(1/c_k)} pairs (see tr_log)
    const double* log_tab;
    // exponential ziggurat: {W_i, C_i} pairs, then {f_i, df_i} pairs (see exp_sample)
    const double* zig_tab;
    // weight windows (closeout): lower bound per mesh voxel and group, or null
    const double* ww_lo;
    double ww_up, ww_surv;
    int ww_max_split;
};

// Per-run parameters.
struct RunParams {
    uint64_t n_hist;
    uint32_t key0, key1;               // (seed_lo, seed_hi ^ tag)
    uint32_t id_hi;                    // batch index (eigenvalue) or 0
    uint32_t id_base;                  // first history of a fixed-source shard (random-stream id offset)
    uint32_t max_events;
    int eig;
    double inv_k;
    int want_log;
    int remap_every;
    uint64_t max_spin;
    uint64_t max_wait_ns;              // wall-clock limit of one spin-wait (global timer)
    int spill_threshold;
};

// Device global timer in nanoseconds (bounds spin-waits in wall-clock time).
__device__ __forceinline__ uint64_t now_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Structure-of-arrays particle storage (global memory stacks and links).
// Fields: position, direction, cached reciprocals of the direction
// components and of u^2 + v^2 (pure functions of the direction, stored so
// that a surface event does not repeat four divisions), energy (CE) or
// group (MG), packed cell, history index, event count, banked-site count, the
// pending surface flags of the decomposed scheme and the problem index of a
// batched launch; the history's running scalar scores (track length,
// absorption and production, summed in event order); with the lookup event,
// the cached cross sections (Sigma_t, 1/Sigma_t, Sigma_a, nu Sigma_f).
struct SoA {
    double *x, *y, *z, *u, *v, *w, *iu, *iv, *iw, *ia, *E, *t;
    double *hf, *ha, *hp;
    double *wt;                        // weight (weight-window problems)
    unsigned *sid;                     // stream tag of a split copy (weight-window problems)
    double *xst, *xist, *xsa, *xnsf;
    int *g;
    unsigned *cell, *id, *n, *nsites, *pend, *prob;
};

struct Particle {
    double x, y, z, u, v, w;
    double iu, iv, iw, ia;
    double E;
    double t;                          // time since the source (timed problems)
    // the history's scalar scores so far (track length, absorption,
    // production), summed in event order: the same value whatever the
    // schedule; converted to fixed point once, when the history ends
    double hf, ha, hp;
    double xst, xist, xsa, xnsf;       // lookup-event decomposition: cross sections of (material, E or g)
    // weight-window problems: the weight (1 at birth); the stream tag of a
    // split copy (0 for a source history; xored into the stream's high word);
    // copies the closeout asked for after the last event
    double wt;
    unsigned sid, nsplit;
    int g;
    unsigned cell;                     // i | j << 10 | k << 20 | inside << 30
    unsigned id, n, nsites, pend;
    unsigned prob;                     // problem index within a batched launch (0 otherwise)
};

struct ErrorWord {
    int code;
    int where;
};

// Tally accumulators written by kernels: raw fixed-point sums (tr_fixed.cuh),
// converted and normalised after the run.
struct Tallies {
    FixBin *mesh;                      // mesh_size
    FixBin *energy;                    // energy_size
    FixBin *scal;                      // 3: flux, absorption, production
    FixBin *time;                      // n_tbins (timed problems)
    unsigned long long *ev_type;       // 8 event counts
    unsigned long long *fin_type;      // 8 final-type counts
    uint32_t *log_n;
    int32_t *log_cell;
    uint8_t *log_type;
    ErrorWord *err;                    // a contribution beyond the fixed-point range sets ERR_RANGE
    // per history (indexed by the history index): its scalar scores at its
    // end (track length, absorption, production), summed later in a fixed
    // order; null: each ended history adds them to scal in fixed point
    double *hist_f, *hist_a, *hist_p;
};

// Record a contribution beyond the fixed-point range (never expected: it
// needs a single track-length score of 2^39).
__device__ __forceinline__ void tally_range_error(const Tallies& T)
{
    if (T.err) atomicCAS(&T.err->code, 0, ERR_RANGE);
}

// Fission bank (unordered during a batch; ordered by (parent, site) later).
struct Bank {
    double *x, *y, *z;
    int *g;
    unsigned *cell;
    unsigned long long *key;           // parent index << 32 | site sequence
    unsigned long long *count;
    unsigned long long capacity;
    unsigned *site_count;              // per parent: sites banked (written at death)
};

// ---------------------------------------------------------------------------
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                          uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return make_uint4(c0, c1, c2, c3);
}

// ((w >> 12) + 1/2) 2^-52 built directly as a binary64 bit pattern:
// v = 2 (w >> 12) + 1 < 2^53 is normalised with a leading-zero count, so the
// value v 2^-53 is exact and no FP64 instruction is spent.
__device__ __forceinline__ double u01(uint32_t lo, uint32_t hi)
{
    const unsigned long long w = ((unsigned long long)hi << 32) | lo;
    const unsigned long long v = ((w >> 12) << 1) | 1ull;
    const int sh = __clzll((long long)v) - 11;
    const unsigned long long mant = (v << sh) & 0x000FFFFFFFFFFFFFull;
    const unsigned long long ex = (unsigned long long)(1022 - sh);
    return __longlong_as_double((long long)((ex << 52) | mant));
}

struct Stream {
    uint32_t k0, k1, id_lo, id_hi;
    __device__ __forceinline__ uint4 block(uint32_t n, uint32_t j) const { return philox10(n, j, id_lo, id_hi, k0, k1); }
    __device__ __forceinline__ double first(uint32_t n, uint32_t j) const
    {
        const uint4 r = block(n, j);
        return u01(r.x, r.y);
    }
};

// Comparisons answered on the bit patterns with integer instructions (no NaN
// reaches them): non-negative doubles and +inf order like their bit patterns,
// and the sign tests below treat -0.0 exactly as the double comparisons do.
__device__ __forceinline__ long long dbits(double d) { return __double_as_longlong(d); }
__device__ __forceinline__ bool lt_nn(double a, double b) { return dbits(a) < dbits(b); }   // a < b, a, b >= +0
__device__ __forceinline__ bool gt0(double x) { return dbits(x) > 0; }                       // x > 0
__device__ __forceinline__ bool lt0(double x) { return dbits(x) < 0 && (dbits(x) << 1) != 0; }  // x < 0
__device__ __forceinline__ bool ge0(double x) { return !lt0(x); }                            // x >= 0
// floor(x) for x >= 0 from the bits (integer instructions only); 2^31 - 1
// from 2^31 on, as the saturating conversion gives
__device__ __forceinline__ int floor_nn(double x)
{
    const long long b = dbits(x);
    const int e = (int)((b >> 52) & 0x7FF) - 1023;
    if (e < 0) return 0;
    if (e > 30) return 0x7FFFFFFF;
    const long long m = (b & 0x000FFFFFFFFFFFFFll) | 0x0010000000000000ll;
    return (int)(m >> (52 - e));
}
// -x by flipping the sign bit (an integer instruction; the same value)
__device__ __forceinline__ double flip_sign(double x)
{
    return __longlong_as_double(dbits(x) ^ (long long)0x8000000000000000ull);
}
// max(d, +0) with -0 and negatives mapped to +0 (no NaN reaches here)
__device__ __forceinline__ double clamp0(double d) { return dbits(d) <= 0 ? 0.0 : d; }

// ---------------------------------------------------------------------------
// Natural logarithm, table-driven (P. T. P. Tang, ACM TOMS 16 (1990) 378):
// x = 2^e m with m in [sqrt(1/2), sqrt(2)]; c_k = 1 + k/128 is the table point
// nearest m (k from the mantissa bits, integer only); r = m (1/c_k) - 1 in one
// rounding; log x = e ln2 + T_k + log1p(r), with T_k = -log(1/c_k) and
// log1p(r) = r + r^2 q(r), q the Taylor terms through r^7/7 (|r| < 2^-7.4).
// For k = 0, 1/c_k = 1 and r = m - 1 exactly.  ln 2 is split at 40 bits, so
// e LN2_HI is exact.  The table, {1/c_k, T_k} for k = LOG_KMIN..LOG_KMAX,
// is built on the host from the atanh series and travels with the problem.
// ---------------------------------------------------------------------------
constexpr int LOG_KMIN = -38, LOG_KMAX = 54, LOG_TAB_N = LOG_KMAX - LOG_KMIN + 1;

__device__ __forceinline__ double tr_log(const double* __restrict__ tab, double x)
{
    const long long b = __double_as_longlong(x);
    const long long f = b & 0x000FFFFFFFFFFFFFll;
    int e = (int)((b >> 52) & 0x7FF) - 1023;
    long long mb = f | 0x3FF0000000000000ll;
    int k = (int)((f + (1ll << 44)) >> 45);              // m in [1, sqrt 2]: round((m - 1) 128)
    if (mb > 0x3FF6A09E667F3BCDll) {                     // m > sqrt(2): halve m (exact), bump e
        mb -= 0x0010000000000000ll;
        e += 1;
        k = (int)((f + (1ll << 45)) >> 46) - 64;         // m/2 in (sqrt(1/2), 1): round((m/2 - 1) 128)
    }
    const double m = __longlong_as_double(mb);
    const double2 t = __ldg(reinterpret_cast<const double2*>(tab) + (k - LOG_KMIN));
    const double r = __fma_rn(m, t.x, -1.0);
    double q = 1.0 / 7.0;
    q = __fma_rn(q, r, -1.0 / 6.0);
    q = __fma_rn(q, r, 1.0 / 5.0);
    q = __fma_rn(q, r, -0.25);
    q = __fma_rn(q, r, 1.0 / 3.0);
    q = __fma_rn(q, r, -0.5);
    const double p = __fma_rn(q, r * r, r);
    const double de = (double)e;
    return __fma_rn(de, __longlong_as_double(0x3FE62E42FEFA4000ll),
                    __fma_rn(de, __longlong_as_double((long long)0xBD48432A1B0E2634ull), t.y + p));
}

// ---------------------------------------------------------------------------
// Exponential variate (the distance to collision in mean free paths) by the
// ziggurat method of Marsaglia and Tsang (J. Stat. Softw. 5, 2000): 256
// layers of equal area v under f(x) = e^-x.  Layer 0 is the base rectangle
// [0, W_0 = v/f(r)] x [0, f(r)] with the tail beyond r; layer i >= 1 is
// [0, X_i] x [f(X_i), f(X_i+1)], X_1 = r, X_256 = 0.  A try takes layer i
// (low 8 bits of its word pair) and the pair's uniform U: x = U W_i is
// accepted below the inner width C_i (C_0 = r, C_i = X_i+1), about 99 % of
// tries, with one multiplication.  Otherwise, with the uniform U2 of words
// 2-3 of block BLK_ZIG + t: layer 0 returns r - log U2 (the tail is
// memoryless); layer i accepts x if x < -log(fma(U2, df_i, f_i)) (under the
// curve), else try t+1 takes words 0-1 of that block.  The table
// ({W_i, C_i}, {f_i, df_i = f_i+1 - f_i}) is built at problem creation.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double exp_sample(const DevProblem& P, const Stream& S, uint32_t n, uint32_t lo, uint32_t hi)
{
    // (the rejection part stays inline: with ~25 lanes per warp a warp takes
    // it in about a fifth of its steps, and out of line it measured slower)
    const double2* wc = reinterpret_cast<const double2*>(P.zig_tab);
    const double2* fd = wc + ZIG_N;
    int i = (int)(lo & 0xFFu);
    double U = u01(lo, hi);
    double2 t = __ldg(wc + i);
    double x = U * t.x;
    if (lt_nn(x, t.y)) return x;
    for (uint32_t k = 0; k < N_ZIG; ++k) {
        const uint4 w = S.block(n, BLK_ZIG + k);
        const double U2 = u01(w.z, w.w);
        if (i == 0) return t.y - tr_log(P.log_tab, U2);
        const double2 f = __ldg(fd + i);
        const double y = __fma_rn(U2, f.y, f.x);
        if (lt_nn(x, -tr_log(P.log_tab, y))) return x;
        i = (int)(w.x & 0xFFu);
        U = u01(w.x, w.y);
        t = __ldg(wc + i);
        x = U * t.x;
        if (lt_nn(x, t.y)) return x;
    }
    return -tr_log(P.log_tab, U);   // after N_ZIG rejected tries (probability below 1e-100)
}

// ---------------------------------------------------------------------------
// Directions: a point of the unit disk by rejection in the unit square (no
// trig), giving the azimuth and the isotropic direction; lab rotation,
// target-at-rest elastic kinematics.
// ---------------------------------------------------------------------------
// One rejection try t: the point (a, b) and whether 0 < a^2 + b^2 <= 1.
__device__ __forceinline__ bool azimuth_try(const Stream& S, uint32_t n, uint32_t t, double& a, double& b, double& a2,
                                            double& b2, double& s)
{
    const uint4 r = S.block(n, BLK_AZIMUTH + t);
    a = __fma_rn(2.0, u01(r.x, r.y), -1.0);   // 2 xi is exact: the same value as 2.0 * xi - 1.0
    b = __fma_rn(2.0, u01(r.z, r.w), -1.0);
    a2 = a * a;
    b2 = b * b;
    s = a2 + b2;
    return dbits(s) <= dbits(1.0) && gt0(s);   // 0 < s <= 1 (s >= +0)
}

// The first accepted rejection try: (a, b) uniform in the unit disk, s =
// a^2 + b^2.  sm: the lanes of this warp that call it together (a mask every
// one of them passes, computed by a ballot), regrouped after the rejection
// loop; 0 = no regrouping.
__device__ __forceinline__ void disk_point(const Stream& S, uint32_t n, double& a, double& b, double& a2, double& b2,
                                           double& s, unsigned sm)
{
    // tries 0 and 1 run unconditionally in every lane (both accepted: take
    // try 0), the rare remainder loops
    TR_LANES(18);
    double a1, b1, a21, b21, s1;
    bool ok = azimuth_try(S, n, 0u, a, b, a2, b2, s);
    const bool ok1 = azimuth_try(S, n, 1u, a1, b1, a21, b21, s1);
    if (!ok && ok1) {
        a = a1; b = b1; a2 = a21; b2 = b21; s = s1;
        ok = true;
    }
    // (the retries stay inline: with ~16 scattering lanes a warp needs them
    // in about half of its collision passes)
    for (uint32_t t = 2; !ok && t < N_AZIMUTH; ++t) {
        TR_LANES(6);
        ok = azimuth_try(S, n, t, a, b, a2, b2, s);
    }
    if (!ok) {
        a = 1.0; b = 0.0; a2 = 1.0; b2 = 0.0; s = 1.0;
    }
    if (sm) __syncwarp(sm);
    TR_LANES(19);
}

// Azimuth (cos phi, sin phi) = ((a^2 - b^2)/s, 2ab/s) from the disk point.
__device__ __forceinline__ void azimuth(const Stream& S, uint32_t n, double& cphi, double& sphi, unsigned sm = 0u)
{
    double a, b, a2, b2, s;
    disk_point(S, n, a, b, a2, b2, s, sm);
    const double inv_s = sf_rcp(s);   // continuous energy only: on the integer pipe (the same bits)
    cphi = (a2 - b2) * inv_s;
    sphi = (2.0 * (a * b)) * inv_s;
}

// SOFT: the reciprocals on the integer pipe (sf_rcp, the same bits), for
// the continuous-energy scatter, whose kernels are the most FP64-bound.
template <bool SOFT = false>
__device__ __forceinline__ void set_reciprocals(Particle& p)
{
    TR_LANES(20);
    // (bits << 1) != 0 is x != +-0
    // tr_rcp is the correctly rounded reciprocal: the same value as 1.0 / x
    p.iu = (dbits(p.u) << 1) ? (SOFT ? sf_rcp(p.u) : tr_rcp(p.u)) : 0.0;
    p.iv = (dbits(p.v) << 1) ? (SOFT ? sf_rcp(p.v) : tr_rcp(p.v)) : 0.0;
    p.iw = (dbits(p.w) << 1) ? (SOFT ? sf_rcp(p.w) : tr_rcp(p.w)) : 0.0;
    const double a = __fma_rn(p.u, p.u, p.v * p.v);
    p.ia = gt0(a) ? (SOFT ? sf_rcp(a) : tr_rcp(a)) : 0.0;
}

// Isotropic direction (Marsaglia, Ann. Math. Stat. 43 (1972) 645): with the
// disk point (a, b), s = a^2 + b^2, (1 - 2s, 2a sqrt(1 - s), 2b sqrt(1 - s))
// is uniform on the unit sphere; no division and one square root.
// SOFT: the square root and the reciprocals on the integer pipe (the same
// bits; the source pre-sampling kernel, where it measured faster).
template <bool SOFT = false>
__device__ __forceinline__ void iso_dir(const Stream& S, uint32_t n, Particle& p, unsigned sm = 0u)
{
    double a, b, a2, b2, s;
    disk_point(S, n, a, b, a2, b2, s, sm);
    const double t = 2.0 * (SOFT ? sf_sqrt(1.0 - s) : tr_sqrt(1.0 - s));
    p.u = __fma_rn(-2.0, s, 1.0);   // 2 s is exact: the same value as 1.0 - 2.0 * s
    p.v = a * t;
    p.w = b * t;
    set_reciprocals<SOFT>(p);
}

__device__ __forceinline__ void rotate(Particle& p, double mu, double cphi, double sphi)
{
    double t = __fma_rn(-mu, mu, 1.0);
    if (lt0(t)) t = 0.0;
    const double st = sf_sqrt(t);   // the rotation (continuous energy only): square roots on the integer pipe
    const double u = p.u, v = p.v, w = p.w;
    // |w| > 0.9999999999 and w > 0 on the bit patterns (integer instructions)
    if ((dbits(w) & 0x7FFFFFFFFFFFFFFFll) > dbits(0.9999999999)) {
        p.u = st * cphi;
        p.v = st * sphi;
        p.w = gt0(w) ? mu : -mu;
    } else {
        const double sq = sf_sqrt(__fma_rn(-w, w, 1.0));
        const double a1 = st / sq;
        p.u = mu * u + a1 * ((u * w) * cphi - v * sphi);
        p.v = mu * v + a1 * ((v * w) * cphi + u * sphi);
        p.w = mu * w - (st * sq) * cphi;
    }
    set_reciprocals<true>(p);
}

// ---------------------------------------------------------------------------
// Geometry helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int cell_i(unsigned c) { return (int)(c & 1023u); }
__device__ __forceinline__ int cell_j(unsigned c) { return (int)((c >> 10) & 1023u); }
__device__ __forceinline__ int cell_k(unsigned c) { return (int)((c >> 20) & 1023u); }
__device__ __forceinline__ int cell_in(unsigned c) { return (int)(c >> 30); }
__device__ __forceinline__ unsigned pack_cell(int i, int j, int k, int in)
{
    return (unsigned)i | ((unsigned)j << 10) | ((unsigned)k << 20) | ((unsigned)in << 30);
}
__device__ __forceinline__ int cell_lin(const DevProblem& P, unsigned c)
{
    return (cell_k(c) * P.ny + cell_j(c)) * P.nx + cell_i(c);
}
__device__ __forceinline__ int cell_id(const DevProblem& P, unsigned c) { return cell_lin(P, c) * 2 + cell_in(c); }
__device__ __forceinline__ int cell_info(const DevProblem& P, unsigned c) { return __ldg(P.cellinfo + cell_lin(P, c)); }
__device__ __forceinline__ int info_pin(int info) { return (info >> 16) - 1; }
__device__ __forceinline__ int info_mat(int info) { return info & 0xFFFF; }
__device__ __forceinline__ int material(const DevProblem& P, unsigned c)
{
    const int info = cell_info(P, c);
    return cell_in(c) ? info_pin(info) : info_mat(info);
}

// c = (dx^2 + dy^2) - r^2 and k = dx u + dy v about the centre of the cell's pin
__device__ __forceinline__ void pin_terms(const DevProblem& P, const Particle& p, double& c, double& k)
{
    const double dx = p.x - __ldg(P.xc + cell_i(p.cell));
    const double dy = p.y - __ldg(P.yc + cell_j(p.cell));
    c = __fma_rn(dx, dx, dy * dy) - P.r2;
    k = __fma_rn(dx, p.u, dy * p.v);
}

// largest i in [0, n-1] with pl[i] <= x; one cell down when x sits exactly on
// an interior plane and the direction component is negative
__device__ __forceinline__ int locate_axis(const double* pl, int n, double x, double dir)
{
    int lo = 0, hi = n;                 // pl[lo] <= x (or lo = 0), answer in [lo, hi)
    while (hi - lo > 1) {
        TR_LANES(9);
        const int mid = (lo + hi) >> 1;
        if (__ldg(pl + mid) <= x) lo = mid; else hi = mid;
    }
    if (lo > 0 && x == __ldg(pl + lo) && dir < 0.0) lo -= 1;
    return lo;
}

__device__ __forceinline__ void locate(const DevProblem& P, Particle& p)
{
    const int i = locate_axis(P.xp, P.nx, p.x, p.u);
    const int j = locate_axis(P.yp, P.ny, p.y, p.v);
    const int k = locate_axis(P.zp, P.nz, p.z, p.w);
    p.cell = pack_cell(i, j, k, 0);
    if (info_pin(cell_info(P, p.cell)) >= 0) {
        double c, kk;
        pin_terms(P, p, c, kk);
        if (c < 0.0) p.cell |= 1u << 30;
    }
}

// ---------------------------------------------------------------------------
// Cross sections
// ---------------------------------------------------------------------------
// Macroscopic terms of a continuous-energy lookup, kept for the collision
// that follows in the same event, so that it selects its (nuclide, reaction)
// without repeating the union-grid search and the interpolations.
constexpr int CE_KEEP_NUC = 4;
struct CEKeep {
    int n;                             // present nuclides kept, or -1 (more than CE_KEEP_NUC: recompute)
    int nuc[CE_KEEP_NUC];              // their indices, in order
    double mac[3 * CE_KEEP_NUC];       // N (s0 + f (s1 - s0)) per kept nuclide and reaction
    double st, xi;                     // a deferred collision: sigma_t and the reaction draw of its step
};

struct XS {
    double st, inv_st, sa, nsf;
    CEKeep* keep = nullptr;            // continuous energy: where the lookup leaves its terms, if anywhere
};

__device__ __forceinline__ void xs_mg(const DevProblem& P, int m, int g, XS& X)
{
    const int o = m * P.G + g;
    X.st = __ldg(P.sigt + o);
    X.inv_st = __ldg(P.inv_sigt + o);
    X.sa = __ldg(P.sig_a + o);
    X.nsf = __ldg(P.nusigf + o);
}

// Union-grid index: largest u in [0, n_union-2] with ue[u] <= E.  The hash
// buckets the double bit pattern of E (exponent + leading mantissa bits, a
// piecewise-linear log2), giving a short range for a binary search that
// compares bit patterns (all energies are positive).
extern __shared__ __align__(16) unsigned char tr_dyn_smem[];

__device__ __forceinline__ int union_index(const DevProblem& P, double E)
{
    const long long eb = dbits(E);
    long long bkt = (eb >> P.hash_shift) - P.hash_base;
    if (bkt < 0) bkt = 0;
    if (bkt > P.n_hash - 1) bkt = P.n_hash - 1;
    int lo, hi;
    if (P.hash_smem_off) {
        const int* h = reinterpret_cast<const int*>(tr_dyn_smem + P.hash_smem_off);
        lo = h[bkt] - 1;
        hi = h[bkt + 1];
    } else {
        lo = __ldg(P.hash + bkt) - 1;
        hi = __ldg(P.hash + bkt + 1);
    }
    if (lo < 0) lo = 0;
    if (hi > P.n_union - 1) hi = P.n_union - 1;
    // invariant: ue[lo] <= E < ue[hi] (or boundaries)
    if (eb < dbits(__ldg(P.ue + lo))) lo = 0;
    if (eb >= dbits(__ldg(P.ue + hi))) return (hi >= P.n_union - 1) ? P.n_union - 2 : hi;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (dbits(__ldg(P.ue + mid)) <= eb) lo = mid; else hi = mid;
    }
    return lo;
}

// CE macroscopic totals at the particle energy: per present nuclide (density
// > 0, index order) and reaction (elastic, capture, fission) the term
// N * fma(E - E_i, slope_i, s_i), E_i the largest grid point <= E and
// slope_i = (s_i+1 - s_i) / (E_i+1 - E_i) stored per row; sigma_t is the
// running sum, sigma_a the capture + fission part.
__device__ __forceinline__ void xs_ce(const DevProblem& P, int m, double E, XS& X)
{
    const int u = union_index(P, E);
    double cum = 0.0, sa = 0.0;
    int kept = 0;
#pragma unroll 4   // (measured slightly faster: the nuclides' loads issue together)
    for (int n = 0; n < P.n_nuc; ++n) {
        const double N = __ldg(P.dens + m * P.n_nuc + n);
        if (!gt0(N)) continue;
        const int r0 = __ldg(P.uptr + (long long)u * P.n_nuc + n);
        const double dE = E - __ldg(P.nuc_e + r0);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const double s0 = __ldg(P.nuc_sig + 3 * (long long)r0 + r);
            const double mac = N * __fma_rn(dE, __ldg(P.nuc_slope + 3 * (long long)r0 + r), s0);
            if (X.keep && kept < CE_KEEP_NUC) X.keep->mac[3 * kept + r] = mac;
            cum = cum + mac;
            if (r > 0) sa = sa + mac;
        }
        if (X.keep && kept < CE_KEEP_NUC) X.keep->nuc[kept] = n;
        ++kept;
    }
    if (X.keep) X.keep->n = kept <= CE_KEEP_NUC ? kept : -1;
    X.st = cum;
    X.inv_st = sf_rcp(cum);   // on the integer pipe: the FP64 pipe is the CE kernels' bound (the same bits as 1.0 / cum)
    X.sa = sa;
    X.nsf = 0.0;
}

template <bool CE>
__device__ __forceinline__ void xs_lookup(const DevProblem& P, const Particle& p, int m, XS& X)
{
    if (CE) xs_ce(P, m, p.E, X);
    else xs_mg(P, m, p.g, X);
}

__device__ __forceinline__ int sample_chi(const DevProblem& P, int m, double xi)
{
    // the first g with t < cc[g]; if none (rounding), the last group with
    // chi > 0, else G - 1.  Every lane runs all G steps (no early exit that
    // would split the warp).
    const double* cc = P.cum_chi + m * P.G;
    const double t = xi * __ldg(cc + P.G - 1);
    int sel = -1, last = P.G - 1;
    for (int g = 0; g < P.G; ++g) {
        sel = (sel < 0 && lt_nn(t, __ldg(cc + g))) ? g : sel;   // non-negative: integer compares
        last = gt0(__ldg(P.chi + m * P.G + g)) ? g : last;
    }
    return sel >= 0 ? sel : last;
}

__device__ __forceinline__ double cdf_sample(const DevProblem& P, double xi)
{
    // largest k <= n-2 with p[k] <= xi, then linear interpolation
    int lo = 0, hi = P.n_cdf - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(P.cdf_p + mid) <= xi) lo = mid; else hi = mid;
    }
    const double e0 = __ldg(P.cdf_e + lo), e1 = __ldg(P.cdf_e + lo + 1);
    const double p0 = __ldg(P.cdf_p + lo), p1 = __ldg(P.cdf_p + lo + 1);
    return e0 + (xi - p0) * (e1 - e0) / (p1 - p0);
}

}  // namespace tr
