// tr_events.cuh -- the transport events (Sec. 4 of Cuneo et al., M&C 2025):
// source (make_work), step (cross-section lookup, distance to collision vs.
// distance to surface, move, track-length tally), collision and surface
// crossing.  The monolithic task scheme runs step + collision/surface as one
// event; the decomposed scheme runs them as separate events with a remap in
// between.  The event counter n (which keys the random numbers) advances once
// per collision or surface outcome, so both schemes produce identical
// histories.
#pragma once
#include "tr_device.cuh"

namespace tr {

// pending-outcome flags left by the step event for the decomposed scheme
constexpr unsigned PEND_X = 1u, PEND_Y = 2u, PEND_Z = 4u, PEND_CYL = 8u, PEND_ESCAPE = 16u, PEND_COLLIDE = 32u,
                   PEND_CENSUS = 64u;

// Per-thread accumulators: event counts, and the fixed-point sums
// (tr_fixed.cuh) of the scalar scores of the histories this thread ended.
// Those sums live in shared memory (fx: three per thread), or fx is null and
// each ended history goes to its tally bins directly.
struct Acc {
    long long* fx;
    unsigned ev[8];
    unsigned fin[8];
    __device__ __forceinline__ void zero()
    {
        fx = nullptr;
#pragma unroll
        for (int i = 0; i < 8; ++i) ev[i] = fin[i] = 0u;
    }
};

// Shared-memory words per thread for Acc::fx.
constexpr int ACC_FX_WORDS = 3;

// Points acc at this thread's three fixed-point sums in `base` (block-wide
// array of blockDim.x * 3 words) and clears them.
__device__ __forceinline__ void acc_attach(Acc& acc, long long* base)
{
    acc.fx = base + 3 * threadIdx.x;
    acc.fx[0] = acc.fx[1] = acc.fx[2] = 0;
}

// A history's scalar scores at its end, when no per-history buffer is given
// (the allocation-free entry, batched launches, runs above 2^26 histories):
// each rounded once to fixed point and added to this thread's sums (spilled
// to the bin before they could overflow), or straight to the bin.  Out of
// line, so that the kernels' hot loops carry only the call.
static __device__ __noinline__ void acc_history_sums(long long* fx, FixBin* scal, ErrorWord* err, double hf,
                                                     double ha, double hp)
{
    const double h[3] = {hf, ha, hp};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double c = h[k];
        if (fx && fix_small(c)) {
            long long s = fx[k] + fix_round(c);
            if (fix_sum_full(s)) {
                fix_add_sum(scal + k, s);
                s = 0;
            }
            fx[k] = s;
        } else if (dbits(c) << 1) {
            if (!fix_add(scal + k, c) && err) atomicCAS(&err->code, 0, ERR_RANGE);
        }
    }
}

__device__ __forceinline__ Stream make_stream(const RunParams& R, unsigned id)
{
    Stream S;
    S.k0 = R.key0;
    S.k1 = R.key1;
    S.id_lo = R.id_base + id;
    S.id_hi = R.id_hi;
    return S;
}

// The particle's random stream: its history's, with a split copy's stream
// tag xored into the high word (weight-window problems).
template <bool WW>
__device__ __forceinline__ Stream particle_stream(const RunParams& R, const Particle& p)
{
    Stream S = make_stream(R, p.id);
    if (WW) S.id_hi ^= p.sid;
    return S;
}

// ---------------------------------------------------------------------------
// Track-length mesh tally.  A segment never leaves its geometry cell; when
// that cell lies inside one mesh cell on every axis (precomputed per axis)
// the whole length goes to that mesh cell.  Otherwise a 3D DDA (Amanatides &
// Woo) walks the mesh cells the segment p0 + t d, 0 <= t <= L crosses, after
// clipping it to the mesh box.
// ---------------------------------------------------------------------------
// Mesh-tally operations: add the piece to the tally, or weight it by an
// upstream gradient (adjoint).
struct MeshAtomic {
    const Tallies& T;
    __device__ __forceinline__ void operator()(int i, double l) const
    {
        if (!fix_add_nn(T.mesh + i, l)) tally_range_error(T);   // l > 0
    }
};
// The same for weighted particles: each piece times the weight.
struct MeshAtomicW {
    const Tallies& T;
    double wt;
    __device__ __forceinline__ void operator()(int i, double l) const
    {
        if (!fix_add_nn(T.mesh + i, wt * l)) tally_range_error(T);
    }
};
struct MeshWeighted {
    const double* g;
    double f;
    __device__ __forceinline__ void operator()(int i, double l) { f += __ldg(g + i) * l; }
};

// The generic walk (segments that leave their one-cell fast path).
template <class Op>
__device__ __forceinline__ void mesh_tally_dda(const DevProblem& P, Op& op, const Particle& p, double x0, double y0,
                                               double z0, double L, int goff)
{
    const int nx = P.mesh_n[0], ny = P.mesh_n[1], nz = P.mesh_n[2];
    const double INF = __longlong_as_double(0x7FF0000000000000ll);
    double t0 = 0.0, t1 = L;
    // clip per axis (a zero component keeps the start point's slab test)
#define TR_CLIP(D, INV, X0, LO, HI)                                                   \
    if ((D) == 0.0) {                                                                 \
        if ((X0) < (LO) || (X0) >= (HI)) return;                                      \
    } else {                                                                          \
        const double ta = ((LO) - (X0)) * (INV), tb = ((HI) - (X0)) * (INV);           \
        t0 = fmax(t0, fmin(ta, tb));                                                  \
        t1 = fmin(t1, fmax(ta, tb));                                                  \
    }
    TR_CLIP(p.u, p.iu, x0, P.mesh_lo[0], P.mesh_hi[0])
    TR_CLIP(p.v, p.iv, y0, P.mesh_lo[1], P.mesh_hi[1])
    TR_CLIP(p.w, p.iw, z0, P.mesh_lo[2], P.mesh_hi[2])
#undef TR_CLIP
    if (!(t1 > t0)) return;
    // start cell, next crossing parameter and its step per axis
#define TR_START(D, INV, X0, A, N, I, S, TN, DT)                                      \
    int I = (int)floor(((X0) + t0 * (D) - P.mesh_lo[A]) * P.mesh_iw[A]);             \
    I = I < 0 ? 0 : (I > (N) - 1 ? (N) - 1 : I);                                      \
    int S = 0;                                                                        \
    double TN = INF, DT = 0.0;                                                        \
    if (gt0(D)) {                                                                     \
        S = 1;                                                                        \
        TN = (P.mesh_lo[A] + (double)(I + 1) * P.mesh_w[A] - (X0)) * (INV);           \
        DT = P.mesh_w[A] * (INV);                                                     \
    } else if (lt0(D)) {                                                              \
        S = -1;                                                                       \
        TN = (P.mesh_lo[A] + (double)I * P.mesh_w[A] - (X0)) * (INV);                 \
        DT = -P.mesh_w[A] * (INV);                                                    \
    }
    TR_START(p.u, p.iu, x0, 0, nx, ix, sx, tx, dtx)
    TR_START(p.v, p.iv, y0, 1, ny, iy, sy, ty, dty)
    TR_START(p.w, p.iw, z0, 2, nz, iz, sz, tz, dtz)
#undef TR_START
    TR_LANES(7);
    double t = t0;
    for (int guard = 0; guard < (1 << 20); ++guard) {
        TR_LANES(8);
        int ax = 0;
        double tn = tx;
        if (ty < tn) { tn = ty; ax = 1; }
        if (tz < tn) { tn = tz; ax = 2; }
        const double te = fmin(tn, t1);
        if (te > t) {
            op(goff + (iz * ny + iy) * nx + ix, te - t);
            t = te;
        }
        if (!(tn < t1)) break;
        if (ax == 0) {
            ix += sx;
            if (ix < 0 || ix >= nx) break;
            tx += dtx;
        } else if (ax == 1) {
            iy += sy;
            if (iy < 0 || iy >= ny) break;
            ty += dty;
        } else {
            iz += sz;
            if (iz < 0 || iz >= nz) break;
            tz += dtz;
        }
    }
}

// The one-voxel fast path: a segment in a geometry cell that lies inside one
// mesh voxel puts its whole length there.  Returns false when the cell spans
// several voxels (or none) on some axis, and the segment needs the walk.
template <class Op>
__device__ __forceinline__ bool mesh_tally_cell(const DevProblem& P, Op& op, const Particle& p, double L, int goff)
{
    const int vx = __ldg(P.cell2vox + cell_i(p.cell));
    const int vy = __ldg(P.cell2vox + P.nx + cell_j(p.cell));
    const int vz = __ldg(P.cell2vox + P.nx + P.ny + cell_k(p.cell));
    if ((vx | vy | vz) < 0) return false;
    op(goff + (vz * P.mesh_n[1] + vy) * P.mesh_n[0] + vx, L);
    return true;
}

template <class Op>
__device__ __forceinline__ void mesh_tally(const DevProblem& P, Op& op, const Particle& p, double x0, double y0,
                                           double z0, double L, int goff)
{
    if (!mesh_tally_cell(P, op, p, L, goff)) mesh_tally_dda(P, op, p, x0, y0, z0, L, goff);
}

// Deferred mesh walks.  The segments that need the walk come from the few
// lanes of a warp whose particles are in such cells, so inline each FP64 warp
// instruction of the walk serves one or two lanes (the FP64 pipe charges a
// warp instruction the same however few lanes are active).  The monolithic
// asynchronous kernel instead queues them per warp (in global memory, or in
// shared memory for the allocation-free entry) and walks them 32 at a time.  The mesh tally sums fixed-point pieces, so their order
// does not change it, and each piece comes from the same inputs as inline:
// the tallies are the same bits either way.
constexpr int WALKQ_CAP = 64;          // a warp drains 32 entries before each pass: at most 31 + 32 queued
struct WalkQ {
    double x0[WALKQ_CAP], y0[WALKQ_CAP], z0[WALKQ_CAP];
    double u[WALKQ_CAP], v[WALKQ_CAP], w[WALKQ_CAP];
    double iu[WALKQ_CAP], iv[WALKQ_CAP], iw[WALKQ_CAP];
    double len[WALKQ_CAP], wt[WALKQ_CAP];
    int goff[WALKQ_CAP];
    int n;
};
__host__ __device__ constexpr size_t walkq_bytes() { return (sizeof(WalkQ) + 15) & ~size_t(15); }

__device__ __forceinline__ void walk_push(WalkQ* q, const Particle& p, double x0, double y0, double z0, double L,
                                          int goff, double wt, ErrorWord* err)
{
    const int i = q ? atomicAdd(&q->n, 1) : WALKQ_CAP;
    if (i >= WALKQ_CAP) {   // (the drain before every pass rules this out; no queue: a launch error)
        if (err) atomicCAS(&err->code, 0, ERR_CAPACITY);
        return;
    }
    q->x0[i] = x0; q->y0[i] = y0; q->z0[i] = z0;
    q->u[i] = p.u; q->v[i] = p.v; q->w[i] = p.w;
    q->iu[i] = p.iu; q->iv[i] = p.iv; q->iw[i] = p.iw;
    q->len[i] = L;
    q->wt[i] = wt;
    q->goff[i] = goff;
}

// Walks entries [first, n) of a warp's queue with the lanes of m (every lane
// of m calls it).
template <bool WW>
static __device__ __forceinline__ void walk_run(const DevProblem& P, const Tallies& T, const WalkQ* q, int first,
                                                int n, unsigned m)
{
    const int lane = (int)(threadIdx.x & 31);
    const int nl = __popc(m), rank = __popc(m & ((1u << lane) - 1u));
    for (int i = first + rank; i < n; i += nl) {
        Particle d;
        d.u = q->u[i]; d.v = q->v[i]; d.w = q->w[i];
        d.iu = q->iu[i]; d.iv = q->iv[i]; d.iw = q->iw[i];
        if (WW) {
            MeshAtomicW op{T, q->wt[i]};
            mesh_tally_dda(P, op, d, q->x0[i], q->y0[i], q->z0[i], q->len[i], q->goff[i]);
        } else {
            MeshAtomic op{T};
            mesh_tally_dda(P, op, d, q->x0[i], q->y0[i], q->z0[i], q->len[i], q->goff[i]);
        }
    }
}

// Energy-bin flux tally per material: bin = largest b with e[b] <= E < e[b+1].
__device__ __forceinline__ void energy_tally(const DevProblem& P, const Tallies& T, int m, double E, double L)   // L: weighted
{
    const int nb = P.n_ebins;
    // E > 0 and the edges are non-negative (checked at problem creation):
    // compared on their bit patterns (integer instructions)
    const long long eb = dbits(E);
    if (eb < dbits(__ldg(P.e_edges)) || eb >= dbits(__ldg(P.e_edges + nb))) return;
    int lo = 0, hi = nb;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (dbits(__ldg(P.e_edges + mid)) <= eb) lo = mid; else hi = mid;
    }
    if (!fix_add_nn(T.energy + m * nb + lo, L)) tally_range_error(T);   // L > 0
}

// ---------------------------------------------------------------------------
// Source event (make_work): event count 0 draws; leaves n = 1.
// ---------------------------------------------------------------------------
template <bool CE, bool SOFT = false>
__device__ __forceinline__ bool source_particle(const DevProblem& P, const RunParams& R, unsigned id, Particle& p,
                                                const Bank* site, unsigned long long site_idx)
{
    TR_LANES(23);
    const Stream S = make_stream(R, id);
    const uint4 b0 = S.block(0u, BLK_MAIN);
    const double xi_ge = u01(b0.z, b0.w);
    p.id = id;
    p.n = 1u;
    p.nsites = 0u;
    p.pend = 0u;
    p.prob = 0u;
    p.g = 0;
    p.E = 0.0;
    p.t = 0.0;
    p.hf = p.ha = p.hp = 0.0;
    p.wt = 1.0;
    p.sid = p.nsplit = 0u;
    if (site != nullptr || P.src_kind != 0 || P.src_iso) {
        iso_dir<SOFT>(S, 0u, p);
    } else {
        p.u = P.src_dir[0];
        p.v = P.src_dir[1];
        p.w = P.src_dir[2];
        set_reciprocals<SOFT>(p);
    }
    if (site != nullptr) {
        p.x = site->x[site_idx];
        p.y = site->y[site_idx];
        p.z = site->z[site_idx];
        p.cell = site->cell[site_idx];
        p.g = site->g[site_idx];
        return true;
    }
    if (P.src_kind == 0) {
        p.x = P.src_pt[0];
        p.y = P.src_pt[1];
        p.z = P.src_pt[2];
        locate(P, p);
    } else {
        uint32_t t = 0;
        for (; t < N_POS; ++t) {
            TR_LANES(24);
            const uint4 a = S.block(0u, BLK_POS + 2u * t);
            const uint4 b = S.block(0u, BLK_POS + 2u * t + 1u);
            p.x = P.src_lo[0] + u01(a.x, a.y) * (P.src_hi[0] - P.src_lo[0]);
            p.y = P.src_lo[1] + u01(a.z, a.w) * (P.src_hi[1] - P.src_lo[1]);
            p.z = P.src_lo[2] + u01(b.x, b.y) * (P.src_hi[2] - P.src_lo[2]);
            locate(P, p);
            if (P.src_kind == 1) break;
            if (cell_in(p.cell) && __ldg(P.src_mat + info_pin(cell_info(P, p.cell)))) break;
        }
        if (t == N_POS) return false;
    }
    const int m = material(P, p.cell);
    if (!CE) p.g = (P.src_group >= 0) ? P.src_group : sample_chi(P, m, xi_ge);
    else p.E = (P.n_cdf > 1) ? cdf_sample(P, xi_ge) : P.src_energy;
    return true;
}

// ---------------------------------------------------------------------------
// Step event: lookup, distance to collision vs. surface, move, tally.
// Leaves the outcome in p.pend.  Returns the lookup for the collision.
// ---------------------------------------------------------------------------
// Timed problems only, out of line so that untimed steps carry only a branch
// and a call: the track length spent in each uniform bin of [t0, t1]
// (t0 < t1), and a particle's 1/v and distance to census.
static __device__ __noinline__ void time_bins(FixBin* tally, ErrorWord* err, int n_tbins, double tb_w, double t0,
                                              double t1, double inv_v, double wt)
{
    int b = (int)floor(t0 / tb_w);
    if (b < 0) b = 0;
    for (; b < n_tbins; ++b) {
        double lo = (double)b * tb_w, hi = (double)(b + 1) * tb_w;
        if (lo >= t1) break;
        lo = fmax(lo, t0);
        hi = fmin(hi, t1);
        if (hi > lo && !fix_add_nn(tally + b, wt * ((hi - lo) / inv_v)) && err) atomicCAS(&err->code, 0, ERR_RANGE);
    }
}

struct CensusStep {
    double dcen, inv_v;
};

template <bool CE>
static __device__ __noinline__ CensusStep census_step(double v_c, const double* inv_vel, double t_cen, double E, int g,
                                                      double t)
{
    CensusStep r;
    r.inv_v = CE ? 1.0 / (v_c * sqrt(E)) : __ldg(inv_vel + g);
    const double left = t_cen - t;
    r.dcen = left > 0.0 ? left / r.inv_v : 0.0;
    return r;
}

// Forward tally sink: track-length scores into the tallies and the
// particle's running scalar scores.  WW: weighted particles (weight-window
// problems), every score times the particle's weight.
template <bool WW, bool WQ = false>
struct FwdSinkT {
    static constexpr bool kWW = WW;
    const Tallies& T;
    Acc& acc;
    double wt = 1.0;                   // WW: the particle's weight (set by segment for time_segment)
    WalkQ* wq = nullptr;               // WQ: the warp's queue of deferred mesh walks
    template <bool CE>
    __device__ __forceinline__ void segment(const DevProblem& P, Particle& p, double x0, double y0, double z0,
                                            double dist, int m, const XS& X)
    {
        const double dl = WW ? p.wt * dist : dist;
        if (WW) wt = p.wt;
        p.hf += dl;
        p.ha = __fma_rn(dl, X.sa, p.ha);   // tallies: compared within tolerance, fused freely
        if (!CE) p.hp = __fma_rn(dl, X.nsf, p.hp);   // continuous energy: nu Sigma_f = 0
        if (P.has_mesh && gt0(dist)) {
            const int goff = (!CE && P.by_group) ? p.g * P.mesh_vox : 0;
            if (WQ) {
                bool one;
                if (WW) {
                    MeshAtomicW op{T, p.wt};
                    one = mesh_tally_cell(P, op, p, dist, goff);
                } else {
                    MeshAtomic op{T};
                    one = mesh_tally_cell(P, op, p, dist, goff);
                }
                if (!one) walk_push(wq, p, x0, y0, z0, dist, goff, WW ? p.wt : 1.0, T.err);
            } else if (WW) {
                MeshAtomicW op{T, p.wt};
                mesh_tally(P, op, p, x0, y0, z0, dist, goff);
            } else {
                MeshAtomic op{T};
                mesh_tally(P, op, p, x0, y0, z0, dist, goff);
            }
        }
        if (CE && P.n_ebins > 0 && gt0(dist)) energy_tally(P, T, m, p.E, dl);
    }
    // time bins: the (weighted) track length spent in each bin of [t0, t1]
    __device__ __forceinline__ void time_segment(const DevProblem& P, double t0, double t1, double inv_v)
    {
        if (P.n_tbins <= 0 || !(t1 > t0)) return;
        time_bins(T.time, T.err, P.n_tbins, P.tb_w, t0, t1, inv_v, wt);
    }
};
using FwdSink = FwdSinkT<false>;

// CACHED: the cross sections come from the particle (left there by the
// lookup event) instead of a lookup here; the values are the same.
template <bool CE, bool CACHED = false, class Sink>
__device__ __forceinline__ void step_event(const DevProblem& P, const RunParams& R, Particle& p, Sink& sink, XS& X,
                                           double& xi_react)
{
    TR_LANES(1);
    const unsigned c = p.cell;
    const int info = cell_info(P, c);
    const int in = cell_in(c);
    const int pin = info_pin(info) >= 0;
    const int m = in ? info_pin(info) : info_mat(info);
    if (CACHED) {
        X.st = p.xst;
        X.inv_st = p.xist;
        X.sa = p.xsa;
        X.nsf = p.xnsf;
    } else {
        xs_lookup<CE>(P, p, m, X);
    }
    const Stream S = particle_stream<Sink::kWW>(R, p);
    const uint4 b0 = S.block(p.n, BLK_MAIN);
    xi_react = u01(b0.z, b0.w);
    const double dcol = exp_sample(P, S, p.n, b0.x, b0.y) * X.inv_st;
    TR_LANES(2);

    const double INF = __longlong_as_double(0x7FF0000000000000ll);
    const int i = cell_i(c), j = cell_j(c), k = cell_k(c);
    double dx, dy, dz;
    // exit plane chosen by the sign of the component (integer select), then one
    // subtraction and one multiplication for every lane: no divergent paths
    dx = (__ldg(P.xp + i + (gt0(p.u) ? 1 : 0)) - p.x) * p.iu;
    dy = (__ldg(P.yp + j + (gt0(p.v) ? 1 : 0)) - p.y) * p.iv;
    dz = (__ldg(P.zp + k + (gt0(p.w) ? 1 : 0)) - p.z) * p.iw;
    dx = (dbits(p.u) << 1) ? clamp0(dx) : INF;
    dy = (dbits(p.v) << 1) ? clamp0(dy) : INF;
    dz = (dbits(p.w) << 1) ? clamp0(dz) : INF;

    double dcyl = INF;
    if (pin) {
        // one square root of max(disc, 0) serves both cases: inside, the
        // clamped discriminant; outside, a hit needs k < 0 and disc >= 0 and
        // then max(disc, 0) = disc
        double cc, kk;
        pin_terms(P, p, cc, kk);
        const double a = __fma_rn(p.u, p.u, p.v * p.v);
        const double disc = __fma_rn(kk, kk, -(a * cc));
        const double sq = tr_sqrt(lt0(disc) ? 0.0 : disc);
        // inside (sq - k) ia, outside ((-k) - sq) ia = ((-sq) - k) ia (IEEE
        // addition commutes): one subtraction and one product for both
        const double d = ((in ? sq : flip_sign(sq)) - kk) * p.ia;
        const bool hit = gt0(a) && (in || (lt0(kk) && ge0(disc)));
        dcyl = hit ? clamp0(d) : INF;
    }
    TR_LANES(3);
    unsigned flags = 0u;
    double ds;
    if (in) {
        if (lt_nn(dcyl, dz)) {
            ds = dcyl;
            flags = PEND_CYL;
        } else {
            ds = dz;
            flags = PEND_Z;
        }
    } else {
        double dmin = dx;
        if (lt_nn(dy, dmin)) dmin = dy;
        if (lt_nn(dz, dmin)) dmin = dz;
        if (pin && lt_nn(dcyl, dmin)) {
            ds = dcyl;
            flags = PEND_CYL;
        } else {
            ds = dmin;
            if (dbits(dx) == dbits(ds)) flags |= PEND_X;
            if (dbits(dy) == dbits(ds)) flags |= PEND_Y;
            if (dbits(dz) == dbits(ds)) flags |= PEND_Z;
        }
    }
    const bool collided = lt_nn(dcol, ds);
    double dist = collided ? dcol : ds;
    // timed problems: the census ends the history when it comes strictly
    // before the collision or surface
    bool census = false;
    double inv_v = 0.0;
    if (P.timed) {
        const CensusStep c = census_step<CE>(P.v_c, P.inv_vel, P.t_cen, p.E, p.g, p.t);
        inv_v = c.inv_v;
        if (c.dcen < dist) {
            census = true;
            dist = c.dcen;
        }
    }
    const bool escape = !census && !collided && dbits(ds) == dbits(INF);   // no surface ahead: escape
    TR_LANES(4);
    if (!escape) {
        const double x0 = p.x, y0 = p.y, z0 = p.z;
        p.x = __fma_rn(dist, p.u, p.x);
        p.y = __fma_rn(dist, p.v, p.y);
        p.z = __fma_rn(dist, p.w, p.z);
        sink.template segment<CE>(P, p, x0, y0, z0, dist, m, X);
        if (P.timed) {
            const double t0 = p.t;
            p.t = census ? P.t_cen : __fma_rn(dist, inv_v, p.t);
            sink.time_segment(P, t0, p.t, inv_v);
        }
    }
    TR_LANES(5);
    p.pend = escape ? PEND_ESCAPE : (census ? PEND_CENSUS : (collided ? PEND_COLLIDE : flags));
}

// ---------------------------------------------------------------------------
// Collision event.  Returns the event type (SCATTER keeps the history alive).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void bank_sites(const DevProblem& P, const RunParams& R, const Stream& S, Particle& p,
                                           int m, const XS& X, const Bank& B, ErrorWord* err)
{
    const double xf = S.first(p.n, BLK_FISSION);
    const double t = ((X.nsf * X.inv_st) * R.inv_k) + xf;
    const int nf = floor_nn(t);   // t >= 0
    for (int c = 0; c < nf; ++c) {
        const double xs = S.first(p.n, BLK_SITE + (uint32_t)c);
        const int gs = sample_chi(P, m, xs);
        const unsigned long long pos = atomicAdd(B.count, 1ull);
        if (pos < B.capacity) {
            B.x[pos] = p.x;
            B.y[pos] = p.y;
            B.z[pos] = p.z;
            B.g[pos] = gs;
            B.cell[pos] = p.cell;
            B.key[pos] = ((unsigned long long)p.id << 32) | p.nsites;
        } else {
            atomicCAS(&err->code, 0, ERR_CAPACITY);
        }
        p.nsites += 1u;
    }
}

// Multigroup collision up to its direction: fission banking and the
// reaction, the first g' with xi * Sigma_t below the cumulative Sigma_s.
// Returns g', or -1 for absorption.
template <bool WW>
__device__ __forceinline__ int collide_mg_react(const DevProblem& P, const RunParams& R, Particle& p, const XS& X,
                                                double xi_react, const Bank& B, ErrorWord* err, unsigned cm)
{
    const Stream S = particle_stream<WW>(R, p);
    const int m = material(P, p.cell);
    if (R.eig && gt0(X.nsf)) bank_sites(P, R, S, p, m, X, B, err);
    if (cm) __syncwarp(cm);
    const double t = xi_react * X.st;
    const double* cs = P.cum_s + (m * P.G + p.g) * P.G;
    int gp = -1;
    for (int h = 0; h < P.G; ++h) gp = (gp < 0 && lt_nn(t, __ldg(cs + h))) ? h : gp;
    return gp;
}

// cm: the lanes of this warp that run the collision together (a mask every
// one of them passes, from a ballot), or 0.  With a mask the colliding lanes
// are regrouped after the fission banking and the reaction selection (which
// runs every candidate in every lane instead of stopping at the first hit),
// and the scattering lanes after the azimuth loop, so that the FP64 work of
// the direction sampling is issued once for all of them: the FP64 pipe
// charges a warp instruction the same however few lanes are active.
template <bool CE, bool WW = false>
__device__ __forceinline__ int collide_event(const DevProblem& P, const RunParams& R, Particle& p, const XS& X,
                                             double xi_react, const Bank& B, ErrorWord* err, unsigned cm = 0u)
{
    TR_LANES(16);
    const Stream S = particle_stream<WW>(R, p);
    if (!CE) {
        const int gp = collide_mg_react<WW>(P, R, p, X, xi_react, B, err, cm);
        const unsigned sm = cm ? __ballot_sync(cm, gp >= 0) : 0u;
        if (gp < 0) return EV_ABSORB;
        TR_LANES(17);
        p.g = gp;
        iso_dir(S, p.n, p, sm);
        return EV_SCATTER;
    }
    const int m = material(P, p.cell);
    // continuous energy: the lookup terms in order, and the first (nuclide,
    // reaction) with xi * sigma_t below the running sum; if none (rounding),
    // the last term with a positive value.  Nuclides absent from the material
    // (density <= 0) add nothing.  Terms the step's lookup kept are the same
    // values; otherwise they are computed again.
    const double t = xi_react * X.st;
    double cum = 0.0;
    int sel_n = -1, sel_r = -1, last_n = -1, last_r = -1;
    if (X.keep && X.keep->n >= 0) {
        if (cm) __syncwarp(cm);
        int sel = -1, last = -1;
        for (int k = 0; k < 3 * X.keep->n; ++k) {
            const double mac = X.keep->mac[k];
            const double c2 = cum + mac;
            last = gt0(mac) ? k : last;                  // non-negative values: integer compares
            sel = (sel < 0 && lt_nn(t, c2)) ? k : sel;
            cum = c2;
        }
        if (sel >= 0) {
            sel_n = X.keep->nuc[sel / 3];
            sel_r = sel % 3;
        }
        if (last >= 0) {
            last_n = X.keep->nuc[last / 3];
            last_r = last % 3;
        }
    } else {
        const int u = union_index(P, p.E);
        if (cm) __syncwarp(cm);
        for (int n = 0; n < P.n_nuc; ++n) {
            const double N = __ldg(P.dens + m * P.n_nuc + n);
            const bool use = gt0(N);
            const int r0 = __ldg(P.uptr + (long long)u * P.n_nuc + n);
            const double dE = p.E - __ldg(P.nuc_e + r0);
            for (int r = 0; r < 3; ++r) {
                const double s0 = __ldg(P.nuc_sig + 3 * (long long)r0 + r);
                const double mac = N * __fma_rn(dE, __ldg(P.nuc_slope + 3 * (long long)r0 + r), s0);
                const double c2 = use ? cum + mac : cum;
                const bool pos = use && gt0(mac);
                last_n = pos ? n : last_n;
                last_r = pos ? r : last_r;
                const bool take = use && sel_n < 0 && lt_nn(t, c2);
                sel_n = take ? n : sel_n;
                sel_r = take ? r : sel_r;
                cum = c2;
            }
        }
    }
    if (sel_n < 0) {
        sel_n = last_n;
        sel_r = last_r;
    }
    const bool scatter = !(sel_n < 0 || sel_r != 0);
    const unsigned sm = cm ? __ballot_sync(cm, scatter) : 0u;
    if (!scatter) return EV_ABSORB;
    const double A = __ldg(P.awr + sel_n);
    const double mu_cm = __fma_rn(2.0, S.first(p.n, BLK_ANGLE), -1.0);   // 2 xi exact: same as 2 xi - 1
    const double q = (A * A + (2.0 * A) * mu_cm) + 1.0;
    const double E1 = (p.E * q) * __ldg(P.inv_ap1sq + sel_n);
    const double mu = (1.0 + A * mu_cm) / sf_sqrt(q);   // integer-pipe square root (the same bits)
    double cphi, sphi;
    azimuth(S, p.n, cphi, sphi, sm);
    rotate(p, mu, cphi, sphi);
    p.E = E1;
    if (lt_nn(p.E, P.e_cut)) return EV_SCATTER_CUTOFF;
    return EV_SCATTER;
}

// ---------------------------------------------------------------------------
// Surface-crossing event from the step's pending flags.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int surface_event(const DevProblem& P, Particle& p)
{
    TR_LANES(21);
    const unsigned f = p.pend;
    if (f & PEND_CENSUS) return EV_CUTOFF;
    if (f & PEND_ESCAPE) return EV_LEAK;
    if (f & PEND_CYL) {
        p.cell ^= 1u << 30;
        return EV_SURF_INTERNAL;
    }
    int i = cell_i(p.cell), j = cell_j(p.cell), k = cell_k(p.cell), in = cell_in(p.cell);
    bool leak = false, refl = false, moved_xy = false, moved_z = false;
    if (f & PEND_X) {
        const bool hi = gt0(p.u);
        if (hi ? (i == P.nx - 1) : (i == 0)) {
            if (P.bc[hi ? 1 : 0] == 1) {
                p.u = flip_sign(p.u);
                p.iu = flip_sign(p.iu);
                refl = true;
            } else leak = true;
        } else {
            i += hi ? 1 : -1;
            moved_xy = true;
        }
    }
    if (f & PEND_Y) {
        const bool hi = gt0(p.v);
        if (hi ? (j == P.ny - 1) : (j == 0)) {
            if (P.bc[hi ? 3 : 2] == 1) {
                p.v = flip_sign(p.v);
                p.iv = flip_sign(p.iv);
                refl = true;
            } else leak = true;
        } else {
            j += hi ? 1 : -1;
            moved_xy = true;
        }
    }
    if (f & PEND_Z) {
        const bool hi = gt0(p.w);
        if (hi ? (k == P.nz - 1) : (k == 0)) {
            if (P.bc[hi ? 5 : 4] == 1) {
                p.w = flip_sign(p.w);
                p.iw = flip_sign(p.iw);
                refl = true;
            } else leak = true;
        } else {
            k += hi ? 1 : -1;
            moved_z = true;
        }
    }
    if (leak) {
        // the final cell keeps the moves of the other axes crossed in the same event
        p.cell = pack_cell(i, j, k, in);
        return EV_LEAK;
    }
    if (moved_xy || moved_z) {
        p.cell = pack_cell(i, j, k, 0);
        const int pin = info_pin(cell_info(P, p.cell)) >= 0;
        if (pin && !moved_xy) {
            if (in) {
                p.cell |= 1u << 30;
            } else {
                double cc, kk;
                pin_terms(P, p, cc, kk);
                if (cc < 0.0 || (cc == 0.0 && kk < 0.0)) p.cell |= 1u << 30;
            }
        }
    }
    return refl ? EV_SURF_REFLECT : EV_SURF_INTERNAL;
}

// Closeout (the closeout event of the paper's decomposed scheme, Sec. 4:
// weights and weight windows for the particle's next loop iteration; the
// rules are our reading, the same as the oracle's).  The window of the
// tally-mesh voxel holding the particle (i_a = floor((x_a - lo_a) (1 / w_a)),
// outside the mesh: none) and its group has lower bound L (0: none), upper
// bound ww_up L and survival weight ww_surv L.  Below L: Russian roulette,
// survival when xi (the first uniform of block BLK_CLOSE at the particle's
// event count) times the survival weight is below the weight, at the
// survival weight; otherwise the history ends as CUTOFF.  Above the upper
// bound: k = min(ceil(w / U), ww_max_split) copies of weight w / k; the
// particle continues as copy 0 and leaves k - 1 in p.nsplit for the
// scheduler to create (tag of copy c: word 0 of block BLK_SPLIT + c, bit 31
// set).  Returns whether the particle lives on.
__device__ __forceinline__ bool closeout(const DevProblem& P, const RunParams& R, Particle& p, int& type)
{
    const double xs[3] = {p.x, p.y, p.z};
    int idx[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double t = floor((xs[a] - P.mesh_lo[a]) * P.mesh_iw[a]);
        if (!(t >= 0.0) || !(t < (double)P.mesh_n[a])) return true;
        idx[a] = (int)t;
    }
    const int v = (idx[2] * P.mesh_n[1] + idx[1]) * P.mesh_n[0] + idx[0];
    // continuous energy: one window per voxel (G = 1); p.g carries no group
    // there (stacks and spill links do not store it)
    const double L = __ldg(P.ww_lo + (long long)v * P.G + (P.kind == 1 ? 0 : p.g));
    if (!(L > 0.0)) return true;
    const Stream S = particle_stream<true>(R, p);
    if (p.wt < L) {
        const double Sw = P.ww_surv * L;
        if (S.first(p.n, BLK_CLOSE) * Sw < p.wt) {
            p.wt = Sw;
            return true;
        }
        type = EV_CUTOFF;
        return false;
    }
    const double U = P.ww_up * L;
    if (!(p.wt > U)) return true;
    int k = (int)ceil(p.wt / U);
    if (k > P.ww_max_split) k = P.ww_max_split;
    if (k < 2) return true;
    p.wt = p.wt / (double)k;
    p.nsplit = (unsigned)(k - 1);
    return true;
}

// Split copy c (1 .. p.nsplit) of particle p: its state with its own stream
// tag, no pending outcome, its scores starting at 0.
__device__ __forceinline__ Particle split_copy(const RunParams& R, const Particle& p, unsigned c)
{
    Particle q = p;
    const Stream S = particle_stream<true>(R, p);
    q.sid = p.sid ^ (S.block(p.n, BLK_SPLIT + c).x | 0x80000000u);
    q.hf = q.ha = q.hp = 0.0;
    q.nsplit = 0u;
    q.pend = 0u;
    return q;
}

// Close an event: count it, advance n, apply the event cap (and, WW, the
// weight-window closeout).  Returns whether the history continues; on death
// records the final state.  A split copy (p.sid != 0) ends without a log
// entry, its scores going to the per-thread fixed-point sums.
template <bool WW = false>
__device__ __forceinline__ bool finish_event(const DevProblem& P, const RunParams& R, Particle& p, int type,
                                             const Tallies& T, Acc& acc, const Bank& B)
{
    TR_LANES(22);
    const bool sc = type == EV_SCATTER_CUTOFF;
    acc.ev[sc ? EV_SCATTER : type] += 1u;
    if (sc) type = EV_CUTOFF;
    p.n += 1u;
    bool alive = (type == EV_SCATTER || type == EV_SURF_INTERNAL || type == EV_SURF_REFLECT);
    if (alive && p.n >= R.max_events) {
        alive = false;
        type = EV_MAXEV;
    }
    if (WW && alive) alive = closeout(P, R, p, type);
    if (!alive) {
        const bool primary = !WW || p.sid == 0u;
        if (T.hist_f && primary) {
            T.hist_f[p.id] = p.hf;
            T.hist_a[p.id] = p.ha;
            T.hist_p[p.id] = p.hp;
        } else if (T.scal) {
            acc_history_sums(acc.fx, T.scal, T.err, p.hf, p.ha, p.hp);
        }
        acc.fin[type] += 1u;
        if (R.want_log && primary) {
            T.log_n[p.id] = p.n;
            T.log_cell[p.id] = cell_id(P, p.cell);
            T.log_type[p.id] = (uint8_t)type;
        }
        if (R.eig) B.site_count[p.id] = p.nsites;
    }
    return alive;
}

// One monolithic event (step followed by collision or surface crossing).
// em: the lanes of this warp that run this event together (from a ballot), or 0.
// WQ: mesh walks go to the warp's queue wq.
template <bool CE, bool WW = false, bool WQ = false>
__device__ __forceinline__ bool mono_event(const DevProblem& P, const RunParams& R, Particle& p, const Tallies& T,
                                           Acc& acc, const Bank& B, ErrorWord* err, unsigned em = 0u,
                                           WalkQ* wq = nullptr)
{
    TR_LANES(10);
    XS X;
    CEKeep keep;
    if (CE) X.keep = &keep;   // the collision below reuses the lookup's terms
    double xi_react;
    FwdSinkT<WW, WQ> sink{T, acc, 1.0, wq};
    step_event<CE>(P, R, p, sink, X, xi_react);
    const bool coll = p.pend == PEND_COLLIDE;
    const unsigned cm = em ? __ballot_sync(em, coll) : 0u;
    int type;
    if (coll) type = collide_event<CE, WW>(P, R, p, X, xi_react, B, err, cm);
    else type = surface_event(P, p);
    return finish_event<WW>(P, R, p, type, T, acc, B);
}

// Lookup event (decomposition with the lookup as an event of its own): the
// cross sections of the particle's material at its energy or group, kept in
// the particle for the step and collision that follow.  Does not count as an
// event (n unchanged).
template <bool CE>
__device__ __forceinline__ void lookup_event(const DevProblem& P, Particle& p)
{
    XS X;
    xs_lookup<CE>(P, p, material(P, p.cell), X);
    p.xst = X.st;
    p.xist = X.inv_st;
    p.xsa = X.sa;
    p.xnsf = X.nsf;
}

// Decomposed collision event: repeats the lookup (or, CACHED, takes the
// particle's) and the reaction draw.
template <bool CE, bool CACHED = false, bool WW = false>
__device__ __forceinline__ bool split_collide(const DevProblem& P, const RunParams& R, Particle& p, const Tallies& T,
                                             Acc& acc, const Bank& B, ErrorWord* err, unsigned em = 0u)
{
    XS X;
    if (CACHED) {
        X.st = p.xst;
        X.inv_st = p.xist;
        X.sa = p.xsa;
        X.nsf = p.xnsf;
    } else {
        xs_lookup<CE>(P, p, material(P, p.cell), X);
    }
    const Stream S = particle_stream<WW>(R, p);
    const uint4 b0 = S.block(p.n, BLK_MAIN);
    const int type = collide_event<CE, WW>(P, R, p, X, u01(b0.z, b0.w), B, err, em);
    return finish_event<WW>(P, R, p, type, T, acc, B);
}

template <bool WW = false>
__device__ __forceinline__ bool split_surface(const DevProblem& P, const RunParams& R, Particle& p, const Tallies& T,
                                             Acc& acc, const Bank& B)
{
    const int type = surface_event(P, p);
    return finish_event<WW>(P, R, p, type, T, acc, B);
}

// Surface event of the lookup-event decomposition: the next event is a lookup
// when the particle entered another material, else the step (the cached cross
// sections depend only on material and energy).
__device__ __forceinline__ int split_surface_next(const DevProblem& P, const RunParams& R, Particle& p,
                                                  const Tallies& T, Acc& acc, const Bank& B)
{
    const int m0 = material(P, p.cell);
    const int type = surface_event(P, p);
    if (!finish_event(P, R, p, type, T, acc, B)) return Q_DEAD;
    return material(P, p.cell) != m0 ? Q_LOOKUP : Q_STEP;
}

// ---------------------------------------------------------------------------
// SoA load / store
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load_particle(const SoA& s, unsigned long long i, Particle& p, bool ce, bool xs = false,
                                              bool ww = false)
{
    p.nsplit = 0u;
    if (ww) {
        p.wt = s.wt[i];
        p.sid = s.sid[i];
    }
    p.t = s.t[i];
    p.hf = s.hf[i]; p.ha = s.ha[i]; p.hp = s.hp[i];
    if (xs) {
        p.xst = s.xst[i]; p.xist = s.xist[i]; p.xsa = s.xsa[i]; p.xnsf = s.xnsf[i];
    }
    p.x = s.x[i]; p.y = s.y[i]; p.z = s.z[i];
    p.u = s.u[i]; p.v = s.v[i]; p.w = s.w[i];
    p.iu = s.iu[i]; p.iv = s.iv[i]; p.iw = s.iw[i]; p.ia = s.ia[i];
    if (ce) {
        p.E = s.E[i];
        p.g = 0;
    } else {
        p.g = s.g[i];
    }
    p.cell = s.cell[i]; p.id = s.id[i]; p.n = s.n[i]; p.nsites = s.nsites[i]; p.pend = s.pend[i];
    p.prob = s.prob[i];
}

__device__ __forceinline__ void store_particle(const SoA& s, unsigned long long i, const Particle& p, bool ce,
                                               bool xs = false, bool ww = false)
{
    if (ww) {
        s.wt[i] = p.wt;
        s.sid[i] = p.sid;
    }
    s.t[i] = p.t;
    s.hf[i] = p.hf; s.ha[i] = p.ha; s.hp[i] = p.hp;
    if (xs) {
        s.xst[i] = p.xst; s.xist[i] = p.xist; s.xsa[i] = p.xsa; s.xnsf[i] = p.xnsf;
    }
    s.x[i] = p.x; s.y[i] = p.y; s.z[i] = p.z;
    s.u[i] = p.u; s.v[i] = p.v; s.w[i] = p.w;
    s.iu[i] = p.iu; s.iv[i] = p.iv; s.iw[i] = p.iw; s.ia[i] = p.ia;
    if (ce) s.E[i] = p.E; else s.g[i] = p.g;
    s.cell[i] = p.cell; s.id[i] = p.id; s.n[i] = p.n; s.nsites[i] = p.nsites; s.pend[i] = p.pend;
    s.prob[i] = p.prob;
}

// The particle k_presample left for history i, in the state source_particle
// leaves (n = 1, nothing banked or pending, t = 0); false if sampling failed.
template <bool CE>
__device__ __forceinline__ bool load_presampled(const SoA& s, unsigned long long i, Particle& p)
{
    p.x = s.x[i]; p.y = s.y[i]; p.z = s.z[i];
    p.u = s.u[i]; p.v = s.v[i]; p.w = s.w[i];
    p.iu = s.iu[i]; p.iv = s.iv[i]; p.iw = s.iw[i]; p.ia = s.ia[i];
    p.E = CE ? s.E[i] : 0.0;
    p.g = CE ? 0 : s.g[i];
    p.cell = s.cell[i];
    p.id = (unsigned)i;
    p.n = 1u;
    p.nsites = 0u;
    p.pend = 0u;
    p.prob = 0u;
    p.t = 0.0;
    p.hf = p.ha = p.hp = 0.0;
    p.wt = 1.0;
    p.sid = p.nsplit = 0u;
    return s.id[i] == (unsigned)i;
}

// Next queue of a live particle after an event: a step leads to collision or
// surface crossing; those lead back to a step.
__device__ __forceinline__ int next_queue_after_step(const Particle& p)
{
    return p.pend == PEND_COLLIDE ? Q_COLLIDE : Q_SURFACE;
}

// Warp-reduce the per-lane accumulators and add them to the global tallies
// (integer sums: the result does not depend on the order).
__device__ __forceinline__ void flush_acc(const Acc& acc, const Tallies& T)
{
    unsigned long long sl[3] = {0ull, 0ull, 0ull}, sh[3] = {0ull, 0ull, 0ull};
    if (acc.fx) {
#pragma unroll
        for (int k = 0; k < 3; ++k) fix_split_sum(acc.fx[k], sl[k], sh[k]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            sl[k] += __shfl_xor_sync(0xFFFFFFFFu, sl[k], o);
            sh[k] += __shfl_xor_sync(0xFFFFFFFFu, sh[k], o);
        }
    }
    unsigned ev[8], fin[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        ev[i] = __reduce_add_sync(0xFFFFFFFFu, acc.ev[i]);
        fin[i] = __reduce_add_sync(0xFFFFFFFFu, acc.fin[i]);
    }
    if ((threadIdx.x & 31) == 0) {
        if (T.scal) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                if (sl[k]) atomicAdd(&T.scal[k].lo, sl[k]);
                if (sh[k]) atomicAdd(&T.scal[k].hi, sh[k]);
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (ev[i]) atomicAdd(T.ev_type + i, (unsigned long long)ev[i]);
            if (fin[i]) atomicAdd(T.fin_type + i, (unsigned long long)fin[i]);
        }
    }
}

}  // namespace tr
