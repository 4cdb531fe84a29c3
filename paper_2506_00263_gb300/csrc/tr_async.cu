// tr_async.cu -- asynchronous remapping (Sec. 3.2 of Cuneo et al., M&C 2025).
//
// One persistent launch.  Each block owns a shared-memory stash: a pool of
// particle slots (structure of arrays) and, per event type, a queue of slot
// indices.  The block's warps share the stash (the paper's future-work item
// of Sec. 5.2: one stash used by several warps, for higher occupancy);
// metadata changes happen under a short shared-memory lock, while particle
// state is read and written only by the warp that owns the slot.
//
// A warp takes 32 particles of one event type from the fullest queue, runs
// that event with one particle per lane in registers, writes the particles
// back into the slots it owns and pushes each slot onto the queue of its next
// event type.  When no queue holds a full warp's worth, the warp calls
// make_work: it claims source indices with one atomic add and runs their
// source events (or loads the particles k_presample sampled before the
// launch).  Once the source is exhausted, partial queues are run as they are.
// In the monolithic scheme a warp keeps its particles in registers for up to
// remap_every passes, refilling idle lanes with new histories and batching
// the collisions of its lanes, before it deposits them.
//
// Global memory is the last resort (Sec. 3.2): a link arena of 32-particle
// links, organised in linked lists whose (head, tail) pair is packed in one
// 64-bit word.  A warp claims a list by swapping it with the empty list,
// edits it privately and deposits it back, merging with whatever another warp
// deposited meanwhile -- no inter-block synchronisation.  Blocks with surplus
// particles spill full links when some warp of another block is starving;
// starving warps refill from those lists (work stealing).  Every wait is
// bounded by max_spin and ends with TR_ERR_TIMEOUT instead of hanging.
#include "tr_events.cuh"
#include "tr_kernels.h"

namespace tr {

constexpr unsigned FULLM = 0xFFFFFFFFu;
constexpr unsigned long long EMPTY_LIST = ~0ull;
constexpr unsigned NIL = 0xFFFFFFFFu;
constexpr int N_GQ = 32;

struct Stash {
    double *x, *y, *z, *u, *v, *w, *iu, *iv, *iw, *ia, *E, *t;
    double *hf, *ha, *hp;              // the histories' running scalar scores
    double* wt;                        // weight-window problems: weights (else NULL)
    unsigned* sid;                     // weight-window problems: split copies' stream tags (else NULL)
    double *xst, *xist, *xsa, *xnsf;   // lookup-event decomposition only (else NULL)
    int* g;
    unsigned *cell, *id, *n, *nsites, *pend, *prob;
    unsigned short* q[N_QUEUES];       // slot-index queues per event type
    unsigned short* fr;                // free-slot stack
    int* cnt;                          // [0, N_QUEUES) queue counts, [CNT_FREE] free count, [CNT_LOCK] lock,
                                       // [CNT_RUN] warps between a take and its deposit
};
// control words after the queue counts
constexpr int CNT_FREE = N_QUEUES, CNT_LOCK = N_QUEUES + 1, CNT_RUN = N_QUEUES + 2;

__host__ __device__ __forceinline__ size_t stash_bytes(int S, bool xs = false, bool ww = false)
{
    return (size_t)S * ((xs ? 19 : 15) * sizeof(double) + sizeof(int) + 6 * sizeof(unsigned)) +
           (ww ? (size_t)S * (sizeof(double) + sizeof(unsigned)) : 0) +
           (size_t)S * (N_QUEUES + 1) * sizeof(unsigned short) + 16 * sizeof(int);
}

// Dynamic shared memory of one block: the stash, then (8-byte aligned) the
// threads' fixed-point sums of ended histories' scalar scores.
__host__ __device__ __forceinline__ size_t fx_offset(int S, bool xs, bool ww = false)
{
    return (stash_bytes(S, xs, ww) + 15) & ~size_t(15);
}
__host__ __device__ __forceinline__ size_t async_smem_bytes(int S, bool xs, bool ww = false)
{
    return fx_offset(S, xs, ww) + 256 * ACC_FX_WORDS * sizeof(long long);
}

__device__ __forceinline__ Stash carve(unsigned char* base, int S, bool xs, bool ww = false)
{
    Stash s;
    double* d = reinterpret_cast<double*>(base);
    s.x = d; d += S; s.y = d; d += S; s.z = d; d += S;
    s.u = d; d += S; s.v = d; d += S; s.w = d; d += S;
    s.iu = d; d += S; s.iv = d; d += S; s.iw = d; d += S; s.ia = d; d += S;
    s.E = d; d += S;
    s.t = d; d += S;
    s.hf = d; d += S; s.ha = d; d += S; s.hp = d; d += S;
    s.xst = s.xist = s.xsa = s.xnsf = nullptr;
    if (xs) {
        s.xst = d; d += S; s.xist = d; d += S; s.xsa = d; d += S; s.xnsf = d; d += S;
    }
    s.wt = nullptr;
    s.sid = nullptr;
    if (ww) {
        s.wt = d;
        d += S;
    }
    unsigned* u = reinterpret_cast<unsigned*>(d);
    s.g = reinterpret_cast<int*>(u); u += S;
    s.cell = u; u += S; s.id = u; u += S; s.n = u; u += S; s.nsites = u; u += S; s.pend = u; u += S;
    s.prob = u; u += S;
    if (ww) {
        s.sid = u;
        u += S;
    }
    unsigned short* h = reinterpret_cast<unsigned short*>(u);
    for (int q = 0; q < N_QUEUES; ++q) {
        s.q[q] = h;
        h += S;
    }
    s.fr = h;
    h += S;
    size_t off = reinterpret_cast<unsigned char*>(h) - base;
    off = (off + 15) & ~size_t(15);
    s.cnt = reinterpret_cast<int*>(base + off);
    return s;
}

// tm: the problem is timed (or the launch is batched): the particle's time
// travels too; WW: the weight and stream tag (weight-window problems)
template <bool XS, bool WW = false>
__device__ __forceinline__ void slot_load(const Stash& s, int i, Particle& p, bool tm)
{
    p.nsplit = 0u;
    if (WW) {
        p.wt = s.wt[i];
        p.sid = s.sid[i];
    }
    if (tm) p.t = s.t[i];
    p.hf = s.hf[i]; p.ha = s.ha[i]; p.hp = s.hp[i];
    if (XS) {
        p.xst = s.xst[i]; p.xist = s.xist[i]; p.xsa = s.xsa[i]; p.xnsf = s.xnsf[i];
    }
    p.x = s.x[i]; p.y = s.y[i]; p.z = s.z[i];
    p.u = s.u[i]; p.v = s.v[i]; p.w = s.w[i];
    p.iu = s.iu[i]; p.iv = s.iv[i]; p.iw = s.iw[i]; p.ia = s.ia[i];
    p.E = s.E[i]; p.g = s.g[i];
    p.cell = s.cell[i]; p.id = s.id[i]; p.n = s.n[i]; p.nsites = s.nsites[i]; p.pend = s.pend[i];
    p.prob = s.prob[i];
}

template <bool XS, bool WW = false>
__device__ __forceinline__ void slot_store(const Stash& s, int i, const Particle& p, bool tm)
{
    if (WW) {
        s.wt[i] = p.wt;
        s.sid[i] = p.sid;
    }
    if (tm) s.t[i] = p.t;
    s.hf[i] = p.hf; s.ha[i] = p.ha; s.hp[i] = p.hp;
    if (XS) {
        s.xst[i] = p.xst; s.xist[i] = p.xist; s.xsa[i] = p.xsa; s.xnsf[i] = p.xnsf;
    }
    s.x[i] = p.x; s.y[i] = p.y; s.z[i] = p.z;
    s.u[i] = p.u; s.v[i] = p.v; s.w[i] = p.w;
    s.iu[i] = p.iu; s.iv[i] = p.iv; s.iw[i] = p.iw; s.ia[i] = p.ia;
    s.E[i] = p.E; s.g[i] = p.g;
    s.cell[i] = p.cell; s.id[i] = p.id; s.n[i] = p.n; s.nsites[i] = p.nsites; s.pend[i] = p.pend;
    s.prob[i] = p.prob;
}

// Particle state of a global link, read through L2 (ld.global.cg): the link
// was written by another SM, and this SM's L1 may still hold lines from an
// earlier use of the same link.
template <bool XS, bool WW = false>
__device__ __forceinline__ void load_particle_l2(const SoA& s, unsigned long long i, Particle& p)
{
    p.nsplit = 0u;
    if (WW) {
        p.wt = __ldcg(s.wt + i);
        p.sid = __ldcg(s.sid + i);
    }
    if (XS) {
        p.xst = __ldcg(s.xst + i); p.xist = __ldcg(s.xist + i); p.xsa = __ldcg(s.xsa + i); p.xnsf = __ldcg(s.xnsf + i);
    }
    p.x = __ldcg(s.x + i); p.y = __ldcg(s.y + i); p.z = __ldcg(s.z + i);
    p.u = __ldcg(s.u + i); p.v = __ldcg(s.v + i); p.w = __ldcg(s.w + i);
    p.iu = __ldcg(s.iu + i); p.iv = __ldcg(s.iv + i); p.iw = __ldcg(s.iw + i); p.ia = __ldcg(s.ia + i);
    p.E = __ldcg(s.E + i); p.g = __ldcg(s.g + i); p.t = __ldcg(s.t + i);
    p.hf = __ldcg(s.hf + i); p.ha = __ldcg(s.ha + i); p.hp = __ldcg(s.hp + i);
    p.cell = __ldcg(s.cell + i); p.id = __ldcg(s.id + i); p.n = __ldcg(s.n + i);
    p.nsites = __ldcg(s.nsites + i); p.pend = __ldcg(s.pend + i); p.prob = __ldcg(s.prob + i);
}

__device__ __forceinline__ void fail(ErrorWord* err, int code, int where)
{
    if (atomicCAS(&err->code, 0, code) == 0) err->where = where;
}

// Shared-memory lock, taken by lane 0 for the whole warp.  Bounded: the
// spin count and the wall clock are checked every 64 failed tries (a clock
// read per try slowed the contended case); the first tries spin without a
// pause.
__device__ __forceinline__ bool lock_stash(const Stash& s, const RunParams& R, ErrorWord* err)
{
    bool ok = true;
    if ((threadIdx.x & 31) == 0) {
        unsigned long long spins = 0;
        uint64_t t0 = 0;
        while (atomicCAS(s.cnt + CNT_LOCK, 0, 1) != 0) {
            if (spins == 0) t0 = now_ns();
            ++spins;
            if ((spins & 63ull) == 0ull && (spins > R.max_spin || now_ns() - t0 > R.max_wait_ns)) {
                fail(err, ERR_TIMEOUT, 1);
                ok = false;
                break;
            }
            if (spins > 4ull) __nanosleep(32);
        }
        __threadfence_block();
    }
    return __shfl_sync(FULLM, ok, 0);
}

__device__ __forceinline__ void unlock_stash(const Stash& s)
{
    __threadfence_block();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
        __threadfence_block();
        atomicExch(s.cnt + CNT_LOCK, 0);
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// Lock-free global lists: claim by swapping with the empty list, deposit by
// swapping back, merging with whatever was deposited meanwhile.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned list_head(unsigned long long L) { return (unsigned)(L & 0xFFFFFFFFull); }
__device__ __forceinline__ unsigned list_tail(unsigned long long L) { return (unsigned)(L >> 32); }
__device__ __forceinline__ unsigned long long make_list(unsigned h, unsigned t)
{
    return (unsigned long long)h | ((unsigned long long)t << 32);
}

// Called by one lane.  Returns false on timeout or on a corrupt list.
__device__ bool list_deposit(unsigned long long* slot, unsigned long long L, unsigned* next, unsigned long long n_links,
                             const RunParams& R, ErrorWord* err)
{
    unsigned long long spins = 0;
    const uint64_t t0 = now_ns();
    for (;;) {
        __threadfence();
        const unsigned long long cur = atomicExch(slot, EMPTY_LIST);   // claim whatever is there
        if (cur != EMPTY_LIST) {                                        // append it after L
            if (list_tail(L) >= n_links || list_head(cur) >= n_links) {
                fail(err, ERR_INVALID, 8);
                return false;
            }
            next[list_tail(L)] = list_head(cur);
            L = make_list(list_head(L), list_tail(cur));
        }
        __threadfence();
        const unsigned long long old = atomicExch(slot, L);
        if (old == EMPTY_LIST) return true;
        L = old;                                                        // deposited meanwhile: merge again
        if (++spins > R.max_spin || now_ns() - t0 > R.max_wait_ns) {
            fail(err, ERR_TIMEOUT, 2);
            return false;
        }
    }
}

// Pop one link from the lists `q[0..N_GQ)` starting at `start`.  One lane.
// List pointers written by other SMs are read through L2.
__device__ unsigned list_pop(unsigned long long* q, int start, unsigned* next, unsigned long long n_links,
                             const RunParams& R, ErrorWord* err)
{
    for (int t = 0; t < N_GQ; ++t) {
        unsigned long long* slot = q + ((start + t) & (N_GQ - 1));
        if (*(volatile unsigned long long*)slot == EMPTY_LIST) continue;
        const unsigned long long L = atomicExch(slot, EMPTY_LIST);
        if (L == EMPTY_LIST) continue;
        __threadfence();
        const unsigned h = list_head(L);
        if (h >= n_links || list_tail(L) >= n_links) {
            fail(err, ERR_INVALID, 9);
            return NIL;
        }
        if (h != list_tail(L)) {
            const unsigned rest = __ldcg(next + h);
            if (rest >= n_links) {
                fail(err, ERR_INVALID, 10);
                return NIL;
            }
            if (!list_deposit(slot, make_list(rest, list_tail(L)), next, n_links, R, err)) return NIL;
        }
        next[h] = NIL;
        return h;
    }
    return NIL;
}

__device__ __forceinline__ unsigned new_link(const AsyncArgs& A, int start, const RunParams& R, ErrorWord* err)
{
    unsigned l = list_pop(A.ctl->free_q, start, A.link_next, A.n_links, R, err);
    if (l != NIL) return l;
    const unsigned long long k = atomicAdd(&A.ctl->links_made, 1ull);
    if (k < A.n_links) return (unsigned)k;
    return NIL;
}

// Weight-window split copies of this warp's particles (p.nsplit each) into
// free slots of the block's stash, queued for steps (warp-collective).  The
// copies are counted live while the stash is still locked, so no warp can
// take one and end it before it is counted.  A stash without room for them
// is a capacity error.
template <bool XS>
__device__ bool deposit_copies(const Stash& st, const RunParams& R, Particle& p, bool live, AsyncCtl* ctl,
                               ErrorWord* err, bool tm)
{
    const int lane = threadIdx.x & 31;
    const unsigned k = live ? p.nsplit : 0u;
    unsigned incl = k;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(FULLM, incl, o);
        if (lane >= o) incl += y;
    }
    const unsigned total = __shfl_sync(FULLM, incl, 31);
    if (total == 0u) return true;
    const unsigned base = incl - k;
    if (!lock_stash(st, R, err)) return false;
    const int nf = *(volatile int*)(st.cnt + CNT_FREE);
    const int c = *(volatile int*)(st.cnt + Q_STEP);
    const bool ok = nf >= (int)total;
    if (ok) {
        for (unsigned j = 0; j < k; ++j) {
            const Particle q = split_copy(R, p, j + 1u);
            const int sl = st.fr[nf - 1 - (int)(base + j)];
            slot_store<XS, true>(st, sl, q, tm);
            st.q[Q_STEP][c + (int)(base + j)] = (unsigned short)sl;
        }
    }
    __syncwarp();
    if (lane == 0 && ok) {
        atomicAdd(&ctl->live, (unsigned long long)total);
        st.cnt[CNT_FREE] = nf - (int)total;
        st.cnt[Q_STEP] = c + (int)total;
    }
    unlock_stash(st);
    if (!ok) {
        if (lane == 0) fail(err, ERR_CAPACITY, 11);
        return false;
    }
    p.nsplit = 0u;
    return true;
}

// ---------------------------------------------------------------------------
// The persistent kernel
// ---------------------------------------------------------------------------
#ifndef TR_COLL_MIN
#define TR_COLL_MIN 16   // pending collisions that make a warp run its collision pass
#endif
#ifndef TR_COLL_MIN_CE
#define TR_COLL_MIN_CE 16   // the same, continuous energy
#endif
#ifndef TR_DEFER_MIN
#define TR_DEFER_MIN 4      // fewer events between remaps: each pass runs whole events (no deferred collisions)
#endif

// Batch tail of the monolithic loop (source exhausted): a warp left with at
// most TR_TAIL_EXIT live lanes, after TR_TAIL_MINRUN passes, hands its
// particles to the block's other running warps through the stash; a warp with
// a quarter of its lanes idle tops them up from the stash; an idle warp waits
// up to TR_TAIL_WAIT polls for a full warp's worth while other warps run.
#ifndef TR_TAIL_EXIT
#define TR_TAIL_EXIT 16
#endif
#ifndef TR_TAIL_MINRUN
#define TR_TAIL_MINRUN 4
#endif
#ifndef TR_TAIL_WAIT
#define TR_TAIL_WAIT 256
#endif

#ifndef TR_ASYNC_MIN_BLOCKS
#define TR_ASYNC_MIN_BLOCKS 2   // resident blocks per SM the register allocation must allow
#endif

// Source particles sampled ahead of the transport launch: make_work then
// only loads them.  The source event of history i depends on i alone (and its
// fission-bank site), so a pre-sampled particle equals the one make_work
// would sample; the sampling's FP64 work runs in full warps instead of in the
// few lanes a refill serves.
#ifndef TR_PRE_REFILL
#define TR_PRE_REFILL 1   // idle lanes that make a warp refill from pre-sampled sources
#endif

template <bool CE>
__global__ void __launch_bounds__(256) k_presample(DevProblem P, RunParams R, Bank src, int use_src, SoA out)
{
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < R.n_hist; i += stride) {
        Particle p;
        // (directions with the integer-pipe square root and reciprocals: the
        // same bits, and this kernel is FP64-bound)
        const bool ok = source_particle<CE, true>(P, R, (unsigned)i, p, use_src ? &src : nullptr, i);
        out.x[i] = p.x; out.y[i] = p.y; out.z[i] = p.z;
        out.u[i] = p.u; out.v[i] = p.v; out.w[i] = p.w;
        out.iu[i] = p.iu; out.iv[i] = p.iv; out.iw[i] = p.iw; out.ia[i] = p.ia;
        if (CE) out.E[i] = p.E; else out.g[i] = p.g;
        out.cell[i] = p.cell;
        out.id[i] = ok ? (unsigned)i : ~(unsigned)i;   // a failed source keeps another id
    }
}

// Batched launches: problem p owns source indices [hist_off[p], hist_off[p+1]).
__device__ __forceinline__ int find_problem(const unsigned long long* off, int n, unsigned long long gid)
{
    int lo = 0, hi = n;   // off[lo] <= gid < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= gid) lo = mid; else hi = mid;
    }
    return lo;
}

// Batched launches: add a lane's event counts to the tallies of the problem
// they belong to (a lane counts while its particles come from one problem and
// flushes when the problem changes; ended histories add their scalar scores
// to their own problem's bins directly).
__device__ __forceinline__ void flush_lane(Acc& acc, const Tallies& T)
{
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if (acc.ev[i]) atomicAdd(T.ev_type + i, (unsigned long long)acc.ev[i]);
        if (acc.fin[i]) atomicAdd(T.fin_type + i, (unsigned long long)acc.fin[i]);
    }
    acc.zero();
}

// DEC: the task decomposition (DEC_MONO, DEC_SPLIT or DEC_LOOKUP).
// PRE: make_work loads pre-sampled sources (A.pre) instead of sampling them,
// so the sampling code is not part of this kernel.  FUSE (monolithic, fewer
// than TR_DEFER_MIN events between remaps): each pass runs whole events, as
// the paper's monolithic scheme does; a deferred collision would wait for the
// next take.
// WW (monolithic only): weight-window problems -- weighted scores, the
// closeout after every event, split copies deposited into the stash.
template <bool CE, int DEC, bool BATCHED = false, bool PRE = false, bool FUSE = false, bool WW = false>
__global__ void __launch_bounds__(256, TR_ASYNC_MIN_BLOCKS) k_async(DevProblem P, RunParams R, AsyncArgs A, Tallies T, ErrorWord* err)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr bool SPLIT = DEC != DEC_MONO;
    constexpr bool XS = DEC == DEC_LOOKUP;   // cross sections travel with the particle
    static_assert(!WW || (DEC == DEC_MONO && !BATCHED), "weight windows run with the monolithic scheme");
    const int S = A.stash_slots;
    const Stash st = carve(smem, S, XS, WW);
    const int lane = threadIdx.x & 31;
    constexpr int nq = dec_queues(DEC);
    const bool tm = BATCHED || P.timed != 0;   // particle times travel through the stash
    constexpr bool MERGE = !SPLIT && !BATCHED;   // batch-tail consolidation of the monolithic loop
    constexpr bool WALK = !SPLIT && !BATCHED;    // mesh walks deferred to the warp's queue (WalkQ)
    AsyncCtl* ctl = A.ctl;
    WalkQ* wq = nullptr;
    if (WALK && P.has_mesh && P.mesh_walk) {
        if (A.walkq) wq = A.walkq + (size_t)blockIdx.x * 8 + (threadIdx.x >> 5);
        else if (P.walk_smem_off)
            wq = reinterpret_cast<WalkQ*>(smem + P.walk_smem_off + (threadIdx.x >> 5) * walkq_bytes());
    }
    if (wq && lane == 0) wq->n = 0;

    if (threadIdx.x == 0) {
        for (int q = 0; q <= CNT_RUN; ++q) st.cnt[q] = 0;
        st.cnt[CNT_FREE] = S;
    }
    for (int i = threadIdx.x; i < S; i += blockDim.x) st.fr[i] = (unsigned short)(S - 1 - i);
    if (CE && P.hash_smem_off) {
        // the union-grid hash buckets, read by every lookup's first step
        int* h = reinterpret_cast<int*>(smem + P.hash_smem_off);
        for (int i = threadIdx.x; i <= P.n_hash; i += blockDim.x) h[i] = __ldg(P.hash + i);
    }
    __syncthreads();

    Acc acc;
    acc.zero();
    if (!BATCHED) acc_attach(acc, reinterpret_cast<long long*>(smem + fx_offset(S, XS, WW)));
    unsigned long long idle_spins = 0;
    uint64_t idle_t0 = 0;    // when this warp last started waiting for work
    bool idle = false;
    unsigned acc_prob = 0;   // batched: the problem whose scores acc holds
    bool spill_ok = true;   // cleared once the link arena is exhausted
    int tail_wait = 0;      // polls passed over a partial queue while other warps run
    const int qstart = (int)(blockIdx.x * 7 + (threadIdx.x >> 5)) & (N_GQ - 1);

    // warp-uniform reads of the global state (lane 0, broadcast)
    int g_err = 0;
    unsigned long long g_src = 0, g_live = 0;
    unsigned g_hungry = 0;
    auto read_global = [&]() {
        if (lane == 0) {
            g_err = *(volatile int*)&err->code;
            g_src = *(volatile unsigned long long*)&ctl->src_cursor;
            g_live = *(volatile unsigned long long*)&ctl->live;
            g_hungry = *(volatile unsigned*)&ctl->hungry;
        }
        g_err = __shfl_sync(FULLM, g_err, 0);
        g_src = __shfl_sync(FULLM, g_src, 0);
        g_live = __shfl_sync(FULLM, g_live, 0);
        g_hungry = __shfl_sync(FULLM, g_hungry, 0);
    };
    // a deposit keeps the stash lock for the take that follows it (one lock
    // round per event instead of two); the global state is then read before
    // the deposit
    bool held = false;
    for (;;) {
        if (!held) read_global();
        if (g_err != 0) {
            if (held) unlock_stash(st);
            break;
        }
        // ---------------- take work (under the stash lock) ----------------
        if (!held && !lock_stash(st, R, err)) break;
        held = false;
        int cnts[N_QUEUES] = {};
#pragma unroll
        for (int q = 0; q < nq; ++q) cnts[q] = *(volatile int*)(st.cnt + q);
        const int nfree = *(volatile int*)(st.cnt + CNT_FREE);
        const int n_run = *(volatile int*)(st.cnt + CNT_RUN);
        int q = 0;
        for (int k = 1; k < nq; ++k)
            if (cnts[k] > cnts[q]) q = k;
        const bool src_left = g_src < R.n_hist;
        // mode: 0 process a link of queue q, 1 make_work, 2 spill, 3 idle
        int mode, take;
        const int thr = R.spill_threshold < 0 ? -R.spill_threshold : R.spill_threshold;
        const bool want_spill = spill_ok && (R.spill_threshold < 0 ||
                                             (!src_left && g_hungry > 0u));
        if (want_spill && cnts[q] >= thr + 32) {
            mode = 2;
            take = 32;
        } else if (cnts[q] >= 32) {
            mode = 0;
            take = 32;
        } else if (src_left && nfree >= 32) {
            mode = 1;
            take = 32;
        } else if (cnts[q] > 0 && (!MERGE || src_left || n_run == 0 || tail_wait >= TR_TAIL_WAIT ||
                                   R.remap_every < TR_TAIL_MINRUN)) {
            // a partial queue; in the batch tail only once no other warp of the
            // block runs (it would take these particles into its idle lanes)
            // or after TR_TAIL_WAIT polls, unless warps run too few passes to
            // take particles in
            mode = 0;
            take = cnts[q];
        } else {
            mode = 3;
            take = 0;
        }
        tail_wait = (mode == 3 && cnts[q] > 0) ? tail_wait + 1 : 0;
        int slot = -1;
        if (mode == 0 || mode == 2) {
            if (lane < take) slot = st.q[q][cnts[q] - take + lane];
        } else if (mode == 1) {
            slot = st.fr[nfree - 32 + lane];
        }
        __syncwarp();
        if (lane == 0) {
            if (mode == 0 || mode == 2) st.cnt[q] = cnts[q] - take;
            else if (mode == 1) st.cnt[CNT_FREE] = nfree - 32;
            if (MERGE && (mode == 0 || mode == 1)) st.cnt[CNT_RUN] = n_run + 1;
        }
        unlock_stash(st);

        if (mode == 3) {
            // ---------------- starving: steal, or wait for termination ----------------
            if (!idle) {
                idle = true;
                idle_t0 = now_ns();
                if (lane == 0) atomicAdd(&ctl->hungry, 1u);
            }
            unsigned link = NIL;
            if (lane == 0) link = list_pop(ctl->full_q, qstart, A.link_next, A.n_links, R, err);
            link = __shfl_sync(FULLM, link, 0);
            if (link != NIL) {
                // refill: move the link's particles into free slots of this stash
                __threadfence();
                __syncwarp();
                const int fill = __ldcg(A.link_fill + link);
                const int type = __ldcg(A.link_type + link);
                if (link >= A.n_links || fill < 1 || fill > 32 || type < 0 || type >= nq) {
                    if (lane == 0) fail(err, ERR_INVALID, 6);
                    break;
                }
                bool ok = lock_stash(st, R, err);
                if (!ok) break;
                const int nf = *(volatile int*)(st.cnt + CNT_FREE);
                int sl = -1;
                if (lane < fill && nf >= fill) sl = st.fr[nf - fill + lane];
                __syncwarp();
                if (lane == 0 && nf >= fill) st.cnt[CNT_FREE] = nf - fill;
                unlock_stash(st);
                if (nf < fill) {
                    fail(err, ERR_CAPACITY, 3);
                    break;
                }
                bool bad = false;
                if (lane < fill) {
                    Particle p;
                    load_particle_l2<XS, WW>(A.links, (unsigned long long)link * 32 + lane, p);
                    bad = BATCHED && p.prob >= (unsigned)A.n_probs;
                    const DevProblem& PP = (BATCHED && !bad) ? A.probs[p.prob] : P;
                    bad = bad || p.id >= R.n_hist || cell_i(p.cell) >= PP.nx || cell_j(p.cell) >= PP.ny ||
                          cell_k(p.cell) >= PP.nz || sl < 0 || sl >= S || (!CE && (p.g < 0 || p.g >= PP.G));
                    if (!bad && cell_in(p.cell)) bad = info_pin(cell_info(PP, p.cell)) < 0;
                    if (!bad) slot_store<XS, WW>(st, sl, p, tm);
                }
                if (__any_sync(FULLM, bad)) {
                    if (lane == 0) fail(err, ERR_INVALID, 7);
                    break;
                }
                __syncwarp();
                if (lane == 0) {
                    A.link_next[link] = NIL;
                    list_deposit(ctl->free_q + qstart, make_list(link, link), A.link_next, A.n_links, R, err);
                    atomicAdd(&ctl->refills, 1ull);
                }
                idle_t0 = now_ns();   // a refill is progress: restart the wait bound
                idle_spins = 0;
                ok = lock_stash(st, R, err);
                if (!ok) break;
                const int c = *(volatile int*)(st.cnt + type);
                if (lane < fill) st.q[type][c + lane] = (unsigned short)sl;
                __syncwarp();
                if (lane == 0) st.cnt[type] = c + fill;
                unlock_stash(st);
                continue;
            }
            if (!src_left && g_live == 0ull) break;
            // bounded in iterations and in time; the warp-uniform decision
            // comes from lane 0's clock
            bool give_up = ++idle_spins > R.max_spin;
            if (lane == 0) give_up = give_up || now_ns() - idle_t0 > R.max_wait_ns;
            if (__shfl_sync(FULLM, give_up, 0)) {
                if (lane == 0) fail(err, ERR_TIMEOUT, 4);
                break;
            }
            __nanosleep(50);
            continue;
        }
        if (idle) {
            idle = false;
            idle_spins = 0;
            if (lane == 0) atomicSub(&ctl->hungry, 1u);
        }

        if (mode == 2) {
            // ---------------- spill one full link to global memory ----------------
            unsigned link = NIL;
            if (lane == 0) link = new_link(A, qstart, R, err);
            link = __shfl_sync(FULLM, link, 0);
            if (link == NIL) {
                // arena exhausted: keep the particles local and stop spilling
                if (!lock_stash(st, R, err)) break;
                const int c = *(volatile int*)(st.cnt + q);
                st.q[q][c + lane] = (unsigned short)slot;
                __syncwarp();
                if (lane == 0) st.cnt[q] = c + 32;
                unlock_stash(st);
                spill_ok = false;
                continue;
            }
            Particle p;
            slot_load<XS, WW>(st, slot, p, tm);
            store_particle(A.links, (unsigned long long)link * 32 + lane, p, CE, XS, WW);
            __threadfence();
            __syncwarp();
            if (lane == 0) {
                A.link_fill[link] = 32;
                A.link_type[link] = q;
                A.link_next[link] = NIL;
                list_deposit(ctl->full_q + qstart, make_list(link, link), A.link_next, A.n_links, R, err);
                atomicAdd(&ctl->spills, 1ull);
            }
            if (!lock_stash(st, R, err)) break;
            const int nf = *(volatile int*)(st.cnt + CNT_FREE);
            st.fr[nf + lane] = (unsigned short)slot;
            __syncwarp();
            if (lane == 0) st.cnt[CNT_FREE] = nf + 32;
            unlock_stash(st);
            continue;
        }

#ifdef TR_PROFILE_LANES
        {   // exact warp fill per iteration: sites 26 + queue (mode 0) and 30 (make_work)
            const unsigned hm = __ballot_sync(FULLM, slot >= 0);
            if (lane == 0 && hm) {
                const int site = mode == 1 ? 30 : 26 + q;
                atomicAdd(&g_lane_prof[2 * site], 1ull);
                atomicAdd(&g_lane_prof[2 * site + 1], (unsigned long long)__popc(hm));
            }
        }
#endif
        // ---------------- run one event (or make_work) ----------------
        Particle p;
        bool live = false;
        int next = Q_DEAD;
        if (mode == 1) {
            unsigned long long first = 0;
            if (lane == 0) first = atomicAdd(&ctl->src_cursor, 32ull);
            first = __shfl_sync(FULLM, first, 0);
            const unsigned long long id = first + lane;
            __syncwarp();   // reconverge: the event below must run once for all lanes, not per lane group
            if (id < R.n_hist) {
                TR_LANES(11);
                if (BATCHED) {
                    const int pi = find_problem(A.hist_off, A.n_probs, id);
                    RunParams RR = R;
                    RR.key1 = R.key1 ^ (uint32_t)pi;
                    const unsigned lid = (unsigned)(id - __ldg(A.hist_off + pi));
                    live = source_particle<CE>(A.probs[pi], RR, lid, p, nullptr, 0);
                    p.prob = (unsigned)pi;
                    if ((unsigned)pi != acc_prob) {
                        flush_lane(acc, A.tallies[acc_prob]);
                        acc_prob = (unsigned)pi;
                    }
                    acc.ev[EV_SOURCE] += 1u;
                } else {
                    if constexpr (PRE) live = load_presampled<CE>(A.pre, id, p);
                    else live = source_particle<CE>(P, R, (unsigned)id, p, A.use_src ? &A.src : nullptr, id);
                    acc.ev[EV_SOURCE] += 1u;
                }
                if (!live) fail(err, ERR_INVALID, 5);
                next = XS ? Q_LOOKUP : Q_STEP;
            }
            const unsigned made = __popc(__ballot_sync(FULLM, live));
            if (lane == 0 && made) atomicAdd(&ctl->live, (unsigned long long)made);
        } else {
            // mode 0 (warp-uniform): lanes beyond a partial link hold no slot and stay idle
            if (slot >= 0) slot_load<XS, WW>(st, slot, p, tm);
            __syncwarp();   // reconverge: the event below must run once for all lanes, not per lane group
            const unsigned em = __ballot_sync(FULLM, slot >= 0);   // the lanes that hold a particle
            if (slot >= 0) {
                __syncwarp(em);
                TR_LANES(0);
                live = true;
                // batched: the particle's own problem, random-stream tag and tallies
                const DevProblem& PP = BATCHED ? A.probs[p.prob] : P;
                const Tallies& TT = BATCHED ? A.tallies[p.prob] : T;
                RunParams RR = R;
                if (BATCHED) {
                    RR.key1 = R.key1 ^ p.prob;
                    if (p.prob != acc_prob) {
                        flush_lane(acc, A.tallies[acc_prob]);
                        acc_prob = p.prob;
                    }
                }
                if (!SPLIT) {
                    // Up to remap_every passes.  While the source lasts, a lane
                    // whose history ended starts the next source history in
                    // place (make_work inside the loop), so the warp stays full;
                    // the live count needs no update for that (the lane's death
                    // and its new history cancel).  A step that ends in a
                    // collision leaves the collision pending; a pass runs either
                    // the steps (with their surface crossings) of the lanes with
                    // nothing pending, or, once TR_COLL_MIN lanes are pending
                    // (or nothing else can step), their collisions together, so
                    // the FP64 work of the collision is issued for many lanes
                    // at once.  A multigroup collision recomputes its lookup and
                    // reaction draw from the counter-based keys; a continuous-
                    // energy one reuses what its step kept.  Histories are the
                    // same.  (Below TR_DEFER_MIN passes the FUSE variant runs
                    // whole events instead.)
                    // Every lane holding a slot stays in the loop, so the
                    // ballots name em; a pending collision survives a remap in
                    // p.pend.  Once the source is exhausted (the batch tail),
                    // histories end and lanes empty; the block's warps then
                    // consolidate through the stash: a warp with a quarter of
                    // its lanes idle takes waiting particles into them, and a
                    // warp left with few live lanes deposits its particles for
                    // the others, so fewer, fuller warps issue the FP64 work.
                    bool src_more = !BATCHED && src_left;
                    const int leader = __ffs(em) - 1;
                    bool pend_coll = live && p.pend == PEND_COLLIDE;
                    // continuous energy: a collision deferred in the lane that made
                    // its step reuses the step's lookup terms (ck); one that
                    // arrived pending from the stash computes them again
                    CEKeep ck;
                    bool ck_ok = false;
                    for (int r = 0; r < R.remap_every; ++r) {
                        // weight windows: a pass that left split copies ends
                        // the take, so that the whole warp deposits them
                        if (WW && __any_sync(em, live && p.nsplit != 0u)) break;
                        if (MERGE && r > 0 && !src_more && em == FULLM) {
                            const unsigned dead = __ballot_sync(FULLM, !live);
                            const int nd = __popc(dead);
                            if (4 * nd >= 32) {
                                int avail = 0, others = 0;
                                if (lane == 0) {
                                    avail = *(volatile int*)(st.cnt + Q_STEP);
                                    others = *(volatile int*)(st.cnt + CNT_RUN) - 1;
                                }
                                avail = __shfl_sync(FULLM, avail, 0);
                                others = __shfl_sync(FULLM, others, 0);
                                if (avail > 0) {
                                    // top up: the first k idle lanes adopt waiting
                                    // particles and free their own slots
                                    if (!lock_stash(st, R, err)) break;
                                    const int c = *(volatile int*)(st.cnt + Q_STEP);
                                    const int nf = *(volatile int*)(st.cnt + CNT_FREE);
                                    const int k = c < nd ? c : nd;
                                    const int rank = __popc(dead & ((1u << lane) - 1u));
                                    const bool adopt = !live && rank < k;
                                    int ns = -1;
                                    if (adopt) {
                                        ns = st.q[Q_STEP][c - k + rank];
                                        st.fr[nf + rank] = (unsigned short)slot;
                                    }
                                    __syncwarp();
                                    if (lane == 0) {
                                        st.cnt[Q_STEP] = c - k;
                                        st.cnt[CNT_FREE] = nf + k;
                                    }
                                    unlock_stash(st);
                                    // the adopted particles were already counted live;
                                    // the k histories they replace ended here
                                    if (lane == 0 && k > 0) atomicAdd(&ctl->live, 0ull - (unsigned long long)k);
                                    if (adopt) {
                                        slot = ns;
                                        slot_load<XS, WW>(st, slot, p, tm);
                                        live = true;
                                        pend_coll = p.pend == PEND_COLLIDE;
                                        ck_ok = false;
                                    }
                                } else if (32 - nd <= TR_TAIL_EXIT && r >= TR_TAIL_MINRUN && others > 0) {
                                    break;   // deposit: the block's running warps take these
                                }
                            }
                        }
                        if (!BATCHED && r > 0 && src_more) {
                            // refill once a quarter of the warp is idle (the source
                            // sampling then runs for several lanes at once), or,
                            // with pre-sampled sources (a load), once
                            // TR_PRE_REFILL lanes are idle
                            const unsigned dead = __ballot_sync(em, !live);
                            const int nd = __popc(dead);
                            if ((PRE ? nd >= TR_PRE_REFILL : 4 * nd >= __popc(em)) || dead == em) {
                                unsigned long long first = 0;
                                if (lane == leader) first = atomicAdd(&ctl->src_cursor, (unsigned long long)__popc(dead));
                                first = __shfl_sync(em, first, leader);
                                if (first + __popc(dead) >= R.n_hist) src_more = false;
                                if (!live) {
                                    const unsigned long long gid = first + __popc(dead & ((1u << lane) - 1u));
                                    if (gid < R.n_hist) {
                                        if constexpr (PRE) live = load_presampled<CE>(A.pre, gid, p);
                                        else live = source_particle<CE>(P, R, (unsigned)gid, p,
                                                                        A.use_src ? &A.src : nullptr, gid);
                                        if (!live) fail(err, ERR_INVALID, 5);
                                        acc.ev[EV_SOURCE] += 1u;
                                        pend_coll = false;
                                    }
                                }
                            }
                        }
                        const unsigned lm = __ballot_sync(em, live);
                        if (!lm) break;
                        if constexpr (WALK) {
                            // drain 32 deferred mesh walks once 32 are queued, before a
                            // pass that may queue 32 more
                            if (wq) {
                                __syncwarp(em);
                                int nq_w = *(volatile int*)&wq->n;
                                nq_w = nq_w < WALKQ_CAP ? nq_w : WALKQ_CAP;
                                if (nq_w >= 32) {
                                    walk_run<WW>(PP, TT, wq, nq_w - 32, nq_w, em);
                                    __syncwarp(em);
                                    if (lane == leader) wq->n = nq_w - 32;
                                    __syncwarp(em);
                                }
                            }
                        }
                        TR_LANES(12);
                        if (!src_more) TR_LANES(25);
                        if (live) TR_LANES(13);
                        if (live && !src_more) TR_LANES(31);
                        if constexpr (FUSE) {
                            if (live) live = mono_event<CE, WW, WALK>(PP, RR, p, TT, acc, A.bank, err, lm, wq);
                            continue;
                        }
                        if constexpr (CE) {
                            // A pass is either the collision pass (warp-uniform
                            // choice) or the step pass; either way each lane ends
                            // at most one event.  Continuous energy closes it with
                            // one finish_event below (one inlined copy of the
                            // closing code and of the collision, whether the lane
                            // kept its step's lookup terms or computes them again:
                            // measured faster); multigroup keeps a closing copy per
                            // path (measured faster there).
                            const unsigned pm = __ballot_sync(em, live && pend_coll);
                            const bool cpass = pm == lm || __popc(pm) >= TR_COLL_MIN_CE;
                            int type = -1;
                            if (cpass) {
                                if (live && pend_coll) {
                                    TR_LANES(15);
                                    tr::XS X;
                                    double xr;
                                    X.keep = &ck;
                                    if (ck_ok) {
                                        // the step's lookup terms, sigma_t and reaction draw
                                        X.st = ck.st;
                                        X.inv_st = X.sa = X.nsf = 0.0;
                                        xr = ck.xi;
                                    } else {
                                        // arrived pending from the stash: the lookup
                                        // and the draw again, the same values
                                        xs_lookup<CE>(PP, p, material(PP, p.cell), X);
                                        const Stream S = particle_stream<WW>(RR, p);
                                        const uint4 b0 = S.block(p.n, BLK_MAIN);
                                        xr = u01(b0.z, b0.w);
                                    }
                                    type = collide_event<CE, WW>(PP, RR, p, X, xr, A.bank, err, pm);
                                    pend_coll = false;
                                    p.pend = 0u;
                                }
                            } else if (live && !pend_coll) {
                                TR_LANES(14);
                                tr::XS X;
                                X.keep = &ck;
                                double xr;
                                FwdSinkT<WW, WALK> sink{TT, acc, 1.0, wq};
                                step_event<CE>(PP, RR, p, sink, X, xr);
                                if (p.pend == PEND_COLLIDE) {
                                    pend_coll = true;
                                    ck_ok = true;
                                    ck.st = X.st;
                                    ck.xi = xr;
                                } else {
                                    type = surface_event(PP, p);
                                    p.pend = 0u;
                                }
                            }
                            if (type >= 0) live = finish_event<WW>(PP, RR, p, type, TT, acc, A.bank);
                            continue;
                        }
                        const unsigned pm = __ballot_sync(em, live && pend_coll);
                        if (pm == lm || __popc(pm) >= TR_COLL_MIN) {
                            if (live && pend_coll) {
                                TR_LANES(15);
                                live = split_collide<CE, false, WW>(PP, RR, p, TT, acc, A.bank, err, pm);
                                pend_coll = false;
                                p.pend = 0u;
                            }
                        } else if (live && !pend_coll) {
                            TR_LANES(14);
                            tr::XS X;
                            double xr;
                            FwdSinkT<WW, WALK> sink{TT, acc, 1.0, wq};
                            step_event<CE>(PP, RR, p, sink, X, xr);
                            if (p.pend == PEND_COLLIDE) {
                                pend_coll = true;
                            } else {
                                live = finish_event<WW>(PP, RR, p, surface_event(PP, p), TT, acc, A.bank);
                                p.pend = 0u;
                            }
                        }
                    }
                    next = live ? Q_STEP : Q_DEAD;
                } else if (DEC == DEC_STREAM) {
                    // streaming: a deferred collision (collision queue) first,
                    // then steps and surface crossings inline; the next
                    // collision sends the particle back to the collision queue
                    next = Q_STEP;
                    if (q == Q_COLLIDE) {
                        live = split_collide<CE, false>(PP, RR, p, TT, acc, A.bank, err, em);
                        next = live ? Q_STEP : Q_DEAD;
                    }
                    unsigned lm = em;
                    for (int r = 0; r < R.remap_every; ++r) {
                        const bool go = live && next == Q_STEP;
                        lm = __ballot_sync(lm, go);
                        if (!go) break;
                        tr::XS X;
                        double xr;
                        FwdSink sink{TT, acc};
                        step_event<CE>(PP, RR, p, sink, X, xr);
                        if (p.pend == PEND_COLLIDE) {
                            next = Q_COLLIDE;
                        } else {
                            live = split_surface(PP, RR, p, TT, acc, A.bank);
                            next = live ? Q_STEP : Q_DEAD;
                        }
                    }
                } else if (q == Q_STEP) {
                    tr::XS X;
                    double xr;
                    FwdSink sink{TT, acc};
                    step_event<CE, XS>(PP, RR, p, sink, X, xr);
                    next = next_queue_after_step(p);
                } else if (q == Q_COLLIDE) {
                    live = split_collide<CE, XS>(PP, RR, p, TT, acc, A.bank, err, em);
                    next = live ? (XS ? Q_LOOKUP : Q_STEP) : Q_DEAD;
                } else if (XS && q == Q_LOOKUP) {
                    lookup_event<CE>(PP, p);
                    next = Q_STEP;
                } else if (XS) {
                    next = split_surface_next(PP, RR, p, TT, acc, A.bank);
                    live = next != Q_DEAD;
                } else {
                    live = split_surface(PP, RR, p, TT, acc, A.bank);
                    next = live ? Q_STEP : Q_DEAD;
                }
                if (!live) next = Q_DEAD;
            }
            const unsigned died = __popc(__ballot_sync(FULLM, slot >= 0 && !live));
            if (lane == 0 && died) atomicAdd(&ctl->live, 0ull - (unsigned long long)died);
        }
        if (live) slot_store<XS, WW>(st, slot, p, tm);
        // ---------------- deposit (under the stash lock) ----------------
        __syncwarp();
        if constexpr (WW) {
            if (!deposit_copies<XS>(st, R, p, live, ctl, err, tm)) break;   // split copies first
        }
        read_global();
        if (!lock_stash(st, R, err)) break;
        const bool has = slot >= 0;
        if (MERGE && lane == 0) st.cnt[CNT_RUN] -= 1;
        for (int qq = 0; qq <= N_QUEUES; ++qq) {
            if (qq < N_QUEUES && qq >= nq) continue;   // queues this decomposition never fills
            const bool mine = has && (qq == N_QUEUES ? next == Q_DEAD : next == qq);
            const unsigned mask = __ballot_sync(FULLM, mine);
            if (!mask) continue;
            int* cp = st.cnt + (qq == N_QUEUES ? CNT_FREE : qq);
            const int c = *(volatile int*)cp;
            if (mine) {
                const int pos = c + __popc(mask & ((1u << lane) - 1u));
                if (qq == N_QUEUES) st.fr[pos] = (unsigned short)slot;
                else st.q[qq][pos] = (unsigned short)slot;
            }
            __syncwarp();
            if (lane == 0) *cp = c + __popc(mask);
            __syncwarp();
        }
        // (not with forced spills, a diagnostic setting: they need queues
        // that build up between other warps' deposits and takes)
        held = R.spill_threshold >= 0;
        if (!held) unlock_stash(st);
    }
    if (idle && lane == 0) atomicSub(&ctl->hungry, 1u);
    if constexpr (WALK) {
        if (wq) {   // the warp's remaining deferred mesh walks
            __syncwarp();
            const int nq_w = *(volatile int*)&wq->n;
            walk_run<WW>(P, T, wq, 0, nq_w < WALKQ_CAP ? nq_w : WALKQ_CAP, FULLM);
        }
    }
    if (BATCHED) flush_lane(acc, A.tallies[acc_prob]);
    else flush_acc(acc, T);
}

}  // namespace tr

namespace tr {

template <bool CE, int DEC, bool BATCHED = false, bool PRE = false, bool FUSE = false, bool WW = false>
static cudaError_t prepare_async(size_t smem)
{
    return cudaFuncSetAttribute(k_async<CE, DEC, BATCHED, PRE, FUSE, WW>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <bool CE, int DEC, bool BATCHED = false, bool PRE = false, bool FUSE = false, bool WW = false>
static int occupancy_async(size_t smem)
{
    int nb = 0;
    if (prepare_async<CE, DEC, BATCHED, PRE, FUSE, WW>(smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_async<CE, DEC, BATCHED, PRE, FUSE, WW>, 256, smem) !=
        cudaSuccess)
        return 0;
    return nb;
}

// Continuous energy: the union-grid hash buckets (n_hash + 1 ints) are staged
// in each block's shared memory, after the stash and the score sums, when
// they fit there at TR_ASYNC_MIN_BLOCKS blocks per SM (228 KB per SM, 1 KB of
// it reserved per block) and take at most TR_HASH_SMEM_MAX bytes.  Returns
// the byte offset (0: not staged); *total becomes the block's dynamic shared
// memory.
#ifndef TR_HASH_SMEM_MAX
#define TR_HASH_SMEM_MAX (64 * 1024)
#endif
static size_t hash_stage(const DevProblem& P, size_t smem, size_t* total)
{
    *total = smem;
    if (P.kind != 1 || !P.hash || P.n_hash < 1) return 0;
    const size_t off = (smem + 15) & ~size_t(15);
    const size_t bytes = (size_t)(P.n_hash + 1) * sizeof(int);
    if (bytes > TR_HASH_SMEM_MAX || (off + bytes + 1024) * TR_ASYNC_MIN_BLOCKS > 228 * 1024) return 0;
    *total = off + bytes;
    return off;
}

// Dynamic shared memory of a non-batched launch: the stash and the score
// sums; with walk_smem, the monolithic kernel's mesh-walk queues (one WalkQ
// per warp) when the problem has cells that lie in no single mesh voxel; the
// union-grid hash when it fits.  Sets the offsets in P; returns the bytes.
static size_t async_layout(DevProblem& P, int dec, int stash_slots, bool walk_smem)
{
    size_t smem = async_smem_bytes(stash_slots, dec == DEC_LOOKUP, P.ww_lo != nullptr);
    P.walk_smem_off = 0;
    if (walk_smem && dec == DEC_MONO && P.has_mesh && P.mesh_walk) {
        const size_t off = (smem + 15) & ~size_t(15);
        P.walk_smem_off = (int)off;
        smem = off + 8 * walkq_bytes();   // 256 threads: 8 warps
    }
    size_t total;
    P.hash_smem_off = (int)hash_stage(P, smem, &total);
    return total;
}

size_t walk_queue_bytes(int blocks) { return (size_t)blocks * 8 * sizeof(WalkQ); }

int async_max_blocks_per_sm(const DevProblem& Pin, int dec, int stash_slots, bool pre, bool walk_smem)
{
    DevProblem P = Pin;
    const size_t smem = async_layout(P, dec, stash_slots, walk_smem);
    if (P.ww_lo) {
        return P.kind == 1 ? occupancy_async<true, DEC_MONO, false, false, false, true>(smem)
                           : occupancy_async<false, DEC_MONO, false, false, false, true>(smem);
    }
    if (pre && dec == DEC_MONO)
        return P.kind == 1 ? occupancy_async<true, DEC_MONO, false, true>(smem)
                           : occupancy_async<false, DEC_MONO, false, true>(smem);
    if (P.kind == 1) {
        if (dec == DEC_STREAM) return occupancy_async<true, DEC_STREAM>(smem);
        if (dec == DEC_LOOKUP) return occupancy_async<true, DEC_LOOKUP>(smem);
        return dec == DEC_SPLIT ? occupancy_async<true, DEC_SPLIT>(smem) : occupancy_async<true, DEC_MONO>(smem);
    }
    if (dec == DEC_STREAM) return occupancy_async<false, DEC_STREAM>(smem);
    if (dec == DEC_LOOKUP) return occupancy_async<false, DEC_LOOKUP>(smem);
    return dec == DEC_SPLIT ? occupancy_async<false, DEC_SPLIT>(smem) : occupancy_async<false, DEC_MONO>(smem);
}

template <bool CE, int DEC, bool BATCHED = false, bool PRE = false, bool FUSE = false, bool WW = false>
static cudaError_t launch_async_t(const DevProblem& P, const RunParams& R, const AsyncArgs& A, const Tallies& T,
                                  ErrorWord* err, int blocks, cudaStream_t st, size_t smem)
{
    const cudaError_t e = prepare_async<CE, DEC, BATCHED, PRE, FUSE, WW>(smem);
    if (e != cudaSuccess) return e;
    k_async<CE, DEC, BATCHED, PRE, FUSE, WW><<<blocks, 256, smem, st>>>(P, R, A, T, err);
    return cudaGetLastError();
}

// The monolithic kernel for a run: pre-sampled sources or not, whole events
// per pass (fewer than TR_DEFER_MIN events between remaps) or deferred collisions.
template <bool CE>
static cudaError_t launch_async_mono(const DevProblem& P, const RunParams& R, const AsyncArgs& A, const Tallies& T,
                                     ErrorWord* err, int blocks, cudaStream_t st, size_t smem)
{
    const bool fuse = R.remap_every < TR_DEFER_MIN;
    if (P.ww_lo)   // weight windows: sources sampled in the loop
        return fuse ? launch_async_t<CE, DEC_MONO, false, false, true, true>(P, R, A, T, err, blocks, st, smem)
                    : launch_async_t<CE, DEC_MONO, false, false, false, true>(P, R, A, T, err, blocks, st, smem);
    if (A.use_pre)
        return fuse ? launch_async_t<CE, DEC_MONO, false, true, true>(P, R, A, T, err, blocks, st, smem)
                    : launch_async_t<CE, DEC_MONO, false, true>(P, R, A, T, err, blocks, st, smem);
    return fuse ? launch_async_t<CE, DEC_MONO, false, false, true>(P, R, A, T, err, blocks, st, smem)
                : launch_async_t<CE, DEC_MONO>(P, R, A, T, err, blocks, st, smem);
}

cudaError_t launch_async(const DevProblem& Pin, const RunParams& R, const AsyncArgs& A, const Tallies& T,
                         ErrorWord* err, int blocks, cudaStream_t st, int* smem_bytes_out)
{
    DevProblem P = Pin;
    const size_t smem = async_layout(P, A.dec, A.stash_slots, A.walkq == nullptr);
    if (smem_bytes_out) *smem_bytes_out = (int)smem;
    count_launches(1);
    if (A.dec == DEC_MONO)
        return P.kind == 1 ? launch_async_mono<true>(P, R, A, T, err, blocks, st, smem)
                           : launch_async_mono<false>(P, R, A, T, err, blocks, st, smem);
    if (P.kind == 1) {
        if (A.dec == DEC_STREAM) return launch_async_t<true, DEC_STREAM>(P, R, A, T, err, blocks, st, smem);
        if (A.dec == DEC_LOOKUP) return launch_async_t<true, DEC_LOOKUP>(P, R, A, T, err, blocks, st, smem);
        return launch_async_t<true, DEC_SPLIT>(P, R, A, T, err, blocks, st, smem);
    }
    if (A.dec == DEC_STREAM) return launch_async_t<false, DEC_STREAM>(P, R, A, T, err, blocks, st, smem);
    if (A.dec == DEC_LOOKUP) return launch_async_t<false, DEC_LOOKUP>(P, R, A, T, err, blocks, st, smem);
    return launch_async_t<false, DEC_SPLIT>(P, R, A, T, err, blocks, st, smem);
}

cudaError_t launch_presample(const DevProblem& P, const RunParams& R, const AsyncArgs& A, int blocks, cudaStream_t st)
{
    count_launches(1);
    if (P.kind == 1) k_presample<true><<<blocks, 256, 0, st>>>(P, R, A.src, A.use_src, A.pre);
    else k_presample<false><<<blocks, 256, 0, st>>>(P, R, A.src, A.use_src, A.pre);
    return cudaGetLastError();
}

// Batched launches (multigroup; monolithic or decomposed).
int async_batched_max_blocks_per_sm(int dec, int stash_slots)
{
    const size_t smem = async_smem_bytes(stash_slots, false);
    return dec == DEC_SPLIT ? occupancy_async<false, DEC_SPLIT, true>(smem) : occupancy_async<false, DEC_MONO, true>(smem);
}

cudaError_t launch_async_batched(const DevProblem& P0, const RunParams& R, const AsyncArgs& A, ErrorWord* err,
                                 int blocks, cudaStream_t st)
{
    const size_t smem = async_smem_bytes(A.stash_slots, false);
    const Tallies T{};
    count_launches(1);
    if (A.dec == DEC_SPLIT) return launch_async_t<false, DEC_SPLIT, true>(P0, R, A, T, err, blocks, st, smem);
    if (R.remap_every < TR_DEFER_MIN)
        return launch_async_t<false, DEC_MONO, true, false, true>(P0, R, A, T, err, blocks, st, smem);
    return launch_async_t<false, DEC_MONO, true>(P0, R, A, T, err, blocks, st, smem);
}

}  // namespace tr

#ifdef TR_PROFILE_LANES
// Diagnostic builds only: copy and clear the lane-occupancy counters.
extern "C" int tr_profile_lanes_read(unsigned long long* out, int n)
{
    if (n > 64) n = 64;
    if (cudaMemcpyFromSymbol(out, tr::g_lane_prof, n * sizeof(unsigned long long)) != cudaSuccess) return 1;
    unsigned long long z[64] = {};
    return cudaMemcpyToSymbol(tr::g_lane_prof, z, sizeof(z)) != cudaSuccess;
}
#endif
