// tr_stack.cu -- stack-based remapping (Sec. 3.1 of Cuneo et al., M&C 2025)
// and the per-batch kernels of the power iteration.
//
// Stack-based remapping keeps, per event type, one global input and one
// global output buffer used as pop-only / push-only stacks.  Warps pop 32
// particles with one atomic add, hold each particle in registers while its
// event runs, and push survivors with one atomic add per warp and destination
// (ballot / match_any ranks).  A warp calls make_work only once the input
// stacks have been claimed completely, and only while the output stacks have
// room (the launch threshold of Sec. 3.1); the host relaunches until the
// source is exhausted and the stacks are empty.
#include "tr_events.cuh"
#include "tr_kernels.h"

#include <atomic>

namespace tr {

constexpr unsigned FULL = 0xFFFFFFFFu;

// warp-aggregated push of `p` (if `live`) onto stack `dst` of the output set;
// a push beyond the capacity (which the launch-threshold rule prevents) is not
// written and raises a capacity error
__device__ __forceinline__ void push_to(const SoA* outs, unsigned long long* out_count, int dst, bool live,
                                        const Particle& p, bool ce, unsigned long long cap, ErrorWord* err,
                                        bool xs = false, bool ww = false)
{
    const int lane = threadIdx.x & 31;
    const unsigned act = __ballot_sync(FULL, live);
    if (!act) return;
    const int key = live ? dst : -1;
    const unsigned grp = __match_any_sync(FULL, key);
    const int leader = __ffs(grp) - 1;
    unsigned long long base = 0;
    if (live && lane == leader) base = atomicAdd(out_count + dst, (unsigned long long)__popc(grp));
    base = __shfl_sync(FULL, base, leader);
    if (live) {
        const unsigned long long pos = base + __popc(grp & ((1u << lane) - 1u));
        if (pos < cap) store_particle(outs[dst], pos, p, ce, xs, ww);
        else atomicCAS(&err->code, 0, ERR_CAPACITY);
    }
}

struct StackArgs {
    SoA in[N_QUEUES], out[N_QUEUES];
    StackCtl* ctl;
    Bank bank;        // fission bank written this batch
    Bank src;         // source sites of this batch (eigenvalue batches after the first)
    int use_src;
};

// Weight-window split copies (p.nsplit each) pushed onto the output step
// stack (warp-collective).
__device__ __forceinline__ void push_copies(const SoA* outs, unsigned long long* out_count, bool live, Particle& p,
                                            const RunParams& R, bool ce, unsigned long long cap, ErrorWord* err)
{
    const unsigned k = live ? p.nsplit : 0u;
    const unsigned kmax = __reduce_max_sync(FULL, k);
    for (unsigned c = 1; c <= kmax; ++c) {
        const bool has = c <= k;
        Particle q;
        if (has) q = split_copy(R, p, c);
        push_to(outs, out_count, Q_STEP, has, q, ce, cap, err, false, true);
    }
    p.nsplit = 0u;
}

// Monolithic ("step") event scheme: one stack pair, R events per pop.  WW:
// weight-window problems (weighted scores, closeout, split copies pushed
// onto the output stack).
template <bool CE, bool WW = false>
__global__ void __launch_bounds__(256) k_stack_mono(DevProblem P, const RunParams* Rd, StackArgs A, Tallies T,
                                                   ErrorWord* err)
{
    const int lane = threadIdx.x & 31;
    StackCtl* ctl = A.ctl;
    if (ctl->done) return;   // the loop ended after the previous round
    const RunParams R = *Rd;
    const unsigned long long in_count = ctl->in_count[Q_STEP];
    const unsigned long long cap = ctl->capacity;
    __shared__ long long fx[256 * ACC_FX_WORDS];
    Acc acc;
    acc.zero();
    acc_attach(acc, fx);
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&ctl->pop, 32ull);
        base = __shfl_sync(FULL, base, 0);
        Particle p;
        bool live = false;
        if (base < in_count) {
            const unsigned long long i = base + lane;
            if (i < in_count) {
                load_particle(A.in[Q_STEP], i, p, CE, false, WW);
                live = true;
            }
            __syncwarp();
            for (int r = 0; r < R.remap_every; ++r) {
                const unsigned em = __ballot_sync(FULL, live);   // every lane of the warp is here
                if (!em) break;
                if (live) live = mono_event<CE, WW>(P, R, p, T, acc, A.bank, err, em);
                __syncwarp();
                if (WW) push_copies(A.out, ctl->out_count, live, p, R, CE, cap, err);
            }
        } else {
            // make_work: the input stack is fully claimed; create sources
            // while the output stack keeps room for every input survivor
            unsigned long long first = ~0ull;
            if (lane == 0 && *(volatile unsigned long long*)&ctl->src_cursor < R.n_hist) {
                const unsigned long long r = atomicAdd(&ctl->reserve[Q_STEP], 32ull);
                if (r + 32ull <= cap) first = atomicAdd(&ctl->src_cursor, 32ull);
            }
            first = __shfl_sync(FULL, first, 0);
            if (first >= R.n_hist) break;
            const unsigned long long id = first + lane;
            __syncwarp();
            if (id < R.n_hist) {
                live = source_particle<CE>(P, R, (unsigned)id, p, A.use_src ? &A.src : nullptr, id);
                if (!live) atomicCAS(&err->code, 0, ERR_INVALID);
                acc.ev[EV_SOURCE] += 1u;
            }
        }
        push_to(A.out, ctl->out_count, Q_STEP, live, p, CE, cap, err, false, WW);
    }
    flush_acc(acc, T);
}

// Decomposed schemes: the event stacks (step / collision / surface, and with
// DEC_LOOKUP the lookup) processed in one launch; each warp's 32 virtual
// indices fall in one stack (ranges padded to 32), so a warp runs one event
// type.  With DEC_LOOKUP every collision and surface crossing is followed by a
// lookup, so each output stack receives at most one input stack's particles
// (plus reserved sources) and cannot overflow.
template <bool CE, int DEC>
__global__ void __launch_bounds__(256) k_stack_split(DevProblem P, const RunParams* Rd, StackArgs A, Tallies T,
                                                    ErrorWord* err)
{
    if (A.ctl->done) return;   // the loop ended after the previous round
    const RunParams R = *Rd;
    constexpr int nq = dec_queues(DEC);
    constexpr bool XS = DEC == DEC_LOOKUP;
    constexpr int FIRST = XS ? Q_LOOKUP : Q_STEP;   // where sources start
    const int lane = threadIdx.x & 31;
    StackCtl* ctl = A.ctl;
    unsigned long long cnt[nq], start[nq + 1];
    start[0] = 0;
#pragma unroll
    for (int q = 0; q < nq; ++q) {
        cnt[q] = ctl->in_count[q];
        start[q + 1] = start[q] + ((cnt[q] + 31ull) & ~31ull);
    }
    const unsigned long long cap = ctl->capacity;
    __shared__ long long fx[256 * ACC_FX_WORDS];
    Acc acc;
    acc.zero();
    acc_attach(acc, fx);
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&ctl->pop, 32ull);
        base = __shfl_sync(FULL, base, 0);
        Particle p;
        bool live = false;
        int dst = XS ? Q_LOOKUP : Q_STEP;
        if (base < start[nq]) {
            int q = 0;
#pragma unroll
            for (int k = 1; k < nq; ++k)
                if (base >= start[k]) q = k;
            const unsigned long long i = base - start[q] + lane;
            if (i < cnt[q]) load_particle(A.in[q], i, p, CE, XS);
            __syncwarp();
            const unsigned em = __ballot_sync(FULL, i < cnt[q]);   // the lanes that hold a particle
            if (i < cnt[q]) {
                live = true;
                if (q == Q_STEP) {
                    tr::XS X;
                    double xr;
                    FwdSink sink{T, acc};
                    step_event<CE, XS>(P, R, p, sink, X, xr);
                    dst = next_queue_after_step(p);
                } else if (q == Q_COLLIDE) {
                    live = split_collide<CE, XS>(P, R, p, T, acc, A.bank, err, em);
                } else if (XS && q == Q_LOOKUP) {
                    lookup_event<CE>(P, p);
                    dst = Q_STEP;
                } else {
                    live = split_surface(P, R, p, T, acc, A.bank);
                }
            }
        } else {
            unsigned long long first = ~0ull;
            if (lane == 0 && *(volatile unsigned long long*)&ctl->src_cursor < R.n_hist) {
                const unsigned long long r = atomicAdd(&ctl->reserve[FIRST], 32ull);
                if (r + 32ull <= cap) first = atomicAdd(&ctl->src_cursor, 32ull);
            }
            first = __shfl_sync(FULL, first, 0);
            if (first >= R.n_hist) break;
            const unsigned long long id = first + lane;
            __syncwarp();
            if (id < R.n_hist) {
                live = source_particle<CE>(P, R, (unsigned)id, p, A.use_src ? &A.src : nullptr, id);
                if (!live) atomicCAS(&err->code, 0, ERR_INVALID);
                acc.ev[EV_SOURCE] += 1u;
            }
        }
        push_to(A.out, ctl->out_count, dst, live, p, CE, cap, err, XS);
    }
    flush_acc(acc, T);
}

// The step between two stack rounds (one thread): the host loop's
// bookkeeping done on the device, so that the rounds run as a graph loop
// with no host round trip.  Sources go where the survivors of the previous
// round's collision and surface stacks go (the launch-threshold rule).
__global__ void k_stack_next(StackCtl* ctl, const RunParams* Rd, ErrorWord* err, cudaGraphConditionalHandle cond)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (ctl->done) {
        cudaGraphSetConditional(cond, 0u);
        return;
    }
    ctl->rounds += 1;
    unsigned long long tot = 0;
    bool over = false;
    for (int q = 0; q < N_QUEUES; ++q) {
        const unsigned long long c = ctl->out_count[q];
        over = over || c > ctl->capacity;
        ctl->in_count[q] = c;
        tot += c;
        ctl->out_count[q] = 0;
        ctl->reserve[q] = 0;
    }
    if (over) atomicCAS(&err->code, 0, ERR_CAPACITY);
    ctl->pop = 0;
    if (ctl->dec == DEC_MONO) ctl->reserve[Q_STEP] = ctl->in_count[Q_STEP];
    else ctl->reserve[ctl->dec == DEC_LOOKUP ? Q_LOOKUP : Q_STEP] = ctl->in_count[Q_COLLIDE] + ctl->in_count[Q_SURFACE];
    bool finished = (tot == 0 && ctl->src_cursor >= Rd->n_hist) || over || *(volatile int*)&err->code != 0;
    if (!finished && ctl->rounds >= ctl->max_rounds) {
        atomicCAS(&err->code, 0, ERR_TIMEOUT);
        finished = true;
    }
    if (finished) ctl->done = 1;
    __threadfence();
    cudaGraphSetConditional(cond, finished ? 0u : 1u);
}

// ---------------------------------------------------------------------------
// Scan: exclusive prefix sum of n 32-bit counts into 64-bit offsets, total in
// out[n].  Three phases: tile sums, scan of tile sums, tile scans.
// ---------------------------------------------------------------------------
constexpr int SCAN_TILE = 2048;

__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long v, unsigned long long* sh,
                                                              unsigned long long& total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned long long s = lane < nw ? sh[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(FULL, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) sh[lane] = s;
    }
    __syncthreads();
    total = sh[nw - 1];
    const unsigned long long res = x - v + (wid > 0 ? sh[wid - 1] : 0ull);
    __syncthreads();
    return res;
}

__global__ void __launch_bounds__(1024) k_scan_tiles(const unsigned* __restrict__ in, unsigned long long n,
                                                     unsigned long long* __restrict__ tile_sum)
{
    __shared__ unsigned long long sh[32];
    const unsigned long long b = (unsigned long long)blockIdx.x * SCAN_TILE;
    unsigned long long s = 0;
    for (unsigned long long i = b + threadIdx.x; i < b + SCAN_TILE && i < n; i += blockDim.x) s += in[i];
    unsigned long long tot;
    block_excl_scan(s, sh, tot);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_sums(unsigned long long* __restrict__ tile_sum, unsigned long long nt,
                                                    unsigned long long* __restrict__ total_out)
{
    __shared__ unsigned long long sh[32];
    unsigned long long carry = 0;
    for (unsigned long long c = 0; c < nt; c += blockDim.x) {
        const unsigned long long i = c + threadIdx.x;
        const unsigned long long v = i < nt ? tile_sum[i] : 0ull;
        unsigned long long tot;
        const unsigned long long e = block_excl_scan(v, sh, tot);
        if (i < nt) tile_sum[i] = carry + e;
        carry += tot;
    }
    if (threadIdx.x == 0) *total_out = carry;
}

__global__ void __launch_bounds__(1024) k_scan_apply(const unsigned* __restrict__ in, unsigned long long n,
                                                     const unsigned long long* __restrict__ tile_sum,
                                                     unsigned long long* __restrict__ out)
{
    __shared__ unsigned long long sh[32];
    const unsigned long long b = (unsigned long long)blockIdx.x * SCAN_TILE;
    constexpr int PER = SCAN_TILE / 1024;
    unsigned long long loc[PER];
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const unsigned long long i = b + (unsigned long long)threadIdx.x * PER + k;
        loc[k] = i < n ? in[i] : 0u;
        s += loc[k];
    }
    unsigned long long tot;
    unsigned long long e = block_excl_scan(s, sh, tot) + tile_sum[blockIdx.x];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const unsigned long long i = b + (unsigned long long)threadIdx.x * PER + k;
        if (i < n) out[i] = e;
        e += loc[k];
    }
}

// ---------------------------------------------------------------------------
// Power-iteration kernels
// ---------------------------------------------------------------------------
// Order the bank by (parent history, site sequence): destination =
// offset[parent] + sequence, offsets from the scan of per-parent counts.
__global__ void k_bank_order(Bank in, unsigned long long m, const unsigned long long* __restrict__ offset, Bank out,
                             ErrorWord* err)
{
    for (unsigned long long s = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; s < m;
         s += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long key = in.key[s];
        const unsigned long long dst = offset[key >> 32] + (key & 0xFFFFFFFFull);
        if (dst >= m) {
            atomicCAS(&err->code, 0, ERR_INVALID);
            continue;
        }
        out.x[dst] = in.x[s];
        out.y[dst] = in.y[s];
        out.z[dst] = in.z[s];
        out.g[dst] = in.g[s];
        out.cell[dst] = in.cell[s];
        out.key[dst] = key;
    }
}

// Splitting roulette: site s gets floor(r) copies plus one with probability
// r - floor(r); the draw is Philox keyed by (seed, population tag) with counter
// (batch, 0, s).
__global__ void k_pop_copies(unsigned long long m, uint32_t key0, uint32_t key1, uint32_t batch, unsigned fl,
                             double fr, unsigned* __restrict__ copies)
{
    for (unsigned long long s = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; s < m;
         s += (unsigned long long)gridDim.x * blockDim.x) {
        const uint4 r = philox10(batch, 0u, (uint32_t)s, (uint32_t)(s >> 32), key0, key1);
        copies[s] = fl + (u01(r.x, r.y) < fr ? 1u : 0u);
    }
}

// (copies beyond the output's capacity are not written: they raise a
// capacity error, which the host reads with the batch's other status words)
__global__ void k_pop_write(Bank in, unsigned long long m, const unsigned* __restrict__ copies,
                            const unsigned long long* __restrict__ offset, Bank out, unsigned long long cap,
                            ErrorWord* err)
{
    for (unsigned long long s = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; s < m;
         s += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long o = offset[s];
        unsigned c = copies[s];
        if (o + c > cap) {
            atomicCAS(&err->code, 0, ERR_CAPACITY);
            c = o < cap ? (unsigned)(cap - o) : 0u;
        }
        for (unsigned k = 0; k < c; ++k) {
            out.x[o + k] = in.x[s];
            out.y[o + k] = in.y[s];
            out.z[o + k] = in.z[s];
            out.g[o + k] = in.g[s];
            out.cell[o + k] = in.cell[s];
        }
    }
}

// Fixed-order reduction of the per-history scalar scores: block b sums the
// HIST_CHUNK histories [b HIST_CHUNK, (b + 1) HIST_CHUNK) -- thread t the
// elements t, t + 256, ... in turn, then a fixed tree over the threads --
// into partial[3 b + k]; one block then sums the partials the same way and
// writes each total, rounded once to fixed point, to its scalar bin.  The
// order depends on n alone, so the sums are the same for any schedule.
constexpr int HIST_CHUNK = 4096;

__device__ __forceinline__ double block_sum_fixed(double v, double* sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] = sh[threadIdx.x] + sh[threadIdx.x + w];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(256) k_hist_partial(const double* __restrict__ hf, const double* __restrict__ ha,
                                                      const double* __restrict__ hp, unsigned long long n,
                                                      double* __restrict__ partial)
{
    __shared__ double sh[256];
    const unsigned long long b0 = (unsigned long long)blockIdx.x * HIST_CHUNK;
    const double* src[3] = {hf, ha, hp};
    for (int k = 0; k < 3; ++k) {
        double s = 0.0;
        for (unsigned long long i = b0 + threadIdx.x; i < b0 + HIST_CHUNK && i < n; i += blockDim.x) s = s + src[k][i];
        const double t = block_sum_fixed(s, sh);
        if (threadIdx.x == 0) partial[3 * (unsigned long long)blockIdx.x + k] = t;
    }
}

__global__ void __launch_bounds__(256) k_hist_final(const double* __restrict__ partial, unsigned long long nb,
                                                    FixBin* scal, ErrorWord* err)
{
    __shared__ double sh[256];
    for (int k = 0; k < 3; ++k) {
        double s = 0.0;
        for (unsigned long long b = threadIdx.x; b < nb; b += blockDim.x) s = s + partial[3 * b + k];
        const double t = block_sum_fixed(s, sh);
        if (threadIdx.x == 0) {
            unsigned long long lo, hi;
            if (!fix_split(t, lo, hi)) atomicCAS(&err->code, 0, ERR_RANGE);
            scal[k].lo += lo;
            scal[k].hi += hi;
        }
    }
}

// The same for a batched launch: problem p = blockIdx.y reduces its
// histories [0, off[p+1] - off[p]) from its own per-history arrays, chunk
// blockIdx.x of at most `maxch`, into partial[(p maxch + chunk) 3 + k]; then
// one block per problem sums its chunks in order into its scalar bins.
__global__ void __launch_bounds__(256) k_hist_partial_batched(const Tallies* __restrict__ tal,
                                                              const unsigned long long* __restrict__ off, int maxch,
                                                              double* __restrict__ partial)
{
    __shared__ double sh[256];
    const int p = blockIdx.y;
    const unsigned long long n = off[p + 1] - off[p];
    const unsigned long long b0 = (unsigned long long)blockIdx.x * HIST_CHUNK;
    if (b0 >= n && blockIdx.x > 0) return;   // the whole block leaves together
    const Tallies T = tal[p];
    const double* src[3] = {T.hist_f, T.hist_a, T.hist_p};
    for (int k = 0; k < 3; ++k) {
        double s = 0.0;
        for (unsigned long long i = b0 + threadIdx.x; i < b0 + HIST_CHUNK && i < n; i += blockDim.x) s = s + src[k][i];
        const double t = block_sum_fixed(s, sh);
        if (threadIdx.x == 0) partial[((unsigned long long)p * maxch + blockIdx.x) * 3 + k] = t;
    }
}

__global__ void __launch_bounds__(256) k_hist_final_batched(const Tallies* __restrict__ tal,
                                                            const unsigned long long* __restrict__ off, int maxch,
                                                            const double* __restrict__ partial, ErrorWord* err)
{
    __shared__ double sh[256];
    const int p = blockIdx.x;
    const unsigned long long n = off[p + 1] - off[p];
    const unsigned long long nb = n ? (n + HIST_CHUNK - 1) / HIST_CHUNK : 0;
    FixBin* scal = tal[p].scal;
    for (int k = 0; k < 3; ++k) {
        double s = 0.0;
        for (unsigned long long b = threadIdx.x; b < nb; b += blockDim.x)
            s = s + partial[((unsigned long long)p * maxch + b) * 3 + k];
        const double t = block_sum_fixed(s, sh);
        if (threadIdx.x == 0 && nb) {
            unsigned long long lo, hi;
            if (!fix_split(t, lo, hi)) atomicCAS(&err->code, 0, ERR_RANGE);
            scal[k].lo += lo;
            scal[k].hi += hi;
        }
    }
}

// Active-batch statistics: sum and sum of squares of (bin value) / n per bin.
__global__ void k_eig_accumulate(const FixBin* __restrict__ raw, int n, double inv_n, double* __restrict__ sum,
                                 double* __restrict__ sq)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v = fix_value(raw[i]) * inv_n;
        sum[i] += v;
        sq[i] += v * v;
    }
}

__global__ void k_scale(const double* __restrict__ in, int n, double s, double* __restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = in[i] * s;
}

// Bin values (fixed-point sums) times s.
__global__ void k_fix_scale(const FixBin* __restrict__ in, int n, double s, double* __restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = fix_value(in[i]) * s;
}

// Many conversions in one launch: job j writes the values of in[0..n) times s to out.
__global__ void k_scale_jobs(const ScaleJob* __restrict__ jobs, int n_jobs)
{
    for (int j = blockIdx.y; j < n_jobs; j += gridDim.y) {
        const ScaleJob J = jobs[j];
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < J.n; i += gridDim.x * blockDim.x)
            J.out[i] = fix_value(J.in[i]) * J.s;
    }
}

__global__ void k_eig_finish(const double* __restrict__ sum, const double* __restrict__ sq, int n, double na,
                             double* __restrict__ mean, double* __restrict__ sd)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double m = sum[i] / na;
        const double var = (sq[i] / na - m * m) / (na - 1.0);
        mean[i] = m;
        sd[i] = var > 0.0 ? sqrt(var) : 0.0;
    }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
static std::atomic<unsigned long long> g_launches{0};
unsigned long long launch_count() { return g_launches.load(); }
void count_launches(unsigned long long n) { g_launches += n; }

static int grid_for(unsigned long long n, int threads, int max_blocks)
{
    unsigned long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > (unsigned long long)max_blocks) b = max_blocks;
    return (int)b;
}

// The run's parameters and initial control block, written by the device
// from kernel arguments (a copy from pageable host memory would first wait
// for the stream).
__global__ void k_stack_setup(RunParams R, StackCtl h, RunParams* Rd, StackCtl* ctl)
{
    if (threadIdx.x == 0) {
        *Rd = R;
        *ctl = h;
    }
}

cudaError_t launch_stack_setup(const RunParams& R, const StackCtl& h, RunParams* Rd, StackCtl* ctl, cudaStream_t st)
{
    count_launches(1);
    k_stack_setup<<<1, 32, 0, st>>>(R, h, Rd, ctl);
    return cudaGetLastError();
}

cudaError_t launch_stack_next(StackCtl* ctl, const RunParams* Rd, ErrorWord* err, cudaGraphConditionalHandle cond,
                              cudaStream_t st)
{
    count_launches(1);
    k_stack_next<<<1, 32, 0, st>>>(ctl, Rd, err, cond);
    return cudaGetLastError();
}

cudaError_t launch_stack(const DevProblem& P, const RunParams* R, const SoA* in, const SoA* out, StackCtl* ctl,
                         const Tallies& T, const Bank& bank, const Bank* src, ErrorWord* err, int dec, int blocks,
                         cudaStream_t st)
{
    StackArgs A;
    for (int q = 0; q < N_QUEUES; ++q) {
        A.in[q] = in[q];
        A.out[q] = out[q];
    }
    A.ctl = ctl;
    A.bank = bank;
    A.use_src = src != nullptr;
    if (src) A.src = *src;
    else A.src = bank;
    count_launches(1);
    if (dec == DEC_LOOKUP) {
        if (P.kind == 1) k_stack_split<true, DEC_LOOKUP><<<blocks, 256, 0, st>>>(P, R, A, T, err);
        else k_stack_split<false, DEC_LOOKUP><<<blocks, 256, 0, st>>>(P, R, A, T, err);
    } else if (dec == DEC_SPLIT) {
        if (P.kind == 1) k_stack_split<true, DEC_SPLIT><<<blocks, 256, 0, st>>>(P, R, A, T, err);
        else k_stack_split<false, DEC_SPLIT><<<blocks, 256, 0, st>>>(P, R, A, T, err);
    } else if (P.ww_lo) {
        if (P.kind == 1) k_stack_mono<true, true><<<blocks, 256, 0, st>>>(P, R, A, T, err);
        else k_stack_mono<false, true><<<blocks, 256, 0, st>>>(P, R, A, T, err);
    } else {
        if (P.kind == 1) k_stack_mono<true><<<blocks, 256, 0, st>>>(P, R, A, T, err);
        else k_stack_mono<false><<<blocks, 256, 0, st>>>(P, R, A, T, err);
    }
    return cudaGetLastError();
}

cudaError_t launch_scan(const unsigned* in, unsigned long long n, unsigned long long* tile_sum, unsigned long long* out,
                        unsigned long long* total, cudaStream_t st)
{
    const unsigned long long nt = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (n == 0) return cudaMemsetAsync(total, 0, sizeof(unsigned long long), st);
    count_launches(3);
    k_scan_tiles<<<(unsigned)nt, 1024, 0, st>>>(in, n, tile_sum);
    k_scan_sums<<<1, 1024, 0, st>>>(tile_sum, nt, total);
    k_scan_apply<<<(unsigned)nt, 1024, 0, st>>>(in, n, tile_sum, out);
    return cudaGetLastError();
}

cudaError_t launch_bank_order(const Bank& in, unsigned long long m, const unsigned long long* offset, const Bank& out,
                              ErrorWord* err, cudaStream_t st)
{
    if (m == 0) return cudaSuccess;
    count_launches(1);
    k_bank_order<<<grid_for(m, 256, 4096), 256, 0, st>>>(in, m, offset, out, err);
    return cudaGetLastError();
}

cudaError_t launch_pop_copies(unsigned long long m, uint32_t key0, uint32_t key1, uint32_t batch, unsigned fl,
                              double fr, unsigned* copies, cudaStream_t st)
{
    if (m == 0) return cudaSuccess;
    count_launches(1);
    k_pop_copies<<<grid_for(m, 256, 4096), 256, 0, st>>>(m, key0, key1, batch, fl, fr, copies);
    return cudaGetLastError();
}

cudaError_t launch_pop_write(const Bank& in, unsigned long long m, const unsigned* copies,
                             const unsigned long long* offset, const Bank& out, unsigned long long cap, ErrorWord* err,
                             cudaStream_t st)
{
    if (m == 0) return cudaSuccess;
    count_launches(1);
    k_pop_write<<<grid_for(m, 256, 4096), 256, 0, st>>>(in, m, copies, offset, out, cap, err);
    return cudaGetLastError();
}

__global__ void k_gather(Gather g)
{
    for (int k = 0; k < g.n; ++k) {
        const unsigned char* src = static_cast<const unsigned char*>(g.src[k]);
        unsigned char* dst = static_cast<unsigned char*>(g.dst[k]);
        for (unsigned i = threadIdx.x; i < g.bytes[k]; i += blockDim.x) dst[i] = src[i];
    }
}

cudaError_t launch_gather(const Gather& g, cudaStream_t st)
{
    if (g.n <= 0) return cudaSuccess;
    count_launches(1);
    k_gather<<<1, 256, 0, st>>>(g);
    return cudaGetLastError();
}

cudaError_t launch_eig_accumulate(const FixBin* raw, int n, double inv_n, double* sum, double* sq, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    count_launches(1);
    k_eig_accumulate<<<grid_for(n, 256, 1024), 256, 0, st>>>(raw, n, inv_n, sum, sq);
    return cudaGetLastError();
}

cudaError_t launch_scale(const double* in, int n, double s, double* out, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    count_launches(1);
    k_scale<<<grid_for(n, 256, 1024), 256, 0, st>>>(in, n, s, out);
    return cudaGetLastError();
}

cudaError_t launch_hist_reduce(const Tallies& T, unsigned long long n, double* partial, cudaStream_t st)
{
    if (n == 0 || !T.hist_f) return cudaSuccess;
    const unsigned long long nb = (n + HIST_CHUNK - 1) / HIST_CHUNK;
    count_launches(2);
    k_hist_partial<<<(unsigned)nb, 256, 0, st>>>(T.hist_f, T.hist_a, T.hist_p, n, partial);
    k_hist_final<<<1, 256, 0, st>>>(partial, nb, T.scal, T.err);
    return cudaGetLastError();
}

cudaError_t launch_hist_reduce_batched(const Tallies* tal, const unsigned long long* off, int n_probs, int maxch,
                                      double* partial, ErrorWord* err, cudaStream_t st)
{
    if (n_probs <= 0 || maxch <= 0) return cudaSuccess;
    count_launches(2);
    k_hist_partial_batched<<<dim3((unsigned)maxch, (unsigned)n_probs), 256, 0, st>>>(tal, off, maxch, partial);
    k_hist_final_batched<<<(unsigned)n_probs, 256, 0, st>>>(tal, off, maxch, partial, err);
    return cudaGetLastError();
}

cudaError_t launch_fix_scale(const FixBin* in, int n, double s, double* out, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    count_launches(1);
    k_fix_scale<<<grid_for(n, 256, 1024), 256, 0, st>>>(in, n, s, out);
    return cudaGetLastError();
}

cudaError_t launch_scale_jobs(const ScaleJob* jobs, int n_jobs, cudaStream_t st)
{
    if (n_jobs <= 0) return cudaSuccess;
    count_launches(1);
    k_scale_jobs<<<dim3(32, n_jobs < 65535 ? n_jobs : 65535), 256, 0, st>>>(jobs, n_jobs);
    return cudaGetLastError();
}

cudaError_t launch_eig_finish(const double* sum, const double* sq, int n, double na, double* mean, double* sd,
                              cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    count_launches(1);
    k_eig_finish<<<grid_for(n, 256, 1024), 256, 0, st>>>(sum, sq, n, na, mean, sd);
    return cudaGetLastError();
}

}  // namespace tr
