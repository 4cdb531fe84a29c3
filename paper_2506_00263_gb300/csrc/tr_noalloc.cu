// tr_noalloc.cu -- tr_run_fixed_source_noalloc: a fixed-source run of the
// asynchronous scheme that allocates no memory.
//
// Some callers cannot allocate device memory while they run: for example a
// host application that reserves the GPU's memory for its own pool at
// start-up and forbids further allocations, or a latency-sensitive loop that
// cannot accept the implicit device synchronisation of cudaMalloc/cudaFree.
// This entry point serves them.  Its scratch -- the error word, the event
// counters, the scheduler's control block, a small global link arena for
// spilled particles and the tally accumulators (fixed-point sums, converted
// into the caller's arrays at the end) -- lives in the file-scope array below, which every GPU
// that loads the library holds until the process exits.  The caller passes
// the inputs (a problem created earlier) and the outputs (device arrays for
// the tallies).  Nothing here calls cudaMalloc, cudaFree, an event or stream
// creation, or any allocating library routine.
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/tr.h"
#include "tr_kernels.h"

using namespace tr;

namespace tr {
void set_last_error(const char* msg);   // tr_capi.cu: the thread-local message of tr_last_error()
}

namespace {

constexpr unsigned long long NOALLOC_LINKS = TR_NOALLOC_MAX_QUEUE_CAPACITY / 32;
constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
// per particle slot of the link arena: 15 doubles + 7 32-bit words (as carve_links below)
constexpr size_t LINK_SOA_BYTES = 22 * 256 + NOALLOC_LINKS * 32 * (15 * 8 + 7 * 4);
constexpr size_t OFF_ERR = 0;
constexpr size_t OFF_COUNTS = align256(OFF_ERR + sizeof(ErrorWord));
constexpr size_t OFF_CTL = align256(OFF_COUNTS + 16 * sizeof(unsigned long long));
constexpr size_t OFF_NEXT = align256(OFF_CTL + sizeof(AsyncCtl));
constexpr size_t OFF_TYPE = align256(OFF_NEXT + NOALLOC_LINKS * 4);
constexpr size_t OFF_FILL = align256(OFF_TYPE + NOALLOC_LINKS * 4);
constexpr size_t OFF_LINKS = align256(OFF_FILL + NOALLOC_LINKS * 4);
constexpr size_t OFF_TALLY = align256(OFF_LINKS + LINK_SOA_BYTES);
constexpr size_t SCRATCH_USED = OFF_TALLY + (size_t)TR_NOALLOC_MAX_TALLY_BINS * sizeof(FixBin);
static_assert(SCRATCH_USED <= TR_NOALLOC_SCRATCH_BYTES, "static scratch too small for its layout");

}  // namespace

// The scratch shared by every call on a device (contents persist between calls).
static __device__ __align__(256) unsigned char g_noalloc_scratch[TR_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char* g_addr[MAX_DEVICES] = {};

tr_status fail(tr_status s, const char* m)
{
    tr::set_last_error(m);   // reported by tr_last_error()
    return s;
}

// Device address of the scratch array on `dev`, looked up once per device
// with that device current (the host-side symbol is only a stand-in).
tr_status scratch_address(int dev, unsigned char** out)
{
    if (dev < 0 || dev >= MAX_DEVICES) return fail(TR_ERR_INVALID, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        int prev = -1;
        if (cudaGetDevice(&prev) != cudaSuccess) return fail(TR_ERR_CUDA, "cudaGetDevice failed");
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) return fail(TR_ERR_CUDA, "cudaSetDevice failed");
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (prev != dev) cudaSetDevice(prev);
        if (e != cudaSuccess || !p) return fail(TR_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
        g_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_addr[dev];
    return TR_OK;
}

void carve_links(unsigned char* b, unsigned long long n, SoA& s)
{
    auto take = [&](size_t sz) {
        unsigned char* p = b;
        b += align256(n * sz);
        return p;
    };
    s.x = (double*)take(8); s.y = (double*)take(8); s.z = (double*)take(8);
    s.u = (double*)take(8); s.v = (double*)take(8); s.w = (double*)take(8);
    s.iu = (double*)take(8); s.iv = (double*)take(8); s.iw = (double*)take(8); s.ia = (double*)take(8);
    s.E = (double*)take(8);
    s.t = (double*)take(8);
    s.hf = (double*)take(8); s.ha = (double*)take(8); s.hp = (double*)take(8);
    s.xst = s.xist = s.xsa = s.xnsf = nullptr;   // the lookup-event decomposition is not offered here
    s.wt = nullptr;                              // nor are weight windows
    s.sid = nullptr;
    s.g = (int*)take(4);
    s.cell = (unsigned*)take(4); s.id = (unsigned*)take(4); s.n = (unsigned*)take(4);
    s.nsites = (unsigned*)take(4); s.pend = (unsigned*)take(4); s.prob = (unsigned*)take(4);
}

#define NA_CUDA(call)                                                            \
    do {                                                                         \
        if ((call) != cudaSuccess) return fail(TR_ERR_CUDA, #call " failed");    \
    } while (0)

}  // namespace

// Accessors of the problem needed here (defined in tr_capi.cu).
namespace tr {
const DevProblem* problem_device_data(const tr_problem* pr, int* device, cudaStream_t* stream, int* sms);
}

extern "C" tr_status tr_run_fixed_source_noalloc(tr_problem* problem, const tr_run_opts* o, double* mesh_out,
                                                 double* energy_out, double* scalars_out, tr_run_stats* stats)
{
    if (!problem || !o) return fail(TR_ERR_INVALID, "NULL problem or options");
    if (o->scheme != TR_SCHEME_ASYNC) return fail(TR_ERR_INVALID, "the no-allocation run uses the asynchronous scheme");
    if (o->decomposition != TR_DECOMP_MONO && o->decomposition != TR_DECOMP_SPLIT)
        return fail(TR_ERR_INVALID, "decomposition must be TR_DECOMP_MONO or TR_DECOMP_SPLIT");
    if (o->want_event_log) return fail(TR_ERR_INVALID, "the no-allocation run keeps no event log");
    if (o->n_histories >= (1ull << 32) || o->first_history + o->n_histories > (1ull << 32))
        return fail(TR_ERR_INVALID, "histories must stay below 2^32");
    if (o->queue_capacity > TR_NOALLOC_MAX_QUEUE_CAPACITY)
        return fail(TR_ERR_INVALID, "queue_capacity exceeds the static link arena (TR_NOALLOC_MAX_QUEUE_CAPACITY)");
    if (o->remap_every < 0 || o->blocks_per_sm < 0 || o->stash_slots < 0 || o->max_spin < 0)
        return fail(TR_ERR_INVALID, "negative tuning option");
    if (o->decomposition == TR_DECOMP_SPLIT && o->remap_every > 1)
        return fail(TR_ERR_INVALID, "remap_every > 1 applies to the monolithic scheme only");
    int dev = 0, sms = 0;
    cudaStream_t st = nullptr;
    const DevProblem* Pp = problem_device_data(problem, &dev, &st, &sms);
    const DevProblem& P = *Pp;
    DeviceGuard dg(dev);   // the problem's device, current until return
    if ((P.mesh_size > 0 && !mesh_out) || (P.energy_size > 0 && !energy_out) || !scalars_out)
        return fail(TR_ERR_INVALID, "an output array for a present tally is NULL");
    if (P.timed) return fail(TR_ERR_INVALID, "timed problems have no output here: use tr_run_fixed_source");
    if (P.ww_lo) return fail(TR_ERR_INVALID, "weight windows need tr_run_fixed_source");
    const size_t n_bins = (size_t)P.mesh_size + (size_t)P.energy_size + 3;
    if (n_bins > TR_NOALLOC_MAX_TALLY_BINS)
        return fail(TR_ERR_INVALID, "mesh + energy tally bins + 3 exceed TR_NOALLOC_MAX_TALLY_BINS");
    // default stash: 288 slots for the monolithic scheme (its particles stay in
    // registers; a smaller stash leaves more of the shared L1 array as cache:
    // lattice 2.78e9 events/s at 288 slots, 2.74e9 at 512), 512 otherwise
    int S = o->stash_slots > 0 ? o->stash_slots : (o->decomposition == TR_DECOMP_MONO ? 288 : 512);
    S = (S + 31) & ~31;
    if (S < 32 * 9 || S > 16384) return fail(TR_ERR_INVALID, "stash_slots must be in 288..16384");

    unsigned char* base = nullptr;
    tr_status s = scratch_address(dev, &base);
    if (s != TR_OK) return s;

    ErrorWord* err = reinterpret_cast<ErrorWord*>(base + OFF_ERR);
    unsigned long long* counts = reinterpret_cast<unsigned long long*>(base + OFF_COUNTS);
    AsyncArgs A{};
    A.ctl = reinterpret_cast<AsyncCtl*>(base + OFF_CTL);
    A.link_next = reinterpret_cast<unsigned*>(base + OFF_NEXT);
    A.link_type = reinterpret_cast<int*>(base + OFF_TYPE);
    A.link_fill = reinterpret_cast<int*>(base + OFF_FILL);
    carve_links(base + OFF_LINKS, NOALLOC_LINKS * 32, A.links);
    A.n_links = o->queue_capacity ? (o->queue_capacity + 31) / 32 : NOALLOC_LINKS;
    A.use_src = 0;
    A.dec = o->decomposition;
    A.stash_slots = S;

    RunParams R{};
    R.n_hist = o->n_histories;
    R.key0 = (uint32_t)o->seed;
    R.key1 = (uint32_t)(o->seed >> 32) ^ o->problem_tag;
    R.id_base = (uint32_t)o->first_history;
    R.max_events = o->max_events ? o->max_events : 10000000u;
    R.inv_k = 1.0;
    R.remap_every = o->remap_every > 0 ? o->remap_every : 1;
    R.max_spin = o->max_spin > 0 ? (uint64_t)o->max_spin : (1ull << 24);
    R.max_wait_ns = (uint64_t)(o->max_wait_ms ? o->max_wait_ms : 60000u) * 1000000ull;
    R.spill_threshold = o->spill_threshold ? o->spill_threshold : 64;

    // the array keeps the previous call's contents: clear what must start at zero
    // (the control block's list words start as empty lists, all bits set)
    NA_CUDA(cudaMemsetAsync(err, 0, sizeof(ErrorWord), st));
    NA_CUDA(cudaMemsetAsync(counts, 0, 16 * sizeof(unsigned long long), st));
    NA_CUDA(cudaMemsetAsync(A.ctl, 0, sizeof(AsyncCtl), st));
    NA_CUDA(cudaMemsetAsync(A.ctl->free_q, 0xFF, sizeof(A.ctl->free_q), st));
    NA_CUDA(cudaMemsetAsync(A.ctl->full_q, 0xFF, sizeof(A.ctl->full_q), st));
    FixBin* bins = reinterpret_cast<FixBin*>(base + OFF_TALLY);
    NA_CUDA(cudaMemsetAsync(bins, 0, n_bins * sizeof(FixBin), st));

    Tallies T{};
    T.scal = bins;
    T.mesh = bins + 3;
    T.energy = bins + 3 + P.mesh_size;
    T.ev_type = counts;
    T.fin_type = counts + 8;
    T.err = err;
    if (o->n_histories > 0) {
        // (mesh-walk queues, if the problem needs them, in shared memory: nothing to allocate)
        const int maxb = async_max_blocks_per_sm(P, A.dec, S, false, true);
        if (maxb < 1) return fail(TR_ERR_INVALID, "stash does not fit in shared memory");
        const int bps = o->blocks_per_sm > 0 ? (o->blocks_per_sm < maxb ? o->blocks_per_sm : maxb) : maxb;
        int smem = 0;
        NA_CUDA(launch_async(P, R, A, T, err, sms * bps, st, &smem));
    }
    ErrorWord he{};
    AsyncCtl hc;
    unsigned long long hcnt[16];
    NA_CUDA(cudaMemcpyAsync(&he, err, sizeof(he), cudaMemcpyDeviceToHost, st));
    NA_CUDA(cudaMemcpyAsync(&hc, A.ctl, sizeof(hc), cudaMemcpyDeviceToHost, st));
    NA_CUDA(cudaMemcpyAsync(hcnt, counts, sizeof(hcnt), cudaMemcpyDeviceToHost, st));
    NA_CUDA(cudaStreamSynchronize(st));
    if (he.code == ERR_TIMEOUT) return fail(TR_ERR_TIMEOUT, "a device spin-wait exceeded max_spin or max_wait_ms");
    if (he.code == ERR_CAPACITY) return fail(TR_ERR_CAPACITY, "the static link arena overflowed");
    if (he.code == ERR_RANGE) return fail(TR_ERR_CAPACITY, "a tally contribution exceeded the fixed-point range");
    if (he.code != 0) return fail(TR_ERR_INVALID, "device reported invalid state");
    if (hc.live != 0) return fail(TR_ERR_STATE, "run ended with live particles");
    // tallies: means per source particle, into the caller's arrays
    const double inv = o->n_histories ? 1.0 / (double)o->n_histories : 0.0;
    NA_CUDA(launch_fix_scale(T.mesh, P.mesh_size, inv, mesh_out, st));
    NA_CUDA(launch_fix_scale(T.energy, P.energy_size, inv, energy_out, st));
    NA_CUDA(launch_fix_scale(T.scal, 3, inv, scalars_out, st));
    NA_CUDA(cudaStreamSynchronize(st));
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->histories = o->n_histories;
        for (int i = 0; i < 8; ++i) {
            stats->events_by_type[i] = hcnt[i];
            stats->final_by_type[i] = hcnt[8 + i];
            if (i != EV_SOURCE) stats->events += hcnt[i];
        }
        stats->launches = o->n_histories > 0 ? 1 : 0;
        stats->spills = hc.spills;
        stats->refills = hc.refills;
    }
    return TR_OK;
}
