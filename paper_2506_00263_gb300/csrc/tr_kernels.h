// tr_kernels.h -- host-callable launchers of the device kernels.
#pragma once
#include "tr_device.cuh"

namespace tr {

// Makes a device current for the duration of an entry point and restores the
// caller's current device on every return path.
struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) changed = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (changed) cudaSetDevice(prev);
    }
    DeviceGuard(const DeviceGuard&) = delete;
    DeviceGuard& operator=(const DeviceGuard&) = delete;
};

// Number of kernels launched through the launchers below (process-wide).
unsigned long long launch_count();
void count_launches(unsigned long long n);

// Control block of the stack scheme (device memory): one round's counters,
// advanced between rounds on the device by k_stack_next.
struct StackCtl {
    unsigned long long in_count[N_QUEUES];    // particles in each input stack
    unsigned long long out_count[N_QUEUES];   // pushes into each output stack
    unsigned long long reserve[N_QUEUES];     // output-stack reservations (make_work threshold)
    unsigned long long pop;            // virtual pop cursor over the input stacks
    unsigned long long src_cursor;     // next source index (make_work)
    unsigned long long capacity;       // particles per stack
    unsigned long long rounds;         // rounds (stack-kernel launches) completed
    unsigned long long max_rounds;     // a loop still running after this many rounds ends with ERR_TIMEOUT
    int done;                          // the loop has ended: a stack kernel launched now returns at once
    int dec;                           // task decomposition (the reservation rule depends on it)
};

// Control block of the asynchronous scheme (device memory).
struct AsyncCtl {
    unsigned long long src_cursor;     // next source index (make_work)
    unsigned long long live;           // particles created and not yet ended
    unsigned long long spills, refills;
    unsigned long long free_q[32];     // lock-free queues of empty global links: head | tail << 32
    unsigned long long full_q[32];     // lock-free queues of filled global links
    unsigned long long links_made;     // links taken from the arena's never-used tail
    unsigned hungry;                   // warps currently starving for work
};

// One stack round from the buffer set `in` to `out`; the run parameters are
// read from device memory (Rd), so that a captured launch serves every batch.
cudaError_t launch_stack(const DevProblem& P, const RunParams* Rd, const SoA* in, const SoA* out, StackCtl* ctl,
                         const Tallies& T, const Bank& bank, const Bank* src, ErrorWord* err, int dec, int blocks,
                         cudaStream_t st);
// Between two rounds: check the output stacks' counts against the capacity,
// make them the next round's inputs, reset the round's cursors and
// reservations, and decide whether another round runs (sources left or
// particles in flight, no error, fewer than max_rounds rounds); the decision
// goes to the graph's loop condition.
cudaError_t launch_stack_next(StackCtl* ctl, const RunParams* Rd, ErrorWord* err, cudaGraphConditionalHandle cond,
                              cudaStream_t st);
// Write the run parameters and the initial control block to device memory
// from kernel arguments, in stream order.
cudaError_t launch_stack_setup(const RunParams& R, const StackCtl& h, RunParams* Rd, StackCtl* ctl, cudaStream_t st);

struct WalkQ;   // a warp's deferred mesh walks (tr_events.cuh)

struct AsyncArgs {
    SoA links;                         // global link arena: n_links * 32 particle slots
    unsigned* link_next;               // per link: next link in its list
    int* link_type;                    // per link: event type of its particles
    int* link_fill;                    // per link: number of particles
    unsigned long long n_links;
    AsyncCtl* ctl;
    Bank bank, src;
    int use_src;
    SoA pre;                           // source particles sampled before the launch (x..ia, E or g, cell, id)
    int use_pre;                       // 1: make_work loads its particles from pre instead of sampling them
    int dec;                           // task decomposition: DEC_MONO, DEC_SPLIT, DEC_LOOKUP
    int stash_slots;
    // batched launches: per-problem descriptors, tallies and history offsets
    const DevProblem* probs;
    const Tallies* tallies;
    const unsigned long long* hist_off;   // n_probs + 1 cumulative history counts
    int n_probs;
    // monolithic scheme, problems whose mesh tally needs walks: one queue per
    // warp of the grid in global memory (walk_queue_bytes), or NULL: the
    // queues take shared memory (async_max_blocks_per_sm with walk_smem)
    WalkQ* walkq;
};

cudaError_t launch_async(const DevProblem& P, const RunParams& R, const AsyncArgs& A, const Tallies& T, ErrorWord* err,
                         int blocks, cudaStream_t st, int* smem_bytes_out);
int async_max_blocks_per_sm(const DevProblem& P, int dec, int stash_slots, bool pre = false, bool walk_smem = false);
size_t walk_queue_bytes(int blocks);   // AsyncArgs::walkq of a launch of this many blocks
// Samples the source particles of histories [0, R.n_hist) into A.pre.
cudaError_t launch_presample(const DevProblem& P, const RunParams& R, const AsyncArgs& A, int blocks, cudaStream_t st);
cudaError_t launch_async_batched(const DevProblem& P0, const RunParams& R, const AsyncArgs& A, ErrorWord* err,
                                 int blocks, cudaStream_t st);
int async_batched_max_blocks_per_sm(int dec, int stash_slots);
struct ScaleJob {
    const FixBin* in;
    double* out;
    int n;
    double s;
};
cudaError_t launch_scale_jobs(const ScaleJob* jobs, int n_jobs, cudaStream_t st);

cudaError_t launch_adjoint(const DevProblem& P, const RunParams& R, const double* g_mesh, const double* g_scal,
                           double* F, double* d_sigt, double* d_sigs, double* d_nusigf, ErrorWord* err, int sms,
                           unsigned long long* cursors, const SoA* pre, cudaStream_t st);
cudaError_t launch_scan(const unsigned* in, unsigned long long n, unsigned long long* tile_sum, unsigned long long* out,
                        unsigned long long* total, cudaStream_t st);
cudaError_t launch_bank_order(const Bank& in, unsigned long long m, const unsigned long long* offset, const Bank& out,
                              ErrorWord* err, cudaStream_t st);
cudaError_t launch_pop_copies(unsigned long long m, uint32_t key0, uint32_t key1, uint32_t batch, unsigned fl,
                              double fr, unsigned* copies, cudaStream_t st);
cudaError_t launch_pop_write(const Bank& in, unsigned long long m, const unsigned* copies,
                             const unsigned long long* offset, const Bank& out, unsigned long long cap, ErrorWord* err,
                             cudaStream_t st);
// Up to 8 small device-to-device copies in one single-block launch, so that
// the host reads a batch's status words (gathered in one buffer) with one
// copy: one host round trip instead of one per word.
struct Gather {
    const void* src[8];
    void* dst[8];
    unsigned bytes[8];
    int n;
};
cudaError_t launch_gather(const Gather& g, cudaStream_t st);
cudaError_t launch_eig_accumulate(const FixBin* raw, int n, double inv_n, double* sum, double* sq, cudaStream_t st);
cudaError_t launch_scale(const double* in, int n, double s, double* out, cudaStream_t st);
// The per-history scalar scores of histories [0, n) (T.hist_*) summed in a
// fixed order and added to T.scal; partial: 3 ceil(n / 4096) doubles of scratch.
cudaError_t launch_hist_reduce(const Tallies& T, unsigned long long n, double* partial, cudaStream_t st);
inline unsigned long long hist_partials(unsigned long long n) { return 3 * ((n + 4095) / 4096) + 3; }
// Batched launches: problem p's histories [0, off[p+1] - off[p]) reduced from
// tal[p].hist_* into tal[p].scal; maxch = the most 4096-history chunks of
// any problem; partial: 3 n_probs maxch doubles of scratch.
cudaError_t launch_hist_reduce_batched(const Tallies* tal, const unsigned long long* off, int n_probs, int maxch,
                                      double* partial, ErrorWord* err, cudaStream_t st);
inline int hist_chunks(unsigned long long n) { return (int)((n + 4095) / 4096); }
// out[i] = (value of fixed-point bin in[i]) * s
cudaError_t launch_fix_scale(const FixBin* in, int n, double s, double* out, cudaStream_t st);
cudaError_t launch_eig_finish(const double* sum, const double* sq, int n, double na, double* mean, double* sd,
                              cudaStream_t st);

}  // namespace tr
