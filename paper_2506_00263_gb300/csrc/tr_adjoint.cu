// tr_adjoint.cu -- derivatives of the fixed-source tallies with respect to the
// multigroup cross sections (tr_sensitivities).
//
// For L = sum_b g_b T_b (T the tallies per source particle, g the upstream
// gradients) the estimator per history is the score-function (likelihood
// ratio) sum in causal form plus the pathwise terms of the reaction-rate
// tallies.  With F = sum_k f_k the history's weighted score (f_k the weighted
// contribution of segment k) and F_before the part already completed:
//   flight ending in a collision  d/dSt[m][g] += (1/St - len) (F - F_before)
//   flight ending at a surface    d/dSt[m][g] += (-len) (F - F_before)
//   then F_before += f_k
//   scatter g -> h                d/dSs[m][g][h] += (1/Ss) (F - F_before), d/dSt -= (1/St) (F - F_before)
//   absorption                    d/dSt += (1/Sa - 1/St) (F - F_before), d/dSs[m][g][*] -= (1/Sa) (F - F_before)
//   pathwise, per segment         d/dSt += g_abs len, d/dSs[m][g][*] -= g_abs len, d/dnuSf += g_prod len
// Histories are not stored: pass 1 recomputes each history from its Philox
// keys to get F, pass 2 recomputes it again and accumulates the terms.  Both
// passes keep one history per lane (its running F in registers) and refill a
// lane from a global cursor the moment its history ends; collisions wait
// until many lanes have one and then run together; the derivative arrays are
// accumulated per block in shared memory when they fit, with the terms that
// add one value to a whole scattering row d/dSs[m][g][*] summed once per row
// and spread over the row when the block flushes.  The source particles come
// pre-sampled (one buffer serves both passes) when a buffer is given.
#include <algorithm>

#include "tr_events.cuh"
#include "tr_kernels.h"

namespace tr {

// Adjoint tally sink: the upstream-gradient-weighted contribution of the
// segment, plus what the flight score needs.
struct AdjSink {
    static constexpr bool kWW = false;   // derivatives are offered for analog runs
    const double* g_mesh;
    const double* g_scal;
    double f, len;
    int m;
    template <bool CE>
    __device__ __forceinline__ void segment(const DevProblem& P, const Particle& p, double x0, double y0, double z0,
                                            double dist, int mat, const XS& X)
    {
        double s = 0.0;
        if (g_mesh && P.has_mesh && gt0(dist)) {
            const int goff = P.by_group ? p.g * P.mesh_vox : 0;
            MeshWeighted op{g_mesh, 0.0};
            mesh_tally(P, op, p, x0, y0, z0, dist, goff);
            s = op.f;
        }
        if (g_scal)
            s = s + ((__ldg(g_scal) * dist + __ldg(g_scal + 1) * (dist * X.sa)) + __ldg(g_scal + 2) * (dist * X.nsf));
        f = s;
        len = dist;
        m = mat;
    }
    // derivatives are offered for untimed problems only
    __device__ __forceinline__ void time_segment(const DevProblem&, double, double, double) {}
};

struct AdjArgs {
    const double* g_mesh;
    const double* g_scal;
    double* F;              // per-history weighted score (pass 1 out, pass 2 in)
    double* d_sigt;         // [m][g]
    double* d_sigs;         // [m][g][h]
    double* d_nusigf;       // [m][g]
    unsigned long long* cursor;   // next history to start (zeroed before each pass)
    int use_smem;
    SoA pre;                // pre-sampled source particles (use_pre)
    int use_pre;
};

#ifndef TR_ADJ_BLOCKS
#define TR_ADJ_BLOCKS 2   // resident blocks per SM the register allocation targets (and the grid uses)
#endif

template <bool PASS2>
__global__ void __launch_bounds__(256, TR_ADJ_BLOCKS) k_adjoint(DevProblem P, RunParams R, AdjArgs A, ErrorWord* err)
{
    extern __shared__ double sgrad[];
    const int G = P.G, MG = P.n_mat * P.G, MGG = MG * P.G;
    double* gst = A.d_sigt;
    double* gss = A.d_sigs;
    double* gnf = A.d_nusigf;
    double* grow = nullptr;   // shared memory only: one value added to every h of row [m][g]
    if (PASS2 && A.use_smem) {
        for (int i = threadIdx.x; i < 3 * MG + MGG; i += blockDim.x) sgrad[i] = 0.0;
        __syncthreads();
        gst = sgrad;
        gss = sgrad + MG;
        gnf = sgrad + MG + MGG;
        grow = sgrad + 2 * MG + MGG;
    }
    Acc acc;
    acc.zero();
    const Tallies T{};
    const Bank B{};
    constexpr unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    // each lane carries one history at a time and takes the next one from the
    // global cursor as soon as its history ends, so lanes stay busy until the
    // histories run out; one event per lane per pass of the loop
    Particle p;
    bool alive = false, exhausted = false, pend = false;
    double F = 0.0, before = 0.0;
    unsigned long long id = 0;
    for (;;) {
        const unsigned need = __ballot_sync(FULL, !alive);
        if (need && !exhausted) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(A.cursor, (unsigned long long)__popc(need));
            base = __shfl_sync(FULL, base, 0);
            if (base + __popc(need) >= R.n_hist) exhausted = true;   // the same in every lane
            if (!alive) {
                const unsigned long long mine = base + __popc(need & ((1u << lane) - 1u));
                if (mine < R.n_hist) {
                    id = mine;
                    alive = A.use_pre ? load_presampled<false>(A.pre, id, p)
                                      : source_particle<false>(P, R, (unsigned)id, p, nullptr, 0);
                    if (!alive) atomicCAS(&err->code, 0, ERR_INVALID);
                    F = PASS2 ? A.F[id] : 0.0;
                    before = 0.0;
                    pend = false;
                }
            }
        }
        const unsigned am = __ballot_sync(FULL, alive);
        if (!am) {
            if (exhausted) break;
            continue;
        }
        // a step that ends in a collision leaves it pending; collisions run
        // together once 16 lanes hold one (or nothing else can step)
        const unsigned pm = __ballot_sync(FULL, alive && pend);
        const bool coll_pass = (am & ~pm) == 0u || __popc(pm) >= 16;
        if (coll_pass) {
            if (alive && pend) {
                // the step's lookup and reaction draw again, from the same keys
                XS X;
                const int m = material(P, p.cell);
                xs_lookup<false>(P, p, m, X);
                const Stream S = make_stream(R, p.id);
                const uint4 b0 = S.block(p.n, BLK_MAIN);
                const int mg = m * G + p.g;
                const int type = collide_event<false>(P, R, p, X, u01(b0.z, b0.w), B, err, pm);
                if (PASS2) {
                    const double after = F - before;
                    if (type == EV_SCATTER) {
                        const double ss = __ldg(P.sigs + mg * G + p.g);
                        atomicAdd(gss + mg * G + p.g, __drcp_rn(ss) * after);
                        atomicAdd(gst + mg, (-X.inv_st) * after);
                    } else {
                        const double inv_sa = __drcp_rn(__ldg(P.sig_a + mg));
                        atomicAdd(gst + mg, (inv_sa - X.inv_st) * after);
                        if (grow) atomicAdd(grow + mg, (-inv_sa) * after);
                        else for (int h = 0; h < G; ++h) atomicAdd(gss + mg * G + h, (-inv_sa) * after);
                    }
                }
                pend = false;
                alive = finish_event(P, R, p, type, T, acc, B);
                if (!alive && !PASS2) A.F[id] = F;
            }
        } else if (alive && !pend) {
            AdjSink sink{A.g_mesh, A.g_scal, 0.0, 0.0, 0};
            XS X;
            double xr;
            const int g0 = p.g;
            step_event<false>(P, R, p, sink, X, xr);
            const bool coll = p.pend == PEND_COLLIDE;
            if (p.pend == PEND_ESCAPE) {
                alive = finish_event(P, R, p, surface_event(P, p), T, acc, B);
            } else {
                const int mg = sink.m * G + g0;
                if (!PASS2) {
                    F += sink.f;
                } else {
                    const double sf = coll ? X.inv_st - sink.len : -sink.len;
                    atomicAdd(gst + mg, sf * (F - before));
                    if (A.g_scal) {
                        const double ga = __ldg(A.g_scal + 1) * sink.len;
                        atomicAdd(gst + mg, ga);
                        if (grow) atomicAdd(grow + mg, -ga);
                        else for (int h = 0; h < G; ++h) atomicAdd(gss + mg * G + h, -ga);
                        atomicAdd(gnf + mg, __ldg(A.g_scal + 2) * sink.len);
                    }
                    before = before + sink.f;
                }
                if (coll) pend = true;
                else alive = finish_event(P, R, p, surface_event(P, p), T, acc, B);
            }
            if (!alive && !PASS2) A.F[id] = F;
        }
    }
    if (PASS2 && A.use_smem) {
        __syncthreads();
        for (int i = threadIdx.x; i < MG; i += blockDim.x) {
            if (sgrad[i] != 0.0) atomicAdd(A.d_sigt + i, sgrad[i]);
            if (sgrad[MG + MGG + i] != 0.0) atomicAdd(A.d_nusigf + i, sgrad[MG + MGG + i]);
        }
        for (int i = threadIdx.x; i < MGG; i += blockDim.x) {
            const double v = sgrad[MG + i] + grow[i / G];
            if (v != 0.0) atomicAdd(A.d_sigs + i, v);
        }
    }
}

cudaError_t launch_adjoint(const DevProblem& P, const RunParams& R, const double* g_mesh, const double* g_scal,
                           double* F, double* d_sigt, double* d_sigs, double* d_nusigf, ErrorWord* err, int sms,
                           unsigned long long* cursors, const SoA* pre, cudaStream_t st)
{
    cudaError_t e0 = cudaMemsetAsync(cursors, 0, 2 * sizeof(unsigned long long), st);
    if (e0 != cudaSuccess) return e0;
    AdjArgs A;
    A.g_mesh = g_mesh;
    A.g_scal = g_scal;
    A.F = F;
    A.d_sigt = d_sigt;
    A.d_sigs = d_sigs;
    A.d_nusigf = d_nusigf;
    A.use_pre = pre != nullptr;
    if (pre) A.pre = *pre;
    const size_t n = (size_t)P.n_mat * P.G * (P.G + 3);
    const size_t smem = n * sizeof(double);
    A.use_smem = smem <= 96 * 1024 ? 1 : 0;
    if (A.use_smem) {
        const cudaError_t e = cudaFuncSetAttribute(k_adjoint<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int blocks = sms * TR_ADJ_BLOCKS;
    count_launches(2);
    A.cursor = cursors;
    k_adjoint<false><<<blocks, 256, 0, st>>>(P, R, A, err);
    A.cursor = cursors + 1;
    k_adjoint<true><<<blocks, 256, A.use_smem ? smem : 0, st>>>(P, R, A, err);
    return cudaGetLastError();
}

}  // namespace tr
