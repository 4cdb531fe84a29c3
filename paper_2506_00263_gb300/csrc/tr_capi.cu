// tr_capi.cu -- the C ABI (include/tr.h): problem creation, run drivers for
// the stack-based and asynchronous schemes, power iteration, tally readout.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <chrono>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/tr.h"
#include "tr_kernels.h"

#ifndef TR_HASH_MANT
#define TR_HASH_MANT 10  // union-grid hash: leading mantissa bits of E per bucket
#endif

using namespace tr;

static thread_local std::string g_err;

static tr_status set_err(tr_status s, const std::string& msg)
{
    g_err = msg;
    return s;
}

#define TR_CUDA(call)                                                                              \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return set_err(TR_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));       \
    } while (0)

struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct tr_problem {
    tr_device_ctx ctx{};
    cudaStream_t stream = nullptr;
    int sms = 0;
    DevProblem dp{};
    std::vector<void*> owned;                 // problem data, freed at destroy
    std::map<std::string, Buf> ws;            // run workspaces, grown on demand
    // tallies: raw accumulators, results, eigenvalue statistics
    FixBin *raw_mesh = nullptr, *raw_energy = nullptr, *raw_scal = nullptr, *raw_time = nullptr;   // fixed-point sums
    double *res_mesh = nullptr, *res_energy = nullptr, *res_scal = nullptr, *res_time = nullptr;
    double *sd_mesh = nullptr, *sd_energy = nullptr, *sd_scal = nullptr;
    double *sum_all = nullptr, *sq_all = nullptr;   // mesh | energy | scalars concatenated
    unsigned long long* counts = nullptr;     // ev_type[8], fin_type[8]
    ErrorWord* err = nullptr;
    uint32_t* log_n = nullptr;
    int32_t* log_cell = nullptr;
    uint8_t* log_type = nullptr;
    size_t log_cap = 0, log_count = 0;
    bool have_run = false;
    bool have_std = false;
    bool have_fixed = false;                  // last completed run was fixed source (for sensitivities)
    tr_run_opts last_fixed{};
    // batched launches led by this problem: the captured CUDA graph and its key
    std::vector<unsigned char> ckpt;          // state of a power iteration stopped early (tr_eig_checkpoint)
    uint64_t fingerprint = 0;                 // hash of the geometry, cross sections, source and tally descriptions
    uint64_t xs_generation = 0;               // cross-section updates (tr_problem_set_xs) so far
    unsigned long long hist_cap = 0;          // stride of the per-history score arrays (histories)
    std::vector<double> hplanes[3];           // host copies of the planes (checkpoint validation)
    std::vector<int> hpin;                    // host copy: 1 where the cell holds a pin
    cudaGraphExec_t batch_graph = nullptr;
    std::map<std::vector<unsigned long long>, cudaGraphExec_t> stack_graphs;   // stack-scheme loops by buffers
    std::map<std::vector<int>, int> async_occupancy;   // resident blocks per SM by (decomposition, stash, pre-sampling)
    std::vector<unsigned long long> batch_key;
    unsigned long long batch_graph_launches = 0;
};

// ---------------------------------------------------------------------------
// memory
// ---------------------------------------------------------------------------
static void* dev_alloc(tr_problem* pr, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    void* p = nullptr;
    if (pr->ctx.alloc) {
        p = pr->ctx.alloc(bytes, pr->ctx.stream, pr->ctx.user);
    } else if (cudaMallocAsync(&p, bytes, pr->stream) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

static void dev_free(tr_problem* pr, void* p)
{
    if (!p) return;
    if (pr->ctx.free) pr->ctx.free(p, pr->ctx.stream, pr->ctx.user);
    else cudaFreeAsync(p, pr->stream);
}

static void* own(tr_problem* pr, size_t bytes)
{
    void* p = dev_alloc(pr, bytes);
    if (p) pr->owned.push_back(p);
    return p;
}

template <class T>
static T* upload(tr_problem* pr, const T* src, size_t n, bool* ok)
{
    T* d = (T*)own(pr, n * sizeof(T));
    if (!d) {
        *ok = false;
        return nullptr;
    }
    if (n && cudaMemcpyAsync(d, src, n * sizeof(T), cudaMemcpyHostToDevice, pr->stream) != cudaSuccess) *ok = false;
    // the host vectors may die right after return: make the copy complete
    if (cudaStreamSynchronize(pr->stream) != cudaSuccess) *ok = false;
    return d;
}

static void* workspace(tr_problem* pr, const char* name, size_t bytes)
{
    Buf& b = pr->ws[name];
    if (b.p && b.bytes >= bytes) return b.p;
    if (b.p) dev_free(pr, b.p);
    b.p = dev_alloc(pr, bytes);
    b.bytes = b.p ? bytes : 0;
    return b.p;
}

// ---------------------------------------------------------------------------
// Logarithm table for tr_log (Tang's table-driven method): for each table
// point c_k = 1 + k/128, the pair {1/c_k, -log(1/c_k)}, the logarithm taken
// from the atanh series: x = 2^e m, m in [sqrt(1/2), sqrt(2)], s = (m-1)/(m+1),
// log m = 2 s sum_{j<10} s^(2j)/(2j+1) (Horner in s^2, one fma a step),
// log x = fma(e, LN2_HI, fma(e, LN2_LO, log m)).
// ---------------------------------------------------------------------------
static double bits_double(uint64_t b)
{
    double d;
    std::memcpy(&d, &b, 8);
    return d;
}

static double log_series(double x)
{
    uint64_t b;
    std::memcpy(&b, &x, 8);
    int e = (int)((b >> 52) & 0x7FF) - 1023;
    double m = bits_double((b & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull);
    if (m > bits_double(0x3FF6A09E667F3BCDull)) {
        m = m * 0.5;
        e += 1;
    }
    const double s = (m - 1.0) / (m + 1.0);
    const double z = s * s;
    double p = 1.0 / 19.0;
    const double c[9] = {1.0 / 17.0, 1.0 / 15.0, 1.0 / 13.0, 1.0 / 11.0, 1.0 / 9.0, 1.0 / 7.0, 1.0 / 5.0, 1.0 / 3.0, 1.0};
    for (double ci : c) p = std::fma(p, z, ci);
    const double r = (s + s) * p;
    const double de = (double)e;
    return std::fma(de, bits_double(0x3FE62E42FEFA4000ull), std::fma(de, bits_double(0xBD48432A1B0E2634ull), r));
}

static std::vector<double> log_table()
{
    std::vector<double> t(2 * LOG_TAB_N);
    for (int k = LOG_KMIN; k <= LOG_KMAX; ++k) {
        const double c = (double)(128 + k) / 128.0;
        const double ic = 1.0 / c;
        t[2 * (k - LOG_KMIN)] = ic;
        t[2 * (k - LOG_KMIN) + 1] = -log_series(ic);
    }
    return t;
}

// Exponential ziggurat table for exp_sample (Marsaglia and Tsang's r and v for
// 256 layers): X_1 = r, f_1 = v/(r+1) (the base area v = (r+1) e^-r), then
// f_i+1 = f_i + v/X_i and X_i+1 = -log f_i+1 with the library's own log, so
// one thread builds it on the device; X_256 = 0, f_256 = 1.  Out: {W_i, C_i}
// pairs (W_0 = v/f_1, C_0 = r; W_i = X_i, C_i = X_i+1), then {f_i, df_i}.
__global__ void k_zig_table(DevProblem P, double* out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double r = 7.69711747013104972;
    const double v = 0.0039496598225815571993;
    double X = r, F = v / (r + 1.0);
    out[0] = v / F;
    out[1] = r;
    out[2 * ZIG_N] = 0.0;
    out[2 * ZIG_N + 1] = 0.0;
    for (int i = 1; i < ZIG_N; ++i) {
        double Xn = 0.0, Fn = 1.0;
        if (i < ZIG_N - 1) {
            Fn = F + v / X;
            Xn = -tr_log(P.log_tab, Fn);
        }
        out[2 * i] = X;
        out[2 * i + 1] = Xn;
        out[2 * ZIG_N + 2 * i] = F;
        out[2 * ZIG_N + 2 * i + 1] = Fn - F;
        X = Xn;
        F = Fn;
    }
}

// Derived multigroup tables from sigma_t and sigma_s, one thread per (m, g),
// with the operations and order problem creation uses on the host: 1/sigma_t,
// the running sum of sigma_s[m][g][h] over h, sigma_a = sigma_t - sum.  A
// non-positive or non-finite sigma_t, or a negative or non-finite sigma_s,
// sets *bad.
__global__ void k_mg_derived(int MG, int G, const double* __restrict__ st, const double* __restrict__ ss,
                             double* inv, double* sa, double* cum, int* bad)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < MG; i += gridDim.x * blockDim.x) {
        const double t = st[i];
        if (!(t > 0.0) || !isfinite(t)) atomicExch(bad, 1);
        inv[i] = 1.0 / t;
        double c = 0.0;
        for (int h = 0; h < G; ++h) {
            const double v = ss[(size_t)i * G + h];
            if (!(v >= 0.0) || !isfinite(v)) atomicExch(bad, 1);
            c = c + v;
            cum[(size_t)i * G + h] = c;
        }
        sa[i] = t - c;
    }
}

// ---------------------------------------------------------------------------
// problem creation
// ---------------------------------------------------------------------------
static bool ascending(const double* p, int n)
{
    for (int i = 0; i < n; ++i)
        if (!(p[i] < p[i + 1])) return false;
    return true;
}

static long long dbl_bits(double d)
{
    long long b;
    std::memcpy(&b, &d, 8);
    return b;
}

// FNV-1a, 64 bits, over a byte range (the problem fingerprint a checkpoint
// must match).
static uint64_t fnv1a(uint64_t h, const void* p, size_t n)
{
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 0x100000001B3ull;
    }
    return h;
}

extern "C" tr_status tr_problem_create(const tr_geometry_desc* G, const tr_xs_desc* X, const tr_source_desc* S,
                                       const tr_tally_desc* Tl, int32_t n_tallies, const tr_device_ctx* ctx,
                                       tr_problem** out)
{
    if (!out) return set_err(TR_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!G || !X || !S || !ctx) return set_err(TR_ERR_INVALID, "NULL description");
    if (n_tallies < 0 || n_tallies > 1 || (n_tallies == 1 && !Tl))
        return set_err(TR_ERR_INVALID, "n_tallies must be 0 or 1");
    if (G->nx < 1 || G->ny < 1 || G->nz < 1 || G->nx > 1023 || G->ny > 1023 || G->nz > 1023)
        return set_err(TR_ERR_INVALID, "grid dimensions must be in 1..1023");
    if (!G->x_planes || !G->y_planes || !G->z_planes || !G->cell_material)
        return set_err(TR_ERR_INVALID, "geometry arrays missing");
    if (!ascending(G->x_planes, G->nx) || !ascending(G->y_planes, G->ny) || !ascending(G->z_planes, G->nz))
        return set_err(TR_ERR_INVALID, "planes must be strictly ascending");
    if (!std::isfinite(G->x_planes[0]) || !std::isfinite(G->x_planes[G->nx]) || !std::isfinite(G->y_planes[0]) ||
        !std::isfinite(G->y_planes[G->ny]))
        return set_err(TR_ERR_INVALID, "x and y extents must be finite");
    for (int f = 0; f < 6; ++f)
        if (G->bc[f] != TR_BC_VACUUM && G->bc[f] != TR_BC_REFLECT) return set_err(TR_ERR_INVALID, "bad boundary code");
    if (X->kind != TR_XS_MG && X->kind != TR_XS_CE) return set_err(TR_ERR_INVALID, "bad cross-section kind");
    const int M = X->n_materials;
    if (M < 1 || M > 256) return set_err(TR_ERR_INVALID, "n_materials must be in 1..256");
    const size_t ncell = (size_t)G->nx * G->ny * G->nz;
    for (size_t c = 0; c < ncell; ++c) {
        if (G->cell_material[c] < 0 || G->cell_material[c] >= M) return set_err(TR_ERR_INVALID, "cell material out of range");
        if (G->pin_material && (G->pin_material[c] >= M)) return set_err(TR_ERR_INVALID, "pin material out of range");
    }
    if (G->pin_material && !(G->pin_radius >= 0.0)) return set_err(TR_ERR_INVALID, "negative pin radius");

    tr_problem* pr = new tr_problem();
    pr->ctx = *ctx;
    pr->stream = (cudaStream_t)ctx->stream;
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
        delete pr;
        cudaGetLastError();
        return set_err(TR_ERR_CUDA, "cudaSetDevice failed");
    }
    cudaDeviceGetAttribute(&pr->sms, cudaDevAttrMultiProcessorCount, ctx->device);
    DevProblem& P = pr->dp;
    bool ok = true;
    auto fail_out = [&](tr_status s, const std::string& m) {
        tr_problem_destroy(pr);
        return set_err(s, m);
    };

    const std::vector<double> lt = log_table();
    P.log_tab = upload(pr, lt.data(), lt.size(), &ok);
    {
        double* zt = (double*)own(pr, 4 * ZIG_N * sizeof(double));
        if (!zt || !P.log_tab) {
            ok = false;
        } else {
            P.zig_tab = zt;
            count_launches(1);
            k_zig_table<<<1, 32, 0, pr->stream>>>(P, zt);
            if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(pr->stream) != cudaSuccess) ok = false;
        }
    }

    // geometry
    P.nx = G->nx; P.ny = G->ny; P.nz = G->nz;
    P.xp = upload(pr, G->x_planes, G->nx + 1, &ok);
    P.yp = upload(pr, G->y_planes, G->ny + 1, &ok);
    P.zp = upload(pr, G->z_planes, G->nz + 1, &ok);
    std::vector<double> xc(G->nx), yc(G->ny);
    for (int i = 0; i < G->nx; ++i) xc[i] = 0.5 * (G->x_planes[i] + G->x_planes[i + 1]);
    for (int j = 0; j < G->ny; ++j) yc[j] = 0.5 * (G->y_planes[j] + G->y_planes[j + 1]);
    P.xc = upload(pr, xc.data(), xc.size(), &ok);
    P.yc = upload(pr, yc.data(), yc.size(), &ok);
    std::vector<int> info(ncell);
    for (size_t c = 0; c < ncell; ++c) {
        const int pm = G->pin_material ? G->pin_material[c] : -1;
        info[c] = G->cell_material[c] | ((pm < 0 ? 0 : pm + 1) << 16);
    }
    P.cellinfo = upload(pr, info.data(), ncell, &ok);
    for (int f = 0; f < 6; ++f) P.bc[f] = G->bc[f];
    P.r2 = G->pin_radius * G->pin_radius;
    pr->hplanes[0].assign(G->x_planes, G->x_planes + G->nx + 1);
    pr->hplanes[1].assign(G->y_planes, G->y_planes + G->ny + 1);
    pr->hplanes[2].assign(G->z_planes, G->z_planes + G->nz + 1);
    pr->hpin.resize(ncell);
    for (size_t c = 0; c < ncell; ++c) pr->hpin[c] = (G->pin_material && G->pin_material[c] >= 0) ? 1 : 0;
    uint64_t fp = 0xCBF29CE484222325ull;
    for (int a = 0; a < 3; ++a) fp = fnv1a(fp, pr->hplanes[a].data(), pr->hplanes[a].size() * 8);
    fp = fnv1a(fp, info.data(), ncell * 4);
    fp = fnv1a(fp, G->bc, sizeof(G->bc));
    fp = fnv1a(fp, &G->pin_radius, 8);
    if (X->kind == TR_XS_MG && X->sigma_t && X->sigma_s && X->nu_sigma_f && X->chi && X->n_groups > 0) {
        const size_t MGn = (size_t)M * X->n_groups;
        fp = fnv1a(fp, X->sigma_t, MGn * 8);
        fp = fnv1a(fp, X->sigma_s, MGn * X->n_groups * 8);
        fp = fnv1a(fp, X->nu_sigma_f, MGn * 8);
        fp = fnv1a(fp, X->chi, MGn * 8);
    }
    fp = fnv1a(fp, &S->kind, sizeof(S->kind));
    fp = fnv1a(fp, S->lo, sizeof(S->lo));
    fp = fnv1a(fp, S->hi, sizeof(S->hi));
    if (S->source_material) fp = fnv1a(fp, S->source_material, (size_t)M);
    pr->fingerprint = fp;

    // cross sections
    P.kind = X->kind;
    P.n_mat = M;
    if (X->kind == TR_XS_MG) {
        const int Gn = X->n_groups;
        if (Gn < 1 || Gn > 128 || !X->sigma_t || !X->sigma_s || !X->nu_sigma_f || !X->chi)
            return fail_out(TR_ERR_INVALID, "multigroup data missing or n_groups out of 1..128");
        P.G = Gn;
        const size_t MG = (size_t)M * Gn;
        std::vector<double> inv(MG), sa(MG), cs(MG * Gn), cc(MG);
        for (int m = 0; m < M; ++m) {
            double c = 0.0;
            for (int g = 0; g < Gn; ++g) {
                c = c + X->chi[m * Gn + g];
                cc[m * Gn + g] = c;
            }
            for (int g = 0; g < Gn; ++g) {
                const double st = X->sigma_t[m * Gn + g];
                if (!(st > 0.0)) return fail_out(TR_ERR_INVALID, "sigma_t must be positive");
                inv[m * Gn + g] = 1.0 / st;
                double s = 0.0;
                for (int h = 0; h < Gn; ++h) {
                    const double v = X->sigma_s[((size_t)m * Gn + g) * Gn + h];
                    if (v < 0.0) return fail_out(TR_ERR_INVALID, "negative sigma_s");
                    s = s + v;
                    cs[((size_t)m * Gn + g) * Gn + h] = s;
                }
                sa[m * Gn + g] = st - s;
            }
        }
        P.sigt = upload(pr, X->sigma_t, MG, &ok);
        P.inv_sigt = upload(pr, inv.data(), MG, &ok);
        P.sig_a = upload(pr, sa.data(), MG, &ok);
        P.nusigf = upload(pr, X->nu_sigma_f, MG, &ok);
        P.cum_s = upload(pr, cs.data(), MG * Gn, &ok);
        P.cum_chi = upload(pr, cc.data(), MG, &ok);
        P.chi = upload(pr, X->chi, MG, &ok);
        P.sigs = upload(pr, X->sigma_s, MG * Gn, &ok);
    } else {
        const int Nn = X->n_nuclides;
        if (Nn < 1 || Nn > 16 || !X->nuc_offset || !X->nuc_energy || !X->nuc_sigma || !X->nuc_awr || !X->density)
            return fail_out(TR_ERR_INVALID, "continuous-energy data missing or n_nuclides out of 1..16");
        P.G = 1;
        P.n_nuc = Nn;
        const long long rows = X->nuc_offset[Nn];
        // per grid row and reaction the slope (s[i+1] - s[i]) / (E[i+1] - E[i])
        std::vector<double> slope(3 * (size_t)rows, 0.0);
        for (int n = 0; n < Nn; ++n) {
            const long long a = X->nuc_offset[n], b = X->nuc_offset[n + 1];
            if (b - a < 2 || !ascending(X->nuc_energy + a, (int)(b - a - 1)))
                return fail_out(TR_ERR_INVALID, "each nuclide grid needs >= 2 ascending points");
            for (long long r = a; r + 1 < b; ++r)
                for (int k = 0; k < 3; ++k)
                    slope[3 * r + k] = (X->nuc_sigma[3 * (r + 1) + k] - X->nuc_sigma[3 * r + k]) /
                                       (X->nuc_energy[r + 1] - X->nuc_energy[r]);
        }
        // union grid: all nuclide energies, sorted and unique; per union point
        // and nuclide the largest nuclide row with E_row <= E_union (clamped
        // to the nuclide's last interval)
        std::vector<double> ue(X->nuc_energy, X->nuc_energy + rows);
        std::sort(ue.begin(), ue.end());
        ue.erase(std::unique(ue.begin(), ue.end()), ue.end());
        const long long U = (long long)ue.size();
        std::vector<int> uptr((size_t)U * Nn);
        for (int n = 0; n < Nn; ++n) {
            const long long a = X->nuc_offset[n], b = X->nuc_offset[n + 1];
            long long i = a;
            for (long long u = 0; u < U; ++u) {
                while (i + 1 < b && X->nuc_energy[i + 1] <= ue[u]) ++i;
                long long r = std::min(i, b - 2);
                uptr[(size_t)u * Nn + n] = (int)r;
            }
        }
        // hash on the bit pattern of E: exponent plus TR_HASH_MANT leading
        // mantissa bits (2^TR_HASH_MANT buckets per octave)
        const int shift = 52 - TR_HASH_MANT;
        const long long base = dbl_bits(ue[0]) >> shift, top = dbl_bits(ue[U - 1]) >> shift;
        const int nh = (int)(top - base + 1);
        std::vector<int> hash(nh + 1);
        long long u = 0;
        for (int b = 0; b <= nh; ++b) {
            while (u < U && (dbl_bits(ue[u]) >> shift) - base < b) ++u;
            hash[b] = (int)u;
        }
        std::vector<double> iap(Nn);
        for (int n = 0; n < Nn; ++n) {
            const double A = X->nuc_awr[n];
            iap[n] = 1.0 / ((A + 1.0) * (A + 1.0));
        }
        P.nuc_e = upload(pr, X->nuc_energy, rows, &ok);
        P.nuc_sig = upload(pr, X->nuc_sigma, rows * 3, &ok);
        P.nuc_slope = upload(pr, slope.data(), 3 * (size_t)rows, &ok);
        P.dens = upload(pr, X->density, (size_t)M * Nn, &ok);
        P.awr = upload(pr, X->nuc_awr, Nn, &ok);
        P.inv_ap1sq = upload(pr, iap.data(), Nn, &ok);
        P.e_cut = X->energy_cutoff;
        P.n_union = (int)U;
        P.ue = upload(pr, ue.data(), U, &ok);
        P.uptr = upload(pr, uptr.data(), uptr.size(), &ok);
        P.n_hash = nh;
        P.hash_shift = shift;
        P.hash_base = base;
        P.hash = upload(pr, hash.data(), hash.size(), &ok);
    }

    // source
    if (S->kind < 0 || S->kind > 2) return fail_out(TR_ERR_INVALID, "bad source kind");
    P.src_kind = S->kind;
    P.src_iso = S->isotropic ? 1 : 0;
    P.src_group = S->group;
    if (X->kind == TR_XS_MG && S->group >= P.G) return fail_out(TR_ERR_INVALID, "source group out of range");
    for (int a = 0; a < 3; ++a) {
        P.src_pt[a] = S->point[a];
        P.src_dir[a] = S->direction[a];
        P.src_lo[a] = S->lo[a];
        P.src_hi[a] = S->hi[a];
    }
    P.src_energy = S->energy;
    std::vector<unsigned char> sm(M, 1);
    if (S->source_material) std::memcpy(sm.data(), S->source_material, M);
    P.src_mat = upload(pr, sm.data(), M, &ok);
    P.n_cdf = 0;
    if (X->kind == TR_XS_CE && S->n_cdf > 1) {
        if (!S->cdf_energy || !S->cdf_prob) return fail_out(TR_ERR_INVALID, "source CDF arrays missing");
        P.n_cdf = S->n_cdf;
        P.cdf_e = upload(pr, S->cdf_energy, S->n_cdf, &ok);
        P.cdf_p = upload(pr, S->cdf_prob, S->n_cdf, &ok);
    }

    // tallies
    P.has_mesh = 0;
    P.mesh_vox = 0;
    P.mesh_size = 0;
    P.energy_size = 0;
    P.n_ebins = 0;
    if (n_tallies == 1 && Tl->has_mesh) {
        P.has_mesh = 1;
        long long nv = 1;
        for (int a = 0; a < 3; ++a) {
            if (Tl->mesh_n[a] < 1 || !(Tl->mesh_hi[a] > Tl->mesh_lo[a])) return fail_out(TR_ERR_INVALID, "bad mesh");
            P.mesh_n[a] = Tl->mesh_n[a];
            P.mesh_lo[a] = Tl->mesh_lo[a];
            P.mesh_hi[a] = Tl->mesh_hi[a];
            P.mesh_w[a] = (Tl->mesh_hi[a] - Tl->mesh_lo[a]) / (double)Tl->mesh_n[a];
            P.mesh_iw[a] = 1.0 / P.mesh_w[a];
            nv *= Tl->mesh_n[a];
        }
        if (nv > (1ll << 26)) return fail_out(TR_ERR_INVALID, "mesh too large");
        P.mesh_vox = (int)nv;
        P.by_group = (Tl->by_group && X->kind == TR_XS_MG) ? 1 : 0;
        P.mesh_size = (int)(nv * (P.by_group ? P.G : 1));
    }
    // per axis: the mesh cell that contains geometry cell i (a segment never
    // leaves its geometry cell, so its whole length goes there), or -1
    {
        std::vector<int> c2v((size_t)P.nx + P.ny + P.nz, -1);
        if (P.has_mesh) {
            const double* pl[3] = {G->x_planes, G->y_planes, G->z_planes};
            const int ng[3] = {G->nx, G->ny, G->nz};
            size_t off = 0;
            for (int a = 0; a < 3; ++a) {
                for (int i = 0; i < ng[a]; ++i) {
                    const double g0 = pl[a][i], g1 = pl[a][i + 1];
                    if (!std::isfinite(g0) || !std::isfinite(g1)) continue;
                    const double mid = 0.5 * (g0 + g1);
                    const double kf = std::floor((mid - P.mesh_lo[a]) * P.mesh_iw[a]);
                    if (kf < 0.0 || kf >= (double)P.mesh_n[a]) continue;
                    const int k = (int)kf;
                    const double m0 = P.mesh_lo[a] + (double)k * P.mesh_w[a];
                    const double m1 = P.mesh_lo[a] + (double)(k + 1) * P.mesh_w[a];
                    const double tol = 1e-12 * std::max(std::max(std::fabs(m0), std::fabs(m1)), P.mesh_w[a]);
                    if (g0 >= m0 - tol && g1 <= m1 + tol) c2v[off + i] = k;
                }
                off += ng[a];
            }
        }
        P.mesh_walk = (P.has_mesh && std::find(c2v.begin(), c2v.end(), -1) != c2v.end()) ? 1 : 0;
        P.walk_smem_off = 0;
        P.cell2vox = upload(pr, c2v.data(), c2v.size(), &ok);
    }
    if (n_tallies == 1 && Tl->n_energy_bins > 0) {
        if (!Tl->energy_edges || !ascending(Tl->energy_edges, Tl->n_energy_bins) || !(Tl->energy_edges[0] >= 0.0))
            return fail_out(TR_ERR_INVALID, "energy edges must be ascending and non-negative");
        P.n_ebins = Tl->n_energy_bins;
        P.e_edges = upload(pr, Tl->energy_edges, Tl->n_energy_bins + 1, &ok);
        P.energy_size = M * Tl->n_energy_bins;
    }
    // time: census and time bins
    P.timed = 0;
    P.n_tbins = 0;
    P.t_cen = 0.0;
    P.tb_w = 0.0;
    P.inv_vel = nullptr;
    P.v_c = 2.99792458e10 * std::sqrt(2.0 / 939.56542052e6);   // v = c sqrt(2 E / m_n c^2), E in eV
    if (n_tallies == 1 && (Tl->t_census != 0.0 || Tl->n_time_bins != 0)) {
        if (!(Tl->t_census > 0.0) || !std::isfinite(Tl->t_census) || Tl->n_time_bins < 0 || Tl->n_time_bins > 4096)
            return fail_out(TR_ERR_INVALID, "t_census must be finite and > 0, n_time_bins in 0..4096");
        if (X->kind == TR_XS_MG) {
            if (!X->inv_velocity) return fail_out(TR_ERR_INVALID, "a timed multigroup problem needs inv_velocity");
            for (int g = 0; g < X->n_groups; ++g)
                if (!(X->inv_velocity[g] > 0.0) || !std::isfinite(X->inv_velocity[g]))
                    return fail_out(TR_ERR_INVALID, "inv_velocity must be finite and > 0");
            P.inv_vel = upload(pr, X->inv_velocity, X->n_groups, &ok);
        }
        P.timed = 1;
        P.t_cen = Tl->t_census;
        P.n_tbins = Tl->n_time_bins;
        P.tb_w = P.n_tbins > 0 ? P.t_cen / (double)P.n_tbins : 0.0;
    }
    // weight windows on the tally mesh (the closeout event)
    P.ww_lo = nullptr;
    if (n_tallies == 1 && Tl->ww_lower) {
        if (!P.has_mesh) return fail_out(TR_ERR_INVALID, "weight windows need the tally mesh");
        if (!(Tl->ww_upper > 1.0) || !(Tl->ww_survival > 0.0) || !(Tl->ww_survival <= Tl->ww_upper) ||
            !std::isfinite(Tl->ww_upper) || Tl->ww_max_split < 2 || Tl->ww_max_split > WW_MAX_SPLIT)
            return fail_out(TR_ERR_INVALID,
                            "weight windows need ww_upper > 1, 0 < ww_survival <= ww_upper, 2 <= ww_max_split <= 64");
        const size_t nw = (size_t)P.mesh_vox * P.G;
        for (size_t i = 0; i < nw; ++i)
            if (!(Tl->ww_lower[i] >= 0.0) || !std::isfinite(Tl->ww_lower[i]))
                return fail_out(TR_ERR_INVALID, "weight-window lower bounds must be finite and non-negative");
        P.ww_lo = upload(pr, Tl->ww_lower, nw, &ok);
        P.ww_up = Tl->ww_upper;
        P.ww_surv = Tl->ww_survival;
        P.ww_max_split = Tl->ww_max_split;
    }
    const size_t ms = std::max(P.mesh_size, 1), es = std::max(P.energy_size, 1);
    pr->raw_mesh = (FixBin*)own(pr, ms * sizeof(FixBin));
    pr->raw_energy = (FixBin*)own(pr, es * sizeof(FixBin));
    pr->raw_scal = (FixBin*)own(pr, 4 * sizeof(FixBin));
    pr->res_mesh = (double*)own(pr, ms * 8);
    pr->res_energy = (double*)own(pr, es * 8);
    pr->res_scal = (double*)own(pr, 4 * 8);
    pr->sd_mesh = (double*)own(pr, ms * 8);
    pr->sd_energy = (double*)own(pr, es * 8);
    pr->sd_scal = (double*)own(pr, 4 * 8);
    pr->raw_time = (FixBin*)own(pr, std::max(P.n_tbins, 1) * sizeof(FixBin));
    pr->res_time = (double*)own(pr, std::max(P.n_tbins, 1) * 8);
    pr->sum_all = (double*)own(pr, (ms + es + 4) * 8);
    pr->sq_all = (double*)own(pr, (ms + es + 4) * 8);
    pr->counts = (unsigned long long*)own(pr, 16 * 8);
    pr->err = (ErrorWord*)own(pr, sizeof(ErrorWord));
    if (!ok || !pr->raw_mesh || !pr->raw_energy || !pr->raw_scal || !pr->res_mesh || !pr->res_energy ||
        !pr->res_scal || !pr->sd_mesh || !pr->sd_energy || !pr->sd_scal || !pr->sum_all || !pr->sq_all ||
        !pr->counts || !pr->err || !pr->raw_time || !pr->res_time)
        return fail_out(TR_ERR_NOMEM, "device allocation or upload failed");
    if (cudaStreamSynchronize(pr->stream) != cudaSuccess) return fail_out(TR_ERR_CUDA, "stream sync failed");
    *out = pr;
    return TR_OK;
}

extern "C" tr_status tr_problem_set_xs(tr_problem* pr, const double* sigma_t, const double* sigma_s,
                                       const double* nu_sigma_f, int32_t on_device)
{
    if (!pr || !sigma_t || !sigma_s || !nu_sigma_f) return set_err(TR_ERR_INVALID, "NULL argument");
    if (pr->dp.kind != TR_XS_MG) return set_err(TR_ERR_INVALID, "tr_problem_set_xs needs multigroup data");
    DeviceGuard dg(pr->ctx.device);
    DevProblem& P = pr->dp;
    const cudaStream_t st = pr->stream;
    const size_t MG = (size_t)P.n_mat * P.G;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    int* bad = (int*)workspace(pr, "set_xs_flag", sizeof(int));
    if (!bad) return set_err(TR_ERR_NOMEM, "workspace allocation failed");
    // new values land in scratch first: a refused update leaves the problem as it was
    double* nst = (double*)workspace(pr, "set_xs_st", MG * 8);
    double* nss = (double*)workspace(pr, "set_xs_ss", MG * P.G * 8);
    double* ninv = (double*)workspace(pr, "set_xs_inv", MG * 8);
    double* nsa = (double*)workspace(pr, "set_xs_sa", MG * 8);
    double* ncum = (double*)workspace(pr, "set_xs_cum", MG * P.G * 8);
    if (!nst || !nss || !ninv || !nsa || !ncum) return set_err(TR_ERR_NOMEM, "workspace allocation failed");
    TR_CUDA(cudaMemcpyAsync(nst, sigma_t, MG * 8, kind, st));
    TR_CUDA(cudaMemcpyAsync(nss, sigma_s, MG * P.G * 8, kind, st));
    TR_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
    count_launches(1);
    k_mg_derived<<<(unsigned)std::min<size_t>((MG + 127) / 128, 1024), 128, 0, st>>>((int)MG, P.G, nst, nss, ninv, nsa,
                                                                                    ncum, bad);
    TR_CUDA(cudaGetLastError());
    int hbad = 0;
    TR_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    TR_CUDA(cudaStreamSynchronize(st));
    if (hbad) return set_err(TR_ERR_INVALID, "sigma_t must be positive and finite, sigma_s non-negative and finite");
    TR_CUDA(cudaMemcpyAsync(const_cast<double*>(P.sigt), nst, MG * 8, cudaMemcpyDeviceToDevice, st));
    TR_CUDA(cudaMemcpyAsync(const_cast<double*>(P.sigs), nss, MG * P.G * 8, cudaMemcpyDeviceToDevice, st));
    TR_CUDA(cudaMemcpyAsync(const_cast<double*>(P.inv_sigt), ninv, MG * 8, cudaMemcpyDeviceToDevice, st));
    TR_CUDA(cudaMemcpyAsync(const_cast<double*>(P.sig_a), nsa, MG * 8, cudaMemcpyDeviceToDevice, st));
    TR_CUDA(cudaMemcpyAsync(const_cast<double*>(P.cum_s), ncum, MG * P.G * 8, cudaMemcpyDeviceToDevice, st));
    TR_CUDA(cudaMemcpyAsync(const_cast<double*>(P.nusigf), nu_sigma_f, MG * 8, kind, st));
    // results and checkpoints of earlier runs no longer describe this problem
    pr->have_run = pr->have_std = pr->have_fixed = false;
    pr->ckpt.clear();
    ++pr->xs_generation;
    pr->fingerprint = fnv1a(pr->fingerprint, &pr->xs_generation, sizeof(pr->xs_generation));
    return TR_OK;
}

extern "C" void tr_problem_destroy(tr_problem* pr)
{
    if (!pr) return;
    DeviceGuard dg(pr->ctx.device);
    cudaStreamSynchronize(pr->stream);
    if (pr->batch_graph) cudaGraphExecDestroy(pr->batch_graph);
    for (auto& kv : pr->stack_graphs) cudaGraphExecDestroy(kv.second);
    for (auto& kv : pr->ws) dev_free(pr, kv.second.p);
    for (void* p : pr->owned) dev_free(pr, p);
    if (pr->log_n) dev_free(pr, pr->log_n);
    if (pr->log_cell) dev_free(pr, pr->log_cell);
    if (pr->log_type) dev_free(pr, pr->log_type);
    cudaStreamSynchronize(pr->stream);
    cudaGetLastError();
    delete pr;
}

// ---------------------------------------------------------------------------
// run helpers
// ---------------------------------------------------------------------------
// Largest history count whose sources are sampled ahead of the asynchronous
// monolithic launch (16.8M: 2.6 GB of particle records); larger runs sample
// inside the launch, with the same results.
constexpr unsigned long long PRESAMPLE_MAX_HIST = 1ull << 24;
// Largest history count whose scalar scores are stored per history and
// reduced in a fixed order after the launch (1.6 GB of scores at 2^26).
constexpr unsigned long long HIST_MAX = 1ull << 26;

static bool carve_soa(tr_problem* pr, const char* name, unsigned long long cap, SoA& s)
{
    const size_t n = (size_t)cap;
    const size_t bytes = n * (20 * 8 + 8 * 4) + 28 * 256;
    unsigned char* b = (unsigned char*)workspace(pr, name, bytes);
    if (!b) return false;
    auto take = [&](size_t sz) {
        unsigned char* p = b;
        b += (n * sz + 255) & ~size_t(255);
        return p;
    };
    s.x = (double*)take(8); s.y = (double*)take(8); s.z = (double*)take(8);
    s.u = (double*)take(8); s.v = (double*)take(8); s.w = (double*)take(8);
    s.iu = (double*)take(8); s.iv = (double*)take(8); s.iw = (double*)take(8); s.ia = (double*)take(8);
    s.E = (double*)take(8);
    s.t = (double*)take(8);
    s.hf = (double*)take(8); s.ha = (double*)take(8); s.hp = (double*)take(8);
    s.xst = (double*)take(8); s.xist = (double*)take(8); s.xsa = (double*)take(8); s.xnsf = (double*)take(8);
    s.wt = (double*)take(8);
    s.g = (int*)take(4);
    s.sid = (unsigned*)take(4);
    s.cell = (unsigned*)take(4); s.id = (unsigned*)take(4); s.n = (unsigned*)take(4);
    s.nsites = (unsigned*)take(4); s.pend = (unsigned*)take(4); s.prob = (unsigned*)take(4);
    return true;
}

static bool carve_bank(tr_problem* pr, const char* name, unsigned long long cap, Bank& B, bool with_key)
{
    const size_t n = (size_t)cap;
    const size_t bytes = n * (3 * 8 + 4 + 4 + 8) + 8 * 256;
    unsigned char* b = (unsigned char*)workspace(pr, name, bytes);
    if (!b) return false;
    auto take = [&](size_t sz) {
        unsigned char* p = b;
        b += (n * sz + 255) & ~size_t(255);
        return p;
    };
    B.x = (double*)take(8); B.y = (double*)take(8); B.z = (double*)take(8);
    B.g = (int*)take(4); B.cell = (unsigned*)take(4);
    B.key = with_key ? (unsigned long long*)take(8) : nullptr;
    B.count = (unsigned long long*)take(8);
    B.capacity = cap;
    B.site_count = nullptr;
    return true;
}

static tr_status decode_err(const ErrorWord& h)
{
    if (h.code == ERR_CAPACITY) return set_err(TR_ERR_CAPACITY, "a queue, link arena or fission bank overflowed");
    if (h.code == ERR_RANGE)
        return set_err(TR_ERR_CAPACITY, "a tally contribution exceeded the fixed-point range (|score| >= 2^39)");
    if (h.code == ERR_TIMEOUT)
        return set_err(TR_ERR_TIMEOUT, "a device spin-wait exceeded max_spin or max_wait_ms (site " + std::to_string(h.where) + ")");
    if (h.code != 0) return set_err(TR_ERR_INVALID, "device reported invalid state (code " + std::to_string(h.code) + ")");
    return TR_OK;
}

static tr_status check_err(tr_problem* pr)
{
    ErrorWord h{};
    TR_CUDA(cudaMemcpyAsync(&h, pr->err, sizeof(h), cudaMemcpyDeviceToHost, pr->stream));
    TR_CUDA(cudaStreamSynchronize(pr->stream));
    return decode_err(h);
}

// Status words read back after a launch, gathered on the device into one
// buffer so that the host reads them with a single copy.
struct Readback {
    AsyncCtl hc;
    StackCtl sc;
    ErrorWord err;
    unsigned long long count[2];
    FixBin scal[3];
};

static tr_status ensure_log(tr_problem* pr, size_t n)
{
    if (pr->log_cap >= n) return TR_OK;
    if (pr->log_n) dev_free(pr, pr->log_n);
    if (pr->log_cell) dev_free(pr, pr->log_cell);
    if (pr->log_type) dev_free(pr, pr->log_type);
    pr->log_n = (uint32_t*)dev_alloc(pr, n * 4);
    pr->log_cell = (int32_t*)dev_alloc(pr, n * 4);
    pr->log_type = (uint8_t*)dev_alloc(pr, n);
    pr->log_cap = (pr->log_n && pr->log_cell && pr->log_type) ? n : 0;
    if (!pr->log_cap) return set_err(TR_ERR_NOMEM, "event log allocation failed");
    return TR_OK;
}

static tr_status validate_opts(const tr_run_opts* o)
{
    if (!o) return set_err(TR_ERR_INVALID, "opts is NULL");
    if (o->scheme != TR_SCHEME_STACK && o->scheme != TR_SCHEME_ASYNC) return set_err(TR_ERR_INVALID, "bad scheme");
    if (o->decomposition < TR_DECOMP_MONO || o->decomposition > TR_DECOMP_STREAM)
        return set_err(TR_ERR_INVALID, "bad decomposition");
    if (o->decomposition == TR_DECOMP_STREAM && o->scheme != TR_SCHEME_ASYNC)
        return set_err(TR_ERR_INVALID, "the streaming decomposition is offered by the asynchronous scheme");
    if (o->n_histories >= (1ull << 32)) return set_err(TR_ERR_INVALID, "n_histories must be < 2^32 per run");
    if (o->first_history + o->n_histories > (1ull << 32))
        return set_err(TR_ERR_INVALID, "first_history + n_histories must not exceed 2^32");
    if (o->remap_every < 0 || o->blocks_per_sm < 0 || o->stash_slots < 0 || o->max_spin < 0)
        return set_err(TR_ERR_INVALID, "negative tuning option");
    if (o->decomposition != TR_DECOMP_MONO && o->decomposition != TR_DECOMP_STREAM && o->remap_every > 1)
        return set_err(TR_ERR_INVALID, "remap_every > 1 applies to the monolithic and streaming schemes only");
    return TR_OK;
}

static Tallies make_tallies(tr_problem* pr, bool log)
{
    Tallies T;
    T.mesh = pr->raw_mesh;
    T.energy = pr->raw_energy;
    T.scal = pr->raw_scal;
    T.time = pr->raw_time;
    T.ev_type = pr->counts;
    T.fin_type = pr->counts + 8;
    T.log_n = log ? pr->log_n : nullptr;
    T.log_cell = log ? pr->log_cell : nullptr;
    T.log_type = log ? pr->log_type : nullptr;
    T.err = pr->err;
    T.hist_f = T.hist_a = T.hist_p = nullptr;
    return T;
}

static tr_status zero_raw(tr_problem* pr)
{
    const DevProblem& P = pr->dp;
    TR_CUDA(cudaMemsetAsync(pr->raw_mesh, 0, std::max(P.mesh_size, 1) * sizeof(FixBin), pr->stream));
    TR_CUDA(cudaMemsetAsync(pr->raw_energy, 0, std::max(P.energy_size, 1) * sizeof(FixBin), pr->stream));
    TR_CUDA(cudaMemsetAsync(pr->raw_scal, 0, 4 * sizeof(FixBin), pr->stream));
    TR_CUDA(cudaMemsetAsync(pr->raw_time, 0, std::max(P.n_tbins, 1) * sizeof(FixBin), pr->stream));
    return TR_OK;
}

struct TransportOut {
    unsigned long long launches = 0, spills = 0, refills = 0;
    double kernel_ms = 0.0;
    // in: a device counter to read with the launch's status (the fission
    // bank's size), or null; out (when `have_readback`): its value and the
    // scalar tallies' raw bins
    const unsigned long long* want_count = nullptr;
    bool have_readback = false;
    unsigned long long count = 0;
    FixBin scal[3] = {};
};

// The status words of a transport launch, gathered on the device and read
// with one copy: the scheme's control block, the error word, the scalar
// bins and, if given, a counter of the caller's (the fission bank's size).
static tr_status read_status(tr_problem* pr, const AsyncCtl* actl, const StackCtl* sctl,
                             const unsigned long long* count, Readback& rb)
{
    Readback* drb = (Readback*)workspace(pr, "readback", sizeof(Readback));
    if (!drb) return set_err(TR_ERR_NOMEM, "readback buffer allocation failed");
    Gather g{};
    auto add = [&g](const void* src, void* dst, size_t bytes) {
        g.src[g.n] = src;
        g.dst[g.n] = dst;
        g.bytes[g.n] = (unsigned)bytes;
        ++g.n;
    };
    if (actl) add(actl, &drb->hc, sizeof(AsyncCtl));
    if (sctl) add(sctl, &drb->sc, sizeof(StackCtl));
    add(pr->err, &drb->err, sizeof(ErrorWord));
    add(pr->raw_scal, drb->scal, 3 * sizeof(FixBin));
    if (count) add(count, &drb->count[0], sizeof(unsigned long long));
    TR_CUDA(launch_gather(g, pr->stream));
    TR_CUDA(cudaMemcpyAsync(&rb, drb, sizeof(rb), cudaMemcpyDeviceToHost, pr->stream));
    TR_CUDA(cudaStreamSynchronize(pr->stream));
    return TR_OK;
}

// Device time of one kernel launch: events recorded around it on the stream.
struct LaunchTimer {
    cudaEvent_t a = nullptr, b = nullptr;
    LaunchTimer()
    {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~LaunchTimer()
    {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
    float elapsed()
    {
        float ms = 0.f;
        cudaEventSynchronize(b);
        cudaEventElapsedTime(&ms, a, b);
        return ms;
    }
};

// One transport pass over n histories (fixed source, or one eigenvalue batch).
static tr_status transport(tr_problem* pr, const tr_run_opts* o, RunParams R, const Bank& bank, const Bank* src,
                           TransportOut& out)
{
    const DevProblem& P = pr->dp;
    const cudaStream_t st = pr->stream;
    const int dec = o->decomposition;   // DEC_MONO, DEC_SPLIT, DEC_LOOKUP (same values as TR_DECOMP_*)
    Tallies T = make_tallies(pr, R.want_log != 0);
    if (R.n_hist == 0) return TR_OK;
    // scalar scores: each ended history stores its sums (by history index),
    // reduced in a fixed order after the launch (runs above HIST_MAX
    // histories round them into per-thread fixed-point sums instead)
    double* hist_partial = nullptr;
    if (R.n_hist <= HIST_MAX) {
        // the arrays' stride only grows (in steps of 2^16 histories), so
        // their addresses, which a captured stack-scheme loop bakes in, stay
        // put from batch to batch
        pr->hist_cap = std::max(pr->hist_cap, (R.n_hist + 65535) & ~65535ull);
        double* h = (double*)workspace(pr, "hist_sums", 3 * pr->hist_cap * sizeof(double));
        hist_partial = (double*)workspace(pr, "hist_partial", hist_partials(pr->hist_cap) * sizeof(double));
        if (!h || !hist_partial) return set_err(TR_ERR_NOMEM, "history score buffer allocation failed");
        T.hist_f = h;
        T.hist_a = h + pr->hist_cap;
        T.hist_p = h + 2 * pr->hist_cap;
    }
    if (o->scheme == TR_SCHEME_STACK) {
        // default: the histories (split copies of weight-window problems: room for 8 per history)
        unsigned long long cap = o->queue_capacity ? o->queue_capacity
                                                   : std::min<unsigned long long>(P.ww_lo ? 8 * R.n_hist + 4096 : R.n_hist,
                                                                                  1ull << 22);
        cap = std::max<unsigned long long>((cap + 31) & ~31ull, 64);
        const int nst = dec_queues(dec);
        SoA bufs[2][N_QUEUES] = {};
        const char* names[2][N_QUEUES] = {{"s0a", "s0b", "s0c", "s0d"}, {"s1a", "s1b", "s1c", "s1d"}};
        for (int h = 0; h < 2; ++h)
            for (int q = 0; q < nst; ++q)
                if (!carve_soa(pr, names[h][q], cap, bufs[h][q])) return set_err(TR_ERR_NOMEM, "stack allocation failed");
        StackCtl* dctl = (StackCtl*)workspace(pr, "stackctl", sizeof(StackCtl));
        RunParams* dR = (RunParams*)workspace(pr, "stack_params", sizeof(RunParams));
        if (!dctl || !dR) return set_err(TR_ERR_NOMEM, "control block allocation failed");
        const int bps = o->blocks_per_sm > 0 ? o->blocks_per_sm : 4;
        const int blocks = pr->sms * bps;
        // the rounds run as a graph loop (a conditional WHILE node): each
        // iteration is two rounds, set 0 -> set 1 and set 1 -> set 0, each
        // followed by k_stack_next, which advances the control block and sets
        // the loop condition; no host round trip between rounds
        std::vector<unsigned long long> key = {(unsigned long long)dec, (unsigned long long)blocks, cap,
                                               (unsigned long long)(uintptr_t)dctl, (unsigned long long)(uintptr_t)dR,
                                               (unsigned long long)(uintptr_t)pr->err, (unsigned long long)(src != nullptr)};
        for (int hh = 0; hh < 2; ++hh)
            for (int q = 0; q < nst; ++q) key.push_back((unsigned long long)(uintptr_t)bufs[hh][q].x);
        for (const void* q : {(const void*)T.mesh, (const void*)T.energy, (const void*)T.scal, (const void*)T.time,
                              (const void*)T.hist_f, (const void*)T.hist_a,
                              (const void*)T.ev_type, (const void*)T.log_n, (const void*)T.log_cell,
                              (const void*)T.log_type, (const void*)bank.x, (const void*)bank.count,
                              (const void*)bank.site_count, (const void*)bank.key, (const void*)(src ? src->x : nullptr),
                              (const void*)(src ? src->cell : nullptr)})
            key.push_back((unsigned long long)(uintptr_t)q);
        key.push_back(bank.capacity);
        key.push_back(src ? src->capacity : 0ull);
        cudaGraphExec_t exec = nullptr;
        auto it = pr->stack_graphs.find(key);
        if (it != pr->stack_graphs.end()) {
            exec = it->second;
        } else {
            if (pr->stack_graphs.size() >= 8) {
                for (auto& kv : pr->stack_graphs) cudaGraphExecDestroy(kv.second);
                pr->stack_graphs.clear();
            }
            cudaGraph_t g = nullptr;
            TR_CUDA(cudaGraphCreate(&g, 0));
            cudaGraphConditionalHandle cond;
            cudaError_t ce = cudaGraphConditionalHandleCreate(&cond, g, 1u, cudaGraphCondAssignDefault);
            cudaGraphNodeParams np = {};
            cudaGraphNode_t node;
            if (ce == cudaSuccess) {
                np.type = cudaGraphNodeTypeConditional;
                np.conditional.handle = cond;
                np.conditional.type = cudaGraphCondTypeWhile;
                np.conditional.size = 1;
                ce = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
            }
            cudaStream_t cs = nullptr;
            if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
            tr_status cap_status = TR_OK;
            if (ce == cudaSuccess) {
                cudaGraph_t body = np.conditional.phGraph_out[0];
                const unsigned long long c0 = launch_count();
                ce = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
                if (ce == cudaSuccess) {
                    cudaError_t le = launch_stack(P, dR, bufs[0], bufs[1], dctl, T, bank, src, pr->err, dec, blocks, cs);
                    if (le == cudaSuccess) le = launch_stack_next(dctl, dR, pr->err, cond, cs);
                    if (le == cudaSuccess)
                        le = launch_stack(P, dR, bufs[1], bufs[0], dctl, T, bank, src, pr->err, dec, blocks, cs);
                    if (le == cudaSuccess) le = launch_stack_next(dctl, dR, pr->err, cond, cs);
                    cudaGraph_t captured = nullptr;
                    ce = cudaStreamEndCapture(cs, &captured);
                    if (le != cudaSuccess) ce = le;
                }
                count_launches(0ull - (launch_count() - c0));   // captured, not launched
                cudaStreamDestroy(cs);
            }
            if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, g, 0);
            cudaGraphDestroy(g);
            if (ce != cudaSuccess) {
                cudaGetLastError();
                cap_status = set_err(TR_ERR_CUDA, std::string("stack-scheme graph: ") + cudaGetErrorString(ce));
                return cap_status;
            }
            pr->stack_graphs[key] = exec;
        }
        StackCtl h{};
        h.capacity = cap;
        h.max_rounds = 4ull * R.max_events + 1000000ull;
        h.dec = dec;
        TR_CUDA(launch_stack_setup(R, h, dR, dctl, st));
        LaunchTimer lt;
        TR_CUDA(cudaEventRecord(lt.a, st));
        TR_CUDA(cudaGraphLaunch(exec, st));
        TR_CUDA(cudaEventRecord(lt.b, st));
        // the fixed-order reduction of the per-history scores, then one read
        // of the status words (after a failed loop the sums are discarded)
        TR_CUDA(launch_hist_reduce(T, R.n_hist, hist_partial, st));
        Readback rb;
        tr_status rs = read_status(pr, nullptr, dctl, out.want_count, rb);
        if (rs != TR_OK) return rs;
        h = rb.sc;
        out.kernel_ms += lt.elapsed();
        const unsigned long long launched = 4ull * ((h.rounds + 1) / 2);   // whole loop iterations
        count_launches(launched);
        out.launches += h.rounds;
        if (rb.err.code == ERR_CAPACITY) return set_err(TR_ERR_CAPACITY, "stack overflow");
        if (rb.err.code == ERR_TIMEOUT) return set_err(TR_ERR_TIMEOUT, "stack loop did not terminate");
        tr_status es = decode_err(rb.err);
        if (es != TR_OK) return es;
        out.have_readback = true;
        out.count = rb.count[0];
        std::memcpy(out.scal, rb.scal, sizeof(out.scal));
        return TR_OK;
    }
    // asynchronous scheme: one persistent launch
    // default stash: 288 slots for the monolithic scheme (its particles stay in
    // registers; a smaller stash leaves more of the shared L1 array as cache:
    // lattice 2.78e9 events/s at 288 slots, 2.74e9 at 512), 512 otherwise
    int S = o->stash_slots > 0 ? o->stash_slots : (o->decomposition == TR_DECOMP_MONO && !P.ww_lo ? 288 : 512);
    S = (S + 31) & ~31;
    if (S < 32 * 9 || S > 16384) return set_err(TR_ERR_INVALID, "stash_slots must be in 288..16384");
    const unsigned long long n_links = o->queue_capacity ? (o->queue_capacity + 31) / 32 : 8192;
    AsyncArgs A{};
    if (!carve_soa(pr, "links", n_links * 32, A.links)) return set_err(TR_ERR_NOMEM, "link arena allocation failed");
    A.link_next = (unsigned*)workspace(pr, "link_next", n_links * 4);
    A.link_type = (int*)workspace(pr, "link_type", n_links * 4);
    A.link_fill = (int*)workspace(pr, "link_fill", n_links * 4);
    A.ctl = (AsyncCtl*)workspace(pr, "asyncctl", sizeof(AsyncCtl));
    if (!A.link_next || !A.link_type || !A.link_fill || !A.ctl) return set_err(TR_ERR_NOMEM, "link arena allocation failed");
    A.n_links = n_links;
    A.bank = bank;
    A.use_src = src != nullptr;
    A.src = src ? *src : bank;
    A.dec = dec;
    A.stash_slots = S;
    // monolithic scheme: sample the sources ahead of the launch (make_work loads them)
    if (dec == DEC_MONO && R.n_hist <= PRESAMPLE_MAX_HIST && !P.ww_lo) {
        if (!carve_soa(pr, "presample", R.n_hist, A.pre)) return set_err(TR_ERR_NOMEM, "source buffer allocation failed");
        A.use_pre = 1;
    }
    // the control block: zero, with empty global link queues (all ones);
    // set by the device (a copy from pageable host memory would first wait
    // for the stream)
    static_assert(offsetof(AsyncCtl, full_q) == offsetof(AsyncCtl, free_q) + sizeof(AsyncCtl::free_q),
                  "the two queue arrays are contiguous");
    TR_CUDA(cudaMemsetAsync(A.ctl, 0, sizeof(AsyncCtl), st));
    TR_CUDA(cudaMemsetAsync(A.ctl->free_q, 0xFF, sizeof(AsyncCtl::free_q) + sizeof(AsyncCtl::full_q), st));
    AsyncCtl hc;
    // resident blocks per SM: an occupancy query, once per configuration
    const std::vector<int> okey = {A.dec, S, A.use_pre, P.kind, P.ww_lo != nullptr};
    auto oc = pr->async_occupancy.find(okey);
    int maxb = 0;
    if (oc != pr->async_occupancy.end()) {
        maxb = oc->second;
    } else {
        maxb = async_max_blocks_per_sm(P, A.dec, S, A.use_pre != 0);
        pr->async_occupancy[okey] = maxb;
    }
    if (maxb < 1) return set_err(TR_ERR_INVALID, "stash does not fit in shared memory");
    const int bps = o->blocks_per_sm > 0 ? std::min(o->blocks_per_sm, maxb) : maxb;
    // monolithic scheme: the warps' deferred mesh walks queue in global memory
    // (L2-resident; in shared memory they would halve the L1 cache)
    if (dec == DEC_MONO && P.has_mesh && P.mesh_walk) {
        A.walkq = (WalkQ*)workspace(pr, "walkq", walk_queue_bytes(pr->sms * bps));
        if (!A.walkq) return set_err(TR_ERR_NOMEM, "mesh-walk queue allocation failed");
    }
    int smem = 0;
    LaunchTimer lt;
    TR_CUDA(cudaEventRecord(lt.a, st));
    if (A.use_pre) TR_CUDA(launch_presample(P, R, A, pr->sms * 8, st));
    TR_CUDA(launch_async(P, R, A, T, pr->err, pr->sms * bps, st, &smem));
    TR_CUDA(cudaEventRecord(lt.b, st));
    out.launches += 1;
    // the fixed-order reduction of the per-history scores follows the launch
    // in the stream (after a failed launch its sums are discarded)
    TR_CUDA(launch_hist_reduce(T, R.n_hist, hist_partial, st));
    // one host round trip: control block, error word, the caller's counter
    // and the scalar bins, gathered on the device
    Readback rb;
    tr_status rs = read_status(pr, A.ctl, nullptr, out.want_count, rb);
    if (rs != TR_OK) return rs;
    hc = rb.hc;
    out.kernel_ms += lt.elapsed();
    tr_status es = decode_err(rb.err);
    if (es == TR_ERR_TIMEOUT)
        return set_err(es, g_err + "; live " + std::to_string(hc.live) + ", source cursor " +
                               std::to_string(hc.src_cursor) + " of " + std::to_string(R.n_hist) + ", spills " +
                               std::to_string(hc.spills) + ", refills " + std::to_string(hc.refills) + ", hungry warps " +
                               std::to_string(hc.hungry));
    if (es != TR_OK) return es;
    out.spills += hc.spills;
    out.refills += hc.refills;
    if (hc.live != 0) return set_err(TR_ERR_STATE, "asynchronous run ended with live particles");
    out.have_readback = true;
    out.count = rb.count[0];
    std::memcpy(out.scal, rb.scal, sizeof(out.scal));
    return TR_OK;
}

static RunParams base_params(const tr_run_opts* o, unsigned long long n)
{
    RunParams R{};
    R.n_hist = n;
    R.key0 = (uint32_t)o->seed;
    R.key1 = (uint32_t)(o->seed >> 32) ^ o->problem_tag;
    R.id_hi = 0;
    R.max_events = o->max_events ? o->max_events : 10000000u;
    R.eig = 0;
    R.inv_k = 1.0;
    R.want_log = o->want_event_log ? 1 : 0;
    R.remap_every = o->remap_every > 0 ? o->remap_every : 1;
    R.max_spin = o->max_spin > 0 ? (uint64_t)o->max_spin : (1ull << 24);
    R.max_wait_ns = (uint64_t)(o->max_wait_ms ? o->max_wait_ms : 60000u) * 1000000ull;
    R.spill_threshold = o->spill_threshold ? o->spill_threshold : 64;
    R.id_base = (uint32_t)o->first_history;
    return R;
}

extern "C" tr_status tr_run_fixed_source(tr_problem* pr, const tr_run_opts* o, tr_run_stats* stats)
{
    if (!pr) return set_err(TR_ERR_INVALID, "problem is NULL");
    DeviceGuard dg(pr->ctx.device);
    tr_status s = validate_opts(o);
    if (s != TR_OK) return s;
    const DevProblem& P = pr->dp;
    const cudaStream_t st = pr->stream;
    if (P.ww_lo && o->decomposition != TR_DECOMP_MONO)
        return set_err(TR_ERR_INVALID, "weight windows run with the monolithic scheme");
    RunParams R = base_params(o, o->n_histories);
    if (R.want_log) {
        s = ensure_log(pr, std::max<unsigned long long>(o->n_histories, 1));
        if (s != TR_OK) return s;
    }
    s = zero_raw(pr);
    if (s != TR_OK) return s;
    TR_CUDA(cudaMemsetAsync(pr->counts, 0, 16 * 8, st));
    TR_CUDA(cudaMemsetAsync(pr->err, 0, sizeof(ErrorWord), st));
    Bank bank{};
    cudaEvent_t e0, e1;
    TR_CUDA(cudaEventCreate(&e0));
    TR_CUDA(cudaEventCreate(&e1));
    TR_CUDA(cudaEventRecord(e0, st));
    TransportOut to;
    s = transport(pr, o, R, bank, nullptr, to);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != TR_OK) {
        pr->have_run = false;
        return s;
    }
    const double inv = o->n_histories ? 1.0 / (double)o->n_histories : 0.0;
    TR_CUDA(launch_fix_scale(pr->raw_mesh, P.mesh_size, inv, pr->res_mesh, st));
    TR_CUDA(launch_fix_scale(pr->raw_energy, P.energy_size, inv, pr->res_energy, st));
    TR_CUDA(launch_fix_scale(pr->raw_scal, 3, inv, pr->res_scal, st));
    TR_CUDA(launch_fix_scale(pr->raw_time, P.n_tbins, inv, pr->res_time, st));
    unsigned long long cnt[16];
    TR_CUDA(cudaMemcpyAsync(cnt, pr->counts, sizeof(cnt), cudaMemcpyDeviceToHost, st));
    TR_CUDA(cudaStreamSynchronize(st));
    pr->have_run = true;
    pr->have_std = false;
    pr->have_fixed = true;
    pr->last_fixed = *o;
    pr->log_count = R.want_log ? o->n_histories : 0;
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->histories = o->n_histories;
        unsigned long long ev = 0;
        for (int i = 0; i < 8; ++i) {
            stats->events_by_type[i] = cnt[i];
            stats->final_by_type[i] = cnt[8 + i];
            if (i != EV_SOURCE) ev += cnt[i];
        }
        stats->events = ev;
        stats->launches = to.launches;
        stats->spills = to.spills;
        stats->refills = to.refills;
        stats->seconds = ms * 1e-3;
        stats->transport_seconds = to.kernel_ms * 1e-3;
    }
    return TR_OK;
}

// ---------------------------------------------------------------------------
// power iteration
// ---------------------------------------------------------------------------
// Serialised power-iteration state (tr_eig_checkpoint): this header, then
// k_batch, ktl_batch (doubles) and n_source (u64) for the batches done, the
// active-batch tally sums and sums of squares (nall + 1 doubles each), and the
// source bank of the next batch (x, y, z doubles, g int32, cell uint32).
struct EigCkpt {
    char magic[8];
    uint64_t n_per_batch, seed, N;
    uint32_t n_inactive, n_active, problem_tag, b_next;
    int32_t scheme, decomposition, mesh_size, energy_size, n_mat, G, nall, pad;
    double k0, bank_factor, k, ksum, ksq, kernel_ms;
    uint64_t tlaunch;
    uint64_t fingerprint;              // the problem's (geometry, cross sections, source, tallies)
    unsigned long long counts[16];
};
static const char EIG_MAGIC[8] = {'T', 'R', 'E', 'I', 'G', 'C', 'K', '2'};

static size_t eig_ckpt_bytes(uint32_t b_next, int nall, unsigned long long N)
{
    return sizeof(EigCkpt) + (size_t)b_next * 24 + (size_t)(nall + 1) * 16 + (size_t)N * 32;
}

extern "C" tr_status tr_eig_checkpoint(const tr_problem* pr, void* buf, size_t cap, size_t* bytes)
{
    if (!pr || !bytes) return set_err(TR_ERR_INVALID, "NULL argument");
    if (pr->ckpt.empty()) return set_err(TR_ERR_STATE, "no power iteration stopped early");
    *bytes = pr->ckpt.size();
    if (!buf) return TR_OK;
    if (cap < pr->ckpt.size()) return set_err(TR_ERR_INVALID, "checkpoint buffer too small");
    std::memcpy(buf, pr->ckpt.data(), pr->ckpt.size());
    return TR_OK;
}

extern "C" tr_status tr_run_power_iteration(tr_problem* pr, const tr_eig_opts* eo, tr_eig_result* res)
{
    if (!pr || !eo || !res) return set_err(TR_ERR_INVALID, "NULL argument");
    DeviceGuard dg(pr->ctx.device);
    if (pr->dp.kind != TR_XS_MG) return set_err(TR_ERR_INVALID, "power iteration needs multigroup data");
    if (pr->dp.ww_lo) return set_err(TR_ERR_INVALID, "weight windows are offered for fixed-source runs");
    if (pr->dp.timed) return set_err(TR_ERR_INVALID, "timed problems run fixed source only");
    tr_status s = validate_opts(&eo->run);
    if (s != TR_OK) return s;
    if (eo->n_per_batch < 1 || eo->n_active < 2) return set_err(TR_ERR_INVALID, "need n_per_batch >= 1 and n_active >= 2");
    const DevProblem& P = pr->dp;
    const cudaStream_t st = pr->stream;
    const double factor = eo->bank_capacity_factor > 0.0 ? eo->bank_capacity_factor : 4.0;
    const unsigned long long cap = (unsigned long long)std::ceil(factor * (double)eo->n_per_batch) + 64;
    if (cap >= (1ull << 32)) return set_err(TR_ERR_INVALID, "bank capacity must stay below 2^32");
    Bank bank, ordered, source;
    if (!carve_bank(pr, "bank", cap, bank, true) || !carve_bank(pr, "ordered", cap, ordered, true) ||
        !carve_bank(pr, "source", cap, source, false))
        return set_err(TR_ERR_NOMEM, "bank allocation failed");
    unsigned* site_count = (unsigned*)workspace(pr, "site_count", cap * 4);
    unsigned* copies = (unsigned*)workspace(pr, "copies", cap * 4);
    unsigned long long* offs = (unsigned long long*)workspace(pr, "offsets", cap * 8);
    unsigned long long* tiles = (unsigned long long*)workspace(pr, "scan_tiles", ((cap + 2047) / 2048 + 1) * 8);
    unsigned long long* total = (unsigned long long*)workspace(pr, "scan_total", 8);
    if (!site_count || !copies || !offs || !tiles || !total) return set_err(TR_ERR_NOMEM, "bank allocation failed");
    bank.site_count = site_count;
    const tr_run_opts* o = &eo->run;
    if (o->first_history != 0) return set_err(TR_ERR_INVALID, "first_history applies to fixed-source runs only");
    RunParams R = base_params(o, eo->n_per_batch);
    R.eig = 1;
    if (R.want_log) {
        s = ensure_log(pr, cap);
        if (s != TR_OK) return s;
    }
    const int ms = std::max(P.mesh_size, 0), es = std::max(P.energy_size, 0);
    const int nall = ms + es + 3;
    TR_CUDA(cudaMemsetAsync(pr->sum_all, 0, (size_t)(nall + 1) * 8, st));
    TR_CUDA(cudaMemsetAsync(pr->sq_all, 0, (size_t)(nall + 1) * 8, st));
    TR_CUDA(cudaMemsetAsync(pr->counts, 0, 16 * 8, st));
    TR_CUDA(cudaMemsetAsync(pr->err, 0, sizeof(ErrorWord), st));
    const uint32_t nb = eo->n_inactive + eo->n_active;
    double k = eo->k0 > 0.0 ? eo->k0 : 1.0;
    unsigned long long N = eo->n_per_batch;
    double ksum = 0.0, ksq = 0.0;
    std::vector<FixBin> scal(3);
    bool have_src = false;
    double kernel_ms = 0.0;
    unsigned long long tlaunch = 0;
    std::vector<double> kh, ktlh;         // per-batch eigenvalue history (kept for checkpoints)
    std::vector<uint64_t> nsh;
    uint32_t b0 = 0;
    pr->ckpt.clear();
    if (eo->resume_from) {
        // continue a run stopped early: check the signature, restore the state
        const unsigned char* q = (const unsigned char*)eo->resume_from;
        EigCkpt h;
        if (eo->resume_bytes < sizeof(h)) return set_err(TR_ERR_INVALID, "checkpoint too short");
        std::memcpy(&h, q, sizeof(h));
        if (std::memcmp(h.magic, EIG_MAGIC, 8) != 0) return set_err(TR_ERR_INVALID, "not a checkpoint");
        const double k0 = eo->k0 > 0.0 ? eo->k0 : 1.0;
        if (h.n_per_batch != eo->n_per_batch || h.n_inactive != eo->n_inactive || h.n_active != eo->n_active ||
            h.seed != o->seed || h.problem_tag != o->problem_tag || h.scheme != o->scheme ||
            h.decomposition != o->decomposition || h.k0 != k0 || h.bank_factor != factor ||
            h.mesh_size != P.mesh_size || h.energy_size != P.energy_size || h.n_mat != P.n_mat || h.G != P.G ||
            h.nall != nall || h.b_next < 1 || h.b_next >= nb || h.fingerprint != pr->fingerprint)
            return set_err(TR_ERR_STATE, "checkpoint does not match this problem and these options");
        if (h.N > cap || eo->resume_bytes != eig_ckpt_bytes(h.b_next, nall, h.N))
            return set_err(TR_ERR_INVALID, "checkpoint size mismatch");
        // every restored site must lie in the problem: group in range, the
        // packed cell inside the grid (with the pin bit only where a pin
        // is), the position finite and within that cell's planes; the
        // transport kernels index their tables with these values
        {
            const unsigned char* bq = q + sizeof(h) + 24 * (size_t)h.b_next + 16 * (size_t)(nall + 1);
            const size_t n8 = (size_t)h.N * 8, n4 = (size_t)h.N * 4;
            for (unsigned long long i = 0; i < h.N; ++i) {
                double x[3];
                int32_t g;
                uint32_t c;
                for (int a = 0; a < 3; ++a) std::memcpy(&x[a], bq + a * n8 + 8 * i, 8);
                std::memcpy(&g, bq + 3 * n8 + 4 * i, 4);
                std::memcpy(&c, bq + 3 * n8 + n4 + 4 * i, 4);
                const int ci[3] = {(int)(c & 1023u), (int)((c >> 10) & 1023u), (int)((c >> 20) & 1023u)};
                const int nn[3] = {P.nx, P.ny, P.nz};
                bool bad = g < 0 || g >= P.G || (c >> 31) != 0;
                for (int a = 0; a < 3 && !bad; ++a)
                    bad = ci[a] >= nn[a] || !std::isfinite(x[a]) || x[a] < pr->hplanes[a][ci[a]] ||
                          x[a] > pr->hplanes[a][ci[a] + 1];
                if (!bad && (c >> 30))
                    bad = !pr->hpin[((size_t)ci[2] * P.ny + ci[1]) * P.nx + ci[0]];
                if (bad) return set_err(TR_ERR_INVALID, "checkpoint source site " + std::to_string(i) +
                                                        " lies outside the problem");
            }
        }
        q += sizeof(h);
        kh.assign((const double*)q, (const double*)q + h.b_next);
        q += 8 * (size_t)h.b_next;
        ktlh.assign((const double*)q, (const double*)q + h.b_next);
        q += 8 * (size_t)h.b_next;
        nsh.resize(h.b_next);
        std::memcpy(nsh.data(), q, 8 * (size_t)h.b_next);
        q += 8 * (size_t)h.b_next;
        TR_CUDA(cudaMemcpyAsync(pr->sum_all, q, (size_t)(nall + 1) * 8, cudaMemcpyHostToDevice, st));
        q += (size_t)(nall + 1) * 8;
        TR_CUDA(cudaMemcpyAsync(pr->sq_all, q, (size_t)(nall + 1) * 8, cudaMemcpyHostToDevice, st));
        q += (size_t)(nall + 1) * 8;
        const size_t n8 = (size_t)h.N * 8, n4 = (size_t)h.N * 4;
        TR_CUDA(cudaMemcpyAsync(source.x, q, n8, cudaMemcpyHostToDevice, st));
        TR_CUDA(cudaMemcpyAsync(source.y, q + n8, n8, cudaMemcpyHostToDevice, st));
        TR_CUDA(cudaMemcpyAsync(source.z, q + 2 * n8, n8, cudaMemcpyHostToDevice, st));
        TR_CUDA(cudaMemcpyAsync(source.g, q + 3 * n8, n4, cudaMemcpyHostToDevice, st));
        TR_CUDA(cudaMemcpyAsync(source.cell, q + 3 * n8 + n4, n4, cudaMemcpyHostToDevice, st));
        TR_CUDA(cudaMemcpyAsync(pr->counts, h.counts, sizeof(h.counts), cudaMemcpyHostToDevice, st));
        TR_CUDA(cudaStreamSynchronize(st));   // the host buffer may go away on return
        b0 = h.b_next;
        k = h.k;
        N = h.N;
        ksum = h.ksum;
        ksq = h.ksq;
        kernel_ms = h.kernel_ms;
        tlaunch = h.tlaunch;
        have_src = true;
    }
    const uint32_t stop = (eo->stop_after > 0 && eo->stop_after < nb) ? eo->stop_after : nb;
    if (stop <= b0) return set_err(TR_ERR_INVALID, "stop_after must lie beyond the resumed batch");
    for (uint32_t b = 0; b < b0; ++b) {
        if (res->k_batch) res->k_batch[b] = kh[b];
        if (res->ktl_batch) res->ktl_batch[b] = ktlh[b];
        if (res->n_source) res->n_source[b] = nsh[b];
    }
    cudaEvent_t e0, e1;
    TR_CUDA(cudaEventCreate(&e0));
    TR_CUDA(cudaEventCreate(&e1));
    TR_CUDA(cudaEventRecord(e0, st));
    for (uint32_t b = b0; b < nb; ++b) {
        s = zero_raw(pr);
        if (s != TR_OK) return s;
        TR_CUDA(cudaMemsetAsync(bank.count, 0, 8, st));
        R.id_hi = b;
        R.inv_k = 1.0 / k;
        R.n_hist = N;
        TransportOut to;
        to.want_count = bank.count;
        s = transport(pr, o, R, bank, have_src ? &source : nullptr, to);
        if (s != TR_OK) return s;
        kernel_ms += to.kernel_ms;
        tlaunch += to.launches;
        // the bank's size and the scalar bins (read with the launch's status
        // by the asynchronous scheme; the stack scheme reads them here)
        unsigned long long M = 0;
        if (to.have_readback) {
            M = to.count;
            std::memcpy(scal.data(), to.scal, 3 * sizeof(FixBin));
        } else {
            TR_CUDA(cudaMemcpyAsync(&M, bank.count, 8, cudaMemcpyDeviceToHost, st));
            TR_CUDA(cudaMemcpyAsync(scal.data(), pr->raw_scal, 3 * sizeof(FixBin), cudaMemcpyDeviceToHost, st));
            TR_CUDA(cudaStreamSynchronize(st));
        }
        if (M > cap) return set_err(TR_ERR_CAPACITY, "fission bank overflow");
        const double kb = k * ((double)M / (double)N);
        if (res->k_batch) res->k_batch[b] = kb;
        const double prod = fix_value(scal[2]);
        if (res->ktl_batch) res->ktl_batch[b] = prod / (double)N;
        if (res->n_source) res->n_source[b] = N;
        kh.push_back(kb);
        ktlh.push_back(prod / (double)N);
        nsh.push_back(N);
        if (b >= eo->n_inactive) {
            const double inv = 1.0 / (double)N;
            TR_CUDA(launch_eig_accumulate(pr->raw_mesh, ms, inv, pr->sum_all, pr->sq_all, st));
            TR_CUDA(launch_eig_accumulate(pr->raw_energy, es, inv, pr->sum_all + ms, pr->sq_all + ms, st));
            TR_CUDA(launch_eig_accumulate(pr->raw_scal, 3, inv, pr->sum_all + ms + es, pr->sq_all + ms + es, st));
            ksum += kb;
            ksq += kb * kb;
        }
        k = kb;
        if (M == 0) return set_err(TR_ERR_STATE, "the fission source died out");
        if (b + 1 == nb) {
            pr->log_count = R.want_log ? N : 0;
            break;
        }
        // order the bank by (parent, site sequence); splitting roulette back
        // to n_per_batch.  The host reads the two scan totals and the error
        // word once, after the population is written (the kernels bound
        // every index by its buffer and report overflows in the error word).
        Readback* drb = (Readback*)workspace(pr, "readback", sizeof(Readback));
        if (!drb) return set_err(TR_ERR_NOMEM, "readback buffer allocation failed");
        TR_CUDA(launch_scan(site_count, N, tiles, offs, total, st));
        Gather g1{};
        g1.src[0] = total;
        g1.dst[0] = &drb->count[0];
        g1.bytes[0] = sizeof(unsigned long long);
        g1.n = 1;
        TR_CUDA(launch_gather(g1, st));
        TR_CUDA(launch_bank_order(bank, M, offs, ordered, pr->err, st));
        const double r = (double)eo->n_per_batch / (double)M;
        const double fl = std::floor(r), fr = r - fl;
        TR_CUDA(launch_pop_copies(M, R.key0, (uint32_t)(o->seed >> 32) ^ TAG_POP, b, (unsigned)fl, fr, copies, st));
        TR_CUDA(launch_scan(copies, M, tiles, offs, total, st));
        TR_CUDA(launch_pop_write(ordered, M, copies, offs, source, cap, pr->err, st));
        Gather g2{};
        g2.src[0] = total;
        g2.dst[0] = &drb->count[1];
        g2.bytes[0] = sizeof(unsigned long long);
        g2.src[1] = pr->err;
        g2.dst[1] = &drb->err;
        g2.bytes[1] = sizeof(ErrorWord);
        g2.n = 2;
        TR_CUDA(launch_gather(g2, st));
        Readback rb;
        TR_CUDA(cudaMemcpyAsync(&rb, drb, sizeof(rb), cudaMemcpyDeviceToHost, st));
        TR_CUDA(cudaStreamSynchronize(st));
        const unsigned long long tot = rb.count[0], nn = rb.count[1];
        if (tot != M) return set_err(TR_ERR_STATE, "bank site counts disagree with the bank size");
        if (nn > cap) return set_err(TR_ERR_CAPACITY, "source bank overflow after population control");
        if (nn >= (1ull << 32)) return set_err(TR_ERR_CAPACITY, "batch too large");
        s = decode_err(rb.err);
        if (s != TR_OK) return s;
        N = nn;
        have_src = true;
        if (b + 1 == stop) {
            // stop early: keep the state before batch b + 1 for tr_eig_checkpoint
            EigCkpt h{};
            std::memcpy(h.magic, EIG_MAGIC, 8);
            h.n_per_batch = eo->n_per_batch;
            h.seed = o->seed;
            h.N = N;
            h.n_inactive = eo->n_inactive;
            h.n_active = eo->n_active;
            h.problem_tag = o->problem_tag;
            h.b_next = b + 1;
            h.scheme = o->scheme;
            h.decomposition = o->decomposition;
            h.mesh_size = P.mesh_size;
            h.energy_size = P.energy_size;
            h.n_mat = P.n_mat;
            h.G = P.G;
            h.nall = nall;
            h.k0 = eo->k0 > 0.0 ? eo->k0 : 1.0;
            h.bank_factor = factor;
            h.k = k;
            h.ksum = ksum;
            h.ksq = ksq;
            h.kernel_ms = kernel_ms;
            h.tlaunch = tlaunch;
            h.fingerprint = pr->fingerprint;
            TR_CUDA(cudaMemcpyAsync(h.counts, pr->counts, sizeof(h.counts), cudaMemcpyDeviceToHost, st));
            std::vector<unsigned char> buf(eig_ckpt_bytes(h.b_next, nall, N));
            unsigned char* q = buf.data() + sizeof(h);
            std::memcpy(q, kh.data(), 8 * kh.size());
            q += 8 * kh.size();
            std::memcpy(q, ktlh.data(), 8 * ktlh.size());
            q += 8 * ktlh.size();
            std::memcpy(q, nsh.data(), 8 * nsh.size());
            q += 8 * nsh.size();
            TR_CUDA(cudaMemcpyAsync(q, pr->sum_all, (size_t)(nall + 1) * 8, cudaMemcpyDeviceToHost, st));
            q += (size_t)(nall + 1) * 8;
            TR_CUDA(cudaMemcpyAsync(q, pr->sq_all, (size_t)(nall + 1) * 8, cudaMemcpyDeviceToHost, st));
            q += (size_t)(nall + 1) * 8;
            const size_t n8 = (size_t)N * 8, n4 = (size_t)N * 4;
            TR_CUDA(cudaMemcpyAsync(q, source.x, n8, cudaMemcpyDeviceToHost, st));
            TR_CUDA(cudaMemcpyAsync(q + n8, source.y, n8, cudaMemcpyDeviceToHost, st));
            TR_CUDA(cudaMemcpyAsync(q + 2 * n8, source.z, n8, cudaMemcpyDeviceToHost, st));
            TR_CUDA(cudaMemcpyAsync(q + 3 * n8, source.g, n4, cudaMemcpyDeviceToHost, st));
            TR_CUDA(cudaMemcpyAsync(q + 3 * n8 + n4, source.cell, n4, cudaMemcpyDeviceToHost, st));
            TR_CUDA(cudaStreamSynchronize(st));
            std::memcpy(buf.data(), &h, sizeof(h));
            TR_CUDA(cudaEventRecord(e1, st));
            TR_CUDA(cudaEventSynchronize(e1));
            float msec = 0.f;
            cudaEventElapsedTime(&msec, e0, e1);
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            pr->ckpt.swap(buf);
            std::memset(res->final_by_type, 0, sizeof(res->final_by_type));
            res->k_mean = res->k_std = 0.0;
            res->histories = h.counts[EV_SOURCE];
            res->events = 0;
            for (int i = 1; i < 8; ++i) res->events += h.counts[i];
            for (int i = 0; i < 8; ++i) res->final_by_type[i] = h.counts[8 + i];
            res->seconds = msec * 1e-3;
            res->transport_seconds = kernel_ms * 1e-3;
            res->transport_launches = tlaunch;
            res->batches_done = b + 1;
            pr->have_run = false;   // tallies are final only at the end of the run
            pr->have_std = false;
            pr->have_fixed = false;
            return TR_OK;
        }
    }
    TR_CUDA(cudaEventRecord(e1, st));
    TR_CUDA(cudaEventSynchronize(e1));
    float msec = 0.f;
    cudaEventElapsedTime(&msec, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double na = (double)eo->n_active;
    TR_CUDA(launch_eig_finish(pr->sum_all, pr->sq_all, ms, na, pr->res_mesh, pr->sd_mesh, st));
    TR_CUDA(launch_eig_finish(pr->sum_all + ms, pr->sq_all + ms, es, na, pr->res_energy, pr->sd_energy, st));
    TR_CUDA(launch_eig_finish(pr->sum_all + ms + es, pr->sq_all + ms + es, 3, na, pr->res_scal, pr->sd_scal, st));
    unsigned long long cnt[16];
    TR_CUDA(cudaMemcpyAsync(cnt, pr->counts, sizeof(cnt), cudaMemcpyDeviceToHost, st));
    TR_CUDA(cudaStreamSynchronize(st));
    res->k_mean = ksum / na;
    const double var = (ksq / na - res->k_mean * res->k_mean) / (na - 1.0);
    res->k_std = var > 0.0 ? std::sqrt(var) : 0.0;
    unsigned long long ev = 0;
    for (int i = 0; i < 8; ++i) {
        res->final_by_type[i] = cnt[8 + i];
        if (i != EV_SOURCE) ev += cnt[i];
    }
    res->histories = cnt[EV_SOURCE];
    res->events = ev;
    res->seconds = msec * 1e-3;
    res->transport_seconds = kernel_ms * 1e-3;
    res->transport_launches = tlaunch;
    res->batches_done = nb;
    pr->have_run = true;
    pr->have_std = true;
    pr->have_fixed = false;
    return TR_OK;
}

// ---------------------------------------------------------------------------
// sensitivities
// ---------------------------------------------------------------------------
extern "C" tr_status tr_sensitivities(tr_problem* pr, const tr_run_opts* o, const double* d_grad_mesh,
                                      const double* d_grad_scalars, double* d_sigt, double* d_sigs, double* d_nusigf)
{
    if (!pr || !o || !d_sigt || !d_sigs || !d_nusigf) return set_err(TR_ERR_INVALID, "NULL argument");
    DeviceGuard dg(pr->ctx.device);
    if (pr->dp.kind != TR_XS_MG) return set_err(TR_ERR_INVALID, "sensitivities need multigroup data");
    if (pr->dp.ww_lo) return set_err(TR_ERR_INVALID, "sensitivities are offered for analog runs");
    if (pr->dp.timed) return set_err(TR_ERR_INVALID, "sensitivities are offered for untimed problems");
    tr_status s = validate_opts(o);
    if (s != TR_OK) return s;
    const tr_run_opts& L = pr->last_fixed;
    if (!pr->have_fixed || L.n_histories != o->n_histories || L.seed != o->seed || L.problem_tag != o->problem_tag ||
        L.max_events != o->max_events || L.first_history != o->first_history)
        return set_err(TR_ERR_STATE, "tr_sensitivities needs a prior tr_run_fixed_source with the same histories");
    const DevProblem& P = pr->dp;
    const cudaStream_t st = pr->stream;
    const size_t MG = (size_t)P.n_mat * P.G;
    TR_CUDA(cudaMemsetAsync(d_sigt, 0, MG * 8, st));
    TR_CUDA(cudaMemsetAsync(d_sigs, 0, MG * P.G * 8, st));
    TR_CUDA(cudaMemsetAsync(d_nusigf, 0, MG * 8, st));
    if (o->n_histories == 0) {
        TR_CUDA(cudaStreamSynchronize(st));
        return TR_OK;
    }
    double* F = (double*)workspace(pr, "adjoint_F", o->n_histories * 8);
    if (!F) return set_err(TR_ERR_NOMEM, "adjoint workspace allocation failed");
    TR_CUDA(cudaMemsetAsync(pr->err, 0, sizeof(ErrorWord), st));
    RunParams R = base_params(o, o->n_histories);
    R.want_log = 0;
    unsigned long long* cursors = (unsigned long long*)workspace(pr, "adj_cursors", 16);
    if (!cursors) return set_err(TR_ERR_NOMEM, "workspace allocation failed");
    // both passes start the same histories: sample their sources once
    AsyncArgs S{};
    const bool pre = o->n_histories <= PRESAMPLE_MAX_HIST;
    if (pre) {
        if (!carve_soa(pr, "presample", o->n_histories, S.pre)) return set_err(TR_ERR_NOMEM, "source buffer allocation failed");
        TR_CUDA(launch_presample(P, R, S, pr->sms * 8, st));
    }
    TR_CUDA(launch_adjoint(P, R, d_grad_mesh, d_grad_scalars, F, d_sigt, d_sigs, d_nusigf, pr->err, pr->sms, cursors,
                           pre ? &S.pre : nullptr, st));
    s = check_err(pr);
    if (s != TR_OK) return s;
    const double inv = 1.0 / (double)o->n_histories;
    TR_CUDA(launch_scale(d_sigt, (int)MG, inv, d_sigt, st));
    TR_CUDA(launch_scale(d_sigs, (int)(MG * P.G), inv, d_sigs, st));
    TR_CUDA(launch_scale(d_nusigf, (int)MG, inv, d_nusigf, st));
    TR_CUDA(cudaStreamSynchronize(st));
    return TR_OK;
}

// ---------------------------------------------------------------------------
// batched launches
// ---------------------------------------------------------------------------
namespace {

struct BatchTuning {
    int blocks_per_sm, stash_slots, remap_every;
};

std::mutex g_tune_mu;
std::map<std::vector<unsigned long long>, BatchTuning> g_tune_cache;

std::vector<unsigned long long> batch_signature(tr_problem* const* probs, int32_t n, const uint64_t* nh,
                                                const tr_run_opts* o)
{
    std::vector<unsigned long long> k;
    k.reserve(2 * (size_t)n + 16);
    for (int32_t i = 0; i < n; ++i) {
        k.push_back((unsigned long long)(uintptr_t)probs[i]);
        k.push_back(nh[i]);
    }
    k.push_back(o->seed);
    k.push_back((unsigned long long)o->decomposition);
    k.push_back(o->queue_capacity);
    k.push_back((unsigned long long)o->blocks_per_sm);
    k.push_back((unsigned long long)o->stash_slots);
    k.push_back((unsigned long long)o->remap_every);
    k.push_back((unsigned long long)o->max_spin);
    k.push_back((unsigned long long)o->max_wait_ms);
    k.push_back(o->max_events);
    k.push_back((unsigned long long)o->want_event_log);
    k.push_back((unsigned long long)(uint32_t)o->spill_threshold);
    k.push_back(o->problem_tag);
    return k;
}

}  // namespace

// Enqueue one batched run (everything from zeroing to normalisation) on the
// leader's stream; used directly and under stream capture.
static tr_status enqueue_batched(tr_problem* lead, tr_problem* const* probs, int32_t n, const tr_run_opts* o,
                                 const BatchTuning& tune, DevProblem* d_probs, Tallies* d_tal,
                                 unsigned long long* d_off, ScaleJob* d_jobs, int n_jobs, const AsyncArgs& A0,
                                 unsigned long long total, int maxch, double* hist_partial)
{
    const cudaStream_t st = lead->stream;
    for (int32_t i = 0; i < n; ++i) {
        tr_problem* p = probs[i];
        TR_CUDA(cudaMemsetAsync(p->raw_mesh, 0, std::max(p->dp.mesh_size, 1) * sizeof(FixBin), st));
        TR_CUDA(cudaMemsetAsync(p->raw_energy, 0, std::max(p->dp.energy_size, 1) * sizeof(FixBin), st));
        TR_CUDA(cudaMemsetAsync(p->raw_scal, 0, 4 * sizeof(FixBin), st));
        TR_CUDA(cudaMemsetAsync(p->raw_time, 0, std::max(p->dp.n_tbins, 1) * sizeof(FixBin), st));
        TR_CUDA(cudaMemsetAsync(p->counts, 0, 16 * 8, st));
    }
    TR_CUDA(cudaMemsetAsync(lead->err, 0, sizeof(ErrorWord), st));
    AsyncArgs A = A0;
    TR_CUDA(cudaMemsetAsync(A.ctl, 0, sizeof(AsyncCtl), st));
    TR_CUDA(cudaMemsetAsync(A.ctl->free_q, 0xFF, sizeof(A.ctl->free_q), st));
    TR_CUDA(cudaMemsetAsync(A.ctl->full_q, 0xFF, sizeof(A.ctl->full_q), st));
    A.probs = d_probs;
    A.tallies = d_tal;
    A.hist_off = d_off;
    A.n_probs = n;
    A.stash_slots = tune.stash_slots;
    RunParams R = base_params(o, total);
    R.remap_every = tune.remap_every;
    R.want_log = o->want_event_log ? 1 : 0;
    if (total > 0) TR_CUDA(launch_async_batched(lead->dp, R, A, lead->err, lead->sms * tune.blocks_per_sm, st));
    if (hist_partial) TR_CUDA(launch_hist_reduce_batched(d_tal, d_off, n, maxch, hist_partial, lead->err, st));
    TR_CUDA(launch_scale_jobs(d_jobs, n_jobs, st));
    return TR_OK;
}

extern "C" tr_status tr_run_batched(tr_problem* const* probs, int32_t n, const uint64_t* n_histories,
                                    const tr_run_opts* opts, tr_run_stats* stats)
{
    if (!probs || n < 1 || !n_histories || !opts) return set_err(TR_ERR_INVALID, "NULL argument or n < 1");
    tr_status s = validate_opts(opts);
    if (s != TR_OK) return s;
    if (opts->scheme != TR_SCHEME_ASYNC) return set_err(TR_ERR_INVALID, "batched runs use the asynchronous scheme");
    if (opts->decomposition != TR_DECOMP_MONO && opts->decomposition != TR_DECOMP_SPLIT)
        return set_err(TR_ERR_INVALID, "batched runs use the monolithic or decomposed scheme");
    if (opts->first_history != 0) return set_err(TR_ERR_INVALID, "first_history applies to single runs only");
    tr_problem* lead = probs[0];
    if (!lead) return set_err(TR_ERR_INVALID, "NULL problem in the batch");
    DeviceGuard dg(lead->ctx.device);
    unsigned long long total = 0;
    for (int32_t i = 0; i < n; ++i) {
        if (!probs[i]) return set_err(TR_ERR_INVALID, "NULL problem in the batch");
        if (probs[i]->dp.kind != TR_XS_MG) return set_err(TR_ERR_INVALID, "batched runs need multigroup problems");
        if (probs[i]->dp.ww_lo) return set_err(TR_ERR_INVALID, "batched runs are analog (no weight windows)");
        if (probs[i]->ctx.device != lead->ctx.device) return set_err(TR_ERR_INVALID, "all problems on one device");
        if (n_histories[i] >= (1ull << 32)) return set_err(TR_ERR_INVALID, "n_histories must be < 2^32 per problem");
        for (int32_t j = 0; j < i; ++j)
            if (probs[j] == probs[i]) return set_err(TR_ERR_INVALID, "a problem appears twice in the batch");
        total += n_histories[i];
    }
    if (opts->problem_tag & TAG_POP) return set_err(TR_ERR_INVALID, "problem_tag must be below 2^31");
    const cudaStream_t st = lead->stream;
    // outputs and logs allocated before any capture
    for (int32_t i = 0; i < n; ++i) {
        if (opts->want_event_log) {
            s = ensure_log(probs[i], std::max<unsigned long long>(n_histories[i], 1));
            if (s != TR_OK) return s;
        }
        if (probs[i]->stream != st) TR_CUDA(cudaStreamSynchronize(probs[i]->stream));
    }
    // autotuning of the options left at 0: blocks per SM, stash slots, remap frequency
    BatchTuning tune{opts->blocks_per_sm, opts->stash_slots ? (opts->stash_slots + 31) & ~31 : 0, opts->remap_every};
    if (tune.stash_slots && (tune.stash_slots < 32 * 9 || tune.stash_slots > 16384))
        return set_err(TR_ERR_INVALID, "stash_slots must be in 288..16384");
    const std::vector<unsigned long long> key = batch_signature(probs, n, n_histories, opts);
    const bool need_tune = tune.blocks_per_sm == 0 || tune.stash_slots == 0 || tune.remap_every == 0;
    if (need_tune) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) tune = it->second;
    }
    // device tables of the batch (leader's workspace)
    DevProblem* d_probs = (DevProblem*)workspace(lead, "batch_probs", sizeof(DevProblem) * n);
    Tallies* d_tal = (Tallies*)workspace(lead, "batch_tallies", sizeof(Tallies) * n);
    unsigned long long* d_off = (unsigned long long*)workspace(lead, "batch_off", 8 * (size_t)(n + 1));
    ScaleJob* d_jobs = (ScaleJob*)workspace(lead, "batch_jobs", sizeof(ScaleJob) * 3 * (size_t)n);
    const unsigned long long n_links = opts->queue_capacity ? (opts->queue_capacity + 31) / 32 : 8192;
    AsyncArgs A{};
    if (!d_probs || !d_tal || !d_off || !d_jobs || !carve_soa(lead, "links", n_links * 32, A.links))
        return set_err(TR_ERR_NOMEM, "batch table allocation failed");
    A.link_next = (unsigned*)workspace(lead, "link_next", n_links * 4);
    A.link_type = (int*)workspace(lead, "link_type", n_links * 4);
    A.link_fill = (int*)workspace(lead, "link_fill", n_links * 4);
    A.ctl = (AsyncCtl*)workspace(lead, "asyncctl", sizeof(AsyncCtl));
    if (!A.link_next || !A.link_type || !A.link_fill || !A.ctl) return set_err(TR_ERR_NOMEM, "link arena allocation failed");
    A.n_links = n_links;
    A.dec = opts->decomposition;
    std::vector<DevProblem> hp(n);
    std::vector<Tallies> ht(n);
    std::vector<unsigned long long> hoff(n + 1, 0);
    std::vector<ScaleJob> hj;
    for (int32_t i = 0; i < n; ++i) hoff[i + 1] = hoff[i] + n_histories[i];
    // scalar scores stored per history (each member in its own range) and
    // reduced per member in a fixed order after the launch, as single runs do
    double* hist = nullptr;
    double* hist_partial = nullptr;
    int maxch = 0;
    unsigned long long hstride = 0;
    if (total <= HIST_MAX) {
        hstride = (total + 65535) & ~65535ull;
        for (int32_t i = 0; i < n; ++i) maxch = std::max(maxch, hist_chunks(n_histories[i]));
        hist = (double*)workspace(lead, "batch_hist", 3 * std::max(hstride, 1ull) * sizeof(double));
        hist_partial = (double*)workspace(lead, "batch_hist_partial",
                                          3 * (size_t)n * (size_t)std::max(maxch, 1) * sizeof(double));
        if (!hist || !hist_partial) return set_err(TR_ERR_NOMEM, "history score buffer allocation failed");
    }
    for (int32_t i = 0; i < n; ++i) {
        hp[i] = probs[i]->dp;
        ht[i] = make_tallies(probs[i], opts->want_event_log != 0);
        ht[i].err = lead->err;   // the batch's one error word
        if (hist) {
            ht[i].hist_f = hist + hoff[i];
            ht[i].hist_a = hist + hstride + hoff[i];
            ht[i].hist_p = hist + 2 * hstride + hoff[i];
        }
        const double inv = n_histories[i] ? 1.0 / (double)n_histories[i] : 0.0;
        if (probs[i]->dp.mesh_size) hj.push_back({probs[i]->raw_mesh, probs[i]->res_mesh, probs[i]->dp.mesh_size, inv});
        if (probs[i]->dp.energy_size)
            hj.push_back({probs[i]->raw_energy, probs[i]->res_energy, probs[i]->dp.energy_size, inv});
        hj.push_back({probs[i]->raw_scal, probs[i]->res_scal, 3, inv});
        if (probs[i]->dp.n_tbins) hj.push_back({probs[i]->raw_time, probs[i]->res_time, probs[i]->dp.n_tbins, inv});
    }
    TR_CUDA(cudaMemcpyAsync(d_probs, hp.data(), sizeof(DevProblem) * n, cudaMemcpyHostToDevice, st));
    TR_CUDA(cudaMemcpyAsync(d_tal, ht.data(), sizeof(Tallies) * n, cudaMemcpyHostToDevice, st));
    TR_CUDA(cudaMemcpyAsync(d_off, hoff.data(), 8 * (size_t)(n + 1), cudaMemcpyHostToDevice, st));
    TR_CUDA(cudaMemcpyAsync(d_jobs, hj.data(), sizeof(ScaleJob) * hj.size(), cudaMemcpyHostToDevice, st));
    TR_CUDA(cudaStreamSynchronize(st));

    if (need_tune && (tune.blocks_per_sm == 0 || tune.stash_slots == 0 || tune.remap_every == 0)) {
        // time candidate settings on a sample (1/16 of each problem's histories)
        std::vector<uint64_t> sample(n);
        unsigned long long stotal = 0;
        std::vector<unsigned long long> soff(n + 1, 0);
        for (int32_t i = 0; i < n; ++i) {
            sample[i] = std::min<uint64_t>(n_histories[i], std::max<uint64_t>(64, n_histories[i] / 16));
            soff[i + 1] = soff[i] + sample[i];
            stotal += sample[i];
        }
        unsigned long long* d_soff = (unsigned long long*)workspace(lead, "batch_soff", 8 * (size_t)(n + 1));
        if (!d_soff) return set_err(TR_ERR_NOMEM, "autotune allocation failed");
        TR_CUDA(cudaMemcpyAsync(d_soff, soff.data(), 8 * (size_t)(n + 1), cudaMemcpyHostToDevice, st));
        // candidates: a field set by the caller stays fixed
        const std::vector<int> c_bps = tune.blocks_per_sm ? std::vector<int>{tune.blocks_per_sm} : std::vector<int>{1, 2};
        const std::vector<int> c_S = tune.stash_slots ? std::vector<int>{tune.stash_slots} : std::vector<int>{288, 512, 1024};
        // batched runs do not refill lanes inside the loop, so long loops idle
        // them: on the full 256-box workload 2 / 4 / 8 / 16 / 64 events per
        // remap ran at 1.72 / 1.72 / 1.78 / 1.51 / 0.90e9 events/s, while
        // samples of 1/16 of the histories favoured 16
        const std::vector<int> c_rm = tune.remap_every ? std::vector<int>{tune.remap_every}
                                      : A.dec          ? std::vector<int>{1}
                                                       : std::vector<int>{2, 4, 8};
        std::vector<BatchTuning> cands;
        for (int bps : c_bps)
            for (int S : c_S)
                for (int rm : c_rm)
                    if (async_batched_max_blocks_per_sm(A.dec, S) >= bps) cands.push_back({bps, S, rm});
        if (cands.empty()) return set_err(TR_ERR_INVALID, "no feasible tuning candidate");
        cudaEvent_t e0, e1;
        TR_CUDA(cudaEventCreate(&e0));
        TR_CUDA(cudaEventCreate(&e1));
        float best = 1e30f;
        BatchTuning pick = cands[0];
        for (const BatchTuning& t : cands) {
            TR_CUDA(cudaEventRecord(e0, st));
            s = enqueue_batched(lead, probs, n, opts, t, d_probs, d_tal, d_soff, d_jobs, 0, A, stotal, maxch,
                                hist_partial);
            if (s != TR_OK) return s;
            TR_CUDA(cudaEventRecord(e1, st));
            TR_CUDA(cudaEventSynchronize(e1));
            s = check_err(lead);
            if (s != TR_OK) return s;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                pick = t;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        tune = pick;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = tune;
    }
    if (async_batched_max_blocks_per_sm(A.dec, tune.stash_slots) < tune.blocks_per_sm)
        return set_err(TR_ERR_INVALID, "blocks_per_sm does not fit with this stash size");

    // the run: replay the captured graph when this leader ran the same batch last
    // the graph bakes in device addresses: any reallocated buffer forces a new capture
    std::vector<unsigned long long> gkey = key;
    gkey.push_back((unsigned long long)tune.blocks_per_sm);
    gkey.push_back((unsigned long long)tune.stash_slots);
    gkey.push_back((unsigned long long)tune.remap_every);
    for (const void* q : {(const void*)d_probs, (const void*)d_tal, (const void*)d_off, (const void*)d_jobs,
                          (const void*)A.links.x, (const void*)A.link_next, (const void*)A.link_type,
                          (const void*)A.link_fill, (const void*)A.ctl, (const void*)lead->err, (const void*)hist,
                          (const void*)hist_partial})
        gkey.push_back((unsigned long long)(uintptr_t)q);
    gkey.push_back((unsigned long long)maxch);
    for (int32_t i = 0; i < n; ++i)
        for (const void* q : {(const void*)probs[i]->raw_mesh, (const void*)probs[i]->raw_energy,
                              (const void*)probs[i]->raw_scal, (const void*)probs[i]->raw_time,
                              (const void*)probs[i]->counts})
            gkey.push_back((unsigned long long)(uintptr_t)q);
    gkey.push_back(hj.size());
    if (!lead->batch_graph || lead->batch_key != gkey) {
        if (lead->batch_graph) {
            cudaGraphExecDestroy(lead->batch_graph);
            lead->batch_graph = nullptr;
        }
        cudaStream_t cap;
        TR_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        const unsigned long long c0 = launch_count();
        TR_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        // capture on a private stream: the leader's stream is swapped for the capture
        cudaStream_t saved = lead->stream;
        lead->stream = cap;
        s = enqueue_batched(lead, probs, n, opts, tune, d_probs, d_tal, d_off, d_jobs, (int)hj.size(), A, total, maxch,
                            hist_partial);
        lead->stream = saved;
        const cudaError_t ce = cudaStreamEndCapture(cap, &g);
        cudaStreamDestroy(cap);
        // captured launches did not run: take them off the counter, count them at each replay
        lead->batch_graph_launches = launch_count() - c0;
        count_launches(0ull - lead->batch_graph_launches);
        if (s != TR_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (ce != cudaSuccess) return set_err(TR_ERR_CUDA, std::string("stream capture: ") + cudaGetErrorString(ce));
        const cudaError_t ie = cudaGraphInstantiate(&lead->batch_graph, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            lead->batch_graph = nullptr;
            return set_err(TR_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
        }
        lead->batch_key = gkey;
    }
    cudaEvent_t e0, e1;
    TR_CUDA(cudaEventCreate(&e0));
    TR_CUDA(cudaEventCreate(&e1));
    TR_CUDA(cudaEventRecord(e0, st));
    TR_CUDA(cudaGraphLaunch(lead->batch_graph, st));
    count_launches(lead->batch_graph_launches);
    TR_CUDA(cudaEventRecord(e1, st));
    AsyncCtl hc;
    TR_CUDA(cudaMemcpyAsync(&hc, A.ctl, sizeof(hc), cudaMemcpyDeviceToHost, st));
    std::vector<unsigned long long> cnt(16 * (size_t)n);
    for (int32_t i = 0; i < n; ++i)
        TR_CUDA(cudaMemcpyAsync(cnt.data() + 16 * (size_t)i, probs[i]->counts, 16 * 8, cudaMemcpyDeviceToHost, st));
    TR_CUDA(cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    s = check_err(lead);
    if (s == TR_ERR_TIMEOUT)
        return set_err(s, g_err + "; live " + std::to_string(hc.live) + ", spills " + std::to_string(hc.spills) +
                              ", refills " + std::to_string(hc.refills));
    if (s != TR_OK) return s;
    if (hc.live != 0) return set_err(TR_ERR_STATE, "batched run ended with live particles");
    for (int32_t i = 0; i < n; ++i) {
        tr_problem* p = probs[i];
        p->have_run = true;
        p->have_std = false;
        p->have_fixed = true;
        p->last_fixed = *opts;
        p->last_fixed.n_histories = n_histories[i];
        p->last_fixed.problem_tag = opts->problem_tag ^ (uint32_t)i;
        p->log_count = opts->want_event_log ? n_histories[i] : 0;
        if (stats) {
            tr_run_stats& S = stats[i];
            std::memset(&S, 0, sizeof(S));
            S.histories = n_histories[i];
            for (int k = 0; k < 8; ++k) {
                S.events_by_type[k] = cnt[16 * (size_t)i + k];
                S.final_by_type[k] = cnt[16 * (size_t)i + 8 + k];
                if (k != EV_SOURCE) S.events += S.events_by_type[k];
            }
            S.launches = 1;
            S.spills = hc.spills;
            S.refills = hc.refills;
            S.seconds = ms * 1e-3;
            S.transport_seconds = ms * 1e-3;
            S.used_blocks_per_sm = tune.blocks_per_sm;
            S.used_stash_slots = tune.stash_slots;
            S.used_remap_every = tune.remap_every;
        }
    }
    return TR_OK;
}

// ---------------------------------------------------------------------------
// readout
// ---------------------------------------------------------------------------
extern "C" size_t tr_tally_size(const tr_problem* pr, int32_t id)
{
    if (!pr) return 0;
    if (id == TR_TALLY_MESH) return (size_t)pr->dp.mesh_size;
    if (id == TR_TALLY_ENERGY) return (size_t)pr->dp.energy_size;
    if (id == TR_TALLY_SCALARS) return 3;
    if (id == TR_TALLY_TIME) return (size_t)pr->dp.n_tbins;
    return 0;
}

static tr_status copy_tally(const tr_problem* pr, int32_t id, double* out, size_t n, int32_t on_dev, bool sd)
{
    if (!pr || !out) return set_err(TR_ERR_INVALID, "NULL argument");
    DeviceGuard dg(pr->ctx.device);
    if (!pr->have_run) return set_err(TR_ERR_STATE, "no completed run");
    if (sd && !pr->have_std) return set_err(TR_ERR_STATE, "standard deviations come from power iteration only");
    const size_t want = tr_tally_size(pr, id);
    if (id < 0 || id > 3 || n != want) return set_err(TR_ERR_INVALID, "tally id or size mismatch");
    if (n == 0) return TR_OK;
    const double* src = id == TR_TALLY_MESH ? (sd ? pr->sd_mesh : pr->res_mesh)
                      : id == TR_TALLY_ENERGY ? (sd ? pr->sd_energy : pr->res_energy)
                      : id == TR_TALLY_TIME ? pr->res_time
                                              : (sd ? pr->sd_scal : pr->res_scal);
    TR_CUDA(cudaMemcpyAsync(out, src, n * 8, on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, pr->stream));
    TR_CUDA(cudaStreamSynchronize(pr->stream));
    return TR_OK;
}

extern "C" tr_status tr_tallies(const tr_problem* pr, int32_t id, double* out, size_t n, int32_t on_dev)
{
    return copy_tally(pr, id, out, n, on_dev, false);
}

extern "C" tr_status tr_tally_stddev(const tr_problem* pr, int32_t id, double* out, size_t n, int32_t on_dev)
{
    return copy_tally(pr, id, out, n, on_dev, true);
}

extern "C" tr_status tr_event_log(const tr_problem* pr, uint32_t* n_events, int32_t* final_cell, uint8_t* final_type,
                                  size_t n)
{
    if (!pr) return set_err(TR_ERR_INVALID, "problem is NULL");
    if (!pr->have_run || pr->log_count == 0) return set_err(TR_ERR_STATE, "no event log (set want_event_log)");
    DeviceGuard dg(pr->ctx.device);
    if (n != pr->log_count) return set_err(TR_ERR_INVALID, "n must equal the histories of the logged run");
    if (n_events) TR_CUDA(cudaMemcpyAsync(n_events, pr->log_n, n * 4, cudaMemcpyDeviceToHost, pr->stream));
    if (final_cell) TR_CUDA(cudaMemcpyAsync(final_cell, pr->log_cell, n * 4, cudaMemcpyDeviceToHost, pr->stream));
    if (final_type) TR_CUDA(cudaMemcpyAsync(final_type, pr->log_type, n, cudaMemcpyDeviceToHost, pr->stream));
    TR_CUDA(cudaStreamSynchronize(pr->stream));
    return TR_OK;
}

extern "C" const char* tr_last_error(void) { return g_err.c_str(); }

namespace tr {
void set_last_error(const char* msg) { g_err = msg; }

const DevProblem* problem_device_data(const tr_problem* pr, int* device, cudaStream_t* stream, int* sms)
{
    *device = pr->ctx.device;
    *stream = pr->stream;
    *sms = pr->sms;
    return &pr->dp;
}
}  // namespace tr

extern "C" uint64_t tr_kernel_launch_count(void) { return tr::launch_count(); }

extern "C" const char* tr_version(void) { return "tr 0.1 (sm_103a)"; }
