// tr_selftest.cu -- device-side checks of the arithmetic building blocks, for
// the test suite: the library's Philox-4x32-10 (Salmon et al., SC'11) beside a
// call of CUDA's own curand Philox4x32-10 on the same counters and keys; the
// table-driven logarithm as the transport kernels evaluate it; and the
// exponential ziggurat table the transport kernels read; the integer-pipe
// reciprocal, square root and division beside the IEEE hardware sequences;
// and an issue-rate probe of the arithmetic pipes for the roofline's ALU
// denominator.  The transport itself never calls these.
#include <curand_kernel.h>

#include <cstring>
#include <string>

#include "../../include/tr.h"
#include "tr_kernels.h"
#include "tr_softfp.cuh"

using namespace tr;

namespace tr {
void set_last_error(const char* msg);
const DevProblem* problem_device_data(const tr_problem* pr, int* device, cudaStream_t* stream, int* sms);
}  // namespace tr

namespace {

__global__ void k_philox_pair(const uint4* __restrict__ ctr, const uint2* __restrict__ key, size_t n, uint4* ours,
                              uint4* lib)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const uint4 c = ctr[i];
        const uint2 k = key[i];
        ours[i] = philox10(c.x, c.y, c.z, c.w, k.x, k.y);
        lib[i] = curand_Philox4x32_10(c, k);
    }
}

__global__ void k_log(const double* __restrict__ tab, const double* __restrict__ x, size_t n, double* out)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = tr_log(tab, x[i]);
}

// y1 ~ 2^115 / m for a mantissa m in [2^52, 2^53), within a few units: the
// FP32 seed and second-order fixed-point Newton step of sf_rcp
// (tr_softfp.cuh), which is exact (2^63) for m = 2^52.
__device__ __forceinline__ unsigned long long recip115(unsigned long long m)
{
    const float rf = __frcp_rn(__uint2float_rn((unsigned)(m >> 21)));
    const unsigned long long y0 = __float2uint_rz(rf * 0x1p61f);          // ~ 2^82 / m, <= 2^30
    const long long d = (long long)(0ull - m * y0);                        // 2^82 - m y0
    const long long c1 = __mul64hi(d, (long long)(y0 << 15));             // y0 2^33 t
    const long long c2 = __mul64hi(c1, d) >> 18;                           // y0 2^33 t^2
    return (y0 << 33) + (unsigned long long)(c1 + c2);
}

// Quotient a / b on the integer and FP32 pipes, correctly rounded (ties to
// even), for finite nonzero normal a and b with a normal result; anything
// else takes the hardware division.  Measured in the continuous-energy
// scatter's two divisions, it returned the same bits and ran 0.3 % slower
// than the IEEE division there, so the transport kernels do not use it; it
// stays here with its bitwise check.  With the mantissas ma, mb and k = 54 (ma >= mb) or 55, the
// quotient's 55 leading bits are Q = floor(ma 2^k / mb) in [2^54, 2^55): an
// estimate from the reciprocal 2^115 / mb is corrected to the exact Q by the
// remainder ma 2^k - Q mb (a signed 64-bit word), and Q's two low bits with
// the remainder's sign decide the rounding of the 53-bit mantissa Q / 4.
__device__ __forceinline__ double sf_div(double a, double b)
{
    const unsigned long long ba = (unsigned long long)__double_as_longlong(a);
    const unsigned long long bb = (unsigned long long)__double_as_longlong(b);
    const unsigned ea = (unsigned)(ba >> 52) & 0x7FFu, eb = (unsigned)(bb >> 52) & 0x7FFu;
    if (ea - 1u > 2045u || eb - 1u > 2045u) return __ddiv_rn(a, b);
    const unsigned long long ma = (ba & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    const unsigned long long mb = (bb & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    const unsigned lt = ma < mb ? 1u : 0u;
    const int E = (int)ea - (int)eb + 1023 - (int)lt;
    if (E < 1 || E > 2045) return __ddiv_rn(a, b);   // (2046 is reached only by rounding: kept out)
    const unsigned long long hi = __umul64hi(ma << 11, recip115(mb));   // (exactly 2^63 for mb = 2^52)
    unsigned long long q = hi >> (8u - lt);
    long long r = (long long)((ma << (54u + lt)) - q * mb);   // ma 2^k - q mb, small
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        if (r < 0) {
            q -= 1ull;
            r += (long long)mb;
        }
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        if (r >= (long long)mb) {
            q += 1ull;
            r -= (long long)mb;
        }
    }
    unsigned long long mant = q >> 2;
    const unsigned long long guard = (q >> 1) & 1ull;
    const bool sticky = (q & 1ull) || r != 0;
    mant += (guard && (sticky || (mant & 1ull))) ? 1ull : 0ull;
    unsigned long long eo = (unsigned long long)E;
    if (mant == 0x0020000000000000ull) {   // rounded up to 2^53
        mant = 0x0010000000000000ull;
        eo += 1ull;
    }
    return __longlong_as_double((long long)(((ba ^ bb) & 0x8000000000000000ull) | (eo << 52) |
                                            (mant - 0x0010000000000000ull)));
}

__global__ void k_softfp(int op, const double* __restrict__ x, size_t n, double* out)
{
    if (op >= 4) {   // quotients of the pairs (x[2i], x[2i + 1])
        for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n / 2; i += (size_t)gridDim.x * blockDim.x)
            out[i] = op == 4 ? sf_div(x[2 * i], x[2 * i + 1]) : __ddiv_rn(x[2 * i], x[2 * i + 1]);
        return;
    }
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double v = x[i];
        out[i] = op == 0 ? sf_rcp(v) : op == 1 ? __drcp_rn(v) : op == 2 ? sf_sqrt(v) : __dsqrt_rn(v);
    }
}

// Issue-rate probe of the arithmetic pipes, the roofline's denominators: eight
// independent dependency chains per thread.  OP 0..4: FP64 add, mul, fma,
// division, square root (IEEE, correctly rounded); 5: FP32 fma; 6: INT32
// multiply-add; 7: FP64 fma in only the first `lanes` lanes of each warp;
// 8 / 9: reciprocal, IEEE sequence / integer-pipe sf_rcp; 10 / 11: square
// root, IEEE sequence / sf_sqrt.
constexpr int PROBE_ITERS = 4096;

template <int OP>
__global__ void __launch_bounds__(256) k_issue(double* out, double a0, double b, int lanes)
{
    double x[8];
    float f[8];
    unsigned u[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        x[j] = a0 + 1e-3 * j + 1e-9 * threadIdx.x;
        f[j] = (float)x[j];
        u[j] = 2654435761u * (threadIdx.x + j);
    }
    const bool on = OP != 7 || (int)(threadIdx.x & 31) < lanes;
    if (on) {
#pragma unroll 4
        for (int i = 0; i < PROBE_ITERS; ++i) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (OP == 0) x[j] = __dadd_rn(x[j], b);
                if (OP == 1) x[j] = __dmul_rn(x[j], b);
                if (OP == 2 || OP == 7) x[j] = __fma_rn(x[j], b, b);
                if (OP == 3) x[j] = __ddiv_rn(b, x[j]);
                if (OP == 4) x[j] = __dsqrt_rn(__dadd_rn(x[j], b));
                if (OP == 5) f[j] = __fmaf_rn(f[j], (float)b, (float)b);
                if (OP == 6) u[j] = u[j] * u[j] + 12345u;   // not affine: the chain cannot be folded
                if (OP == 8) x[j] = __drcp_rn(x[j]);
                if (OP == 9) x[j] = sf_rcp(x[j]);
                if (OP == 10) x[j] = __dsqrt_rn(__dadd_rn(x[j], b));
                if (OP == 11) x[j] = sf_sqrt(__dadd_rn(x[j], b));
            }
        }
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j] + (double)f[j] + (double)u[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

tr_status fail(tr_status s, const std::string& m)
{
    tr::set_last_error(m.c_str());
    return s;
}

// Device scratch for one call (a diagnostic: allocation is fine here).
struct Scratch {
    void* p = nullptr;
    ~Scratch()
    {
        if (p) cudaFree(p);
    }
};

#define ST_CUDA(call)                                                                          \
    do {                                                                                       \
        const cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) return fail(TR_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

}  // namespace

extern "C" tr_status tr_selftest_philox(const uint32_t* ctr, const uint32_t* key, size_t n, uint32_t* ours,
                                        uint32_t* curand_out)
{
    if (!ctr || !key || !ours || !curand_out) return fail(TR_ERR_INVALID, "NULL argument");
    if (n == 0) return TR_OK;
    if (n > (1u << 26)) return fail(TR_ERR_INVALID, "n must be at most 2^26");
    Scratch s;
    const size_t b4 = n * sizeof(uint4), b2 = n * sizeof(uint2);
    ST_CUDA(cudaMalloc(&s.p, 3 * b4 + b2));
    uint4* d_ctr = static_cast<uint4*>(s.p);
    uint4* d_ours = d_ctr + n;
    uint4* d_lib = d_ours + n;
    uint2* d_key = reinterpret_cast<uint2*>(d_lib + n);
    ST_CUDA(cudaMemcpy(d_ctr, ctr, b4, cudaMemcpyHostToDevice));
    ST_CUDA(cudaMemcpy(d_key, key, b2, cudaMemcpyHostToDevice));
    count_launches(1);
    k_philox_pair<<<(unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256>>>(d_ctr, d_key, n, d_ours,
                                                                                        d_lib);
    ST_CUDA(cudaGetLastError());
    ST_CUDA(cudaMemcpy(ours, d_ours, b4, cudaMemcpyDeviceToHost));
    ST_CUDA(cudaMemcpy(curand_out, d_lib, b4, cudaMemcpyDeviceToHost));
    return TR_OK;
}

extern "C" tr_status tr_selftest_log(const tr_problem* problem, const double* x, size_t n, double* out)
{
    if (!problem || !x || !out) return fail(TR_ERR_INVALID, "NULL argument");
    if (n == 0) return TR_OK;
    if (n > (1u << 26)) return fail(TR_ERR_INVALID, "n must be at most 2^26");
    for (size_t i = 0; i < n; ++i) {
        uint64_t b;
        std::memcpy(&b, &x[i], 8);
        const unsigned e = (unsigned)((b >> 52) & 0x7FFu);
        if ((b >> 63) || e == 0 || e == 0x7FF)
            return fail(TR_ERR_INVALID, "inputs must be positive, finite and normal");
    }
    int dev = 0, sms = 0;
    cudaStream_t st = nullptr;
    const DevProblem* P = problem_device_data(problem, &dev, &st, &sms);
    DeviceGuard dg(dev);
    Scratch s;
    ST_CUDA(cudaMalloc(&s.p, 2 * n * sizeof(double)));
    double* d_x = static_cast<double*>(s.p);
    double* d_out = d_x + n;
    ST_CUDA(cudaMemcpyAsync(d_x, x, n * 8, cudaMemcpyHostToDevice, st));
    count_launches(1);
    k_log<<<(unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, st>>>(P->log_tab, d_x, n, d_out);
    ST_CUDA(cudaGetLastError());
    ST_CUDA(cudaMemcpyAsync(out, d_out, n * 8, cudaMemcpyDeviceToHost, st));
    ST_CUDA(cudaStreamSynchronize(st));
    return TR_OK;
}

extern "C" tr_status tr_selftest_zig_table(const tr_problem* problem, double* out)
{
    if (!problem || !out) return fail(TR_ERR_INVALID, "NULL argument");
    int dev = 0, sms = 0;
    cudaStream_t st = nullptr;
    const DevProblem* P = problem_device_data(problem, &dev, &st, &sms);
    DeviceGuard dg(dev);
    ST_CUDA(cudaMemcpyAsync(out, P->zig_tab, 4 * ZIG_N * sizeof(double), cudaMemcpyDeviceToHost, st));
    ST_CUDA(cudaStreamSynchronize(st));
    return TR_OK;
}

extern "C" tr_status tr_selftest_issue_rate(int32_t op, int32_t lanes, double* per_second)
{
    if (!per_second || op < 0 || op > 11 || (op == 7 && (lanes < 1 || lanes > 32)))
        return fail(TR_ERR_INVALID, "op must be 0..11 (lanes 1..32 for op 7)");
    int dev = 0, sms = 0;
    ST_CUDA(cudaGetDevice(&dev));
    ST_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int threads = 256, blocks = sms * 8;
    Scratch s;
    ST_CUDA(cudaMalloc(&s.p, (size_t)threads * blocks * sizeof(double)));
    double* d = static_cast<double*>(s.p);
    cudaEvent_t e0, e1;
    ST_CUDA(cudaEventCreate(&e0));
    ST_CUDA(cudaEventCreate(&e1));
    const double b = op == 0 ? 1e-9 : op == 1 ? 1.0000001 : op == 3 ? 1.5 : (op == 4 || op >= 10) ? 0.25 : 0.5;
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {   // the second launch is timed
        cudaEventRecord(e0);
        count_launches(1);
        switch (op) {
        case 0: k_issue<0><<<blocks, threads>>>(d, 1.0, b, 32); break;
        case 1: k_issue<1><<<blocks, threads>>>(d, 1.0, b, 32); break;
        case 2: k_issue<2><<<blocks, threads>>>(d, 1.0, b, 32); break;
        case 3: k_issue<3><<<blocks, threads>>>(d, 1.0, b, 32); break;
        case 4: k_issue<4><<<blocks, threads>>>(d, 1.0, b, 32); break;
        case 5: k_issue<5><<<blocks, threads>>>(d, 1.0, b, 32); break;
        case 6: k_issue<6><<<blocks, threads>>>(d, 1.0, b, 32); break;
        case 7: k_issue<7><<<blocks, threads>>>(d, 1.0, b, lanes); break;
        case 8: k_issue<8><<<blocks, threads>>>(d, 1.0, b, 32); break;
        case 9: k_issue<9><<<blocks, threads>>>(d, 1.0, b, 32); break;
        case 10: k_issue<10><<<blocks, threads>>>(d, 1.0, b, 32); break;
        default: k_issue<11><<<blocks, threads>>>(d, 1.0, b, 32); break;
        }
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ST_CUDA(cudaGetLastError());
    const double chains = (double)threads * blocks * 8.0 * PROBE_ITERS;
    // op 7: FP64 warp instructions per second (one per warp per chain step)
    *per_second = (op == 7 ? chains / 32.0 : chains) / (ms * 1e-3);
    return TR_OK;
}

extern "C" tr_status tr_selftest_softfp(int32_t op, const double* x, size_t n, double* out)
{
    if (!x || !out || op < 0 || op > 5) return fail(TR_ERR_INVALID, "op must be 0..5 and x, out non-NULL");
    if (op >= 4 && (n & 1)) return fail(TR_ERR_INVALID, "ops 4 and 5 take pairs: n must be even");
    if (n == 0) return TR_OK;
    if (n > (1u << 26)) return fail(TR_ERR_INVALID, "n must be at most 2^26");
    Scratch s;
    ST_CUDA(cudaMalloc(&s.p, 2 * n * sizeof(double)));
    double* d_x = static_cast<double*>(s.p);
    double* d_out = d_x + n;
    ST_CUDA(cudaMemcpy(d_x, x, n * 8, cudaMemcpyHostToDevice));
    count_launches(1);
    k_softfp<<<(unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256>>>(op, d_x, n, d_out);
    ST_CUDA(cudaGetLastError());
    ST_CUDA(cudaMemcpy(out, d_out, (op >= 4 ? n / 2 : n) * 8, cudaMemcpyDeviceToHost));
    return TR_OK;
}
