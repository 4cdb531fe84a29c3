// tr_selftest.cu -- device-side checks of the arithmetic building blocks, for
// the test suite: the library's Philox-4x32-10 (Salmon et al., SC'11) beside a
// call of CUDA's own curand Philox4x32-10 on the same counters and keys; the
// table-driven logarithm as the transport kernels evaluate it; and the
// exponential ziggurat table the transport kernels read.  The transport
// itself never calls these.
#include <curand_kernel.h>

#include <cstring>
#include <string>

#include "../../include/tr.h"
#include "tr_kernels.h"

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
