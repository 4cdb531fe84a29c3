// fp64_rate.cu -- issue-rate probe for the roofline peak: FP64 add / mul / fma /
// div / sqrt, FP32 fma and INT32 imad thread-operations per clock per SM,
// eight independent chains per thread, 8 blocks of 256 threads per SM.
// Build: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o fp64_rate fp64_rate.cu
#include <cstdio>
#include <cuda_runtime.h>
#define ITERS 4096
template<int OP> __global__ void k(double* out, double a0, double b0) {
  double x0 = a0 + threadIdx.x * 1e-9, x1 = x0 + 1e-3, x2 = x0 + 2e-3, x3 = x0 + 3e-3;
  double x4 = x0 + 4e-3, x5 = x0 + 5e-3, x6 = x0 + 6e-3, x7 = x0 + 7e-3;
  const double b = b0;
  #pragma unroll 4
  for (int i = 0; i < ITERS; ++i) {
    if (OP == 0) { x0 = __dadd_rn(x0, b); x1 = __dadd_rn(x1, b); x2 = __dadd_rn(x2, b); x3 = __dadd_rn(x3, b);
                   x4 = __dadd_rn(x4, b); x5 = __dadd_rn(x5, b); x6 = __dadd_rn(x6, b); x7 = __dadd_rn(x7, b); }
    if (OP == 1) { x0 = __dmul_rn(x0, b); x1 = __dmul_rn(x1, b); x2 = __dmul_rn(x2, b); x3 = __dmul_rn(x3, b);
                   x4 = __dmul_rn(x4, b); x5 = __dmul_rn(x5, b); x6 = __dmul_rn(x6, b); x7 = __dmul_rn(x7, b); }
    if (OP == 2) { x0 = __fma_rn(x0, b, b); x1 = __fma_rn(x1, b, b); x2 = __fma_rn(x2, b, b); x3 = __fma_rn(x3, b, b);
                   x4 = __fma_rn(x4, b, b); x5 = __fma_rn(x5, b, b); x6 = __fma_rn(x6, b, b); x7 = __fma_rn(x7, b, b); }
    if (OP == 3) { x0 = __ddiv_rn(b, x0); x1 = __ddiv_rn(b, x1); x2 = __ddiv_rn(b, x2); x3 = __ddiv_rn(b, x3);
                   x4 = __ddiv_rn(b, x4); x5 = __ddiv_rn(b, x5); x6 = __ddiv_rn(b, x6); x7 = __ddiv_rn(b, x7); }
    if (OP == 4) { x0 = __dsqrt_rn(x0 + b); x1 = __dsqrt_rn(x1 + b); x2 = __dsqrt_rn(x2 + b); x3 = __dsqrt_rn(x3 + b);
                   x4 = __dsqrt_rn(x4 + b); x5 = __dsqrt_rn(x5 + b); x6 = __dsqrt_rn(x6 + b); x7 = __dsqrt_rn(x7 + b); }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
__global__ void kf(float* out, float a0, float b) {
  float x[8]; for (int j = 0; j < 8; ++j) x[j] = a0 + j * 1e-3f + threadIdx.x * 1e-7f;
  #pragma unroll 4
  for (int i = 0; i < ITERS * 8; ++i) {
    #pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = __fmaf_rn(x[j], b, b);
  }
  float s = 0; for (int j = 0; j < 8; ++j) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void ki(unsigned* out, unsigned a0, unsigned b) {
  unsigned x[8]; for (int j = 0; j < 8; ++j) x[j] = a0 + j + threadIdx.x;
  #pragma unroll 4
  for (int i = 0; i < ITERS * 8; ++i) {
    #pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = x[j] * b + b;
  }
  unsigned s = 0; for (int j = 0; j < 8; ++j) s ^= x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void kh(unsigned* out, unsigned a0, unsigned b) {
  unsigned x[8]; for (int j = 0; j < 8; ++j) x[j] = a0 + j + threadIdx.x;
  #pragma unroll 4
  for (int i = 0; i < ITERS * 8; ++i) {
    #pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = __umulhi(x[j], b) ^ b;
  }
  unsigned s = 0; for (int j = 0; j < 8; ++j) s ^= x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
// DFMA chains executed by only the first K lanes of every warp: if the time
// does not fall with K, an FP64 warp instruction costs the same pipe time
// however many lanes are active.
__global__ void kpart(double* out, double a0, double b, int K) {
  double x[8]; for (int j = 0; j < 8; ++j) x[j] = a0 + j * 1e-3 + threadIdx.x * 1e-9;
  if ((int)(threadIdx.x & 31) < K) {
    #pragma unroll 4
    for (int i = 0; i < ITERS; ++i) {
      #pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = __fma_rn(x[j], b, b);
    }
  }
  double s = 0; for (int j = 0; j < 8; ++j) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
int main() {
  int dev = 0; cudaDeviceProp p; cudaGetDeviceProperties(&p, dev);
  int sms = p.multiProcessorCount; int clk = 0; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
  printf("name=%s sms=%d clock_khz=%d cc=%d.%d\n", p.name, sms, clk, p.major, p.minor);
  int threads = 256, blocks = sms * 8; size_t n = (size_t)threads * blocks;
  double* d; cudaMalloc(&d, n * 8); cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  const char* names[5] = {"dadd", "dmul", "dfma", "ddiv", "dsqrt"};
  for (int op = 0; op < 5; ++op) {
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(e0);
      if (op == 0) k<0><<<blocks, threads>>>(d, 1.0, 1e-9);
      if (op == 1) k<1><<<blocks, threads>>>(d, 1.0, 1.0000001);
      if (op == 2) k<2><<<blocks, threads>>>(d, 1.0, 0.5);
      if (op == 3) k<3><<<blocks, threads>>>(d, 1.0, 1.5);
      if (op == 4) k<4><<<blocks, threads>>>(d, 1.0, 0.25);
      cudaEventRecord(e1); cudaEventSynchronize(e1);
      float ms; cudaEventElapsedTime(&ms, e0, e1);
      double ops = (double)n * ITERS * 8;
      if (rep == 1) printf("%s: %.3f ms, %.3e ops/s, %.3f ops/clk/SM @%.0fMHz(nominal)\n", names[op], ms, ops / (ms * 1e-3),
             ops / (ms * 1e-3) / sms / (clk * 1e3), clk / 1e3);
    }
  }
  for (int rep = 0; rep < 2; ++rep) {
    cudaEventRecord(e0); kf<<<blocks, threads>>>((float*)d, 1.0f, 0.5f); cudaEventRecord(e1); cudaEventSynchronize(e1);
    float ms; cudaEventElapsedTime(&ms, e0, e1); double ops = (double)n * ITERS * 64;
    if (rep) printf("ffma: %.3f ms, %.3e ops/s, %.3f ops/clk/SM\n", ms, ops / (ms * 1e-3), ops / (ms * 1e-3) / sms / (clk * 1e3));
  }
  for (int rep = 0; rep < 2; ++rep) {
    cudaEventRecord(e0); ki<<<blocks, threads>>>((unsigned*)d, 1u, 2654435761u); cudaEventRecord(e1); cudaEventSynchronize(e1);
    float ms; cudaEventElapsedTime(&ms, e0, e1); double ops = (double)n * ITERS * 64;
    if (rep) printf("imad: %.3f ms, %.3e ops/s, %.3f ops/clk/SM\n", ms, ops / (ms * 1e-3), ops / (ms * 1e-3) / sms / (clk * 1e3));
  }
  for (int rep = 0; rep < 2; ++rep) {
    cudaEventRecord(e0); kh<<<blocks, threads>>>((unsigned*)d, 1u, 2654435761u); cudaEventRecord(e1); cudaEventSynchronize(e1);
    float ms; cudaEventElapsedTime(&ms, e0, e1); double ops = (double)n * ITERS * 64;
    if (rep) printf("umulhi+xor: %.3f ms, %.3e pairs/s, %.3f pairs/clk/SM\n", ms, ops / (ms * 1e-3), ops / (ms * 1e-3) / sms / (clk * 1e3));
  }
  for (int K : {32, 16, 8, 1}) {
    float ms = 0;
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(e0); kpart<<<blocks, threads>>>(d, 1.0, 0.5, K); cudaEventRecord(e1); cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
    }
    double winst = (double)n / 32 * ITERS * 8;
    printf("dfma with %2d active lanes/warp: %.3f ms, %.3e warp-inst/s, %.3f warp-inst/clk/SM\n", K, ms,
           winst / (ms * 1e-3), winst / (ms * 1e-3) / sms / (clk * 1e3));
  }
  cudaError_t err = cudaGetLastError(); printf("err=%s\n", cudaGetErrorString(err));
  cudaFree(d); return err == cudaSuccess ? 0 : 1;
}
