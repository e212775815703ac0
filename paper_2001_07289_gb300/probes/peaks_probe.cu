// Throughput probe (diagnostic, not part of the library): FP64 FMA, FP32 FMA,
// FP64 mma.sync (dependent chain) and a plain HBM read, on the current GPU.
#include <cstdio>
#include <cuda_runtime.h>
template <typename T>
__global__ void fma_chain(T* out, int iters, T a, T b) {
  T x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
__global__ void dmma_chain(double* out, int iters) {
  double a = 1.0001, b = 0.9999, c0 = 0, c1 = 0;
  double d0, d1;
  for (int i = 0; i < iters; ++i) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%4,%5};"
                 : "=d"(d0), "=d"(d1) : "d"(a), "d"(b), "d"(c0), "d"(c1));
    c0 = d0 * 1e-30; c1 = d1 * 1e-30;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = c0 + c1;
}
__global__ void readbw(const double2* __restrict__ in, double* out, long long n) {
  double s = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double2 v = in[i]; s += v.x + v.y;
  }
  if (s == 12345.0) out[0] = s;
}
int main() {
  int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  double* out; cudaMalloc(&out, 1 << 26);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1); float ms;
  int blocks = sms * 8, threads = 256, iters = 4096;
  for (int rep = 0; rep < 2; ++rep) {
    cudaEventRecord(e0); fma_chain<double><<<blocks, threads>>>(out, iters, 1.0000001, 1e-9); cudaEventRecord(e1); cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    printf("fp64 fma: %.3f TFLOP/s\n", 2.0 * 8 * iters * (double)blocks * threads / ms / 1e9);
    cudaEventRecord(e0); fma_chain<float><<<blocks, threads>>>((float*)out, iters * 16, 1.0000001f, 1e-9f); cudaEventRecord(e1); cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    printf("fp32 fma: %.3f TFLOP/s\n", 2.0 * 8 * iters * 16 * (double)blocks * threads / ms / 1e9);
    cudaEventRecord(e0); dmma_chain<<<blocks, threads>>>(out, iters); cudaEventRecord(e1); cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    printf("fp64 dmma (dependent chain per warp): %.3f TFLOP/s\n", 2.0 * 8 * 8 * 4 * iters * (double)blocks * threads / 32 / ms / 1e9);
  }
  long long n = (1LL << 31) / 32;  // 2 GiB of double2
  double2* in; if (cudaMalloc(&in, n * 16) == cudaSuccess) {
    cudaMemset(in, 0, n * 16);
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0); readbw<<<sms * 8, 512>>>(in, out, n); cudaEventRecord(e1); cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1); printf("hbm read: %.1f GB/s\n", n * 16.0 / ms / 1e6);
    }
  }
  printf("status %s\n", cudaGetErrorString(cudaDeviceSynchronize()));
  return 0;
}
