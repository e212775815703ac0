// Streaming probe (diagnostic, not part of the library): per-CTA throughput of
// 1-D bulk copies (cp.async.bulk into a shared-memory ring with mbarrier
// completion, no compute) for several chunk sizes and ring depths, against
// plain 16-byte loads, with 64 and 152 CTAs.
#include <cstdio>
#include <cuda_runtime.h>
#include <stdint.h>
__device__ inline unsigned sa(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__global__ void tma_stream(const char* src, long long per_cta, int chb, int nbuf, float* out) {
  extern __shared__ __align__(128) unsigned char sm[];
  uint64_t* bar = (uint64_t*)(sm + (size_t)nbuf * chb);
  const char* base = src + per_cta * blockIdx.x;
  int nch = (int)(per_cta / chb);
  if (threadIdx.x == 0) {
    for (int s = 0; s < nbuf; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sa(&bar[s])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  float acc = 0.f;
  if (threadIdx.x == 0)
    for (int c = 0; c < nch && c < nbuf; ++c) {
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(&bar[c])), "r"(chb) : "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(sa(sm + (size_t)c * chb)), "l"(base + (long long)c * chb), "r"(chb), "r"(sa(&bar[c])) : "memory");
    }
  for (int c = 0; c < nch; ++c) {
    int slot = c % nbuf;
    unsigned par = (c / nbuf) & 1;
    if (threadIdx.x == 0) {
      for (long long i = 0; i < (1LL << 24); ++i) {
        unsigned ok;
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0,1,0,p; }" : "=r"(ok) : "r"(sa(&bar[slot])), "r"(par) : "memory");
        if (ok) break;
      }
    }
    __syncthreads();
    acc += ((const float*)(sm + (size_t)slot * chb))[threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0 && c + nbuf < nch) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(&bar[slot])), "r"(chb) : "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(sa(sm + (size_t)slot * chb)), "l"(base + (long long)(c + nbuf) * chb), "r"(chb), "r"(sa(&bar[slot])) : "memory");
    }
  }
  if (acc == 1234.5f) out[0] = acc;
}
__global__ void ldg_stream(const float4* src, long long per_cta_f4, float* out) {
  const float4* base = src + per_cta_f4 * blockIdx.x;
  float acc = 0.f;
  for (long long i = threadIdx.x; i < per_cta_f4; i += blockDim.x * 8) {
    float4 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) { long long j = i + (long long)u * blockDim.x; v[u] = j < per_cta_f4 ? base[j] : make_float4(0,0,0,0); }
#pragma unroll
    for (int u = 0; u < 8; ++u) acc += v[u].x + v[u].y + v[u].z + v[u].w;
  }
  if (acc == 1234.5f) out[0] = acc;
}
int main() {
  long long per_cta = 24LL << 20;  // 24 MiB per CTA
  int maxcta = 152;
  char* src; cudaMalloc(&src, per_cta * maxcta); cudaMemset(src, 0, per_cta * maxcta);
  float* out; cudaMalloc(&out, 64);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1); float ms;
  cudaFuncSetAttribute(tma_stream, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  int ctas[2] = {64, 152};
  for (int ci = 0; ci < 2; ++ci) {
    int n = ctas[ci];
    int cfg[][2] = {{32768, 4}, {24576, 6}, {16384, 8}, {8192, 16}, {49152, 4}, {4096, 32}};
    for (auto& c : cfg) {
      size_t smem = (size_t)c[0] * c[1] + 8 * c[1];
      for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0); tma_stream<<<n, 512, smem>>>(src, per_cta, c[0], c[1], out); cudaEventRecord(e1); cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep) printf("tma ctas %3d chunk %6d nbuf %2d: %7.1f GB/s total, %6.1f GB/s per CTA\n", n, c[0], c[1], per_cta * n / ms / 1e6, per_cta / ms / 1e6);
      }
    }
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(e0); ldg_stream<<<n, 512>>>((const float4*)src, per_cta / 16, out); cudaEventRecord(e1); cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep) printf("ldg ctas %3d 512 thr x8 float4: %7.1f GB/s total, %6.1f GB/s per CTA\n", n, per_cta * n / ms / 1e6, per_cta / ms / 1e6);
    }
  }
  printf("status %s\n", cudaGetErrorString(cudaDeviceSynchronize()));
}
