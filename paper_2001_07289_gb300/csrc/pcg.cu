// PCG vector kernels (FP64) with deterministic reductions: every dot product
// is accumulated into RED_BLOCKS fixed per-block partials and summed by one
// block in a fixed order, so repeated runs are bitwise identical.  The CG
// scalars live on the device; only ||r||^2 crosses to the host per iteration
// (the stopping test on the residual 2-norm of Section 5).
#include "common.cuh"
#include "kernels.h"

namespace bddc {

__device__ inline double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ inline void block_partial_p(double v, double* partial) {
  __shared__ double ws[32];
  v = wsum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) ws[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = (lane < (int)(blockDim.x >> 5)) ? ws[lane] : 0.0;
    v = wsum(v);
    if (lane == 0) partial[blockIdx.x] = v;
  }
}

__global__ void k_dot(const double* __restrict__ a, const double* __restrict__ b, long long n,
                      double* __restrict__ partial) {
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s = fma(a[i], b[i], s);
  block_partial_p(s, partial);
}

void launch_dot(const double* a, const double* b, long long n, double* partial, cudaStream_t st) {
  BDDC_COUNT(1);
  k_dot<<<RED_BLOCKS, 256, 0, st>>>(a, b, n, partial);
}

// op: 0 rz = sum (initial r.z);  1 pq -> alpha = rz/pq (hist[it] = alpha),
//     flag if pq <= 0 or not finite;  2 rr = sum;  3 rz_new -> beta =
//     rz_new/rz (hist[it] = beta), rz = rz_new;  4 bb = sum.
__global__ void k_finalize(const double* __restrict__ partial, double* scal, int op, double* hist, int it,
                           int* flag) {
  __shared__ double ws[32];
  double v = 0.0;
  for (int i = threadIdx.x; i < RED_BLOCKS; i += blockDim.x) v += partial[i];
  v = wsum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) ws[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
    switch (op) {
      case 0: scal[0] = s; break;
      case 1: {
        scal[1] = s;
        double a = scal[0] / s;
        if (!(s > 0.0) || !isfinite(a)) { *flag = 1; a = 0.0; }
        scal[2] = a;
        if (hist) hist[it] = a;
        break;
      }
      case 2: scal[3] = s; break;
      case 3: {
        scal[4] = s;
        double b = s / scal[0];
        if (!isfinite(b)) { *flag = 1; b = 0.0; }
        scal[5] = b;
        scal[0] = s;
        if (hist) hist[it] = b;
        break;
      }
      case 4: scal[6] = s; break;
    }
  }
}

void launch_finalize(const double* partial, double* scal, int op, double* hist, int it, int* flag, cudaStream_t st) {
  BDDC_COUNT(1);
  k_finalize<<<1, 256, 0, st>>>(partial, scal, op, hist, it, flag);
}

// x += alpha p; r -= alpha q; partials of r.r
__global__ void k_update_xr(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                            const double* __restrict__ q, const double* __restrict__ scal, long long n,
                            double* __restrict__ partial) {
  const double a = scal[2];
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    x[i] = fma(a, p[i], x[i]);
    double ri = fma(-a, q[i], r[i]);
    r[i] = ri;
    s = fma(ri, ri, s);
  }
  block_partial_p(s, partial);
}

void launch_update_xr(double* x, double* r, const double* p, const double* q, const double* scal, long long n,
                      double* partial, cudaStream_t st) {
  BDDC_COUNT(1);
  k_update_xr<<<RED_BLOCKS, 256, 0, st>>>(x, r, p, q, scal, n, partial);
}

// p = z + beta p
__global__ void k_update_p(double* __restrict__ p, const double* __restrict__ z, const double* __restrict__ scal,
                           long long n) {
  const double b = scal[5];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = fma(b, p[i], z[i]);
}

void launch_update_p(double* p, const double* z, const double* scal, long long n, cudaStream_t st) {
  BDDC_COUNT(1);
  k_update_p<<<RED_BLOCKS, 256, 0, st>>>(p, z, scal, n);
}

}  // namespace bddc
