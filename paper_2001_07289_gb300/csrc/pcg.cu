// PCG vector kernels (FP64) with deterministic reductions: every dot product
// is accumulated into RED_BLOCKS fixed per-block partials and summed by one
// block in a fixed order, so repeated runs are bitwise identical.  The CG
// scalars and the stopping test (the residual 2-norm rule of Section 5) live
// on the device, so a PCG loop needs no host round trip per iteration.
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
  pdl_enter();
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s = fma(a[i], b[i], s);
  block_partial_p(s, partial);
}

void launch_dot(const double* a, const double* b, long long n, double* partial, cudaStream_t st) {
  BDDC_COUNT(1);
  launch_pdl(k_dot, dim3(RED_BLOCKS), dim3(256), 0, st, a, b, n, partial);
}

// r.z and r.zp in one pass: partials of the first in partial[0, RED_BLOCKS),
// of the second in partial[RED_BLOCKS, 2 RED_BLOCKS)
__global__ void k_dot2(const double* __restrict__ r, const double* __restrict__ z, const double* __restrict__ zp,
                       long long n, double* __restrict__ partial) {
  pdl_enter();
  double s = 0.0, t = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double ri = r[i];
    s = fma(ri, z[i], s);
    t = fma(ri, zp[i], t);
  }
  block_partial_p(s, partial);
  __syncthreads();
  block_partial_p(t, partial + RED_BLOCKS);
}

void launch_dot2(const double* r, const double* z, const double* zp, long long n, double* partial, cudaStream_t st) {
  BDDC_COUNT(1);
  launch_pdl(k_dot2, dim3(RED_BLOCKS), dim3(256), 0, st, r, z, zp, n, partial);
}

// One block sums the partials in a fixed order and updates the CG scalars and
// the control block ctl = {it, continue, converged, breakdown}.
//   op 4 (start):  bb = sum; threshold rtol ||b||_2 (Section 5 stopping rule),
//                  it = 0, converged iff b = 0, continue iff not converged.
//   op 3 (beta):   rz_new = sum; beta = 0 on the first iteration, else
//                  rz_new / rz (hist[it - 1] = beta); rz = rz_new.
//   op 5 (flexible beta): as op 3 with beta = (rz_new - r.z_prev) / rz, where
//                  r.z_prev is the sum of the second partial array.
//   op 1 (alpha):  pq = sum; alpha = rz / pq (hist[it] = alpha); breakdown if
//                  pq <= 0 or alpha is not finite.
//   op 2 (test):   rr = sum; ++it; converged iff ||r||_2 <= threshold and no
//                  breakdown; continue iff neither and it < maxit.
// With use_cond the continue flag also sets the condition of the enclosing
// graph's while node, which is what ends a PCG loop captured in a graph: it
// grows by one per body, so the loop runs at most maxit times.
__device__ inline double fixed_order_sum(const double* __restrict__ partial, double* ws) {
  double v = 0.0;
  for (int i = threadIdx.x; i < RED_BLOCKS; i += blockDim.x) v += partial[i];
  v = wsum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) ws[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
  __syncthreads();
  return s;
}

__global__ void k_finalize(const double* __restrict__ partial, double* scal, int op, double* hist, int* ctl,
                           int maxit, double rtol, cudaGraphConditionalHandle cond, int use_cond) {
  pdl_enter();
  __shared__ double ws[32];
  const double s = fixed_order_sum(partial, ws);
  // op 5: the second sum, r_{k+1}.z_k
  const double s2 = op == 5 ? fixed_order_sum(partial + RED_BLOCKS, ws) : 0.0;
  if (threadIdx.x == 0) {
    int cont = -1;
    switch (op) {
      case 4: {
        scal[6] = s;
        scal[7] = rtol * sqrt(s);
        const int conv = s == 0.0;
        ctl[0] = 0;
        ctl[2] = conv;
        ctl[3] = 0;
        cont = (!conv && maxit > 0) ? 1 : 0;
        break;
      }
      case 3: {
        scal[4] = s;
        const int it = ctl[0];
        double b = 0.0;
        if (it > 0) {
          b = s / scal[0];
          if (!isfinite(b)) { ctl[3] = 1; b = 0.0; }
          if (hist) hist[it - 1] = b;
        }
        scal[5] = b;
        scal[0] = s;
        break;
      }
      case 5: {
        // Polak-Ribiere (flexible) beta: r_{k+1}.(z_{k+1} - z_k) / r_k.z_k
        scal[4] = s;
        const int it = ctl[0];
        double b = 0.0;
        if (it > 0) {
          b = (s - s2) / scal[0];
          if (!isfinite(b)) { ctl[3] = 1; b = 0.0; }
          if (hist) hist[it - 1] = b;
        }
        scal[5] = b;
        scal[0] = s;
        break;
      }
      case 1: {
        scal[1] = s;
        double a = scal[0] / s;
        if (!(s > 0.0) || !isfinite(a)) { ctl[3] = 1; a = 0.0; }
        scal[2] = a;
        if (hist) hist[ctl[0]] = a;
        break;
      }
      case 2: {
        scal[3] = s;
        const int it = ctl[0] + 1;
        ctl[0] = it;
        const int brk = ctl[3];
        const int conv = !brk && sqrt(s) <= scal[7];
        ctl[2] = conv;
        cont = (!brk && !conv && it < maxit) ? 1 : 0;
        break;
      }
    }
    if (cont >= 0) {
      ctl[1] = cont;
      if (use_cond) cudaGraphSetConditional(cond, (unsigned)cont);
    }
  }
}

void launch_finalize(const double* partial, double* scal, int op, double* hist, int* ctl, int maxit, double rtol,
                     const cudaGraphConditionalHandle* cond, cudaStream_t st) {
  BDDC_COUNT(1);
  launch_pdl(k_finalize, dim3(1), dim3(256), 0, st, partial, scal, op, hist, ctl, maxit, rtol,
             cond ? *cond : (cudaGraphConditionalHandle)0, cond ? 1 : 0);
}

// Sets the condition of a graph's while node from ctl[1] (the continue flag).
__global__ void k_loop_condition(const int* ctl, cudaGraphConditionalHandle cond) {
  pdl_enter();
  if (threadIdx.x == 0) cudaGraphSetConditional(cond, ctl[1] ? 1u : 0u);
}

void launch_loop_condition(const int* ctl, cudaGraphConditionalHandle cond, cudaStream_t st) {
  BDDC_COUNT(1);
  launch_pdl(k_loop_condition, dim3(1), dim3(32), 0, st, ctl, cond);
}

// x += alpha p; r -= alpha q; partials of r.r
__global__ void k_update_xr(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                            const double* __restrict__ q, const double* __restrict__ scal, long long n,
                            double* __restrict__ partial) {
  pdl_enter();
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
  launch_pdl(k_update_xr, dim3(RED_BLOCKS), dim3(256), 0, st, x, r, p, q, scal, n, partial);
}

// p = z + beta p
__global__ void k_update_p(double* __restrict__ p, const double* __restrict__ z, const double* __restrict__ scal,
                           long long n) {
  pdl_enter();
  const double b = scal[5];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = fma(b, p[i], z[i]);
}

void launch_update_p(double* p, const double* z, const double* scal, long long n, cudaStream_t st) {
  BDDC_COUNT(1);
  launch_pdl(k_update_p, dim3(RED_BLOCKS), dim3(256), 0, st, p, z, scal, n);
}

// p = z + beta p and zp = z (the flexible recurrence keeps the last z)
__global__ void k_update_p_keep(double* __restrict__ p, double* __restrict__ zp, const double* __restrict__ z,
                                const double* __restrict__ scal, long long n) {
  pdl_enter();
  const double b = scal[5];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double zi = z[i];
    p[i] = fma(b, p[i], zi);
    zp[i] = zi;
  }
}

void launch_update_p_keep(double* p, double* zp, const double* z, const double* scal, long long n, cudaStream_t st) {
  BDDC_COUNT(1);
  launch_pdl(k_update_p_keep, dim3(RED_BLOCKS), dim3(256), 0, st, p, zp, z, scal, n);
}

}  // namespace bddc
