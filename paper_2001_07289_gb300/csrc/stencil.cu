// Grid kernels on the global node vector (FP64): the matrix-free Q1 operator,
// the adjoint gradient, the weighted injection E onto Gamma and input checks.
//
// Operator (Section 2, eq. weakform, with Remark 1's per-element alpha): the
// element matrix of a cube of side h is h*K with K = 1/3 on the diagonal, 0
// between nodes one coordinate apart and -1/12 between nodes two or three
// coordinates apart.  Hence for an interior node a
//     (A x)_a = h/12 * sum_{e containing a} alpha_e (4 x_a - sum_{b in e,
//               b two or three coordinates from a} x_b).
#include "common.cuh"
#include "kernels.h"

namespace bddc {

long long g_launches = 0;

__device__ inline double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block reduction into partial[blockIdx.x]; every thread must call it.
__device__ inline void block_partial(double v, double* partial) {
  __shared__ double ws[32];
  v = warp_sum_d(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) ws[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = (lane < (int)(blockDim.x >> 5)) ? ws[lane] : 0.0;
    v = warp_sum_d(v);
    if (lane == 0) partial[blockIdx.x] = v;
  }
}

// y = A x on the full node grid (x's Dirichlet entries read as 0, y's written
// 0).  If dot_partial != nullptr also accumulates x.y into per-block partials.
__global__ void __launch_bounds__(256)
k_operator(MeshDev m, const double* __restrict__ alpha, const double* __restrict__ x, double* __restrict__ y,
           double* __restrict__ dot_partial) {
  pdl_enter();
  const long long N = (long long)m.NX * m.NY * m.NZ;
  const long long sx = 1, sy = m.NX, sz = (long long)m.NX * m.NY;
  double dot = 0.0;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < N;
       g += (long long)gridDim.x * blockDim.x) {
    int i = (int)(g % m.NX), j = (int)((g / m.NX) % m.NY), k = (int)(g / sz);
    double out = 0.0;
    if (!(i == 0 || j == 0 || k == 0 || i == m.nx || j == m.ny || k == m.nz)) {
      // neighbourhood with Dirichlet entries masked
      double xv[27];
#pragma unroll
      for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
          for (int dx = -1; dx <= 1; ++dx) {
            int ii = i + dx, jj = j + dy, kk = k + dz;
            bool bnd = ii == 0 || jj == 0 || kk == 0 || ii == m.nx || jj == m.ny || kk == m.nz;
            xv[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)] = bnd ? 0.0 : x[g + dx * sx + dy * sy + dz * sz];
          }
      double asum = 0.0, acc = 0.0;
#pragma unroll
      for (int oz = 0; oz < 2; ++oz)
#pragma unroll
        for (int oy = 0; oy < 2; ++oy)
#pragma unroll
          for (int ox = 0; ox < 2; ++ox) {
            // element with corner offsets s = (2o-1) around the node
            const int ex = i - 1 + ox, ey = j - 1 + oy, ez = k - 1 + oz;
            const double a = alpha[(long long)ex + (long long)m.nx * (ey + (long long)m.ny * ez)];
            const int px = 2 * ox, py = 2 * oy, pz = 2 * oz;  // index of offset +-1 in xv
            const double far = xv[pz * 9 + py * 3 + 1] + xv[pz * 9 + 3 + px] + xv[9 + py * 3 + px] +
                               xv[pz * 9 + py * 3 + px];
            asum += a;
            acc = fma(a, far, acc);
          }
      out = (m.h / 12.0) * (4.0 * xv[13] * asum - acc);
    }
    y[g] = out;
    if (dot_partial) dot += out * ((i == 0 || j == 0 || k == 0 || i == m.nx || j == m.ny || k == m.nz) ? 0.0 : x[g]);
  }
  if (dot_partial) block_partial(dot, dot_partial);
}

void launch_operator(const MeshDev& m, const double* alpha, const double* x, double* y, double* dot_partial,
                     int nblocks, cudaStream_t st) {
  BDDC_COUNT(1);
  launch_pdl(k_operator, dim3(nblocks), dim3(256), 0, st, m, alpha, x, y, dot_partial);
}

// g_e = -h * lambda_e^T K u_e  (the derivative of J(u(alpha)) in alpha_e when
// A lambda = dJ/du).  With S = sum of the 8 nodal u values and N1(a) the sum
// over the three edge neighbours of a in e:  (K u)_a = (5 u_a + N1(a) - S)/12.
__global__ void k_gradient(MeshDev m, const double* __restrict__ u, const double* __restrict__ lam,
                           double* __restrict__ g) {
  const long long NE = (long long)m.nx * m.ny * m.nz;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < NE;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e % m.nx), j = (int)((e / m.nx) % m.ny), k = (int)(e / ((long long)m.nx * m.ny));
    double uv[8], lv[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      int ii = i + (a & 1), jj = j + ((a >> 1) & 1), kk = k + (a >> 2);
      bool bnd = ii == 0 || jj == 0 || kk == 0 || ii == m.nx || jj == m.ny || kk == m.nz;
      long long gi = nodeid(m.NX, m.NY, ii, jj, kk);
      uv[a] = bnd ? 0.0 : u[gi];
      lv[a] = bnd ? 0.0 : lam[gi];
    }
    double S = 0.0;
#pragma unroll
    for (int a = 0; a < 8; ++a) S += uv[a];
    double q = 0.0;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      double n1 = uv[a ^ 1] + uv[a ^ 2] + uv[a ^ 4];
      q += lv[a] * (5.0 * uv[a] + n1 - S);
    }
    g[e] = -m.h * q / 12.0;
  }
}

void launch_gradient(const MeshDev& m, const double* u, const double* lam, double* g, cudaStream_t st) {
  long long NE = (long long)m.nx * m.ny * m.nz;
  int blocks = (int)std::min<long long>((NE + 255) / 256, 152 * 16);
  BDDC_COUNT(1);
  k_gradient<<<blocks, 256, 0, st>>>(m, u, lam, g);
}

// Weighted injection onto Gamma: z(xi) = sum_i delta_i(xi) v_i(xi) over the
// subdomains holding xi (eq. W); other nodes get 0.  The subdomains of a node
// follow from the per-axis slab tables, so the sum order is fixed.
__global__ void k_interface_gather(MeshDev m, const SubDesc* __restrict__ subs, const double* __restrict__ delta,
                                   const double* __restrict__ vgam, double* __restrict__ z) {
  pdl_enter();
  const long long N = (long long)m.NX * m.NY * m.NZ;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < N;
       g += (long long)gridDim.x * blockDim.x) {
    int c[3] = {(int)(g % m.NX), (int)((g / m.NX) % m.NY), (int)(g / ((long long)m.NX * m.NY))};
    double out = 0.0;
    bool bnd = c[0] == 0 || c[1] == 0 || c[2] == 0 || c[0] == m.nx || c[1] == m.ny || c[2] == m.nz;
    if (!bnd && (m.ax[0].theta[c[0]] || m.ax[1].theta[c[1]] || m.ax[2].theta[c[2]])) {
      int sl[3][2], ns[3];
      for (int d = 0; d < 3; ++d) {
        if (m.ax[d].theta[c[d]]) { ns[d] = 2; sl[d][0] = m.ax[d].slab[c[d] - 1]; sl[d][1] = m.ax[d].slab[c[d]]; }
        else { ns[d] = 1; sl[d][0] = m.ax[d].slab[c[d]]; }
      }
      for (int cz = 0; cz < ns[2]; ++cz)
        for (int cy = 0; cy < ns[1]; ++cy)
          for (int cx = 0; cx < ns[0]; ++cx) {
            int si = sl[0][cx] + m.nsub[0] * (sl[1][cy] + m.nsub[1] * sl[2][cz]);
            const SubDesc& s = subs[si];
            int b = surf_index(c[0] - s.e0[0], c[1] - s.e0[1], c[2] - s.e0[2], s.w[0] + 1, s.w[1] + 1, s.w[2] + 1);
            out += delta[s.offB + b] * vgam[s.offB + b];
          }
    }
    z[g] = out;
  }
}

void launch_interface_gather(const MeshDev& m, const SubDesc* subs, const double* delta, const double* vgam,
                             double* z, cudaStream_t st) {
  long long N = (long long)m.NX * m.NY * m.NZ;
  int blocks = (int)std::min<long long>((N + 255) / 256, 152 * 16);
  BDDC_COUNT(1);
  launch_pdl(k_interface_gather, dim3(blocks), dim3(256), 0, st, m, subs, delta, vgam, z);
}

__global__ void k_check_alpha(const double* __restrict__ a, long long n, int* err) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    double v = a[e];
    if (!(v > 0.0) || !isfinite(v)) {
      if (atomicCAS(err, 0, 1) == 0) err[1] = (int)e;
    }
  }
}

void launch_check_alpha(const double* alpha, long long n, int* err, cudaStream_t st) {
  int blocks = (int)std::min<long long>((n + 255) / 256, 152 * 8);
  BDDC_COUNT(1);
  k_check_alpha<<<blocks, 256, 0, st>>>(alpha, n, err);
}

// dst = src with the Dirichlet-boundary entries set to 0.
__global__ void k_masked_copy(MeshDev m, const double* __restrict__ src, double* __restrict__ dst) {
  const long long N = (long long)m.NX * m.NY * m.NZ;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < N; g += (long long)gridDim.x * blockDim.x) {
    int i = (int)(g % m.NX), j = (int)((g / m.NX) % m.NY), k = (int)(g / ((long long)m.NX * m.NY));
    bool bnd = i == 0 || j == 0 || k == 0 || i == m.nx || j == m.ny || k == m.nz;
    dst[g] = bnd ? 0.0 : src[g];
  }
}

void launch_masked_copy(const MeshDev& m, const double* src, double* dst, cudaStream_t st) {
  long long N = (long long)m.NX * m.NY * m.NZ;
  int blocks = (int)std::min<long long>((N + 255) / 256, 152 * 16);
  BDDC_COUNT(1);
  k_masked_copy<<<blocks, 256, 0, st>>>(m, src, dst);
}

}  // namespace bddc
