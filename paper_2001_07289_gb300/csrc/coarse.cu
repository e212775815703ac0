// Coarse problem of BDDC-SO in FP64: assembly A_c = sum_i R_ci^T A_c^(i) R_ci,
// dense blocked Cholesky A_c = L L^T and the two triangular solves of the
// apply.  The coarse DOFs are the selected (sub)objects (Section 3); the paper
// points to the coarse problem as BDDC-SO's main cost (Sections 1 and 6).
//
// Factor layout: A_c row-major n x n (ld n); after factorisation its lower
// triangle holds L; dinv holds the inverses of the diagonal CNB x CNB tiles of
// L (row-major, ld CNB), so a triangular solve is a sequence of dense
// mat-vecs.
#include "common.cuh"
#include "dense.cuh"
#include "kernels.h"

namespace bddc {

// ---------------------------------------------------------------------------
// assembly: one launch per subdomain colour (subdomains of one colour share
// no coarse DOF), so each entry is summed in a fixed order without atomics.
// ---------------------------------------------------------------------------
__global__ void k_coarse_assemble(const SubDesc* __restrict__ subs, const LocalCoarse* __restrict__ lc,
                                  const int* __restrict__ list, const double* __restrict__ Ac,
                                  double* __restrict__ Acg, long long nc) {
  const SubDesc s = subs[list[blockIdx.x]];
  const int n = s.nc;
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < n * n; e += gridDim.y * blockDim.x) {
    int r = e / n, c = e % n;
    long long gr = lc[s.cofs + r].gid, gc = lc[s.cofs + c].gid;
    Acg[gr * nc + gc] += Ac[s.offAc + e];
  }
}

void launch_coarse_assemble(const LocalLaunch& L, const int* color_subs, const int* color_count_host,
                            const int* color_offset_host, double* Acg, int nc, cudaStream_t st) {
  for (int c = 0; c < 8; ++c) {
    if (color_count_host[c] == 0) continue;
    BDDC_COUNT(1);
    k_coarse_assemble<<<dim3(color_count_host[c], 16), BDDC_THREADS, 0, st>>>(
        L.subs, L.lc, color_subs + color_offset_host[c], L.Ac, Acg, nc);
  }
}

// ---------------------------------------------------------------------------
// blocked right-looking Cholesky
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(BDDC_THREADS)
k_coarse_potrf(double* A, int n, int j, double* dinv, double* scratch, int* err) {
  extern __shared__ __align__(16) unsigned char smraw[];
  DenseSmem<double>& sm = *reinterpret_cast<DenseSmem<double>*>(smraw);
  const int j0 = j * CNB, nb = min(CNB, n - j0);
  double* D = dinv + (long long)j * CNB * CNB;
  bool ok = cta_chol_inv<double>(A + (long long)j0 * n + j0, n, D, CNB, nb, scratch, sm);
  if (!ok && threadIdx.x == 0) {
    if (atomicCAS(err, 0, 5) == 0) err[1] = j;
  }
}

// A[i,j] <- A[i,j] Linv_jj^T for the tiles below the diagonal tile j.
__global__ void __launch_bounds__(BDDC_THREADS)
k_coarse_trsm(double* A, int n, int j, const double* dinv, double* scratch) {
  extern __shared__ __align__(16) unsigned char smraw[];
  DenseSmem<double>& sm = *reinterpret_cast<DenseSmem<double>*>(smraw);
  const int j0 = j * CNB, nbj = min(CNB, n - j0);
  const int i = j + 1 + blockIdx.x;
  const int i0 = i * CNB, nbi = min(CNB, n - i0);
  double* T = scratch + (long long)blockIdx.x * CNB * CNB;
  double* tile = A + (long long)i0 * n + j0;
  for (int e = threadIdx.x; e < nbi * nbj; e += blockDim.x) T[e] = tile[(long long)(e / nbj) * n + e % nbj];
  __syncthreads();
  cta_gemm<double>(nbi, nbj, nbj, 1.0, T, nbj, false, dinv + (long long)j * CNB * CNB, CNB, true, 0.0, tile, n,
                   0, 1, false, sm);
}

// A[i,l] -= A[i,j] A[l,j]^T for j < l <= i (lower tiles of the trailing matrix).
__global__ void __launch_bounds__(BDDC_THREADS)
k_coarse_syrk(double* A, int n, int j, int nt) {
  extern __shared__ __align__(16) unsigned char smraw[];
  DenseSmem<double>& sm = *reinterpret_cast<DenseSmem<double>*>(smraw);
  const int m = nt - j - 1;
  const int i = j + 1 + blockIdx.x / m, l = j + 1 + blockIdx.x % m;
  if (l > i) return;
  const int j0 = j * CNB, nbj = min(CNB, n - j0);
  const int i0 = i * CNB, nbi = min(CNB, n - i0);
  const int l0 = l * CNB, nbl = min(CNB, n - l0);
  cta_gemm<double>(nbi, nbl, nbj, -1.0, A + (long long)i0 * n + j0, n, false, A + (long long)l0 * n + j0, n, true,
                   1.0, A + (long long)i0 * n + l0, n, 0, 0, i == l, sm);
}

void configure_coarse_kernels() {
  int sm = (int)sizeof(DenseSmem<double>);
  cudaFuncSetAttribute(k_coarse_potrf, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_coarse_trsm, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_coarse_syrk, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

void launch_coarse_factor(double* A, int n, double* dinv, double* scratch, int* err, cudaStream_t st) {
  const int nt = (n + CNB - 1) / CNB;
  const size_t sm = sizeof(DenseSmem<double>);
  for (int j = 0; j < nt; ++j) {
    k_coarse_potrf<<<1, BDDC_THREADS, sm, st>>>(A, n, j, dinv, scratch, err);
    BDDC_COUNT(1);
    const int m = nt - j - 1;
    if (m > 0) {
      BDDC_COUNT(2);
      k_coarse_trsm<<<m, BDDC_THREADS, sm, st>>>(A, n, j, dinv, scratch);
      k_coarse_syrk<<<m * m, BDDC_THREADS, sm, st>>>(A, n, j, nt);
    }
  }
}

// ---------------------------------------------------------------------------
// r_c = sum_i R_ci^T rc_i: gather of the local coarse values of the
// subdomains sharing each coarse DOF, in a fixed order.
// ---------------------------------------------------------------------------
__global__ void k_coarse_gather(const int* __restrict__ ptr, const int2* __restrict__ ent,
                                const double* __restrict__ rcl, double* __restrict__ rc, int nc) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < nc; g += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int e = ptr[g]; e < ptr[g + 1]; ++e) s += rcl[ent[e].y];
    rc[g] = s;
  }
}

void launch_coarse_gather(const int* ptr, const int2* ent, const double* rcl, double* rc, int nc, cudaStream_t st) {
  if (nc <= 0) return;
  BDDC_COUNT(1);
  k_coarse_gather<<<(nc + 255) / 256, 256, 0, st>>>(ptr, ent, rcl, rc, nc);
}

// ---------------------------------------------------------------------------
// triangular solves, one launch per tile step
// ---------------------------------------------------------------------------
template <typename T>
__device__ inline T warp_sum_c(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// forward step j: y_j = Dinv_j b_j (all CTAs, CTA 0 stores it), then CTA c
// updates b_i -= L_ij y_j for i = j+1+c.
__global__ void __launch_bounds__(BDDC_THREADS)
k_coarse_fwd(const double* __restrict__ L, int n, int j, const double* __restrict__ dinv, double* b, double* y) {
  __shared__ double bj[CNB], yj[CNB];
  const int j0 = j * CNB, nbj = min(CNB, n - j0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = threadIdx.x; c < nbj; c += blockDim.x) bj[c] = b[j0 + c];
  __syncthreads();
  const double* D = dinv + (long long)j * CNB * CNB;
  for (int r = warp; r < nbj; r += nw) {
    double acc = 0.0;
    for (int c = lane; c <= r; c += 32) acc += D[r * CNB + c] * bj[c];
    acc = warp_sum_c(acc);
    if (lane == 0) yj[r] = acc;
  }
  __syncthreads();
  if (blockIdx.x == 0)
    for (int c = threadIdx.x; c < nbj; c += blockDim.x) y[j0 + c] = yj[c];
  const int i = j + 1 + blockIdx.x;
  const int i0 = i * CNB;
  if (i0 >= n) return;
  const int nbi = min(CNB, n - i0);
  for (int r = warp; r < nbi; r += nw) {
    const double* row = L + (long long)(i0 + r) * n + j0;
    double acc = 0.0;
    for (int c = lane; c < nbj; c += 32) acc += row[c] * yj[c];
    acc = warp_sum_c(acc);
    if (lane == 0) b[i0 + r] -= acc;
  }
}

// backward step j: x_j = Dinv_j^T y_j, then CTA c updates y_l -= L_jl^T x_j
// for l = c < j.  x and y are distinct: every CTA reads tile j of y.
__global__ void __launch_bounds__(BDDC_THREADS)
k_coarse_bwd(const double* __restrict__ L, int n, int j, const double* __restrict__ dinv, double* y, double* x) {
  __shared__ double yjs[CNB], xj[CNB];
  const int j0 = j * CNB, nbj = min(CNB, n - j0);
  for (int c = threadIdx.x; c < nbj; c += blockDim.x) yjs[c] = y[j0 + c];
  __syncthreads();
  const double* D = dinv + (long long)j * CNB * CNB;
  for (int c = threadIdx.x; c < nbj; c += blockDim.x) {
    double acc = 0.0;
    for (int r = c; r < nbj; ++r) acc += D[r * CNB + c] * yjs[r];
    xj[c] = acc;
  }
  __syncthreads();
  if (blockIdx.x == 0)
    for (int c = threadIdx.x; c < nbj; c += blockDim.x) x[j0 + c] = xj[c];
  const int l = blockIdx.x;
  if (l >= j) return;
  const int l0 = l * CNB;
  for (int c = threadIdx.x; c < CNB; c += blockDim.x) {
    double acc = 0.0;
    for (int r = 0; r < nbj; ++r) acc += L[(long long)(j0 + r) * n + l0 + c] * xj[r];
    y[l0 + c] -= acc;
  }
}

// x = A_c^{-1} b: b and y are work vectors (overwritten), x the result.
void launch_coarse_solve(const double* L, int n, const double* dinv, double* b, double* y, double* x,
                         cudaStream_t st) {
  const int nt = (n + CNB - 1) / CNB;
  BDDC_COUNT(2 * nt);
  for (int j = 0; j < nt; ++j) {
    int m = std::max(1, nt - j - 1);
    k_coarse_fwd<<<m, BDDC_THREADS, 0, st>>>(L, n, j, dinv, b, y);
  }
  for (int j = nt - 1; j >= 0; --j) {
    int m = std::max(1, j);
    k_coarse_bwd<<<m, BDDC_THREADS, 0, st>>>(L, n, j, dinv, y, x);
  }
}

}  // namespace bddc
