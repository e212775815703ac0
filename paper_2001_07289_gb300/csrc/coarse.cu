// Coarse vectors and the dense coarse matrix of BDDC-SO (FP64): the gather
// r_c = sum_i R_ci^T rc_i of the local coarse right-hand sides, and the dense
// assembly A_c = sum_i R_ci^T A_c^(i) R_ci kept for small problems as a
// diagnostic (the solver factors A_c by fronts, coarse_mf.cu).  The coarse
// DOFs are the selected (sub)objects of Section 3.
#include "common.cuh"
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

}  // namespace bddc
