// Host-side launchers shared by the translation units of the BDDC-SO library.
#pragma once
#include <cuda_runtime.h>
#include <algorithm>
#include "common.cuh"

namespace bddc {

// Running count of kernel launches issued by this library (host side).
extern long long g_launches;
#define BDDC_COUNT(n) (::bddc::g_launches += (n))

constexpr int CW = 64;       // RHS columns per CTA in the multi-RHS sweeps
constexpr int CNB = 128;     // coarse Cholesky tile

// Everything a batched local kernel needs (device pointers; local type erased).
struct LocalLaunch {
  int nsub;
  const SubDesc* subs;
  MeshDev m;
  const double* alpha;
  const LocalCoarse* lc;
  void *facD, *facN, *scratch, *mscratch;
  long long mscratch_stride;
  void *Y, *G, *Lv, *PA, *Sc, *Phi, *vloc;
  double* Ac;
  double* delta;
  double* vgam;
  double* rcl;
  int* err;
  int maxQD, maxNzD, maxND;   // Dirichlet: plane size, planes, nodes
  int maxQN, maxNzN, maxNN;   // Neumann
  int maxNB, maxNc;
};

// ev (may be null): 3 events recorded after the Dirichlet factorisation, the
// Neumann factorisation and the coarse basis.
template <typename T> void launch_setup_local(const LocalLaunch& L, cudaStream_t st, cudaEvent_t* ev);
template <typename T> void configure_local_kernels();
template <typename T> size_t dense_smem();
template <typename T>
void launch_dirichlet(const LocalLaunch& L, const double* r, const double* t, double* z, int mode, cudaStream_t st);
template <typename T> void launch_neumann(const LocalLaunch& L, const double* r, const double* t, cudaStream_t st);
template <typename T> void launch_neumann_finish(const LocalLaunch& L, const double* uc, cudaStream_t st);
void launch_weights(const LocalLaunch& L, const double* piece_w, cudaStream_t st);
void launch_piece_alpha(const MeshDev& m, const double* alpha, const int* plo, const int* phi, int npx, int npy,
                        int npz, double* pw, cudaStream_t st);

// coarse.cu
void configure_coarse_kernels();
void launch_coarse_assemble(const LocalLaunch& L, const int* color_subs, const int* color_count_host,
                            const int* color_offset_host, double* Acg, int nc, cudaStream_t st);
void launch_coarse_factor(double* Acg, int nc, double* dinv, double* scratch, int* err, cudaStream_t st);
void launch_coarse_gather(const int* ptr, const int2* ent, const double* rcl, double* rc, int nc, cudaStream_t st);
void launch_coarse_solve(const double* L, int nc, const double* dinv, double* b, double* y, double* x,
                         cudaStream_t st);

// stencil.cu
void launch_operator(const MeshDev& m, const double* alpha, const double* x, double* y, double* dot_partial,
                     int nblocks, cudaStream_t st);
void launch_gradient(const MeshDev& m, const double* u, const double* lam, double* g, cudaStream_t st);
void launch_interface_gather(const MeshDev& m, const SubDesc* subs, const double* delta, const double* vgam,
                             double* z, cudaStream_t st);
void launch_check_alpha(const double* alpha, long long n, int* err, cudaStream_t st);
void launch_masked_copy(const MeshDev& m, const double* src, double* dst, cudaStream_t st);

// pcg.cu
constexpr int RED_BLOCKS = 608;  // 4 x 152 SMs: fixed partial count => deterministic sums
void launch_dot(const double* a, const double* b, long long n, double* partial, cudaStream_t st);
// scalars: [0] rz, [1] pq, [2] alpha, [3] rr, [4] rz_new, [5] beta, [6] bb
void launch_finalize(const double* partial, double* scal, int op, double* hist, int it, int* flag,
                     cudaStream_t st);
void launch_update_xr(double* x, double* r, const double* p, const double* q, const double* scal, long long n,
                      double* partial, cudaStream_t st);
void launch_update_p(double* p, const double* z, const double* scal, long long n, cudaStream_t st);

}  // namespace bddc
