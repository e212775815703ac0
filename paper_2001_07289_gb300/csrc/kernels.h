// Host-side launchers shared by the translation units of the BDDC-SO library.
#pragma once
#include <cuda_runtime.h>
#include <algorithm>
#include <functional>
#include <vector>
#include "common.cuh"

namespace bddc {

// Running count of kernel launches issued by this library (host side).
extern long long g_launches;
#define BDDC_COUNT(n) (::bddc::g_launches += (n))

// Launch with programmatic stream serialisation, for kernels that start with
// pdl_enter(): the launch overlaps the previous kernel's tail.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

constexpr int CW = 64;       // RHS columns per CTA in the multi-RHS sweeps

// A size bucket of the apply's per-subdomain kernels: its descriptors in
// longest-first order (device), their number and the depth of the bulk-copy
// ring its launches use.  A launch over a bucket is persistent: clusters take
// the bucket's subdomains in turn.
struct ApplyBucket {
  const SubDesc* subs;
  int count;
  int nb;
};

constexpr int MAX_BUCKETS = 2;

// A bucket of the local factorisations: bucket 0 holds the subdomains whose
// planes fit the tensor-core kernel (FP32 path), bucket 1 the rest; longest
// first.
struct FactorBucket {
  const SubDesc* subs;
  int count;
  int maxQN, maxQD;
};

// Largest local sizes in a bucket (shared-memory sizing of its launches).
struct BucketSizes {
  int maxQD, maxND, maxQN, maxNN, maxNB, maxNc;
};

// Everything a batched local kernel needs (device pointers; local type erased).
struct LocalLaunch {
  int nsub;
  const SubDesc* subs;
  MeshDev m;
  const double* alpha;
  const LocalCoarse* lc;
  const int* lcn;               // local node lists of the coarse DOFs (LocalCoarse::off, count)
  const int* own;               // per local Neumann node (offVec layout): local average index or -1
  void *facD, *facN, *scratch, *mscratch;
  long long mscratch_stride;
  void *Y, *G, *Lv, *PA, *Sc, *Phi, *vloc;
  void* PhiT;                      // transposed copy of Phi for the apply's column accumulations
  const SubDesc* subs_lpt;         // the same descriptors, largest subdomains first
  void* tc;                        // packed 3xTF32 tiles of the Neumann S_k^{-1} (setup, FP32 path) or null
  double* Ac;
  double* delta;
  double* vgam;
  double* rcl;
  int* err;
  int maxQD, maxNzD, maxND;   // Dirichlet: plane size, planes, nodes
  int maxQN, maxNzN, maxNN;   // Neumann
  int maxNB, maxNc;
  // size buckets of the apply: [0] subdomains whose work vectors leave no room
  // for two CTAs per SM with a shallow ring, [1] the others (either may be
  // empty); per bucket the ring depth and CTAs per subdomain (tuned)
  int nbucket = 0;
  ApplyBucket bucket[MAX_BUCKETS] = {};
  BucketSizes bsize[MAX_BUCKETS] = {};
  int bcluster[MAX_BUCKETS] = {1, 1};
  FactorBucket fbucket[2] = {};
  // pinned floating subdomains (selections without point values): their
  // count and the augmented-Lagrangian weight rho per local coarse DOF (cofs)
  int npin = 0;
  double* pen = nullptr;
  int factor_tc = 1;          // bucket 0 on the tensor cores (1) or the CUDA cores (0), tuned
  int negate_sub = -1;        // test hook: subdomain whose local matrix gets a negated pivot (-1: none)
  int negate_neumann = 1;     // ... in its Neumann (1) or Dirichlet (0) matrix
};

// schur_tc.cu: the local factorisations on the tensor cores (FP32 path,
// planes of at most TCS_MAXQ nodes)
constexpr int TCS_MAXQ = 176;
size_t schur_tc_smem(int maxQ);
void configure_schur_tc();
void launch_schur_tc(const LocalLaunch& L, const FactorBucket& B, cudaStream_t st);
// assembly of the local plane blocks; the factorisations of every bucket
// (tc: bucket 0 on the tensor cores)
// tc: the factorisation that follows runs on the tensor cores (FP32 path):
// D_k of its subdomains as in-plane taps (plane_taps)
template <typename T> void launch_assemble(const LocalLaunch& L, int tc, cudaStream_t st);
template <typename T> void launch_factor(const LocalLaunch& L, int tc, cudaStream_t st);

// ev (may be null): 3 events recorded after the Dirichlet factorisation, the
// Neumann factorisation and the coarse basis.
template <typename T> void launch_setup_local(const LocalLaunch& L, cudaStream_t st, cudaEvent_t* ev);
template <typename T> void configure_local_kernels();
template <typename T> size_t dense_smem();
template <typename T>
void launch_dirichlet(const LocalLaunch& L, const double* r, const double* t, double* z, int mode, cudaStream_t st);
// weighted restriction r_i of r - t and the local coarse right-hand sides
// rc_i = Phi_i^T r_i (into L.rcl)
template <typename T> void launch_neumann_rhs(const LocalLaunch& L, const double* r, const double* t, cudaStream_t st);
// constrained Neumann solves y = A_rr^{-1} r_i,r (into L.vloc)
template <typename T> void launch_neumann(const LocalLaunch& L, const double* r, const double* t, cudaStream_t st);
template <typename T> void launch_neumann_finish(const LocalLaunch& L, const double* uc, cudaStream_t st);
void launch_weights(const LocalLaunch& L, const double* piece_w, cudaStream_t st);
// test hook: tries after which the bounded waits of the local kernels report
// a timeout (they then still wait, bounded, for the work they cover)
void set_wait_report_tries(long long tries);
// shared-memory bytes of the apply's per-subdomain kernels for bucket sizes
// bs, ring depth nb and local element size es (the largest over the kernels)
size_t apply_smem(const BucketSizes& bs, int nb, int es);
void launch_piece_alpha(const double* alpha, const long long* pe_off, const int* pe, int np, double* pw,
                        cudaStream_t st);
void launch_piece_alpha_box(const double* alpha, int nx, int ny, const int* plo, const int* phi, int npx, int npy,
                            int npz, double* pw, cudaStream_t st);
void launch_mark_coarse(const LocalLaunch& L, unsigned char* vfix, int* own, cudaStream_t st);
void launch_box_pieces(int nx, int ny, int nz, const int* pa, const int* pb, const int* pc, int npx, int npy,
                       int* epiece, cudaStream_t st);

// coarse.cu
void launch_coarse_assemble(const LocalLaunch& L, const int* color_subs, const int* color_count_host,
                            const int* color_offset_host, double* Acg, int nc, cudaStream_t st);
void launch_coarse_gather(const int* ptr, const int2* ent, const double* rcl, double* rc, int nc, cudaStream_t st);

// coarse_mf.cu: multifrontal FP64 Cholesky of the coarse matrix in a nested-
// dissection order over the subdomain grid.
// Coarse objects by position at subdomain granularity: a "cell" has doubled
// subdomain coordinates per axis, 2s + 1 inside slab s, 2s on the cut plane
// between slabs s - 1 and s (0 and 2 nsub: the domain boundary); an object's
// cell follows from the subdomains that share it.
struct CoarseGeom {
  int nsub[3];
  std::vector<int> cell_ptr;   // CSR over cells (x fastest, (2 nsub + 1) per axis)
  std::vector<int> cell_obj;   // coarse ids of each cell, ascending
};

struct MFPlan {
  int nfront = 0, nlevel = 0, nc = 0;
  // host
  std::vector<int> level_of, np, nu, parent, child_slot;   // per front
  std::vector<long long> foff, doff, woff;                  // front, dinv, work-vector offsets
  std::vector<int> gid;                                     // per front: P then U global ids (concatenated)
  std::vector<long long> gid_off;
  std::vector<int> ord, fr, pp;                             // per coarse dof: order, owning front, pivot pos
  std::vector<std::vector<int>> fronts_at_level;
  std::vector<int> pmap;                                    // child U -> position in parent front
  std::vector<long long> pmap_off;
  long long fpool = 0, dpool = 0, wpool = 0;
  double flops = 0;                                         // FMA count of the partial factorisations
  // device
  int *d_np = nullptr, *d_nu = nullptr, *d_gid = nullptr, *d_fr = nullptr, *d_pp = nullptr, *d_ord = nullptr;
  long long *d_foff = nullptr, *d_doff = nullptr, *d_woff = nullptr, *d_gid_off = nullptr, *d_pmap_off = nullptr;
  int *d_pmap = nullptr, *d_parent = nullptr;
  int *d_ugid = nullptr;            // per front: U ids sorted (for the assembly lookup) ...
  int *d_upos = nullptr;            // ... and their positions in the front
  long long* d_ugid_off = nullptr;
  double *F = nullptr, *Dinv = nullptr, *W = nullptr;
  // solve matrices per front: S_f = [Linv_P; G] (F x np, row-major, ld np),
  // Linv_P = L_P^{-1} and G = L_UP Linv_P
  std::vector<long long> soff;
  long long spool = 0;
  double* S = nullptr;
  double* ST = nullptr;             // S_f^T (np x F, ld F) at the same offsets, for the backward solve
  long long* d_soff = nullptr;
  // L_P^{-1} by recursive doubling: at level q (half block hb = 2^q tiles)
  // the items {front, r, c, hb} cover every tile of the off-diagonal blocks
  // per level of the front tree: [0] diagonal tiles {front, t, t, 0},
  // [1] G tiles {front, ut, st, 0}, [2 + 4q + 2 mode] the tile products of
  // doubling step q {front, r, c, k}, [2 + 4q + 2 mode + 1] their sums
  // {front, r << 16 | c, first product, count}
  std::vector<std::vector<std::vector<int>>> inv_items;
  std::vector<long long> inv_off;              // device offsets of these lists, level by level
  std::vector<int> inv_len;
  std::vector<int> inv_lvl_base;               // per level: first index into inv_off / inv_len
  std::vector<long long> toff;                 // per front: np x np block of the product scratch
  long long tpool = 0;
  long long* d_toff = nullptr;
  double* tscratch = nullptr;                  // L_CA X_AA products of the doubling steps
  double* tpart = nullptr;                     // 32 x 32 tile products before their sums
  std::vector<int> fwd_items_off, bwd_items_off; // per level into the solve work lists
  int* d_solve_items = nullptr;                // int2 {front, chunk} lists for the solves
  std::vector<int> fwd_items_len, bwd_items_len;
  long long blob_lvl_index = 0;                // per front: its index in the level-ordered list
  int maxF = 0;
  // work lists per (level, panel step): int4 {front, i, l, j}, concatenated on the device
  // per (level, panel step j): the fronts still factoring, as int4 entries
  // {front, tiles nt, first trsm item, first syrk item} (prefix counts); the
  // kernels decode their item from the block index, so the lists, whose length
  // grows as nt^3 per front, are not stored item by item
  std::vector<std::vector<int>> step_fronts;
  std::vector<int> step_j, step_ntr, step_nsy;
  std::vector<long long> step_off;            // device offsets of the tables
  int4* d_lists = nullptr;
  double* pscratch = nullptr;       // potrf scratch: 2048 doubles per concurrent diagonal tile
  double* fscratch = nullptr;       // look-ahead potrf scratch in the syrk steps: 2048 doubles per front
  // per level, on the device in one int array: fronts by level, each front's
  // children (CSR aligned with that list), and children by (level, slot)
  int maxslot = 0;
  std::vector<int> lvl_fronts_off;  // per level into the level-ordered front list
  std::vector<int> slot_off;        // per (level, slot) into the slot lists
  long long blob_kptr = 0, blob_klist = 0, blob_slots = 0;
  int* d_blob = nullptr;
};

// host -> device copy of setup metadata, through pinned staging while a
// setup holds it (ordered in st, returns without waiting for st's queued work)
void stage_h2d(void* dst, const void* src, size_t bytes, cudaStream_t st);

void mf_plan(MFPlan& P, const CoarseGeom& g, int nc);
void mf_plan_independent(MFPlan& P, const std::vector<int>& sizes);
// dense local matrices (m x m row-major, global ids per item) into the
// fronts; the listed items share no global id
void mf_add_local(const MFPlan& P, const int* list, int nitems, const int* goff, const int* msz,
                  const long long* moff, const int* gidmap, const double* vals, cudaStream_t st);
// alloc: memory kept for the solves; tmp_alloc: memory needed during setup only
void mf_upload(MFPlan& P, const std::function<void*(size_t)>& alloc,
               const std::function<void*(size_t)>& tmp_alloc, cudaStream_t st);
void mf_assemble(const MFPlan& P, const LocalLaunch& L, const int* color_subs, const int* color_count_host,
                 const int* color_offset_host, cudaStream_t st);
// aux, fork, join (may be null): a second stream and two events; each
// level's solve matrices are then built on aux while st factors the levels
// above it, and st waits for aux before it returns
void mf_factor(const MFPlan& P, int* err, cudaStream_t st, cudaStream_t aux, cudaEvent_t fork, cudaEvent_t join);
// x = A_c^{-1} b; W: work vector pool of P.wpool doubles
void mf_solve(const MFPlan& P, const double* b, double* x, double* W, cudaStream_t st);
void configure_mf_kernels();

// multilevel.cu: the second level of multilevel BDDC-SO, BDDC applied to the
// coarse problem with blocks of g x g x g subdomains (Section 6).  Coarse
// DOFs shared by two or more blocks form the coarse interface Gamma_2; they
// are grouped into level-2 objects by the set of blocks sharing them, each
// constraint the mean of the object's coarse values; weights per block slot
// (w2s): 1 / (blocks sharing the DOF) or diagonal stiffness scaling.  Dense FP64 throughout, on independent multifrontal
// fronts: N, the blocks' augmented matrices A_k + rho_k C_k^T C_k (exact for
// the constrained problems, C_k w being prescribed); D, the blocks' interior
// matrices; C, the level-2 coarse matrix, by fronts of a nested dissection
// of the block grid.  With sub-blocks of `sub` subdomains inside the blocks
// (BDDC-SO on the coarse level), level-2 objects group the Gamma_2 DOFs by
// the set of sub-blocks sharing them.
struct MLPlan {
  int g = 0, sub = 0, nblock = 0, nc = 0, ncc = 0, NB = 0, NI = 0, NO = 0, maxm = 0;
  // host: per block its block-space offset and size, interior offset and
  // size, object-slot offset and count; its subdomains and colour
  std::vector<int> boff, bn, ioff, bni, ooff, bm, bsub_ptr, bsub, bcolor;
  std::vector<int> bgid;              // block-space slot -> coarse id
  std::vector<int> iidx;              // block-space slot -> block-interior slot, -1 on Gamma_2
  std::vector<int> igid;              // block-interior slot -> coarse id
  std::vector<unsigned char> gam2;    // per coarse id: on Gamma_2
  std::vector<double> w2;             // per coarse id: weight (1 inside a block)
  std::vector<int> slot_ptr, slot_ent;  // coarse id -> its block-space slots (ascending block)
  std::vector<int> oobj;              // object slot -> level-2 object
  std::vector<int> obj_ptr, obj_ent;  // level-2 object -> its object slots (ascending block)
  std::vector<int> orow_ptr, orow_ent;  // object slot -> block-space slots of the object's DOFs
  std::vector<int> sub2blk;           // level-1 local-coarse entry (lc index) -> block-space slot
  std::vector<int> nfront_of, dfront_of;   // block -> front of plan N / D (-1: none)
  MFPlan N, D, C;
  // device
  int *d_boff = nullptr, *d_bn = nullptr, *d_ooff = nullptr, *d_bm = nullptr, *d_bsub_ptr = nullptr,
      *d_bsub = nullptr, *d_bgid = nullptr, *d_iidx = nullptr, *d_igid = nullptr, *d_slot_ptr = nullptr,
      *d_slot_ent = nullptr, *d_oobj = nullptr, *d_obj_ptr = nullptr, *d_obj_ent = nullptr,
      *d_orow_ptr = nullptr, *d_orow_ent = nullptr, *d_sub2blk = nullptr, *d_nfront = nullptr,
      *d_dfront = nullptr, *d_bcolor_list = nullptr;
  std::vector<int> color_off, color_cnt;   // blocks by colour (no two of one colour share an object)
  unsigned char* d_gam2 = nullptr;
  double *d_w2 = nullptr, *w2s = nullptr, *rho = nullptr, *X = nullptr, *Psi = nullptr, *Acck = nullptr;
  long long *d_accoff = nullptr;
  std::vector<long long> accoff;      // per block: offset of its m x m level-2 matrix
  // apply work vectors
  double *bI = nullptr, *uIb = nullptr, *sI = nullptr, *u = nullptr, *tl = nullptr, *t = nullptr, *rb = nullptr,
         *y = nullptr, *v = nullptr, *rs = nullptr, *rcc = nullptr, *ucc = nullptr, *vg = nullptr;
  double flops = 0;                   // factorisation multiply-adds of the three plans
};

void ml_plan(MLPlan& P, int g, int sub, const int nsub[3], const std::vector<SubDesc>& subs,
             const std::vector<LocalCoarse>& lc, int nc, const std::vector<int>& cptr, const std::vector<int2>& cent);
void ml_setup(MLPlan& P, const LocalLaunch& L, const std::function<void*(size_t)>& alloc,
              const std::function<void*(size_t)>& tmp_alloc, int stiffness, int* err, cudaStream_t st);
void ml_apply(const MLPlan& P, const LocalLaunch& L, const int* cptr, const int2* cent, const double* rc, double* uc,
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
// scalars: [0] rz, [1] pq, [2] alpha, [3] rr, [4] rz_new, [5] beta, [6] bb,
// [7] stopping threshold; ctl: [0] it, [1] continue, [2] converged, [3] breakdown
void launch_finalize(const double* partial, double* scal, int op, double* hist, int* ctl, int maxit, double rtol,
                     const cudaGraphConditionalHandle* cond, cudaStream_t st);
void launch_loop_condition(const int* ctl, cudaGraphConditionalHandle cond, cudaStream_t st);
void launch_update_xr(double* x, double* r, const double* p, const double* q, const double* scal, long long n,
                      double* partial, cudaStream_t st);
void launch_update_p(double* p, const double* z, const double* scal, long long n, cudaStream_t st);
// flexible (Polak-Ribiere) recurrence: r.z and r.zp into 2 RED_BLOCKS partials;
// p = z + beta p with zp = z
void launch_dot2(const double* r, const double* z, const double* zp, long long n, double* partial, cudaStream_t st);
void launch_update_p_keep(double* p, double* zp, const double* z, const double* scal, long long n, cudaStream_t st);

}  // namespace bddc
