// Multilevel BDDC-SO: the second level (Section 6 names the multilevel
// version as the way past the coarse-problem size of BDDC-SO).  The coarse
// problem A_c u_c = r_c is preconditioned by one application of BDDC on the
// coarse level instead of being solved exactly, with Definition 1 applied
// once more:
//   * coarse "elements": the subdomains and their local coarse matrices
//     A_c^(i) = Phi_i^T A_i Phi_i;
//   * coarse "subdomains": blocks of g x g x g subdomains;
//   * V1 = the block-interior coarse DOFs, V2 = W-tilde_2 with one
//     constraint per level-2 object (Gamma_2 DOFs with equal block sets),
//     the mean of the object's coarse values;
//   * weights 1 / (blocks sharing the DOF), or with Remark 1's rho-weights on
//     the first level stiffness scaling on the second (the diagonal of A_k
//     over its sum across the blocks sharing the DOF); the level-2 coarse
//     problem exact.
// Everything is FP64 and dense per block, factored as independent fronts of
// the multifrontal code (coarse_mf.cu): every tile of every block's front
// goes to its own CTA, and one solve call treats all blocks.  A floating
// block's matrix is singular, so front N_k holds A_k + rho_k C_k^T C_k: the
// constrained problems prescribe C_k w, so their w is unchanged (an
// augmented Lagrangian) and only the level-2 coarse matrix changes,
// Psi^T A_k Psi = S_k^{-1} - rho_k I with S_k = C_k N_k^{-1} C_k^T.
#include <map>
#include <stdexcept>
#include <string>

#include "common.cuh"
#include "dense.cuh"
#include "kernels.h"

namespace bddc {

namespace {

template <typename T>
T* up(const std::vector<T>& v, const std::function<void*(size_t)>& alloc, cudaStream_t st) {
  T* p = (T*)alloc(sizeof(T) * std::max<size_t>(v.size(), 1));
  stage_h2d(p, v.data(), sizeof(T) * v.size(), st);
  return p;
}

}  // namespace

// ---------------------------------------------------------------------------
// host plan
// ---------------------------------------------------------------------------
void ml_plan(MLPlan& P, int g, int sub, const int nsub[3], const std::vector<SubDesc>& subs,
             const std::vector<LocalCoarse>& lc, int nc, const std::vector<int>& cptr, const std::vector<int2>& cent) {
  P = MLPlan();
  P.g = g;
  P.sub = sub;
  P.nc = nc;
  const int nb[3] = {(nsub[0] + g - 1) / g, (nsub[1] + g - 1) / g, (nsub[2] + g - 1) / g};
  const int NBk = nb[0] * nb[1] * nb[2];
  P.nblock = NBk;
  const int S = (int)subs.size();
  std::vector<int> bos(S), pos_(S);
  const int nsb = sub > 0 ? (g + sub - 1) / sub : 1;   // sub-blocks per block and axis
  for (int si = 0; si < S; ++si) {
    const int sx = si % nsub[0], sy = (si / nsub[0]) % nsub[1], sz = si / (nsub[0] * nsub[1]);
    bos[si] = sx / g + nb[0] * (sy / g + nb[1] * (sz / g));
    const int local = sub > 0 ? ((sx % g) / sub + nsb * ((sy % g) / sub + nsb * ((sz % g) / sub))) : 0;
    pos_[si] = bos[si] * nsb * nsb * nsb + local;    // sub-block id
  }
  P.bsub_ptr.assign(NBk + 1, 0);
  for (int si = 0; si < S; ++si) ++P.bsub_ptr[bos[si] + 1];
  for (int k = 0; k < NBk; ++k) P.bsub_ptr[k + 1] += P.bsub_ptr[k];
  P.bsub.assign(S, 0);
  {
    std::vector<int> fill(P.bsub_ptr.begin(), P.bsub_ptr.end() - 1);
    for (int si = 0; si < S; ++si) P.bsub[fill[bos[si]]++] = si;
  }
  P.bcolor.resize(NBk);
  for (int k = 0; k < NBk; ++k) {
    const int bx = k % nb[0], by = (k / nb[0]) % nb[1], bz = k / (nb[0] * nb[1]);
    P.bcolor[k] = (bx & 1) + 2 * (by & 1) + 4 * (bz & 1);
  }
  // blocks and sub-blocks sharing each coarse DOF (ascending)
  std::vector<std::vector<int>> bl(nc), pl(nc);
  for (int j = 0; j < nc; ++j) {
    for (int e = cptr[j]; e < cptr[j + 1]; ++e) {
      bl[j].push_back(bos[cent[e].x]);
      pl[j].push_back(pos_[cent[e].x]);
    }
    for (auto* v : {&bl[j], &pl[j]}) {
      std::sort(v->begin(), v->end());
      v->erase(std::unique(v->begin(), v->end()), v->end());
    }
  }
  P.gam2.assign(nc, 0);
  P.w2.assign(nc, 1.0);
  for (int j = 0; j < nc; ++j)
    if (bl[j].size() >= 2) {
      P.gam2[j] = 1;
      P.w2[j] = 1.0 / (double)bl[j].size();
    }
  // block spaces: each block's DOFs ascending, blocks one after the other
  P.bn.assign(NBk, 0);
  for (int j = 0; j < nc; ++j)
    for (int k : bl[j]) ++P.bn[k];
  P.boff.assign(NBk + 1, 0);
  for (int k = 0; k < NBk; ++k) P.boff[k + 1] = P.boff[k] + P.bn[k];
  P.NB = P.boff[NBk];
  P.bgid.assign(P.NB, 0);
  std::vector<int> blk_of_slot(P.NB, 0);
  P.slot_ptr.assign(nc + 1, 0);
  P.slot_ent.clear();
  {
    std::vector<int> cur(P.boff.begin(), P.boff.end() - 1);
    for (int j = 0; j < nc; ++j) {
      for (int k : bl[j]) {
        const int sl = cur[k]++;
        P.bgid[sl] = j;
        blk_of_slot[sl] = k;
        P.slot_ent.push_back(sl);
      }
      P.slot_ptr[j + 1] = (int)P.slot_ent.size();
    }
  }
  auto slot_of = [&](int j, int k) {
    for (int e = P.slot_ptr[j]; e < P.slot_ptr[j + 1]; ++e)
      if (blk_of_slot[P.slot_ent[e]] == k) return P.slot_ent[e];
    throw std::runtime_error("coarse DOF missing from its block");
  };
  // level-1 local coarse entries -> block-space slots
  P.sub2blk.assign(lc.size(), 0);
  for (int si = 0; si < S; ++si) {
    const SubDesc& s = subs[si];
    for (int a = 0; a < s.nc; ++a) P.sub2blk[s.cofs + a] = slot_of(lc[s.cofs + a].gid, bos[si]);
  }
  // block interiors
  P.iidx.assign(P.NB, -1);
  P.bni.assign(NBk, 0);
  P.ioff.assign(NBk + 1, 0);
  P.igid.clear();
  for (int k = 0; k < NBk; ++k) {
    for (int sl = P.boff[k]; sl < P.boff[k + 1]; ++sl)
      if (!P.gam2[P.bgid[sl]]) {
        P.iidx[sl] = P.bni[k]++;
        P.igid.push_back(P.bgid[sl]);
      }
    P.ioff[k + 1] = P.ioff[k] + P.bni[k];
  }
  P.NI = P.ioff[NBk];
  // level-2 objects: Gamma_2 DOFs by sub-block set (the block set without
  // sub-blocks), numbered by first DOF
  std::map<std::vector<int>, int> sets;
  std::vector<std::vector<int>> odofs, oblk;
  for (int j = 0; j < nc; ++j) {
    if (!P.gam2[j]) continue;
    auto it = sets.find(pl[j]);
    if (it == sets.end()) {
      it = sets.emplace(pl[j], (int)odofs.size()).first;
      odofs.emplace_back();
      oblk.push_back(bl[j]);
    }
    odofs[it->second].push_back(j);
  }
  P.ncc = (int)odofs.size();
  // object slots: per block its objects ascending
  std::vector<std::vector<int>> bobj(NBk);
  for (int q = 0; q < P.ncc; ++q)
    for (int k : oblk[q]) bobj[k].push_back(q);
  P.bm.assign(NBk, 0);
  P.ooff.assign(NBk + 1, 0);
  for (int k = 0; k < NBk; ++k) {
    P.bm[k] = (int)bobj[k].size();
    P.ooff[k + 1] = P.ooff[k] + P.bm[k];
    P.maxm = std::max(P.maxm, P.bm[k]);
  }
  P.NO = P.ooff[NBk];
  P.oobj.assign(P.NO, 0);
  std::vector<std::vector<int>> oslots(P.ncc);
  P.orow_ptr.assign(P.NO + 1, 0);
  P.orow_ent.clear();
  for (int k = 0; k < NBk; ++k)
    for (int r = 0; r < P.bm[k]; ++r) {
      const int os = P.ooff[k] + r, q = bobj[k][r];
      P.oobj[os] = q;
      oslots[q].push_back(os);
      for (int j : odofs[q]) P.orow_ent.push_back(slot_of(j, k));
      P.orow_ptr[os + 1] = (int)P.orow_ent.size();
    }
  P.obj_ptr.assign(P.ncc + 1, 0);
  P.obj_ent.clear();
  for (int q = 0; q < P.ncc; ++q) {
    for (int os : oslots[q]) P.obj_ent.push_back(os);   // ascending block: blocks were visited in order
    P.obj_ptr[q + 1] = (int)P.obj_ent.size();
  }
  P.accoff.assign(NBk + 1, 0);
  for (int k = 0; k < NBk; ++k) P.accoff[k + 1] = P.accoff[k] + (long long)P.bm[k] * P.bm[k];
  // fronts
  P.nfront_of.assign(NBk, -1);
  P.dfront_of.assign(NBk, -1);
  int fn = 0, fd = 0;
  for (int k = 0; k < NBk; ++k) {
    if (P.bn[k] > 0) P.nfront_of[k] = fn++;
    if (P.bni[k] > 0) P.dfront_of[k] = fd++;
  }
  mf_plan_independent(P.N, P.bn);
  mf_plan_independent(P.D, P.bni);
  if (P.ncc > 0) {
    // level-2 coarse: nested dissection of the block grid; an object's cell
    // follows from its block set (2b + 1 inside block b, 2b on the plane of
    // blocks b - 1 and b)
    CoarseGeom G;
    int n3[3];
    for (int d = 0; d < 3; ++d) { G.nsub[d] = nb[d]; n3[d] = 2 * nb[d] + 1; }
    const long long ncell = (long long)n3[0] * n3[1] * n3[2];
    std::vector<long long> cellid(P.ncc);
    for (int q = 0; q < P.ncc; ++q) {
      int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-1, -1, -1};
      for (int k : oblk[q]) {
        const int c[3] = {k % nb[0], (k / nb[0]) % nb[1], k / (nb[0] * nb[1])};
        for (int d = 0; d < 3; ++d) { lo[d] = std::min(lo[d], c[d]); hi[d] = std::max(hi[d], c[d]); }
      }
      int cc[3];
      for (int d = 0; d < 3; ++d) cc[d] = lo[d] == hi[d] ? 2 * lo[d] + 1 : 2 * hi[d];
      cellid[q] = cc[0] + (long long)n3[0] * (cc[1] + (long long)n3[1] * cc[2]);
    }
    G.cell_ptr.assign(ncell + 1, 0);
    for (int q = 0; q < P.ncc; ++q) ++G.cell_ptr[cellid[q] + 1];
    for (long long c = 0; c < ncell; ++c) G.cell_ptr[c + 1] += G.cell_ptr[c];
    G.cell_obj.assign(P.ncc, 0);
    std::vector<int> fill(G.cell_ptr.begin(), G.cell_ptr.end() - 1);
    for (int q = 0; q < P.ncc; ++q) G.cell_obj[fill[cellid[q]]++] = q;
    mf_plan(P.C, G, P.ncc);
  }
  P.flops = P.N.flops + P.D.flops + P.C.flops;
  // blocks by colour
  P.color_off.assign(9, 0);
  P.color_cnt.assign(8, 0);
  for (int k = 0; k < NBk; ++k) ++P.color_cnt[P.bcolor[k]];
  for (int c = 0; c < 8; ++c) P.color_off[c + 1] = P.color_off[c] + P.color_cnt[c];
}

// ---------------------------------------------------------------------------
// set-up kernels (one CTA per block)
// ---------------------------------------------------------------------------

// Block matrices from the subdomains' local coarse matrices, summed
// subdomain by subdomain: A_k into front N_k and its interior part into D_k.
__global__ void k_ml_assemble(const SubDesc* __restrict__ subs, const double* __restrict__ Ac,
                              const int* __restrict__ bsub_ptr, const int* __restrict__ bsub,
                              const int* __restrict__ sub2blk, const int* __restrict__ boff, const int* __restrict__ bn,
                              const int* __restrict__ iidx, const int* __restrict__ nfront,
                              const int* __restrict__ dfront, const long long* __restrict__ nfoff,
                              const long long* __restrict__ dfoff, const int* __restrict__ dnp, double* __restrict__ FN,
                              double* __restrict__ FD) {
  const int k = blockIdx.x;
  if (nfront[k] < 0) return;
  const int n = bn[k], b0 = boff[k];
  double* AN = FN + nfoff[nfront[k]];
  const int fd = dfront[k];
  double* AD = fd >= 0 ? FD + dfoff[fd] : nullptr;
  const int nD = fd >= 0 ? dnp[fd] : 0;
  for (int q = bsub_ptr[k]; q < bsub_ptr[k + 1]; ++q) {
    const SubDesc s = subs[bsub[q]];
    const int m = s.nc;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int a = e / m, b = e % m;
      const int pa = sub2blk[s.cofs + a] - b0, pb = sub2blk[s.cofs + b] - b0;
      const double v = Ac[s.offAc + e];
      AN[(long long)pa * n + pb] += v;
      if (AD) {
        const int ia = iidx[b0 + pa], ib = iidx[b0 + pb];
        if (ia >= 0 && ib >= 0) AD[(long long)ia * nD + ib] += v;
      }
    }
    __syncthreads();   // the next subdomain may add to the same entries
  }
}

// rho_k = the largest diagonal entry of A_k, and rho_k c_r^T c_r for every
// constraint row r of the block (objects are disjoint: no entry twice).
__global__ void k_ml_penalty(const int* __restrict__ boff, const int* __restrict__ bn, const int* __restrict__ ooff,
                             const int* __restrict__ bm, const int* __restrict__ orow_ptr,
                             const int* __restrict__ orow_ent, const int* __restrict__ nfront,
                             const long long* __restrict__ nfoff, double* __restrict__ FN, double* __restrict__ rho) {
  __shared__ double red[BDDC_THREADS];
  const int k = blockIdx.x;
  if (nfront[k] < 0) return;
  const int n = bn[k], b0 = boff[k];
  double* A = FN + nfoff[nfront[k]];
  double mx = 0.0;
  for (int p = threadIdx.x; p < n; p += blockDim.x) mx = fmax(mx, A[(long long)p * n + p]);
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  const double rk = red[0];
  if (threadIdx.x == 0) rho[k] = rk;
  for (int r = 0; r < bm[k]; ++r) {
    const int os = ooff[k] + r, r0 = orow_ptr[os], cnt = orow_ptr[os + 1] - r0;
    const double val = rk / ((double)cnt * cnt);
    for (int e = threadIdx.x; e < cnt * cnt; e += blockDim.x) {
      const int p = orow_ent[r0 + e / cnt] - b0, q = orow_ent[r0 + e % cnt] - b0;
      A[(long long)p * n + q] += val;
    }
  }
}

// Level-2 weights per block-space slot: the diagonal of A_k (before the
// augmented terms) into dsl, then w = 1 / (blocks sharing the DOF) or
// dsl / (sum of dsl over the blocks sharing the DOF).
__global__ void k_ml_diag(const int* __restrict__ boff, const int* __restrict__ bn, const int* __restrict__ nfront,
                          const long long* __restrict__ nfoff, const double* __restrict__ FN, double* __restrict__ dsl) {
  const int k = blockIdx.x;
  if (nfront[k] < 0) return;
  const int n = bn[k];
  const double* A = FN + nfoff[nfront[k]];
  for (int p = threadIdx.x; p < n; p += blockDim.x) dsl[boff[k] + p] = A[(long long)p * n + p];
}

__global__ void k_ml_slot_weights(const int* __restrict__ bgid, const int* __restrict__ slot_ptr,
                                  const int* __restrict__ slot_ent, const double* __restrict__ dsl, int stiffness,
                                  double* __restrict__ w, int NB) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < NB; s += gridDim.x * blockDim.x) {
    const int g = bgid[s], e0 = slot_ptr[g], e1 = slot_ptr[g + 1];
    if (!stiffness) { w[s] = 1.0 / (double)(e1 - e0); continue; }
    double sum = 0.0;
    for (int e = e0; e < e1; ++e) sum += dsl[slot_ent[e]];
    w[s] = dsl[s] / sum;
  }
}

// column c of C^T in every block's space (zero where a block has fewer rows)
__global__ void k_ml_rhs_col(const int* __restrict__ boff, const int* __restrict__ bn, const int* __restrict__ ooff,
                             const int* __restrict__ bm, const int* __restrict__ orow_ptr,
                             const int* __restrict__ orow_ent, int c, double* __restrict__ b) {
  const int k = blockIdx.x;
  for (int p = threadIdx.x; p < bn[k]; p += blockDim.x) b[boff[k] + p] = 0.0;
  __syncthreads();
  if (c < bm[k]) {
    const int os = ooff[k] + c, r0 = orow_ptr[os], cnt = orow_ptr[os + 1] - r0;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) b[orow_ent[r0 + e]] = 1.0 / cnt;
  }
}

// S_k = C_k X_k (X_k = N_k^{-1} C_k^T), S_k^{-1} by Cholesky and explicit
// inverse, the level-2 local coarse matrix S_k^{-1} - rho_k I, and
// Psi_k = X_k S_k^{-1}.  X and Psi: column c of every block at c * NB.
__global__ void __launch_bounds__(BDDC_THREADS)
k_ml_schur(const int* __restrict__ boff, const int* __restrict__ bn, const int* __restrict__ ooff,
           const int* __restrict__ bm, const int* __restrict__ orow_ptr, const int* __restrict__ orow_ent,
           const long long* __restrict__ accoff, const double* __restrict__ rho, const double* __restrict__ X, int NB,
           double* __restrict__ Sw, double* __restrict__ Lw, double* __restrict__ Dg, double* __restrict__ Acck,
           double* __restrict__ Psi, int* err) {
  extern __shared__ __align__(128) unsigned char smraw[];
  DenseSmem<double>& sm = *reinterpret_cast<DenseSmem<double>*>(smraw);
  const int k = blockIdx.x, m = bm[k];
  if (m == 0) return;
  const long long o = accoff[k];
  double* S = Sw + o;
  double* Linv = Lw + o;
  double* diag = Dg + 32LL * ooff[k] + 1024LL * k;   // ceil(m/32) 32 x 32 tiles fit in 32 m + 1024
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int r = e / m, c = e % m;
    const int os = ooff[k] + r, r0 = orow_ptr[os], cnt = orow_ptr[os + 1] - r0;
    double s = 0.0;
    for (int q = 0; q < cnt; ++q) s += X[(long long)c * NB + orow_ent[r0 + q]];
    S[e] = s / cnt;
  }
  __syncthreads();
  const bool ok = cta_chol_inv<double>(S, m, Linv, m, m, diag, sm);
  if (!ok && threadIdx.x == 0) set_error(err, 4, k);
  cta_gemm<double>(m, m, m, 1.0, Linv, m, true, Linv, m, false, 0.0, S, m, 2, 2, false, sm);   // S^{-1}
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) Acck[o + e] = S[e] - ((e / m == e % m) ? rho[k] : 0.0);
  const int n = bn[k], b0 = boff[k];
  for (int e = threadIdx.x; e < n * m; e += blockDim.x) {
    const int p = e / m, c = e % m;
    double s = 0.0;
    for (int r = 0; r < m; ++r) s += X[(long long)r * NB + b0 + p] * S[r * m + c];
    Psi[(long long)c * NB + b0 + p] = s;
  }
}

// ---------------------------------------------------------------------------
// apply kernels
// ---------------------------------------------------------------------------
__global__ void k_ml_gather(const int* __restrict__ map, const double* __restrict__ src, double* __restrict__ dst,
                            int n) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) dst[s] = src[map[s]];
}

__global__ void k_ml_scatter(const int* __restrict__ map, const double* __restrict__ src, double* __restrict__ dst,
                             int n) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) dst[map[s]] = src[s];
}

// t_i = A_c^(i) u|_i on every subdomain's local coarse entries
__global__ void k_ml_local_matvec(const SubDesc* __restrict__ subs, const LocalCoarse* __restrict__ lc,
                                  const double* __restrict__ Ac, const double* __restrict__ u, double* __restrict__ tl) {
  const SubDesc s = subs[blockIdx.x];
  const int m = s.nc;
  for (int a = threadIdx.x; a < m; a += blockDim.x) {
    double acc = 0.0;
    const double* row = Ac + s.offAc + (long long)a * m;
    for (int b = 0; b < m; ++b) acc = fma(row[b], u[lc[s.cofs + b].gid], acc);
    tl[s.cofs + a] = acc;
  }
}

// r_k = D_2 R_k (r_c - A_c u_I) on Gamma_2, zero inside the blocks
__global__ void k_ml_block_rhs(const int* __restrict__ bgid, const unsigned char* __restrict__ gam2,
                               const double* __restrict__ w2s, const double* __restrict__ rc,
                               const double* __restrict__ t, double* __restrict__ rb, int NB) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < NB; s += gridDim.x * blockDim.x) {
    const int g = bgid[s];
    rb[s] = gam2[g] ? w2s[s] * (rc[g] - t[g]) : 0.0;
  }
}

// Psi_k^T r_k per object slot, a warp per row (fixed order)
__global__ void k_ml_psiT(const int* __restrict__ boff, const int* __restrict__ bn, const int* __restrict__ ooff,
                          const int* __restrict__ bm, const double* __restrict__ Psi, int NB,
                          const double* __restrict__ rb, double* __restrict__ rs) {
  const int k = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int n = bn[k], b0 = boff[k];
  for (int c = warp; c < bm[k]; c += nw) {
    double acc = 0.0;
    for (int p = lane; p < n; p += 32) acc = fma(Psi[(long long)c * NB + b0 + p], rb[b0 + p], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) rs[ooff[k] + c] = acc;
  }
}

// dst[i] = sum over ent[ptr[i] .. ptr[i+1]) of w[ent] src[ent] (w NULL: 1;
// mask: 0 -> dst 0), in the order of the list
__global__ void k_ml_csr_sum(const int* __restrict__ ptr, const int* __restrict__ ent, const double* __restrict__ src,
                             const double* __restrict__ w, const unsigned char* __restrict__ mask,
                             double* __restrict__ dst, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (mask && !mask[i]) { dst[i] = 0.0; continue; }
    double s = 0.0;
    for (int e = ptr[i]; e < ptr[i + 1]; ++e) s += (w ? w[ent[e]] : 1.0) * src[ent[e]];
    dst[i] = s;
  }
}

// v_k = Psi_k (u_cc|_k - C_k y_k) + y_k, y_k = N_k^{-1} r_k
__global__ void k_ml_block_finish(const int* __restrict__ boff, const int* __restrict__ bn,
                                  const int* __restrict__ ooff, const int* __restrict__ bm,
                                  const int* __restrict__ orow_ptr, const int* __restrict__ orow_ent,
                                  const int* __restrict__ oobj, const double* __restrict__ Psi, int NB,
                                  const double* __restrict__ ucc, const double* __restrict__ y,
                                  double* __restrict__ v) {
  extern __shared__ double dsh[];
  const int k = blockIdx.x, m = bm[k], n = bn[k], b0 = boff[k];
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
    const int os = ooff[k] + r, r0 = orow_ptr[os], cnt = orow_ptr[os + 1] - r0;
    double s = 0.0;
    for (int q = 0; q < cnt; ++q) s += y[orow_ent[r0 + q]];
    dsh[r] = ucc[oobj[os]] - s / cnt;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    double acc = y[b0 + p];
    for (int r = 0; r < m; ++r) acc = fma(Psi[(long long)r * NB + b0 + p], dsh[r], acc);
    v[b0 + p] = acc;
  }
}

// u_c = v_Gamma on Gamma_2 (zero inside), then u_I - A_II^{-1} A_IGamma v_Gamma inside
__global__ void k_ml_combine(const int* __restrict__ igid, const double* __restrict__ uIb,
                             const double* __restrict__ sI, double* __restrict__ uc, int NI) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < NI; s += gridDim.x * blockDim.x)
    uc[igid[s]] = uIb[s] - sI[s];
}

// ---------------------------------------------------------------------------
// host drivers
// ---------------------------------------------------------------------------
namespace {
inline int grid_of_n(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 4096)); }
}  // namespace

void ml_setup(MLPlan& P, const LocalLaunch& L, const std::function<void*(size_t)>& alloc,
              const std::function<void*(size_t)>& tmp_alloc, int stiffness, int* err, cudaStream_t st) {
  const int NBk = P.nblock;
  P.d_boff = up(P.boff, alloc, st);
  P.d_bn = up(P.bn, alloc, st);
  P.d_ooff = up(P.ooff, alloc, st);
  P.d_bm = up(P.bm, alloc, st);
  P.d_bsub_ptr = up(P.bsub_ptr, alloc, st);
  P.d_bsub = up(P.bsub, alloc, st);
  P.d_bgid = up(P.bgid, alloc, st);
  P.d_iidx = up(P.iidx, alloc, st);
  P.d_igid = up(P.igid, alloc, st);
  P.d_slot_ptr = up(P.slot_ptr, alloc, st);
  P.d_slot_ent = up(P.slot_ent, alloc, st);
  P.d_oobj = up(P.oobj, alloc, st);
  P.d_obj_ptr = up(P.obj_ptr, alloc, st);
  P.d_obj_ent = up(P.obj_ent, alloc, st);
  P.d_orow_ptr = up(P.orow_ptr, alloc, st);
  P.d_orow_ent = up(P.orow_ent, alloc, st);
  P.d_sub2blk = up(P.sub2blk, alloc, st);
  P.d_nfront = up(P.nfront_of, alloc, st);
  P.d_dfront = up(P.dfront_of, alloc, st);
  P.d_gam2 = up(P.gam2, alloc, st);
  P.d_w2 = up(P.w2, alloc, st);
  P.d_accoff = up(P.accoff, alloc, st);
  {
    std::vector<int> lst;
    for (int c = 0; c < 8; ++c)
      for (int k = 0; k < NBk; ++k)
        if (P.bcolor[k] == c) lst.push_back(k);
    P.d_bcolor_list = up(lst, alloc, st);
  }
  configure_mf_kernels();
  mf_upload(P.N, alloc, tmp_alloc, st);
  mf_upload(P.D, alloc, tmp_alloc, st);
  if (P.ncc > 0) mf_upload(P.C, alloc, tmp_alloc, st);
  P.rho = (double*)alloc(sizeof(double) * std::max(NBk, 1));
  // block matrices, their augmented terms and factors
  BDDC_COUNT(2);
  k_ml_assemble<<<NBk, BDDC_THREADS, 0, st>>>(L.subs, L.Ac, P.d_bsub_ptr, P.d_bsub, P.d_sub2blk, P.d_boff, P.d_bn,
                                             P.d_iidx, P.d_nfront, P.d_dfront, P.N.d_foff, P.D.d_foff, P.D.d_np,
                                             P.N.F, P.D.F);
  {
    double* dsl = (double*)tmp_alloc(sizeof(double) * (size_t)std::max(P.NB, 1));
    P.w2s = (double*)alloc(sizeof(double) * (size_t)std::max(P.NB, 1));
    BDDC_COUNT(2);
    k_ml_diag<<<NBk, BDDC_THREADS, 0, st>>>(P.d_boff, P.d_bn, P.d_nfront, P.N.d_foff, P.N.F, dsl);
    k_ml_slot_weights<<<grid_of_n(P.NB), 256, 0, st>>>(P.d_bgid, P.d_slot_ptr, P.d_slot_ent, dsl, stiffness, P.w2s,
                                                       P.NB);
  }
  k_ml_penalty<<<NBk, BDDC_THREADS, 0, st>>>(P.d_boff, P.d_bn, P.d_ooff, P.d_bm, P.d_orow_ptr, P.d_orow_ent,
                                            P.d_nfront, P.N.d_foff, P.N.F, P.rho);
  mf_factor(P.N, err, st, nullptr, nullptr, nullptr);
  mf_factor(P.D, err, st, nullptr, nullptr, nullptr);
  // X = N^{-1} C^T, column by column for all blocks at once
  const long long NB = std::max(P.NB, 1);
  P.X = (double*)tmp_alloc(sizeof(double) * (size_t)NB * std::max(P.maxm, 1));
  P.Psi = (double*)alloc(sizeof(double) * (size_t)NB * std::max(P.maxm, 1));
  double* bcol = (double*)tmp_alloc(sizeof(double) * (size_t)NB);
  for (int c = 0; c < P.maxm; ++c) {
    BDDC_COUNT(1);
    k_ml_rhs_col<<<NBk, BDDC_THREADS, 0, st>>>(P.d_boff, P.d_bn, P.d_ooff, P.d_bm, P.d_orow_ptr, P.d_orow_ent, c,
                                              bcol);
    mf_solve(P.N, bcol, P.X + (size_t)c * NB, P.N.W, st);
  }
  // level-2 local coarse matrices and bases
  const long long nacc = std::max<long long>(P.accoff[NBk], 1);
  double* Sw = (double*)tmp_alloc(sizeof(double) * (size_t)nacc);
  double* Lw = (double*)tmp_alloc(sizeof(double) * (size_t)nacc);
  double* Dg = (double*)tmp_alloc(sizeof(double) * (32 * (size_t)std::max(P.NO, 1) + 1024 * (size_t)NBk));
  P.Acck = (double*)tmp_alloc(sizeof(double) * (size_t)nacc);
  if (P.maxm > 0) {
    const size_t sm = sizeof(DenseSmem<double>);
    cudaFuncSetAttribute(k_ml_schur, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    BDDC_COUNT(1);
    k_ml_schur<<<NBk, BDDC_THREADS, sm, st>>>(P.d_boff, P.d_bn, P.d_ooff, P.d_bm, P.d_orow_ptr, P.d_orow_ent,
                                             P.d_accoff, P.rho, P.X, (int)NB, Sw, Lw, Dg, P.Acck, P.Psi, err);
  }
  if (P.ncc > 0) {
    // S_k^{-1} - rho_k I into the level-2 fronts, one colour of blocks at a time
    for (int c = 0; c < 8; ++c)
      mf_add_local(P.C, P.d_bcolor_list + P.color_off[c], P.color_cnt[c], P.d_ooff, P.d_bm, P.d_accoff, P.d_oobj,
                   P.Acck, st);
    mf_factor(P.C, err, st, nullptr, nullptr, nullptr);
  }
  // apply work vectors
  const size_t nc = std::max(P.nc, 1), ni = std::max(P.NI, 1), no = std::max(P.NO, 1),
               ncc = std::max(P.ncc, 1);
  P.bI = (double*)alloc(sizeof(double) * ni);
  P.uIb = (double*)alloc(sizeof(double) * ni);
  P.sI = (double*)alloc(sizeof(double) * ni);
  P.u = (double*)alloc(sizeof(double) * nc);
  P.tl = (double*)alloc(sizeof(double) * std::max<size_t>(P.sub2blk.size(), 1));
  P.t = (double*)alloc(sizeof(double) * nc);
  P.rb = (double*)alloc(sizeof(double) * (size_t)NB);
  P.y = (double*)alloc(sizeof(double) * (size_t)NB);
  P.v = (double*)alloc(sizeof(double) * (size_t)NB);
  P.rs = (double*)alloc(sizeof(double) * no);
  P.rcc = (double*)alloc(sizeof(double) * ncc);
  P.ucc = (double*)alloc(sizeof(double) * ncc);
  P.vg = (double*)alloc(sizeof(double) * nc);
}

// u_c = M2 r_c: the coarse level's BDDC preconditioner (Definition 1)
void ml_apply(const MLPlan& P, const LocalLaunch& L, const int* cptr, const int2* cent, const double* rc, double* uc,
              cudaStream_t st) {
  const int NBk = P.nblock, nc = P.nc;
  // V1: u_I = A_II^{-1} r_I, block by block
  if (P.NI > 0) {
    BDDC_COUNT(1);
    k_ml_gather<<<grid_of_n(P.NI), 256, 0, st>>>(P.d_igid, rc, P.bI, P.NI);
    mf_solve(P.D, P.bI, P.uIb, P.D.W, st);
  }
  cudaMemsetAsync(P.u, 0, sizeof(double) * (size_t)nc, st);
  if (P.NI > 0) {
    BDDC_COUNT(1);
    k_ml_scatter<<<grid_of_n(P.NI), 256, 0, st>>>(P.d_igid, P.uIb, P.u, P.NI);
  }
  // r_k = D_2 R_k (r_c - A_c u_I)
  BDDC_COUNT(2);
  k_ml_local_matvec<<<L.nsub, BDDC_THREADS, 0, st>>>(L.subs, L.lc, L.Ac, P.u, P.tl);
  launch_coarse_gather(cptr, cent, P.tl, P.t, nc, st);
  k_ml_block_rhs<<<grid_of_n(P.NB), 256, 0, st>>>(P.d_bgid, P.d_gam2, P.w2s, rc, P.t, P.rb, P.NB);
  // level-2 coarse correction
  if (P.ncc > 0) {
    BDDC_COUNT(2);
    k_ml_psiT<<<NBk, BDDC_THREADS, 0, st>>>(P.d_boff, P.d_bn, P.d_ooff, P.d_bm, P.Psi, std::max(P.NB, 1), P.rb,
                                           P.rs);
    k_ml_csr_sum<<<grid_of_n(P.ncc), 256, 0, st>>>(P.d_obj_ptr, P.d_obj_ent, P.rs, nullptr, nullptr, P.rcc, P.ncc);
    mf_solve(P.C, P.rcc, P.ucc, P.C.W, st);
  }
  // constrained block problems and v_k = Psi_k (u_cc - C_k y) + y
  mf_solve(P.N, P.rb, P.y, P.N.W, st);
  BDDC_COUNT(2);
  k_ml_block_finish<<<NBk, BDDC_THREADS, sizeof(double) * std::max(P.maxm, 1), st>>>(
      P.d_boff, P.d_bn, P.d_ooff, P.d_bm, P.d_orow_ptr, P.d_orow_ent, P.d_oobj, P.Psi, std::max(P.NB, 1), P.ucc,
      P.y, P.v);
  // v_Gamma = sum_k R_k^T D_2 v_k, then the harmonic extension into the blocks
  k_ml_csr_sum<<<grid_of_n(nc), 256, 0, st>>>(P.d_slot_ptr, P.d_slot_ent, P.v, P.w2s, P.d_gam2, uc, nc);
  if (P.NI > 0) {
    BDDC_COUNT(4);
    k_ml_local_matvec<<<L.nsub, BDDC_THREADS, 0, st>>>(L.subs, L.lc, L.Ac, uc, P.tl);
    launch_coarse_gather(cptr, cent, P.tl, P.t, nc, st);
    k_ml_gather<<<grid_of_n(P.NI), 256, 0, st>>>(P.d_igid, P.t, P.bI, P.NI);
    mf_solve(P.D, P.bI, P.sI, P.D.W, st);
    k_ml_combine<<<grid_of_n(P.NI), 256, 0, st>>>(P.d_igid, P.uIb, P.sI, uc, P.NI);
  }
}

}  // namespace bddc
