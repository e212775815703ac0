// Multifrontal FP64 Cholesky of the BDDC-SO coarse matrix.
//
// The coarse DOFs are the (sub)objects of Theta-hat on Gamma (Section 3); two
// of them are coupled only through a shared subdomain, and the paper points at
// the size of this coarse problem as BDDC-SO's cost (Sections 1 and 6).  The
// elimination order is a nested dissection of the box-subdomain grid: a box of
// subdomains is split at its middle Theta plane along its longest axis; the
// objects on that plane strictly inside the box are the box's pivots (its
// separator), eliminated after both halves.  A front holds its pivots P and
// the objects on the closed box boundary U (all eliminated later); the
// objects a front's pivots couple to after elimination lie in P u U.
//
// Numeric phase, tree level by tree level (deepest first): extend-add of the
// children's update matrices, then a tiled right-looking partial Cholesky of
// every front of the level at once (potrf of the 32x32 diagonal tile with its
// explicit inverse, trsm of the tiles below it, syrk of the trailing tiles,
// which include the update block U x U).  Afterwards every front gets its
// solve matrix [Linv_P; G] with Linv_P = L_P^{-1} (recursive doubling over
// the diagonal tiles' inverses, all fronts at once: for L = [[A, 0], [B, C]],
// L^{-1} has the off-diagonal block -C^{-1} B A^{-1}) and G = L_UP Linv_P, so each
// level of a triangular solve is one parallel mat-vec over all the level's
// fronts (rows split across CTAs forward, columns backward).  Everything is
// summed in a fixed order (no atomics).
#include <array>
#include <cstdint>
#include <stdexcept>
#include <string>

#include "common.cuh"
#include "dense.cuh"
#include "kernels.h"

namespace bddc {

// Factor tiles are 32 wide: FP64 issue on this GPU is about two FMAs per
// clock per SM, so a 64-wide tile step on one CTA would be long and the
// chain of diagonal-tile steps short of parallel work.  Both solves are row
// dot products (forward on S_f, backward on its transpose) in chunks of FSR
// rows, so a level spreads over many CTAs.
constexpr int FNB = 32;
constexpr int FSR = 8;    // rows per CTA in the solves, one per warp

__host__ __device__ inline int mf_ntiles(int np, int nu) { return (np + FNB - 1) / FNB + (nu + FNB - 1) / FNB; }
__host__ __device__ inline void mf_tile(int t, int np, int nu, int& r0, int& nr) {
  const int npt = (np + FNB - 1) / FNB;
  if (t < npt) { r0 = t * FNB; nr = min(FNB, np - r0); }
  else { int u = t - npt; r0 = np + u * FNB; nr = min(FNB, nu - u * FNB); }
}

// ---------------------------------------------------------------------------
// symbolic analysis (host)
// ---------------------------------------------------------------------------
namespace {

struct Box { int s0[3], s1[3]; };

struct Builder {
  const CoarseGeom& g;
  MFPlan& P;
  int nc3[3];
  std::vector<std::vector<int>> piv, upd;   // per front
  std::vector<std::vector<int>> children;
  std::vector<int> depth;
  Builder(const CoarseGeom& g_, MFPlan& P_) : g(g_), P(P_) {
    for (int d = 0; d < 3; ++d) nc3[d] = 2 * g.nsub[d] + 1;
  }

  // objects of one cell, ascending
  void cell(int cx, int cy, int cz, std::vector<int>& out) const {
    const long long c = cx + (long long)nc3[0] * (cy + (long long)nc3[1] * cz);
    for (int q = g.cell_ptr[c]; q < g.cell_ptr[c + 1]; ++q) out.push_back(g.cell_obj[q]);
  }

  // creates the fronts of this box and of its descendants; the ids of the
  // fronts without a parent inside the box are collected into `kids`
  void build(const Box& b, std::vector<int>& kids) {
    int ext[3] = {b.s1[0] - b.s0[0], b.s1[1] - b.s0[1], b.s1[2] - b.s0[2]};
    if (ext[0] <= 1 && ext[1] <= 1 && ext[2] <= 1) return;
    int ax = 0;
    for (int d = 1; d < 3; ++d)
      if (ext[d] > ext[ax]) ax = d;
    const int mid = b.s0[ax] + ext[ax] / 2;
    int lo[3], hi[3];   // closed cell range of the box
    for (int d = 0; d < 3; ++d) { lo[d] = 2 * b.s0[d]; hi[d] = 2 * b.s1[d]; }
    // separator: cells on the cut plane of `mid`, strictly inside the box
    std::vector<int> sep;
    {
      int a1 = (ax + 1) % 3, a2 = (ax + 2) % 3;
      int c[3];
      c[ax] = 2 * mid;
      for (int j = lo[a2] + 1; j < hi[a2]; ++j)
        for (int i = lo[a1] + 1; i < hi[a1]; ++i) {
          c[a1] = i; c[a2] = j;
          cell(c[0], c[1], c[2], sep);
        }
    }
    Box c0 = b, c1 = b;
    c0.s1[ax] = mid;
    c1.s0[ax] = mid;
    std::vector<int> my_kids;
    build(c0, my_kids);
    build(c1, my_kids);
    if (sep.empty()) {  // nothing to eliminate here: the children attach to the ancestor
      for (int k : my_kids) kids.push_back(k);
      return;
    }
    // update set: objects in the cells of the closed box boundary
    std::vector<int> u;
    for (int cz = lo[2]; cz <= hi[2]; ++cz)
      for (int cy = lo[1]; cy <= hi[1]; ++cy) {
        const bool yz_bnd = cy == lo[1] || cy == hi[1] || cz == lo[2] || cz == hi[2];
        for (int cx = lo[0]; cx <= hi[0]; cx = (yz_bnd || cx == hi[0]) ? cx + 1 : hi[0]) cell(cx, cy, cz, u);
      }
    std::sort(u.begin(), u.end());
    const int f = (int)piv.size();
    piv.push_back(sep);
    upd.push_back(u);
    children.push_back(my_kids);
    depth.push_back(0);
    kids.push_back(f);
  }
};


}  // namespace

namespace {
// The numeric plan of a front tree: pivots and update sets per front, the
// children of every front, and the fronts without a parent (depth 0).
struct FrontTree {
  std::vector<std::vector<int>> piv, upd, children;
  std::vector<int> depth;
};

void set_tree_depth(FrontTree& B, int f, int d) {
  B.depth[f] = d;
  for (int c : B.children[f]) set_tree_depth(B, c, d + 1);
}

void mf_plan_tree(MFPlan& P, FrontTree& B, const std::vector<int>& tops, int nc);
}  // namespace

void mf_plan(MFPlan& P, const CoarseGeom& g, int nc) {
  P = MFPlan();
  P.nc = nc;
  if (nc == 0) return;
  Builder Bd(g, P);
  Box root;
  for (int d = 0; d < 3; ++d) { root.s0[d] = 0; root.s1[d] = g.nsub[d]; }
  std::vector<int> tops;
  Bd.build(root, tops);
  FrontTree T;
  T.piv = std::move(Bd.piv);
  T.upd = std::move(Bd.upd);
  T.children = std::move(Bd.children);
  T.depth = std::move(Bd.depth);
  mf_plan_tree(P, T, tops, nc);
}

// Independent dense fronts: front k eliminates ids off_k .. off_k + size_k - 1
// (consecutive, in order) and updates nothing; all at depth 0, factored side
// by side, and one solve treats every front at once.
void mf_plan_independent(MFPlan& P, const std::vector<int>& sizes) {
  P = MFPlan();
  int nc = 0;
  for (int n : sizes) nc += n;
  P.nc = nc;
  if (nc == 0) return;
  FrontTree T;
  std::vector<int> tops;
  int off = 0;
  for (int n : sizes) {
    if (n == 0) continue;
    std::vector<int> pv(n);
    for (int q = 0; q < n; ++q) pv[q] = off + q;
    off += n;
    tops.push_back((int)T.piv.size());
    T.piv.push_back(std::move(pv));
    T.upd.emplace_back();
    T.children.emplace_back();
    T.depth.push_back(0);
  }
  mf_plan_tree(P, T, tops, nc);
}

namespace {
void mf_plan_tree(MFPlan& P, FrontTree& B, const std::vector<int>& tops, int nc) {
  const int nf = (int)B.piv.size();
  P.nfront = nf;
  P.parent.assign(nf, -1);
  P.child_slot.assign(nf, 0);
  for (int f = 0; f < nf; ++f)
    for (size_t k = 0; k < B.children[f].size(); ++k) {
      P.parent[B.children[f][k]] = f;
      P.child_slot[B.children[f][k]] = (int)k;
    }
  for (int t : tops) set_tree_depth(B, t, 0);
  // several top fronts can exist only if the root box had no separator; they
  // are independent and all sit at depth 0
  P.level_of = B.depth;
  P.nlevel = 0;
  for (int f = 0; f < nf; ++f) P.nlevel = std::max(P.nlevel, P.level_of[f] + 1);
  P.fronts_at_level.assign(P.nlevel, {});
  for (int f = 0; f < nf; ++f) P.fronts_at_level[P.level_of[f]].push_back(f);
  // elimination order: fronts are created in post-order (children first)
  P.ord.assign(nc, -1);
  P.fr.assign(nc, -1);
  P.pp.assign(nc, -1);
  int pos = 0;
  P.np.resize(nf);
  P.nu.resize(nf);
  P.foff.resize(nf);
  P.doff.resize(nf);
  P.woff.resize(nf);
  P.gid_off.resize(nf + 1);
  long long fo = 0, dof = 0, wo = 0;
  P.gid_off[0] = 0;
  for (int f = 0; f < nf; ++f) {
    for (size_t k = 0; k < B.piv[f].size(); ++k) {
      int o = B.piv[f][k];
      if (P.fr[o] != -1) throw std::runtime_error("coarse object in two separators");
      P.ord[o] = pos++;
      P.fr[o] = f;
      P.pp[o] = (int)k;
    }
    P.np[f] = (int)B.piv[f].size();
    P.nu[f] = (int)B.upd[f].size();
    const long long F = P.np[f] + P.nu[f];
    P.foff[f] = fo; fo += F * F;
    P.doff[f] = dof; dof += (long long)((P.np[f] + FNB - 1) / FNB) * FNB * FNB;
    P.woff[f] = wo; wo += F;
    for (int o : B.piv[f]) P.gid.push_back(o);
    for (int o : B.upd[f]) P.gid.push_back(o);
    P.gid_off[f + 1] = (long long)P.gid.size();
    // partial factorisation, in multiply-adds: Cholesky of the pivot block
    // np^3/6, the panel solve L_UP = A_UP L_P^-T nu np^2/2, the update of the
    // U block nu^2 np/2
    const double np = P.np[f], nu = P.nu[f];
    P.flops += np * np * np / 6.0 + nu * np * np / 2.0 + nu * nu * np / 2.0;
  }
  if (pos != nc) throw std::runtime_error("nested dissection missed coarse objects");
  P.fpool = fo; P.dpool = dof; P.wpool = wo;
  // solve matrices and the work lists that build them
  P.soff.resize(nf);
  long long so = 0;
  for (int f = 0; f < nf; ++f) {
    P.soff[f] = so;
    so += (long long)(P.np[f] + P.nu[f]) * P.np[f];
  }
  P.spool = so;
  P.inv_items.assign(P.nlevel, std::vector<std::vector<int>>(2));
  // output tiles of the doubling steps {front, r, c, k0, k1}, by level and
  // (step, mode)
  std::vector<std::vector<std::vector<std::array<int, 5>>>> raw(P.nlevel);
  P.toff.resize(nf);
  long long to = 0;
  for (int f = 0; f < nf; ++f) {
    const int npt = (P.np[f] + FNB - 1) / FNB, nut = (P.nu[f] + FNB - 1) / FNB;
    P.toff[f] = to;
    to += (long long)P.np[f] * P.np[f];
    std::vector<std::vector<int>>& lv = P.inv_items[P.level_of[f]];
    for (int t = 0; t < npt; ++t) lv[0].insert(lv[0].end(), {f, t, t, 0});
    // doubling: blocks of 2 hb tiles, A = first hb tiles, C = the rest.  Each
    // output tile (r, c) is a sum of tile products over a K range (mode 0:
    // k in [c, cstart), mode 1: k in [cstart, r]); one CTA per product
    // (lists 2 + 4q + {0, 2}) and one per output tile summing the products
    // in order (lists 2 + 4q + {1, 3}), so the long sums of the last steps
    // spread over many SMs and the result does not depend on scheduling.
    int q = 0;
    for (int hb = 1; hb < npt; hb *= 2, ++q) {
      while ((int)lv.size() < 2 + 4 * (q + 1)) lv.emplace_back();
      if ((int)raw[P.level_of[f]].size() < 2 * (q + 1)) raw[P.level_of[f]].resize(2 * (q + 1));
      for (int b0 = 0; b0 + hb < npt; b0 += 2 * hb) {
        const int cstart = b0 + hb;
        for (int r = cstart; r < std::min(b0 + 2 * hb, npt); ++r)
          for (int c = b0; c < cstart; ++c)
            for (int mode = 0; mode < 2; ++mode) {
              const int k0 = mode ? cstart : c, k1 = mode ? r + 1 : cstart;
              raw[P.level_of[f]][2 * q + mode].push_back({f, r, c, k0, k1});
            }
      }
    }
    for (int u = 0; u < nut; ++u)
      for (int s2 = 0; s2 < npt; ++s2) lv[1].insert(lv[1].end(), {f, u, s2, 0});
    // solve matrices: Linv_P = L_P^-1 (np^3/6), G = L_UP Linv_P (nu np^2/2)
    P.flops += (double)P.np[f] * P.np[f] * P.np[f] / 6.0 + (double)P.nu[f] * P.np[f] * P.np[f] / 2.0;
  }
  P.tpool = to;
  // products over K chunks of ks tiles, ks chosen per list so that it has at
  // most about 2048 products besides one per output tile
  for (int l = 0; l < P.nlevel; ++l)
    for (size_t qm = 0; qm < raw[l].size(); ++qm) {
      long long total = 0;
      for (const auto& t : raw[l][qm]) total += t[4] - t[3];
      const int ks = (int)std::max<long long>(1, (total + 2047) / 2048);
      std::vector<int>& parts = P.inv_items[l][2 + 2 * qm];
      std::vector<int>& sums = P.inv_items[l][2 + 2 * qm + 1];
      for (const auto& t : raw[l][qm]) {
        const int first = (int)parts.size() / 4;
        int cnt = 0;
        for (int k = t[3]; k < t[4]; k += ks, ++cnt) parts.insert(parts.end(), {t[0], t[1], t[2], k | (std::min(ks, t[4] - k) << 16)});
        sums.insert(sums.end(), {t[0], (t[1] << 16) | t[2], first, cnt});
      }
    }
  // child update rows -> positions in the parent front: a table of each
  // object's position in the current parent, stamped with the parent's id
  P.pmap_off.assign(nf + 1, 0);
  {
    std::vector<long long> cnt(nf + 1, 0);
    for (int f = 0; f < nf; ++f) cnt[f + 1] = cnt[f] + (P.parent[f] >= 0 ? (long long)B.upd[f].size() : 0);
    P.pmap_off = cnt;
    P.pmap.assign(cnt[nf], 0);
    std::vector<int> pos(nc, -1), stamp(nc, -1);
    std::vector<std::vector<int>> kids_of(nf);
    for (int f = 0; f < nf; ++f)
      if (P.parent[f] >= 0) kids_of[P.parent[f]].push_back(f);
    for (int p = 0; p < nf; ++p) {
      if (kids_of[p].empty()) continue;
      const int* gp = P.gid.data() + P.gid_off[p];
      const int Fp = P.np[p] + P.nu[p];
      for (int q = 0; q < Fp; ++q) { pos[gp[q]] = q; stamp[gp[q]] = p; }
      for (int c : kids_of[p]) {
        long long w = P.pmap_off[c];
        for (int o : B.upd[c]) {
          if (stamp[o] != p) throw std::runtime_error("update set not nested in the parent front");
          P.pmap[w++] = pos[o];
        }
      }
    }
  }
  // front tables per (level, panel step): the trsm items of front f at step j
  // are the tiles i = j+1 .. nt-1 below the panel, the syrk items the pairs
  // j+1 <= k <= i < nt of the trailing lower triangle
  P.step_fronts.clear(); P.step_j.clear(); P.step_ntr.clear(); P.step_nsy.clear();
  for (int l = P.nlevel - 1; l >= 0; --l) {
    int maxpt = 0;
    for (int f : P.fronts_at_level[l]) maxpt = std::max(maxpt, (P.np[f] + FNB - 1) / FNB);
    for (int j = 0; j < maxpt; ++j) {
      std::vector<int> tab;
      long long ntr = 0, nsy = 0;
      for (int f : P.fronts_at_level[l]) {
        const int npt = (P.np[f] + FNB - 1) / FNB, nt = mf_ntiles(P.np[f], P.nu[f]);
        if (j >= npt) continue;
        const long long m = nt - j - 1;
        tab.insert(tab.end(), {f, nt, (int)ntr, (int)nsy});
        ntr += m;
        nsy += m * (m + 1) / 2;
      }
      if (nsy > INT32_MAX) throw std::runtime_error("coarse front too large for one panel step");
      P.step_fronts.push_back(tab);
      P.step_j.push_back(j);
      P.step_ntr.push_back((int)ntr);
      P.step_nsy.push_back((int)nsy);
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// device kernels
// ---------------------------------------------------------------------------
struct MFDev {
  const int *np, *nu, *gid, *fr, *pp, *ord, *pmap, *parent;
  const long long *foff, *doff, *woff, *gid_off, *pmap_off, *soff, *toff;
  double *F, *Dinv, *W, *S, *T, *ST;
};

// One FNB x FNB FP64 output tile on one CTA of 256 threads (a 16 x 16 grid,
// FNB/16 rows by FNB/16 columns per thread): C = beta C + alpha sum_k
// A[i][k] op(B)[k][j] with op(B)[k][j] = B[k][j] (TB false) or B[j][k] (TB
// true), k < K, row-major operands; with lower only j <= i is written.
// m, n <= FNB.  K runs in FNB-deep slices staged in shared memory (As, Bs:
// FNB x (FNB + 1) each); at two FP64 FMAs per clock per SM the slice's
// arithmetic hides its loads, so every warp computes rather than blocking
// registers.  beta = 0 does not read C.
static_assert(FNB == 16 || FNB == 32, "tile width: 16 or 32");
template <bool TB>
__device__ void tile_gemm_f64(int m, int n, int K, double alpha, const double* __restrict__ A, long long lda,
                              const double* __restrict__ B, long long ldb, double beta, double* C, long long ldc,
                              bool lower, double* As, double* Bs) {
  constexpr int TP = FNB / 16, LD = FNB + 1;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  double acc[TP][TP];
#pragma unroll
  for (int a = 0; a < TP; ++a)
#pragma unroll
    for (int b = 0; b < TP; ++b) acc[a][b] = 0.0;
  for (int k0 = 0; k0 < K; k0 += FNB) {
    const int kb = min(FNB, K - k0);
    for (int idx = tid; idx < FNB * FNB; idx += BDDC_THREADS) {
      const int r = idx / FNB, kk = idx % FNB;
      As[r * LD + kk] = (r < m && kk < kb) ? A[r * lda + k0 + kk] : 0.0;
      if (TB) Bs[kk * LD + r] = (r < n && kk < kb) ? B[r * ldb + k0 + kk] : 0.0;
      else Bs[r * LD + kk] = (r < kb && kk < n) ? B[(long long)(k0 + r) * ldb + kk] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < FNB; ++kk) {
      double av[TP], bv[TP];
#pragma unroll
      for (int q = 0; q < TP; ++q) {
        av[q] = As[(TP * ty + q) * LD + kk];
        bv[q] = Bs[kk * LD + tx + 16 * q];
      }
#pragma unroll
      for (int a = 0; a < TP; ++a)
#pragma unroll
        for (int b = 0; b < TP; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < TP; ++a)
#pragma unroll
    for (int b = 0; b < TP; ++b) {
      const int r = TP * ty + a, c = tx + 16 * b;
      if (r < m && c < n && (!lower || c <= r)) {
        double* p = C + r * ldc + c;
        *p = (beta == 0.0) ? alpha * acc[a][b] : fma(beta, *p, alpha * acc[a][b]);
      }
    }
}

__device__ inline int mf_pos(const MFDev& d, int f, int o) {
  if (d.fr[o] == f) return d.pp[o];
  const int np = d.np[f], nu = d.nu[f];
  const int* ub = d.gid + d.gid_off[f] + np;
  int lo = 0, hi = nu - 1;
  while (lo <= hi) {
    int m = (lo + hi) >> 1;
    int v = ub[m];
    if (v == o) return np + m;
    if (v < o) lo = m + 1; else hi = m - 1;
  }
  return -1;  // not reached for a consistent plan
}

// original entries of the subdomain coarse matrices, one launch per colour
__global__ void k_mf_assemble(MFDev d, const SubDesc* __restrict__ subs, const LocalCoarse* __restrict__ lc,
                              const int* __restrict__ list, const double* __restrict__ Ac) {
  const SubDesc s = subs[list[blockIdx.x]];
  const int n = s.nc;
  // the fronts are factored from their lower triangles only: entry (a, b),
  // b <= a, goes to the lower of its two front positions; rows over the
  // warps, the lanes along a row
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int a = blockIdx.y * nw + warp; a < n; a += gridDim.y * nw) {
    const int ga = lc[s.cofs + a].gid;
    for (int b = lane; b <= a; b += 32) {
      const int gb = lc[s.cofs + b].gid;
      const int f = d.fr[d.ord[ga] <= d.ord[gb] ? ga : gb];
      const int ra = mf_pos(d, f, ga), rb = mf_pos(d, f, gb);
      if (ra < 0 || rb < 0) continue;
      const long long F = d.np[f] + d.nu[f];
      d.F[d.foff[f] + (long long)max(ra, rb) * F + min(ra, rb)] += Ac[s.offAc + (long long)a * n + b];
    }
  }
}

// Dense local matrices added into the fronts: item list[blockIdx.x] has an
// m x m row-major matrix at vals + moff[item] on the global ids
// gidmap[goff[item] ..]; the items of one launch share no global id.
__global__ void k_mf_add_local(MFDev d, const int* __restrict__ list, const int* __restrict__ goff,
                               const int* __restrict__ msz, const long long* __restrict__ moff,
                               const int* __restrict__ gidmap, const double* __restrict__ vals) {
  const int it = list[blockIdx.x], m = msz[it];
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < m * m; e += gridDim.y * blockDim.x) {
    const int ga = gidmap[goff[it] + e / m], gb = gidmap[goff[it] + e % m];
    const int f = d.fr[d.ord[ga] <= d.ord[gb] ? ga : gb];
    const int ra = mf_pos(d, f, ga), rb = mf_pos(d, f, gb);
    if (ra < 0 || rb < 0) continue;
    const long long F = d.np[f] + d.nu[f];
    d.F[d.foff[f] + ra * F + rb] += vals[moff[it] + e];
  }
}

// child update matrices (lower triangle) into the parents; one launch per slot
__global__ void k_mf_extend_add(MFDev d, const int* __restrict__ kids) {
  pdl_enter();
  const int c = kids[blockIdx.x];
  const int p = d.parent[c];
  const int npc = d.np[c], nuc = d.nu[c];
  const long long Fc = npc + nuc, Fp = d.np[p] + d.nu[p];
  const int* map = d.pmap + d.pmap_off[c];
  const double* C = d.F + d.foff[c];
  double* Pm = d.F + d.foff[p];
  // rows i of the update block round-robin over (blockIdx.y, warp), the
  // lanes along the row's columns j <= i: no triangular index inversion,
  // whose square root would run on the slow FP64 pipe for every entry
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = blockIdx.y * nw + warp; i < nuc; i += gridDim.y * nw) {
    const int pi = map[i];
    const double* crow = C + (long long)(npc + i) * Fc + npc;
    for (int j = lane; j <= i; j += 32) {
      const int pj = map[j];
      const int r = max(pi, pj), q = min(pi, pj);
      Pm[(long long)r * Fp + q] += crow[j];
    }
  }
}

// Entry of a step's front table whose item range holds item b: the last
// entry with first item <= b (syrk: field w, trsm: field z); empty ranges
// are passed over because the next entry has the same first item.
__device__ inline int mf_find_front(const int4* __restrict__ tab, int n, int b, bool syrk) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const int first = syrk ? tab[mid].w : tab[mid].z;
    if (first <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(BDDC_THREADS)
k_mf_potrf(MFDev d, const int4* __restrict__ tab, double* scratch, int* err) {
  pdl_enter();
  extern __shared__ __align__(128) unsigned char smraw[];
  DenseSmem<double>& sm = *reinterpret_cast<DenseSmem<double>*>(smraw);
  const int f = tab[blockIdx.x].x, j = 0;   // the first panel of each front
  const int np = d.np[f], nu = d.nu[f];
  const long long F = np + nu;
  int r0, nr;
  mf_tile(j, np, nu, r0, nr);
  double* A = d.F + d.foff[f];
  bool ok = cta_chol_inv<double>(A + r0 * F + r0, (int)F, d.Dinv + d.doff[f] + (long long)j * FNB * FNB, FNB, nr,
                                 scratch + (long long)blockIdx.x * 2 * 1024, sm);
  if (!ok && threadIdx.x == 0)
    if (atomicCAS(err, 0, 5) == 0) err[1] = f;
}

// A[i,j] <- A[i,j] Dinv_j^T (tile in shared memory)
__global__ void __launch_bounds__(BDDC_THREADS)
k_mf_trsm(MFDev d, const int4* __restrict__ tab, int nfr, int j) {
  pdl_enter();
  extern __shared__ __align__(128) unsigned char smraw[];
  double* T = reinterpret_cast<double*>(smraw);       // FNB x (FNB+1)
  double* D = T + FNB * (FNB + 1);                    // FNB x (FNB+1)
  const int4 fe = tab[mf_find_front(tab, nfr, (int)blockIdx.x, false)];
  const int f = fe.x, i = j + 1 + ((int)blockIdx.x - fe.z);
  const int np = d.np[f], nu = d.nu[f];
  const long long F = np + nu;
  int ri, ni, rj, nj;
  mf_tile(i, np, nu, ri, ni);
  mf_tile(j, np, nu, rj, nj);
  double* A = d.F + d.foff[f];
  const double* Dg = d.Dinv + d.doff[f] + (long long)j * FNB * FNB;
  for (int e = threadIdx.x; e < FNB * FNB; e += blockDim.x) {
    int r = e / FNB, c = e % FNB;
    T[r * (FNB + 1) + c] = (r < ni && c < nj) ? A[(ri + r) * F + rj + c] : 0.0;
    D[r * (FNB + 1) + c] = (r < nj && c < nj) ? Dg[r * FNB + c] : 0.0;
  }
  __syncthreads();
  // lanes along the rows, one output column per warp at a time, so that the
  // triangular loop (k <= c) has the same length in every lane of a warp;
  // warp w takes the columns w, 15 - w, 16 + w, 31 - w (66 multiply-adds)
  static_assert(FNB == 32 && BDDC_THREADS == 256, "column split for 32-wide tiles and 8 warps");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cols[4] = {warp, 15 - warp, 16 + warp, 31 - warp};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = cols[q];
    if (c >= nj) continue;
    double s = 0.0;
    for (int k = 0; k <= c; ++k) s = fma(T[lane * (FNB + 1) + k], D[c * (FNB + 1) + k], s);
    if (lane < ni) A[(ri + lane) * F + rj + c] = s;
  }
}

// A[i,l] -= A[i,j] A[l,j]^T
// A[i,l] -= A[i,j] A[l,j]^T.  Look-ahead: the CTA that updates the diagonal
// tile of the next pivot panel (i = l = j + 1 < pivot tiles) holds its final
// value and factors it right away (Cholesky and explicit inverse), so the
// next panel's trsm does not wait for a separate potrf launch.
__global__ void __launch_bounds__(BDDC_THREADS)
k_mf_syrk(MFDev d, const int4* __restrict__ tab, int nfr, int j, double* pscratch, int* err) {
  pdl_enter();
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ double As[32 * 33], Bs[32 * 33];
  const int4 fe = tab[mf_find_front(tab, nfr, (int)blockIdx.x, true)];
  // local index t -> (r, c), c <= r, of the trailing triangle
  const int t = (int)blockIdx.x - fe.w;
  int r = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  while (r > 0 && r * (r + 1) / 2 > t) --r;
  while ((r + 1) * (r + 2) / 2 <= t) ++r;
  const int f = fe.x, i = j + 1 + r, l = j + 1 + (t - r * (r + 1) / 2);
  const int np = d.np[f], nu = d.nu[f];
  const long long F = np + nu;
  int ri, ni, rl, nl, rj, nj;
  mf_tile(i, np, nu, ri, ni);
  mf_tile(l, np, nu, rl, nl);
  mf_tile(j, np, nu, rj, nj);
  double* A = d.F + d.foff[f];
  tile_gemm_f64<true>(ni, nl, nj, -1.0, A + ri * F + rj, F, A + rl * F + rj, F, 1.0, A + ri * F + rl, F, i == l,
                      As, Bs);
  if (i == l && i == j + 1 && i < (np + FNB - 1) / FNB) {
    __syncthreads();
    DenseSmem<double>& sm = *reinterpret_cast<DenseSmem<double>*>(smraw);
    const bool ok = cta_chol_inv<double>(A + ri * F + ri, (int)F, d.Dinv + d.doff[f] + (long long)i * FNB * FNB, FNB,
                                         ni, pscratch + (long long)f * 2048, sm);
    if (!ok && threadIdx.x == 0)
      if (atomicCAS(err, 0, 5) == 0) err[1] = f;
  }
}

__device__ inline double mf_wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}


// ---------------------------------------------------------------------------
// solve matrices: X = L_P^{-1} by tile rows (X_tt = Dinv_t,
// X_ts = -Dinv_t sum_{k=s}^{t-1} L_tk X_ks) and G = L_UP X.
// ---------------------------------------------------------------------------
__global__ void k_mf_inv_diag(MFDev d, const int4* __restrict__ work) {
  pdl_enter();
  const int4 w = work[blockIdx.x];
  const int f = w.x, t = w.y;
  const int np = d.np[f];
  const int r0 = t * FNB, nr = min(FNB, np - r0);
  double* X = d.S + d.soff[f];
  const double* Dg = d.Dinv + d.doff[f] + (long long)t * FNB * FNB;
  for (int e = threadIdx.x; e < nr * nr; e += blockDim.x) {
    int r = e / nr, c = e % nr;
    X[(long long)(r0 + r) * np + r0 + c] = (c <= r) ? Dg[r * FNB + c] : 0.0;
  }
}

// One partial product of a doubling step, item {front, r, c, k | nk << 16}
// (K tiles k .. k + nk - 1), into its own 32 x 32 slot of the product scratch
// (in item order):
//   mode 0: sum_k L[r][k] X[k][c]   (T = L_CA X_AA)
//   mode 1: sum_k X[r][k] T[k][c]   (X_CA = -X_CC T)
__global__ void __launch_bounds__(BDDC_THREADS)
k_mf_trtri_part(MFDev d, const int4* __restrict__ work, int mode, double* __restrict__ part) {
  pdl_enter();
  __shared__ double As[32 * 33], Bs[32 * 33];
  const int4 w = work[blockIdx.x];
  const int f = w.x, r = w.y, c = w.z, k = w.w & 0xffff, kt = w.w >> 16;
  const int np = d.np[f], nu = d.nu[f];
  const long long F = np + nu;
  const int r0 = r * FNB, nr = min(FNB, np - r0), c0 = c * FNB, nc = min(FNB, np - c0);
  const int k0 = k * FNB, nk = min(FNB * kt, np - k0);
  const double* L = d.F + d.foff[f];
  const double* X = d.S + d.soff[f];
  const double* T = d.T + d.toff[f];
  double* out = part + (long long)blockIdx.x * FNB * FNB;
  if (mode == 0)
    tile_gemm_f64<false>(nr, nc, nk, 1.0, L + r0 * F + k0, F, X + (long long)k0 * np + c0, np, 0.0, out, FNB, false,
                         As, Bs);
  else
    tile_gemm_f64<false>(nr, nc, nk, 1.0, X + (long long)r0 * np + k0, np, T + (long long)k0 * np + c0, np, 0.0, out,
                         FNB, false, As, Bs);
}

// Sum of the products of one output tile in item order, item {front,
// r << 16 | c, first product, count}: mode 0 into T, mode 1 (negated) into X.
__global__ void __launch_bounds__(BDDC_THREADS)
k_mf_trtri_sum(MFDev d, const int4* __restrict__ work, int mode, const double* __restrict__ part) {
  pdl_enter();
  const int4 w = work[blockIdx.x];
  const int f = w.x, r = w.y >> 16, c = w.y & 0xffff;
  const int np = d.np[f];
  const int r0 = r * FNB, nr = min(FNB, np - r0), c0 = c * FNB, nc = min(FNB, np - c0);
  double* dst = (mode == 0 ? d.T + d.toff[f] : d.S + d.soff[f]) + (long long)r0 * np + c0;
  for (int e = threadIdx.x; e < FNB * FNB; e += blockDim.x) {
    const int i = e / FNB, j = e % FNB;
    if (i >= nr || j >= nc) continue;
    double acc = 0.0;
    for (int q = 0; q < w.w; ++q) acc += part[(long long)(w.z + q) * FNB * FNB + e];
    dst[(long long)i * np + j] = mode == 0 ? acc : -acc;
  }
}

__global__ void __launch_bounds__(BDDC_THREADS)
k_mf_g(MFDev d, const int4* __restrict__ work) {
  pdl_enter();
  __shared__ double As[32 * 33], Bs[32 * 33];
  const int4 w = work[blockIdx.x];
  const int f = w.x, ut = w.y, st = w.z;
  const int np = d.np[f], nu = d.nu[f];
  const long long F = np + nu;
  const int u0 = ut * FNB, nuu = min(FNB, nu - u0);
  const int s0 = st * FNB, ns = min(FNB, np - s0);
  const double* L = d.F + d.foff[f];
  double* S = d.S + d.soff[f];
  // G[u, s cols] = L_UP[u, s0:np] X[s0:np, s cols]   (X lower: zero for k < s0)
  tile_gemm_f64<false>(nuu, ns, np - s0, 1.0, L + (np + u0) * F + s0, F, S + (long long)s0 * np + s0, np, 0.0,
                       S + (long long)(np + u0) * np + s0, np, false, As, Bs);
}

// S_f^T for the backward solve, 32 x 32 tiles through shared memory;
// grid (front, tile stride)
__global__ void k_mf_transpose(MFDev d) {
  pdl_enter();
  __shared__ double t[32][33];
  const int f = blockIdx.x;
  const int np = d.np[f], F = np + d.nu[f];
  const double* S = d.S + d.soff[f];
  double* ST = d.ST + d.soff[f];
  const int tc = (np + 31) / 32, ntile = ((F + 31) / 32) * tc;
  for (int tile = blockIdx.y; tile < ntile; tile += gridDim.y) {
    const int r0 = (tile / tc) * 32, c0 = (tile % tc) * 32;
    for (int idx = threadIdx.x; idx < 1024; idx += blockDim.x) {
      const int i = idx >> 5, j = idx & 31;
      t[i][j] = (r0 + i < F && c0 + j < np) ? S[(long long)(r0 + i) * np + c0 + j] : 0.0;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 1024; idx += blockDim.x) {
      const int i = idx >> 5, j = idx & 31;
      if (c0 + i < np && r0 + j < F) ST[(long long)(c0 + i) * F + r0 + j] = t[j][i];
    }
    __syncthreads();
  }
}

// sum over c in [c0, c1) of row[c] w[c] by one warp: lanes stride the row
// with eight independent chains so that eight loads per lane are in flight
__device__ inline double mf_row_dot(const double* __restrict__ row, const double* w, int c0, int c1) {
  const int lane = threadIdx.x & 31;
  double a[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  int c = c0 + lane;
  for (; c + 224 < c1; c += 256) {
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = fma(row[c + 32 * u], w[c + 32 * u], a[u]);
  }
  for (; c < c1; c += 32) a[0] = fma(row[c], w[c], a[0]);
  return mf_wsum(((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7])));
}

// forward, one launch per level; work item {front, chunk of FSR rows}:
// w_P = b_P + children's update vectors at P, w_U likewise at U;
// rows r < np: W[r] = (Linv_P w_P)[r];  rows r >= np: W[r] = w_U[r-np] - (G w_P)[r-np]
__global__ void __launch_bounds__(BDDC_THREADS)
k_mf_fwd(MFDev d, const int2* __restrict__ items, const int* __restrict__ kid_ptr, const int* __restrict__ kid_list,
         const int* __restrict__ lvl_index, const double* __restrict__ b) {
  pdl_enter();
  extern __shared__ __align__(128) unsigned char smraw[];
  double* w = reinterpret_cast<double*>(smraw);
  const int2 it = items[blockIdx.x];
  const int f = it.x, chunk = it.y;
  const int np = d.np[f], nu = d.nu[f], F = np + nu;
  const int* g = d.gid + d.gid_off[f];
  for (int k = threadIdx.x; k < F; k += blockDim.x) w[k] = (k < np) ? b[g[k]] : 0.0;
  __syncthreads();
  const int li = lvl_index[f];
  for (int q = kid_ptr[li]; q < kid_ptr[li + 1]; ++q) {
    const int c = kid_list[q];
    const int* map = d.pmap + d.pmap_off[c];
    const double* wc = d.W + d.woff[c] + d.np[c];
    for (int k = threadIdx.x; k < d.nu[c]; k += blockDim.x) w[map[k]] += wc[k];
    __syncthreads();
  }
  const int r = chunk * FSR + (threadIdx.x >> 5);
  if (r < F) {
    const double acc = mf_row_dot(d.S + d.soff[f] + (long long)r * np, w, 0, (r < np) ? r + 1 : np);
    if ((threadIdx.x & 31) == 0) d.W[d.woff[f] + r] = (r < np) ? acc : w[r] - acc;
  }
}

// backward, one launch per level; work item {front, chunk of FSR pivots}:
// x_P[c] = sum_{c<=r<np} Linv_P[r][c] y_P[r] - sum_u G[u][c] x_U[u], i.e. row c
// of S_f^T against [y_P; x_U]
__global__ void __launch_bounds__(BDDC_THREADS)
k_mf_bwd(MFDev d, const int2* __restrict__ items, double* x) {
  pdl_enter();
  extern __shared__ __align__(128) unsigned char smraw[];
  double* vec = reinterpret_cast<double*>(smraw);        // [y_P; x_U]
  const int2 it = items[blockIdx.x];
  const int f = it.x, chunk = it.y;
  const int np = d.np[f], nu = d.nu[f], F = np + nu;
  const int* g = d.gid + d.gid_off[f];
  const double* Wf = d.W + d.woff[f];
  for (int k = threadIdx.x; k < F; k += blockDim.x) vec[k] = (k < np) ? Wf[k] : x[g[k]];
  __syncthreads();
  const int c = chunk * FSR + (threadIdx.x >> 5);
  if (c < np) {
    const double* row = d.ST + d.soff[f] + (long long)c * F;
    const double pos = mf_row_dot(row, vec, c, np);
    const double neg = mf_row_dot(row, vec, np, F);
    if ((threadIdx.x & 31) == 0) x[g[c]] = pos - neg;
  }
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
namespace {
MFDev dev_of(const MFPlan& P) {
  MFDev d;
  d.np = P.d_np; d.nu = P.d_nu; d.gid = P.d_gid; d.fr = P.d_fr; d.pp = P.d_pp; d.ord = P.d_ord;
  d.pmap = P.d_pmap; d.parent = P.d_parent;
  d.foff = P.d_foff; d.doff = P.d_doff; d.woff = P.d_woff; d.gid_off = P.d_gid_off; d.pmap_off = P.d_pmap_off;
  d.F = P.F; d.Dinv = P.Dinv; d.W = P.W;
  d.S = P.S; d.soff = P.d_soff;
  d.T = P.tscratch; d.toff = P.d_toff; d.ST = P.ST;
  return d;
}

template <typename T>
T* up(const std::vector<T>& v, const std::function<void*(size_t)>& alloc, cudaStream_t st) {
  T* p = (T*)alloc(sizeof(T) * std::max<size_t>(v.size(), 1));
  stage_h2d(p, v.data(), sizeof(T) * v.size(), st);
  return p;
}

}  // namespace

void configure_mf_kernels() {
  int sm = (int)sizeof(DenseSmem<double>);
  cudaFuncSetAttribute(k_mf_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_mf_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_mf_potrf, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_mf_syrk, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_mf_trsm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(2 * FNB * (FNB + 1) * sizeof(double)));
}

void mf_upload(MFPlan& P, const std::function<void*(size_t)>& alloc,
               const std::function<void*(size_t)>& tmp_alloc, cudaStream_t st) {
  if (P.nfront == 0) return;
  P.d_np = up(P.np, alloc, st);
  P.d_nu = up(P.nu, alloc, st);
  P.d_gid = up(P.gid, alloc, st);
  P.d_fr = up(P.fr, alloc, st);
  P.d_pp = up(P.pp, alloc, st);
  P.d_ord = up(P.ord, alloc, st);
  P.d_pmap = up(P.pmap, alloc, st);
  P.d_parent = up(P.parent, alloc, st);
  P.d_foff = up(P.foff, alloc, st);
  P.d_doff = up(P.doff, alloc, st);
  P.d_woff = up(P.woff, alloc, st);
  P.d_gid_off = up(P.gid_off, alloc, st);
  P.d_pmap_off = up(P.pmap_off, alloc, st);
  P.F = (double*)tmp_alloc(sizeof(double) * P.fpool);
  P.Dinv = (double*)tmp_alloc(sizeof(double) * std::max<long long>(P.dpool, 1));
  P.W = (double*)alloc(sizeof(double) * P.wpool);
  P.S = (double*)alloc(sizeof(double) * std::max<long long>(P.spool, 1));
  P.ST = (double*)alloc(sizeof(double) * std::max<long long>(P.spool, 1));
  P.d_soff = up(P.soff, alloc, st);
  cudaMemsetAsync(P.F, 0, sizeof(double) * P.fpool, st);
  cudaMemsetAsync(P.S, 0, sizeof(double) * P.spool, st);
  // work lists
  std::vector<int> all;
  P.step_off.clear();
  for (const std::vector<int>& tab : P.step_fronts) {
    P.step_off.push_back((long long)all.size() / 4);
    all.insert(all.end(), tab.begin(), tab.end());
  }
  P.inv_off.clear(); P.inv_len.clear(); P.inv_lvl_base.clear();
  for (const auto& lv : P.inv_items) {
    P.inv_lvl_base.push_back((int)P.inv_off.size());
    for (const std::vector<int>& v : lv) {
      P.inv_off.push_back((long long)all.size() / 4);
      P.inv_len.push_back((int)v.size() / 4);
      all.insert(all.end(), v.begin(), v.end());
    }
  }
  P.inv_lvl_base.push_back((int)P.inv_off.size());
  P.tscratch = (double*)tmp_alloc(sizeof(double) * std::max<long long>(P.tpool, 1));
  {
    // tile products of the doubling steps; the solve matrices of all levels
    // are built in one stream, one list at a time
    size_t maxparts = 1;
    for (const auto& lv : P.inv_items)
      for (size_t q = 2; q < lv.size(); q += 2) maxparts = std::max(maxparts, lv[q].size() / 4);
    P.tpart = (double*)tmp_alloc(sizeof(double) * FNB * FNB * maxparts);
  }
  P.d_toff = up(P.toff, alloc, st);
  P.d_lists = (int4*)tmp_alloc(sizeof(int) * std::max<size_t>(all.size(), 4));
  stage_h2d(P.d_lists, all.data(), sizeof(int) * all.size(), st);
  // per level: fronts, their children (for the solves), children by slot (extend-add)
  std::vector<int> lv;
  P.lvl_fronts_off.assign(P.nlevel + 1, 0);
  for (int l = 0; l < P.nlevel; ++l) {
    P.lvl_fronts_off[l] = (int)lv.size();
    for (int f : P.fronts_at_level[l]) lv.push_back(f);
  }
  P.lvl_fronts_off[P.nlevel] = (int)lv.size();
  std::vector<std::vector<int>> kids(P.nfront);
  P.maxslot = 0;
  for (int f = 0; f < P.nfront; ++f)
    if (P.parent[f] >= 0) {
      kids[P.parent[f]].push_back(f);
      P.maxslot = std::max(P.maxslot, P.child_slot[f] + 1);
    }
  for (auto& k : kids) std::sort(k.begin(), k.end(), [&](int a, int b) { return P.child_slot[a] < P.child_slot[b]; });
  std::vector<int> kptr, klist;
  for (int f : lv) {
    kptr.push_back((int)klist.size());
    for (int c : kids[f]) klist.push_back(c);
  }
  kptr.push_back((int)klist.size());
  std::vector<int> slots;
  P.slot_off.assign((size_t)P.nlevel * P.maxslot + 1, 0);
  for (int l = 0; l < P.nlevel; ++l)
    for (int s2 = 0; s2 < P.maxslot; ++s2) {
      P.slot_off[(size_t)l * P.maxslot + s2] = (int)slots.size();
      for (int f : P.fronts_at_level[l])
        for (int c : kids[f])
          if (P.child_slot[c] == s2) slots.push_back(c);
    }
  P.slot_off[(size_t)P.nlevel * P.maxslot] = (int)slots.size();
  std::vector<int> blob(lv);
  std::vector<int> lvl_index(P.nfront, 0);
  for (size_t q = 0; q < lv.size(); ++q) lvl_index[lv[q]] = (int)q;
  P.blob_lvl_index = (long long)blob.size();
  blob.insert(blob.end(), lvl_index.begin(), lvl_index.end());
  P.blob_kptr = (long long)blob.size();
  blob.insert(blob.end(), kptr.begin(), kptr.end());
  P.blob_klist = (long long)blob.size();
  blob.insert(blob.end(), klist.begin(), klist.end());
  P.blob_slots = (long long)blob.size();
  blob.insert(blob.end(), slots.begin(), slots.end());
  P.d_blob = up(blob, alloc, st);
  int maxpo = 1;
  for (const std::vector<int>& tab : P.step_fronts) maxpo = std::max(maxpo, (int)tab.size() / 4);
  P.pscratch = (double*)tmp_alloc(sizeof(double) * 2048 * (size_t)maxpo);
  P.fscratch = (double*)tmp_alloc(sizeof(double) * 2048 * (size_t)P.nfront);
  // solve work lists: per level fwd items {front, row chunk}, bwd items {front, column chunk}
  std::vector<int> items;
  P.fwd_items_off.assign(P.nlevel, 0); P.fwd_items_len.assign(P.nlevel, 0);
  P.bwd_items_off.assign(P.nlevel, 0); P.bwd_items_len.assign(P.nlevel, 0);
  P.maxF = 0;
  for (int l = 0; l < P.nlevel; ++l) {
    P.fwd_items_off[l] = (int)items.size() / 2;
    for (int f : P.fronts_at_level[l]) {
      const int F = P.np[f] + P.nu[f];
      P.maxF = std::max(P.maxF, F);
      for (int c = 0; c < (F + FSR - 1) / FSR; ++c) items.insert(items.end(), {f, c});
    }
    P.fwd_items_len[l] = (int)items.size() / 2 - P.fwd_items_off[l];
    P.bwd_items_off[l] = (int)items.size() / 2;
    for (int f : P.fronts_at_level[l])
      for (int c = 0; c < (P.np[f] + FSR - 1) / FSR; ++c) items.insert(items.end(), {f, c});
    P.bwd_items_len[l] = (int)items.size() / 2 - P.bwd_items_off[l];
  }
  P.d_solve_items = up(items, alloc, st);
}

void mf_assemble(const MFPlan& P, const LocalLaunch& L, const int* color_subs, const int* color_count_host,
                 const int* color_offset_host, cudaStream_t st) {
  if (P.nfront == 0) return;
  MFDev d = dev_of(P);
  for (int c = 0; c < 8; ++c) {
    if (color_count_host[c] == 0) continue;
    BDDC_COUNT(1);
    k_mf_assemble<<<dim3(color_count_host[c], 32), BDDC_THREADS, 0, st>>>(d, L.subs, L.lc,
                                                                          color_subs + color_offset_host[c], L.Ac);
  }
}

void mf_add_local(const MFPlan& P, const int* list, int nitems, const int* goff, const int* msz,
                  const long long* moff, const int* gidmap, const double* vals, cudaStream_t st) {
  if (P.nfront == 0 || nitems == 0) return;
  MFDev d = dev_of(P);
  BDDC_COUNT(1);
  k_mf_add_local<<<dim3(nitems, 16), BDDC_THREADS, 0, st>>>(d, list, goff, msz, moff, gidmap, vals);
}

static void CK_MF(cudaError_t e) {
  if (e != cudaSuccess) throw std::runtime_error(std::string("coarse factor: ") + cudaGetErrorString(e));
}

// the kernels of the panel-step chain and of the solves start with
// pdl_enter(): launched with programmatic stream serialisation
template <typename... KArgs, typename... Args>
static void launch_mf(void (*kern)(KArgs...), dim3 grid, size_t smem, cudaStream_t st, Args... args) {
  CK_MF(launch_pdl(kern, grid, dim3(BDDC_THREADS), smem, st, args...));
}

// Solve matrices of the fronts of one level: Linv_P by tile rows (diagonal
// inverses, then the doubling steps), then G = L_UP Linv_P.  They read only
// the level's own factor, final once its last panel step is done.
static void mf_solve_matrices(const MFPlan& P, const MFDev& d, int l, cudaStream_t st) {
  const int b = P.inv_lvl_base[l], e = P.inv_lvl_base[l + 1];
  if (P.inv_len[b]) { BDDC_COUNT(1); launch_mf(k_mf_inv_diag, dim3(P.inv_len[b]), 0, st, d, P.d_lists + P.inv_off[b]); }
  for (int q = b + 2; q + 3 < e; q += 4)
    for (int mode = 0; mode < 2; ++mode) {
      const int lp = q + 2 * mode, ls = lp + 1;
      if (!P.inv_len[lp]) continue;
      BDDC_COUNT(2);
      launch_mf(k_mf_trtri_part, dim3(P.inv_len[lp]), 0, st, d, P.d_lists + P.inv_off[lp], mode, P.tpart);
      launch_mf(k_mf_trtri_sum, dim3(P.inv_len[ls]), 0, st, d, P.d_lists + P.inv_off[ls], mode, (const double*)P.tpart);
    }
  if (P.inv_len[b + 1]) { BDDC_COUNT(1); launch_mf(k_mf_g, dim3(P.inv_len[b + 1]), 0, st, d, P.d_lists + P.inv_off[b + 1]); }
}

void mf_factor(const MFPlan& P, int* err, cudaStream_t st, cudaStream_t aux, cudaEvent_t fork, cudaEvent_t join) {
  if (P.nfront == 0) return;
  MFDev d = dev_of(P);
  const int* slots = P.d_blob + P.blob_slots;
  const size_t dsm = sizeof(DenseSmem<double>);
  const size_t tsm = 2 * FNB * (FNB + 1) * sizeof(double);
  const bool two = aux && fork && join;
  size_t step = 0;
  for (int l = P.nlevel - 1; l >= 0; --l) {
    for (int s = 0; s < P.maxslot; ++s) {
      const int a = P.slot_off[(size_t)l * P.maxslot + s], b = P.slot_off[(size_t)l * P.maxslot + s + 1];
      if (b > a) {
        BDDC_COUNT(1);
        launch_mf(k_mf_extend_add, dim3(b - a, 32), 0, st, d, slots + a);
      }
    }
    int maxpt = 0;
    for (int f : P.fronts_at_level[l]) maxpt = std::max(maxpt, (P.np[f] + FNB - 1) / FNB);
    for (int j = 0; j < maxpt; ++j, ++step) {
      const int nfr = (int)P.step_fronts[step].size() / 4, ntr = P.step_ntr[step], nsy = P.step_nsy[step];
      const int4* tab = P.d_lists + P.step_off[step];
      // the first panel's diagonal tiles of the level; later ones are
      // factored inside the previous step's syrk (look-ahead)
      if (nfr && j == 0) { BDDC_COUNT(1); launch_mf(k_mf_potrf, dim3(nfr), dsm, st, d, tab, P.pscratch, err); }
      if (ntr) { BDDC_COUNT(1); launch_mf(k_mf_trsm, dim3(ntr), tsm, st, d, tab, nfr, j); }
      if (nsy) { BDDC_COUNT(1); launch_mf(k_mf_syrk, dim3(nsy), dsm, st, d, tab, nfr, j, P.fscratch, err); }
    }
    if (two) {
      CK_MF(cudaEventRecord(fork, st));
      CK_MF(cudaStreamWaitEvent(aux, fork, 0));
    }
    mf_solve_matrices(P, d, l, two ? aux : st);
  }
  if (two) {
    CK_MF(cudaEventRecord(join, aux));
    CK_MF(cudaStreamWaitEvent(st, join, 0));
  }
  BDDC_COUNT(1);
  launch_mf(k_mf_transpose, dim3(P.nfront, 16), 0, st, d);
}

void mf_solve(const MFPlan& P, const double* b, double* x, double* W, cudaStream_t st) {
  if (P.nfront == 0) return;
  MFDev d = dev_of(P);
  d.W = W;
  const int* kptr = P.d_blob + P.blob_kptr;
  const int* klist = P.d_blob + P.blob_klist;
  const int* lidx = P.d_blob + P.blob_lvl_index;
  const int2* items = reinterpret_cast<const int2*>(P.d_solve_items);
  const size_t sm = sizeof(double) * (size_t)P.maxF;
  for (int l = P.nlevel - 1; l >= 0; --l) {
    BDDC_COUNT(1);
    launch_mf(k_mf_fwd, dim3(P.fwd_items_len[l]), sm, st, d, items + P.fwd_items_off[l], kptr, klist, lidx, b);
  }
  for (int l = 0; l < P.nlevel; ++l) {
    BDDC_COUNT(1);
    launch_mf(k_mf_bwd, dim3(P.bwd_items_len[l]), sm, st, d, items + P.bwd_items_off[l], x);
  }
}

}  // namespace bddc
