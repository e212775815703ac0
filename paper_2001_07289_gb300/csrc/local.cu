// Per-subdomain (batched) kernels of BDDC-SO: local assembly, block-tridiagonal
// Cholesky factorisations of the Dirichlet and constrained Neumann problems,
// the coarse basis Phi_i, and the local steps of the preconditioner apply.
//
// Method (Section 3 with Definition 1; the two-level split of the W-tilde
// problem as in Dohrmann 2003, cited in Section 1):
//   * A_II^(i): stiffness of the interior nodes of Omega_i (not on Gamma).
//   * A^(i): Neumann stiffness of Omega_i.  Primal point values (vertices of
//     Theta-hat on Gamma) are eliminated: their rows/columns, and those of the
//     Dirichlet-boundary nodes, are replaced by identity rows, which keeps the
//     local grid regular.  Means over (sub)edges/(sub)faces are Lagrange rows
//     C_r, handled through S_c = C_r A_rr^{-1} C_r^T.
//   * Phi_i solves [A C^T; C 0][Phi; Lambda] = [0; I]; with Y = A_rr^{-1}
//     [-A_rv | C_r^T] = [Y_v | X]:  Lambda_v = S_c^{-1} C_r Y_v,
//     Phi_rv = Y_v - X Lambda_v, Phi_ra = X S_c^{-1}, and
//     Phi^T A Phi = [[ (A Phi_v)_V , -Lambda_v^T ], [ -Lambda_v , S_c^{-1} ]].
//   * Apply: the constrained Neumann solution is w_r = y - Phi_ra C_r y with
//     y = A_rr^{-1} r_r, so v_i = Phi_i (u_c|_i - [0; C_r y]) + y.
//
// Local matrices are stored as z-plane blocks (see common.cuh); the factor of
// each diagonal block is kept as its explicit inverse, so every sweep is a
// sequence of dense products.
#include <cooperative_groups.h>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include "common.cuh"
#include "dense.cuh"
#include "kernels.h"
#include "stream.cuh"
#include "umma.cuh"

namespace bddc {

namespace cg = cooperative_groups;

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------

// Entry A(a, a+d) of the stiffness restricted to the elements of box s:
// h * K(d) * (sum of alpha over the elements holding both nodes), where the
// unit-cube matrix K is 1/3 on the diagonal, 0 for nodes one coordinate apart
// and -1/12 for nodes two or three coordinates apart.
__device__ inline double box_entry(const MeshDev& m, const double* __restrict__ alpha,
                                   const SubDesc& s, int ax, int ay, int az, int dx, int dy, int dz) {
  int hd = abs(dx) + abs(dy) + abs(dz);
  if (hd == 1) return 0.0;
  int a[3] = {ax, ay, az}, d[3] = {dx, dy, dz}, lo[3], hi[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (d[c] > 0) { lo[c] = a[c]; hi[c] = a[c]; }
    else if (d[c] < 0) { lo[c] = a[c] - 1; hi[c] = a[c] - 1; }
    else { lo[c] = a[c] - 1; hi[c] = a[c]; }
    lo[c] = max(lo[c], s.e0[c]);
    hi[c] = min(hi[c], s.e0[c] + s.w[c] - 1);
  }
  double sum = 0.0;
  for (int k = lo[2]; k <= hi[2]; ++k)
    for (int j = lo[1]; j <= hi[1]; ++j)
      for (int i = lo[0]; i <= hi[0]; ++i)
        sum += alpha[(long long)i + (long long)m.nx * (j + (long long)m.ny * k)];
  return m.h * (hd == 0 ? (1.0 / 3.0) : (-1.0 / 12.0)) * sum;
}

// Local Neumann node fixed to zero in A_rr: on the Dirichlet boundary or a
// primal point value (a selected one-node vertex object, eliminated).
__device__ inline bool neumann_fixed(const MeshDev& m, const SubDesc& s, int ix, int iy, int iz) {
  int gx = s.e0[0] + ix, gy = s.e0[1] + iy, gz = s.e0[2] + iz;
  if (on_dirichlet(m, gx, gy, gz)) return true;
  return m.vfix[nodeid(m.NX, m.NY, gx, gy, gz)] != 0;
}

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

template <typename T>
__device__ inline T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// assembly of the plane blocks
// ---------------------------------------------------------------------------

// grid: (subdomain, plane k, chunk); writes the diagonal block D_k to slot k
// (dense Q x Q) and the coupling B_k = A_{k,k-1} to slot gz+k-1 as its nine
// stencil diagonals: Bd[o][i] = B_k[i][i + dx + dy gx], o = 3 (dy+1) + dx+1
// (zero where the neighbour is off the plane).
// Pinned floating subdomains (selections without point values: the local
// Neumann matrix A has the constants as kernel).  The factor holds
// A~ = A + sum_k rho_k c_k^T c_k over the constraint rows c_k (averages)
// whose nodes lie in one z-plane of the box, rho_k = the sum of A's diagonal
// over the row's nodes; each term stays inside one diagonal plane block.
// Every constrained problem prescribes C w, so c_k w is known and
// [A~ C^T; C 0] has the same w as [A C^T; C 0] (an augmented Lagrangian):
// the constrained solves and Phi need no correction, and only the local
// coarse matrix changes, Phi^T A Phi = S~_c^{-1} - diag(rho).  pen holds
// rho_k per local coarse DOF (0 for rows not penalised and in subdomains not
// pinned); computed here, one CTA per subdomain, a thread per row.
__global__ void k_pin_penalty(const SubDesc* __restrict__ subs, MeshDev m, const double* __restrict__ alpha,
                              const LocalCoarse* __restrict__ lc, const int* __restrict__ lcn,
                              double* __restrict__ pen) {
  const SubDesc s = subs[blockIdx.x];
  const int px = s.w[0] + 1, py = s.w[1] + 1, Q = px * py;
  for (int j = threadIdx.x; j < s.nc; j += blockDim.x) {
    const LocalCoarse c = lc[s.cofs + j];
    double rho = 0.0;
    if (s.pin && j >= s.nv) {
      const int z0 = lcn[c.off] / Q;
      bool one_plane = true;
      for (int q = 0; q < c.count; ++q) {
        const int l = lcn[c.off + q];
        one_plane = one_plane && l / Q == z0;
        const int ix = l % px, iy = (l / px) % py, iz = l / Q;
        rho += box_entry(m, alpha, s, s.e0[0] + ix, s.e0[1] + iy, s.e0[2] + iz, 0, 0, 0);
      }
      if (!one_plane) rho = 0.0;
    }
    pen[s.cofs + j] = rho;
  }
}

// D_k as a dense Q x Q block in slot k, or (tc, see plane_taps) as its nine
// in-plane taps per node in the factorisation scratch; B_k as nine taps per
// node in slot nz + k - 1.
template <typename T>
__global__ void k_assemble(const SubDesc* __restrict__ subs, MeshDev m, const double* __restrict__ alpha,
                           T* __restrict__ fac, int neumann, const LocalCoarse* __restrict__ lc,
                           const int* __restrict__ own, const double* __restrict__ pen, T* __restrict__ scratch,
                           int tc) {
  const SubDesc s = subs[blockIdx.x];
  const Grid g = grid_of(s, neumann);
  const int k = blockIdx.y;
  if (k >= g.gz) return;
  const int Q = g.gx * g.gy;
  T* base = fac + (neumann ? s.offN : s.offD);
  long long toff = 0;
  const bool taps = plane_taps(s, neumann, tc, TCS_MAXQ, &toff);
  // a plane block has Q^2 + 9Q < 2^31 entries: 32-bit index arithmetic
  const int nd = taps ? 9 * Q : Q * Q;
  const long long SS = slot_stride(Q);
  const int n1 = (k > 0) ? 9 * Q : 0;
  for (int e = (int)(blockIdx.z * blockDim.x + threadIdx.x); e < nd + n1; e += (int)(gridDim.z * blockDim.x)) {
    int a, bx, by, bz, dx, dy;
    if (e < nd && !taps) {
      a = e / Q;
      const int b = e % Q;
      bx = b % g.gx; by = b / g.gx; bz = k;
      dx = bx - a % g.gx; dy = by - a / g.gx;
    } else {
      const int o = (e < nd ? e : e - nd) / Q;
      a = (e < nd ? e : e - nd) % Q;
      dx = o % 3 - 1; dy = o / 3 - 1;
      bx = a % g.gx + dx; by = a / g.gx + dy; bz = e < nd ? k : k - 1;
    }
    const int ax = a % g.gx, ay = a / g.gx, dz = bz - k;
    double v = 0.0;
    if (abs(dx) <= 1 && abs(dy) <= 1 && bx >= 0 && bx < g.gx && by >= 0 && by < g.gy) {
      bool fa = neumann && neumann_fixed(m, s, ax, ay, k);
      bool fb = neumann && neumann_fixed(m, s, bx, by, bz);
      if (fa || fb) v = (dx == 0 && dy == 0 && dz == 0) ? 1.0 : 0.0;
      else v = box_entry(m, alpha, s, s.e0[0] + g.off + ax, s.e0[1] + g.off + ay, s.e0[2] + g.off + k,
                         dx, dy, dz);
    }
    // pinned floating subdomain: rho_k c_k^T c_k of the rows of this plane (see k_pin_penalty)
    if (neumann && s.pin && e < nd) {
      const int ja = own[s.offVec + (long long)k * Q + a], jb = own[s.offVec + (long long)k * Q + (e % Q)];
      if (ja >= 0 && ja == jb) {
        const double cnt = (double)lc[s.cofs + ja].count;
        v += pen[s.cofs + ja] / (cnt * cnt);
      }
    }
    if (e >= nd) base[(long long)(g.gz + k - 1) * SS + (e - nd)] = (T)v;
    else if (taps) scratch[toff + 9LL * Q * k + e] = (T)v;
    else base[(long long)k * SS + e] = (T)v;
  }
}

// ---------------------------------------------------------------------------
// batched block-tridiagonal factorisation by inverse Schur complements:
//   S_0 = D_0,  S_k = D_k - B_k S_{k-1}^{-1} B_k^T,  slot k <- S_k^{-1}.
// B_k has nine stencil entries per row, so the sandwich costs 18 Q^2
// multiply-adds (T = S_{k-1}^{-1} B_k^T, then S_k = D_k - B_k T).  S_k is
// inverted by the symmetric sweep of its lower triangle (Gauss-Jordan
// without pivoting, stable for SPD matrices): for pivot p with d = A[p][p],
//   A[i][j] -= A[i][p] A[j][p] / d   (i, j != p),
//   A[i][p] <- A[i][p] / d,   A[p][p] <- -1 / d,
// which leaves -S^{-1} after all Q pivots.  The packed lower triangle lives in
// shared memory when it fits (else in the scratch, L2-resident).  One barrier per
// pivot: the pivot column is double-buffered and the threads owning column
// p + 1 publish it, and the reciprocal of the next pivot, as they update it.
// 512 threads; thread t owns the entries with i = t/16 (mod 32) and
// j = t (mod 16).
// grid (subdomain, problem): y = 0 Neumann, y = 1 Dirichlet (concurrent).
// ---------------------------------------------------------------------------
__host__ __device__ inline long long packed_size(int Q) { return (long long)Q * (Q + 1) / 2; }

constexpr int SCHUR_THREADS = 512;   // 32 x 16 owner grid

// Register-resident plane step for Q <= 32 RI and Q <= 16 RJ (FP32): thread
// (tr, tc) = (t / 16, t % 16) holds the entries (tr + 32 a, tc + 16 b) of S_k
// in x[a][b] (entries above the diagonal or past Q are carried along and never
// used).  The pivots go in blocks K of SB = 16: the sweep over the pivots of K
// equals, with D = X_KK,
//   X_ij <- X_ij - X_iK D^{-1} X_Kj,  X_iK <- X_iK D^{-1},  X_KK <- -D^{-1}
// (i, j outside K), so one warp inverts D by 16 single-pivot sweeps, the block
// forms W = X_:K D^{-1}, and every thread applies the rank-16 update to its
// registers: three barriers per 16 pivots.  Tm: Q x Q shared memory that
// holds S_{k-1}^{-1} on entry (for k > 0), S_{k-1}^{-1} B_k^T while S_k is
// formed, and S_k^{-1} on return; pw: the panel buffers (schur_panel_floats).
// Writes S_k^{-1} to slot.
constexpr int SB = 16;    // pivots per block (the column block of one tc stride)
constexpr int PST = 18;   // row stride of the panel buffers: 8-byte rows, conflict-free LDS.64
constexpr int PNR = 192;  // panel rows: max(32 RI, 16 RJ) of the register grid
__host__ __device__ constexpr int schur_panel_floats() { return 4 * PNR * PST + SB * (SB + 1); }

template <int RI, int RJ>
__device__ void schur_plane_regs(int Q, int gx, int gy, int k, float* __restrict__ slot,
                                 const float* __restrict__ Bd, float* __restrict__ pw, float* __restrict__ Tm,
                                 int* err, int code, int sub_id) {
  static_assert(32 * RI <= PNR && 16 * RJ <= PNR, "panel rows");
  const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
  if (k > 0) {
    // T = S_{k-1}^{-1} B_k^T in place in Tm, which holds S_{k-1}^{-1} (both
    // triangles) from the previous plane: T[i][j] = sum_o S[i][j + off_o] w_o(j)
    // is a stencil along row i, so a warp takes whole rows, reads the row's
    // taps into registers and writes the row back.  Lane l keeps the nine
    // weights of its columns j = l + 32 m (zero for taps off the plane, whose
    // index is clamped to j).
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int MJ = PNR / 32;
    float w[MJ][9];
    int jc[MJ];
    unsigned okm[MJ];
#pragma unroll
    for (int m = 0; m < MJ; ++m) {
      const int j = lane + 32 * m, jj = min(j, Q - 1), jx = jj % gx, jy = jj / gx;
      jc[m] = jj;
      okm[m] = 0;
#pragma unroll
      for (int o = 0; o < 9; ++o) {
        const int dx = o % 3 - 1, dy = o / 3 - 1;
        const bool ok = j < Q && jx + dx >= 0 && jx + dx < gx && jy + dy >= 0 && jy + dy < gy;
        w[m][o] = ok ? Bd[o * Q + jj] : 0.0f;
        okm[m] |= ok ? (1u << o) : 0u;
      }
    }
    for (int i = warp; i < Q; i += SCHUR_THREADS / 32) {
      float* row = Tm + i * Q;
      float acc[MJ];
#pragma unroll
      for (int m = 0; m < MJ; ++m) {
        float a = 0.0f;
#pragma unroll
        for (int o = 0; o < 9; ++o) {
          const int dx = o % 3 - 1, dy = o / 3 - 1;
          const int idx = ((okm[m] >> o) & 1u) ? jc[m] + dx + dy * gx : jc[m];
          a = fmaf(row[idx], w[m][o], a);
        }
        acc[m] = a;
      }
      __syncwarp();
#pragma unroll
      for (int m = 0; m < MJ; ++m)
        if (lane + 32 * m < Q) row[lane + 32 * m] = acc[m];
    }
    __syncthreads();
  }
  float x[RI][RJ];
#pragma unroll
  for (int ai = 0; ai < RI; ++ai) {
    const int i = tr + 32 * ai, ix = i % gx, iy = i / gx;
#pragma unroll
    for (int bj = 0; bj < RJ; ++bj) {
      const int j = tc + 16 * bj;
      float v = 0.0f;
      if (i < Q && j <= i) {
        v = slot[i * Q + j];
        if (k > 0) {
          float acc = 0.0f;
#pragma unroll
          for (int o = 0; o < 9; ++o) {
            const int dx = o % 3 - 1, dy = o / 3 - 1;
            const bool ok = ix + dx >= 0 && ix + dx < gx && iy + dy >= 0 && iy + dy < gy;
            const float wv = ok ? Bd[o * Q + i] : 0.0f;
            acc += wv * Tm[(ok ? i + dx + dy * gx : i) * Q + j];
          }
          v -= acc;
        }
      }
      x[ai][bj] = v;
    }
  }
  float* Dm = pw + 4 * PNR * PST;   // D^{-1}, SB x (SB + 1)
  const int nb = (Q + SB - 1) / SB;
  for (int kb = 0; kb < nb; ++kb) {
    const int p0 = kb * SB;
    // double-buffered panels: a buffer is rewritten two blocks later, after
    // the three barriers of the block in between
    float* P = pw + (kb & 1) * 2 * PNR * PST;   // P[i][c] = X(i, p0 + c)
    float* W = P + PNR * PST;                   // W[i][c] = (X_:K D^{-1})(i, c)
    const int bj0 = p0 >> 4;                     // K = columns tc + 16 bj0
    const int ai0 = p0 >> 5, tr0 = p0 & 31;      // K = rows tr + 32 ai0, tr in [tr0, tr0 + 16)
    // (a) the panel from the lower triangle: entries (i, p0 + c) with
    // i >= p0 + c from the owners of column p0 + c, the rest from the owners
    // of row p0 + c; zero past Q (and in the columns of a short last block)
    {
      const int pc = p0 + tc;
#pragma unroll
      for (int bj = 0; bj < RJ; ++bj)
        if (bj == bj0) {
#pragma unroll
          for (int ai = 0; ai < RI; ++ai) {
            const int i = tr + 32 * ai;
            if (pc >= Q || i >= Q) P[i * PST + tc] = 0.0f;
            else if (i >= pc) P[i * PST + tc] = x[ai][bj];
          }
        }
      const int c = tr - tr0, pr = p0 + c;
      if (c >= 0 && c < SB && pr < Q) {
#pragma unroll
        for (int ai = 0; ai < RI; ++ai)
          if (ai == ai0) {
#pragma unroll
            for (int bj = 0; bj < RJ; ++bj) {
              const int j = tc + 16 * bj;
              if (j < pr) P[j * PST + c] = x[ai][bj];
            }
          }
      }
    }
    __syncthreads();
    // (b) D^{-1} by one warp: lane m < 16 holds row m of D (identity rows and
    // columns stand in for pivots past Q), 16 single-pivot sweeps
    if (threadIdx.x < 32) {
      const int m = threadIdx.x & 15;
      float a[SB];
#pragma unroll
      for (int c = 0; c < SB; ++c)
        a[c] = (p0 + m < Q && p0 + c < Q) ? P[(p0 + m) * PST + c] : (m == c ? 1.0f : 0.0f);
#pragma unroll
      for (int q = 0; q < SB; ++q) {
        float d = __shfl_sync(0xffffffffu, a[q], q);
        if (!(d > 0.0f)) {
          if (threadIdx.x == 0) set_error(err, code, sub_id);
          d = 1.0f;
        }
        const float r = __frcp_rn(d);
        const float cr = a[q] * r;
#pragma unroll
        for (int c = 0; c < SB; ++c)
          if (c != q) {
            const float rowq = __shfl_sync(0xffffffffu, a[c], q);
            a[c] = (m == q) ? rowq * r : a[c] - cr * rowq;
          }
        a[q] = (m == q) ? -r : cr;
      }
      if (threadIdx.x < SB)
#pragma unroll
        for (int c = 0; c < SB; ++c) Dm[m * (SB + 1) + c] = -a[c];
    }
    __syncthreads();
    // (c) W = X_:K D^{-1} for the rows outside K (zero elsewhere; unused)
    {
      float dcol[SB];
#pragma unroll
      for (int c = 0; c < SB; ++c) dcol[c] = Dm[c * (SB + 1) + tc];
#pragma unroll
      for (int ai = 0; ai < RI; ++ai) {
        const int i = tr + 32 * ai;
        float w = 0.0f;
        if (i < Q && (i < p0 || i >= p0 + SB)) {
          const float2* pr = reinterpret_cast<const float2*>(P + i * PST);
#pragma unroll
          for (int c2 = 0; c2 < SB / 2; ++c2) {
            const float2 v = pr[c2];
            w = fmaf(v.x, dcol[2 * c2], w);
            w = fmaf(v.y, dcol[2 * c2 + 1], w);
          }
        }
        W[i * PST + tc] = w;
      }
    }
    __syncthreads();
    // (d) rank-16 update X_ij -= W_i. P_j. (right for i, j outside K; the
    // K rows and columns are overwritten next).  Register blocks with
    // bj >= 2 ai + 2 hold only entries above the diagonal (j >= 32 ai + 32 > i),
    // which nothing reads: they are skipped.
#pragma unroll
    for (int c2 = 0; c2 < SB / 2; ++c2) {
      float2 pj[RJ];
#pragma unroll
      for (int bj = 0; bj < RJ; ++bj) pj[bj] = reinterpret_cast<const float2*>(P + (tc + 16 * bj) * PST)[c2];
#pragma unroll
      for (int ai = 0; ai < RI; ++ai) {
        const float2 wi = reinterpret_cast<const float2*>(W + (tr + 32 * ai) * PST)[c2];
#pragma unroll
        for (int bj = 0; bj < RJ; ++bj) {
          if (bj >= 2 * ai + 2) continue;
          x[ai][bj] = fmaf(-wi.x, pj[bj].x, x[ai][bj]);
          x[ai][bj] = fmaf(-wi.y, pj[bj].y, x[ai][bj]);
        }
      }
    }
    // (e) X_iK = W_iK, X_KK = -D^{-1}; rows of K: X_Kj = W_jK
#pragma unroll
    for (int bj = 0; bj < RJ; ++bj)
      if (bj == bj0) {
#pragma unroll
        for (int ai = 0; ai < RI; ++ai) {
          const int i = tr + 32 * ai;
          x[ai][bj] = (i >= p0 && i < p0 + SB) ? -Dm[(i - p0) * (SB + 1) + tc] : W[i * PST + tc];
        }
      }
    {
      const int c = tr - tr0;
      if (c >= 0 && c < SB) {
#pragma unroll
        for (int ai = 0; ai < RI; ++ai)
          if (ai == ai0) {
#pragma unroll
            for (int bj = 0; bj < RJ; ++bj)
              if (bj != bj0) x[ai][bj] = W[(tc + 16 * bj) * PST + c];
          }
      }
    }
  }
#pragma unroll
  for (int ai = 0; ai < RI; ++ai) {
    const int i = tr + 32 * ai;
#pragma unroll
    for (int bj = 0; bj < RJ; ++bj) {
      const int j = tc + 16 * bj;
      if (i < Q && j <= i) {
        slot[i * Q + j] = -x[ai][bj];
        slot[j * Q + i] = -x[ai][bj];
        Tm[i * Q + j] = -x[ai][bj];   // S_k^{-1} for the next plane's T
        Tm[j * Q + i] = -x[ai][bj];
      }
    }
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(SCHUR_THREADS)
k_btschur(const SubDesc* __restrict__ subs, T* __restrict__ facN, T* __restrict__ facD, T* __restrict__ scratch,
          long long smem_cap, int* err) {
  extern __shared__ __align__(128) unsigned char smraw[];
  const SubDesc s = subs[blockIdx.x];
  const int neumann = blockIdx.y == 0;
  const Grid g = grid_of(s, neumann);
  if (g.gz == 0) return;
  const int Q = g.gx * g.gy, gx = g.gx, gy = g.gy;
  const long long SS = slot_stride(Q), QQ = (long long)Q * Q;
  T* base = neumann ? facN + s.offN : facD + s.offD;
  const int QN = (s.w[0] + 1) * (s.w[1] + 1);
  T* Tm = scratch + s.offW + (neumann ? 0 : 2LL * QN * QN + 1024LL * ((max(QN, s.na) + 31) / 32));
  T* cb = reinterpret_cast<T*>(smraw);     // pivot columns, 2 x Q
  T* rb = cb + 2 * Q;                      // reciprocals of the pivots, 2
  T* A = (packed_size(Q) <= smem_cap) ? rb + 2 : Tm + QQ;
  const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;   // 32 x 16 owner grid
  // register path: FP32 planes of up to 176 nodes (6 x 11 entries per thread)
  constexpr int RI = 6, RJ = 11;
  // shared memory: Tm (Q x Q), then the panel buffers at a 16-byte boundary
  float* Tm_s = reinterpret_cast<float*>(smraw);
  float* pw = Tm_s + (((long long)Q * Q + 3) & ~3LL);
  const bool regs = std::is_same<T, float>::value && Q <= 32 * RI && Q <= 16 * RJ &&
                    (((long long)Q * Q + 3) & ~3LL) + schur_panel_floats() <= smem_cap;
  for (int k = 0; k < g.gz; ++k) {
    T* slot = base + (long long)k * SS;
    if (regs) {
      if constexpr (std::is_same<T, float>::value)
        schur_plane_regs<RI, RJ>(Q, gx, gy, k, slot, k > 0 ? base + (long long)(g.gz + k - 1) * SS : nullptr, pw,
                                 Tm_s, err, neumann ? 3 : 2, s.id);
      continue;
    }
    if (k > 0) {
      const T* Sp = base + (long long)(k - 1) * SS;       // S_{k-1}^{-1}, full
      const T* Bd = base + (long long)(g.gz + k - 1) * SS;
      // T = S_{k-1}^{-1} B_k^T:  T[i][j] = sum_o Sp[i][j + off_o] Bd[o][j]
      for (long long e = threadIdx.x; e < QQ; e += blockDim.x) {
        const int i = (int)(e / Q), j = (int)(e % Q), jx = j % gx, jy = j / gx;
        T acc = T(0);
#pragma unroll
        for (int o = 0; o < 9; ++o) {
          const int dx = o % 3 - 1, dy = o / 3 - 1;
          if (jx + dx >= 0 && jx + dx < gx && jy + dy >= 0 && jy + dy < gy)
            acc += Sp[(long long)i * Q + j + dx + dy * gx] * Bd[o * Q + j];
        }
        Tm[e] = acc;
      }
      __syncthreads();
      // S_k = D_k - B_k T (lower triangle, packed)
      for (int i = tr; i < Q; i += 32) {
        const int ix = i % gx, iy = i / gx;
        const long long ro = (long long)i * (i + 1) / 2;
        for (int j = tc; j <= i; j += 16) {
          T acc = T(0);
#pragma unroll
          for (int o = 0; o < 9; ++o) {
            const int dx = o % 3 - 1, dy = o / 3 - 1;
            if (ix + dx >= 0 && ix + dx < gx && iy + dy >= 0 && iy + dy < gy)
              acc += Bd[o * Q + i] * Tm[(long long)(i + dx + dy * gx) * Q + j];
          }
          A[ro + j] = slot[(long long)i * Q + j] - acc;
        }
      }
    } else {
      for (int i = tr; i < Q; i += 32) {
        const long long ro = (long long)i * (i + 1) / 2;
        for (int j = tc; j <= i; j += 16) A[ro + j] = slot[(long long)i * Q + j];
      }
    }
    __syncthreads();
    // first pivot column and reciprocal
    for (int i = threadIdx.x; i < Q; i += blockDim.x) cb[i] = A[(long long)i * (i + 1) / 2];
    if (threadIdx.x == 0) {
      T d = A[0];
      if (!(d > T(0))) { set_error(err, neumann ? 3 : 2, s.id); d = T(1); }
      rb[0] = T(1) / d;
    }
    __syncthreads();
    for (int p = 0; p < Q; ++p) {
      const T* c = cb + (p & 1) * Q;
      T* cn = cb + ((p + 1) & 1) * Q;
      const T r = rb[p & 1];
      const int q = p + 1;
      for (int i = tr; i < Q; i += 32) {
        const T ci = c[i], cir = ci * r;
        const long long ro = (long long)i * (i + 1) / 2;
        for (int j = tc; j <= i; j += 16) {
          T v;
          if (i == p) v = (j == p) ? -r : c[j] * r;
          else if (j == p) v = cir;
          else v = A[ro + j] - cir * c[j];
          A[ro + j] = v;
          if (j == q && i >= q) {
            cn[i] = v;
            if (i == q) {
              T d = v;
              if (!(d > T(0))) { set_error(err, neumann ? 3 : 2, s.id); d = T(1); }
              rb[q & 1] = T(1) / d;
            }
          } else if (i == q && j < q) {
            cn[j] = v;
          }
        }
      }
      __syncthreads();
    }
    // slot k <- S_k^{-1} = -A, both triangles
    for (int i = tr; i < Q; i += 32) {
      const long long ro = (long long)i * (i + 1) / 2;
      for (int j = tc; j <= i; j += 16) {
        const T v = -A[ro + j];
        slot[(long long)i * Q + j] = v;
        slot[(long long)j * Q + i] = v;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// multi-RHS solves: Y <- A_rr^{-1} Y with the Neumann factor (Y: nN x nc,
// row-major, ld nc).  grid: (subdomain, column chunk of CW columns).
//   forward  k = 1..nz-1:  Y_k -= B_k (S_{k-1}^{-1} Y_{k-1})
//   backward k = nz-1..0:  Y_k <- S_k^{-1} (Y_k - B_{k+1}^T Y_{k+1})
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(BDDC_THREADS)
k_btsolve_multi(const SubDesc* __restrict__ subs, const T* __restrict__ fac, T* __restrict__ Y,
                T* __restrict__ scratch, long long scratch_stride) {
  extern __shared__ __align__(128) unsigned char smraw[];
  DenseSmem<T>& sm = *reinterpret_cast<DenseSmem<T>*>(smraw);
  const SubDesc s = subs[blockIdx.y];   // chunks of one subdomain launch side by side (L2 reuse of its factor)
  const int c0 = blockIdx.x * CW;
  if (c0 >= s.nc) return;
  const int cw = min(CW, s.nc - c0);
  const Grid g = grid_of(s, 1);
  const int Q = g.gx * g.gy, nz = g.gz, ld = s.nc, gx = g.gx, gy = g.gy;
  const long long SS = slot_stride(Q);
  const T* base = fac + s.offN;
  T* Yb = Y + s.offY + c0;
  T* U = scratch + ((long long)blockIdx.y * gridDim.x + blockIdx.x) * scratch_stride;   // Q x cw
  for (int k = 1; k < nz; ++k) {
    T* Yk = Yb + (long long)k * Q * ld;
    cta_gemm<T>(Q, cw, Q, T(1), base + (long long)(k - 1) * SS, Q, false, Yk - (long long)Q * ld, ld, false, T(0),
                U, cw, 0, 0, false, sm);
    const T* Bd = base + (long long)(nz + k - 1) * SS;
    const int c = threadIdx.x % CW;
    if (c < cw)
      for (int i = threadIdx.x / CW; i < Q; i += BDDC_THREADS / CW) {
        const int ix = i % gx, iy = i / gx;
        T acc = T(0);
#pragma unroll
        for (int o = 0; o < 9; ++o) {
          const int dx = o % 3 - 1, dy = o / 3 - 1;
          if (ix + dx >= 0 && ix + dx < gx && iy + dy >= 0 && iy + dy < gy)
            acc += Bd[o * Q + i] * U[(i + dx + dy * gx) * cw + c];
        }
        Yk[(long long)i * ld + c] -= acc;
      }
    __syncthreads();
  }
  for (int k = nz - 1; k >= 0; --k) {
    T* Yk = Yb + (long long)k * Q * ld;
    const int c = threadIdx.x % CW;
    if (k == nz - 1) {
      if (c < cw)
        for (int l = threadIdx.x / CW; l < Q; l += BDDC_THREADS / CW) U[l * cw + c] = Yk[(long long)l * ld + c];
    } else {
      const T* Bd = base + (long long)(nz + k) * SS;       // B_{k+1}
      const T* Yn = Yk + (long long)Q * ld;
      if (c < cw)
        for (int l = threadIdx.x / CW; l < Q; l += BDDC_THREADS / CW) {
          const int lx = l % gx, ly = l / gx;
          T acc = T(0);
#pragma unroll
          for (int o = 0; o < 9; ++o) {
            const int dx = o % 3 - 1, dy = o / 3 - 1;
            if (lx - dx >= 0 && lx - dx < gx && ly - dy >= 0 && ly - dy < gy) {
              const int i = l - dx - dy * gx;
              acc += Bd[o * Q + i] * Yn[(long long)i * ld + c];
            }
          }
          U[l * cw + c] = Yk[(long long)l * ld + c] - acc;
        }
    }
    __syncthreads();
    cta_gemm<T>(Q, cw, Q, T(1), base + (long long)k * SS, Q, false, U, cw, false, T(0), Yk, ld, 0, 0, false, sm);
  }
}

// ---------------------------------------------------------------------------
// The same multi-RHS solves on the tensor cores (FP32 local path, Q <= 256):
// every product S^{-1} X (Q x Q times Q x 128) runs as tcgen05.mma kind::tf32
// with 3xTF32 splitting, two M tiles of 128 rows, accumulators in TMEM
// (2 x 128 columns), K streamed in chunks of 32 through two shared-memory
// stages (A hi/lo 2 x 32 KiB, B hi/lo 2 x 16 KiB each) so that staging chunk
// n + 1 overlaps the MMAs of chunk n.  grid: (subdomain, 128-column chunk),
// 256 threads; thread 0 issues the MMAs, every wait is bounded.
// ---------------------------------------------------------------------------
constexpr int TC_N = 128, TC_KC = 32;
constexpr unsigned TC_A_BYTES = 2u * 2u * 128u * TC_KC * 4u;   // up to two 128-row tiles, hi and lo
constexpr unsigned TC_B_BYTES = (unsigned)TC_N * TC_KC * 4u;
constexpr unsigned TC_STAGE_BYTES = TC_A_BYTES + 2u * TC_B_BYTES;

// Packs the Neumann S_k^{-1} into the tiles the tensor cores read: per
// (plane, K chunk of 32), for each 128-row tile a hi and a lo tile (3xTF32
// split) in the canonical K-major order, so that the products load their A
// operand with one bulk copy per chunk.  grid: (subdomain, plane, K chunk).
__global__ void k_tc_pack(const SubDesc* __restrict__ subs, const float* __restrict__ facN, float* __restrict__ tiles) {
  const SubDesc s = subs[blockIdx.x];
  const Grid g = grid_of(s, 1);
  const int Q = g.gx * g.gy, k = blockIdx.y, kc = blockIdx.z;
  if (k >= g.gz || kc >= tc_kchunks(Q)) return;
  const float* S = facN + s.offN + (long long)k * slot_stride(Q);
  float* dst = tiles + s.offTC + ((long long)k * tc_kchunks(Q) + kc) * tc_chunk_floats(Q);
  for (int e = threadIdx.x; e < tc_mtiles(Q) * 4096; e += blockDim.x) {
    const int m = e >> 12, ei = e & 4095;
    const int q = ei & 3, rr = (ei >> 2) & 7, cc = (ei >> 5) & 7, gg = ei >> 8;
    const int r = m * 128 + gg * 8 + rr, col = kc * TC_KC + cc * 4 + q;
    const float x = (r < Q && col < Q) ? S[r * Q + col] : 0.0f;
    const float hi = umma::to_tf32(x);
    dst[m * 8192 + ei] = hi;
    dst[m * 8192 + 4096 + ei] = umma::to_tf32(x - hi);
  }
}

struct TcState {
  unsigned char* stage;   // 2 stages of TC_STAGE_BYTES
  uint64_t* bar;          // per stage: the MMAs that read it have completed
  uint64_t* tbar;         // per stage: the bulk copy of its A tiles has landed
  uint32_t tmem;
  int next;               // chunks issued so far (stage = next & 1)
};

// TMEM <- S (Q x Q, packed tiles of one plane) X (Q x ncol, ld ldx); on
// return the products are complete and visible to every thread
__device__ void tc_product(TcState& G, const float* __restrict__ Atiles, int Q, const float* __restrict__ X,
                           long long ldx, int ncol, int* err) {
  const int nkc = tc_kchunks(Q), nmt = tc_mtiles(Q);
  const uint32_t idesc = umma::idesc_tf32(128, TC_N);
  for (int kc = 0; kc < nkc; ++kc) {
    const int b = G.next & 1;
    unsigned char* st = G.stage + (size_t)b * TC_STAGE_BYTES;
    if (threadIdx.x == 0) {
      if (G.next >= 2) mbar_wait_bounded(&G.bar[b], (unsigned)(((G.next >> 1) - 1) & 1), err);
      bulk_load(st, Atiles + (long long)kc * tc_chunk_floats(Q), (unsigned)nmt * 32768u, &G.tbar[b]);
    }
    __syncthreads();
    float* Bhi = reinterpret_cast<float*>(st + TC_A_BYTES);
    float* Blo = reinterpret_cast<float*>(st + TC_A_BYTES + TC_B_BYTES);
    const int k0 = kc * TC_KC;
    // B: row n of B is column n of X (K-major operand); all loads of a thread
    // are issued before any conversion so that their latencies overlap
    constexpr int NB = TC_N * TC_KC / BDDC_THREADS;
    float xb[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const int e = threadIdx.x + j * BDDC_THREADS;
      const int kk = e / TC_N, n = e % TC_N, k = k0 + kk;
      xb[j] = (n < ncol && k < Q) ? X[(long long)k * ldx + n] : 0.0f;
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const int e = threadIdx.x + j * BDDC_THREADS;
      const unsigned o = umma::kmajor_offset(e % TC_N, e / TC_N, TC_KC) >> 2;
      const float hi = umma::to_tf32(xb[j]);
      Bhi[o] = hi;
      Blo[o] = umma::to_tf32(xb[j] - hi);
    }
    fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
      mbar_wait_bounded(&G.tbar[b], (unsigned)((G.next >> 1) & 1), err);
      umma::fence_after_sync();
      const unsigned sbo = (TC_KC / 4) * 128;
      const unsigned a0 = umma::smem_u32(st);
      const unsigned b_hi = umma::smem_u32(Bhi), b_lo = umma::smem_u32(Blo);
#pragma unroll
      for (int ks = 0; ks < TC_KC / 8; ++ks) {
        const unsigned ko = ks * 256;   // 8 TF32 values = two core matrices along K
        const uint64_t bh = umma::smem_desc(b_hi + ko, 128, sbo), bl = umma::smem_desc(b_lo + ko, 128, sbo);
        for (int m = 0; m < nmt; ++m) {
          const unsigned a_hi = a0 + m * 32768u, a_lo = a_hi + 16384u;
          const uint64_t ah = umma::smem_desc(a_hi + ko, 128, sbo), al = umma::smem_desc(a_lo + ko, 128, sbo);
          const uint32_t d = G.tmem + (uint32_t)(m * TC_N);
          umma::mma_tf32(d, ah, bh, idesc, kc > 0 || ks > 0);
          umma::mma_tf32(d, ah, bl, idesc, true);
          umma::mma_tf32(d, al, bh, idesc, true);
        }
      }
      umma::commit(&G.bar[b]);
    }
    ++G.next;
  }
  if (threadIdx.x == 0) mbar_wait_bounded(&G.bar[(G.next - 1) & 1], (unsigned)(((G.next - 1) >> 1) & 1), err);
  __syncthreads();
  umma::fence_after_sync();
}

// The product's rows also go to a shared-memory copy (row i at i * TC_N) in
// the stage area past the readback's transpose buffers, where the stencil that
// follows reads its nine taps per entry.
constexpr unsigned TC_TB_BYTES = 8u * 32u * 33u * 4u;   // per-warp 32 x 33 transpose buffers
__device__ inline float* tc_rows(const TcState& G) {
  return reinterpret_cast<float*>(G.stage + ((TC_TB_BYTES + 127u) & ~127u));
}

// dst[i][n] = product row i (i < Q, n < ncol), ld ldd (dst may be null), and
// the shared copy tc_rows(G); warps 0-3 read the first 128 rows, warps 4-7
// the second.  A lane holds one row, so each warp turns its 32 x 32 blocks
// around in shared memory (the stages are idle once the products are
// complete) and stores whole row segments.
__device__ void tc_readback(const TcState& G, int Q, int ncol, float* __restrict__ dst, long long ldd) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, m = warp >> 2, quad = warp & 3;
  const int row0 = m * 128 + quad * 32;
  float* tb = reinterpret_cast<float*>(G.stage) + warp * 32 * 33;
  float* rows = tc_rows(G);
  for (int c = 0; c < TC_N; c += 32) {
    float v[32];
    umma::ld32(G.tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(m * TC_N + c), v);
#pragma unroll
    for (int j = 0; j < 32; ++j) tb[lane * 33 + j] = v[j];
    __syncwarp();
    for (int r = 0; r < 32 && row0 + r < Q; ++r) {
      const float x = (c + lane < ncol) ? tb[r * 33 + lane] : 0.0f;
      rows[(row0 + r) * TC_N + c + lane] = x;
      if (dst && c + lane < ncol) dst[(long long)(row0 + r) * ldd + c + lane] = x;
    }
    __syncwarp();
  }
  umma::fence_before_sync();
  __syncthreads();
}

// Stencil steps of the tensor-core solves, one column per thread.  The taps
// come from the shared copy of the last product (src, row stride TC_N); the
// loads of Y_k come from L2, so a thread first issues them for RS rows and
// then does the arithmetic of those rows.
// Bd: nine diagonals of the coupling in shared memory.
//   forward:  Y_k[i][c] -= sum_o Bd[o][i] U[i + off_o][c]
//   backward: U[l][c] = Y_k[l][c] - sum_o Bd[o][l - off_o] Y_{k+1}[l - off_o][c]
template <bool FWD>
__device__ void tc_stencil(int Q, int gx, int gy, int cw, const float* Bd, const float* __restrict__ src,
                           float* __restrict__ Yk, long long ld, float* __restrict__ U) {
  constexpr int RS = 24, STEP = BDDC_THREADS / TC_N;
  const int c = threadIdx.x % TC_N;
  if (c >= cw) return;
  for (int i0 = threadIdx.x / TC_N; i0 < Q; i0 += STEP * RS) {
    float y[RS];
#pragma unroll
    for (int u = 0; u < RS; ++u) {
      const int i = min(i0 + u * STEP, Q - 1);
      y[u] = Yk[(long long)i * ld + c];
    }
#pragma unroll
    for (int u = 0; u < RS; ++u) {
      const int i = i0 + u * STEP;
      if (i >= Q) break;
      const int ix = i % gx, iy = i / gx;
      float acc = 0.0f;
#pragma unroll
      for (int o = 0; o < 9; ++o) {
        const int dx = o % 3 - 1, dy = o / 3 - 1;
        const int sx = FWD ? dx : -dx, sy = FWD ? dy : -dy;
        const bool ok = ix + sx >= 0 && ix + sx < gx && iy + sy >= 0 && iy + sy < gy;
        const int j = ok ? i + sx + sy * gx : i;
        const float wv = ok ? Bd[o * Q + (FWD ? i : j)] : 0.0f;
        acc = fmaf(wv, src[j * TC_N + c], acc);
      }
      if (FWD) Yk[(long long)i * ld + c] = y[u] - acc;
      else U[i * TC_N + c] = y[u] - acc;
    }
  }
}

__global__ void __launch_bounds__(BDDC_THREADS, 1)
k_btsolve_multi_tc(const SubDesc* __restrict__ subs, const float* __restrict__ fac,
                   const float* __restrict__ tiles, float* __restrict__ Y, float* __restrict__ scratch,
                   long long scratch_stride, int* err) {
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ __align__(8) uint64_t bars[4];
  __shared__ uint32_t tmem_slot;
  const SubDesc s = subs[blockIdx.y];   // chunks of one subdomain launch side by side (L2 reuse of its factor)
  const int c0 = blockIdx.x * TC_N;
  if (c0 >= s.nc) return;
  const int cw = min(TC_N, s.nc - c0);
  const Grid g = grid_of(s, 1);
  const int Q = g.gx * g.gy, nz = g.gz, ld = s.nc, gx = g.gx, gy = g.gy;
  const long long SS = slot_stride(Q);
  const float* base = fac + s.offN;
  float* Yb = Y + s.offY + c0;
  float* U = scratch + ((long long)blockIdx.y * gridDim.x + blockIdx.x) * scratch_stride;   // Q x TC_N
  if (threadIdx.x == 0) {
    for (int q = 0; q < 4; ++q) mbar_init(&bars[q], 1);
    fence_barrier_init();
  }
  if (threadIdx.x < 32) umma::tmem_alloc(&tmem_slot, 2 * TC_N);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  TcState G{smraw, bars, bars + 2, tmem_slot, 0};
  const float* At = tiles + s.offTC;
  float* Bs = reinterpret_cast<float*>(smraw + 2 * TC_STAGE_BYTES);   // nine coupling diagonals
  const long long plane_floats = (long long)tc_kchunks(Q) * tc_chunk_floats(Q);
  for (int k = 1; k < nz; ++k) {
    float* Yk = Yb + (long long)k * Q * ld;
    tc_product(G, At + (long long)(k - 1) * plane_floats, Q, Yk - (long long)Q * ld, ld, cw, err);
    tc_readback(G, Q, cw, nullptr, 0);
    const float* Bg = base + (long long)(nz + k - 1) * SS;
    for (int e = threadIdx.x; e < 9 * Q; e += blockDim.x) Bs[e] = Bg[e];
    __syncthreads();
    tc_stencil<true>(Q, gx, gy, cw, Bs, tc_rows(G), Yk, ld, nullptr);
    __syncthreads();
  }
  for (int k = nz - 1; k >= 0; --k) {
    float* Yk = Yb + (long long)k * Q * ld;
    if (k == nz - 1) {
      tc_product(G, At + (long long)k * plane_floats, Q, Yk, ld, cw, err);
    } else {
      const float* Bg = base + (long long)(nz + k) * SS;       // B_{k+1}
      for (int e = threadIdx.x; e < 9 * Q; e += blockDim.x) Bs[e] = Bg[e];
      __syncthreads();
      tc_stencil<false>(Q, gx, gy, cw, Bs, tc_rows(G), Yk, ld, U);   // taps: Y_{k+1}, kept by the readback
      __syncthreads();
      tc_product(G, At + (long long)k * plane_floats, Q, U, TC_N, cw, err);
    }
    tc_readback(G, Q, cw, Yk, ld);
  }
  if (threadIdx.x < 32) umma::tmem_dealloc(G.tmem, 2 * TC_N);
}

// ---------------------------------------------------------------------------
// coarse basis
// ---------------------------------------------------------------------------

// F = [-A_rv | C_r^T] on the local Neumann grid (rows), into Y.  own: per
// local Neumann node (at the subdomain's vector offset) the local index of
// the average containing it, -1 if none.
template <typename T>
__global__ void k_coarse_rhs(const SubDesc* __restrict__ subs, MeshDev m, const double* __restrict__ alpha,
                             const LocalCoarse* __restrict__ lc, const int* __restrict__ own, T* __restrict__ Y) {
  const SubDesc s = subs[blockIdx.x];
  const int px = s.w[0] + 1, py = s.w[1] + 1, pz = s.w[2] + 1;
  const long long nN = (long long)px * py * pz;
  T* Yb = Y + s.offY;
  for (long long e = (long long)blockIdx.y * blockDim.x + threadIdx.x; e < nN * s.nc;
       e += (long long)gridDim.y * blockDim.x) {
    int r = (int)(e / s.nc), j = (int)(e % s.nc);
    int ix = r % px, iy = (r / px) % py, iz = r / (px * py);
    double v = 0.0;
    if (!neumann_fixed(m, s, ix, iy, iz)) {
      const LocalCoarse c = lc[s.cofs + j];
      if (j < s.nv) {
        int dx = c.v[0] - ix, dy = c.v[1] - iy, dz = c.v[2] - iz;
        if (abs(dx) <= 1 && abs(dy) <= 1 && abs(dz) <= 1)
          v = -box_entry(m, alpha, s, s.e0[0] + ix, s.e0[1] + iy, s.e0[2] + iz, dx, dy, dz);
      } else if (own[s.offVec + r] == j) {
        v = 1.0 / c.count;
      }
    }
    Yb[e] = (T)v;
  }
}

// G = C_r Y (na x nc): means of Y's columns over the averaging objects.
template <typename T>
__global__ void k_constraint_means(const SubDesc* __restrict__ subs, const LocalCoarse* __restrict__ lc,
                                   const int* __restrict__ lcn, const T* __restrict__ Y, T* __restrict__ G) {
  const SubDesc s = subs[blockIdx.x];
  const T* Yb = Y + s.offY;
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < s.na * s.nc; e += gridDim.y * blockDim.x) {
    int a = e / s.nc, j = e % s.nc;
    const LocalCoarse c = lc[s.cofs + s.nv + a];
    T sum = T(0);
    for (int q = 0; q < c.count; ++q) sum += Yb[(long long)lcn[c.off + q] * s.nc + j];
    G[s.offG + e] = sum / T(c.count);
  }
}

// S_c = G[:, nv:] -> S_c^{-1} (into Sc) and Lambda_v = S_c^{-1} G[:, :nv] (into Lv).
template <typename T>
__global__ void __launch_bounds__(BDDC_THREADS)
k_schur(const SubDesc* __restrict__ subs, T* __restrict__ G, T* __restrict__ Sc, T* __restrict__ Lv,
        T* __restrict__ scratch, int* err) {
  extern __shared__ __align__(128) unsigned char smraw[];
  DenseSmem<T>& sm = *reinterpret_cast<DenseSmem<T>*>(smraw);
  const SubDesc s = subs[blockIdx.x];
  const int na = s.na, nv = s.nv, nc = s.nc;
  if (na == 0) return;
  T* Gs = G + s.offG;
  T* S = Gs + nv;               // na x na, ld nc; factored in place
  T* Linv = Sc + s.offSc;       // na x na
  T* diag = scratch + s.offW;
  bool ok = cta_chol_inv<T>(S, nc, Linv, na, na, diag, sm);
  if (!ok && threadIdx.x == 0) set_error(err, 4, s.id);
  // S_c^{-1} = Linv^T Linv -> into the free S region, then back to Sc
  cta_gemm<T>(na, na, na, T(1), Linv, na, true, Linv, na, false, T(0), S, nc, 2, 2, false, sm);
  for (int e = threadIdx.x; e < na * na; e += blockDim.x) Linv[e] = S[(long long)(e / na) * nc + e % na];
  __syncthreads();
  if (nv > 0)
    cta_gemm<T>(na, nv, na, T(1), Linv, na, false, Gs, nc, false, T(0), Lv + s.offL, nv, 0, 0, false, sm);
}

// Row-chunked products on the nN rows of Y:
//   mode 0: Y[:, :nv] -= X Lambda_v         (Phi_rv)
//   mode 1: PA = X S_c^{-1}                  (Phi_ra)
// grid: (subdomain, row chunk of RB rows).
constexpr int RB = 128;
template <typename T>
__global__ void __launch_bounds__(BDDC_THREADS)
k_phi_rows(const SubDesc* __restrict__ subs, T* __restrict__ Y, const T* __restrict__ Lv,
           const T* __restrict__ Sc, T* __restrict__ PA, int mode) {
  extern __shared__ __align__(128) unsigned char smraw[];
  DenseSmem<T>& sm = *reinterpret_cast<DenseSmem<T>*>(smraw);
  const SubDesc s = subs[blockIdx.x];
  const int nN = (s.w[0] + 1) * (s.w[1] + 1) * (s.w[2] + 1);
  const int r0 = blockIdx.y * RB;
  if (r0 >= nN || s.na == 0) return;
  const int rows = min(RB, nN - r0);
  T* Yr = Y + s.offY + (long long)r0 * s.nc;
  if (mode == 0) {
    if (s.nv == 0) return;
    cta_gemm<T>(rows, s.nv, s.na, T(-1), Yr + s.nv, s.nc, false, Lv + s.offL, s.nv, false, T(1), Yr, s.nc,
                0, 0, false, sm);
  } else {
    cta_gemm<T>(rows, s.na, s.na, T(1), Yr + s.nv, s.nc, false, Sc + s.offSc, s.na, false, T(0),
                PA + s.offPA + (long long)r0 * s.na, s.na, 0, 0, false, sm);
  }
}

// Phi on the box surface: vertex columns from Y (+1 at the vertex itself),
// average columns from PA.
template <typename T>
__global__ void k_phi_surface(const SubDesc* __restrict__ subs, const LocalCoarse* __restrict__ lc,
                              const T* __restrict__ Y, const T* __restrict__ PA, T* __restrict__ Phi) {
  const SubDesc s = subs[blockIdx.x];
  const int px = s.w[0] + 1, py = s.w[1] + 1, pz = s.w[2] + 1;
  for (long long e = (long long)blockIdx.y * blockDim.x + threadIdx.x; e < (long long)s.nB * s.nc;
       e += (long long)gridDim.y * blockDim.x) {
    int b = (int)(e / s.nc), j = (int)(e % s.nc);
    int ix, iy, iz;
    surf_coords(b, px, py, pz, ix, iy, iz);
    long long node = (long long)ix + px * (iy + (long long)py * iz);
    T v;
    if (j < s.nv) {
      const LocalCoarse c = lc[s.cofs + j];
      v = Y[s.offY + node * s.nc + j];
      if (c.v[0] == ix && c.v[1] == iy && c.v[2] == iz) v = T(1);
    } else {
      v = PA[s.offPA + node * s.na + (j - s.nv)];
    }
    Phi[s.offPhi + e] = v;
  }
}

// Local coarse matrix Phi^T A Phi (FP64, nc x nc).
template <typename T>
__global__ void k_local_coarse_matrix(const SubDesc* __restrict__ subs, MeshDev m,
                                      const double* __restrict__ alpha, const LocalCoarse* __restrict__ lc,
                                      const T* __restrict__ Y, const T* __restrict__ Lv,
                                      const T* __restrict__ Sc, const double* __restrict__ pen,
                                      double* __restrict__ Ac) {
  const SubDesc s = subs[blockIdx.x];
  const int px = s.w[0] + 1, py = s.w[1] + 1, pz = s.w[2] + 1;
  const int nc = s.nc, nv = s.nv;
  double* A = Ac + s.offAc;
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < nc * nc; e += gridDim.y * blockDim.x) {
    int r = e / nc, c = e % nc;
    double v;
    if (r < nv && c < nv) {
      // (A Phi_v)[vertex r, column c], symmetrised
      double both[2];
      for (int t = 0; t < 2; ++t) {
        int row = t ? c : r, col = t ? r : c;
        const LocalCoarse vr = lc[s.cofs + row];
        const LocalCoarse vc = lc[s.cofs + col];
        double acc = 0.0;
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              int bx = vr.v[0] + dx, by = vr.v[1] + dy, bz = vr.v[2] + dz;
              if (bx < 0 || by < 0 || bz < 0 || bx >= px || by >= py || bz >= pz) continue;
              if (on_dirichlet(m, s.e0[0] + bx, s.e0[1] + by, s.e0[2] + bz)) continue;
              double phi;
              if (bx == vc.v[0] && by == vc.v[1] && bz == vc.v[2]) phi = 1.0;
              else phi = (double)Y[s.offY + ((long long)bx + px * (by + (long long)py * bz)) * nc + col];
              if (phi == 0.0) continue;
              acc += box_entry(m, alpha, s, s.e0[0] + vr.v[0], s.e0[1] + vr.v[1], s.e0[2] + vr.v[2],
                               dx, dy, dz) * phi;
            }
        both[t] = acc;
      }
      v = 0.5 * (both[0] + both[1]);
    } else if (r >= nv && c >= nv) {
      int a = r - nv, b = c - nv;
      v = 0.5 * ((double)Sc[s.offSc + (long long)a * s.na + b] + (double)Sc[s.offSc + (long long)b * s.na + a]);
      if (s.pin && r == c) v -= pen[s.cofs + r];   // Phi^T A Phi of a pinned subdomain (k_pin_penalty)
    } else if (r >= nv) {
      v = -(double)Lv[s.offL + (long long)(r - nv) * nv + c];
    } else {
      v = -(double)Lv[s.offL + (long long)(c - nv) * nv + r];
    }
    A[e] = v;
  }
}

// Weights on the box surface of subdomain i (eq. (W), Remark 1): over the
// sub-subdomains (pieces) of the elements around a node, the sum of their
// weights inside Omega_i over the sum of all (pw = NULL: every piece counts
// 1, the cardinality rule).  The pieces around a node are the distinct
// labels of its up to eight elements, visited z, y, x.
__global__ void k_weights(const SubDesc* __restrict__ subs, MeshDev m, const double* __restrict__ pw,
                          double* __restrict__ delta) {
  const SubDesc s = subs[blockIdx.x];
  const int px = s.w[0] + 1, py = s.w[1] + 1, pz = s.w[2] + 1;
  int slabS[3];
  for (int d = 0; d < 3; ++d) slabS[d] = m.ax[d].slab[s.e0[d]];
  for (int b = blockIdx.y * blockDim.x + threadIdx.x; b < s.nB; b += gridDim.y * blockDim.x) {
    int ix, iy, iz;
    surf_coords(b, px, py, pz, ix, iy, iz);
    const int gc[3] = {s.e0[0] + ix, s.e0[1] + iy, s.e0[2] + iz};
    if (on_dirichlet(m, gc[0], gc[1], gc[2])) { delta[s.offB + b] = 0.0; continue; }
    int seen[8], n = 0;
    double num = 0.0, den = 0.0;
    for (int dz = -1; dz <= 0; ++dz)
      for (int dy = -1; dy <= 0; ++dy)
        for (int dx = -1; dx <= 0; ++dx) {
          const int ex = gc[0] + dx, ey = gc[1] + dy, ez = gc[2] + dz;   // inside: node off the boundary
          const int p = m.epiece[ex + (long long)m.nx * (ey + (long long)m.ny * ez)];
          bool dup = false;
          for (int q = 0; q < n; ++q) dup = dup || seen[q] == p;
          if (dup) continue;
          seen[n++] = p;
          const double w = pw ? pw[p] : 1.0;
          den += w;
          if (m.ax[0].slab[ex] == slabS[0] && m.ax[1].slab[ey] == slabS[1] && m.ax[2].slab[ez] == slabS[2]) num += w;
        }
    delta[s.offB + b] = num / den;
  }
}

// Device tables of the local kernels, from the coarse-DOF lists: the
// point-value flag of every node (vfix, zeroed before; a vertex shared by
// several subdomains gets the same value from each) and every subdomain's
// local-node -> average map (own at the vector offsets, -1 before; the
// objects of one subdomain are disjoint).  One CTA per subdomain.
__global__ void k_mark_coarse(const SubDesc* __restrict__ subs, const LocalCoarse* __restrict__ lc,
                              const int* __restrict__ lcn, int NX, int NY, unsigned char* __restrict__ vfix,
                              int* __restrict__ own) {
  const SubDesc s = subs[blockIdx.x];
  for (int j = threadIdx.x; j < s.nc; j += blockDim.x) {
    const LocalCoarse c = lc[s.cofs + j];
    if (j < s.nv) {
      vfix[nodeid(NX, NY, s.e0[0] + c.v[0], s.e0[1] + c.v[1], s.e0[2] + c.v[2])] = 1;
    } else {
      for (int q = 0; q < c.count; ++q) own[s.offVec + lcn[c.off + q]] = j;
    }
  }
}

// Box sub-subdomains: piece of every element from the per-axis piece
// numbers, a + npx (b + npy c).
__global__ void k_box_pieces(int nx, int ny, int nz, const int* __restrict__ pa, const int* __restrict__ pb,
                             const int* __restrict__ pc, int npx, int npy, int* __restrict__ epiece) {
  const long long ne = (long long)nx * ny * nz;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % nx), j = (int)((e / nx) % ny), k = (int)(e / ((long long)nx * ny));
    epiece[e] = pa[i] + npx * (pb[j] + npy * pc[k]);
  }
}

// Mean alpha of every box sub-subdomain: its element box [lo, hi) per axis
// (concatenated x, y, z tables), summed over k, j, i ascending.
__global__ void k_piece_alpha_box(const double* __restrict__ alpha, int nx, int ny, const int* __restrict__ plo,
                                  const int* __restrict__ phi, int npx, int npy, int npz, double* __restrict__ pw) {
  const long long np = (long long)npx * npy * npz;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(p % npx), b = (int)((p / npx) % npy), c = (int)(p / ((long long)npx * npy));
    const int x0 = plo[a], x1 = phi[a], y0 = plo[npx + b], y1 = phi[npx + b], z0 = plo[npx + npy + c],
              z1 = phi[npx + npy + c];
    double sum = 0.0;
    for (int k = z0; k < z1; ++k)
      for (int j = y0; j < y1; ++j)
        for (int i = x0; i < x1; ++i) sum += alpha[(long long)i + (long long)nx * (j + (long long)ny * k)];
    pw[p] = sum / ((double)(x1 - x0) * (y1 - y0) * (z1 - z0));
  }
}

// Mean alpha of every sub-subdomain (piece): its elements listed in
// ascending order (pe_off, pe), summed in that order.
__global__ void k_piece_alpha(const double* __restrict__ alpha, const long long* __restrict__ pe_off,
                              const int* __restrict__ pe, int np, double* __restrict__ pw) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
    double sum = 0.0;
    for (long long q = pe_off[p]; q < pe_off[p + 1]; ++q) sum += alpha[pe[q]];
    pw[p] = sum / (double)(pe_off[p + 1] - pe_off[p]);
  }
}

// ---------------------------------------------------------------------------
// transposed copy of Phi (nB x nc -> nc x nB) for the apply's column
// accumulations.  grid: (subdomain, 1, 32x32 tile stride)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_transpose(const SubDesc* __restrict__ subs, const T* __restrict__ src, T* __restrict__ dst) {
  __shared__ T tile[32][33];
  const SubDesc s = subs[blockIdx.x];
  const int rows = s.nB, cols = s.nc;
  if (rows == 0 || cols == 0) return;
  const int tc = (cols + 31) / 32, tr = (rows + 31) / 32;
  const T* A = src + s.offPhi;
  T* B = dst + s.offPhi;
  for (int t = blockIdx.z; t < tr * tc; t += gridDim.z) {
    const int r0 = (t / tc) * 32, c0 = (t % tc) * 32;
    for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
      int r = e / 32, c = e % 32;
      if (r0 + r < rows && c0 + c < cols) tile[r][c] = A[(long long)(r0 + r) * cols + c0 + c];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
      int c = e / 32, r = e % 32;
      if (r0 + r < rows && c0 + c < cols) B[(long long)(c0 + c) * rows + r0 + r] = tile[r][c];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// column accumulation over streamed row chunks: acc[c] += sum_r A[r][c] x[r].
// With ncol <= blockDim the threads form G = blockDim / ncol row groups (one
// column each); otherwise every thread owns up to 4 columns.
// ---------------------------------------------------------------------------
struct ColLayout {
  int ncol, G, grp, col;  // col < 0: idle thread
};
__device__ inline ColLayout col_layout(int ncol) {
  ColLayout L;
  L.ncol = ncol;
  if (ncol <= (int)blockDim.x) {
    L.G = blockDim.x / ncol;
    L.grp = threadIdx.x / ncol;
    L.col = (L.grp < L.G) ? (int)(threadIdx.x % ncol) : -1;
  } else {
    L.G = 1; L.grp = 0; L.col = threadIdx.x;
  }
  return L;
}

template <typename A, typename T, typename X>
__device__ inline void col_accumulate(const ColLayout& L, const T* __restrict__ ch, int nr, const X* __restrict__ x,
                                      A acc[4]) {
  if (L.col < 0) return;
  if (L.G > 1) {
    // one column per thread: four rows per step on separate partial sums, so
    // that their shared-memory loads are in flight together
    const int c = L.col, G = L.G;
    A a0 = A(0), a1 = A(0), a2 = A(0), a3 = A(0);
    int r = L.grp;
    for (; r + 3 * G < nr; r += 4 * G) {
      a0 += (A)ch[(long long)r * L.ncol + c] * (A)x[r];
      a1 += (A)ch[(long long)(r + G) * L.ncol + c] * (A)x[r + G];
      a2 += (A)ch[(long long)(r + 2 * G) * L.ncol + c] * (A)x[r + 2 * G];
      a3 += (A)ch[(long long)(r + 3 * G) * L.ncol + c] * (A)x[r + 3 * G];
    }
    for (; r < nr; r += G) a0 += (A)ch[(long long)r * L.ncol + c] * (A)x[r];
    acc[0] += (a0 + a1) + (a2 + a3);
    return;
  }
  for (int r = L.grp; r < nr; r += L.G) {
    const A xv = (A)x[r];
    const T* row = ch + (long long)r * L.ncol;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = L.col + q * (int)blockDim.x;
      if (q > 0 && L.G > 1) break;
      if (c < L.ncol) acc[q] += (A)row[c] * xv;
    }
  }
}

// Sums the row-group partials (every thread calls; contains a barrier) and
// hands each column's total to out(c, total) on the group-0 threads.
template <typename A, typename Out>
__device__ inline void col_finish(const ColLayout& L, A acc[4], A* part, Out out) {
  if (L.G > 1) {
    if (L.col >= 0) part[L.grp * L.ncol + L.col] = acc[0];
    __syncthreads();
    if (L.col >= 0 && L.grp == 0) {
      A s = A(0);
      for (int g = 0; g < L.G; ++g) s += part[g * L.ncol + L.col];
      out(L.col, s);
    }
    __syncthreads();
  } else if (L.col >= 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = L.col + q * (int)blockDim.x;
      if (c < L.ncol) out(c, acc[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[q] = A(0);
}

// ---------------------------------------------------------------------------
// single-RHS solve (apply): v <- A^{-1} v with the inverse Schur complements
//   forward  k = 1..nz-1:  t = S_{k-1}^{-1} v_{k-1};  v_k -= B_k t
//   backward k = nz-1..0:  v_k <- S_k^{-1} (v_k - B_{k+1}^T v_{k+1})
// The 2 nz - 1 symmetric slots stream through the ring in that order and
// their products are column accumulations (S^{-1} is symmetric, so rows are
// columns); the nine-diagonal B_k and B_{k+1}^T products run between them.
// A subdomain is solved by a cluster of two CTAs: each streams one half of
// the rows of every slot, and the two partial column sums meet through
// distributed shared memory (rank 0's plus rank 1's, the same on both CTAs,
// so both keep identical copies of v and t).  Each CTA streams the coupling
// diagonals itself and runs the stencils redundantly.  Every CTA finishes
// every slot and passes the same cluster barriers in the same order, whatever
// its share of rows.  v (nz*Q), t (Q), part (blockDim), pb (2 Q) in shared
// memory.
// ---------------------------------------------------------------------------
// rows of a row-major matrix (cols entries of es bytes per row) per rank when
// nrank CTAs share it: ceil(rows / nrank) rounded up to the row step that
// keeps a 16-byte alignment
__device__ inline int split_rows(int rows, int cols, int es, int nrank) {
  int step = 1;
  while ((step * cols * es) % 16) ++step;
  const int h = (rows + nrank - 1) / nrank;
  return (h + step - 1) / step * step;
}

template <typename T>
__device__ void sweep_stream(Ring& ring, const T* __restrict__ fac, int gx, int gy, int nz, T* v, T* t, T* part,
                             T* pb, int* err) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank(), nrank = (int)cluster.num_blocks();
  const int Q = gx * gy;
  const int R = rows_per_chunk(Q, (int)sizeof(T));
  // this CTA's rows of every slot: [rlo, rhi), in chunks of R rows; the split
  // keeps every chunk start on a 16-byte boundary (bulk copies require it)
  const int half = split_rows(Q, Q, (int)sizeof(T), nrank);
  const int rlo = min(Q, rank * half), rhi = min(Q, rlo + half);
  const int nch = (rhi - rlo + R - 1) / R;
  const int ngs = nch + 1;                 // slot chunks plus the coupling's diagonals
  const int nlead = 2 * (nz - 1);          // groups followed by a stencil step
  const long long SS = slot_stride(Q);
  auto slot_of = [&](int bi) { return bi < nz - 1 ? bi : 2 * nz - 2 - bi; };
  auto locate = [&](int c, int& bi, int& lc) {
    if (c < nlead * ngs) { bi = c / ngs; lc = c % ngs; }
    else { bi = nlead; lc = c - nlead * ngs; }
  };
  const ColLayout L = col_layout(Q);
  T acc[4] = {T(0), T(0), T(0), T(0)};
  // partial sums of the slot of group bi -> both CTAs' shares added in rank
  // order -> dst (double-buffered by group, so that a CTA never overwrites a
  // buffer its peer may still read)
  auto finish = [&](int bi, T* dst) {
    if (nrank == 1) {   // a CTA of its own: straight to the destination
      col_finish<T>(L, acc, part, [&](int cc, T sum) { dst[cc] = sum; });
      if (L.G == 1) __syncthreads();   // (with row groups col_finish ends with one)
      return;
    }
    T* mine = pb + (bi & 1) * Q;
    col_finish<T>(L, acc, part, [&](int cc, T sum) { mine[cc] = sum; });
    cluster.sync();
    for (int c = threadIdx.x; c < Q; c += blockDim.x) {
      T s = T(0);
      for (int r = 0; r < nrank; ++r) s += cluster.map_shared_rank(mine, r)[c];
      dst[c] = s;
    }
    __syncthreads();
  };
  auto src = [&](int c, const void*& p, unsigned& bytes) {
    int bi, lc;
    locate(c, bi, lc);
    const int k = slot_of(bi);
    if (lc == nch) {
      const int kb = bi < nz - 1 ? k + 1 : k;       // coupling of the stencil step
      p = fac + (long long)(nz + kb - 1) * SS;
      bytes = (unsigned)(9 * Q * sizeof(T));
    } else {
      const int r0 = rlo + lc * R, nr = min(R, rhi - r0);
      p = fac + k * SS + (long long)r0 * Q;
      bytes = (unsigned)(nr * Q * sizeof(T));
    }
  };
  auto use = [&](int c, const unsigned char* raw) {
    int bi, lc;
    locate(c, bi, lc);
    const int k = slot_of(bi);
    const bool fwd = bi < nz - 1;
    if (lc < nch) {
      const int r0 = rlo + lc * R, nr = min(R, rhi - r0);
      const T* in = (fwd || bi == nz - 1) ? v + (long long)k * Q : t;
      col_accumulate<T, T, T>(L, reinterpret_cast<const T*>(raw), nr, in + r0, acc);
      return;
    }
    // every row of the slot is consumed before outputs overwrite inputs (with
    // row groups on one CTA, col_finish's barrier after the partials does it)
    if (nrank > 1 || L.G == 1) __syncthreads();
    finish(bi, fwd ? t : v + (long long)k * Q);
    const T* Bd = reinterpret_cast<const T*>(raw);
    if (fwd) {
      // v_{k+1} -= B_{k+1} t
      T* vn = v + (long long)(k + 1) * Q;
      for (int i = threadIdx.x; i < Q; i += blockDim.x) {
        const int ix = i % gx, iy = i / gx;
        T a = T(0);
#pragma unroll
        for (int o = 0; o < 9; ++o) {
          const int dx = o % 3 - 1, dy = o / 3 - 1;
          if (ix + dx >= 0 && ix + dx < gx && iy + dy >= 0 && iy + dy < gy) a += Bd[o * Q + i] * t[i + dx + dy * gx];
        }
        vn[i] -= a;
      }
    } else {
      // t = v_{k-1} - B_k^T v_k
      const T* vk = v + (long long)k * Q;
      const T* vp = v + (long long)(k - 1) * Q;
      for (int l = threadIdx.x; l < Q; l += blockDim.x) {
        const int lx = l % gx, ly = l / gx;
        T a = T(0);
#pragma unroll
        for (int o = 0; o < 9; ++o) {
          const int dx = o % 3 - 1, dy = o / 3 - 1;
          if (lx - dx >= 0 && lx - dx < gx && ly - dy >= 0 && ly - dy < gy) {
            const int i = l - dx - dy * gx;
            a += Bd[o * Q + i] * vk[i];
          }
        }
        t[l] = vp[l] - a;
      }
    }
    // the next slot's accumulation reads what the stencil wrote; warps are
    // not otherwise held together between chunks
    __syncthreads();
  };
  ring_run(ring, nlead * ngs + nch, src, use, err);
  // the last slot (backward, plane 0) has no stencil step after it
  finish(nlead, v);
  if (nrank > 1) cluster.sync();   // the peer's last reads of this CTA's buffers are done
}

// The apply's per-subdomain kernels are persistent over a bucket (see
// ApplyBucket): cluster c of the launch takes the bucket's subdomains c,
// c + clusters, ... in their longest-first order, with one ring for all of
// them (its bookkeeping runs on across subdomains).

// Dirichlet solves of the apply.  mode 0: z_I = A_II^{-1} r_I;
// mode 1: z_I = A_II^{-1} (r_I - t_I).  Writes the interior nodes of z only.
template <typename T>
__global__ void __launch_bounds__(APPLY_THREADS)
k_dirichlet_solve(ApplyBucket B, MeshDev m, const T* __restrict__ fac, const double* __restrict__ r,
                  const double* __restrict__ t, double* __restrict__ z, int mode, int* err) {
  extern __shared__ __align__(128) unsigned char smraw[];
  pdl_enter();
  // clusters of one or two CTAs (the launch decides), one subdomain at a time
  const int csz = (int)cg::this_cluster().num_blocks();
  Ring ring = ring_at(smraw, B.nb);
  T* part = reinterpret_cast<T*>(smraw + ring_bytes(B.nb));
  ring_init(ring);
  for (int si = (int)blockIdx.x / csz; si < B.count; si += (int)gridDim.x / csz) {
    const SubDesc s = B.subs[si];
    const Grid g = grid_of(s, 0);
    if (g.gz == 0) continue;
    const int Q = g.gx * g.gy, n = Q * g.gz;
    T* v = part + APPLY_THREADS;
    T* tq = v + n;
    T* pb = tq + Q;
    __syncthreads();   // the previous subdomain's stores from v are done
    for (int l = threadIdx.x; l < n; l += blockDim.x) {
      int ix = l % g.gx, iy = (l / g.gx) % g.gy, iz = l / Q;
      long long gi = nodeid(m.NX, m.NY, s.e0[0] + 1 + ix, s.e0[1] + 1 + iy, s.e0[2] + 1 + iz);
      double val = r[gi];
      if (mode) val -= t[gi];
      v[l] = (T)val;
    }
    __syncthreads();
    sweep_stream<T>(ring, fac + s.offD, g.gx, g.gy, g.gz, v, tq, part, pb, err);
    if (cg::this_cluster().block_rank() == 0)
      for (int l = threadIdx.x; l < n; l += blockDim.x) {
        int ix = l % g.gx, iy = (l / g.gx) % g.gy, iz = l / Q;
        long long gi = nodeid(m.NX, m.NY, s.e0[0] + 1 + ix, s.e0[1] + 1 + iy, s.e0[2] + 1 + iz);
        z[gi] = (double)v[l];
      }
  }
}

// Weighted restriction r_i = D_i R_i (r - t) on the box surface into rg;
// returns through set_v whether node b also starts the Neumann right-hand
// side (the primal vertices are eliminated and keep zero).
template <typename T, typename F>
__device__ inline void neumann_restrict(const SubDesc& s, const MeshDev& m, const double* __restrict__ delta,
                                        const double* __restrict__ r, const double* __restrict__ t, F&& put) {
  const int px = s.w[0] + 1, py = s.w[1] + 1, pz = s.w[2] + 1;
  for (int b = threadIdx.x; b < s.nB; b += blockDim.x) {
    int ix, iy, iz;
    surf_coords(b, px, py, pz, ix, iy, iz);
    long long gi = nodeid(m.NX, m.NY, s.e0[0] + ix, s.e0[1] + iy, s.e0[2] + iz);
    double d = delta[s.offB + b];
    double val = (d == 0.0) ? 0.0 : d * (r[gi] - t[gi]);
    put(b, ix + px * (iy + py * iz), !neumann_fixed(m, s, ix, iy, iz), (T)val);
  }
}

// The local coarse right-hand side rc_i = Phi_i^T r_i of the weighted
// restriction r_i = D_i R_i (r - t), in the local precision: columns of Phi
// accumulate over streamed rows, the rows split between the CTAs of the
// cluster and their partial sums added in rank order.
template <typename T>
__global__ void __launch_bounds__(APPLY_THREADS)
k_neumann_rhs(ApplyBucket B, MeshDev m, const T* __restrict__ Phi, const double* __restrict__ delta,
              const double* __restrict__ r, const double* __restrict__ t, double* __restrict__ rcl, int* err) {
  extern __shared__ __align__(128) unsigned char smraw[];
  pdl_enter();
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank(), nrank = (int)cluster.num_blocks();
  Ring ring = ring_at(smraw, B.nb);
  T* part = reinterpret_cast<T*>(smraw + ring_bytes(B.nb));
  ring_init(ring);
  for (int si = (int)blockIdx.x / nrank; si < B.count; si += (int)gridDim.x / nrank) {
  const SubDesc s = B.subs[si];
  if (s.nc == 0) continue;   // both CTAs of the cluster see the same subdomain
  T* rg = part + APPLY_THREADS;
  T* pb = rg + s.nB + 1;   // nc partial sums
  __syncthreads();          // the previous subdomain's reads of rg are done
  neumann_restrict<T>(s, m, delta, r, t, [&](int b, int, bool, T val) { rg[b] = val; });
  __syncthreads();
  const int R = rows_per_chunk(s.nc, (int)sizeof(T));
  const int half = split_rows(s.nB, s.nc, (int)sizeof(T), nrank);
  const int rlo = min(s.nB, rank * half), rhi = min(s.nB, rlo + half);
  const int nch = (rhi - rlo + R - 1) / R;
  const T* P = Phi + s.offPhi;
  const ColLayout L = col_layout(s.nc);
  T acc[4] = {T(0), T(0), T(0), T(0)};
  auto src = [&](int c, const void*& p, unsigned& bytes) {
    const int r0 = rlo + c * R, nr = min(R, rhi - r0);
    p = P + (long long)r0 * s.nc;
    bytes = (unsigned)(nr * s.nc * sizeof(T));
  };
  auto use = [&](int c, const unsigned char* raw) {
    const int r0 = rlo + c * R, nr = min(R, rhi - r0);
    col_accumulate<T, T, T>(L, reinterpret_cast<const T*>(raw), nr, rg + r0, acc);
  };
  ring_run(ring, nch, src, use, err);
  if (nrank == 1) {
    col_finish<T>(L, acc, part, [&](int cc, T sum) { rcl[s.cofs + cc] = (double)sum; });
  } else {
    col_finish<T>(L, acc, part, [&](int cc, T sum) { pb[cc] = sum; });
    cluster.sync();
    if (rank == 0)
      for (int c = threadIdx.x; c < s.nc; c += blockDim.x) {
        T sum = T(0);
        for (int q = 0; q < nrank; ++q) sum += cluster.map_shared_rank(pb, q)[c];
        rcl[s.cofs + c] = (double)sum;
      }
    cluster.sync();   // the peer's reads of this CTA's partial sums are done
  }
  }
}

// The constrained Neumann solve y = A_rr^{-1} r_i,r (into vloc) of the
// weighted restriction r_i = D_i R_i (r - t).
template <typename T>
__global__ void __launch_bounds__(APPLY_THREADS)
k_neumann_solve(ApplyBucket B, MeshDev m, const T* __restrict__ fac, const double* __restrict__ delta,
                const double* __restrict__ r, const double* __restrict__ t, T* __restrict__ vloc, int* err) {
  extern __shared__ __align__(128) unsigned char smraw[];
  pdl_enter();
  // clusters of one or two CTAs (the launch decides), one subdomain at a time
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank(), csz = (int)cluster.num_blocks();
  Ring ring = ring_at(smraw, B.nb);
  T* part = reinterpret_cast<T*>(smraw + ring_bytes(B.nb));
  ring_init(ring);
  for (int si = (int)blockIdx.x / csz; si < B.count; si += (int)gridDim.x / csz) {
  const SubDesc s = B.subs[si];
  const int px = s.w[0] + 1, py = s.w[1] + 1, pz = s.w[2] + 1;
  const int Q = px * py, n = Q * pz;
  T* v = part + APPLY_THREADS;
  T* tq = v + n;
  T* pb = tq + Q;   // 2 Q partial sums
  __syncthreads();  // the previous subdomain's stores from v are done
  for (int l = threadIdx.x; l < n; l += blockDim.x) v[l] = T(0);
  __syncthreads();
  neumann_restrict<T>(s, m, delta, r, t, [&](int, int l, bool free_node, T val) {
    if (free_node) v[l] = val;
  });
  __syncthreads();
  sweep_stream<T>(ring, fac + s.offN, px, py, pz, v, tq, part, pb, err);
  if (rank == 0)
    for (int l = threadIdx.x; l < n; l += blockDim.x) vloc[s.offVec + l] = v[l];
  }
}

// v_i on the box surface: Phi_i (u_c|_i - [0; C_r y]) + y, as a column
// accumulation over the rows of Phi_i^T.
template <typename T>
__global__ void __launch_bounds__(APPLY_THREADS)
k_neumann_finish(ApplyBucket B, const LocalCoarse* __restrict__ lc, const int* __restrict__ lcn,
                 const T* __restrict__ PhiT, const T* __restrict__ vloc, const double* __restrict__ uc,
                 double* __restrict__ vgam, int* err) {
  extern __shared__ __align__(128) unsigned char smraw[];
  pdl_enter();
  Ring ring = ring_at(smraw, B.nb);
  T* part = reinterpret_cast<T*>(smraw + ring_bytes(B.nb));
  T* ut = part + APPLY_THREADS;
  ring_init(ring);
  for (int si = (int)blockIdx.x; si < B.count; si += (int)gridDim.x) {
  const SubDesc s = B.subs[si];
  const int px = s.w[0] + 1, py = s.w[1] + 1, pz = s.w[2] + 1;
  const T* y = vloc + s.offVec;
  __syncthreads();   // the previous subdomain's reads of ut are done
  for (int j = threadIdx.x; j < s.nc; j += blockDim.x) {
    const LocalCoarse c = lc[s.cofs + j];
    double val = uc[c.gid];
    if (j >= s.nv) {
      double sum = 0.0;
      for (int q = 0; q < c.count; ++q) sum += (double)y[lcn[c.off + q]];
      val -= sum / c.count;
    }
    ut[j] = (T)val;
  }
  __syncthreads();
  auto out = [&](int b, T sum) {
    int ix, iy, iz;
    surf_coords(b, px, py, pz, ix, iy, iz);
    vgam[s.offB + b] = (double)sum + (double)y[ix + px * (iy + py * iz)];
  };
  const ColLayout L = col_layout(s.nB);
  T acc[4] = {T(0), T(0), T(0), T(0)};
  if (s.nc > 0) {
    const int R = rows_per_chunk(s.nB, (int)sizeof(T));
    const int nch = (s.nc + R - 1) / R;
    const T* P = PhiT + s.offPhi;
    auto src = [&](int c, const void*& p, unsigned& bytes) {
      const int r0 = c * R, nr = min(R, s.nc - r0);
      p = P + (long long)r0 * s.nB;
      bytes = (unsigned)(nr * s.nB * sizeof(T));
    };
    auto use = [&](int c, const unsigned char* raw) {
      const int r0 = c * R, nr = min(R, s.nc - r0);
      col_accumulate<T, T, T>(L, reinterpret_cast<const T*>(raw), nr, ut + r0, acc);
    };
    ring_run(ring, nch, src, use, err);
  }
  col_finish<T>(L, acc, part, out);
  }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
template <typename T>
size_t dense_smem() { return sizeof(DenseSmem<T>); }

// Test hook (host-side fault injection): negates the first diagonal entry of
// one subdomain's assembled local matrix, Neumann or Dirichlet, so that its
// factorisation meets a non-positive pivot.  One thread.
template <typename T>
__global__ void k_debug_negate(const SubDesc* __restrict__ subs, T* __restrict__ fac, int sub, int neumann,
                               T* __restrict__ scratch, int tc) {
  const SubDesc s = subs[sub];
  long long toff = 0;
  if (plane_taps(s, neumann, tc, TCS_MAXQ, &toff)) {
    const Grid g = grid_of(s, neumann);
    T* c = scratch + toff + 4LL * g.gx * g.gy;   // centre tap of node 0, plane 0
    *c = -*c;
    return;
  }
  T* base = fac + (neumann ? s.offN : s.offD);
  base[0] = -base[0];
}

void set_wait_report_tries(long long tries) {
  cudaMemcpyToSymbol(g_wait_report_tries, &tries, sizeof(tries));
}

template <typename T>
void launch_assemble(const LocalLaunch& L, int tc, cudaStream_t st) {
  const int S = L.nsub;
  T* facD = (T*)L.facD; T* facN = (T*)L.facN; T* W = (T*)L.scratch;
  tc = (tc && std::is_same<T, float>::value) ? 1 : 0;   // the tensor-core factorisation reads plane taps
  // local assembly (Dirichlet and Neumann plane blocks)
  if (L.maxQD > 0) {
    k_assemble<T><<<dim3(S, L.maxNzD, 8), BDDC_THREADS, 0, st>>>(L.subs, L.m, L.alpha, facD, 0, L.lc, L.own, L.pen,
                                                                 W, tc);
    BDDC_COUNT(1);
  }
  if (L.npin) {
    k_pin_penalty<<<S, BDDC_THREADS, 0, st>>>(L.subs, L.m, L.alpha, L.lc, L.lcn, L.pen);
    BDDC_COUNT(1);
  }
  k_assemble<T><<<dim3(S, L.maxNzN, 8), BDDC_THREADS, 0, st>>>(L.subs, L.m, L.alpha, facN, 1, L.lc, L.own, L.pen,
                                                               W, tc);
  BDDC_COUNT(1);
  if (L.negate_sub >= 0) {
    k_debug_negate<T><<<1, 1, 0, st>>>(L.subs, L.negate_neumann ? facN : facD, L.negate_sub, L.negate_neumann, W, tc);
    BDDC_COUNT(1);
  }
}

// Both factorisations of every subdomain, per factorisation bucket: bucket
// 0 (FP32, planes of at most TCS_MAXQ nodes) on the tensor cores when tc is
// set, else like bucket 1 with the CUDA-core sweep (y = 0 Neumann, y = 1
// Dirichlet in one launch; the packed Schur matrix takes the shared memory
// left after the pivot columns).
template <typename T>
void launch_factor(const LocalLaunch& L, int tc, cudaStream_t st) {
  T* facD = (T*)L.facD; T* facN = (T*)L.facN; T* W = (T*)L.scratch;
  for (int b = 0; b < 2; ++b) {
    const FactorBucket& B = L.fbucket[b];
    if (B.count == 0) continue;
    if (b == 0 && tc && std::is_same<T, float>::value) {
      launch_schur_tc(L, B, st);   // rank-16 updates on the tensor cores, matrix in TMEM
      continue;
    }
    const int maxQ = std::max(B.maxQN, B.maxQD);
    const size_t smb = 227 * 1024;
    const long long cap = (long long)(smb / sizeof(T)) - 2LL * maxQ - 2;
    k_btschur<T><<<dim3(B.count, B.maxQD > 0 ? 2 : 1), SCHUR_THREADS, smb, st>>>(B.subs, facN, facD, W, cap, L.err);
    BDDC_COUNT(1);
  }
}

template <typename T>
void launch_setup_local(const LocalLaunch& L, cudaStream_t st, cudaEvent_t* ev) {
  const int S = L.nsub;
  T* facN = (T*)L.facN; T* W = (T*)L.scratch;
  size_t sm = dense_smem<T>();
  launch_assemble<T>(L, L.factor_tc, st);
  if (ev) cudaEventRecord(ev[0], st);
  launch_factor<T>(L, L.factor_tc, st);
  if (ev) cudaEventRecord(ev[1], st);
  // coarse basis
  T* Y = (T*)L.Y; T* G = (T*)L.G; T* Lv = (T*)L.Lv; T* PA = (T*)L.PA; T* Sc = (T*)L.Sc; T* Phi = (T*)L.Phi;
  if (L.maxNc > 0) {  // one subdomain has no interface and no coarse space
    k_coarse_rhs<T><<<dim3(S, 64), BDDC_THREADS, 0, st>>>(L.subs, L.m, L.alpha, L.lc, L.own, Y);
    if (std::is_same<T, float>::value && L.tc) {
      k_tc_pack<<<dim3(S, L.maxNzN, tc_kchunks(L.maxQN)), BDDC_THREADS, 0, st>>>(L.subs, (const float*)L.facN,
                                                                               (float*)L.tc);
      const int nch = (L.maxNc + TC_N - 1) / TC_N;
      k_btsolve_multi_tc<<<dim3(nch, S), BDDC_THREADS, 2 * TC_STAGE_BYTES + 9 * 256 * sizeof(float), st>>>(
          L.subs_lpt, (const float*)L.facN, (const float*)L.tc, (float*)L.Y, (float*)L.mscratch, L.mscratch_stride,
          L.err);
      BDDC_COUNT(1);
    } else {
      const int nch = (L.maxNc + CW - 1) / CW;
      k_btsolve_multi<T><<<dim3(nch, S), BDDC_THREADS, sm, st>>>(L.subs_lpt, facN, Y, (T*)L.mscratch,
                                                                   L.mscratch_stride);
    }
    k_constraint_means<T><<<dim3(S, 16), BDDC_THREADS, 0, st>>>(L.subs, L.lc, L.lcn, Y, G);
    k_schur<T><<<S, BDDC_THREADS, sm, st>>>(L.subs, G, Sc, Lv, W, L.err);
    int nrc = (L.maxNN + RB - 1) / RB;
    k_phi_rows<T><<<dim3(S, nrc), BDDC_THREADS, sm, st>>>(L.subs, Y, Lv, Sc, PA, 0);
    k_phi_rows<T><<<dim3(S, nrc), BDDC_THREADS, sm, st>>>(L.subs, Y, Lv, Sc, PA, 1);
    k_phi_surface<T><<<dim3(S, 32), BDDC_THREADS, 0, st>>>(L.subs, L.lc, Y, PA, Phi);
    k_transpose<T><<<dim3(S, 1, 64), 256, 0, st>>>(L.subs, Phi, (T*)L.PhiT);
    k_local_coarse_matrix<T><<<dim3(S, 32), BDDC_THREADS, 0, st>>>(L.subs, L.m, L.alpha, L.lc, Y, Lv, Sc, L.pen,
                                                                     L.Ac);
    BDDC_COUNT(9);
  }
  if (ev) cudaEventRecord(ev[2], st);
}

template <typename T>
void configure_local_kernels() {
  size_t sm = dense_smem<T>();
  cudaFuncSetAttribute(k_btschur<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (std::is_same<T, float>::value) configure_schur_tc();
  cudaFuncSetAttribute(k_btsolve_multi<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaFuncSetAttribute(k_btsolve_multi_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(2 * TC_STAGE_BYTES + 9 * 256 * sizeof(float)));
  cudaFuncSetAttribute(k_schur<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaFuncSetAttribute(k_phi_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaFuncSetAttribute(k_dirichlet_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  cudaFuncSetAttribute(k_neumann_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  cudaFuncSetAttribute(k_neumann_rhs<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  cudaFuncSetAttribute(k_neumann_finish<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

void launch_weights(const LocalLaunch& L, const double* piece_w, cudaStream_t st) {
  BDDC_COUNT(1);
  k_weights<<<dim3(L.nsub, 8), BDDC_THREADS, 0, st>>>(L.subs, L.m, piece_w, L.delta);
}

void launch_mark_coarse(const LocalLaunch& L, unsigned char* vfix, int* own, cudaStream_t st) {
  BDDC_COUNT(1);
  k_mark_coarse<<<L.nsub, BDDC_THREADS, 0, st>>>(L.subs, L.lc, L.lcn, L.m.NX, L.m.NY, vfix, own);
}

void launch_box_pieces(int nx, int ny, int nz, const int* pa, const int* pb, const int* pc, int npx, int npy,
                       int* epiece, cudaStream_t st) {
  const long long ne = (long long)nx * ny * nz;
  BDDC_COUNT(1);
  k_box_pieces<<<(int)std::min<long long>((ne + 255) / 256, 8192), 256, 0, st>>>(nx, ny, nz, pa, pb, pc, npx, npy,
                                                                                 epiece);
}

void launch_piece_alpha_box(const double* alpha, int nx, int ny, const int* plo, const int* phi, int npx, int npy,
                            int npz, double* pw, cudaStream_t st) {
  const long long np = (long long)npx * npy * npz;
  BDDC_COUNT(1);
  k_piece_alpha_box<<<(int)std::min<long long>((np + 255) / 256, 4096), 256, 0, st>>>(alpha, nx, ny, plo, phi, npx,
                                                                                      npy, npz, pw);
}

void launch_piece_alpha(const double* alpha, const long long* pe_off, const int* pe, int np, double* pw,
                        cudaStream_t st) {
  int blocks = std::min((np + 255) / 256, 4096);
  BDDC_COUNT(1);
  k_piece_alpha<<<blocks, 256, 0, st>>>(alpha, pe_off, pe, np, pw);
}

// CTAs of `kern` (APPLY_THREADS threads, smem bytes) resident on the current
// device at once; cached per (device, kernel, smem)
int resident_ctas(const void* kern, size_t smem) {
  static std::mutex mu;
  static std::map<std::tuple<int, const void*, size_t>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto key = std::make_tuple(dev, kern, smem);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, APPLY_THREADS, smem);
  const int n = std::max(1, per_sm) * std::max(1, sms);
  cache[key] = n;
  return n;
}

// per-subdomain apply kernels: persistent clusters of csize CTAs (one or
// two) over one bucket; as many clusters as fit on the GPU at once, at most
// one per subdomain
template <typename... KArgs, typename... Args>
void launch_clustered(void (*kern)(KArgs...), const ApplyBucket& b, int csize, size_t smem, cudaStream_t st,
                      Args... args) {
  const int clusters = std::max(1, std::min(b.count, resident_ctas((const void*)kern, smem) / csize));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(clusters * csize));
  cfg.blockDim = dim3(APPLY_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  // the apply kernels start with pdl_enter(): the launch overlaps the
  // previous kernel's tail
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

size_t apply_smem(const BucketSizes& bs, int nb, int es) {
  const size_t vec = std::max({(size_t)bs.maxNN + 3 * (size_t)bs.maxQN, (size_t)bs.maxND + 3 * (size_t)bs.maxQD,
                               (size_t)bs.maxNB + 1 + bs.maxNc});
  return ring_bytes(nb) + (size_t)es * (APPLY_THREADS + vec + 2);
}

template <typename T>
void launch_dirichlet(const LocalLaunch& L, const double* r, const double* t, double* z, int mode, cudaStream_t st) {
  if (L.maxQD == 0) return;
  for (int b = 0; b < L.nbucket; ++b) {
    if (L.bucket[b].count == 0 || L.bsize[b].maxQD == 0) continue;
    BDDC_COUNT(1);
    const size_t sm = ring_bytes(L.bucket[b].nb) +
                      sizeof(T) * ((size_t)APPLY_THREADS + L.bsize[b].maxND + 3 * (size_t)L.bsize[b].maxQD + 2);
    launch_clustered(k_dirichlet_solve<T>, L.bucket[b], L.bcluster[b], sm, st, L.bucket[b], L.m, (const T*)L.facD, r,
                     t, z, mode, L.err);
  }
}

template <typename T>
void launch_neumann_rhs(const LocalLaunch& L, const double* r, const double* t, cudaStream_t st) {
  if (L.maxNc == 0) return;
  for (int b = 0; b < L.nbucket; ++b) {
    if (L.bucket[b].count == 0) continue;
    const size_t sm = ring_bytes(L.bucket[b].nb) +
                      sizeof(T) * ((size_t)APPLY_THREADS + L.bsize[b].maxNB + 1 + L.bsize[b].maxNc + 2);
    BDDC_COUNT(1);
    launch_clustered(k_neumann_rhs<T>, L.bucket[b], L.bcluster[b], sm, st, L.bucket[b], L.m, (const T*)L.Phi, L.delta,
                     r, t, L.rcl, L.err);
  }
}

template <typename T>
void launch_neumann(const LocalLaunch& L, const double* r, const double* t, cudaStream_t st) {
  for (int b = 0; b < L.nbucket; ++b) {
    if (L.bucket[b].count == 0) continue;
    const size_t sm = ring_bytes(L.bucket[b].nb) +
                      sizeof(T) * ((size_t)APPLY_THREADS + L.bsize[b].maxNN + 3 * (size_t)L.bsize[b].maxQN + 2);
    BDDC_COUNT(1);
    launch_clustered(k_neumann_solve<T>, L.bucket[b], L.bcluster[b], sm, st, L.bucket[b], L.m, (const T*)L.facN,
                     L.delta, r, t, (T*)L.vloc, L.err);
  }
}

template <typename T>
void launch_neumann_finish(const LocalLaunch& L, const double* uc, cudaStream_t st) {
  for (int b = 0; b < L.nbucket; ++b) {
    if (L.bucket[b].count == 0) continue;
    const size_t sm = ring_bytes(L.bucket[b].nb) + sizeof(T) * ((size_t)APPLY_THREADS + L.bsize[b].maxNc + 1);
    BDDC_COUNT(1);
    launch_clustered(k_neumann_finish<T>, L.bucket[b], 1, sm, st, L.bucket[b], L.lc, L.lcn, (const T*)L.PhiT,
                     (const T*)L.vloc, uc, L.vgam, L.err);
  }
}

template void launch_setup_local<float>(const LocalLaunch&, cudaStream_t, cudaEvent_t*);
template void launch_assemble<float>(const LocalLaunch&, int, cudaStream_t);
template void launch_factor<float>(const LocalLaunch&, int, cudaStream_t);
template void launch_setup_local<double>(const LocalLaunch&, cudaStream_t, cudaEvent_t*);
template void configure_local_kernels<float>();
template void configure_local_kernels<double>();
template void launch_dirichlet<float>(const LocalLaunch&, const double*, const double*, double*, int, cudaStream_t);
template void launch_dirichlet<double>(const LocalLaunch&, const double*, const double*, double*, int, cudaStream_t);
template void launch_neumann<float>(const LocalLaunch&, const double*, const double*, cudaStream_t);
template void launch_neumann_rhs<float>(const LocalLaunch&, const double*, const double*, cudaStream_t);
template void launch_neumann_rhs<double>(const LocalLaunch&, const double*, const double*, cudaStream_t);
template void launch_neumann<double>(const LocalLaunch&, const double*, const double*, cudaStream_t);
template void launch_neumann_finish<float>(const LocalLaunch&, const double*, cudaStream_t);
template void launch_neumann_finish<double>(const LocalLaunch&, const double*, cudaStream_t);
template size_t dense_smem<float>();
template size_t dense_smem<double>();

}  // namespace bddc
