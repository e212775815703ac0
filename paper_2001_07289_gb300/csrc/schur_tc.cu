// Batched block-tridiagonal factorisation by inverse Schur complements on the
// fifth-generation tensor cores (FP32 local path, planes of at most 176 nodes).
//
// Same recurrence as k_btschur (local.cu): S_0 = D_0, S_k = D_k - B_k
// S_{k-1}^{-1} B_k^T, slot k <- S_k^{-1}, for the local Dirichlet matrix
// A_II^(i) and the vertex-eliminated Neumann matrix A_rr^(i) of every
// subdomain (Section 3: the V1 = U_I and V2 = W-tilde local problems).
//
// S_k lives in tensor memory as the FP32 accumulator of one or two 128-row
// tiles: row i at lane i % 128 of tile i / 128, column j at TMEM column
// 256 (i / 128) + j.  It is inverted by the symmetric Gauss-Jordan sweep in
// blocks K of 16 pivots.  With D = X_KK, P = X_:K and W = P D^{-1}, one block is
//   X_ij <- X_ij - W_i P_j^T   (i, j outside K),
//   X_iK <- W_i,  X_KK <- -D^{-1},  X_Kj <- W_j^T,
// and -S^{-1} remains after the last block.  The rank-16 part is one
// tcgen05.mma kind::tf32 per tile and K step of 8 (3xTF32: A = -W, B = P, each
// split into hi and lo TF32 parts, three products), issued by one thread and
// accumulated in place in TMEM; then the pivot column block is overwritten
// with W and -D^{-1} (tcgen05.st).  The pivot rows are not rewritten: the
// result is symmetric, and a pivoted row is never read again, because
//   - a later panel X_:K' takes its entries in pivoted rows i from the row
//     block K' instead (X_iK' = X_K'i: column i was set when i was pivoted and
//     has been updated like every other entry since), and
//   - the finished inverse is read from the upper triangle: entry (j, i),
//     j <= i, lies in the column of the later pivot i.
// The 16 x 16 inverse D^{-1} (one warp), the panel product W and the operand
// staging run on the CUDA cores, as does the Schur sandwich that forms S_k:
// T = S_{k-1}^{-1} B_k^T in place in shared memory (row stencils, B_k has nine
// entries per row), then S_k = D_k - B_k T stored into TMEM row by row.
//
// grid (subdomain, problem): y = 0 Neumann, y = 1 Dirichlet (concurrent), one
// CTA of 384 threads per SM (the whole TMEM).  Warp w owns TMEM lanes
// 32 (w % 4) ... + 31; the three warps of a lane quadrant share its column
// work; the last warp also runs the look-ahead of the pivot blocks.
#include "common.cuh"
#include "kernels.h"
#include "stream.cuh"
#include "umma.cuh"

namespace bddc {

namespace {

constexpr int TCS_THREADS = 384;
constexpr int TCS_NGRP = TCS_THREADS / 128;   // warps per TMEM lane quadrant
constexpr int TCS_PS = 20;           // row stride (floats) of the panel and W buffers: 16-byte rows
constexpr int TCS_MAXROWS = 256;     // two 128-row tiles
// shared memory, bytes.  One union region first: T (Q x TS floats plus slack
// for the last row's 16-column reads) while S_k is formed and S_k^{-1} is
// extracted, and the MMA operands during the sweep, when T is dead: A (two
// tiles x hi/lo x 128 rows x 16 TF32) and B (hi/lo x 176 rows x 16).
// Then the panel, W, two D^{-1} (16 x 16, by block parity), the next pivot
// block before the current update, the look-ahead warp's copy of the next
// panel rows, the pivot-row broadcast buffers, barrier and TMEM slot.
constexpr unsigned TCS_BPART = TCS_MAXQ * 64;                  // one B part
constexpr unsigned TCS_B_OFF = 2 * 2 * 8192;                   // after the A parts
constexpr unsigned TCS_U = ((4 * (TCS_MAXQ * 180 + 16) > TCS_B_OFF + 2 * TCS_BPART ? 4 * (TCS_MAXQ * 180 + 16)
                                                                                   : TCS_B_OFF + 2 * TCS_BPART) +
                            1023) & ~1023u;
constexpr unsigned TCS_P = TCS_U, TCS_W = TCS_P + TCS_MAXROWS * TCS_PS * 4, TCS_D = TCS_W + TCS_MAXROWS * TCS_PS * 4,
                   TCS_O = TCS_D + 2 * 16 * 16 * 4, TCS_L = TCS_O + 16 * 16 * 4, TCS_R = TCS_L + 16 * 16 * 4,
                   TCS_BAR = TCS_R + 2 * 16 * 4, TCS_END = TCS_BAR + 16;
constexpr int TCS_LW = TCS_THREADS / 32 - 1;   // the look-ahead warp
constexpr int TCS_WORK = TCS_THREADS - 32;     // threads staging operands

// T's row stride: a multiple of 4 floats (16-byte rows) with an odd number of
// 16-byte units, so that eight rows' float4 loads hit distinct banks
__host__ __device__ inline int tcs_ts(int Q) { return (((Q + 3) / 4) | 1) * 4; }

// x = hi + lo in TF32 parts (hi the TF32 rounding of x, lo that of x - hi):
// 22 significant bits
__device__ inline void split2(float4 x, float4* p) {
  const float xs[4] = {x.x, x.y, x.z, x.w};
  float h[4], l[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    h[c] = umma::to_tf32(xs[c]);
    l[c] = umma::to_tf32(xs[c] - h[c]);
  }
  p[0] = make_float4(h[0], h[1], h[2], h[3]);
  p[1] = make_float4(l[0], l[1], l[2], l[3]);
}

// named barriers: 1 = the staging warps among themselves; 2 = the look-ahead
// warp has copied its inputs (it arrives, the others wait before they
// overwrite the panel and Dold)
__device__ inline void bar_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ inline void bar_arrive(int id, int n) { asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory"); }

}  // namespace

size_t schur_tc_smem(int) { return TCS_END; }

__global__ void __launch_bounds__(TCS_THREADS, 1)
k_btschur_tc(const SubDesc* __restrict__ subs, float* __restrict__ facN, float* __restrict__ facD,
             const float* __restrict__ scratch, int* err) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  const SubDesc s = subs[blockIdx.x];
  const int neumann = blockIdx.y == 0;
  const Grid g = grid_of(s, neumann);
  if (g.gz == 0) return;
  long long toff = 0;
  const bool taps = plane_taps(s, neumann, 1, TCS_MAXQ, &toff);   // D_k as in-plane taps (k_assemble)
  const int Q = g.gx * g.gy, gx = g.gx, gy = g.gy;
  const int Qp = (Q + 15) & ~15, TS = tcs_ts(Q), nmt = (Q + 127) / 128, nch = Qp / 16, nb = Qp / 16;
  const long long SS = slot_stride(Q);
  float* base = neumann ? facN + s.offN : facD + s.offD;
  unsigned char* Aop = smraw;                  // part t of tile m at m * 16384 + t * 8192
  unsigned char* Bop = smraw + TCS_B_OFF;      // part t at t * TCS_BPART
  float* P = reinterpret_cast<float*>(smraw + TCS_P);
  float* W = reinterpret_cast<float*>(smraw + TCS_W);
  float* Dm = reinterpret_cast<float*>(smraw + TCS_D);      // D^{-1} of block kb at Dm + 256 (kb & 1)
  float* Dold = reinterpret_cast<float*>(smraw + TCS_O);    // X_K'K' of the next block before this update
  float* Lp = reinterpret_cast<float*>(smraw + TCS_L);      // the next block's rows of this panel
  float* prow = reinterpret_cast<float*>(smraw + TCS_R);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smraw + TCS_BAR);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smraw + TCS_BAR + 8);
  float* Tm = reinterpret_cast<float*>(smraw);   // the union region
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, q = warp & 3, grp = warp >> 2;
  const int code = neumann ? 3 : 2;
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  if (warp == 0) umma::tmem_alloc(tslot, 512);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t lanes = tmem + ((uint32_t)(32 * q) << 16);   // this warp's lane quadrant
  // the MMA descriptors are the same for every block (fixed operand buffers)
  // [m][ks][0..1] A hi/lo of tile m, [2..3] B hi/lo, at K step ks
  uint64_t dsc[2][2][4] = {};
  const uint32_t idesc = umma::idesc_tf32(128, Qp);
  if (tid == 0) {
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
      for (int ks = 0; ks < 2; ++ks)
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          dsc[m][ks][t] = umma::smem_desc(umma::smem_u32(Aop + m * 16384u + t * 8192u) + ks * 256u, 128, 512);
          dsc[m][ks][2 + t] = umma::smem_desc(umma::smem_u32(Bop + t * TCS_BPART) + ks * 256u, 128, 512);
        }
  }
  unsigned nmma = 0;   // completed MMA groups: parity of the next wait

  // panel rows i >= p (from the column block at p, warps of tile grp)
  auto panel_columns = [&](int p) {
    if (grp < nmt && 128 * grp + 32 * q + 31 >= p && 128 * grp + 32 * q < Q) {
      const int i = 128 * grp + 32 * q + lane;
      float v[16];
      umma::ld16(lanes + 256u * grp + (uint32_t)p, v);
      if (i >= p && i < Q) {
        float4* dst = reinterpret_cast<float4*>(P + i * TCS_PS);
#pragma unroll
        for (int u = 0; u < 4; ++u) dst[u] = make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
      }
    }
  };

  // D^{-1} by one warp: lane r (and r + 16) holds row r of D in a[] (identity
  // rows and columns stand in for pivots past Q, set by the caller); the pivot
  // row reaches every lane through shared memory (two buffers); 16 single-
  // pivot sweeps leave -D^{-1} in a[], stored as D^{-1} to dst (16 x 16)
  auto invert16 = [&](float* a, int pbase, float* dst) {
    const int r = lane & 15;
#pragma unroll
    for (int pv = 0; pv < 16; ++pv) {
      float4* pb = reinterpret_cast<float4*>(prow + (pv & 1) * 16);
      if (lane == pv)
#pragma unroll
        for (int u = 0; u < 4; ++u) pb[u] = make_float4(a[4 * u], a[4 * u + 1], a[4 * u + 2], a[4 * u + 3]);
      __syncwarp();
      float pr[16];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4 t = pb[u];
        pr[4 * u] = t.x; pr[4 * u + 1] = t.y; pr[4 * u + 2] = t.z; pr[4 * u + 3] = t.w;
      }
      float d = pr[pv];
      if (!(d > 0.0f)) {
        if (lane == 0 && pbase + pv < Q) set_error(err, code, s.id);
        d = 1.0f;
      }
      const float rc = __frcp_rn(d);
      const float cr = a[pv] * rc;
#pragma unroll
      for (int c = 0; c < 16; ++c)
        if (c != pv) a[c] = (r == pv) ? pr[c] * rc : fmaf(-cr, pr[c], a[c]);
      a[pv] = (r == pv) ? -rc : cr;
    }
    if (lane < 16) {
      float4* dr = reinterpret_cast<float4*>(dst + r * 16);
#pragma unroll
      for (int u = 0; u < 4; ++u) dr[u] = make_float4(-a[4 * u], -a[4 * u + 1], -a[4 * u + 2], -a[4 * u + 3]);
    }
  };
  // X_{p..p+15, p..p+15} (current TMEM contents) into Dold, by the warp whose
  // lane quadrant holds those rows
  auto read_block = [&](int p) {
    const int mq = p >> 7, qq = (p >> 5) & 3, half = (p >> 4) & 1;
    if (warp == qq) {
      float v[16];
      umma::ld16(lanes + 256u * mq + (uint32_t)p, v);
      if ((lane >> 4) == half)
#pragma unroll
        for (int c = 0; c < 16; ++c) Dold[(lane & 15) * 16 + c] = v[c];
    }
  };

  for (int k = 0; k < g.gz; ++k) {
    float* slot = base + (long long)k * SS;
    const float* Bd = k > 0 ? base + (long long)(g.gz + k - 1) * SS : nullptr;
    if (k > 0) {
      // T = S_{k-1}^{-1} B_k^T in place (Tm holds S_{k-1}^{-1}, both
      // triangles): T[i][j] = sum_o S[i][j + off_o] w_o(j) is a stencil along
      // row i; a warp takes whole rows, lane l the columns l + 32 u
      constexpr int MJ = (TCS_MAXQ + 31) / 32;
      float wj[MJ][9];
      int jc[MJ];
      unsigned okm[MJ];
#pragma unroll
      for (int u = 0; u < MJ; ++u) {
        const int j = lane + 32 * u, jj = min(j, Q - 1), jx = jj % gx, jy = jj / gx;
        jc[u] = jj;
        okm[u] = 0;
#pragma unroll
        for (int o = 0; o < 9; ++o) {
          const int dx = o % 3 - 1, dy = o / 3 - 1;
          const bool ok = j < Q && jx + dx >= 0 && jx + dx < gx && jy + dy >= 0 && jy + dy < gy;
          wj[u][o] = ok ? Bd[o * Q + jj] : 0.0f;
          okm[u] |= ok ? (1u << o) : 0u;
        }
      }
      for (int i = warp; i < Q; i += TCS_THREADS / 32) {
        float* row = Tm + i * TS;
        float acc[MJ];
#pragma unroll
        for (int u = 0; u < MJ; ++u) {
          float a = 0.0f;
#pragma unroll
          for (int o = 0; o < 9; ++o) {
            const int dx = o % 3 - 1, dy = o / 3 - 1;
            const int idx = ((okm[u] >> o) & 1u) ? jc[u] + dx + dy * gx : jc[u];
            a = fmaf(row[idx], wj[u][o], a);
          }
          acc[u] = a;
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < MJ; ++u)
          if (lane + 32 * u < Q) row[lane + 32 * u] = acc[u];
      }
      __syncthreads();
    }
    // S_k = D_k - B_k T into TMEM: work items (tile m, 16-column chunk cc),
    // item it to the warps of each lane quadrant in turn; zero past Q.
    // Lane = row i; the taps T[i + off_o][16 cc ...] are float4 loads.
    for (int it = grp; it < nmt * nch; it += TCS_NGRP) {
      const int m = it / nch, cc = it % nch;
      const int i = 128 * m + 32 * q + lane;
      float v[16];
      if (taps) {
        // the row's nine taps land in columns i - gx - 1 .. i + gx + 1
#pragma unroll
        for (int c = 0; c < 16; ++c) v[c] = 0.0f;
        if (i < Q && 16 * cc <= i + gx + 1 && 16 * cc + 15 >= i - gx - 1) {
          const float* Dt = scratch + toff + 9LL * Q * k;
          const int ix = i % gx, iy = i / gx;
#pragma unroll
          for (int o = 0; o < 9; ++o) {
            const int dx = o % 3 - 1, dy = o / 3 - 1;
            if (ix + dx < 0 || ix + dx >= gx || iy + dy < 0 || iy + dy >= gy) continue;
            const int c0 = i + dx + dy * gx - 16 * cc;
            if (c0 < 0 || c0 >= 16) continue;
            const float dv = Dt[o * Q + i];
#pragma unroll
            for (int c = 0; c < 16; ++c) v[c] = (c == c0) ? dv : v[c];
          }
        }
      } else {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int j = 16 * cc + c;
          v[c] = (i < Q && j < Q) ? slot[(long long)j * Q + i] : 0.0f;   // D_k symmetric: coalesced
        }
      }
      if (k > 0 && i < Q) {
        const int ix = i % gx, iy = i / gx;
#pragma unroll
        for (int o = 0; o < 9; ++o) {
          const int dx = o % 3 - 1, dy = o / 3 - 1;
          if (ix + dx >= 0 && ix + dx < gx && iy + dy >= 0 && iy + dy < gy) {
            const float wv = Bd[o * Q + i];
            const float4* t4 = reinterpret_cast<const float4*>(Tm + (i + dx + dy * gx) * TS + 16 * cc);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float4 t = t4[u];
              v[4 * u] = fmaf(-wv, t.x, v[4 * u]);
              v[4 * u + 1] = fmaf(-wv, t.y, v[4 * u + 1]);
              v[4 * u + 2] = fmaf(-wv, t.z, v[4 * u + 2]);
              v[4 * u + 3] = fmaf(-wv, t.w, v[4 * u + 3]);
            }
          }
        }
#pragma unroll
        for (int c = 0; c < 16; ++c)
          if (16 * cc + c >= Q) v[c] = 0.0f;
      }
      umma::st16(lanes + 256u * m + 16u * cc, v);
    }
    umma::wait_st();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    panel_columns(0);
    if (16 < Q) read_block(16);
    __syncthreads();
    if (warp == TCS_LW) {
      const int r = lane & 15;
      float a[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) a[c] = (r < Q && c < Q) ? P[r * TCS_PS + c] : (r == c ? 1.0f : 0.0f);
      invert16(a, 0, Dm);
    }
    __syncthreads();

    // Block kb: D^{-1} of K is ready in Dm + 256 (kb & 1).  The look-ahead warp
    // forms the next pivot block D' = X_K'K' - W_K' P_K'^T from the values
    // before this update (Dold) and this panel, and inverts it while the other
    // warps stage the operands, run the MMA and fix up the column block.
    for (int kb = 0; kb < nb; ++kb) {
      const int p0 = 16 * kb, p1 = p0 + 16;
      const float* Di = Dm + 256 * (kb & 1);
      const bool ahead = kb + 1 < nb;
      float lo[16];   // look-ahead warp: row r of D' (from Dold), then of -D'^{-1}
      if (warp == TCS_LW) {
        // the look-ahead: copy rows K' of this panel (to Lp) and Dold, let the
        // others go on, then W_K' = (rows K' of P) D^{-1} and D' = Dold -
        // W_K' P_K'^T in the arithmetic (order of terms) of the staging and of
        // (f), and D'^{-1} for block kb + 1; rows and columns past Q identity
        if (ahead) {
          const int r = lane & 15;
          float la[16];
          const float4* pr = reinterpret_cast<const float4*>(P + (p1 + r) * TCS_PS);
          const float4* dr = reinterpret_cast<const float4*>(Dold + r * 16);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float4 t = p1 + r < Q ? pr[u] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            la[4 * u] = t.x; la[4 * u + 1] = t.y; la[4 * u + 2] = t.z; la[4 * u + 3] = t.w;
            const float4 o = dr[u];
            lo[4 * u] = o.x; lo[4 * u + 1] = o.y; lo[4 * u + 2] = o.z; lo[4 * u + 3] = o.w;
          }
#pragma unroll
          for (int c = 0; c < 16; ++c)
            if (!(p1 + r < Q && p1 + c < Q)) lo[c] = (r == c) ? 1.0f : 0.0f;
          if (lane < 16) {
            float4* lr = reinterpret_cast<float4*>(Lp + r * 16);
#pragma unroll
            for (int u = 0; u < 4; ++u) lr[u] = make_float4(la[4 * u], la[4 * u + 1], la[4 * u + 2], la[4 * u + 3]);
          }
          __syncwarp();
          __threadfence_block();   // Lp and the reads of P and Dold are done before the others go on
          bar_arrive(2, TCS_THREADS);
          float w[16];
#pragma unroll
          for (int c = 0; c < 16; ++c) w[c] = 0.0f;
#pragma unroll
          for (int c2 = 0; c2 < 16; ++c2) {
            const float4* d4 = reinterpret_cast<const float4*>(Di + c2 * 16);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float4 dd = d4[u];
              w[4 * u] = fmaf(la[c2], dd.x, w[4 * u]);
              w[4 * u + 1] = fmaf(la[c2], dd.y, w[4 * u + 1]);
              w[4 * u + 2] = fmaf(la[c2], dd.z, w[4 * u + 2]);
              w[4 * u + 3] = fmaf(la[c2], dd.w, w[4 * u + 3]);
            }
          }
          if (p1 + r < Q)
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (p1 + j < Q) {
                const float4* l4 = reinterpret_cast<const float4*>(Lp + j * 16);
                float a = lo[j];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                  const float4 t = l4[u];
                  a = fmaf(-w[4 * u], t.x, a);
                  a = fmaf(-w[4 * u + 1], t.y, a);
                  a = fmaf(-w[4 * u + 2], t.z, a);
                  a = fmaf(-w[4 * u + 3], t.w, a);
                }
                lo[j] = a;
              }
          invert16(lo, p1, Dm + 256 * ((kb + 1) & 1));
        }
      } else {
        // (c) W = P D^{-1} on the rows outside K (zero elsewhere) and the MMA
        // operands A = -W (M x 16) and B = P (Qp x 16), rows of K and past Q
        // zero, as hi and lo TF32 parts in the canonical K-major layout (SBO
        // 512, LBO 128): items (row i, four columns 4 g4), consecutive threads
        // on consecutive rows
        const int R = 128 * nmt;
        for (int e = tid; e < R * 4; e += TCS_WORK) {
          const int i = e % R, g4 = e / R;
          const bool live = i < Q && (i < p0 || i >= p1);
          // B leaves out the next pivot block's columns too: their update is
          // done on the CUDA cores, in the same arithmetic as the look-ahead
          const bool bcol = live && !(ahead && i >= p1 && i < p1 + 16);
          float4 w = make_float4(0.0f, 0.0f, 0.0f, 0.0f), pp = w;
          if (live) {
            const float4* pr = reinterpret_cast<const float4*>(P + i * TCS_PS);
            const float4* d4 = reinterpret_cast<const float4*>(Di) + g4;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float4 pv = pr[u];
              const float pvs[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
              for (int t = 0; t < 4; ++t) {
                const float4 dd = d4[(4 * u + t) * 4];
                w.x = fmaf(pvs[t], dd.x, w.x);
                w.y = fmaf(pvs[t], dd.y, w.y);
                w.z = fmaf(pvs[t], dd.z, w.z);
                w.w = fmaf(pvs[t], dd.w, w.w);
              }
            }
            if (bcol) pp = pr[g4];
          }
          reinterpret_cast<float4*>(W + i * TCS_PS)[g4] = w;
          float4 parts[2];
          split2(make_float4(-w.x, -w.y, -w.z, -w.w), parts);
          const unsigned o = umma::kmajor_offset(i & 127, 4 * g4, 16);
          unsigned char* ab = Aop + (i >> 7) * 16384u;
#pragma unroll
          for (int t = 0; t < 2; ++t) *reinterpret_cast<float4*>(ab + t * 8192u + o) = parts[t];
          if (i < Qp) {
            split2(pp, parts);
            const unsigned ob = umma::kmajor_offset(i, 4 * g4, 16);
#pragma unroll
            for (int t = 0; t < 2; ++t) *reinterpret_cast<float4*>(Bop + t * TCS_BPART + ob) = parts[t];
          }
        }
        fence_proxy_async();
        bar_sync(1, TCS_WORK);
      }
      // (d) X += (-W) P^T on every tile, two K steps of 8, three TF32 products
      if (tid == 0) {
        umma::fence_after_sync();
#pragma unroll
        for (int m = 0; m < 2; ++m)
          if (m < nmt) {
            const uint32_t d = tmem + 256u * m;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
              umma::mma_tf32(d, dsc[m][ks][0], dsc[m][ks][2], idesc, true);   // hi hi
              umma::mma_tf32(d, dsc[m][ks][0], dsc[m][ks][3], idesc, true);   // hi lo
              umma::mma_tf32(d, dsc[m][ks][1], dsc[m][ks][2], idesc, true);   // lo hi
            }
          }
        umma::commit(bar);
      }
      if (warp != TCS_LW) {
        // (e) the update has landed in TMEM (and no longer reads the operands)
        mbar_wait_bounded(bar, nmma & 1u, err);
        umma::fence_after_sync();
        if (ahead) bar_sync(2, TCS_THREADS);   // the look-ahead warp has its inputs
        // (f) pivot column block: W outside K, -D^{-1} inside; at the same
        // time the next block's panel: rows >= p1 from its column block, rows
        // of K from W (X_{p1 + c, i} = W_{p1 + c, i - p0}), rows < p0 from
        // the row block p1 ... p1 + 15 (columns of earlier pivots, untouched
        // by (f)); and the block after next as it stands now (Dold)
        if (grp < nmt && 128 * grp + 32 * q < Q) {
          const int i = 128 * grp + 32 * q + lane;
          float v[16];
          const bool inK = i >= p0 && i < p1;
          const float4* src = reinterpret_cast<const float4*>(inK ? Di + (i - p0) * 16 : W + i * TCS_PS);
          const float sg = inK ? -1.0f : 1.0f;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float4 t = src[u];
            v[4 * u] = sg * t.x; v[4 * u + 1] = sg * t.y; v[4 * u + 2] = sg * t.z; v[4 * u + 3] = sg * t.w;
          }
          umma::st16(lanes + 256u * grp + (uint32_t)p0, v);
        }
        if (ahead) {
          // rows >= p1 of the next panel: X_{i, K'} before this update (the
          // MMA left those columns out) minus W_i P_K'^T, term by term in the
          // order the look-ahead warp uses for D'
          if (grp < nmt && 128 * grp + 32 * q + 31 >= p1 && 128 * grp + 32 * q < Q) {
            const int i = 128 * grp + 32 * q + lane;
            float v[16];
            umma::ld16(lanes + 256u * grp + (uint32_t)p1, v);
            if (i >= p1 && i < Q) {
              float w[16];
              const float4* wr = reinterpret_cast<const float4*>(W + i * TCS_PS);
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const float4 t = wr[u];
                w[4 * u] = t.x; w[4 * u + 1] = t.y; w[4 * u + 2] = t.z; w[4 * u + 3] = t.w;
              }
              float4* dst = reinterpret_cast<float4*>(P + i * TCS_PS);
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                float o4[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                  const int j = 4 * u + t;
                  float a = v[j];
#pragma unroll
                  for (int c = 0; c < 16; ++c) a = fmaf(-w[c], Lp[j * 16 + c], a);
                  o4[t] = a;
                }
                dst[u] = make_float4(o4[0], o4[1], o4[2], o4[3]);
              }
            }
          }
          // (the look-ahead warp belongs to lane quadrant 3 and is busy: that
          // quadrant's chunks go to its other warps)
          const int m1 = p1 >> 7, q1 = (p1 >> 5) & 3, half = (p1 >> 4) & 1;
          const int nq = q1 == (TCS_LW & 3) ? TCS_NGRP - 1 : TCS_NGRP;
          if (q == q1)
            for (int cc = grp; cc < kb; cc += nq) {
              float v[16];
              umma::ld16(lanes + 256u * m1 + 16u * cc, v);
              if ((lane >> 4) == half) {
                const int r = lane & 15;
#pragma unroll
                for (int c = 0; c < 16; ++c) P[(16 * cc + c) * TCS_PS + r] = v[c];
              }
            }
          if (tid < 256) {
            const int r = tid >> 4, c = tid & 15;   // panel row p0 + r, column c
            P[(p0 + r) * TCS_PS + c] = (p1 + c < Q) ? W[(p1 + c) * TCS_PS + r] : 0.0f;
          }
          if (p1 + 16 < Q) read_block(p1 + 16);
        }
        umma::wait_st();
      }
      ++nmma;
      umma::fence_before_sync();
      __syncthreads();
      umma::fence_after_sync();
    }
    // slot k <- S_k^{-1} = -X from the upper triangle, through Tm (both
    // triangles, kept for the next plane's sandwich) for coalesced stores
    for (int it = grp; it < nmt * nch; it += TCS_NGRP) {
      const int m = it / nch, cc = it % nch;
      if (128 * m + 32 * q >= Q) continue;   // the whole warp
      float v[16];
      umma::ld16(lanes + 256u * m + 16u * cc, v);
      const int j = 128 * m + 32 * q + lane;
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int i = 16 * cc + c;
        if (j < Q && i < Q && j <= i) {
          Tm[j * TS + i] = -v[c];
          Tm[i * TS + j] = -v[c];
        }
      }
    }
    __syncthreads();
    for (int e = tid; e < Q * Q; e += TCS_THREADS) slot[e] = Tm[(e / Q) * TS + e % Q];
    __syncthreads();
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tmem, 512);
}

void configure_schur_tc() {
  cudaFuncSetAttribute(k_btschur_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)schur_tc_smem(TCS_MAXQ));
}

void launch_schur_tc(const LocalLaunch& L, const FactorBucket& B, cudaStream_t st) {
  BDDC_COUNT(1);
  k_btschur_tc<<<dim3(B.count, B.maxQD > 0 ? 2 : 1), TCS_THREADS, schur_tc_smem(std::max(B.maxQN, B.maxQD)), st>>>(
      B.subs, (float*)L.facN, (float*)L.facD, (const float*)L.scratch, L.err);
}

}  // namespace bddc
