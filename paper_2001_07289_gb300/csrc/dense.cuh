// CTA-level dense building blocks for the batched local factorisations.
//
// One thread block (BDDC_THREADS = 256 threads) works on matrices that live in
// global memory (L2-resident at these sizes), staging 64 x 16 / 16 x 64 tiles
// through shared memory; each thread owns a 4 x 4 register tile of a 64 x 64
// output tile.  Triangular operands skip the K-range that multiplies known
// zeros.  These routines are called from kernels that give one CTA to one
// subdomain (or one RHS chunk of one subdomain).
#pragma once
#include <type_traits>

#include "common.cuh"

namespace bddc {

constexpr int GBM = 64, GBN = 64, GBK = 16, GPAD = 1;
constexpr int TILE = 32, TLD = 33;

template <typename T>
struct DenseSmem {
  T As[GBK][GBM + GPAD];
  T Bs[GBK][GBN + GPAD];
  T t0[TILE * TLD];
  T t1[TILE * TLD];
  T t2[TILE * TLD];
  T rd[TILE];
  T lv[TILE];
  T r2[TILE];
  int flag;
};

// C(MxN) = alpha * op(A) * op(B) + beta * C  (beta == 0: C is not read).
//   op(A)[i,k] = TA ? A[k*lda+i] : A[i*lda+k]
//   op(B)[k,j] = TB ? B[j*ldb+k] : B[k*ldb+j]
//   triA: 0 none, 1 op(A) lower (zero for k>i), 2 op(A) upper (zero for k<i)
//   triB: 0 none, 1 op(B) upper (zero for k>j), 2 op(B) lower (zero for k<j)
//   lowerC: skip output tiles strictly above the diagonal.
// C must not alias A or B.  Ends with __syncthreads().
template <typename T>
__device__ void cta_gemm(int M, int N, int K, T alpha,
                         const T* __restrict__ A, int lda, bool TA,
                         const T* __restrict__ B, int ldb, bool TB,
                         T beta, T* C, int ldc, int triA, int triB, bool lowerC,
                         DenseSmem<T>& sm) {
  const int tid = threadIdx.x;
  // output mapping: warp w owns the 16x32 sub-block (rows 16*(w>>1), cols
  // 32*(w&1)) of the 64x64 tile; lane (lr, lc) owns its 4x4 cells.  Warps
  // whose sub-block lies outside M x N skip the multiply-adds entirely.
  const int warp = tid >> 5, lane = tid & 31;
  const int orow = 16 * (warp >> 1) + 4 * (lane >> 3), ocol = 32 * (warp & 1) + 4 * (lane & 7);
  const int tilesM = (M + GBM - 1) / GBM, tilesN = (N + GBN - 1) / GBN;
  // element e of a 64x16 (A) or 16x64 (B) slice handled by this thread
  int aii[4], akk[4], bjj[4], bkk[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int e = tid + BDDC_THREADS * r;
    if (TA) { aii[r] = e & 63; akk[r] = e >> 6; } else { aii[r] = e >> 4; akk[r] = e & 15; }
    if (TB) { bjj[r] = e >> 4; bkk[r] = e & 15; } else { bjj[r] = e & 63; bkk[r] = e >> 6; }
  }
  for (int t = 0; t < tilesM * tilesN; ++t) {
    const int i0 = (t / tilesN) * GBM, j0 = (t % tilesN) * GBN;
    if (lowerC && j0 > i0 + GBM - 1) continue;
    int kbeg = 0, kend = K;
    if (triA == 1) kend = min(kend, i0 + GBM);
    if (triA == 2) kbeg = max(kbeg, i0);
    if (triB == 1) kend = min(kend, j0 + GBN);
    if (triB == 2) kbeg = max(kbeg, j0);
    T acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = T(0);
    const bool wactive = (i0 + 16 * (warp >> 1) < M) && (j0 + 32 * (warp & 1) < N) &&
                         !(lowerC && j0 + 32 * (warp & 1) > i0 + 16 * (warp >> 1) + 15);
    // register prefetch of the first K-slice; the next slice's global loads
    // are issued before the current slice is multiplied out of shared memory
    T ra[4], rb[4];
    auto fetch = [&](int k0) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int gi = i0 + aii[r], gk = k0 + akk[r];
        ra[r] = (gi < M && gk < kend) ? (TA ? A[(long long)gk * lda + gi] : A[(long long)gi * lda + gk]) : T(0);
        const int gj = j0 + bjj[r], gk2 = k0 + bkk[r];
        rb[r] = (gj < N && gk2 < kend) ? (TB ? B[(long long)gj * ldb + gk2] : B[(long long)gk2 * ldb + gj]) : T(0);
      }
    };
    if (kbeg < kend) fetch(kbeg);
    for (int k0 = kbeg; k0 < kend; k0 += GBK) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        sm.As[akk[r]][aii[r]] = ra[r];
        sm.Bs[bkk[r]][bjj[r]] = rb[r];
      }
      __syncthreads();
      if (k0 + GBK < kend) fetch(k0 + GBK);
      if (wactive) {
#pragma unroll
        for (int kk = 0; kk < GBK; ++kk) {
          T a[4], b[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) a[r] = sm.As[kk][orow + r];
#pragma unroll
          for (int c = 0; c < 4; ++c) b[c] = sm.Bs[kk][ocol + c];
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int gi = i0 + orow + r;
      if (gi >= M) continue;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        int gj = j0 + ocol + c;
        if (gj >= N) continue;
        T* p = C + (long long)gi * ldc + gj;
        *p = (beta == T(0)) ? alpha * acc[r][c] : alpha * acc[r][c] + beta * (*p);
      }
    }
  }
  __syncthreads();
}

// Thread map of the 32 x 32 tile routines: thread t owns row t / 8 and the
// columns t % 8 + 8q, q = 0..3 (no integer division in the loops); warp w
// holds rows 4w .. 4w + 3, so it skips the column groups past its last row
// and the steps that no longer touch its rows.  FP64 runs at a small fraction
// of the FP32 rate, so the routines keep floating-point instructions to one
// multiply-add per touched entry and per step.

__device__ inline float rsqrt_t(float x) { return rsqrtf(x); }
__device__ inline double rsqrt_t(double x) { return rsqrt(x); }

// Unblocked Cholesky of an n x n (n <= 32) tile in shared memory (ld TLD),
// lower triangle in place, one barrier per column.  Step c updates the
// trailing entries with the unscaled column c: S[i][j] -= (S[i][c] / d_c)
// S[j][c] (d_c the pivot), one product per row and one multiply-add per
// entry; column c - 1 is scaled to L (times 1/sqrt(d)) in step c, when nothing
// reads it, and the diagonal gets sqrt(d) at the end.  The thread that
// finishes S[c+1][c+1] takes its reciprocal square root right away.  A
// non-positive (or NaN) pivot sets sm.flag and is replaced by 1 so that the
// computation stays finite.
template <typename T>
__device__ void tile_chol(T* S, int n, DenseSmem<T>& sm) {
  const int tid = threadIdx.x, i = tid >> 3, cg = tid & 7, wlast = 4 * (tid >> 5) + 3;
  auto pivot = [&](int c, T d) {
    if (!(d > T(0))) { sm.flag = 1; d = T(1); }
    const T rl = rsqrt_t(d);
    sm.lv[c] = d * rl;       // sqrt(d)
    sm.rd[c] = rl;           // 1 / sqrt(d): scales column c
    sm.r2[c] = rl * rl;      // 1 / d: the update's factor
  };
  if (tid == 0 && n > 0) pivot(0, S[0]);
  __syncthreads();
  for (int c = 0; c < n; ++c) {
    if (wlast >= c && i >= c && i < n) {
      const T t = S[i * TLD + c] * sm.r2[c];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (8 * q > wlast) break;
        const int j = cg + 8 * q;
        if (c > 0 && j == c - 1 && i > j) S[i * TLD + j] *= sm.rd[j];   // L column c - 1
        if (j > c && j <= i) {
          const T v = S[i * TLD + j] - t * S[j * TLD + c];
          S[i * TLD + j] = v;
          if (i == c + 1 && j == c + 1) pivot(c + 1, v);
        }
      }
    }
    __syncthreads();
  }
  if (tid < n) S[tid * TLD + tid] = sm.lv[tid];
  __syncthreads();
}

// X = L^{-1} for a lower n x n tile (both ld TLD); zeros above the diagonal.
// rdiag: n entries of scratch for the reciprocal diagonal.  Right-looking
// substitution, every thread of the CTA taking part: row i collects
// -sum_{m<i} L[i][m] X[m][.] over the steps m = 0 .. i-1 and is scaled by
// 1/L[i][i] in its last one (X[i][i] = 1/L[i][i] from the start), so step k
// reads the finished row k and costs one multiply-add per entry.
template <typename T>
__device__ void tile_inv(const T* L, T* X, int n, T* rdiag) {
  const int tid = threadIdx.x, i = tid >> 3, cg = tid & 7, wlast = 4 * (tid >> 5) + 3;
  if (tid < n) rdiag[tid] = T(1) / L[tid * TLD + tid];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j = cg + 8 * q;
    X[i * TLD + j] = (i == j && i < n) ? rdiag[i] : T(0);
  }
  __syncthreads();
  for (int k = 0; k + 1 < n; ++k) {
    if (wlast > k && i > k && i < n) {
      const T lik = L[i * TLD + k];
      const bool last = (i == k + 1);
      const T ri = last ? rdiag[i] : T(1);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (8 * q > k) break;
        const int j = cg + 8 * q;
        if (j <= k) {
          const T v = X[i * TLD + j] - lik * X[k * TLD + j];
          X[i * TLD + j] = last ? v * ri : v;
        }
      }
    }
    __syncthreads();
  }
}

// FP64 Cholesky and inverse of an n x n (n <= 32) tile in registers of
// warps 0-3, one warp per SM sub-partition (FP64 issue costs about the same
// per warp instruction whether one lane or 32 are active, so each FP64
// instruction on the pivot chain counts): lane i holds row i, warp w the
// columns j = w + 4m (m < 8) of the factor (a) and of the inverse (y).
// Columns are published through shared memory with two counters instead of
// a barrier per column: when column k of L is out, the owner of column k + 1
// applies it to that column, takes the pivot (reciprocal square root) and
// publishes column k + 1 at once; only then does it, like the other warps,
// apply column k to its remaining columns and take the inverse's step k:
// Y[i][j] -= (L[i][k] / L[k][k]) Y[k][j] (row k of Y from lane k), with
// X[i][j] = Y[i][j] / L[i][i] at the end.  The chain of pivots thus waits on
// one multiply-add per column, not on the slowest warp's whole step.  The
// operations per entry and their order are those of the plain right-looking
// algorithm.  In: t0 lower triangle of S (ld TLD).  Out: t0 = L (zeros
// above), X (full, zeros above the diagonal).  Uses sm.As (columns of L, ld
// 32), sm.t2 (L[i][k] / L[k][k] by k, ld 32), sm.rd, sm.r2 (the two
// counters).  A non-positive pivot, or a publication wait that runs past its
// bound, sets sm.flag (the pivot is replaced by 1).
__device__ inline void tile_chol_inv_f64(double* t0, double* X, int n, DenseSmem<double>& sm) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* colL = &sm.As[0][0];
  double* colT = sm.t2;
  volatile int* pubL = reinterpret_cast<volatile int*>(sm.r2);
  volatile int* pubT = pubL + 1;
  if (threadIdx.x == 0) { pubL[0] = 0; pubT[0] = 0; }
  __syncthreads();
  if (warp < 4 && n > 0) {
    double a[8], y[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int j = warp + 4 * m;
      a[m] = (lane < n && j < n && j <= lane) ? t0[lane * TLD + j] : 0.0;
      y[m] = (lane == j) ? 1.0 : 0.0;
    }
    // waits (all lanes) until counter p reaches v; bounded
    auto wait_for = [&](volatile int* p, int v) {
      long long tries = 0;
      while (*p < v) {
        if (++tries > (1LL << 24)) {
          sm.flag = 1;
          break;
        }
      }
      __threadfence_block();
    };
    // pivot of column c, held in col by this warp: publishes L's column c,
    // then L[i][c] / L[c][c] and 1 / L[c][c]; returns the L column
    auto pivot = [&](int c, double col) -> double {
      double d = __shfl_sync(0xffffffffu, col, c);
      const long long bits = __double_as_longlong(d);
      if (!(bits > 0 && bits < 0x7ff0000000000000LL)) {   // not a positive finite number
        if (lane == 0) sm.flag = 1;
        d = 1.0;
        col = (lane == c) ? 1.0 : col;
      }
      const double rl = rsqrt(d);
      const double l = (lane >= c) ? col * rl : 0.0;
      colL[c * 32 + lane] = l;
      __threadfence_block();
      __syncwarp();
      if (lane == 0) *pubL = c + 1;
      colT[c * 32 + lane] = (lane > c) ? l * rl : 0.0;
      if (lane == 0) sm.rd[c] = rl;
      __threadfence_block();
      __syncwarp();
      wait_for(pubT, c);   // the counters only grow: column c - 1 first
      if (lane == 0) *pubT = c + 1;
      return l;
    };
    if (warp == 0) a[0] = pivot(0, a[0]);
    for (int k = 0; k < n; ++k) {
      wait_for(pubL, k + 1);
      const double lk = colL[k * 32 + lane];
      const int cn = k + 1;
      const bool owner = cn < n && (cn & 3) == warp;
      if (owner) {
        const int mm = cn >> 2;
        double col = a[0];
#pragma unroll
        for (int m = 1; m < 8; ++m) col = (m == mm) ? a[m] : col;
        col = pivot(cn, fma(-lk, colL[k * 32 + cn], col));
#pragma unroll
        for (int m = 0; m < 8; ++m) a[m] = (m == mm) ? col : a[m];
      }
      // column k on this warp's columns j > k (minus the pivot column just
      // taken), and the inverse's step k on its columns j <= k.  An FP64
      // instruction whose predicate is off still costs its issue slot, so
      // the ranges are entered by a jump (switch with fall-through) instead
      // of predicating all eight.  Columns j >= n hold zeros and stay zero.
      const int m0 = (k >= warp) ? ((k - warp) >> 2) + 1 : 0;   // first column j > k
#define BDDC_FSTEP(m) a[m] = fma(-lk, colL[k * 32 + warp + 4 * (m)], a[m])
      switch (owner ? m0 + 1 : m0) {
        case 0: BDDC_FSTEP(0); [[fallthrough]];
        case 1: BDDC_FSTEP(1); [[fallthrough]];
        case 2: BDDC_FSTEP(2); [[fallthrough]];
        case 3: BDDC_FSTEP(3); [[fallthrough]];
        case 4: BDDC_FSTEP(4); [[fallthrough]];
        case 5: BDDC_FSTEP(5); [[fallthrough]];
        case 6: BDDC_FSTEP(6); [[fallthrough]];
        case 7: BDDC_FSTEP(7); [[fallthrough]];
        default: break;
      }
#undef BDDC_FSTEP
      if (k + 1 < n) {
        wait_for(pubT, k + 1);
        const double lt = colT[k * 32 + lane];   // zero for lane <= k
#define BDDC_ISTEP(m) y[m] = fma(-lt, __shfl_sync(0xffffffffu, y[m], k), y[m])
        switch (m0) {
          case 8: BDDC_ISTEP(7); [[fallthrough]];
          case 7: BDDC_ISTEP(6); [[fallthrough]];
          case 6: BDDC_ISTEP(5); [[fallthrough]];
          case 5: BDDC_ISTEP(4); [[fallthrough]];
          case 4: BDDC_ISTEP(3); [[fallthrough]];
          case 3: BDDC_ISTEP(2); [[fallthrough]];
          case 2: BDDC_ISTEP(1); [[fallthrough]];
          case 1: BDDC_ISTEP(0); [[fallthrough]];
          default: break;
        }
#undef BDDC_ISTEP
      }
    }
    wait_for(pubT, n);
    const double ri = (lane < n) ? sm.rd[lane] : 0.0;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int j = warp + 4 * m;
      t0[lane * TLD + j] = (lane < n && j <= lane) ? a[m] : 0.0;
      X[lane * TLD + j] = y[m] * ri;
    }
  }
  __syncthreads();
}

// Blocked right-looking Cholesky S = L L^T (S n x n SPD, lower part read,
// overwritten by L) followed by the explicit inverse Linv = L^{-1} (written in
// full, zeros above the diagonal).  diag: scratch for ceil(n/32) 32x32 tiles.
// Returns false if a pivot was not positive.
template <typename T>
__device__ bool cta_chol_inv(T* S, int lds, T* Linv, int ldl, int n, T* diag, DenseSmem<T>& sm) {
  const int tid = threadIdx.x;
  if (tid == 0) sm.flag = 0;
  __syncthreads();
  const int nt = (n + TILE - 1) / TILE;
  for (int jb = 0; jb < nt; ++jb) {
    const int j0 = jb * TILE, nb = min(TILE, n - j0);
    for (int idx = tid; idx < TILE * TILE; idx += BDDC_THREADS) {
      int i = idx / TILE, j = idx % TILE;
      sm.t0[i * TLD + j] = (i < nb && j <= i) ? S[(long long)(j0 + i) * lds + j0 + j] : T(0);
    }
    __syncthreads();
    if constexpr (std::is_same<T, double>::value) {
      tile_chol_inv_f64(sm.t0, sm.t1, nb, sm);
    } else {
      tile_chol(sm.t0, nb, sm);
      tile_inv(sm.t0, sm.t1, nb, sm.rd);
    }
    {
      const int i = tid >> 3, cg = tid & 7;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = cg + 8 * q;
        if (i < nb && j < nb) {
          if (j <= i) S[(long long)(j0 + i) * lds + j0 + j] = sm.t0[i * TLD + j];
          diag[jb * TILE * TILE + i * TILE + j] = sm.t1[i * TLD + j];
        }
      }
    }
    // panel below the diagonal tile: P = P * Tinv^T, 32 rows at a time
    // through shared memory, every thread producing 4 outputs
    __syncthreads();
    for (int p0 = j0 + nb; p0 < n; p0 += TILE) {
      const int pr = min(TILE, n - p0);
      for (int idx = tid; idx < TILE * TILE; idx += BDDC_THREADS) {
        int i = idx / TILE, k = idx % TILE;
        sm.t2[i * TLD + k] = (i < pr && k < nb) ? S[(long long)(p0 + i) * lds + j0 + k] : T(0);
      }
      __syncthreads();
      {
        const int i = tid >> 3, cg = tid & 7;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int c = cg + 8 * q;
          if (i < pr && c < nb) {
            T acc = T(0);
            for (int k = 0; k <= c; ++k) acc += sm.t2[i * TLD + k] * sm.t1[c * TLD + k];
            S[(long long)(p0 + i) * lds + j0 + c] = acc;
          }
        }
      }
      __syncthreads();
    }
    const int m = n - j0 - nb;
    if (m > 0) {
      const T* P = S + (long long)(j0 + nb) * lds + j0;
      cta_gemm<T>(m, m, nb, T(-1), P, lds, false, P, lds, true, T(1),
                  S + (long long)(j0 + nb) * lds + j0 + nb, lds, 0, 0, true, sm);
    }
  }
  // Linv, row block by row block: X_ib,<ib = -Tinv_ib (L_ib,<ib X_<ib,<ib)
  for (int ib = 0; ib < nt; ++ib) {
    const int i0 = ib * TILE, nb = min(TILE, n - i0);
    for (int idx = tid; idx < TILE * TILE; idx += BDDC_THREADS) {
      int i = idx / TILE, j = idx % TILE;
      sm.t1[i * TLD + j] = diag[ib * TILE * TILE + i * TILE + j];
    }
    __syncthreads();
    if (ib > 0) {
      cta_gemm<T>(nb, i0, i0, T(1), S + (long long)i0 * lds, lds, false, Linv, ldl, false, T(0),
                  Linv + (long long)i0 * ldl, ldl, 0, 2, false, sm);
      for (int j = tid; j < i0; j += BDDC_THREADS) {
        T w[TILE];
#pragma unroll
        for (int k = 0; k < TILE; ++k) w[k] = (k < nb) ? Linv[(long long)(i0 + k) * ldl + j] : T(0);
#pragma unroll
        for (int r = 0; r < TILE; ++r) {
          if (r >= nb) break;
          T s = T(0);
#pragma unroll
          for (int k = 0; k < TILE; ++k)
            if (k <= r) s += sm.t1[r * TLD + k] * w[k];
          Linv[(long long)(i0 + r) * ldl + j] = -s;
        }
      }
    }
    for (int idx = tid; idx < nb * (n - i0); idx += BDDC_THREADS) {
      int i = idx / (n - i0), j = idx % (n - i0);
      Linv[(long long)(i0 + i) * ldl + i0 + j] = (j < nb) ? sm.t1[i * TLD + j] : T(0);
    }
    __syncthreads();
  }
  return sm.flag == 0;
}

}  // namespace bddc
