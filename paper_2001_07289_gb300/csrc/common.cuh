// Shared definitions of the BDDC-SO CUDA library (device side).
//
// Layouts
//   * global node vectors: FP64, node (i,j,k) at i + NX*(j + NY*k), NX = nx+1.
//   * alpha: FP64 per element, (i,j,k) at i + nx*(j + ny*k).
//   * subdomain i is the element box [e0, e0+w) per axis; its local Neumann
//     grid has p = w+1 nodes per axis, its Dirichlet (interior) grid q = w-1.
//   * local plane-block factors: for a grid of Q = gx*gy nodes per z-plane and
//     gz planes, slot k (k = 0..gz-1) holds S_k^{-1}, the inverse of the k-th
//     Schur complement of the block-tridiagonal matrix (symmetric, full Q x Q,
//     row-major), and slot gz + k - 1 (k = 1..gz-1) the coupling
//     B_k = A_{k,k-1} as nine stencil diagonals (9 x Q).
//   * box-surface ("boundary list") order: all nodes of the local Neumann grid
//     with at least one coordinate at 0 or p-1, in lexicographic order.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define BDDC_THREADS 256

namespace bddc {

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may have its CTAs scheduled while the previous kernel of the
// stream finishes; they wait here for its completion (and its memory) before
// reading anything, then let the next kernel be scheduled in turn.  Without
// that launch attribute both instructions do nothing.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" :::);
}

struct SubDesc {
  int id;             // index of the subdomain (x fastest over the box grid)
  int e0[3];          // element origin of the box
  int w[3];           // box widths in elements
  int nB;             // box-surface nodes
  int nv, na, nc;     // local coarse DOFs: point values, averages, total
  int cofs;           // first entry of this subdomain in the local-coarse table
                      // (also the offset of its nc-vector of local coarse values)
  int color;          // (sx&1) + 2(sy&1) + 4(sz&1): same colour => no shared objects
  int pin;            // 1: floating subdomain without a point value, whose local
                      // Neumann factor carries augmented-Lagrangian terms
  long long offD;     // Dirichlet factor slots (local type)
  long long offN;     // Neumann factor slots (local type)
  long long offW;     // factorisation scratch: 2*QN^2 + 1024*ceil(QN/32) (local type)
  long long offY;     // setup: Y = A_rr^{-1} F, nN x nc (local type)
  long long offG;     // setup: C_r Y, na x nc (local type)
  long long offL;     // setup: Lambda_v, na x nv (local type)
  long long offPA;    // setup: Phi_ra = X S_c^{-1}, nN x na (local type)
  long long offSc;    // setup: S_c^{-1}, na x na (local type)
  long long offAc;    // setup: Phi^T A Phi, nc x nc (FP64)
  long long offPhi;   // Phi on the box surface: nB x nc, row-major (local type)
  long long offB;     // per-surface-node arrays: nB (weights, v_Gamma)
  long long offVec;   // apply: local Neumann vector, nN (local type)
  long long offTC;    // setup: canonical 3xTF32 tiles of the Neumann S_k^{-1} (FP32 path)
};

// Tensor-core tiles of one Neumann plane inverse: per K chunk of 32 columns
// and per 128-row tile a hi and a lo tile of 128 x 32 TF32 values (16 KiB
// each) in the canonical K-major order; floats per (plane, K chunk).
__host__ __device__ inline int tc_mtiles(int Q) { return (Q + 127) / 128; }
__host__ __device__ inline int tc_kchunks(int Q) { return (Q + 31) / 32; }
__host__ __device__ inline long long tc_chunk_floats(int Q) { return (long long)tc_mtiles(Q) * 8192; }

// A coarse DOF as seen from one subdomain: its global number and the list of
// the object's nodes on the local Neumann grid (entries off .. off + count - 1
// of the local-node table, linear index ix + px (iy + py iz), ascending); v is
// the first node's local position (the node itself for a point value).
struct LocalCoarse {
  int gid;
  int off;            // first entry in the local-node table
  int count;          // nodes in the object
  short v[3];
};

// Per-axis tables (global), concatenated for the three axes.
struct AxisTables {
  const int* theta;    // node -> 1 on a Theta cut plane (interior), 0 else
  const int* slab;     // element -> slab index, size n
  const int* slab_lo;  // slab -> first element
  const int* slab_hi;  // slab -> one past last element
  int n;               // elements on this axis
  int nslab;
};

struct MeshDev {
  int nx, ny, nz;
  int NX, NY, NZ;      // nodes per axis
  const unsigned char* vfix;  // per node: 1 for a point-value coarse DOF (eliminated as primal)
  const int* epiece;   // per element: sub-subdomain (piece) number
  double h;
  AxisTables ax[3];
  int nsub[3];
};

// Stride between the plane blocks of a factor (elements): Q*Q padded so that
// every block starts 256-byte aligned and a chunk rounded up to 16 bytes
// stays inside its slot.
__host__ __device__ inline long long slot_stride(int Q) {
  return ((long long)Q * Q + 4 + 63) / 64 * 64;
}

// Padded element count of a dense array that is streamed in 16-byte chunks.
__host__ __device__ inline long long padded(long long n) { return (n + 4 + 63) / 64 * 64; }

__host__ __device__ inline long long nodeid(int NX, int NY, int i, int j, int k) {
  return (long long)i + (long long)NX * ((long long)j + (long long)NY * k);
}

__device__ inline bool on_dirichlet(const MeshDev& m, int i, int j, int k) {
  return i == 0 || j == 0 || k == 0 || i == m.nx || j == m.ny || k == m.nz;
}

// Local grid of subdomain s: the Neumann grid (w+1 nodes per axis) or the
// Dirichlet grid of interior nodes (w-1 per axis, empty if some w < 2).
struct Grid {
  int gx, gy, gz, off;  // local grid sizes; global coordinate = e0 + off + local
};
__device__ inline Grid grid_of(const SubDesc& s, int neumann) {
  Grid g;
  if (neumann) { g.gx = s.w[0] + 1; g.gy = s.w[1] + 1; g.gz = s.w[2] + 1; g.off = 0; }
  else { g.gx = s.w[0] - 1; g.gy = s.w[1] - 1; g.gz = s.w[2] - 1; g.off = 1; }
  if (g.gx <= 0 || g.gy <= 0 || g.gz <= 0) { g.gx = g.gy = g.gz = 0; }
  return g;
}

// In-plane stencil taps of the plane blocks D_k for the tensor-core
// factorisation (FP32 path): nine values per node, tap o = (dx + 1) + 3 (dy + 1)
// of node a at o Q + a, plane k after k 9Q values, in the subdomain's
// factorisation scratch (Neumann part first, then Dirichlet, as the CUDA-core
// sweep lays it out).  Used when the subdomain goes to the tensor-core kernel
// (tc, planes of at most maxq nodes in both problems), its Neumann matrix
// carries no augmented-Lagrangian term (dense in the plane) and the taps fit
// the scratch part; off receives the part's first entry.
__device__ inline bool plane_taps(const SubDesc& s, int neumann, int tc, int maxq, long long* off) {
  const Grid gN = grid_of(s, 1), gD = grid_of(s, 0);
  const long long QN = (long long)gN.gx * gN.gy, QD = (long long)gD.gx * gD.gy;
  const long long partN = 2 * QN * QN + 1024 * ((max((int)QN, s.na) + 31) / 32);
  const long long partD = 2 * QD * QD + 1024 * ((QD + 31) / 32);
  *off = s.offW + (neumann ? 0 : partN);
  const Grid& g = neumann ? gN : gD;
  const long long taps = 9LL * g.gx * g.gy * g.gz;
  return tc && QN <= maxq && QD <= maxq && !(neumann && s.pin) && taps <= (neumann ? partN : partD);
}

// First device-side failure wins: error code and the subdomain (or front) id.
__device__ inline void set_error(int* err, int code, int sub) {
  if (atomicCAS(err, 0, code) == 0) err[1] = sub;
}

// Box-surface list of a px x py x pz grid.
__host__ __device__ inline int surf_count(int px, int py, int pz) {
  int ring = 2 * px + 2 * (py - 2);
  return 2 * px * py + (pz - 2) * ring;
}

__host__ __device__ inline int surf_index(int ix, int iy, int iz, int px, int py, int pz) {
  int P = px * py;
  int ring = 2 * px + 2 * (py - 2);
  if (iz == 0) return iy * px + ix;
  if (iz == pz - 1) return P + (pz - 2) * ring + iy * px + ix;
  int base = P + (iz - 1) * ring;
  if (iy == 0) return base + ix;
  if (iy == py - 1) return base + px + 2 * (py - 2) + ix;
  return base + px + 2 * (iy - 1) + (ix == 0 ? 0 : 1);
}

__host__ __device__ inline void surf_coords(int b, int px, int py, int pz, int& ix, int& iy, int& iz) {
  int P = px * py;
  int ring = 2 * px + 2 * (py - 2);
  if (b < P) { iz = 0; iy = b / px; ix = b % px; return; }
  b -= P;
  if (b < (pz - 2) * ring) {
    iz = 1 + b / ring;
    int r = b % ring;
    if (r < px) { iy = 0; ix = r; return; }
    r -= px;
    if (r < 2 * (py - 2)) { iy = 1 + r / 2; ix = (r & 1) ? px - 1 : 0; return; }
    r -= 2 * (py - 2);
    iy = py - 1; ix = r; return;
  }
  b -= (pz - 2) * ring;
  iz = pz - 1; iy = b / px; ix = b % px;
}

}  // namespace bddc
