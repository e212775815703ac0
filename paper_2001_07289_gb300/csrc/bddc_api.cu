// C ABI of the BDDC-SO library (include/bddc_so.h): host-side metadata of the
// partition and the sub-partition, buffer layout, and the sequencing of the
// device kernels for setup, preconditioner apply, operator, PCG and gradient.
//
// Metadata (Section 3, the remark on local subdivision): on every axis the
// Theta cut planes split the elements into slabs and each slab of width w is
// cut into s = ceil(w/L) pieces at floor(k w / s).  The piece boundaries on an
// axis ("points") and the open intervals between them ("items") make every
// node a tuple of per-axis items; a DOF's set of containing sub-subdomains is
// determined by that tuple, so the (sub)objects are exactly the tuples that
// lie on Gamma (some item is a Theta plane), avoid the Dirichlet boundary and
// hold at least one node.  A vertex is a tuple of three points (a point
// value); edges and faces carry the mean over their nodes.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <string>
#include <tuple>
#include <vector>

#include "bddc_so.h"
#include "common.cuh"
#include "kernels.h"
#include "stream.cuh"

using namespace bddc;

namespace {

struct BddcError : std::runtime_error {
  int code;
  BddcError(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define CK(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      throw BddcError(e_ == cudaErrorMemoryAllocation ? BDDC_ERR_OOM : BDDC_ERR_CUDA,              \
                      std::string(#call) + ": " + cudaGetErrorString(e_));                         \
  } while (0)

thread_local std::string g_setup_error;

// Test hooks set by bddc_debug_inject (process-wide): the subdomain whose
// local matrix the next setups assemble with a negated pivot, and the tries
// after which bounded device waits report a timeout.
struct DebugHooks {
  int negate_sub = -1;
  int negate_neumann = 1;
};
DebugHooks g_debug;
std::mutex g_debug_mu;

// Device blocks of destroyed handles (and the setup scratch of live ones) are
// kept per device and handed to later allocations of the same size class: a
// solver that sets up one problem after another with the same shapes then
// stops paying cudaMalloc and cudaFree in every setup.  Size classes waste at
// most 1/8 above 1 MiB.  The cache holds at most an eighth of the device's
// memory (16 GiB at most); a failed cudaMalloc empties it and retries.
class BlockCache {
 public:
  static size_t round(size_t b) {
    if (b <= (size_t(1) << 20)) return (b + 511) & ~size_t(511);
    size_t p = size_t(1) << 20;
    while (p < b) p <<= 1;
    const size_t step = p >> 3;
    return (b + step - 1) / step * step;
  }
  void* take(int dev, size_t rb) {
    std::lock_guard<std::mutex> lk(mu_);
    auto& m = free_[dev & 15];
    auto it = m.find(rb);
    if (it == m.end()) return nullptr;
    void* p = it->second;
    m.erase(it);
    held_[dev & 15] -= rb;
    return p;
  }
  void put(int dev, void* p, size_t rb) {
    std::lock_guard<std::mutex> lk(mu_);
    if (limit_[dev & 15] == 0) {
      size_t fr = 0, tot = 0;
      cudaMemGetInfo(&fr, &tot);
      limit_[dev & 15] = std::min<size_t>(tot / 8, size_t(16) << 30);
    }
    if (held_[dev & 15] + rb > limit_[dev & 15]) { cudaFree(p); return; }
    free_[dev & 15].emplace(rb, p);
    held_[dev & 15] += rb;
  }
  void release(int dev) {
    std::lock_guard<std::mutex> lk(mu_);
    for (auto& kv : free_[dev & 15]) cudaFree(kv.second);
    free_[dev & 15].clear();
    held_[dev & 15] = 0;
  }

 private:
  std::mutex mu_;
  std::multimap<size_t, void*> free_[16];
  size_t held_[16] = {0};
  size_t limit_[16] = {0};
};

BlockCache& block_cache() {
  static BlockCache* c = new BlockCache();   // never destroyed: handles may outlive static teardown
  return *c;
}

struct AxisHost {
  int n = 0;
  std::vector<int> cuts, pts;
  std::vector<int> item, theta, hat;       // per node
  std::vector<int> slab, piece;            // per element
  std::vector<int> slab_lo, slab_hi, piece_lo, piece_hi;
  std::vector<int> item_lo, item_hi, item_kind;  // kind: 0 interval, 1 piece point, 2 Theta point, 3 boundary

  void build(int n_, const int* c, int nc, int L) {
    n = n_;
    cuts.assign(c, c + nc);
    for (int i = 0; i < nc; ++i)
      if (cuts[i] <= 0 || cuts[i] >= n || (i > 0 && cuts[i] <= cuts[i - 1]))
        throw BddcError(BDDC_ERR_ARG, "cut planes must be strictly increasing inside (0, n)");
    std::vector<int> b;
    b.push_back(0);
    for (int v : cuts) b.push_back(v);
    b.push_back(n);
    slab.assign(n, 0);
    piece.assign(n, 0);
    pts.clear();
    pts.push_back(0);
    int p = 0;
    for (size_t s = 0; s + 1 < b.size(); ++s) {
      int lo = b[s], hi = b[s + 1], w = hi - lo;
      int sN = std::max(1, (w + L - 1) / L);
      slab_lo.push_back(lo);
      slab_hi.push_back(hi);
      std::vector<int> bd;
      bd.push_back(lo);
      for (int k = 1; k < sN; ++k) bd.push_back(lo + (int)(((long long)k * w) / sN));
      bd.push_back(hi);
      for (size_t q = 0; q + 1 < bd.size(); ++q) {
        piece_lo.push_back(bd[q]);
        piece_hi.push_back(bd[q + 1]);
        for (int e = bd[q]; e < bd[q + 1]; ++e) { slab[e] = (int)s; piece[e] = p; }
        ++p;
        pts.push_back(bd[q + 1]);
      }
    }
    // pts now holds every piece boundary once, increasing (0 .. n)
    item.assign(n + 1, 0);
    theta.assign(n + 1, 0);
    hat.assign(n + 1, 0);
    const int np = (int)pts.size();
    item_lo.assign(2 * np - 1, 0);
    item_hi.assign(2 * np - 1, 0);
    item_kind.assign(2 * np - 1, 0);
    for (int j = 0; j < np; ++j) {
      int t = pts[j];
      item[t] = 2 * j;
      hat[t] = 1;
      bool is_cut = std::binary_search(cuts.begin(), cuts.end(), t);
      theta[t] = is_cut ? 1 : 0;
      item_lo[2 * j] = item_hi[2 * j] = t;
      item_kind[2 * j] = (t == 0 || t == n) ? 3 : (is_cut ? 2 : 1);
      if (j + 1 < np) {
        item_lo[2 * j + 1] = t + 1;
        item_hi[2 * j + 1] = pts[j + 1] - 1;
        item_kind[2 * j + 1] = 0;
        for (int u = t + 1; u < pts[j + 1]; ++u) item[u] = 2 * j + 1;
      }
    }
  }
  int nitem() const { return (int)item_kind.size(); }
  bool empty(int it) const { return item_lo[it] > item_hi[it]; }
};

}  // namespace

struct bddc_handle {
  int device = 0;
  bddc_mesh mesh{};
  bddc_options opt{};
  int local_double = 1;
  AxisHost ax[3];
  std::vector<SubDesc> subs;
  std::vector<LocalCoarse> lc;
  int n_coarse = 0, n_vertices = 0, max_nc = 0;
  int n_pinned = 0;               // floating subdomains without a point-value coarse DOF, pinned
  int pin_missing = -1;           // a pinned subdomain without an average in one z-plane
  // sub-subdomains: per-element labels (Theta-hat given) or boxes of size L
  bool labels = false;
  std::vector<int> label_in;            // the caller's labels until renumbered
  std::vector<int> epiece, piece_sub;   // labels: per element dense piece number; per piece: subdomain
  int n_pieces = 0;
  // coarse objects (selected), by coarse id: type (0 vertex, 1 edge, 2 face),
  // cell (3 doubled subdomain coordinates), global nodes (CSR, ascending)
  std::vector<int> okind, ocell;
  std::vector<long long> onoff;
  std::vector<int> onodes;        // node coordinates (x, y, z) per object node
  std::vector<int> lcn;           // local node lists of the coarse DOFs
  long long n_nodes = 0, n_free = 0;
  LocalLaunch L{};
  MeshDev m{};
  // device buffers (pointer, rounded size), returned to the block cache
  std::vector<std::pair<void*, size_t>> allocs;
  size_t bytes = 0, factor_bytes = 0;
  double* alpha = nullptr;       // private copy of alpha
  double* Ac_copy = nullptr;      // dense coarse matrix, kept for small problems (diagnostics)
  CoarseGeom geom;
  MFPlan mf;
  MLPlan ml;                      // second level (options.ml_block > 0)
  int *cptr = nullptr, *color_subs = nullptr;
  int2* cent = nullptr;
  int color_count[8] = {0}, color_off[8] = {0};
  double *rc = nullptr, *uc = nullptr;
  double *uI = nullptr, *t = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
  double *partial = nullptr, *scal = nullptr, *hist_a = nullptr, *hist_b = nullptr;
  int* ctl = nullptr;             // PCG control block {it, continue, converged, breakdown}
  int flexible = 0;               // PCG beta by the flexible (Polak-Ribiere) rule; zp keeps the last z
  double* zp = nullptr;
  int* err = nullptr;
  // PCG loop as one CUDA graph (use_graph): a kernel setting the loop condition,
  // then a while node whose body is one PCG iteration writing into xw
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t cap = nullptr;
  // the coarse solve of the apply runs on aux beside the Neumann sweeps;
  // fork and join order it against the caller's stream
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t setup_ev[7] = {};   // phase boundaries of the setup
  double* xw = nullptr;
  long long graph_body_launches = 0;
  double* pinned = nullptr;
  int hist_cap = 0;
  long long n_surface_total = 0, n_local_nodes_total = 0;  // sizes of vgam and vloc
  float setup_ms = 0.f;
  float phase_ms[6] = {0, 0, 0, 0, 0, 0};
  long long launch_base = 0;
  std::vector<std::pair<void*, size_t>> setup_only;
  std::vector<int> h_cptr, h_clist;   // coarse DOF -> owners (CSR), colour lists
  std::vector<int2> h_cent;
  std::string error;

  void* dalloc(size_t b, bool setup_tmp = false) {
    if (b == 0) b = 16;
    const size_t rb = BlockCache::round(b);
    void* ptr = block_cache().take(device, rb);
    if (!ptr) {
      cudaError_t e = cudaMalloc(&ptr, rb);
      if (e != cudaSuccess) {
        cudaGetLastError();
        block_cache().release(device);
        e = cudaMalloc(&ptr, rb);
      }
      if (e != cudaSuccess) {
        cudaGetLastError();
        throw BddcError(BDDC_ERR_OOM, "cudaMalloc of " + std::to_string(b) + " bytes failed");
      }
    }
    (setup_tmp ? setup_only : allocs).emplace_back(ptr, rb);
    if (!setup_tmp) bytes += b;
    return ptr;
  }
  template <typename T> T* dnew(size_t count, bool setup_tmp = false) {
    return (T*)dalloc(sizeof(T) * count, setup_tmp);
  }
  // callers make sure no queued work still uses the blocks (setup ends with
  // a stream synchronisation; the destructor synchronises the device, as
  // cudaFree would)
  void free_setup_only() {
    for (auto& v : setup_only) block_cache().put(device, v.first, v.second);
    setup_only.clear();
  }
  ~bddc_handle() {
    cudaDeviceSynchronize();
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    if (aux) cudaStreamDestroy(aux);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    for (cudaEvent_t e : setup_ev)
      if (e) cudaEventDestroy(e);
    free_setup_only();
    for (auto& v : allocs) block_cache().put(device, v.first, v.second);
    if (pinned) cudaFreeHost(pinned);
  }
};

namespace {

// Pinned staging for the uploads of a setup: host vectors are copied into
// page-locked blocks and sent with cudaMemcpyAsync, which then returns without
// waiting for the work queued before it (a copy from pageable memory may wait,
// and the setup's host work between launches would then leave the GPU idle).
// One setup at a time holds the pool; setups end with a stream
// synchronisation, after which its blocks are free again.  The blocks live for
// the process.
struct PinnedPool {
  std::mutex mu;
  std::vector<std::pair<char*, size_t>> blocks;
  size_t blk = 0, off = 0;
  void* take(size_t bytes) {
    bytes = (bytes + 63) & ~size_t(63);
    while (blk < blocks.size() && off + bytes > blocks[blk].second) { ++blk; off = 0; }
    if (blk == blocks.size()) {
      const size_t sz = std::max<size_t>(bytes, blocks.empty() ? (size_t(4) << 20) : 2 * blocks.back().second);
      char* p = nullptr;
      if (cudaMallocHost((void**)&p, sz) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
      }
      blocks.emplace_back(p, sz);
      off = 0;
    }
    void* r = blocks[blk].first + off;
    off += bytes;
    return r;
  }
};
PinnedPool& pinned_pool() {
  static PinnedPool* p = new PinnedPool;
  return *p;
}
thread_local PinnedPool* t_stage = nullptr;

// Holds the pool for one setup on the calling thread; on exit waits for the
// stream, so that no copy from the pool is still in flight.
struct StageSession {
  std::unique_lock<std::mutex> lk;
  cudaStream_t st;
  explicit StageSession(cudaStream_t s) : lk(pinned_pool().mu), st(s) {
    pinned_pool().blk = 0;
    pinned_pool().off = 0;
    t_stage = &pinned_pool();
  }
  ~StageSession() {
    t_stage = nullptr;
    cudaStreamSynchronize(st);
  }
};

}  // namespace

void bddc::stage_h2d(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return;
  void* hp = t_stage ? t_stage->take(bytes) : nullptr;
  if (hp) {
    std::memcpy(hp, src, bytes);
    CK(cudaMemcpyAsync(dst, hp, bytes, cudaMemcpyHostToDevice, st));
  } else {
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));
  }
}

namespace {

template <typename T>
T* upload(bddc_handle* h, const std::vector<T>& v, cudaStream_t st) {
  T* d = h->dnew<T>(std::max<size_t>(v.size(), 1));
  stage_h2d(d, v.data(), sizeof(T) * v.size(), st);
  return d;
}

// Sub-subdomain of every element: the box pieces of size L (per-axis piece
// numbers, x fastest) or the given labels, renumbered densely by first
// appearance; and the subdomain of every piece.
void build_pieces(bddc_handle* h) {
  const bddc_mesh& M = h->mesh;
  const long long NE = (long long)M.nx * M.ny * M.nz;
  const AxisHost* ax = h->ax;
  const int nsx = (int)ax[0].slab_lo.size(), nsy = (int)ax[1].slab_lo.size();
  auto sub_of = [&](int i, int j, int k) { return ax[0].slab[i] + nsx * (ax[1].slab[j] + nsy * ax[2].slab[k]); };
  if (!h->labels) {   // the element table is computed on the device (k_box_pieces)
    h->epiece.clear();
    const int npx = (int)ax[0].piece_lo.size(), npy = (int)ax[1].piece_lo.size(), npz = (int)ax[2].piece_lo.size();
    h->n_pieces = npx * npy * npz;
    h->piece_sub.assign(h->n_pieces, 0);
    for (int c = 0; c < npz; ++c)
      for (int b = 0; b < npy; ++b)
        for (int a = 0; a < npx; ++a)
          h->piece_sub[a + npx * (b + npy * c)] = sub_of(ax[0].piece_lo[a], ax[1].piece_lo[b], ax[2].piece_lo[c]);
    return;
  }
  std::map<int, int> dense;
  h->piece_sub.clear();
  h->epiece.assign(NE, 0);
  for (int k = 0; k < M.nz; ++k)
    for (int j = 0; j < M.ny; ++j)
      for (int i = 0; i < M.nx; ++i) {
        const long long e = i + (long long)M.nx * (j + (long long)M.ny * k);
        const int lab = h->label_in[e];
        const int si = sub_of(i, j, k);
        auto it = dense.find(lab);
        if (it == dense.end()) {
          it = dense.emplace(lab, (int)h->piece_sub.size()).first;
          h->piece_sub.push_back(si);
        } else if (h->piece_sub[it->second] != si) {
          throw BddcError(BDDC_ERR_ARG, "sub-subdomain label " + std::to_string(lab) + " spans two subdomains");
        }
        h->epiece[e] = it->second;
      }
  h->n_pieces = (int)h->piece_sub.size();
}

// The selected coarse objects, numbered in a fixed order: item tuples of the
// box pieces (x fastest), or for labels connected components (nodes sharing
// an element) of interface nodes with equal sets of surrounding pieces, in
// the order of their first node.  Type by the number of pieces sharing the
// object (Section 3): 2 face, 3 or 4 edge, more vertex; in box pieces the
// item tuples with 1, 2 or 3 point items.
void build_objects(bddc_handle* h, bool keep_v, bool keep_e, bool keep_f) {
  const bddc_mesh& M = h->mesh;
  const AxisHost* ax = h->ax;
  const int NX = M.nx + 1, NY = M.ny + 1, NZ = M.nz + 1;
  const int nsx = (int)ax[0].slab_lo.size(), nsy = (int)ax[1].slab_lo.size();
  auto keep = [&](int kind) { return kind == 0 ? keep_v : (kind == 1 ? keep_e : keep_f); };
  h->okind.clear();
  h->ocell.clear();
  h->onoff.assign(1, 0);
  h->onodes.clear();
  if (!h->labels) {
    int nit[3];
    for (int d = 0; d < 3; ++d) nit[d] = ax[d].nitem();
    {
      // capacity: objects lie on the cut planes; at most the items of those planes
      long long nodes = 0, items = 0;
      for (int d = 0; d < 3; ++d) {
        const int a1 = (d + 1) % 3, a2 = (d + 2) % 3;
        nodes += (long long)ax[d].cuts.size() * (ax[a1].n + 1) * (ax[a2].n + 1);
        items += (long long)ax[d].cuts.size() * nit[a1] * nit[a2];
      }
      h->onodes.reserve(3 * nodes);
      h->okind.reserve(items);
      h->ocell.reserve(3 * items);
      h->onoff.reserve(items + 1);
    }
    for (int iz = 0; iz < nit[2]; ++iz)
      for (int iy = 0; iy < nit[1]; ++iy)
        for (int ix = 0; ix < nit[0]; ++ix) {
          const int it[3] = {ix, iy, iz};
          bool ok = true, on_gamma = false;
          for (int d = 0; d < 3; ++d) {
            const int k = ax[d].item_kind[it[d]];
            if (k == 3 || ax[d].empty(it[d])) ok = false;
            if (k == 2) on_gamma = true;
          }
          const int pts = !(ix & 1) + !(iy & 1) + !(iz & 1);
          const int kind = pts == 3 ? 0 : (pts == 2 ? 1 : 2);
          if (!ok || !on_gamma || !keep(kind)) continue;
          h->okind.push_back(kind);
          for (int d = 0; d < 3; ++d) {
            const int sl = ax[d].slab[ax[d].item_lo[it[d]]];   // element right of the item's first node
            h->ocell.push_back(ax[d].item_kind[it[d]] == 2 ? 2 * sl : 2 * sl + 1);
          }
          for (int z = ax[2].item_lo[iz]; z <= ax[2].item_hi[iz]; ++z)
            for (int y = ax[1].item_lo[iy]; y <= ax[1].item_hi[iy]; ++y)
              for (int x = ax[0].item_lo[ix]; x <= ax[0].item_hi[ix]; ++x) h->onodes.insert(h->onodes.end(), {x, y, z});
          h->onoff.push_back((long long)h->onodes.size() / 3);
        }
    return;
  }
  // interface nodes (off the Dirichlet boundary, on a cut plane) and the
  // sorted set of pieces of their eight elements
  const long long NN = (long long)NX * NY * NZ;
  std::vector<int> key_of(NN, -1);
  std::map<std::vector<int>, int> keys;
  std::vector<std::vector<int>> key_list;
  for (int z = 1; z < M.nz; ++z)
    for (int y = 1; y < M.ny; ++y)
      for (int x = 1; x < M.nx; ++x) {
        if (!ax[0].theta[x] && !ax[1].theta[y] && !ax[2].theta[z]) continue;
        std::vector<int> k;
        for (int dz = -1; dz <= 0; ++dz)
          for (int dy = -1; dy <= 0; ++dy)
            for (int dx = -1; dx <= 0; ++dx)
              k.push_back(h->epiece[(x + dx) + (long long)M.nx * ((y + dy) + (long long)M.ny * (z + dz))]);
        std::sort(k.begin(), k.end());
        k.erase(std::unique(k.begin(), k.end()), k.end());
        auto it = keys.find(k);
        if (it == keys.end()) {
          it = keys.emplace(k, (int)key_list.size()).first;
          key_list.push_back(k);
        }
        key_of[nodeid(NX, NY, x, y, z)] = it->second;
      }
  std::vector<char> seen(NN, 0);
  std::vector<long long> comp, stack;
  for (long long n0 = 0; n0 < NN; ++n0) {
    if (key_of[n0] < 0 || seen[n0]) continue;
    const int key = key_of[n0];
    comp.clear();
    stack.assign(1, n0);
    seen[n0] = 1;
    while (!stack.empty()) {
      const long long u = stack.back();
      stack.pop_back();
      comp.push_back(u);
      const int ux = (int)(u % NX), uy = (int)((u / NX) % NY), uz = (int)(u / ((long long)NX * NY));
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            const int x = ux + dx, y = uy + dy, z = uz + dz;
            if (x < 0 || y < 0 || z < 0 || x >= NX || y >= NY || z >= NZ) continue;
            const long long v = nodeid(NX, NY, x, y, z);
            if (seen[v] || key_of[v] != key) continue;
            seen[v] = 1;
            stack.push_back(v);
          }
    }
    const std::vector<int>& k = key_list[key];
    const int np = (int)k.size();
    const int kind = np == 2 ? 2 : (np <= 4 ? 1 : 0);
    if (!keep(kind)) continue;
    int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-1, -1, -1};
    for (int p : k) {
      const int si = h->piece_sub[p];
      const int sc[3] = {si % nsx, (si / nsx) % nsy, si / (nsx * nsy)};
      for (int d = 0; d < 3; ++d) { lo[d] = std::min(lo[d], sc[d]); hi[d] = std::max(hi[d], sc[d]); }
    }
    h->okind.push_back(kind);
    for (int d = 0; d < 3; ++d) h->ocell.push_back(lo[d] == hi[d] ? 2 * lo[d] + 1 : 2 * hi[d]);
    std::sort(comp.begin(), comp.end());
    for (long long u : comp)
      h->onodes.insert(h->onodes.end(), {(int)(u % NX), (int)((u / NX) % NY), (int)(u / ((long long)NX * NY))});
    h->onoff.push_back((long long)h->onodes.size() / 3);
  }
}

void build_metadata(bddc_handle* h) {
  int nsub[3];
  for (int d = 0; d < 3; ++d) nsub[d] = (int)h->ax[d].slab_lo.size();
  const int sel = h->opt.selection;
  const bool keep_verts = sel == BDDC_SEL_VEF || sel == BDDC_SEL_VE || sel == BDDC_SEL_VF || sel == BDDC_SEL_V;
  const bool keep_edges = sel == BDDC_SEL_VEF || sel == BDDC_SEL_VE || sel == BDDC_SEL_EF;
  const bool keep_faces = sel == BDDC_SEL_VEF || sel == BDDC_SEL_VF || sel == BDDC_SEL_F || sel == BDDC_SEL_EF;
  build_pieces(h);
  build_objects(h, keep_verts, keep_edges, keep_faces);
  const int nc = (int)h->okind.size();
  // point values: one-node vertex objects, eliminated as primal DOFs
  int nvert = 0;
  for (int g = 0; g < nc; ++g)
    if (h->okind[g] == 0 && h->onoff[g + 1] - h->onoff[g] == 1) ++nvert;
  h->n_coarse = nc;
  h->n_vertices = nvert;
  h->n_pinned = 0;
  h->pin_missing = -1;
  // cells -> objects (CSR, ascending) for the nested dissection
  {
    CoarseGeom& G = h->geom;
    int n3[3];
    for (int d = 0; d < 3; ++d) { G.nsub[d] = nsub[d]; n3[d] = 2 * nsub[d] + 1; }
    const long long ncell = (long long)n3[0] * n3[1] * n3[2];
    G.cell_ptr.assign(ncell + 1, 0);
    auto cid = [&](int g) {
      return h->ocell[3 * g] + (long long)n3[0] * (h->ocell[3 * g + 1] + (long long)n3[1] * h->ocell[3 * g + 2]);
    };
    for (int g = 0; g < nc; ++g) ++G.cell_ptr[cid(g) + 1];
    for (long long c = 0; c < ncell; ++c) G.cell_ptr[c + 1] += G.cell_ptr[c];
    G.cell_obj.assign(nc, 0);
    std::vector<int> fill(G.cell_ptr.begin(), G.cell_ptr.end() - 1);
    for (int g = 0; g < nc; ++g) G.cell_obj[fill[cid(g)]++] = g;
  }
  // objects of every subdomain (ascending coarse id): a cell coordinate
  // 2s + 1 lies in slab s, 2s on the plane of slabs s - 1 and s
  const int S = nsub[0] * nsub[1] * nsub[2];
  std::vector<std::vector<int>> sub_objs(S);
  h->lcn.reserve(2 * h->onodes.size() / 3 + 8 * (size_t)nc);
  h->lc.reserve(2 * (size_t)nc + 8 * (size_t)nc / 4);
  for (int g = 0; g < nc; ++g) {
    int r0[3], r1[3];
    for (int d = 0; d < 3; ++d) {
      const int c = h->ocell[3 * g + d];
      if (c & 1) { r0[d] = r1[d] = (c - 1) / 2; }
      else { r0[d] = c / 2 - 1; r1[d] = c / 2; }
    }
    for (int sz = r0[2]; sz <= r1[2]; ++sz)
      for (int sy = r0[1]; sy <= r1[1]; ++sy)
        for (int sx = r0[0]; sx <= r1[0]; ++sx) sub_objs[sx + nsub[0] * (sy + nsub[1] * sz)].push_back(g);
  }
  h->lcn.clear();
  h->subs.assign(S, SubDesc{});
  h->lc.clear();
  // (coarse id, subdomain, local position) of every local coarse DOF, in
  // subdomain order; a counting sort by coarse id gives the owner lists
  std::vector<int> own_g;
  std::vector<int2> own_e;
  std::vector<LocalCoarse> verts, avgs;
  long long offD = 0, offN = 0, offW = 0, offY = 0, offG = 0, offL = 0, offPA = 0, offSc = 0, offAc = 0, offPhi = 0,
            offB = 0, offVec = 0, offTC = 0;
  LocalLaunch& L = h->L;
  L.maxQD = L.maxNzD = L.maxND = L.maxQN = L.maxNzN = L.maxNN = L.maxNB = L.maxNc = 0;
  for (int sz = 0; sz < nsub[2]; ++sz)
    for (int sy = 0; sy < nsub[1]; ++sy)
      for (int sx = 0; sx < nsub[0]; ++sx) {
        const int si = sx + nsub[0] * (sy + nsub[1] * sz);
        SubDesc& s = h->subs[si];
        s.id = si;
        const int sl[3] = {sx, sy, sz};
        for (int d = 0; d < 3; ++d) {
          s.e0[d] = h->ax[d].slab_lo[sl[d]];
          s.w[d] = h->ax[d].slab_hi[sl[d]] - s.e0[d];
        }
        s.color = (sx & 1) + 2 * (sy & 1) + 4 * (sz & 1);
        const int px = s.w[0] + 1, py = s.w[1] + 1, pz = s.w[2] + 1;
        // local coarse DOFs: point values first, then averages, each by coarse
        // id; node lists on the local Neumann grid
        verts.clear();
        avgs.clear();
        for (int g : sub_objs[si]) {
          LocalCoarse c;
          c.gid = g;
          c.count = (int)(h->onoff[g + 1] - h->onoff[g]);
          c.off = (int)h->lcn.size();
          for (long long q = h->onoff[g]; q < h->onoff[g + 1]; ++q) {
            const int x = h->onodes[3 * q] - s.e0[0], y = h->onodes[3 * q + 1] - s.e0[1],
                      z = h->onodes[3 * q + 2] - s.e0[2];
            if (x < 0 || y < 0 || z < 0 || x > s.w[0] || y > s.w[1] || z > s.w[2])
              throw std::runtime_error("coarse object outside a subdomain that shares it");
            if (q == h->onoff[g]) { c.v[0] = (short)x; c.v[1] = (short)y; c.v[2] = (short)z; }
            h->lcn.push_back(x + px * (y + py * z));
          }
          const bool point = h->okind[g] == 0 && c.count == 1;
          (point ? verts : avgs).push_back(c);
        }
        s.nv = (int)verts.size();
        s.na = (int)avgs.size();
        s.nc = s.nv + s.na;
        s.cofs = (int)h->lc.size();
        for (auto& c : verts) h->lc.push_back(c);
        for (auto& c : avgs) h->lc.push_back(c);
        {
          // floating: no face of the box on the Dirichlet boundary; without a
          // point value its local Neumann matrix has the constants as kernel
          // and gets pinned (augmented-Lagrangian terms, see k_pin_penalty),
          // which needs an average whose nodes lie in one z-plane of the box
          const int nd[3] = {h->mesh.nx, h->mesh.ny, h->mesh.nz};
          bool floating = true;
          for (int d = 0; d < 3; ++d)
            if (s.e0[d] == 0 || s.e0[d] + s.w[d] == nd[d]) floating = false;
          s.pin = (floating && s.nv == 0) ? 1 : 0;
          h->n_pinned += s.pin;
          if (s.pin) {
            bool one = false;
            for (const LocalCoarse& c : avgs) {
              bool same = true;
              for (int q = 1; q < c.count; ++q) same = same && h->lcn[c.off + q] / (px * py) == h->lcn[c.off] / (px * py);
              one = one || same;
            }
            if (!one && h->pin_missing < 0) h->pin_missing = si;   // refused by the setup
          }
        }
        for (int j = 0; j < s.nc; ++j) {
          own_g.push_back(h->lc[s.cofs + j].gid);
          own_e.push_back(make_int2(si, s.cofs + j));
        }
        s.nB = surf_count(px, py, pz);
        const int QN = px * py, NN = QN * pz;
        const int qx = s.w[0] - 1, qy = s.w[1] - 1, qz = s.w[2] - 1;
        const bool hasI = qx > 0 && qy > 0 && qz > 0;
        const int QD = hasI ? qx * qy : 0, nzD = hasI ? qz : 0;
        s.offD = offD; offD += hasI ? (long long)(2 * nzD - 1) * slot_stride(QD) : 0;
        s.offN = offN; offN += (long long)(2 * pz - 1) * slot_stride(QN);
        s.offW = offW;   // Neumann scratch, then Dirichlet scratch (factored concurrently)
        offW += 2LL * QN * QN + 1024LL * ((std::max(QN, s.na) + 31) / 32) + 2LL * QD * QD + 1024LL * ((QD + 31) / 32);
        s.offY = offY; offY += (long long)NN * s.nc;
        s.offG = offG; offG += (long long)s.na * s.nc;
        s.offL = offL; offL += (long long)s.na * s.nv;
        s.offPA = offPA; offPA += (long long)NN * s.na;
        s.offSc = offSc; offSc += (long long)s.na * s.na;
        s.offAc = offAc; offAc += (long long)s.nc * s.nc;
        s.offPhi = offPhi; offPhi += padded((long long)s.nB * s.nc);
        s.offB = offB; offB += s.nB;
        s.offVec = offVec; offVec += NN;
        s.offTC = offTC; offTC += (long long)pz * tc_kchunks(QN) * tc_chunk_floats(QN);
        L.maxQD = std::max(L.maxQD, QD); L.maxNzD = std::max(L.maxNzD, nzD); L.maxND = std::max(L.maxND, QD * nzD);
        L.maxQN = std::max(L.maxQN, QN); L.maxNzN = std::max(L.maxNzN, pz); L.maxNN = std::max(L.maxNN, NN);
        L.maxNB = std::max(L.maxNB, s.nB); L.maxNc = std::max(L.maxNc, s.nc);
        h->max_nc = std::max(h->max_nc, s.nc);
      }
  L.nsub = S;
  // multi-RHS scratch per (subdomain, column chunk): Q x 128 covers both the
  // 64-column CUDA-core chunks and the 128-column tensor-core chunks
  h->L.mscratch_stride = (long long)L.maxQN * 128;
  // coarse owners CSR, owners of a coarse DOF in subdomain order (stable
  // counting sort of the subdomain-ordered list)
  std::vector<int> ptr(nc + 1, 0);
  for (int g : own_g) ++ptr[g + 1];
  for (int g = 0; g < nc; ++g) ptr[g + 1] += ptr[g];
  std::vector<int2> ent(own_e.size());
  {
    std::vector<int> fill(ptr.begin(), ptr.end() - 1);
    for (size_t q = 0; q < own_g.size(); ++q) ent[fill[own_g[q]]++] = own_e[q];
  }
  // colour lists
  std::vector<int> clist;
  for (int c = 0; c < 8; ++c) {
    h->color_off[c] = (int)clist.size();
    for (int si = 0; si < S; ++si)
      if (h->subs[si].color == c) clist.push_back(si);
    h->color_count[c] = (int)clist.size() - h->color_off[c];
  }
  h->h_cptr = std::move(ptr);
  h->h_cent = std::move(ent);
  h->h_clist = std::move(clist);
}

}  // namespace

// ---------------------------------------------------------------------------
// setup
// ---------------------------------------------------------------------------
namespace {

// ring depth of the shallow apply configuration and the shared memory one CTA
// may take so that two fit on an SM (228 KB per SM, 1 KB reserved per CTA)
constexpr int SMALL_RING = 4;
constexpr size_t SMALL_SMEM = 113 * 1024;

bool dbl_local(const bddc_handle* h) { return h->local_double != 0; }

BucketSizes sizes_of(const SubDesc& d) {
  BucketSizes z{};
  const bool hasI = d.w[0] > 1 && d.w[1] > 1 && d.w[2] > 1;
  z.maxQD = hasI ? (d.w[0] - 1) * (d.w[1] - 1) : 0;
  z.maxND = hasI ? z.maxQD * (d.w[2] - 1) : 0;
  z.maxQN = (d.w[0] + 1) * (d.w[1] + 1);
  z.maxNN = z.maxQN * (d.w[2] + 1);
  z.maxNB = d.nB;
  z.maxNc = d.nc;
  return z;
}

void grow(BucketSizes& a, const BucketSizes& b) {
  a.maxQD = std::max(a.maxQD, b.maxQD); a.maxND = std::max(a.maxND, b.maxND);
  a.maxQN = std::max(a.maxQN, b.maxQN); a.maxNN = std::max(a.maxNN, b.maxNN);
  a.maxNB = std::max(a.maxNB, b.maxNB); a.maxNc = std::max(a.maxNc, b.maxNc);
}

struct Layout {
  long long D, N, W, Y, G, L, PA, Sc, Ac, Phi, B, Vec, TC;
};

Layout layout_of(const bddc_handle* h) {
  Layout o{};
  for (const SubDesc& s : h->subs) {
    const int px = s.w[0] + 1, py = s.w[1] + 1, pz = s.w[2] + 1;
    const int QN = px * py, NN = QN * pz;
    const int qx = s.w[0] - 1, qy = s.w[1] - 1, qz = s.w[2] - 1;
    const bool hasI = qx > 0 && qy > 0 && qz > 0;
    const int QD = hasI ? qx * qy : 0;
    o.D = std::max(o.D, s.offD + (hasI ? (long long)(2 * qz - 1) * slot_stride(QD) : 0));
    o.N = std::max(o.N, s.offN + (long long)(2 * pz - 1) * slot_stride(QN));
    o.W = std::max(o.W, s.offW + 2LL * QN * QN + 1024LL * ((std::max(QN, s.na) + 31) / 32) + 2LL * QD * QD +
                            1024LL * ((QD + 31) / 32));
    o.Y = std::max(o.Y, s.offY + (long long)NN * s.nc);
    o.G = std::max(o.G, s.offG + (long long)s.na * s.nc);
    o.L = std::max(o.L, s.offL + (long long)s.na * s.nv);
    o.PA = std::max(o.PA, s.offPA + (long long)NN * s.na);
    o.Sc = std::max(o.Sc, s.offSc + (long long)s.na * s.na);
    o.Ac = std::max(o.Ac, s.offAc + (long long)s.nc * s.nc);
    o.Phi = std::max(o.Phi, s.offPhi + padded((long long)s.nB * s.nc));
    o.B = std::max(o.B, s.offB + s.nB);
    o.Vec = std::max(o.Vec, s.offVec + NN);
    o.TC = std::max(o.TC, s.offTC + (long long)pz * tc_kchunks(QN) * tc_chunk_floats(QN));
  }
  return o;
}

// Autotuner of the local factorisations: for the planes that fit it, the
// tensor-core kernel or the CUDA-core register sweep.  The first setup of a
// shape (subdomains, largest planes, bucket size) in the process assembles
// and factors the local matrices once with each and keeps the faster (the
// tensor cores unless the sweep is at least 3 % faster) for every later
// setup of that shape; the setup itself then assembles and factors again.
struct FactorKey {
  int nsub, qn, qd, n0;
  bool operator<(const FactorKey& o) const {
    return std::tie(nsub, qn, qd, n0) < std::tie(o.nsub, o.qn, o.qd, o.n0);
  }
};
std::mutex g_ftune_mu;
std::map<FactorKey, int> g_ftune;

void tune_factor(bddc_handle* h, cudaStream_t st) {
  LocalLaunch& L = h->L;
  L.factor_tc = 1;
  if (h->local_double || L.fbucket[0].count == 0) return;
  const FactorKey key{L.nsub, L.fbucket[0].maxQN, L.fbucket[0].maxQD, L.fbucket[0].count};
  {
    std::lock_guard<std::mutex> lk(g_ftune_mu);
    auto it = g_ftune.find(key);
    if (it != g_ftune.end()) { L.factor_tc = it->second; return; }
  }
  configure_local_kernels<float>();
  cudaEvent_t e[4];
  for (auto& x : e) CK(cudaEventCreate(&x));
  for (int v = 0; v < 2; ++v) {
    launch_assemble<float>(L, 1 - v, st);
    CK(cudaEventRecord(e[2 * v], st));
    launch_factor<float>(L, 1 - v, st);
    CK(cudaEventRecord(e[2 * v + 1], st));
  }
  CK(cudaEventSynchronize(e[3]));
  float t_tc = 0.f, t_cc = 0.f;
  CK(cudaEventElapsedTime(&t_tc, e[0], e[1]));
  CK(cudaEventElapsedTime(&t_cc, e[2], e[3]));
  for (auto& x : e) cudaEventDestroy(x);
  L.factor_tc = t_cc < 0.97f * t_tc ? 0 : 1;
  std::lock_guard<std::mutex> lk(g_ftune_mu);
  g_ftune[key] = L.factor_tc;
}

void check_err_flags(bddc_handle* h, cudaStream_t st) {
  int e[2] = {0, -1};
  CK(cudaMemcpyAsync(e, h->err, sizeof(e), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (e[0] == 0) return;
  const char* what[] = {"", "alpha must be finite and > 0 (element ", "non-positive pivot in the Dirichlet factor of subdomain ",
                        "non-positive pivot in the Neumann factor of subdomain ",
                        "non-positive pivot in S_c of subdomain ", "non-positive pivot in the coarse factor, front ",
                        "", "a bounded device wait ran past its limit in block "};
  // the flags are cleared once read, so that a later call on the handle
  // reports only its own failures
  const int clear[2] = {0, -1};
  CK(cudaMemcpyAsync(h->err, clear, sizeof(clear), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  const int code = std::min(std::max(e[0], 0), 7);
  std::string msg = std::string(what[code]) + std::to_string(e[1]) + (code == 1 ? ")" : "");
  throw BddcError(code == 1 ? BDDC_ERR_ARG : code == 7 ? BDDC_ERR_TIMEOUT : BDDC_ERR_NOT_SPD, msg);
}

template <typename T>
void setup_local(bddc_handle* h, cudaStream_t st, cudaEvent_t* ev) {
  configure_local_kernels<T>();
  launch_setup_local<T>(h->L, st, ev);
}

void do_setup(bddc_handle* h, const double* alpha_dev, cudaStream_t st) {
  const bddc_mesh& M = h->mesh;
  CK(cudaGetDevice(&h->device));
  h->n_nodes = (long long)(M.nx + 1) * (M.ny + 1) * (M.nz + 1);
  h->n_free = (long long)(M.nx - 1) * (M.ny - 1) * (M.nz - 1);
  build_metadata(h);
  if (h->pin_missing >= 0)
    throw BddcError(BDDC_ERR_UNSUPPORTED, "floating subdomain " + std::to_string(h->pin_missing) +
                                              " has neither a point value nor an average within one z-plane");
  {
    // the apply streams rows of plane blocks and of Phi through the shared-
    // memory ring and keeps one subdomain's vectors in shared memory
    const int es = h->local_double ? 8 : 4;
    const LocalLaunch& L = h->L;
    const size_t ring = (size_t)NBUF * CHB + 16 * NBUF;
    const size_t vec = std::max({(size_t)L.maxNN + 3 * (size_t)L.maxQN, (size_t)L.maxND + 3 * (size_t)L.maxQD,
                                 (size_t)L.maxNB + 1 + L.maxNc});
    const size_t smem = ring + (size_t)es * (APPLY_THREADS + vec + 2);
    bool rows_ok = true;
    for (const SubDesc& s : h->subs) {
      const int QN = (s.w[0] + 1) * (s.w[1] + 1);
      if (rows_per_chunk(QN, es) < 1 || (s.nc > 0 && (rows_per_chunk(s.nc, es) < 1 || rows_per_chunk(s.nB, es) < 1)))
        rows_ok = false;
      if ((size_t)9 * QN * es > (size_t)CHB) rows_ok = false;   // a coupling's diagonals stream as one chunk
    }
    if (!rows_ok || L.maxQN > 2048 || L.maxNB > 2048 || L.maxNc > 2048 || smem > 227 * 1024)
      throw BddcError(BDDC_ERR_UNSUPPORTED, "subdomains too large for the streamed local solves "
                                            "(at most 341 FP64 / 682 FP32 nodes per plane and 1024 coarse DOFs)");
  }
  {
    int lo = 0, hi = 0;
    CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    // the coarse chain is latency-bound: its blocks go first when SMs free up
    CK(cudaStreamCreateWithPriority(&h->aux, cudaStreamNonBlocking, hi));
    CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
  }
  h->launch_base = g_launches;
  // events: 0 start, 1 weights done, 2 Dirichlet, 3 Neumann, 4 basis, 5 assembly, 6 coarse factor
  cudaEvent_t* ev = h->setup_ev;
  for (int k = 0; k < 7; ++k) CK(cudaEventCreate(&ev[k]));
  CK(cudaEventRecord(ev[0], st));
  // flags and alpha
  h->err = h->dnew<int>(2);
  int init[2] = {0, -1};
  stage_h2d(h->err, init, sizeof(init), st);
  const long long NE = (long long)M.nx * M.ny * M.nz;
  h->alpha = h->dnew<double>(NE);
  CK(cudaMemcpyAsync(h->alpha, alpha_dev, sizeof(double) * NE, cudaMemcpyDeviceToDevice, st));
  // alpha's check sets the first error code; it is read with every other
  // device-side failure at the end of setup (nothing below can hang or fault
  // on a bad alpha: every loop is bounded by sizes and every wait by a count)
  launch_check_alpha(h->alpha, NE, h->err, st);
  // axis tables
  MeshDev& m = h->m;
  m.nx = M.nx; m.ny = M.ny; m.nz = M.nz;
  m.NX = M.nx + 1; m.NY = M.ny + 1; m.NZ = M.nz + 1;
  {
    // point-value flags (marked below from the coarse lists) and the piece of
    // every element: the given labels, or the box pieces computed here
    unsigned char* vf = h->dnew<unsigned char>((size_t)h->n_nodes);
    CK(cudaMemsetAsync(vf, 0, (size_t)h->n_nodes, st));
    m.vfix = vf;
    if (h->labels) {
      m.epiece = upload(h, h->epiece, st);
    } else {
      int* ep = h->dnew<int>((size_t)NE);
      const int* pa = upload(h, h->ax[0].piece, st);
      const int* pb = upload(h, h->ax[1].piece, st);
      const int* pc = upload(h, h->ax[2].piece, st);
      launch_box_pieces(M.nx, M.ny, M.nz, pa, pb, pc, (int)h->ax[0].piece_lo.size(), (int)h->ax[1].piece_lo.size(),
                        ep, st);
      m.epiece = ep;
    }
  }
  m.h = M.h;
  for (int d = 0; d < 3; ++d) {
    AxisHost& a = h->ax[d];
    m.ax[d].theta = upload(h, a.theta, st);
    m.ax[d].slab = upload(h, a.slab, st);
    m.ax[d].slab_lo = upload(h, a.slab_lo, st);
    m.ax[d].slab_hi = upload(h, a.slab_hi, st);
    m.ax[d].n = a.n;
    m.ax[d].nslab = (int)a.slab_lo.size();
    m.nsub[d] = (int)a.slab_lo.size();
  }
  const bool dbl = h->local_double;
  const size_t es = dbl ? sizeof(double) : sizeof(float);
  Layout lay = layout_of(h);
  h->n_surface_total = lay.B;
  h->n_local_nodes_total = lay.Vec;
  LocalLaunch& L = h->L;
  L.m = m;
  L.alpha = h->alpha;
  L.subs = upload(h, h->subs, st);
  {
    // longest first: the per-subdomain kernels of uneven partitions take the
    // subdomains in decreasing order of plane work (Q^2 per plane, Neumann
    // grid), so that the large ones do not start last
    std::vector<SubDesc> lpt(h->subs);
    auto work = [](const SubDesc& d) {
      const double q = (double)(d.w[0] + 1) * (d.w[1] + 1);
      return q * q * (d.w[2] + 1);
    };
    std::stable_sort(lpt.begin(), lpt.end(), [&](const SubDesc& a, const SubDesc& b) { return work(a) > work(b); });
    L.subs_lpt = upload(h, lpt, st);
    // size buckets of the apply: a subdomain whose work vectors leave room
    // for two CTAs per SM with a ring of SMALL_RING buffers goes to bucket 1,
    // the rest to bucket 0; both keep the longest-first order, start with
    // the deepest ring and one CTA per subdomain, and are tuned below
    const int es = dbl_local(h) ? 8 : 4;
    std::vector<SubDesc> bk[MAX_BUCKETS];
    BucketSizes bz[MAX_BUCKETS] = {};
    for (const SubDesc& d : lpt) {
      const BucketSizes one = sizes_of(d);
      const int b = apply_smem(one, SMALL_RING, es) <= SMALL_SMEM ? 1 : 0;
      bk[b].push_back(d);
      grow(bz[b], one);
    }
    std::vector<SubDesc> all(bk[0]);
    all.insert(all.end(), bk[1].begin(), bk[1].end());
    const SubDesc* dev = upload(h, all, st);
    // factorisation buckets: planes that fit the tensor-core kernel (FP32
    // path) first, the rest second, both longest first
    std::vector<SubDesc> fb[2];
    FactorBucket fz[2] = {};
    for (const SubDesc& d : lpt) {
      const BucketSizes one = sizes_of(d);
      const int b = (!dbl_local(h) && one.maxQN <= TCS_MAXQ && one.maxQD <= TCS_MAXQ) ? 0 : 1;
      fb[b].push_back(d);
      fz[b].maxQN = std::max(fz[b].maxQN, one.maxQN);
      fz[b].maxQD = std::max(fz[b].maxQD, one.maxQD);
    }
    std::vector<SubDesc> fall(fb[0]);
    fall.insert(fall.end(), fb[1].begin(), fb[1].end());
    const SubDesc* fdev = upload(h, fall, st);
    for (int b = 0; b < 2; ++b) {
      fz[b].subs = fdev + (b ? fb[0].size() : 0);
      fz[b].count = (int)fb[b].size();
      L.fbucket[b] = fz[b];
    }
    L.nbucket = MAX_BUCKETS;
    for (int b = 0; b < MAX_BUCKETS; ++b) {
      L.bucket[b] = ApplyBucket{dev + (b ? bk[0].size() : 0), (int)bk[b].size(), NBUF};
      L.bsize[b] = bz[b];
      L.bcluster[b] = 1;
    }
  }
  {
    std::lock_guard<std::mutex> lk(g_debug_mu);
    L.negate_sub = -1;
    if (g_debug.negate_sub >= 0 && g_debug.negate_sub < (int)h->subs.size()) {
      const SubDesc& s = h->subs[g_debug.negate_sub];
      const bool hasI = s.w[0] > 1 && s.w[1] > 1 && s.w[2] > 1;
      if (g_debug.negate_neumann || hasI) {
        L.negate_sub = g_debug.negate_sub;
        L.negate_neumann = g_debug.negate_neumann;
      }
    }
  }
  L.lc = upload(h, h->lc, st);
  L.lcn = upload(h, h->lcn, st);
  {
    int* own = h->dnew<int>((size_t)std::max(h->n_local_nodes_total, 1LL));
    CK(cudaMemsetAsync(own, 0xFF, sizeof(int) * (size_t)std::max(h->n_local_nodes_total, 1LL), st));
    L.own = own;
    launch_mark_coarse(L, const_cast<unsigned char*>(m.vfix), own, st);
  }
  L.facD = h->dalloc(es * lay.D);
  L.facN = h->dalloc(es * lay.N);
  L.Phi = h->dalloc(es * lay.Phi);
  L.PhiT = h->dalloc(es * lay.Phi);
  h->factor_bytes = es * (lay.D + lay.N + 2 * lay.Phi);   // inverse Schur slots, Phi and Phi^T
  L.delta = h->dnew<double>(lay.B);
  L.vgam = h->dnew<double>(lay.B);
  L.vloc = h->dalloc(es * lay.Vec);
  L.rcl = h->dnew<double>(h->lc.size());
  L.npin = h->n_pinned;
  if (L.npin) {
    L.pen = h->dnew<double>(std::max<size_t>(h->lc.size(), 1));
  }
  L.err = h->err;
  L.scratch = h->dalloc(es * lay.W, true);
  L.Y = h->dalloc(es * lay.Y, true);
  L.G = h->dalloc(es * lay.G, true);
  L.Lv = h->dalloc(es * lay.L, true);
  L.PA = h->dalloc(es * lay.PA, true);
  L.Sc = h->dalloc(es * lay.Sc, true);
  // the local coarse matrices stay for the apply of the multilevel coarse level
  L.Ac = (double*)h->dalloc(sizeof(double) * lay.Ac, h->opt.ml_block <= 0);
  const int nch = (L.maxNc + CW - 1) / CW;
  L.mscratch = h->dalloc(es * (size_t)L.nsub * nch * L.mscratch_stride, true);
  // packed tensor-core tiles of the Neumann factors (FP32 path, planes of at
  // most 256 nodes), setup only
  L.tc = (!dbl && L.maxQN <= 256) ? h->dalloc(sizeof(float) * (size_t)std::max(lay.TC, 1LL), true) : nullptr;
  // weights (eq. W or Remark 1)
  double* pw = nullptr;
  if (h->opt.weights == BDDC_W_RHO && !h->labels) {
    std::vector<int> plo, phi;
    int npc[3];
    for (int d = 0; d < 3; ++d) {
      npc[d] = (int)h->ax[d].piece_lo.size();
      plo.insert(plo.end(), h->ax[d].piece_lo.begin(), h->ax[d].piece_lo.end());
      phi.insert(phi.end(), h->ax[d].piece_hi.begin(), h->ax[d].piece_hi.end());
    }
    pw = (double*)h->dalloc(sizeof(double) * (size_t)h->n_pieces, true);
    launch_piece_alpha_box(h->alpha, M.nx, M.ny, upload(h, plo, st), upload(h, phi, st), npc[0], npc[1], npc[2], pw,
                           st);
  } else if (h->opt.weights == BDDC_W_RHO) {
    // elements of every piece, ascending (counting sort of the element labels)
    const int np = h->n_pieces;
    std::vector<long long> pe_off(np + 1, 0);
    for (int p : h->epiece) ++pe_off[p + 1];
    for (int p = 0; p < np; ++p) pe_off[p + 1] += pe_off[p];
    std::vector<int> pe(h->epiece.size());
    {
      std::vector<long long> fill(pe_off.begin(), pe_off.end() - 1);
      for (size_t e = 0; e < h->epiece.size(); ++e) pe[fill[h->epiece[e]]++] = (int)e;
    }
    const long long* dpo = upload(h, pe_off, st);
    const int* dpe = upload(h, pe, st);
    pw = (double*)h->dalloc(sizeof(double) * (size_t)np, true);
    launch_piece_alpha(h->alpha, dpo, dpe, np, pw, st);
  }
  launch_weights(L, pw, st);
  tune_factor(h, st);
  CK(cudaEventRecord(ev[1], st));
  // local factorisations and coarse basis
  if (dbl) setup_local<double>(h, st, ev + 2); else setup_local<float>(h, st, ev + 2);
  CK(cudaGetLastError());
  // coarse problem (FP64)
  const int nc = h->n_coarse;
  h->cptr = upload(h, h->h_cptr, st);
  h->cent = upload(h, h->h_cent, st);
  h->color_subs = upload(h, h->h_clist, st);
  if ((long long)nc * nc <= (1LL << 22)) {   // dense copy for bddc_get_coarse_matrix
    h->Ac_copy = h->dnew<double>((size_t)nc * nc);
    CK(cudaMemsetAsync(h->Ac_copy, 0, sizeof(double) * (size_t)nc * nc, st));
    launch_coarse_assemble(L, h->color_subs, h->color_count, h->color_off, h->Ac_copy, nc, st);
  }
  if (h->opt.ml_block > 0) {
    // multilevel: the coarse problem gets BDDC on blocks of subdomains
    const int nsub3[3] = {(int)h->ax[0].slab_lo.size(), (int)h->ax[1].slab_lo.size(), (int)h->ax[2].slab_lo.size()};
    ml_plan(h->ml, h->opt.ml_block, h->opt.ml_sub, nsub3, h->subs, h->lc, nc, h->h_cptr, h->h_cent);
    CK(cudaEventRecord(ev[5], st));
    ml_setup(h->ml, L, [h](size_t b) { return h->dalloc(b); }, [h](size_t b) { return h->dalloc(b, true); },
             h->opt.weights == BDDC_W_RHO, h->err, st);
    h->factor_bytes += 2 * sizeof(double) * (size_t)(h->ml.N.spool + h->ml.D.spool + h->ml.C.spool);
    CK(cudaEventRecord(ev[6], st));
  } else {
    mf_plan(h->mf, h->geom, nc);
    mf_upload(h->mf, [h](size_t b) { return h->dalloc(b); }, [h](size_t b) { return h->dalloc(b, true); }, st);
    h->factor_bytes += 2 * sizeof(double) * (size_t)h->mf.spool;   // solve matrices and their transposes
    configure_mf_kernels();
    mf_assemble(h->mf, L, h->color_subs, h->color_count, h->color_off, st);
    CK(cudaEventRecord(ev[5], st));
    mf_factor(h->mf, h->err, st, h->aux, h->ev_fork, h->ev_join);
    CK(cudaEventRecord(ev[6], st));
  }
  CK(cudaGetLastError());
  // apply / PCG work vectors
  const long long N = h->n_nodes;
  h->rc = h->dnew<double>(std::max(nc, 1));
  h->uc = h->dnew<double>(std::max(nc, 1));
  h->uI = h->dnew<double>(N);
  CK(cudaMemsetAsync(h->uI, 0, sizeof(double) * N, st));
  h->t = h->dnew<double>(N);
  h->r = h->dnew<double>(N);
  h->z = h->dnew<double>(N);
  h->p = h->dnew<double>(N);
  h->q = h->dnew<double>(N);
  h->partial = h->dnew<double>(2 * RED_BLOCKS);
  h->flexible = h->opt.beta_rule == BDDC_BETA_FLEXIBLE;
  if (h->flexible) h->zp = h->dnew<double>(N);
  h->scal = h->dnew<double>(8);
  h->ctl = h->dnew<int>(4);
  h->hist_cap = h->opt.maxit > 0 ? h->opt.maxit : 2000;
  h->hist_a = h->dnew<double>(h->hist_cap);
  h->hist_b = h->dnew<double>(h->hist_cap);
  CK(cudaMallocHost((void**)&h->pinned, 64));
}

// The end of a setup: waits for the queued work, reads the device-side error
// flags and the phase times, returns the setup-only blocks to the cache.
void finish_setup(bddc_handle* h, cudaStream_t st) {
  cudaEvent_t* ev = h->setup_ev;
  check_err_flags(h, st);
  CK(cudaEventElapsedTime(&h->setup_ms, ev[0], ev[6]));
  for (int k = 0; k < 6; ++k) CK(cudaEventElapsedTime(&h->phase_ms[k], ev[k], ev[k + 1]));
  h->free_setup_only();
}

}  // namespace

// ---------------------------------------------------------------------------
// apply, operator, PCG
// ---------------------------------------------------------------------------
namespace {

// The coarse correction and the local Neumann corrections are solved in
// a-orthogonal spaces (Definition 1: each v_k from its own V_k), so once r_c
// is formed the coarse solve runs on the auxiliary stream while the Neumann
// sweeps run on st; v_i needs both.
template <typename T>
void apply_core(bddc_handle* h, const LocalLaunch& L, const double* r, double* z, double* uI, double* t, double* rc,
                double* uc, double* wf, cudaStream_t st) {
  launch_dirichlet<T>(L, r, nullptr, uI, 0, st);                       // V1: u_I = A_II^{-1} r_I
  launch_operator(h->m, h->alpha, uI, t, nullptr, RED_BLOCKS, st);      // A u_I
  launch_neumann_rhs<T>(L, r, t, st);                                  // r_i, Phi_i^T r_i
  CK(cudaEventRecord(h->ev_fork, st));
  CK(cudaStreamWaitEvent(h->aux, h->ev_fork, 0));
  launch_coarse_gather(h->cptr, h->cent, L.rcl, rc, h->n_coarse, h->aux);
  if (h->opt.ml_block > 0)
    ml_apply(h->ml, L, h->cptr, h->cent, rc, uc, h->aux);                // u_c = M2 r_c (coarse-level BDDC)
  else
    mf_solve(h->mf, rc, uc, wf, h->aux);                               // A_c u_c = r_c
  CK(cudaEventRecord(h->ev_join, h->aux));
  launch_neumann<T>(L, r, t, st);                                      // y = A_rr^{-1} r_i,r
  CK(cudaStreamWaitEvent(st, h->ev_join, 0));
  launch_neumann_finish<T>(L, uc, st);                                 // v_i on the surface
  launch_interface_gather(h->m, L.subs, L.delta, L.vgam, z, st);       // E v
  launch_operator(h->m, h->alpha, z, t, nullptr, RED_BLOCKS, st);      // A (E v)
  launch_dirichlet<T>(L, r, t, z, 1, st);                              // (I - P) E v + u_I
}

template <typename T>
void apply_impl(bddc_handle* h, const double* r, double* z, cudaStream_t st) {
  apply_core<T>(h, h->L, r, z, h->uI, h->t, h->rc, h->uc, h->mf.W, st);
}

void apply(bddc_handle* h, const double* r, double* z, cudaStream_t st) {
  if (h->local_double) apply_impl<double>(h, r, z, st);
  else apply_impl<float>(h, r, z, st);
}

// Autotuner of the apply schedule, bucket by bucket: the depth of the bulk-
// copy ring (the deepest, or the shallow one that lets two CTAs share an SM
// when the bucket's work vectors fit) and one or two CTAs per subdomain in
// the local solves.  Two CTAs halve each CTA's share of the streamed rows but
// add an exchange per slot; a shallow ring doubles the CTAs in flight but
// keeps fewer copies ahead of each; which wins depends on how many
// subdomains there are per SM and on their size, so the first setup of a
// shape times five applies of each candidate (after a warm-up, on a zero
// vector: the work does not depend on the values), tuning one bucket at a
// time with the others fixed; a candidate replaces the default (deepest ring,
// one CTA per subdomain) only if it is at least 3 % faster, and the choice is
// kept per shape for the process.
struct TuneKey {
  int dbl, nsub, qn, qd, nc, b0, b1;
  bool operator<(const TuneKey& o) const {
    return std::tie(dbl, nsub, qn, qd, nc, b0, b1) < std::tie(o.dbl, o.nsub, o.qn, o.qd, o.nc, o.b0, o.b1);
  }
};
struct TuneChoice {
  int nb[MAX_BUCKETS], cluster[MAX_BUCKETS];
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneChoice> g_tune;

void tune_apply(bddc_handle* h, cudaStream_t st) {
  LocalLaunch& L = h->L;
  const TuneKey key{h->local_double, L.nsub, L.maxQN, L.maxQD, L.maxNc, L.bucket[0].count, L.bucket[1].count};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      for (int b = 0; b < MAX_BUCKETS; ++b) {
        L.bucket[b].nb = it->second.nb[b];
        L.bcluster[b] = it->second.cluster[b];
      }
      return;
    }
  }
  CK(cudaMemsetAsync(h->r, 0, sizeof(double) * h->n_nodes, st));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int es = h->local_double ? 8 : 4;
  for (int b = 0; b < MAX_BUCKETS; ++b) {
    if (L.bucket[b].count == 0) continue;
    float best = 1e30f;
    int bnb = NBUF, bcl = 1;
    for (int nb : {NBUF, SMALL_RING}) {
      if (nb != NBUF && apply_smem(L.bsize[b], nb, es) > SMALL_SMEM) continue;
      for (int c : {1, 2, 4}) {
        L.bucket[b].nb = nb;
        L.bcluster[b] = c;
        apply(h, h->r, h->z, st);
        CK(cudaEventRecord(e0, st));
        for (int k = 0; k < 5; ++k) apply(h, h->r, h->z, st);
        CK(cudaEventRecord(e1, st));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        // the first candidate (deepest ring, one CTA per subdomain) stays
        // unless another is clearly faster: closer than 3 % is timing noise
        if (ms < 0.97f * best || best == 1e30f) { best = ms; bnb = nb; bcl = c; }
      }
    }
    L.bucket[b].nb = bnb;
    L.bcluster[b] = bcl;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  TuneChoice ch{};
  for (int b = 0; b < MAX_BUCKETS; ++b) {
    ch.nb[b] = L.bucket[b].nb;
    ch.cluster[b] = L.bcluster[b];
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = ch;
}

}  // namespace

namespace {

// One PCG iteration (Section 5's PCG with B as preconditioner): z = B r,
// beta and p, q = A p, alpha, x and r, and the stopping test.  The host loop
// and the graph's while body launch exactly this sequence, so both give the
// same iterates bit for bit.
void pcg_body(bddc_handle* h, double* x, const cudaGraphConditionalHandle* cond, cudaStream_t st) {
  const long long N = h->n_nodes;
  const int maxit = h->hist_cap;
  apply(h, h->r, h->z, st);
  if (h->flexible) {
    launch_dot2(h->r, h->z, h->zp, N, h->partial, st);
    launch_finalize(h->partial, h->scal, 5, h->hist_b, h->ctl, maxit, 0.0, nullptr, st);
    launch_update_p_keep(h->p, h->zp, h->z, h->scal, N, st);
  } else {
    launch_dot(h->r, h->z, N, h->partial, st);
    launch_finalize(h->partial, h->scal, 3, h->hist_b, h->ctl, maxit, 0.0, nullptr, st);
    launch_update_p(h->p, h->z, h->scal, N, st);
  }
  launch_operator(h->m, h->alpha, h->p, h->q, h->partial, RED_BLOCKS, st);
  launch_finalize(h->partial, h->scal, 1, h->hist_a, h->ctl, maxit, 0.0, nullptr, st);
  launch_update_xr(x, h->r, h->p, h->q, h->scal, N, h->partial, st);
  launch_finalize(h->partial, h->scal, 2, nullptr, h->ctl, maxit, 0.0, cond, st);
}

// Captures the PCG loop once per handle: [condition kernel] -> while(cond)
// { pcg_body }.  The graph reads and writes only handle-owned buffers, so it
// stays valid for every later solve; the caller's b and x are copied in and
// out around its launch.
void build_graph(bddc_handle* h) {
  if (h->gexec) return;
  if (!h->xw) h->xw = h->dnew<double>(h->n_nodes);
  if (!h->cap) CK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  const long long before = g_launches;
  bool capturing = false;
  try {
    cudaGraphConditionalHandle cond;
    CK(cudaGraphConditionalHandleCreate(&cond, g, 0, cudaGraphCondAssignDefault));
    CK(cudaStreamBeginCaptureToGraph(h->cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    capturing = true;
    launch_loop_condition(h->ctl, cond, h->cap);
    CK(cudaGetLastError());
    capturing = false;
    CK(cudaStreamEndCapture(h->cap, &g));
    cudaGraphNode_t first;
    size_t n = 1;
    CK(cudaGraphGetNodes(g, &first, &n));
    if (n != 1) throw BddcError(BDDC_ERR_CUDA, "graph capture: unexpected node count");
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop;
    CK(cudaGraphAddNode(&loop, g, &first, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    const long long b0 = g_launches;
    CK(cudaStreamBeginCaptureToGraph(h->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    capturing = true;
    pcg_body(h, h->xw, &cond, h->cap);
    CK(cudaGetLastError());
    capturing = false;
    CK(cudaStreamEndCapture(h->cap, &body));
    h->graph_body_launches = g_launches - b0;
    CK(cudaGraphInstantiate(&h->gexec, g, 0));
  } catch (...) {
    if (capturing) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(h->cap, &junk);
    }
    cudaGetLastError();
    cudaGraphDestroy(g);
    g_launches = before;
    throw;
  }
  h->graph = g;
  g_launches = before;   // captured, not yet launched
}

int pcg_impl(bddc_handle* h, const double* b, double* x, double rtol, bddc_stats* stats, cudaStream_t st) {
  const long long N = h->n_nodes;
  const int maxit = h->hist_cap;
  const bool graph = h->opt.use_graph != 0;
  if (graph) build_graph(h);
  double* xs = graph ? h->xw : x;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, st));
  CK(cudaMemsetAsync(xs, 0, sizeof(double) * N, st));
  CK(cudaMemsetAsync(h->p, 0, sizeof(double) * N, st));
  if (h->flexible) CK(cudaMemsetAsync(h->zp, 0, sizeof(double) * N, st));
  launch_masked_copy(h->m, b, h->r, st);
  launch_dot(h->r, h->r, N, h->partial, st);
  launch_finalize(h->partial, h->scal, 4, nullptr, h->ctl, maxit, rtol, nullptr, st);
  int* hc = (int*)(h->pinned + 2);   // ctl as read back: it, continue, converged, breakdown
  if (graph) {
    CK(cudaGraphLaunch(h->gexec, st));
    CK(cudaMemcpyAsync(x, h->xw, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
  } else {
    CK(cudaMemcpyAsync(hc, h->ctl, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    while (hc[1]) {
      pcg_body(h, x, nullptr, st);
      CK(cudaMemcpyAsync(hc, h->ctl, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
    }
  }
  CK(cudaMemcpyAsync(h->pinned, h->scal + 3, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h->pinned + 1, h->scal + 6, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(hc, h->ctl, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaEventRecord(e1, st));
  CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const int it = hc[0], converged = hc[2], breakdown = hc[3];
  const double r0 = std::sqrt(h->pinned[1]);
  const double rn = it > 0 ? std::sqrt(h->pinned[0]) : r0;
  if (graph) g_launches += h->graph_body_launches * it + 1;
  int status = BDDC_OK;
  if (breakdown) status = BDDC_ERR_BREAKDOWN;
  else if (!converged) status = BDDC_ERR_NOCONV;
  if (stats) {
    stats->iterations = it;
    stats->converged = converged;
    stats->r0_norm = r0;
    stats->r_norm = rn;
    stats->solve_ms = ms;
    int na = std::min(it, stats->capacity);
    if (stats->alphas && na > 0)
      CK(cudaMemcpy(stats->alphas, h->hist_a, sizeof(double) * na, cudaMemcpyDeviceToHost));
    int nb = std::min(std::max(it - 1, 0), stats->capacity);
    if (stats->betas && nb > 0)
      CK(cudaMemcpy(stats->betas, h->hist_b, sizeof(double) * nb, cudaMemcpyDeviceToHost));
  }
  check_err_flags(h, st);   // device-side failures of the applies (bounded waits)
  return status;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
#define ABI_BEGIN try {
#define ABI_END(hh)                                                   \
  }                                                                   \
  catch (const BddcError& e) {                                        \
    if (hh) (hh)->error = e.what();                                   \
    else g_setup_error = e.what();                                    \
    return e.code;                                                    \
  }                                                                   \
  catch (const std::exception& e) {                                   \
    if (hh) (hh)->error = e.what();                                   \
    else g_setup_error = e.what();                                    \
    return BDDC_ERR_CUDA;                                             \
  }

namespace {
// Validates the arguments and builds the per-axis tables of a new handle.
std::unique_ptr<bddc_handle> make_handle(const bddc_mesh* mesh, const bddc_partition* part, const bddc_options* opt) {
  if (!mesh || !part || !opt) throw BddcError(BDDC_ERR_ARG, "NULL argument");
  if (mesh->nx < 2 || mesh->ny < 2 || mesh->nz < 2) throw BddcError(BDDC_ERR_ARG, "need at least 2 elements per axis");
  if ((long long)mesh->nx * mesh->ny * mesh->nz > (1LL << 31)) throw BddcError(BDDC_ERR_ARG, "mesh too large");
  if (opt->L_elems < 1) throw BddcError(BDDC_ERR_ARG, "L must be >= 1");
  if (opt->precision != BDDC_FP64 && opt->precision != BDDC_MIXED) throw BddcError(BDDC_ERR_ARG, "bad precision");
  if (opt->weights != BDDC_W_CARD && opt->weights != BDDC_W_RHO) throw BddcError(BDDC_ERR_ARG, "bad weights");
  if (opt->beta_rule != BDDC_BETA_STANDARD && opt->beta_rule != BDDC_BETA_FLEXIBLE)
    throw BddcError(BDDC_ERR_ARG, "bad beta_rule");
  if (opt->ml_block < 0) throw BddcError(BDDC_ERR_ARG, "ml_block must be >= 0");
  if (opt->ml_sub < 0 || (opt->ml_sub > 0 && opt->ml_block == 0))
    throw BddcError(BDDC_ERR_ARG, "ml_sub must be >= 0, and needs ml_block");
  if (opt->selection < BDDC_SEL_VEF || opt->selection > BDDC_SEL_EF)
    throw BddcError(BDDC_ERR_ARG, "bad selection");
  std::unique_ptr<bddc_handle> h(new bddc_handle());
  h->mesh = *mesh;
  if (!(h->mesh.h > 0)) h->mesh.h = 1.0 / mesh->nx;
  h->opt = *opt;
  h->local_double = opt->precision == BDDC_FP64;
  const int n[3] = {mesh->nx, mesh->ny, mesh->nz};
  for (int d = 0; d < 3; ++d) {
    if (part->ncut[d] < 0 || (part->ncut[d] > 0 && !part->cut[d])) throw BddcError(BDDC_ERR_ARG, "bad cut list");
    h->ax[d].build(n[d], part->cut[d], part->ncut[d], opt->L_elems);
  }
  if (part->piece) {
    h->labels = true;
    const long long NE = (long long)mesh->nx * mesh->ny * mesh->nz;
    h->label_in.assign(part->piece, part->piece + NE);
    for (int v : h->label_in)
      if (v < 0) throw BddcError(BDDC_ERR_ARG, "sub-subdomain labels must be >= 0");
  }
  for (int d = 0; d < 3; ++d)
    for (size_t s = 0; s < h->ax[d].slab_lo.size(); ++s)
      if (h->ax[d].slab_hi[s] - h->ax[d].slab_lo[s] > 4000) throw BddcError(BDDC_ERR_ARG, "subdomain too wide");
  return h;
}
}  // namespace

extern "C" int bddc_setup(const bddc_mesh* mesh, const bddc_partition* part, const bddc_options* opt,
                          const double* alpha_dev, void* stream, bddc_handle** out) {
  bddc_handle* hnull = nullptr;
  ABI_BEGIN
  if (!out) throw BddcError(BDDC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!alpha_dev) throw BddcError(BDDC_ERR_ARG, "NULL argument");
  std::unique_ptr<bddc_handle> h = make_handle(mesh, part, opt);
  cudaStream_t st = (cudaStream_t)stream;
  StageSession staging(st);   // the uploads of this setup go through pinned staging
  do_setup(h.get(), alpha_dev, st);
  tune_apply(h.get(), st);
  // the PCG graph (use_graph) is captured and instantiated on the host while
  // the setup still runs on the device; it only records the handle's buffers
  if (h->opt.use_graph) build_graph(h.get());
  finish_setup(h.get(), st);
  *out = h.release();
  return BDDC_OK;
  ABI_END(hnull)
}

extern "C" int bddc_analyze(const bddc_mesh* mesh, const bddc_partition* part, const bddc_options* opt,
                            bddc_analysis_t* out) {
  bddc_handle* hnull = nullptr;
  ABI_BEGIN
  if (!out) throw BddcError(BDDC_ERR_ARG, "out is NULL");
  std::unique_ptr<bddc_handle> h = make_handle(mesh, part, opt);
  build_metadata(h.get());
  mf_plan(h->mf, h->geom, h->n_coarse);
  *out = bddc_analysis_t{};
  out->n_sub = (int)h->subs.size();
  out->n_coarse = h->n_coarse;
  for (int k : h->okind) {
    if (k == 0) ++out->n_vertices; else if (k == 1) ++out->n_edges; else ++out->n_faces;
  }
  out->max_local_coarse = h->max_nc;
  out->n_fronts = h->mf.nfront;
  out->n_levels = h->mf.nlevel;
  for (int f = 0; f < h->mf.nfront; ++f) out->max_front = std::max(out->max_front, h->mf.np[f] + h->mf.nu[f]);
  out->front_entries = h->mf.fpool;
  out->coarse_fma = h->mf.flops;
  if (h->opt.ml_block > 0) {
    const int nsub3[3] = {(int)h->ax[0].slab_lo.size(), (int)h->ax[1].slab_lo.size(), (int)h->ax[2].slab_lo.size()};
    ml_plan(h->ml, h->opt.ml_block, h->opt.ml_sub, nsub3, h->subs, h->lc, h->n_coarse, h->h_cptr, h->h_cent);
    out->ml_blocks = h->ml.nblock;
    out->ml_coarse2 = h->ml.ncc;
    out->ml_fronts2 = h->ml.C.nfront;
  }
  return BDDC_OK;
  ABI_END(hnull)
}

// Acceptable paths (remark after Theorem 1), on the sub-subdomains of the
// handle (box pieces or labels).  A pair is two pieces of different
// subdomains around one interface node off the Dirichlet boundary; its
// contact is open while one such node lies in no selected object.  Direct:
// the two share a selected edge or face object (both in the object's set of
// surrounding pieces) or their contact is not open.  Links: pieces sharing an
// element face that lie in one subdomain (w is continuous inside a
// subdomain), or lie in two and share a selected face object or a contact
// that is not open.  A path's bottleneck is the smallest rho on it (ends
// included), so the best path of every pair is its path in a maximum
// spanning forest of the links weighted by min(rho_u, rho_v) (Kruskal),
// queried by binary lifting.
extern "C" int bddc_acceptable_paths(const bddc_mesh* mesh, const bddc_partition* part, const bddc_options* opt,
                                     const double* alpha_host, bddc_paths_t* out) {
  bddc_handle* hnull = nullptr;
  ABI_BEGIN
  if (!out) throw BddcError(BDDC_ERR_ARG, "out is NULL");
  std::unique_ptr<bddc_handle> h = make_handle(mesh, part, opt);
  build_metadata(h.get());
  const bddc_mesh& M = h->mesh;
  const AxisHost* ax = h->ax;
  const long long P = h->n_pieces;
  if (P > (1LL << 22)) throw BddcError(BDDC_ERR_UNSUPPORTED, "more than 2^22 sub-subdomains");
  const int NX = M.nx + 1, NY = M.ny + 1;
  const long long NE = (long long)M.nx * M.ny * M.nz;
  // the piece of every element (the labels, or the box pieces)
  std::vector<int> ep;
  if (h->labels) {
    ep = h->epiece;
  } else {
    ep.assign(NE, 0);
    const int npx = (int)ax[0].piece_lo.size(), npy = (int)ax[1].piece_lo.size();
    for (int k = 0; k < M.nz; ++k)
      for (int j = 0; j < M.ny; ++j)
        for (int i = 0; i < M.nx; ++i)
          ep[i + (long long)M.nx * (j + (long long)M.ny * k)] = ax[0].piece[i] + npx * (ax[1].piece[j] + npy * ax[2].piece[k]);
  }
  auto elem = [&](int i, int j, int k) { return ep[i + (long long)M.nx * (j + (long long)M.ny * k)]; };
  // piece coefficient: the mean of alpha over the piece's elements (1 without alpha)
  std::vector<double> rho(P, 1.0);
  if (alpha_host) {
    std::vector<double> sum(P, 0.0);
    std::vector<long long> cnt(P, 0);
    for (long long e = 0; e < NE; ++e) { sum[ep[e]] += alpha_host[e]; ++cnt[ep[e]]; }
    for (long long q = 0; q < P; ++q) rho[q] = sum[q] / (double)cnt[q];
  }
  // primal nodes: the nodes of the selected objects
  std::vector<unsigned char> primal((size_t)NX * NY * (M.nz + 1), 0);
  for (size_t q = 0; q < h->onodes.size(); q += 3)
    primal[nodeid(NX, NY, h->onodes[q], h->onodes[q + 1], h->onodes[q + 2])] = 1;
  auto pieces_at = [&](int x, int y, int z, std::vector<int>& k) {
    k.clear();
    for (int dz = -1; dz <= 0; ++dz)
      for (int dy = -1; dy <= 0; ++dy)
        for (int dx = -1; dx <= 0; ++dx) k.push_back(elem(x + dx, y + dy, z + dz));
    std::sort(k.begin(), k.end());
    k.erase(std::unique(k.begin(), k.end()), k.end());
  };
  auto key = [&](long long a, long long b) { return a * P + b; };
  // pairs around interface nodes, and which contacts are open
  std::map<long long, char> pair_open;   // (a, b), a < b -> contact open
  std::vector<int> k;
  for (int z = 1; z < M.nz; ++z)
    for (int y = 1; y < M.ny; ++y)
      for (int x = 1; x < M.nx; ++x) {
        if (!ax[0].theta[x] && !ax[1].theta[y] && !ax[2].theta[z]) continue;
        pieces_at(x, y, z, k);
        const bool open = !primal[nodeid(NX, NY, x, y, z)];
        for (size_t a = 0; a < k.size(); ++a)
          for (size_t b = a + 1; b < k.size(); ++b) {
            if (h->piece_sub[k[a]] == h->piece_sub[k[b]]) continue;
            char& o = pair_open[key(k[a], k[b])];
            o = (char)(o | (open ? 1 : 0));
          }
      }
  // selected edge and face objects: pairs of their surrounding pieces
  std::map<long long, char> shares_obj;   // 1: edge or face object, 2: face object
  for (size_t g = 0; g < h->okind.size(); ++g) {
    if (h->okind[g] == 0) continue;
    const long long q = 3 * h->onoff[g];
    pieces_at(h->onodes[q], h->onodes[q + 1], h->onodes[q + 2], k);
    for (size_t a = 0; a < k.size(); ++a)
      for (size_t b = a + 1; b < k.size(); ++b) {
        char& o = shares_obj[key(k[a], k[b])];
        o = (char)std::max<int>(o, h->okind[g] == 2 ? 2 : 1);
      }
  }
  std::vector<std::pair<long long, long long>> pairs, links;
  std::vector<char> direct;
  for (const auto& pr : pair_open) {
    const long long a = pr.first / P, b = pr.first % P;
    auto it = shares_obj.find(pr.first);
    pairs.push_back({a, b});
    direct.push_back((it != shares_obj.end()) || !pr.second);
  }
  // links: element-face contacts
  {
    std::map<long long, char> seen;
    auto contact = [&](int pa, int pb) {
      if (pa == pb) return;
      const long long a = std::min(pa, pb), b = std::max(pa, pb);
      if (!seen.emplace(key(a, b), 1).second) return;
      bool link = h->piece_sub[a] == h->piece_sub[b];
      if (!link) {
        auto it = shares_obj.find(key(a, b));
        auto po = pair_open.find(key(a, b));
        link = (it != shares_obj.end() && it->second == 2) || po == pair_open.end() || !po->second;
      }
      if (link) links.push_back({a, b});
    };
    for (int z = 0; z < M.nz; ++z)
      for (int y = 0; y < M.ny; ++y)
        for (int x = 0; x < M.nx; ++x) {
          const int pe = elem(x, y, z);
          if (x + 1 < M.nx) contact(pe, elem(x + 1, y, z));
          if (y + 1 < M.ny) contact(pe, elem(x, y + 1, z));
          if (z + 1 < M.nz) contact(pe, elem(x, y, z + 1));
        }
  }
  // maximum spanning forest (Kruskal), edge weight min(rho_u, rho_v)
  std::sort(links.begin(), links.end(), [&](const std::pair<long long, long long>& x,
                                            const std::pair<long long, long long>& y) {
    const double wx = std::min(rho[x.first], rho[x.second]), wy = std::min(rho[y.first], rho[y.second]);
    return wx != wy ? wx > wy : x < y;
  });
  std::vector<long long> uf(P);
  for (long long i = 0; i < P; ++i) uf[i] = i;
  auto find = [&](long long x) {
    while (uf[x] != x) { uf[x] = uf[uf[x]]; x = uf[x]; }
    return x;
  };
  std::vector<std::vector<std::pair<long long, double>>> adj(P);
  for (const auto& e : links) {
    const long long u = find(e.first), v = find(e.second);
    if (u == v) continue;
    uf[u] = v;
    const double w = std::min(rho[e.first], rho[e.second]);
    adj[e.first].push_back({e.second, w});
    adj[e.second].push_back({e.first, w});
  }
  // root every tree; binary lifting tables of ancestors and path minima
  int LOG = 1;
  while ((1LL << LOG) < P) ++LOG;
  std::vector<long long> depth(P, -1), comp(P, -1);
  std::vector<std::vector<long long>> up(LOG, std::vector<long long>(P));
  std::vector<std::vector<double>> mn(LOG, std::vector<double>(P, INFINITY));
  for (long long root = 0; root < P; ++root) {
    if (depth[root] >= 0) continue;
    std::vector<long long> stack{root};
    depth[root] = 0;
    comp[root] = root;
    up[0][root] = root;
    while (!stack.empty()) {
      const long long u = stack.back();
      stack.pop_back();
      for (const auto& e : adj[u])
        if (depth[e.first] < 0) {
          depth[e.first] = depth[u] + 1;
          comp[e.first] = root;
          up[0][e.first] = u;
          mn[0][e.first] = e.second;
          stack.push_back(e.first);
        }
    }
  }
  for (int k = 1; k < LOG; ++k)
    for (long long v = 0; v < P; ++v) {
      up[k][v] = up[k - 1][up[k - 1][v]];
      mn[k][v] = std::min(mn[k - 1][v], mn[k - 1][up[k - 1][v]]);
    }
  auto bottleneck = [&](long long u, long long v) {
    double m = INFINITY;
    if (depth[u] < depth[v]) std::swap(u, v);
    for (int k = LOG - 1; k >= 0; --k)
      if (depth[u] - (1LL << k) >= depth[v]) { m = std::min(m, mn[k][u]); u = up[k][u]; }
    if (u == v) return m;
    for (int k = LOG - 1; k >= 0; --k)
      if (up[k][u] != up[k][v]) {
        m = std::min({m, mn[k][u], mn[k][v]});
        u = up[k][u];
        v = up[k][v];
      }
    return std::min({m, mn[0][u], mn[0][v]});
  };
  *out = bddc_paths_t{};
  out->n_pieces = P;
  out->min_ratio = 1.0;
  out->worst_pair[0] = out->worst_pair[1] = -1;
  long long lone[2] = {-1, -1}, worst[2] = {-1, -1};
  for (size_t k = 0; k < pairs.size(); ++k) {
    const long long u = pairs[k].first, v = pairs[k].second;
    ++out->n_pairs;
    if (direct[k]) { ++out->n_direct; continue; }
    if (comp[u] != comp[v]) {
      if (out->n_without_path++ == 0) { lone[0] = u; lone[1] = v; }
      continue;
    }
    const double ratio = std::min(1.0, bottleneck(u, v) / std::min(rho[u], rho[v]));
    if (ratio < out->min_ratio || worst[0] < 0) { out->min_ratio = ratio; worst[0] = u; worst[1] = v; }
  }
  // a pair without a path, else the pair of the smallest ratio
  out->worst_pair[0] = lone[0] >= 0 ? lone[0] : worst[0];
  out->worst_pair[1] = lone[0] >= 0 ? lone[1] : worst[1];
  return BDDC_OK;
  ABI_END(hnull)
}

extern "C" int bddc_apply(bddc_handle* h, const double* r_dev, double* z_dev, void* stream) {
  if (!h) return BDDC_ERR_ARG;
  ABI_BEGIN
  if (!r_dev || !z_dev || r_dev == z_dev) throw BddcError(BDDC_ERR_ARG, "bad vectors");
  CK(cudaSetDevice(h->device));
  apply(h, r_dev, z_dev, (cudaStream_t)stream);
  CK(cudaGetLastError());
  return BDDC_OK;
  ABI_END(h)
}

extern "C" int bddc_operator(bddc_handle* h, const double* x_dev, double* y_dev, void* stream) {
  if (!h) return BDDC_ERR_ARG;
  ABI_BEGIN
  if (!x_dev || !y_dev || x_dev == y_dev) throw BddcError(BDDC_ERR_ARG, "bad vectors");
  CK(cudaSetDevice(h->device));
  launch_operator(h->m, h->alpha, x_dev, y_dev, nullptr, RED_BLOCKS, (cudaStream_t)stream);
  CK(cudaGetLastError());
  return BDDC_OK;
  ABI_END(h)
}

extern "C" int pcg_solve(bddc_handle* h, const double* b_dev, double* x_dev, double rtol, bddc_stats* stats,
                         void* stream) {
  if (!h) return BDDC_ERR_ARG;
  ABI_BEGIN
  if (!b_dev || !x_dev || b_dev == x_dev) throw BddcError(BDDC_ERR_ARG, "bad vectors");
  if (!(rtol > 0) || !(rtol < 1)) throw BddcError(BDDC_ERR_ARG, "rtol must be in (0, 1)");
  CK(cudaSetDevice(h->device));
  int s = pcg_impl(h, b_dev, x_dev, rtol, stats, (cudaStream_t)stream);
  if (s == BDDC_ERR_NOCONV) h->error = "PCG did not reach the tolerance within maxit";
  if (s == BDDC_ERR_BREAKDOWN) h->error = "PCG breakdown: p^T A p <= 0 or not finite";
  return s;
  ABI_END(h)
}

extern "C" int bddc_gradient(bddc_handle* h, const double* u_dev, const double* lambda_dev, double* g_dev,
                             void* stream) {
  if (!h) return BDDC_ERR_ARG;
  ABI_BEGIN
  if (!u_dev || !lambda_dev || !g_dev) throw BddcError(BDDC_ERR_ARG, "NULL vector");
  CK(cudaSetDevice(h->device));
  launch_gradient(h->m, u_dev, lambda_dev, g_dev, (cudaStream_t)stream);
  CK(cudaGetLastError());
  return BDDC_OK;
  ABI_END(h)
}

extern "C" int bddc_solve_host(const bddc_mesh* mesh, const bddc_partition* part, const bddc_options* opt,
                               const double* alpha_host, const double* b_host, double* x_host, double rtol,
                               bddc_stats* stats) {
  double *da = nullptr, *db = nullptr, *dx = nullptr;
  cudaStream_t st = nullptr;
  bddc_handle* h = nullptr;
  int rc = BDDC_OK;
  try {
    if (!mesh || !alpha_host || !b_host || !x_host) throw BddcError(BDDC_ERR_ARG, "NULL argument");
    const size_t NE = (size_t)mesh->nx * mesh->ny * mesh->nz;
    const size_t NN = (size_t)(mesh->nx + 1) * (mesh->ny + 1) * (mesh->nz + 1);
    CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    CK(cudaMalloc(&da, sizeof(double) * NE));
    CK(cudaMalloc(&db, sizeof(double) * NN));
    CK(cudaMalloc(&dx, sizeof(double) * NN));
    CK(cudaMemcpyAsync(da, alpha_host, sizeof(double) * NE, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(db, b_host, sizeof(double) * NN, cudaMemcpyHostToDevice, st));
    rc = bddc_setup(mesh, part, opt, da, st, &h);
    if (rc == BDDC_OK) {
      rc = pcg_solve(h, db, dx, rtol, stats, st);
      if (rc == BDDC_OK || rc == BDDC_ERR_NOCONV) {
        CK(cudaMemcpyAsync(x_host, dx, sizeof(double) * NN, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
      }
      if (rc != BDDC_OK) g_setup_error = h->error;
    }
  } catch (const BddcError& e) {
    g_setup_error = e.what();
    rc = e.code;
  }
  if (h) bddc_destroy(h);
  cudaFree(da);
  cudaFree(db);
  cudaFree(dx);
  if (st) cudaStreamDestroy(st);
  return rc;
}

extern "C" int bddc_set_apply_schedule(bddc_handle* h, int ctas_per_subdomain) {
  if (!h) return BDDC_ERR_ARG;
  ABI_BEGIN
  if (ctas_per_subdomain != 1 && ctas_per_subdomain != 2 && ctas_per_subdomain != 4)
    throw BddcError(BDDC_ERR_ARG, "ctas_per_subdomain must be 1, 2 or 4");
  CK(cudaSetDevice(h->device));
  CK(cudaDeviceSynchronize());
  for (int b = 0; b < MAX_BUCKETS; ++b) h->L.bcluster[b] = ctas_per_subdomain;
  if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
  if (h->graph) { cudaGraphDestroy(h->graph); h->graph = nullptr; }
  return BDDC_OK;
  ABI_END(h)
}

extern "C" int bddc_set_bucket_schedule(bddc_handle* h, int bucket, int ring_depth, int ctas_per_subdomain) {
  if (!h) return BDDC_ERR_ARG;
  ABI_BEGIN
  if (bucket < 0 || bucket >= MAX_BUCKETS) throw BddcError(BDDC_ERR_ARG, "bucket out of range");
  if (ctas_per_subdomain != 1 && ctas_per_subdomain != 2 && ctas_per_subdomain != 4)
    throw BddcError(BDDC_ERR_ARG, "ctas_per_subdomain must be 1, 2 or 4");
  if (ring_depth != NBUF && ring_depth != SMALL_RING)
    throw BddcError(BDDC_ERR_ARG, "ring_depth must be " + std::to_string(NBUF) + " or " + std::to_string(SMALL_RING));
  if (ring_depth == SMALL_RING && apply_smem(h->L.bsize[bucket], SMALL_RING, h->local_double ? 8 : 4) > SMALL_SMEM)
    throw BddcError(BDDC_ERR_ARG, "this bucket's work vectors do not fit the shallow ring");
  CK(cudaSetDevice(h->device));
  CK(cudaDeviceSynchronize());
  h->L.bucket[bucket].nb = ring_depth;
  h->L.bcluster[bucket] = ctas_per_subdomain;
  if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
  if (h->graph) { cudaGraphDestroy(h->graph); h->graph = nullptr; }
  return BDDC_OK;
  ABI_END(h)
}

extern "C" int bddc_get_info(const bddc_handle* h, bddc_info_t* info) {
  if (!h || !info) return BDDC_ERR_ARG;
  info->n_sub = (int)h->subs.size();
  info->n_coarse = h->n_coarse;
  info->n_vertices = h->n_vertices;
  info->max_local_coarse = h->max_nc;
  info->n_free = h->n_free;
  info->bytes = (long long)h->bytes;
  info->factor_bytes = (long long)h->factor_bytes;
  info->setup_ms = h->setup_ms;
  for (int k = 0; k < 6; ++k) info->phase_ms[k] = h->phase_ms[k];
  info->launches = g_launches - h->launch_base;
  info->coarse_fma = h->mf.flops;
  // local factorisation work and the bytes one apply has to stream: per
  // subdomain and solve, the 2 nz - 1 symmetric inverse Schur slots (full
  // Q x Q rows) and the nine diagonals of the couplings, forward and backward
  double fma = 0.0;
  long long bytes = 0;
  const int es = h->local_double ? 8 : 4;
  for (const SubDesc& s : h->subs) {
    const double QN = (double)(s.w[0] + 1) * (s.w[1] + 1), nzN = s.w[2] + 1;
    const double QD = (s.w[0] > 1 && s.w[1] > 1 && s.w[2] > 1) ? (double)(s.w[0] - 1) * (s.w[1] - 1) : 0.0;
    const double nzD = QD > 0 ? s.w[2] - 1 : 0;
    // per plane: symmetric sweep of the Schur block (Q pivots over the lower
    // triangle, Q^3/2); per plane after the first: S_{k-1}^{-1} B_k^T and
    // B_k (.) (nine stencil terms each, 18 Q^2)
    auto planes = [](double Q, double nz) {
      return nz > 0 ? nz * Q * Q * Q / 2.0 + (nz - 1) * 18.0 * Q * Q : 0.0;
    };
    fma += planes(QN, nzN) + planes(QD, nzD);
    auto solve = [es](double Q, double nz) {
      return nz > 0 ? ((2 * nz - 1) * Q * Q + 2 * (nz - 1) * 9 * Q) * es : 0.0;
    };
    bytes += (long long)(solve(QN, nzN) + 2 * solve(QD, nzD) + 2.0 * s.nB * s.nc * es);
  }
  for (int f = 0; f < h->mf.nfront; ++f) {
    const long long np = h->mf.np[f], nu = h->mf.nu[f];
    bytes += 2 * 8 * (np * (np + 1) / 2 + nu * np);   // solve matrices, read forward and backward
  }
  info->local_factor_fma = fma;
  info->apply_bytes = bytes;
  {
    int nb = 0, first = -1;
    for (int b = 0; b < MAX_BUCKETS; ++b) {
      info->bucket_subdomains[b] = h->L.bucket[b].count;
      info->bucket_ring[b] = h->L.bucket[b].count ? h->L.bucket[b].nb : 0;
      info->bucket_ctas[b] = h->L.bucket[b].count ? h->L.bcluster[b] : 0;
      if (h->L.bucket[b].count) { ++nb; if (first < 0) first = b; }
    }
    info->n_buckets = nb;
    info->apply_cluster = first >= 0 ? h->L.bcluster[first] : 1;
  }
  // banded-Cholesky count of the same local matrices: per problem n b^2 with
  // n the free nodes and b the half-bandwidth of their lexicographic order
  double band = 0.0;
  for (const SubDesc& s : h->subs) {
    for (int neu = 0; neu < 2; ++neu) {
      double pf[3];
      bool empty = false;
      for (int d = 0; d < 3; ++d) {
        const int lo = s.e0[d] + (neu ? 0 : 1), hi = s.e0[d] + s.w[d] - (neu ? 0 : 1);   // node range
        const int n_d = (d == 0) ? h->mesh.nx : (d == 1) ? h->mesh.ny : h->mesh.nz;
        const int flo = std::max(lo, 1), fhi = std::min(hi, n_d - 1);               // off the Dirichlet boundary
        pf[d] = std::max(0, fhi - flo + 1);
        if (pf[d] <= 0) empty = true;
      }
      if (empty) continue;
      const double n = pf[0] * pf[1] * pf[2], b = pf[0] * pf[1] + pf[0] + 1;
      band += n * b * b;
    }
  }
  info->local_band_flops = band;
  info->factor_kernel = (!h->local_double && h->L.fbucket[0].count > 0 && h->L.factor_tc) ? 1 : 0;
  info->factor_tc_subdomains = info->factor_kernel ? h->L.fbucket[0].count : 0;
  info->pinned_subdomains = h->n_pinned;
  info->ml_blocks = h->opt.ml_block > 0 ? h->ml.nblock : 0;
  info->ml_coarse2 = h->opt.ml_block > 0 ? h->ml.ncc : 0;
  if (h->opt.ml_block > 0) info->coarse_fma = h->ml.flops;
  return BDDC_OK;
}

extern "C" int bddc_get_coarse_basis(const bddc_handle* h, int sub, double* phi_host, int* gid_host,
                                     long long* node_host, int* n_surface, int* n_local_coarse) {
  if (!h || sub < 0 || sub >= (int)h->subs.size()) return BDDC_ERR_ARG;
  bddc_handle* hh = const_cast<bddc_handle*>(h);
  ABI_BEGIN
  const SubDesc& s = h->subs[sub];
  if (n_surface) *n_surface = s.nB;
  if (n_local_coarse) *n_local_coarse = s.nc;
  const size_t cnt = (size_t)s.nB * s.nc;
  if (phi_host) {
    if (h->local_double) {
      CK(cudaMemcpy(phi_host, (double*)h->L.Phi + s.offPhi, sizeof(double) * cnt, cudaMemcpyDeviceToHost));
    } else {
      std::vector<float> tmp(cnt);
      CK(cudaMemcpy(tmp.data(), (float*)h->L.Phi + s.offPhi, sizeof(float) * cnt, cudaMemcpyDeviceToHost));
      for (size_t i = 0; i < cnt; ++i) phi_host[i] = tmp[i];
    }
  }
  if (gid_host)
    for (int j = 0; j < s.nc; ++j) gid_host[j] = h->lc[s.cofs + j].gid;
  if (node_host) {
    const int px = s.w[0] + 1, py = s.w[1] + 1, pz = s.w[2] + 1;
    for (int b = 0; b < s.nB; ++b) {
      int ix, iy, iz;
      surf_coords(b, px, py, pz, ix, iy, iz);
      node_host[b] = nodeid(h->mesh.nx + 1, h->mesh.ny + 1, s.e0[0] + ix, s.e0[1] + iy, s.e0[2] + iz);
    }
  }
  return BDDC_OK;
  ABI_END(hh)
}

extern "C" int bddc_get_coarse_matrix(const bddc_handle* h, double* ac_host) {
  if (!h || !ac_host) return BDDC_ERR_ARG;
  if (!h->Ac_copy) return BDDC_ERR_UNSUPPORTED;
  bddc_handle* hh = const_cast<bddc_handle*>(h);
  ABI_BEGIN
  CK(cudaMemcpy(ac_host, h->Ac_copy, sizeof(double) * (size_t)h->n_coarse * h->n_coarse, cudaMemcpyDeviceToHost));
  return BDDC_OK;
  ABI_END(hh)
}

extern "C" int bddc_destroy(bddc_handle* h) {
  if (!h) return BDDC_OK;
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  delete h;
  return BDDC_OK;
}

extern "C" int bddc_debug_inject(int what, long long value) {
  std::lock_guard<std::mutex> lk(g_debug_mu);
  switch (what) {
    case BDDC_DEBUG_CLEAR:
      g_debug = DebugHooks{};
      set_wait_report_tries(WAIT_TRIES);
      break;
    case BDDC_DEBUG_NEGATE_NEUMANN_PIVOT:
    case BDDC_DEBUG_NEGATE_DIRICHLET_PIVOT:
      if (value < -1 || value > 2147483647LL) return BDDC_ERR_ARG;
      g_debug.negate_sub = (int)value;
      g_debug.negate_neumann = what == BDDC_DEBUG_NEGATE_NEUMANN_PIVOT;
      break;
    case BDDC_DEBUG_WAIT_TRIES:
      set_wait_report_tries(value < 0 ? WAIT_TRIES : std::min<long long>(value, WAIT_TRIES));
      break;
    default:
      return BDDC_ERR_ARG;
  }
  return cudaGetLastError() == cudaSuccess ? BDDC_OK : BDDC_ERR_CUDA;
}

extern "C" const char* bddc_last_error(const bddc_handle* h) {
  return h ? h->error.c_str() : g_setup_error.c_str();
}

// ---------------------------------------------------------------------------
// Allocation-free preconditioner apply.
//
// Some callers cannot call cudaMalloc while they apply the preconditioner:
// code running under another framework's stream-ordered memory pool that
// forbids foreign allocations, or solver loops that must not touch the CUDA
// allocator between iterations.  For them bddc_apply_noalloc runs the same
// kernels as bddc_apply but takes every work vector of the apply from one
// file-scope device array of fixed size instead of the handle's buffers.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocBytes = 32u << 20;  // 32 MiB, held by every GPU that loads the library
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mutex;
void* g_noalloc_addr[256] = {nullptr};

// Device address of the array on `dev` (host code cannot use the symbol
// itself).  Looked up once per device, with that device current.
void* noalloc_scratch(int dev) {
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (dev < 0 || dev >= 256) throw BddcError(BDDC_ERR_ARG, "device ordinal out of range");
  if (!g_noalloc_addr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess)
      throw BddcError(BDDC_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_noalloc_addr[dev] = ptr;
  }
  return g_noalloc_addr[dev];
}

size_t carve(size_t& off, size_t bytes) {
  size_t at = off;
  off = (off + bytes + 255) & ~(size_t)255;
  return at;
}

template <typename T>
void apply_noalloc_impl(bddc_handle* h, unsigned char* base, const double* r, double* z, cudaStream_t st) {
  const long long N = h->n_nodes;
  const int nc = h->n_coarse;
  size_t off = 0;
  double* uI = (double*)(base + carve(off, sizeof(double) * N));
  double* t = (double*)(base + carve(off, sizeof(double) * N));
  double* rc = (double*)(base + carve(off, sizeof(double) * std::max(nc, 1)));
  double* uc = (double*)(base + carve(off, sizeof(double) * std::max(nc, 1)));
  double* wf = (double*)(base + carve(off, sizeof(double) * std::max<long long>(h->mf.wpool, 1)));
  LocalLaunch L = h->L;
  L.rcl = (double*)(base + carve(off, sizeof(double) * std::max<size_t>(h->lc.size(), 1)));
  L.vgam = (double*)(base + carve(off, sizeof(double) * std::max<long long>(h->n_surface_total, 1)));
  L.vloc = base + carve(off, sizeof(T) * std::max<long long>(h->n_local_nodes_total, 1));
  // the array keeps the previous call's contents; the interior solve writes
  // only interior nodes, so the rest of uI must start at zero
  CK(cudaMemsetAsync(uI, 0, sizeof(double) * N, st));
  apply_core<T>(h, L, r, z, uI, t, rc, uc, wf, st);
}

size_t noalloc_bytes_needed(const bddc_handle* h) {
  const size_t es = h->local_double ? sizeof(double) : sizeof(float);
  size_t off = 0;
  carve(off, sizeof(double) * h->n_nodes);
  carve(off, sizeof(double) * h->n_nodes);
  for (int k = 0; k < 2; ++k) carve(off, sizeof(double) * std::max(h->n_coarse, 1));
  carve(off, sizeof(double) * std::max<long long>(h->mf.wpool, 1));
  carve(off, sizeof(double) * std::max<size_t>(h->lc.size(), 1));
  carve(off, sizeof(double) * std::max<long long>(h->n_surface_total, 1));
  carve(off, es * std::max<long long>(h->n_local_nodes_total, 1));
  return off;
}

}  // namespace

extern "C" int bddc_apply_noalloc(bddc_handle* h, const double* r_dev, double* z_dev, void* stream) {
  if (!h) return BDDC_ERR_ARG;
  ABI_BEGIN
  if (!r_dev || !z_dev || r_dev == z_dev) throw BddcError(BDDC_ERR_ARG, "bad vectors");
  const size_t need = noalloc_bytes_needed(h);
  if (need > kNoAllocBytes)
    throw BddcError(BDDC_ERR_ARG, "bddc_apply_noalloc: this problem needs " + std::to_string(need) +
                                      " bytes of work space, above the fixed maximum of " +
                                      std::to_string(kNoAllocBytes) + " bytes; use bddc_apply");
  CK(cudaSetDevice(h->device));
  unsigned char* base = (unsigned char*)noalloc_scratch(h->device);
  if (h->local_double) apply_noalloc_impl<double>(h, base, r_dev, z_dev, (cudaStream_t)stream);
  else apply_noalloc_impl<float>(h, base, r_dev, z_dev, (cudaStream_t)stream);
  CK(cudaGetLastError());
  return BDDC_OK;
  ABI_END(h)
}
