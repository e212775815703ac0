// Streaming of row-major matrices from HBM into shared memory with 1-D bulk
// asynchronous copies (cp.async.bulk, the TMA engine) completing on mbarriers.
//
// A CTA owns a ring of NBUF buffers of CHB bytes.  One thread issues the copy
// of chunk c + NBUF as soon as chunk c has been consumed, so up to NBUF chunks
// (144 KiB) are in flight per SM while the CTA computes.  Only that thread
// polls the chunk's mbarrier; the others wait at a CTA barrier, so waiting
// costs no issue slots and does not compete with the copies for shared memory.  Chunks must start on
// 16-byte boundaries and their byte counts are rounded up to 16; callers pad
// their allocations accordingly.  Every wait is bounded: a wait that gives up
// records error code 7 (timeout) and the kernel carries on to its end.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace bddc {

constexpr int NBUF = 6;
constexpr int CHB = 24576;
constexpr long long WAIT_TRIES = 1LL << 22;

__device__ inline unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ inline void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ inline void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ inline void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ inline void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ inline bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ inline bool mbar_wait_bounded(uint64_t* bar, unsigned parity, int* err) {
  for (long long i = 0; i < WAIT_TRIES; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  if (err && atomicCAS(err, 0, 7) == 0) err[1] = blockIdx.x;
  return false;
}

struct Ring {
  unsigned char* buf;  // NBUF * CHB bytes, 128-byte aligned
  uint64_t* bar;       // NBUF mbarriers
  int base;            // chunks consumed by earlier runs (slot / parity bookkeeping)
};

// Initialise the ring's barriers (all threads call; ends with a barrier).
__device__ inline void ring_init(Ring& r) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < NBUF; ++s) mbar_init(&r.bar[s], 1);
    fence_barrier_init();
  }
  r.base = 0;
  __syncthreads();
}

// Streams nchunks chunks: src(c, &ptr, &bytes) describes chunk c (ptr
// 16-byte aligned, bytes > 0), use(c, smem) consumes it with every thread of
// the CTA.  Ends with a barrier.
template <typename Src, typename Use>
__device__ void ring_run(Ring& r, int nchunks, Src src, Use use, int* err) {
  const int first = r.base;
  if (threadIdx.x == 0) {
    for (int c = 0; c < nchunks && c < NBUF; ++c) {
      const void* p;
      unsigned bytes;
      src(c, p, bytes);
      const int slot = (first + c) % NBUF;
      bulk_load(r.buf + (size_t)slot * CHB, p, (bytes + 15u) & ~15u, &r.bar[slot]);
    }
  }
  for (int c = 0; c < nchunks; ++c) {
    const int g = first + c, slot = g % NBUF;
    if (threadIdx.x == 0) mbar_wait_bounded(&r.bar[slot], (unsigned)((g / NBUF) & 1), err);
    __syncthreads();
    use(c, r.buf + (size_t)slot * CHB);
    __syncthreads();
    if (threadIdx.x == 0 && c + NBUF < nchunks) {
      const void* p;
      unsigned bytes;
      src(c + NBUF, p, bytes);
      fence_proxy_async();
      bulk_load(r.buf + (size_t)slot * CHB, p, (bytes + 15u) & ~15u, &r.bar[slot]);
    }
  }
  r.base = first + nchunks;
}

// Rows of a row-major matrix with `cols` entries of `es` bytes per chunk: the
// largest count that fits a buffer and keeps every chunk start 16-byte aligned
// (0 if no such count exists).
__host__ __device__ inline int rows_per_chunk(int cols, int es) {
  const int row = cols * es;
  int step = 1;
  while ((step * row) % 16) ++step;   // 1, 2 or 4
  const int r = CHB / row;
  return (r / step) * step;
}

}  // namespace bddc
