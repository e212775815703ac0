// Streaming of row-major matrices from HBM into shared memory with 1-D bulk
// asynchronous copies (cp.async.bulk, the TMA engine) completing on mbarriers.
//
// A CTA owns a ring of nb buffers (NBUF or fewer) of CHB bytes with two mbarriers per
// buffer: "full" completes when the buffer's copy has landed, "empty" when
// every warp has finished reading it.  Every thread waits on "full" itself
// and each warp arrives on "empty" after its use of the chunk, so warps run
// ahead of each other up to the ring depth and no block-wide barrier is
// needed per chunk; one thread (the producer) waits on "empty" before it
// refills the buffer with chunk c + nb.  Chunks must start on 16-byte
// boundaries and their byte counts are rounded up to 16; callers pad their
// allocations accordingly.  Every wait is bounded: a wait that runs past its
// limit records error code 7 (timeout), waits (bounded again) for the copy
// it covers and the kernel carries on to its end.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace bddc {

constexpr int NBUF = 6;       // deepest ring (one CTA per SM); shallower rings leave room for two
constexpr int CHB = 24576;
constexpr long long WAIT_TRIES = 1LL << 22;
constexpr int APPLY_THREADS = 512;   // threads of the streaming apply kernels

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

// Tries after which a bounded wait reports a timeout.  WAIT_TRIES unless a
// test lowers it (bddc_debug_inject); one copy per translation unit.
static __device__ long long g_wait_report_tries = WAIT_TRIES;

// Waits for the phase with the given parity.  After g_wait_report_tries
// unsuccessful tries it records error code 7 (timeout) with the block index;
// the copy or MMA the barrier tracks is still this CTA's own work in flight,
// so it then keeps waiting, for at most WAIT_TRIES more tries, before it
// returns.  Returns whether the phase completed.
__device__ inline bool mbar_wait_bounded(uint64_t* bar, unsigned parity, int* err) {
  const long long report = g_wait_report_tries;
  for (long long i = 0; i < report; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  if (err && atomicCAS(err, 0, 7) == 0) err[1] = blockIdx.x;
  for (long long i = 0; i < WAIT_TRIES; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

struct Ring {
  unsigned char* buf;  // nb * CHB bytes, 128-byte aligned
  uint64_t* bar;       // 2 nb mbarriers: full[0..nb), then empty[0..nb)
  int base;            // chunks consumed by earlier runs (slot / parity bookkeeping)
  int nb;              // buffers in the ring (2 .. NBUF)
};

// Shared-memory bytes of a ring of nb buffers with its barriers.
__host__ __device__ inline size_t ring_bytes(int nb) { return (size_t)nb * CHB + 16 * (size_t)nb; }

// A ring of nb buffers at the start of a shared-memory block.
__device__ inline Ring ring_at(unsigned char* smem, int nb) {
  return Ring{smem, reinterpret_cast<uint64_t*>(smem + (size_t)nb * CHB), 0, nb};
}

__device__ inline void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Initialise the ring's barriers (all threads call; ends with a barrier).
__device__ inline void ring_init(Ring& r) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < r.nb; ++s) {
      mbar_init(&r.bar[s], 1);
      mbar_init(&r.bar[r.nb + s], blockDim.x / 32);
    }
    fence_barrier_init();
  }
  r.base = 0;
  __syncthreads();
}

// Streams nchunks chunks: src(c, &ptr, &bytes) describes chunk c (ptr
// 16-byte aligned, bytes > 0), use(c, smem) consumes it with every thread of
// the CTA (use may contain block-wide barriers; every thread calls it for
// every chunk).  Ends with a barrier.
template <typename Src, typename Use>
__device__ void ring_run(Ring& r, int nchunks, Src src, Use use, int* err) {
  const int first = r.base, nb = r.nb;
  uint64_t* full = r.bar;
  uint64_t* empty = r.bar + nb;
  // the producer fills chunk g into slot g % nb once the chunk that last
  // used the slot (g - nb) has been read by every warp
  auto issue = [&](int c) {
    const void* p;
    unsigned bytes;
    src(c, p, bytes);
    const int g = first + c, slot = g % nb;
    if (g >= nb) mbar_wait_bounded(&empty[slot], (unsigned)(((g / nb) - 1) & 1), err);
    fence_proxy_async();
    bulk_load(r.buf + (size_t)slot * CHB, p, (bytes + 15u) & ~15u, &full[slot]);
  };
  if (threadIdx.x == 0)
    for (int c = 0; c < nchunks && c < nb; ++c) issue(c);
  for (int c = 0; c < nchunks; ++c) {
    const int g = first + c, slot = g % nb;
    mbar_wait_bounded(&full[slot], (unsigned)((g / nb) & 1), err);
    use(c, r.buf + (size_t)slot * CHB);
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(&empty[slot]);
    if (threadIdx.x == 0 && c + nb < nchunks) issue(c + nb);
  }
  r.base = first + nchunks;
  __syncthreads();
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
