// tcgen05_ptx.cuh -- inline-PTX wrappers for the sm_100-family async machinery
// the tensor-core sketch kernels use: mbarriers (with bounded waits), TMA tile
// loads, UMMA shared-memory and instruction descriptors, tcgen05.mma /
// commit / fences, TMEM loads, named barriers.
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "spid_internal.cuh"

namespace spid {
namespace tc {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity; false on timeout or abort.
__device__ __noinline__ inline bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                       int* status, bool honour_abort = true) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 127u) == 0) {
      if (honour_abort && *abort_flag) return false;
      if (globaltimer_ns() - t0 > kWaitLimitNs) {
        *abort_flag = 1;
        raise_status(status, kStatusTimeout);
        return false;
      }
    }
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const void* tmap, int c0, int c1, int c2,
                                            int c3, int c4, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
      : "memory");
}

// Load the [64 columns][32 rows] tile of chunk `ch` of a slice: a 2-D map over
// contiguous rows, or (pk.ex > 0) a 5-D map over a box of a global field whose
// 32-row chunks are runs along x (ex a multiple of 32, so x is 16-byte
// aligned).  The chunk's (x, y, z, q) is decoded once per chunk by the caller.
struct ChunkCoord {
  int x, y, z, q;
};

__device__ __forceinline__ ChunkCoord chunk_coord(const Pack& pk, int ch) {
  ChunkCoord c{ch * kChunkRows, 0, 0, 0};
  if (pk.ex > 0) {
    const int t = c.x / pk.ex;
    c.x -= t * pk.ex;
    c.y = t % pk.ey;
    const int t2 = t / pk.ey;
    c.z = t2 % pk.ez;
    c.q = t2 / pk.ez;
  }
  return c;
}

__device__ __forceinline__ void tma_load_chunk(uint32_t dst, const CUtensorMap* tmaps, const Pack& pk,
                                               const ChunkCoord& c, const Slice& sl, uint32_t bar) {
  const void* tm = tmaps + sl.map;
  if (pk.ex > 0) tma_load_5d(dst, tm, sl.tx + c.x, sl.ty + c.y, sl.tz + c.z, sl.tq + c.q, sl.col0, bar);
  else tma_load_2d(dst, tm, sl.tx + c.x, sl.ty + sl.col0, bar);
}

// K-major operand, 128-byte swizzle: 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_kmajor_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu)       // start address
         | ((uint64_t)1 << 16)                    // leading byte offset (unused when swizzled)
         | ((uint64_t)(1024 >> 4) << 32)          // stride byte offset
         | ((uint64_t)1 << 46)                    // descriptor version
         | ((uint64_t)2 << 61);                   // SWIZZLE_128B
}

// Instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major.
__device__ __forceinline__ uint32_t tf32_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32"
      " {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// Barrier among `count` threads (whole warps) on hardware barrier `id` (0 is
// __syncthreads).
__device__ __forceinline__ void named_bar_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}


// K-major operand, 64-byte swizzle: 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t sw64_kmajor_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu)       // start address
         | ((uint64_t)1 << 16)                    // leading byte offset (unused when swizzled)
         | ((uint64_t)(512 >> 4) << 32)           // stride byte offset
         | ((uint64_t)1 << 46)                    // descriptor version
         | ((uint64_t)4 << 61);                   // SWIZZLE_64B
}

// Instruction descriptor: kind::f16 with A = B = BF16, D = F32, both K-major.
__device__ __forceinline__ uint32_t bf16_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

}  // namespace tc
}  // namespace spid
