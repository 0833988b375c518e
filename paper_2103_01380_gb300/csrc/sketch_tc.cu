// sketch_tc.cu -- Gaussian sketch Y = Omega A (Section 2, random projection
// B = Omega A) on the 5th-generation tensor cores of sm_103a.
//
// The contraction is computed transposed, Y^T = A^T Omega^T:
//   MMA M = 128 window columns (snapshots), N = l_pad (rows of Omega),
//   K = rows of A, 32 rows (one 128-byte swizzle row of FP32) per chunk.
// A's columns are contiguous in rows, so a [32 rows x 64 columns] box loaded
// by TMA with 128-byte swizzling is half of the K-major canonical tile the MMA
// reads (a 32- or 16-column box a quarter or an eighth of it, when the plan is
// tuned to narrower slices).  Omega does not depend on the subdomain, so one
// chunk of rows serves a whole pack: up to 512 columns of such boxes (slices of
// subdomains with equal shape) stacked into 4 MMA tiles.  Omega(:, rows) is regenerated from Philox each
// chunk by the generator warps directly into the same swizzled K-major layout;
// the accumulators live in TMEM.
//
// Warp roles (320 threads):
//   warp 0      TMA producer (one elected lane)
//   warp 1      TMEM allocator + MMA issuer (one elected lane)
//   warps 2..9  Omega generators, then the TMEM -> partial-slot epilogue
//               (warp w reads TMEM lanes 32 (w % 4) .. +31; the two warps of a
//               quadrant take alternate 16-column slices)
// Every mbarrier wait is bounded (kWaitLimitNs); on timeout the CTA records
// kStatusTimeout, drains its own copies and MMAs (again bounded), frees TMEM
// and returns.
#include <cuda.h>

#include "sketch_pack.cuh"
#include "spid_internal.cuh"
#include "tcgen05_ptx.cuh"

namespace spid {

namespace {

using namespace tc;

// Omega generation is a chain of Philox rounds and MUFU calls; two generator
// warps per SM sub-partition keep it ahead of HBM even at l = 42.
constexpr int kGenWarps = 8;
constexpr int kGenThreads = 32 * kGenWarps;
constexpr int kTcThreads = 64 + kGenThreads;
constexpr int kTileCols = 128;                 // MMA M
constexpr int kTileBytes = kTileCols * 128;    // 128 columns x 32 FP32 rows
constexpr int kMaxStages = 8;

struct TcArgs {
  SketchArgs s;
  int32_t stages;      // pipeline depth
  int32_t max_tiles;   // MMA tiles per pack (<= 4)
  int32_t acc_stride;  // TMEM columns per tile accumulator (multiple of 32 >= l_pad)
  int32_t tmem_cols;   // power of two >= max_tiles * acc_stride
};

__global__ void __launch_bounds__(kTcThreads, 1) sketch_tf32_kernel(const TcArgs args) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ int epi_last[kMaxPackMembers];
  // 1024-byte alignment for the 128-byte swizzle atoms
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const SketchArgs& a = args.s;
  const int S = args.stages;
  const int l_pad = a.l_pad;
  const int omega_bytes = l_pad * 128;
  unsigned char* smem_A = smem;                                        // S x max_tiles x 16 KB
  unsigned char* smem_O = smem_A + (size_t)S * args.max_tiles * kTileBytes;  // S x l_pad x 128 B
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_O + (size_t)S * omega_bytes);
  uint64_t* full = bars;                       // [S] TMA bytes landed
  uint64_t* empty = bars + kMaxStages;         // [S] MMAs that read the stage completed
  uint64_t* ofull = bars + 2 * kMaxStages;     // [S] Omega written (kGenThreads arrivals)
  uint64_t* accum = bars + 3 * kMaxStages;     // accumulators of a segment complete
  uint64_t* drain = bars + 3 * kMaxStages + 1; // every issued MMA complete
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * kMaxStages + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  const int cta = blockIdx.x + a.cta_base;
  const int seg0 = a.seg_ptr[cta], seg1 = a.seg_ptr[cta + 1];

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_addr(&full[s]), 1);
      mbar_init(smem_addr(&empty[s]), 1);
      mbar_init(smem_addr(&ofull[s]), kGenThreads);
    }
    mbar_init(smem_addr(accum), 1);
    mbar_init(smem_addr(drain), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tmem_slot)),
                 "r"(args.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    // Lane h holds slice h of the current pack (its map and box origin) in
    // registers for the whole segment and issues that slice's box each chunk;
    // lane 0 waits for the stage and arms its barrier first.  A pack has at
    // most 32 slices (512 columns of slices at least 16 wide).
    int it = 0;
    bool ok = true;
    const CUtensorMap* tmaps = static_cast<const CUtensorMap*>(a.tmaps);
    const int slice_bytes = a.slice_cols * 128;   // one box: slice_cols columns x 32 rows
    for (int si = seg0; si < seg1 && ok; ++si) {
      const PackSegment sg = a.psegs[si];
      const Pack pk = a.packs[sg.pack];
      const bool mine = lane < pk.nslices;
      Slice sl{};
      if (mine) sl = a.slices[pk.slice0 + lane];
      for (int ch = sg.chunk0; ch < sg.chunk1; ++ch, ++it) {
        const int st = it % S;
        const uint32_t ph = (uint32_t)(it / S) & 1u;
        const uint32_t fb = smem_addr(&full[st]);
        if (lane == 0) {
          ok = mbar_wait(smem_addr(&empty[st]), ph ^ 1u, abort_flag, a.status);
          if (ok) mbar_arrive_expect_tx(fb, (uint32_t)(pk.nslices * slice_bytes));
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
        // the boxes of a pack's slices sit back to back, so a tile of 128
        // columns is 128 / slice_cols boxes
        unsigned char* dst = smem_A + (size_t)st * args.max_tiles * kTileBytes;
        const ChunkCoord cc = chunk_coord(pk, ch);
        if (mine) tma_load_chunk(smem_addr(dst + lane * slice_bytes), tmaps, pk, cc, sl, fb);
      }
    }
    // Drain: every issued stage's bytes must have landed before the CTA exits.
    if (lane == 0) {
      const int first = it - S > 0 ? it - S : 0;
      for (int j = first; j < it; ++j)
        mbar_wait(smem_addr(&full[j % S]), (uint32_t)(j / S) & 1u, abort_flag, a.status, false);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int it = 0;
      bool ok = true, issued = false;
      const uint32_t idesc = tf32_idesc(kTileCols, l_pad);
      for (int si = seg0; si < seg1 && ok; ++si) {
        const PackSegment sg = a.psegs[si];
        const int nt = (a.packs[sg.pack].nslices * a.slice_cols + kTileCols - 1) / kTileCols;
        for (int ch = sg.chunk0; ch < sg.chunk1; ++ch, ++it) {
          const int st = it % S;
          const uint32_t ph = (uint32_t)(it / S) & 1u;
          if (!mbar_wait(smem_addr(&full[st]), ph, abort_flag, a.status)) { ok = false; break; }
          if (!mbar_wait(smem_addr(&ofull[st]), ph, abort_flag, a.status)) { ok = false; break; }
          tc_fence_after();
          const uint32_t a0 = smem_addr(smem_A + (size_t)st * args.max_tiles * kTileBytes);
          const uint32_t b0 = smem_addr(smem_O + (size_t)st * omega_bytes);
          for (int t = 0; t < nt; ++t) {
            const uint64_t ad = sw128_kmajor_desc(a0 + t * kTileBytes);
            const uint64_t bd = sw128_kmajor_desc(b0);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)   // K = 8 TF32 (32 bytes) per MMA
              umma_tf32(tmem_base + (uint32_t)(t * args.acc_stride), ad + 2 * kk, bd + 2 * kk,
                        idesc, (ch > sg.chunk0 || kk > 0) ? 1u : 0u);
          }
          issued = true;
          umma_commit(smem_addr(&empty[st]));
          if (ch == sg.chunk1 - 1) umma_commit(smem_addr(accum));
        }
      }
      // Every issued MMA must be complete before TMEM is released.
      if (issued) {
        umma_commit(smem_addr(drain));
        mbar_wait(smem_addr(drain), 0u, abort_flag, a.status, false);
      }
    }
  } else {
    // ------------------------------------------------ Omega generators + epilogue
    const int gtid = threadIdx.x - 64;            // 0 .. kGenThreads-1
    const int quad = warp & 3;                    // TMEM lane quadrant of this warp
    const int part = (warp - 2) / 4;              // warps sharing a quadrant split the columns
    const uint2 key = philox_key(a.seed);
    const int groups = l_pad / 4;
    int it = 0, segi = 0;
    bool ok = true;
    // The generator/epilogue warps share named barriers, so their control flow
    // stays uniform for the whole schedule: a wait that gives up only clears
    // `ok`, which switches off the work (and further waits) behind it.
    auto epilogue = [&](int si_done, int seg_index) {
      if (ok) ok = mbar_wait(smem_addr(accum), (uint32_t)seg_index & 1u, abort_flag, a.status);
      ok = __all_sync(0xffffffffu, ok);
      tc_fence_after();
      pack_epilogue(a, a.psegs[si_done], tmem_base, args.acc_stride, quad, part, kGenWarps / 4,
                    lane, gtid, kGenThreads, epi_last, 1, ok);
    };
    for (int si = seg0; si < seg1; ++si, ++segi) {
      const PackSegment sg = a.psegs[si];
      if (si > seg0) epilogue(si - 1, segi - 1);
      const int m = a.packs[sg.pack].m;
      for (int ch = sg.chunk0; ch < sg.chunk1; ++ch, ++it) {
        const int st = it % S;
        const uint32_t ph = (uint32_t)(it / S) & 1u;
        if (ok) ok = mbar_wait(smem_addr(&empty[st]), ph ^ 1u, abort_flag, a.status);
        if (!ok) continue;
        unsigned char* ob = smem_O + (size_t)st * omega_bytes;
        const int r0 = ch * kChunkRows;
        for (int task = gtid; task < kChunkRows * groups; task += kGenThreads) {
          const int k = task % kChunkRows, g = task / kChunkRows;
          float w[4] = {0.f, 0.f, 0.f, 0.f};
          if (4 * g < a.l && r0 + k < m) {
            omega_group<float>(key, (uint32_t)(r0 + k), (uint32_t)g, w);
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (4 * g + u >= a.l) w[u] = 0.f;
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int i = 4 * g + u;   // row of Omega = MMA N index
            const uint32_t off = (uint32_t)((i >> 3) * 1024 + (i & 7) * 128 +
                                            ((((k >> 2) ^ (i & 7))) << 4) + ((k & 3) << 2));
            *reinterpret_cast<float*>(ob + off) = w[u];
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(smem_addr(&ofull[st]));
      }
    }
    if (seg1 > seg0) epilogue(seg1 - 1, segi - 1);
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(args.tmem_cols)
                 : "memory");
  }
}

}  // namespace

int sketch_tc_group_cols() { return kPackSlices * kSliceCols; }

// Dynamic shared memory the TF32 sketch needs for a pipeline of `stages`.
size_t sketch_tc_smem_bytes(int stages, int max_tiles, int l_pad) {
  return 1024 + (size_t)stages * ((size_t)max_tiles * kTileBytes + (size_t)l_pad * 128) +
         (3 * kMaxStages + 2) * sizeof(uint64_t) + 16;
}

int sketch_tc_max_stages() { return kMaxStages; }

cudaError_t launch_sketch_tc(const SketchArgs& s, int grid, int stages, int max_tiles,
                             cudaStream_t st) {
  if (grid <= 0) return cudaSuccess;
  TcArgs a;
  a.s = s;
  a.stages = stages;
  a.max_tiles = max_tiles;
  a.acc_stride = (s.l_pad + 31) / 32 * 32;
  int need = max_tiles * a.acc_stride;
  int cols = 32;
  while (cols < need) cols *= 2;
  a.tmem_cols = cols;
  if (cols > 512 || stages < 1 || stages > kMaxStages || max_tiles < 1 || max_tiles > 4)
    return cudaErrorInvalidValue;
  const size_t smem = sketch_tc_smem_bytes(stages, max_tiles, s.l_pad);
  cudaError_t e = cudaFuncSetAttribute(sketch_tf32_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  sketch_tf32_kernel<<<grid, kTcThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace spid
