// sketch_bf16.cu -- Gaussian sketch Y = Omega A (Section 2, random projection
// B = Omega A) on the tensor cores in BF16 with FP32 accumulation.
//
// Same decomposition and packed schedule as the TF32 kernel (Y^T = A^T
// Omega^T, M = 128 window columns = two 64-column slices, N = l_pad, K = 32
// rows of A per chunk, up to 4 tiles per pack, accumulators in TMEM), with one
// more warp group: the FP32 tiles that TMA lands (128-byte swizzle) are
// converted IN PLACE into BF16 K-major tiles with a 64-byte swizzle -- the
// 16 KB FP32 tile becomes an 8 KB BF16 tile, or, in the split form, an 8 KB
// "hi" tile bf16(a) followed by an 8 KB "lo" tile bf16(a - hi).
//   * BF16:   Y ~ bf16(Omega) bf16(A)                    (8-bit significands)
//   * 3xBF16: Y ~ Oh Ah + Oh Al + Ol Ah, with Ah + Al and Oh + Ol the two-term
//             BF16 splits of A and Omega (about 16-bit significands), three
//             MMAs per K-step; the tensor pipe has the headroom (the sketch
//             is HBM-bound at 2 l flop per 4 bytes).
//
// Warp roles (448 threads):
//   warp 0       TMA producer            warp 1      TMEM allocator + MMA issuer
//   warps 2..9   Omega generators, then the TMEM -> partial-slot epilogue
//   warps 10..13 FP32 -> BF16 converters (thread c owns row c of each tile)
// Every mbarrier wait is bounded; see the TF32 kernel for the abort protocol.
#include <cuda.h>
#include <cuda_bf16.h>

#include "sketch_pack.cuh"
#include "spid_internal.cuh"
#include "tcgen05_ptx.cuh"

namespace spid {

namespace {

using namespace tc;

constexpr int kGenWarps = 8;
constexpr int kGenThreads = 32 * kGenWarps;
constexpr int kConvBase = 64 + kGenThreads;       // first converter thread
constexpr int kThreads = kConvBase + 128;
constexpr int kTileCols = 128;
constexpr int kTileBytes = kTileCols * 128;      // FP32 tile: 128 columns x 32 rows
constexpr int kBf16TileBytes = kTileCols * 64;   // BF16 tile: 128 columns x 32 rows
constexpr int kSliceBytes = kSliceCols * 128;    // FP32 slice: 64 columns x 32 rows (one TMA box)
constexpr int kMaxStages = 8;

struct Bf16Args {
  SketchArgs s;
  int32_t stages;
  int32_t max_tiles;
  int32_t acc_stride;
  int32_t tmem_cols;
};

// byte offset of element (row, k) of a K-major BF16 operand, 64-byte swizzle
__device__ __forceinline__ uint32_t sw64_offset(int row, int k) {
  return (uint32_t)((row >> 3) * 512 + (row & 7) * 64 +
                    ((((k >> 3) ^ ((row >> 1) & 3))) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo_elem, float hi_elem) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo_elem, hi_elem);   // .x at the lower address
  return *reinterpret_cast<const uint32_t*>(&v);
}

template <bool SPLIT>
__global__ void __launch_bounds__(kThreads, 1) sketch_bf16_kernel(const Bf16Args args) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ int epi_last[kMaxPackMembers];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const SketchArgs& a = args.s;
  const int S = args.stages;
  const int l_pad = a.l_pad;
  const int omega_bytes = l_pad * 64 * (SPLIT ? 2 : 1);   // hi (+ lo) BF16 Omega tiles
  unsigned char* smem_A = smem;                                              // S x tiles x 16 KB
  unsigned char* smem_O = smem_A + (size_t)S * args.max_tiles * kTileBytes;  // S x omega_bytes
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_O + (size_t)S * omega_bytes);
  uint64_t* full = bars;                         // [S] TMA bytes landed
  uint64_t* empty = bars + kMaxStages;           // [S] MMAs that read the stage completed
  uint64_t* ofull = bars + 2 * kMaxStages;       // [S] Omega written (128 arrivals)
  uint64_t* cfull = bars + 3 * kMaxStages;       // [S] A converted (128 arrivals)
  uint64_t* accum = bars + 4 * kMaxStages;
  uint64_t* drain = bars + 4 * kMaxStages + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 4 * kMaxStages + 2);
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
      mbar_init(smem_addr(&cfull[s]), 128);
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
    // Lane h holds slice h of the current pack in registers for the whole
    // segment and issues its box each chunk; lane 0 waits for the stage and
    // arms its barrier first.
    int it = 0;
    bool ok = true;
    const CUtensorMap* tmaps = static_cast<const CUtensorMap*>(a.tmaps);
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
          if (ok) mbar_arrive_expect_tx(fb, (uint32_t)(pk.nslices * kSliceBytes));
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
        unsigned char* dst = smem_A + (size_t)st * args.max_tiles * kTileBytes;
        const ChunkCoord cc = chunk_coord(pk, ch);
        if (mine) tma_load_chunk(smem_addr(dst + lane * kSliceBytes), tmaps, pk, cc, sl, fb);
      }
    }
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
      const uint32_t idesc = bf16_idesc(kTileCols, l_pad);
      for (int si = seg0; si < seg1 && ok; ++si) {
        const PackSegment seg = a.psegs[si];
        const int nt = (a.packs[seg.pack].nslices + 1) / 2;
        for (int ch = seg.chunk0; ch < seg.chunk1; ++ch, ++it) {
          const int st = it % S;
          const uint32_t ph = (uint32_t)(it / S) & 1u;
          if (!mbar_wait(smem_addr(&cfull[st]), ph, abort_flag, a.status)) { ok = false; break; }
          if (!mbar_wait(smem_addr(&ofull[st]), ph, abort_flag, a.status)) { ok = false; break; }
          tc_fence_after();
          const uint32_t a0 = smem_addr(smem_A + (size_t)st * args.max_tiles * kTileBytes);
          const uint32_t o0 = smem_addr(smem_O + (size_t)st * omega_bytes);
          const uint64_t oh = sw64_kmajor_desc(o0);
          const uint64_t ol = sw64_kmajor_desc(o0 + l_pad * 64);
          for (int t = 0; t < nt; ++t) {
            const uint64_t ah = sw64_kmajor_desc(a0 + t * kTileBytes);
            const uint64_t al = sw64_kmajor_desc(a0 + t * kTileBytes + kBf16TileBytes);
            const uint32_t d = tmem_base + (uint32_t)(t * args.acc_stride);
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {   // K = 16 BF16 (32 bytes) per MMA
              umma_bf16(d, ah + 2 * kk, oh + 2 * kk, idesc, (ch > seg.chunk0 || kk > 0) ? 1u : 0u);
              if (SPLIT) {
                umma_bf16(d, al + 2 * kk, oh + 2 * kk, idesc, 1u);
                umma_bf16(d, ah + 2 * kk, ol + 2 * kk, idesc, 1u);
              }
            }
          }
          issued = true;
          umma_commit(smem_addr(&empty[st]));
          if (ch == seg.chunk1 - 1) umma_commit(smem_addr(accum));
        }
      }
      if (issued) {
        umma_commit(smem_addr(drain));
        mbar_wait(smem_addr(drain), 0u, abort_flag, a.status, false);
      }
    }
  } else if (threadIdx.x >= kConvBase) {
    // ------------------------------------------------ FP32 -> BF16 converters
    const int row = threadIdx.x - kConvBase;       // 0..127: row (window column) of the tile
    int it = 0;
    bool ok = true;
    // the converters share named barrier 2: uniform control flow, `ok` only
    // switches off the work behind a wait that gave up
    for (int si = seg0; si < seg1; ++si) {
      const PackSegment seg = a.psegs[si];
      const int nt = (a.packs[seg.pack].nslices + 1) / 2;
      for (int ch = seg.chunk0; ch < seg.chunk1; ++ch, ++it) {
        const int st = it % S;
        const uint32_t ph = (uint32_t)(it / S) & 1u;
        if (ok) ok = mbar_wait(smem_addr(&full[st]), ph, abort_flag, a.status);
        for (int t = 0; t < nt; ++t) {
          unsigned char* tile = smem_A + ((size_t)st * args.max_tiles + t) * kTileBytes;
          // read this row's 32 FP32 values (128-byte swizzle) ...
          float x[32];
          const unsigned char* rowp = tile + (row >> 3) * 1024 + (row & 7) * 128;
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const float4 v = ok ? *reinterpret_cast<const float4*>(rowp + ((c ^ (row & 7)) << 4))
                                : make_float4(0.f, 0.f, 0.f, 0.f);
            x[4 * c] = v.x; x[4 * c + 1] = v.y; x[4 * c + 2] = v.z; x[4 * c + 3] = v.w;
          }
          named_bar_sync(2, 128);   // every row read before any BF16 byte overwrites it
          if (!ok) continue;
          // ... and write it back as BF16 (64-byte swizzle), hi tile then lo tile
          unsigned char* hrow = tile + (row >> 3) * 512 + (row & 7) * 64;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            uint4 h, l;
            uint32_t* hp = reinterpret_cast<uint32_t*>(&h);
            uint32_t* lp = reinterpret_cast<uint32_t*>(&l);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float e0 = x[8 * c + 2 * q], e1 = x[8 * c + 2 * q + 1];
              hp[q] = pack_bf16x2(e0, e1);
              if (SPLIT) {
                const __nv_bfloat162 hv = *reinterpret_cast<const __nv_bfloat162*>(&hp[q]);
                lp[q] = pack_bf16x2(e0 - __bfloat162float(hv.x), e1 - __bfloat162float(hv.y));
              }
            }
            const uint32_t off = (uint32_t)((c ^ ((row >> 1) & 3)) << 4);
            *reinterpret_cast<uint4*>(hrow + off) = h;
            if (SPLIT) *reinterpret_cast<uint4*>(hrow + kBf16TileBytes + off) = l;
          }
        }
        if (!ok) continue;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(smem_addr(&cfull[st]));
      }
    }
  } else {
    // ------------------------------------------------ Omega generators + epilogue
    const int gtid = threadIdx.x - 64;            // 0 .. kGenThreads-1
    const int part = (warp - 2) / 4;              // warps sharing a quadrant split the columns
    constexpr int kParts = kGenWarps / 4;
    const int quad = warp & 3;
    const uint2 key = philox_key(a.seed);
    const int groups = l_pad / 4;
    int it = 0, segi = 0;
    bool ok = true;
    // uniform control flow across the group (named barrier 1), as in the TF32 kernel
    auto epilogue = [&](int si_done, int seg_index) {
      if (ok) ok = mbar_wait(smem_addr(accum), (uint32_t)seg_index & 1u, abort_flag, a.status);
      ok = __all_sync(0xffffffffu, ok);
      tc_fence_after();
      pack_epilogue(a, a.psegs[si_done], tmem_base, args.acc_stride, quad, part, kParts, lane,
                    gtid, kGenThreads, epi_last, 1, ok);
    };
    for (int si = seg0; si < seg1; ++si, ++segi) {
      const PackSegment seg = a.psegs[si];
      if (si > seg0) epilogue(si - 1, segi - 1);
      const Pack pb = a.packs[seg.pack];
      for (int ch = seg.chunk0; ch < seg.chunk1; ++ch, ++it) {
        const int st = it % S;
        const uint32_t ph = (uint32_t)(it / S) & 1u;
        if (ok) ok = mbar_wait(smem_addr(&empty[st]), ph ^ 1u, abort_flag, a.status);
        if (!ok) continue;
        unsigned char* ob = smem_O + (size_t)st * omega_bytes;
        const int r0 = ch * kChunkRows;
        // a task makes K-rows k and k + 1 (k even) of Omega rows 4g .. 4g+3:
        // each (row, k pair) is one 4-byte store of two adjacent BF16 values
        for (int task = gtid; task < (kChunkRows / 2) * groups; task += kGenThreads) {
          const int k = 2 * (task % (kChunkRows / 2)), g = task / (kChunkRows / 2);
          float w[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
          for (int h = 0; h < 2; ++h)
            if (4 * g < a.l && r0 + k + h < pb.m) {
              omega_group<float>(key, (uint32_t)(r0 + k + h), (uint32_t)g, w[h]);
#pragma unroll
              for (int u = 0; u < 4; ++u)
                if (4 * g + u >= a.l) w[h][u] = 0.f;
            }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int i = 4 * g + u;   // row of Omega = MMA N index
            const uint32_t off = sw64_offset(i, k);   // k even: 4-byte aligned, k + 1 next
            const uint32_t hp = pack_bf16x2(w[0][u], w[1][u]);
            *reinterpret_cast<uint32_t*>(ob + off) = hp;
            if (SPLIT) {
              const __nv_bfloat162 hv = *reinterpret_cast<const __nv_bfloat162*>(&hp);
              *reinterpret_cast<uint32_t*>(ob + l_pad * 64 + off) =
                  pack_bf16x2(w[0][u] - __bfloat162float(hv.x), w[1][u] - __bfloat162float(hv.y));
            }
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

size_t sketch_bf16_smem_bytes(int stages, int max_tiles, int l_pad, bool split) {
  return 1024 + (size_t)stages * ((size_t)max_tiles * kTileBytes +
                                  (size_t)l_pad * 64 * (split ? 2 : 1)) +
         (4 * kMaxStages + 2) * sizeof(uint64_t) + 16;
}

cudaError_t launch_sketch_bf16(const SketchArgs& s, int grid, int stages, int max_tiles, bool split,
                               cudaStream_t st) {
  if (grid <= 0) return cudaSuccess;
  Bf16Args a;
  a.s = s;
  a.stages = stages;
  a.max_tiles = max_tiles;
  a.acc_stride = (s.l_pad + 31) / 32 * 32;
  const int need = max_tiles * a.acc_stride;
  int cols = 32;
  while (cols < need) cols *= 2;
  a.tmem_cols = cols;
  if (cols > 512 || stages < 1 || stages > kMaxStages || max_tiles < 1 || max_tiles > 4)
    return cudaErrorInvalidValue;
  const size_t smem = sketch_bf16_smem_bytes(stages, max_tiles, s.l_pad, split);
  cudaError_t e;
  if (split) {
    e = cudaFuncSetAttribute(sketch_bf16_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    sketch_bf16_kernel<true><<<grid, kThreads, smem, st>>>(a);
  } else {
    e = cudaFuncSetAttribute(sketch_bf16_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    sketch_bf16_kernel<false><<<grid, kThreads, smem, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace spid
