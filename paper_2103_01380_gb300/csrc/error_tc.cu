// error_tc.cu -- reconstruction A_hat = A(:,J) C (Section 2, column ID form of
// Algorithm 2) fused with the relative Frobenius error of Section 5.1, with the
// rank-k product on the 5th-generation tensor cores.
//
// The CUDA-core pass spends k FMAs per element of A, which at k >= 8 is more
// FP32 issue than the SM has per byte of HBM.  Here a 128-row tile of A_hat
// is one MMA, D[128 x N] = A(rows, J) C(:, cols), with K = k <= 32 and
// N <= 256 columns; the CUDA cores only stream A once and form
// (A - D)^2 and A^2.  FP32 accuracy is kept with a three-term TF32 split:
// x = hi + lo with hi = tf32(x) and lo = x - hi exact in FP32, and
//   D = AJhi Chi + AJhi Clo + AJlo Chi
// (the dropped AJlo Clo and the TF32 rounding of the lo terms are ~2^-21 of
// |AJ||C|), accumulated in FP32 in TMEM.
//
// Thread roles (512 threads = 16 warps, one CTA per SM):
//   all warps    stage C (once per segment) and A(rows, J) (once per tile) into
//                shared memory as hi/lo K-major tiles (128-byte swizzle); after
//                a named barrier thread 0 issues the tile's MMAs into one of
//                two TMEM accumulators (2 x 256 columns, allocated by warp 0);
//                meanwhile every warp drains the previous tile: warp w reads
//                TMEM lanes 32 (w % 4) .. +31 (= rows) and every fourth
//                16-column slice, loads the matching A(row, col) (a coalesced
//                128-byte line per warp per column) and accumulates Kahan sums
//                of e^2 and a^2.
// No separate MMA warp: 17 warps would cap every thread at 96 registers.
// Control flow is uniform across the CTA for the whole schedule: a bounded
// wait that gives up only switches off the work behind it, so every named
// barrier is still reached by every thread.
#include <cuda.h>

#include "error_fold.cuh"
#include "spid_internal.cuh"
#include "tcgen05_ptx.cuh"

namespace spid {

namespace {

using namespace tc;

constexpr int kEpiWarps = 16;
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kThreads = kEpiThreads;
constexpr int kParts = kEpiWarps / 4;                 // warps per TMEM lane quadrant
constexpr int kAjBytes = kErrTcRows * 128;            // 128 rows x 32 TF32 (K-major, SW128)
constexpr int kCBytes = kErrTcCols * 128;             // 256 columns x 32 TF32
constexpr int kChunksPerWarp = kErrTcCols / 16 / kParts;   // 16-column slices per warp per tile
constexpr int kTmemCols = 2 * kErrTcCols;

struct Smem {
  // operand tiles first (1024-byte aligned offsets)
  static constexpr int ch = 0;
  static constexpr int cl = ch + kCBytes;
  static constexpr int aj = cl + kCBytes;            // [2 buffers][hi, lo]
  static constexpr int bars = aj + 4 * kAjBytes;
  static constexpr int total = bars + 4 * 8 + 16;
};

__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// byte offset of element (row, k) of a K-major TF32 operand, 128-byte swizzle
__device__ __forceinline__ uint32_t sw128_offset(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((((k >> 2) ^ (row & 7))) << 4) +
                    ((k & 3) << 2));
}

__device__ __forceinline__ void put_split(unsigned char* hi_tile, unsigned char* lo_tile,
                                          uint32_t off, float x) {
  const float h = tf32_hi(x);
  *reinterpret_cast<float*>(hi_tile + off) = h;
  *reinterpret_cast<float*>(lo_tile + off) = x - h;
}

__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

template <bool WRITE>
__global__ void __launch_bounds__(kThreads, 1) error_tc_kernel(const ErrTcArgs args) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ double red[2][kEpiWarps];
  __shared__ int last_sub;
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const ErrArgs& a = args.e;
  unsigned char* Ch = smem + Smem::ch;
  unsigned char* Cl = smem + Smem::cl;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Smem::bars);
  uint64_t* acc_full = bars;         // [2] D complete (MMA commit)
  uint64_t* drain = bars + 2;        // every issued MMA complete
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  const int gtid = threadIdx.x;
  const int quad = warp & 3;
  const int part = warp >> 2;
  const int seg0 = args.seg_ptr[blockIdx.x], seg1 = args.seg_ptr[blockIdx.x + 1];

  if (threadIdx.x == 0) {
    mbar_init(smem_addr(&acc_full[0]), 1);
    mbar_init(smem_addr(&acc_full[1]), 1);
    mbar_init(smem_addr(drain), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  bool ok = true, issued = false;
  float se = 0.f, ce = 0.f, sa = 0.f, ca = 0.f;   // Kahan sums of e^2 and a^2
  int it = 0;
  for (int si = seg0; si < seg1; ++si) {
    const ErrSeg sg = args.segs[si];
    const int s = sg.sub;
    const int m = a.m[s], n = a.n[s];
    const int kk = a.k[s];
    const int kq = (kk + 7) / 8 * 8;                  // K entries the MMAs read
    const int N = (sg.ncols + 15) / 16 * 16;
    const float* A = static_cast<const float*>(a.window) + a.off[s];
    float* out = WRITE ? static_cast<float*>(a.out) + a.off[s] : nullptr;
    const int64_t ld = a.ld[s];
    const int32_t* Jg = a.J + (int64_t)s * a.k_max;
    // C(:, col0 .. col0 + N) -> Chi / Clo, row = column of A_hat, k = p.  The
    // MMAs of the previous segment are complete: this thread waited for the
    // last of them before draining its D.
    if (ok) {
      const float* Cg = static_cast<const float*>(a.C) + a.coff[s];
      for (int e = gtid; e < N * kq; e += kEpiThreads) {
        const int c = e % N, p = e / N;
        const float x = (p < kk && c < sg.ncols) ? Cg[(int64_t)p * n + sg.col0 + c] : 0.f;
        put_split(Ch, Cl, sw128_offset(c, p), x);
      }
    }
    float av[kChunksPerWarp][16];
    int prev_row0 = 0;
    for (int t = sg.tile0; t <= sg.tile1; ++t, ++it) {
      const bool stage = t < sg.tile1;       // tile t: stage A(rows, J), issue its MMAs
      const bool drain_prev = t > sg.tile0;  // tile t - 1: drain D
      const int pb = (it - 1) & 1;
      const uint32_t pph = (uint32_t)((it - 1) >> 1) & 1u;
      const int row = prev_row0 + quad * 32 + lane;
      const bool rv = row < m;
      // 1. A(row, cols) of tile t - 1, issued before the staging loads
      if (drain_prev && ok) {
#pragma unroll
        for (int j = 0; j < kChunksPerWarp; ++j) {
          const int c16 = 16 * (part + kParts * j);
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int c = c16 + i;
            av[j][i] = (rv && c < sg.ncols) ? __ldg(A + (int64_t)(sg.col0 + c) * ld + row) : 0.f;
          }
        }
      }
      if (stage) {
        // 2. A(rows of tile t, J) -> AJhi / AJlo buffer it & 1, last read by
        //    the MMAs of tile it - 2, which every thread saw complete
        const int b = it & 1;
        const int r0 = t * kErrTcRows;
        unsigned char* hi = smem + Smem::aj + (2 * b) * kAjBytes;
        unsigned char* lo = hi + kAjBytes;
        if (ok) {
          for (int e = gtid; e < kErrTcRows * kq; e += kEpiThreads) {
            const int r = e % kErrTcRows, p = e / kErrTcRows;
            const float x = (p < kk && r0 + r < m) ? __ldg(A + (int64_t)Jg[p] * ld + r0 + r) : 0.f;
            put_split(hi, lo, sw128_offset(r, p), x);
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        // 3. every operand written, and TMEM buffer b drained (tile it - 2)
        tc_fence_before();
        named_bar_sync(1, kEpiThreads);
        if (gtid == 0 && ok) {
          tc_fence_after();
          const uint32_t idesc = tf32_idesc(kErrTcRows, N);
          const uint32_t d = tmem_base + (uint32_t)(b * kErrTcCols);
          const uint64_t ah = sw128_kmajor_desc(smem_addr(hi));
          const uint64_t al = sw128_kmajor_desc(smem_addr(lo));
          const uint64_t bh = sw128_kmajor_desc(smem_addr(Ch));
          const uint64_t bl = sw128_kmajor_desc(smem_addr(Cl));
          for (int ks = 0; ks < kq / 8; ++ks) {   // K = 8 TF32 (32 bytes) per MMA
            umma_tf32(d, ah + 2 * ks, bh + 2 * ks, idesc, ks > 0 ? 1u : 0u);
            umma_tf32(d, ah + 2 * ks, bl + 2 * ks, idesc, 1u);
            umma_tf32(d, al + 2 * ks, bh + 2 * ks, idesc, 1u);
          }
          umma_commit(smem_addr(&acc_full[b]));
          issued = true;
        }
      }
      // 4. drain D of tile t - 1
      if (drain_prev) {
        if (ok) ok = mbar_wait(smem_addr(&acc_full[pb]), pph, abort_flag, args.status);
        ok = __all_sync(0xffffffffu, ok);
        tc_fence_after();
        if (ok) {
#pragma unroll
          for (int j = 0; j < kChunksPerWarp; ++j) {
            const int c16 = 16 * (part + kParts * j);
            if (c16 < N) {   // warp-uniform
              uint32_t r[16];
              tmem_ld16(tmem_base + ((uint32_t)(quad * 32) << 16) +
                            (uint32_t)(pb * kErrTcCols + c16), r);
              tmem_ld_wait();
              float le = 0.f, la = 0.f;
#pragma unroll
              for (int i = 0; i < 16; ++i) {
                const float dv = kk > 0 ? __uint_as_float(r[i]) : 0.f;
                const float x = av[j][i];
                const float df = x - dv;
                le = fmaf(df, df, le);
                la = fmaf(x, x, la);
                if (WRITE && rv && c16 + i < sg.ncols)
                  out[(int64_t)(sg.col0 + c16 + i) * ld + row] = dv;
              }
              kahan_add(se, ce, le);
              kahan_add(sa, ca, la);
            }
          }
        }
      }
      prev_row0 = t * kErrTcRows;
    }
    --it;   // the drain-only pass did not consume a tile
    // ---- segment partial: warp tree in FP32, FP64 across the warps
    float we = se - ce, wa = sa - ca;
    for (int o = 16; o > 0; o >>= 1) {
      we += __shfl_xor_sync(0xffffffffu, we, o);
      wa += __shfl_xor_sync(0xffffffffu, wa, o);
    }
    if (lane == 0) { red[0][warp] = (double)we; red[1][warp] = (double)wa; }
    se = ce = sa = ca = 0.f;
    named_bar_sync(1, kEpiThreads);
    if (gtid == 0) {
      int last = 0;
      if (ok && !*abort_flag) {
        double te = 0.0, ta = 0.0;
        for (int w = 0; w < kEpiWarps; ++w) { te += red[0][w]; ta += red[1][w]; }
        a.part[2 * (int64_t)si] = te;
        a.part[2 * (int64_t)si + 1] = ta;
        __threadfence();
        const int segs_s = a.unit_ptr[s + 1] - a.unit_ptr[s];
        last = (atomicAdd(&a.sub_cnt[s], 1) == segs_s - 1);
      }
      last_sub = last;
    }
    named_bar_sync(1, kEpiThreads);
    if (last_sub && warp == 0) error_fold_subdomain(a, s, lane);
  }
  // every issued MMA complete before TMEM is released
  if (gtid == 0 && issued) {
    umma_commit(smem_addr(drain));
    mbar_wait(smem_addr(drain), 0u, abort_flag, args.status, false);
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(kTmemCols)
                 : "memory");
  }
}

}  // namespace

size_t error_tc_smem_bytes() { return 1024 + (size_t)Smem::total; }

cudaError_t launch_error_tc(const ErrTcArgs& a, int grid, cudaStream_t st) {
  if (grid <= 0) return cudaSuccess;
  if (a.e.k_max > kErrTcKMax) return cudaErrorInvalidValue;
  const size_t smem = error_tc_smem_bytes();
  cudaError_t e;
  if (a.e.out) {
    e = cudaFuncSetAttribute(error_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    error_tc_kernel<true><<<grid, kThreads, smem, st>>>(a);
  } else {
    e = cudaFuncSetAttribute(error_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    error_tc_kernel<false><<<grid, kThreads, smem, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace spid
