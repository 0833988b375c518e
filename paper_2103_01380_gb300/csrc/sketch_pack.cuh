// sketch_pack.cuh -- the part of the tensor-core sketch kernels that depends on
// the packed schedule but not on the MMA format: draining a pack's
// accumulators from TMEM into its problems' partial slots, and the fixed-order
// fold done by the CTA that completes a problem.
#pragma once

#include "spid_internal.cuh"
#include "tcgen05_ptx.cuh"

namespace spid {
namespace tc {

// Accumulator layout: tile t (128 window columns) at TMEM columns
// t * acc_stride, row r of the tile = TMEM lane r; with slices of `slice_cols`
// columns (64, 32 or 16), row r of tile t is column (t 128 + r) % slice_cols
// of slice (t 128 + r) / slice_cols.
// Called by all `nthreads` epilogue threads (whole warps); warp w reads TMEM
// lanes 32 (w % 4) .. +31 and the warps sharing a quadrant (`part` of
// `nparts`) take alternate 16-column slices.  `ok` (uniform per warp) false:
// an earlier bounded wait gave up -- the thread still takes every barrier but
// reads, writes and counts nothing.
__device__ __forceinline__ void pack_epilogue(const SketchArgs& a, const PackSegment& sg,
                                              uint32_t tmem_base, int acc_stride, int quad,
                                              int part, int nparts, int lane, int gtid,
                                              int nthreads, int* last_flags, int barrier_id,
                                              bool ok) {
  const Pack pk = a.packs[sg.pack];
  const int l_pad = a.l_pad;
  const int sc = a.slice_cols;
  const int nt = (pk.nslices * sc + 127) / 128;
  float* partial = static_cast<float*>(a.partial);
  const int row = quad * 32 + lane;                 // TMEM lane = tile row
  for (int t = 0; t < nt && ok; ++t) {
    const int h = (t * 128 + row) / sc;
    const int jj = (t * 128 + row) % sc;
    bool valid = false;
    float* out = nullptr;
    if (h < pk.nslices) {
      const Slice sl = a.slices[pk.slice0 + h];
      if (jj < sl.ncols) {
        valid = true;
        out = partial + a.slot_off[sg.slot0 + sl.member] + (int64_t)(sl.out_col + jj) * l_pad;
      }
    }
    for (int c = 16 * part; c < l_pad; c += 16 * nparts) {
      uint32_t r[16];
      __syncwarp();
      tmem_ld16(tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(t * acc_stride + c), r);
      tmem_ld_wait();
      if (valid) {
        float4* dst = reinterpret_cast<float4*>(out + c);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          dst[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                               __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
      }
    }
  }
  tc_fence_before();
  // every member problem counts this segment; whoever completes it folds it
  __threadfence();
  named_bar_sync(barrier_id, nthreads);
  if (gtid < pk.nprob) {
    const int p = pk.prob0 + gtid;
    const int nslots = a.pslot_ptr[p + 1] - a.pslot_ptr[p];
    last_flags[gtid] = ok && (atomicAdd(&a.prob_cnt[p], 1) == nslots - 1);
  }
  named_bar_sync(barrier_id, nthreads);
  // the problems this segment completed are folded side by side: completed
  // problem j of c gets threads [ceil(j N / c), ceil((j + 1) N / c)) of the N,
  // so their slot loads are in flight together (each element still sums its
  // slots in schedule order)
  __shared__ int done_s[kMaxPackMembers + 1];
  if (gtid == 0) {
    int c = 0;
    for (int q = 0; q < pk.nprob; ++q)
      if (last_flags[q]) done_s[c++] = q;
    done_s[kMaxPackMembers] = c;
  }
  named_bar_sync(barrier_id, nthreads);
  const int c = done_s[kMaxPackMembers];
  if (c > 0) {
    __threadfence();
    const int j = gtid * c / nthreads;
    const int t0 = (j * nthreads + c - 1) / c, t1 = ((j + 1) * nthreads + c - 1) / c;
    reduce_problem_slots<float>(a, pk.prob0 + done_s[j], gtid - t0, t1 - t0);
    if (gtid < c) a.prob_cnt[pk.prob0 + done_s[gtid]] = 0;
  }
  named_bar_sync(barrier_id, nthreads);   // last_flags and done_s are reused by the next segment
}

}  // namespace tc
}  // namespace spid
