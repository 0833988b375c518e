// sketch_simt.cu -- Gaussian sketch Y = Omega A on the CUDA cores (FP64 and
// plain FP32 forms), Section 2 (random projection B = Omega A).
//
// Work decomposition (shared with the tensor-core kernel): the host splits
// every problem (subdomain x column group) into chunks of 32 rows and hands
// each CTA a contiguous, byte-balanced range of chunks ("segments").  A CTA
// keeps the whole column group's partial sketch in registers while it walks
// its rows, regenerating Omega(:, rows) once per chunk and reusing it for all
// columns of the group; at the end of a segment it writes its partial to a
// private slot, and the CTA that completes a problem (an atomic count after a
// device-wide fence) sums that problem's slots in schedule order into Y.
#include "spid_internal.cuh"

namespace spid {

namespace {

template <typename T> struct Vec;
template <> struct Vec<float> { using type = float4; static constexpr int width = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int width = 2; };

template <typename T>
__device__ __forceinline__ void store_vec(T* dst, const typename Vec<T>::type& v);
template <>
__device__ __forceinline__ void store_vec<float>(float* d, const float4& v) {
  *reinterpret_cast<float4*>(d) = v;
}
template <>
__device__ __forceinline__ void store_vec<double>(double* d, const double2& v) {
  *reinterpret_cast<double2*>(d) = v;
}

constexpr int kThreads = 256;
constexpr int kJGroups = 64;  // thread = (i-group in 0..3) x (j-group in 0..63)

// CTAs per SM that a thread's TI x TJ accumulators (in 32-bit registers) leave
// room for; the launch bounds cap registers to match.
constexpr int simt_min_blocks(int acc_regs) {
  return acc_regs <= 8 ? 4 : acc_regs <= 32 ? 3 : acc_regs <= 64 ? 2 : 1;
}

// TI: Omega rows per thread (l_pad = 4 TI); TJ: columns per thread (the
// column group holds up to 64 TJ columns).  A launch uses the smallest TJ that
// holds its widest problem, so narrow column ranges (micro-batches) do not pay
// for a 512-column register tile.
template <typename T, int TI, int TJ>
__global__ void __launch_bounds__(kThreads, simt_min_blocks(TI * TJ * (int)(sizeof(T) / 4)))
sketch_simt_kernel(SketchArgs args) {
  constexpr int LP = 4 * TI;
  constexpr int CG = kJGroups * TJ;
  constexpr int CGP = CG + 1;  // odd row stride: conflict-free transposed stores
  constexpr int VW = Vec<T>::width;
  constexpr int VPC = kChunkRows / VW;  // vectors per column per chunk
  using VT = typename Vec<T>::type;
  // vectors of A each thread stages per chunk; narrow tiles (at most 64 bytes of
  // them) load the next chunk into registers while the current one is computed
  constexpr int NV = (CG * VPC + kThreads - 1) / kThreads;
  constexpr bool kPrefetch = NV * (int)sizeof(VT) <= 64;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int last_flag;
  __shared__ int64_t roff_s[2][kChunkRows];   // boxes: element offsets of a chunk's rows
  T* As = reinterpret_cast<T*>(smem_raw);       // [kChunkRows][CGP]
  T* Om = As + kChunkRows * CGP;                // [kChunkRows][LP]
  // Om must be 16-byte aligned for vector loads
  Om = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(Om) + 15) & ~uintptr_t(15));

  const int tid = threadIdx.x;
  const int ig = tid / kJGroups;
  const int jg = tid % kJGroups;
  const int cta = blockIdx.x + args.cta_base;
  const uint2 key = philox_key(args.seed);
  const T* window = static_cast<const T*>(args.window);
  T* partial = static_cast<T*>(args.partial);
  const int l = args.l;

  const int s0 = args.seg_ptr[cta], s1 = args.seg_ptr[cta + 1];
  for (int si = s0; si < s1; ++si) {
    const Segment seg = args.segs[si];
    const Problem pb = args.probs[seg.prob];
    const T* A = window + pb.off + (int64_t)pb.col0 * pb.ld;
    const int nc = pb.ncols;
    const bool boxed = pb.geo.ex > 0;   // uniform over the CTA

    T acc[TJ][TI];
#pragma unroll
    for (int u = 0; u < TJ; ++u)
#pragma unroll
      for (int v = 0; v < TI; ++v) acc[u][v] = T(0);

    // a box of a global field: rows of one x-run (a multiple of VW long) are
    // contiguous, runs sit at the field's strides; table b holds a chunk's offsets
    auto table = [&](int ch, int b) {
      const int r = ch * kChunkRows + tid;
      if (boxed && tid < kChunkRows) roff_s[b][tid] = (r < pb.m) ? row_offset(pb.geo, r) : 0;
    };
    // A(rows of chunk ch, col group) into registers, 16-byte loads
    auto fetch = [&](int ch, int b, VT* buf) {
      const int r0 = ch * kChunkRows;
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const int v = tid + i * kThreads;
        if (v < nc * VPC) {
          const int c = v / VPC, q = v % VPC;
          const int r = r0 + q * VW;
          const T* src = A + (int64_t)c * pb.ld + (boxed ? roff_s[b][q * VW] : (int64_t)r);
          if (r + VW <= pb.m) {
            buf[i] = __ldg(reinterpret_cast<const VT*>(src));
          } else {
            T* xs = reinterpret_cast<T*>(&buf[i]);
#pragma unroll
            for (int u = 0; u < VW; ++u) xs[u] = (r + u < pb.m) ? src[u] : T(0);
          }
        }
      }
    };
    // ... transposed into As[row][col]; columns of the group past nc stay
    // stale: their accumulators are never stored
    auto put = [&](const VT* buf) {
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const int v = tid + i * kThreads;
        if (v < nc * VPC) {
          const int c = v / VPC, q = v % VPC;
          const T* xs = reinterpret_cast<const T*>(&buf[i]);
#pragma unroll
          for (int u = 0; u < VW; ++u) As[(q * VW + u) * CGP + c] = xs[u];
        }
      }
    };

    // wide tiles: one vector at a time, loaded and stored (no register buffer)
    auto stage_direct = [&](int ch, int b) {
      const int r0 = ch * kChunkRows;
      for (int v = tid; v < nc * VPC; v += kThreads) {
        const int c = v / VPC, q = v % VPC;
        const int r = r0 + q * VW;
        const T* src = A + (int64_t)c * pb.ld + (boxed ? roff_s[b][q * VW] : (int64_t)r);
        T vals[VW];
        if (r + VW <= pb.m) {
          const VT x = __ldg(reinterpret_cast<const VT*>(src));
          const T* xs = reinterpret_cast<const T*>(&x);
#pragma unroll
          for (int u = 0; u < VW; ++u) vals[u] = xs[u];
        } else {
#pragma unroll
          for (int u = 0; u < VW; ++u) vals[u] = (r + u < pb.m) ? src[u] : T(0);
        }
#pragma unroll
        for (int u = 0; u < VW; ++u) As[(q * VW + u) * CGP + c] = vals[u];
      }
    };

    VT buf[kPrefetch ? NV : 1];
    int b = 0;
    if constexpr (kPrefetch) {
      table(seg.chunk0, 0);
      __syncthreads();
      fetch(seg.chunk0, 0, buf);
    }
    for (int ch = seg.chunk0; ch < seg.chunk1; ++ch, b ^= 1) {
      const int r0 = ch * kChunkRows;
      if constexpr (kPrefetch) {
        put(buf);
      } else {
        table(ch, b);
        __syncthreads();
        stage_direct(ch, b);
      }
      // ---- Omega(:, r0 : r0+32) into Om[row][i]
      for (int task = tid; task < kChunkRows * (LP / 4); task += kThreads) {
        const int k = task % kChunkRows, g = task / kChunkRows;
        T w[4] = {T(0), T(0), T(0), T(0)};
        if (4 * g < l && r0 + k < pb.m) {
          omega_group<T>(key, (uint32_t)(r0 + k), (uint32_t)g, w);
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (4 * g + u >= l) w[u] = T(0);
        }
        VT* dst = reinterpret_cast<VT*>(Om + k * LP + 4 * g);
        if constexpr (VW == 4) {
          dst[0] = make_float4(w[0], w[1], w[2], w[3]);
        } else {
          dst[0] = make_double2(w[0], w[1]);
          dst[1] = make_double2(w[2], w[3]);
        }
      }
      const bool more = kPrefetch && ch + 1 < seg.chunk1;
      if (more) table(ch + 1, b ^ 1);
      __syncthreads();
      if constexpr (kPrefetch)
        if (more) fetch(ch + 1, b ^ 1, buf);   // in flight during the FMAs below
      // ---- acc[j][i] += A(r, j) Omega(i, r), rows in ascending order
#pragma unroll 4
      for (int k = 0; k < kChunkRows; ++k) {
        T a[TJ], w[TI];
#pragma unroll
        for (int u = 0; u < TJ; ++u) a[u] = As[k * CGP + jg + kJGroups * u];
#pragma unroll
        for (int v = 0; v < TI; v += VW) {
          const VT x = *reinterpret_cast<const VT*>(Om + k * LP + ig * TI + v);
          const T* xs = reinterpret_cast<const T*>(&x);
#pragma unroll
          for (int u = 0; u < VW; ++u) w[v + u] = xs[u];
        }
#pragma unroll
        for (int u = 0; u < TJ; ++u)
#pragma unroll
          for (int v = 0; v < TI; ++v) acc[u][v] = fma(a[u], w[v], acc[u][v]);
      }
      __syncthreads();
    }
    // ---- partial slot: [col][l_pad]
    T* out = partial + args.slot_off[seg.slot];
#pragma unroll
    for (int u = 0; u < TJ; ++u) {
      const int j = jg + kJGroups * u;
      if (j < nc) {
#pragma unroll
        for (int v = 0; v < TI; v += VW) {
          typename Vec<T>::type x;
          T* xs = reinterpret_cast<T*>(&x);
#pragma unroll
          for (int q = 0; q < VW; ++q) xs[q] = acc[u][v + q];
          store_vec<T>(out + (int64_t)j * LP + ig * TI + v, x);
        }
      }
    }
    // ---- the CTA that completes a problem sums its slots (fixed order)
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      const int nslots = args.pslot_ptr[seg.prob + 1] - args.pslot_ptr[seg.prob];
      last_flag = (atomicAdd(&args.prob_cnt[seg.prob], 1) == nslots - 1);
    }
    __syncthreads();
    if (last_flag) {
      __threadfence();
      reduce_problem_slots<T>(args, seg.prob, tid, kThreads);
      if (tid == 0) args.prob_cnt[seg.prob] = 0;
    }
  }
}

// Batched form: a CTA works through pack segments of the streamed schedule
// (the tensor-core kernels' packs: up to TJ 64-column slices of subdomains of
// one shape), so one Omega chunk serves every slice of the pack.  Thread
// (ig, jg) keeps column jg of each of the TJ slices; the problems a segment
// completes are folded side by side, each on its own share of the threads.
template <typename T, int TI, int TJ>
__global__ void __launch_bounds__(kThreads, simt_min_blocks(TI * TJ * (int)(sizeof(T) / 4)))
sketch_simt_packed_kernel(SketchArgs args) {
  constexpr int LP = 4 * TI;
  constexpr int CG = kJGroups * TJ;
  constexpr int CGP = CG + 1;
  constexpr int VW = Vec<T>::width;
  constexpr int VPC = kChunkRows / VW;
  using VT = typename Vec<T>::type;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int64_t roff_s[kChunkRows];      // boxes: element offsets of the chunk's rows
  __shared__ int64_t base_s[TJ];              // slice u: element offset of its first column
  __shared__ int64_t ld_s[TJ];
  __shared__ int ncols_s[TJ];
  __shared__ int last_s[kMaxPackMembers];
  __shared__ int done_s[kMaxPackMembers + 1];
  T* As = reinterpret_cast<T*>(smem_raw);       // [kChunkRows][CGP]
  T* Om = As + kChunkRows * CGP;                // [kChunkRows][LP]
  Om = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(Om) + 15) & ~uintptr_t(15));

  const int tid = threadIdx.x;
  const int ig = tid / kJGroups;
  const int jg = tid % kJGroups;
  const int cta = blockIdx.x + args.cta_base;
  const uint2 key = philox_key(args.seed);
  const T* window = static_cast<const T*>(args.window);
  T* partial = static_cast<T*>(args.partial);
  const int l = args.l;

  const int s0 = args.seg_ptr[cta], s1 = args.seg_ptr[cta + 1];
  for (int si = s0; si < s1; ++si) {
    const PackSegment sg = args.psegs[si];
    const Pack pk = args.packs[sg.pack];
    const int ns = pk.nslices;                  // <= TJ
    const RowGeom geo = args.probs[pk.prob0].geo;   // one shape (and field) per pack
    const bool boxed = geo.ex > 0;
    __syncthreads();   // the previous segment is done with the slice tables
    if (tid < ns) {
      const Slice sl = args.slices[pk.slice0 + tid];
      const Problem pb = args.probs[sl.prob];
      base_s[tid] = pb.off + (int64_t)sl.col0 * pb.ld;
      ld_s[tid] = pb.ld;
      ncols_s[tid] = sl.ncols;
    }
    T acc[TJ][TI];
#pragma unroll
    for (int u = 0; u < TJ; ++u)
#pragma unroll
      for (int v = 0; v < TI; ++v) acc[u][v] = T(0);

    for (int ch = sg.chunk0; ch < sg.chunk1; ++ch) {
      const int r0 = ch * kChunkRows;
      if (boxed && tid < kChunkRows) roff_s[tid] = (r0 + tid < pk.m) ? row_offset(geo, r0 + tid) : 0;
      __syncthreads();
      // ---- A(r0 : r0+32, every slice's columns) transposed into As[row][64 u + jj]
      for (int v = tid; v < ns * kJGroups * VPC; v += kThreads) {
        const int c = v / VPC, q = v % VPC;
        const int u = c / kJGroups, jj = c % kJGroups;
        const int r = r0 + q * VW;
        T vals[VW];
#pragma unroll
        for (int x = 0; x < VW; ++x) vals[x] = T(0);
        if (jj < ncols_s[u]) {
          const T* src = window + base_s[u] + (int64_t)jj * ld_s[u] + (boxed ? roff_s[q * VW] : (int64_t)r);
          if (r + VW <= pk.m) {
            const VT xv = __ldg(reinterpret_cast<const VT*>(src));
            const T* xs = reinterpret_cast<const T*>(&xv);
#pragma unroll
            for (int x = 0; x < VW; ++x) vals[x] = xs[x];
          } else {
#pragma unroll
            for (int x = 0; x < VW; ++x) vals[x] = (r + x < pk.m) ? src[x] : T(0);
          }
        }
#pragma unroll
        for (int x = 0; x < VW; ++x) As[(q * VW + x) * CGP + c] = vals[x];
      }
      // ---- Omega(:, r0 : r0+32) into Om[row][i], once for the whole pack
      for (int task = tid; task < kChunkRows * (LP / 4); task += kThreads) {
        const int k = task % kChunkRows, g = task / kChunkRows;
        T w[4] = {T(0), T(0), T(0), T(0)};
        if (4 * g < l && r0 + k < pk.m) {
          omega_group<T>(key, (uint32_t)(r0 + k), (uint32_t)g, w);
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (4 * g + u >= l) w[u] = T(0);
        }
        VT* dst = reinterpret_cast<VT*>(Om + k * LP + 4 * g);
        if constexpr (VW == 4) {
          dst[0] = make_float4(w[0], w[1], w[2], w[3]);
        } else {
          dst[0] = make_double2(w[0], w[1]);
          dst[1] = make_double2(w[2], w[3]);
        }
      }
      __syncthreads();
      // ---- acc[u][i] += A(r, column jg of slice u) Omega(i, r), rows ascending
#pragma unroll 4
      for (int k = 0; k < kChunkRows; ++k) {
        T a[TJ], w[TI];
#pragma unroll
        for (int u = 0; u < TJ; ++u) a[u] = As[k * CGP + jg + kJGroups * u];
#pragma unroll
        for (int v = 0; v < TI; v += VW) {
          const VT x = *reinterpret_cast<const VT*>(Om + k * LP + ig * TI + v);
          const T* xs = reinterpret_cast<const T*>(&x);
#pragma unroll
          for (int u = 0; u < VW; ++u) w[v + u] = xs[u];
        }
#pragma unroll
        for (int u = 0; u < TJ; ++u)
#pragma unroll
          for (int v = 0; v < TI; ++v) acc[u][v] = fma(a[u], w[v], acc[u][v]);
      }
      __syncthreads();
    }
    // ---- partial slots: slice u's column jg goes to its problem's slot
#pragma unroll
    for (int u = 0; u < TJ; ++u) {
      if (u < ns && jg < ncols_s[u]) {
        const Slice sl = args.slices[pk.slice0 + u];
        T* out = partial + args.slot_off[sg.slot0 + sl.member] + (int64_t)(sl.out_col + jg) * LP;
#pragma unroll
        for (int v = 0; v < TI; v += VW) {
          VT x;
          T* xs = reinterpret_cast<T*>(&x);
#pragma unroll
          for (int q = 0; q < VW; ++q) xs[q] = acc[u][v + q];
          store_vec<T>(out + ig * TI + v, x);
        }
      }
    }
    // ---- every member problem counts this segment; the completed ones are
    // folded side by side (completed problem j of c on threads
    // [ceil(j N / c), ceil((j + 1) N / c)), each element summing its slots in
    // schedule order)
    __threadfence();
    __syncthreads();
    if (tid < pk.nprob) {
      const int p = pk.prob0 + tid;
      const int nslots = args.pslot_ptr[p + 1] - args.pslot_ptr[p];
      last_s[tid] = (atomicAdd(&args.prob_cnt[p], 1) == nslots - 1);
    }
    __syncthreads();
    if (tid == 0) {
      int c = 0;
      for (int q = 0; q < pk.nprob; ++q)
        if (last_s[q]) done_s[c++] = q;
      done_s[kMaxPackMembers] = c;
    }
    __syncthreads();
    const int c = done_s[kMaxPackMembers];
    if (c > 0) {
      __threadfence();
      const int j = tid * c / kThreads;
      const int t0 = (j * kThreads + c - 1) / c, t1 = ((j + 1) * kThreads + c - 1) / c;
      reduce_problem_slots<T>(args, pk.prob0 + done_s[j], tid - t0, t1 - t0);
      if (tid < c) args.prob_cnt[pk.prob0 + done_s[tid]] = 0;
    }
  }
}

template <typename T, int TI, int TJ>
cudaError_t launch_one(const SketchArgs& a, int grid, cudaStream_t st) {
  constexpr int LP = 4 * TI;
  constexpr int CGP = kJGroups * TJ + 1;
  const size_t smem = sizeof(T) * (size_t)kChunkRows * (CGP + LP) + 16;
  auto k = sketch_simt_kernel<T, TI, TJ>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename T, int TI, int TJ>
cudaError_t launch_packed(const SketchArgs& a, int grid, cudaStream_t st) {
  constexpr int LP = 4 * TI;
  constexpr int CGP = kJGroups * TJ + 1;
  const size_t smem = sizeof(T) * (size_t)kChunkRows * (CGP + LP) + 16;
  auto k = sketch_simt_packed_kernel<T, TI, TJ>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

// Column-group size of the SIMT sketch for a given element size.
int sketch_simt_group_cols(bool fp64) { return fp64 ? kJGroups * 4 : kJGroups * 8; }

// Columns per thread for a launch whose widest problem has max_cols columns.
int sketch_simt_tj(bool fp64, int max_cols) {
  const int cap = fp64 ? 4 : 8;
  int tj = 1;
  while (tj < cap && kJGroups * tj < max_cols) tj *= 2;
  return tj;
}

// CTAs per SM the launch bounds of the (l_pad, tj) variant are built for.
int sketch_simt_ctas_per_sm(bool fp64, int l_pad, int tj) {
  return simt_min_blocks((l_pad / 4) * tj * (fp64 ? 2 : 1));
}

namespace {

template <typename T, int TI, bool PACKED>
cudaError_t launch_tj(const SketchArgs& a, int grid, int tj, cudaStream_t st) {
  switch (tj) {
    case 1: return PACKED ? launch_packed<T, TI, 1>(a, grid, st) : launch_one<T, TI, 1>(a, grid, st);
    case 2: return PACKED ? launch_packed<T, TI, 2>(a, grid, st) : launch_one<T, TI, 2>(a, grid, st);
    case 4: return PACKED ? launch_packed<T, TI, 4>(a, grid, st) : launch_one<T, TI, 4>(a, grid, st);
    case 8:
      if constexpr (sizeof(T) == 4)
        return PACKED ? launch_packed<T, TI, 8>(a, grid, st) : launch_one<T, TI, 8>(a, grid, st);
      break;
  }
  return cudaErrorInvalidValue;
}

template <bool PACKED>
cudaError_t launch_simt(const SketchArgs& a, int grid, bool fp64, int tj, cudaStream_t st) {
  if (grid <= 0) return cudaSuccess;
  if (fp64) {
    switch (a.l_pad) {
      case 16: return launch_tj<double, 4, PACKED>(a, grid, tj, st);
      case 32: return launch_tj<double, 8, PACKED>(a, grid, tj, st);
      case 48: return launch_tj<double, 12, PACKED>(a, grid, tj, st);
      case 64: return launch_tj<double, 16, PACKED>(a, grid, tj, st);
    }
  } else {
    switch (a.l_pad) {
      case 16: return launch_tj<float, 4, PACKED>(a, grid, tj, st);
      case 32: return launch_tj<float, 8, PACKED>(a, grid, tj, st);
      case 48: return launch_tj<float, 12, PACKED>(a, grid, tj, st);
      case 64: return launch_tj<float, 16, PACKED>(a, grid, tj, st);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_sketch_simt(const SketchArgs& a, int grid, bool fp64, int tj, cudaStream_t st) {
  return launch_simt<false>(a, grid, fp64, tj, st);
}

cudaError_t launch_sketch_simt_packed(const SketchArgs& a, int grid, bool fp64, int tj,
                                      cudaStream_t st) {
  return launch_simt<true>(a, grid, fp64, tj, st);
}

}  // namespace spid
