// spid_internal.cuh -- types shared by the host side of libspid and its
// kernels, plus the device helpers every kernel uses (Philox4x32-10,
// Box-Muller, bounded waits, status word).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace spid {

// Sticky device status bits (OR-ed into the plan's status word).
enum : int {
  kStatusTimeout = 1,
  kStatusNonfinite = 2,
  kStatusRankCut = 4,   // informational: the rank guard stopped a factorization early
};

// Where the rows of a subdomain sit inside one column of the window.  A box of
// the solver's global field [t][q][Z][Y][X] has rows r = ((q ez + z) ey + y)
// ex + x (QoI slowest), and row r is element x + y sy + z sz + q sq of the
// column (sy = X, sz = X Y, sq = X Y Z).  ex = 0: the rows are contiguous
// (element r), the blocks layout.
struct RowGeom {
  int32_t ex, ey, ez, pad;
  int64_t sy, sz, sq;
};

__host__ __device__ __forceinline__ int64_t row_offset(const RowGeom& g, int64_t r) {
  if (g.ex == 0) return r;
  const int64_t x = r % g.ex, t = r / g.ex;
  const int64_t y = t % g.ey, t2 = t / g.ey;
  const int64_t z = t2 % g.ez, q = t2 / g.ez;
  return x + y * g.sy + z * g.sz + q * g.sq;
}

// Every spin on an mbarrier gives up after this many nanoseconds, records
// kStatusTimeout and lets the kernel unwind.
constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // 1 s

// Rows of A handled per sketch chunk: one 128-byte swizzle row of FP32.
constexpr int kChunkRows = 32;

// A "problem" is one subdomain restricted to a group of window columns.
struct Problem {
  int32_t sub;     // subdomain index
  int32_t col0;    // first window column
  int32_t ncols;   // number of columns (<= the kernel's column-group size)
  int32_t m;       // rows of the subdomain
  int64_t off;     // element offset of A_s(0,0) in the window
  int64_t ld;      // leading dimension (column stride) in elements
  RowGeom geo;     // row placement inside a column (ex = 0: contiguous)
};

// A contiguous range of row chunks of one problem, processed by one CTA; its
// partial sketch goes to partial slot `slot`.
struct Segment {
  int32_t prob;
  int32_t chunk0;
  int32_t chunk1;
  int32_t slot;
};

// Tensor-core packing: Omega does not depend on the subdomain, so one chunk of
// rows can serve several subdomains at once.  A slice is up to kSliceCols
// columns of one problem (one TMA box of 32 rows; 64 columns by default, 32 or
// 16 in the TF32 sketch when tuned so, which narrows the range of window
// columns -- snapshots -- one chunk touches); a pack is up to 512 columns of
// slices of problems with the same shape, streamed together as 4 MMA tiles of
// 128 rows.
constexpr int kSliceCols = 64;
constexpr int kPackSlices = 8;                 // pack width in 64-column units
constexpr int kMaxPackMembers = 32;            // slices (and problems) per pack, 512 / 16
// Cost of a pack's epilogue (TMEM drain, partial slots, fold) in chunks of
// streaming, for balancing the chunks over the persistent CTAs: measured on
// uneven windows, a 16-chunk pack (m = 512) took about as long as 16 more.
constexpr double kPackOverheadChunks = 16.0;

struct Slice {
  int32_t prob;      // problem index (the fold unit)
  int32_t sub;       // subdomain (tensor map)
  int32_t col0;      // first window column of the slice
  int32_t ncols;     // <= the plan's slice width
  int32_t out_col;   // column of the slice inside its problem's partial slot
  int32_t member;    // index of its problem among the pack's problems
  // The TMA box that loads the slice: tensor map `map`, with the subdomain's
  // first element at coordinate (tx, ty, tz, tq) of that map.  2-D maps load
  // (tx + row, ty + col0); 5-D maps load (tx + x, ty + y, tz + z, tq + q, col0).
  // A subdomain's own map has origin 0; a map shared by many subdomains (one
  // over the whole field, or one per run of equally strided blocks) places it.
  int32_t map;
  int32_t tx, ty, tz, tq;
};

struct Pack {
  int32_t slice0;    // first slice
  int32_t nslices;   // 1 .. 512 / slice width
  int32_t m;         // rows of every member
  int32_t prob0;     // first member problem (members are consecutive problems)
  int32_t nprob;     // number of member problems
  // box geometry shared by every member (ex = 0: 2-D tensor maps over
  // contiguous rows; else 5-D maps (x, y, z, q, column) and a 32-row chunk is
  // one 32-point run along x, ex a multiple of 32)
  int32_t ex, ey, ez;
};

// A contiguous range of row chunks of one pack, processed by one CTA; member
// problem q of the pack writes its partial to slot slot0 + q.
struct PackSegment {
  int32_t pack;
  int32_t chunk0;
  int32_t chunk1;
  int32_t slot0;
};

// Sketch schedule arguments (both sketch kernels).
struct SketchArgs {
  const Problem* probs;
  const Segment* segs;
  const int32_t* seg_ptr;     // CTA c owns segs[seg_ptr[c] .. seg_ptr[c+1])
  const int64_t* slot_off;    // element offset of each partial slot
  void* partial;              // float or double partial sums [slot][ncols][l_pad]
  const void* window;
  const void* tmaps;          // CUtensorMap per subdomain (TF32 kernel only)
  int32_t cta_base;           // first schedule CTA of this launch
  int32_t l;
  int32_t l_pad;
  uint64_t seed;
  int* status;
  // fixed-order reduction of the partial slots into the stored sketch, done by
  // the CTA that completes each problem
  const int32_t* pslot_ptr;   // problem p owns pslots[pslot_ptr[p] .. pslot_ptr[p+1])
  const int32_t* pslots;
  int* prob_cnt;              // [problems] completed-segment counters (zero between calls)
  void* Y;                    // stored sketches, Y_s at yoff[s], [n_s][l_pad]
  const int64_t* yoff;
  // tensor-core schedule: CTA c owns psegs[seg_ptr[c] .. seg_ptr[c+1])
  const Slice* slices;
  const Pack* packs;
  const PackSegment* psegs;
  int32_t slice_cols = kSliceCols;   // columns per slice (TMA box width)
};

template <typename T> struct Vec16;   // 16-byte vector of T
template <> struct Vec16<float> {
  using type = float4;
  static __device__ __forceinline__ float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  static __device__ __forceinline__ void add(float4& s, const float4& x) {
    s.x += x.x; s.y += x.y; s.z += x.z; s.w += x.w;
  }
};
template <> struct Vec16<double> {
  using type = double2;
  static __device__ __forceinline__ double2 zero() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ void add(double2& s, const double2& x) {
    s.x += x.x; s.y += x.y;
  }
};

// Sum problem p's partial slots in schedule order into Y (called by the CTA
// that completed p, after a device-wide fence) with threads t of nt: 16-byte
// loads from L2, four independent vectors per thread, coalesced per warp.
template <typename T>
__device__ __forceinline__ void reduce_problem_slots(const SketchArgs& a, int p, int t, int nt) {
  using V = typename Vec16<T>::type;
  constexpr int U = 4;   // 16-byte vectors per thread per pass
  constexpr int G = 2;   // slots whose loads are in flight together (added in slot order)
  const Problem pb = a.probs[p];
  const int q0 = a.pslot_ptr[p], q1 = a.pslot_ptr[p + 1];
  const T* part = static_cast<const T*>(a.partial);
  V* Y = reinterpret_cast<V*>(static_cast<T*>(a.Y) + a.yoff[pb.sub] +
                              (int64_t)pb.col0 * a.l_pad);
  const int64_t nv = (int64_t)pb.ncols * a.l_pad * sizeof(T) / 16;   // l_pad % 16 == 0
  for (int64_t base = 0; base < nv; base += (int64_t)nt * U) {
    V s[U];
#pragma unroll
    for (int u = 0; u < U; ++u) s[u] = Vec16<T>::zero();
    for (int q = q0; q < q1; q += G) {
      const V* src[G];
#pragma unroll
      for (int g = 0; g < G; ++g)
        src[g] = (q + g < q1) ? reinterpret_cast<const V*>(part + a.slot_off[a.pslots[q + g]]) : nullptr;
      V v[G][U];
#pragma unroll
      for (int g = 0; g < G; ++g)
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t e = base + t + (int64_t)u * nt;
          v[g][u] = (src[g] && e < nv) ? __ldcg(src[g] + e) : Vec16<T>::zero();
        }
#pragma unroll
      for (int g = 0; g < G; ++g)
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (src[g]) Vec16<T>::add(s[u], v[g][u]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t e = base + t + (int64_t)u * nt;
      if (e < nv) Y[e] = s[u];
    }
  }
}

// Batched pivoted QR + rank + coefficients.
struct QrcpArgs {
  const void* Y;          // sketches: Y_s at yoff[s], [n_s][l_pad]
  const int64_t* yoff;
  const int32_t* n;
  void* C;                // C_s at coff[s], k_max x n_s row-major
  const int64_t* coff;
  int32_t* J;             // [S][k_max]
  int32_t* k_out;         // [S]
  int32_t l;
  int32_t k_max;
  double tol;
  double u_mode;
  int32_t sub_base;
  int* status;
};

// Fused reconstruction / error pass.  A work unit is (subdomain, block of
// row_block rows, block of col_block columns); the defaults below, or a shape
// chosen by the plan's autotuner (row_block a multiple of kErrTile, col_block
// 128 or 256).
constexpr int kErrRowBlock = 512;
constexpr int kErrColBlock = 256;
constexpr int kErrTile = 128;
constexpr int kErrMaxK = 64;     // skeleton columns a unit can stage

struct ErrArgs {
  const void* window;
  void* out;                  // reconstruction (same layout), or nullptr
  const int32_t* m;
  const int32_t* n;
  const int64_t* off;
  const int64_t* ld;
  const void* C;
  const int64_t* coff;
  const int32_t* J;
  const int32_t* k;
  int32_t k_max;
  const int32_t* unit_sub;
  const int32_t* unit_row0;
  const int32_t* unit_col0;
  double* part;               // [unit][2] = {e2, a2}
  int32_t unit_base;
  const int32_t* unit_ptr;    // subdomain s owns units [unit_ptr[s], unit_ptr[s+1])
  int* sub_cnt;               // [S] completed-unit counters (zero between calls)
  int* all_cnt;               // completed-subdomain counter (zero between calls)
  double* err;                // [S][2] or nullptr
  double* sub_err;            // plan copy [S][2]
  double* total;              // [4] or nullptr
  int32_t S;
  const int32_t* srows = nullptr;   // rows stored per subdomain for the CF sums (nullptr: m)
  int32_t row_block = kErrRowBlock; // rows of a unit
  int32_t col_block = kErrColBlock; // columns of a unit (C block staged in shared memory)
  // skeleton source: nullptr = the window's columns J (A_hat = A(:, J) C); else
  // an m_s x k block per subdomain at skel_off[s], leading dimension m_s
  // (A_hat = F C, e.g. F = M B(:, I_B) of the coarse-grid SPID)
  const float* skel = nullptr;
  const int64_t* skel_off = nullptr;
  // row placement per subdomain (nullptr: contiguous rows)
  const RowGeom* geo = nullptr;
  // per-QoI totals: subdomain s holds QoI qoi[s] < num_qoi; total[4 + 2 g],
  // total[5 + 2 g] receive that QoI's sum e2, sum a2 (num_qoi = 0: none)
  const int32_t* qoi = nullptr;
  int32_t num_qoi = 0;
};

// Tensor-core error pass (FP32 windows, k_max <= 32): a segment is a run of
// 128-row tiles of one (subdomain, column block of <= 256 columns) processed by
// one CTA; the segments of subdomain s are unit_ptr[s] .. unit_ptr[s + 1].
constexpr int kErrTcRows = 128;
constexpr int kErrTcCols = 256;
constexpr int kErrTcKMax = 32;

struct ErrSeg {
  int32_t sub;
  int32_t col0;
  int32_t ncols;   // <= kErrTcCols
  int32_t tile0;   // first 128-row tile
  int32_t tile1;   // one past the last tile
};

struct ErrTcArgs {
  ErrArgs e;               // unit_* fields unused; part/unit_ptr index segments
  const ErrSeg* segs;
  const int32_t* seg_ptr;  // CTA c owns segs[seg_ptr[c] .. seg_ptr[c + 1])
  int* status;
};

// Detail message returned by spid_last_error() on the calling thread.
void set_last_error(const char* msg);

// Device view of a plan's factors and status (used by the two-stage driver,
// which composes plans).  C_s starts at element coff[s] (k_max x n_s row-major).
struct PlanView {
  int32_t S;
  int32_t k_max;
  size_t esz;
  const int32_t* m;       // device [S]
  const int32_t* n;       // device [S]
  int32_t* k;             // device [S]
  int32_t* J;             // device [S][k_max]
  void* C;
  const int64_t* coff;    // device [S]
  int* status;
  void* Y;                // stored sketches, Y_s at yoff[s], [n_s][l_pad]
  const int64_t* yoff;    // device [S]
  int32_t l;              // rows the QR reads
  int32_t l_pad;          // row stride of the stored sketch
};

// Launchers (one translation unit each).
int sketch_simt_group_cols(bool fp64);
int sketch_simt_tj(bool fp64, int max_cols);
int sketch_simt_ctas_per_sm(bool fp64, int l_pad, int tj);
cudaError_t launch_sketch_simt(const SketchArgs& a, int grid, bool fp64, int tj, cudaStream_t st);
// batched plans: the pack segments of the streamed schedule (tj = slices per pack tile)
cudaError_t launch_sketch_simt_packed(const SketchArgs& a, int grid, bool fp64, int tj,
                                      cudaStream_t st);
int sketch_tc_group_cols();
size_t sketch_tc_smem_bytes(int stages, int max_tiles, int l_pad);
int sketch_tc_max_stages();
size_t sketch_bf16_smem_bytes(int stages, int max_tiles, int l_pad, bool split);
cudaError_t launch_sketch_bf16(const SketchArgs& s, int grid, int stages, int max_tiles, bool split,
                               cudaStream_t st);
cudaError_t launch_sketch_tc(const SketchArgs& s, int grid, int stages, int max_tiles,
                             cudaStream_t st);
int qrcp_cols_per_thread(int n_max, int l_pad, bool fp64);
cudaError_t launch_qrcp(const QrcpArgs& a, int grid, int n_max, int l_pad, bool fp64,
                        cudaStream_t st);
size_t error_smem_bytes(int k_max, int col_block, bool fp64);
size_t error_tc_smem_bytes();
cudaError_t launch_error_tc(const ErrTcArgs& a, int grid, cudaStream_t st);
cudaError_t launch_error(const ErrArgs& a, int units, bool fp64, cudaStream_t st);

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the Philox
// S-box on a 4 x 32-bit counter, with a Weyl-sequence key schedule.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__device__ __forceinline__ uint2 philox_key(uint64_t seed) {
  return make_uint2((uint32_t)(seed & 0xffffffffull), (uint32_t)(seed >> 32));
}

// Box-Muller on a pair of words, FP32: u = (x + 0.5) 2^-32.
__device__ __forceinline__ void box_muller(uint32_t xa, uint32_t xb, float& g0, float& g1) {
  const float ua = fmaf(__uint2float_rn(xa), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
  const float ub = fmaf(__uint2float_rn(xb), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
  const float rad = sqrtf(-2.0f * logf(ua));
  float s, c;
  sincospif(2.0f * ub, &s, &c);
  g0 = rad * c;
  g1 = rad * s;
}

// Box-Muller on a pair of words, FP64.
__device__ __forceinline__ void box_muller(uint32_t xa, uint32_t xb, double& g0, double& g1) {
  const double ua = ((double)xa + 0.5) * 2.3283064365386963e-10;
  const double ub = ((double)xb + 0.5) * 2.3283064365386963e-10;
  const double rad = sqrt(-2.0 * log(ua));
  double s, c;
  sincospi(2.0 * ub, &s, &c);
  g0 = rad * c;
  g1 = rad * s;
}

// Omega(4g .. 4g+3, r) from one Philox call with counter (r, g, 0, 0).
template <typename T>
__device__ __forceinline__ void omega_group(uint2 key, uint32_t r, uint32_t g, T out[4]) {
  const uint4 x = philox4x32_10(make_uint4(r, g, 0u, 0u), key);
  box_muller(x.x, x.y, out[0], out[1]);
  box_muller(x.z, x.w, out[2], out[3]);
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void raise_status(int* status, int bit) {
  if (status) atomicOr(status, bit);
}

}  // namespace spid
