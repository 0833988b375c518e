// subid_internal.cuh -- types shared by the host side and the kernels of the
// coarse-grid (subsampled / single-pass) ID: Section 2 SubID and SPID,
// Algorithms 2 and 3, Section 5.2.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "spid_internal.cuh"

namespace spid {

constexpr int kGatherWarps = 8192;     // warps the coarse gather aims for
constexpr int kSubMaxK = 64;          // k_max bound (coefficient solve keeps k values per column)
constexpr int kSubMaxN = 1024;        // window length bound (one residual norm per column in smem)
constexpr int kSubMaxCoarse = 40960;  // coarse rows bound (one column of B in shared memory)
constexpr int kSubUnitElems = 32768;  // target fine elements per SPID error unit
constexpr int kSubMaxStencil = 16;   // coarse rows per fine row of a point-set interpolation

// Division by a fixed divisor d >= 1 as a multiply-high and a shift
// (Granlund and Montgomery, PLDI'94, Section 4): for 0 <= x < 2^31,
// x / d = (umulhi(x, mul) + x) >> shift with shift = ceil(log2 d) and
// mul = floor(2^32 (2^shift - d) / d) + 1.
struct FastDiv {
  uint32_t d, mul, shift;
};

inline FastDiv make_fastdiv(uint32_t d) {
  uint32_t sh = 0;
  while ((1ull << sh) < d) ++sh;
  const uint64_t m = ((1ull << 32) * ((1ull << sh) - d)) / d + 1;
  return FastDiv{d, (uint32_t)m, sh};
}

__device__ __forceinline__ uint32_t fdiv(uint32_t x, const FastDiv& f) {
  return (__umulhi(x, f.mul) + x) >> f.shift;
}

// One subdomain box and its coarse grid.  Coarse index a of an axis with e
// points and interval s is min(a s, e - 1); count c = (e - 1) / s + 1, plus one
// when (e - 1) % s != 0 (the end point is kept).
struct SubBox {
  int32_t nq, ez, ey, ex;     // QoIs, points along z, y, x
  int32_t cz, cy, cx;         // coarse points along z, y, x
  int32_t sz, sy, sx;         // intervals
  int32_t zc;                 // z planes per SPID error unit
  int32_t zblocks;            // SPID error units per column = ceil(ez / zc)
  FastDiv div_ex, div_plane;  // fine x and (y, x)-plane decodes
  FastDiv div_cx, div_cy, div_cz, div_mc;   // coarse-row decodes
};

// Column stride of the coarse matrix B and its working copy W: m_c rounded up
// to 4 floats, so every column starts 16-byte aligned (rows past m_c are zero).
__host__ __device__ inline int coarse_ld(int mc) { return (mc + 3) & ~3; }

struct SubArgs {
  const SubBox* box;          // [S]
  const int32_t* m;           // [S] fine rows
  const int32_t* n;           // [S]
  const int32_t* mc;          // [S] coarse rows
  const int64_t* off;         // [S] window offsets
  const int64_t* ld;          // [S]
  const int64_t* boff;        // [S] B_s / W_s at boff[s], column-major, column stride
                              // coarse_ld(mc) (W as the coarse reconstruction: stride mc)
  const int64_t* coff;        // [S] sum of n before s (R, C at k_max * coff[s])
  const int64_t* sklo;        // [S] sum of mc before s (Bskel at k_max * sklo[s])
  float* B;                   // gathered coarse matrices
  float* nrm;                 // [sum n][nrm_parts] parts of ||B(:, c)||^2 from the gather
                              // (NaN: a non-finite entry in that part)
  int32_t nrm_parts;
  float* W;                   // MGS working copy; after finalize, the coarse reconstruction
  float* R;                   // k_max x n_s row-major per subdomain
  float* C;                   // k_max x n_s row-major per subdomain
  float* Bskel;               // mc x k_max column-major per subdomain
  int32_t* J;                 // [S][k_max]
  int32_t* k;                 // [S]
  int32_t k_max;
  int32_t S;
  double tol;
  int* status;
};

// SPID error units: subdomain s owns units [uptr[s], uptr[s+1]), unit
// uptr[s] + j * zblocks + b covers column j and z planes [b zc, b zc + zc).
struct SubErrArgs {
  SubArgs a;
  ErrArgs e;                  // fold: m, n, k, part, unit_ptr(= uptr), counters, totals, srows
  const float* window;
  float* out;                 // SPID reconstruction or nullptr
};

cudaError_t launch_subsample(const SubArgs& a, const float* window, int col0, int ncols,
                             int64_t max_work, cudaStream_t st);
size_t subid_qr_smem_bytes(int mc_max, int n_max, int k_max);
cudaError_t launch_subid_qr(const SubArgs& a, int mc_max, int n_max, cudaStream_t st);
cudaError_t launch_coarse_recon(const SubArgs& a, int64_t max_work, cudaStream_t st);
size_t spid_interp_smem_bytes(int mc_max, int e_max);
cudaError_t launch_spid_interp(const SubErrArgs& a, int64_t units, int mc_max, int e_max,
                               cudaStream_t st);
// F = M B(:, I_B): the trilinear interpolation of every coarse skeleton column
// to the fine grid, m_s x k_s column-major at foff[s] (leading dimension m_s).
cudaError_t launch_fine_skeleton(const SubArgs& a, float* F, const int64_t* foff, int m_max,
                                 int e_max, cudaStream_t st);

// Point-set plans: B = A(crow, :); F = M B(:, I_B) with a t-wide stencil
// (iidx, iw: m_s x t per subdomain at ioff[s]); out = F C (no window).
cudaError_t launch_subsample_rows(const SubArgs& a, const float* window, int col0, int ncols,
                                  const int32_t* crow, const int64_t* crow_off, int64_t max_work,
                                  cudaStream_t st);
cudaError_t launch_fine_skeleton_points(const SubArgs& a, float* F, const int64_t* foff,
                                        const int32_t* iidx, const float* iw, const int64_t* ioff,
                                        int t, int m_max, cudaStream_t st);
cudaError_t launch_skeleton_product(const SubArgs& a, const float* F, const int64_t* foff,
                                    float* out, int m_max, int n_max, cudaStream_t st);

}  // namespace spid
