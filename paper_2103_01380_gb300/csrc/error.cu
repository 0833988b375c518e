// error.cu -- reconstruction A_hat = A(:,J) C (Section 2, column ID form of
// Algorithm 2) fused with the relative Frobenius error of Section 5.1:
// ||A - A_hat||_F^2 and ||A||_F^2 per subdomain and over the window, plus the
// compression-factor sums (Section 2, Eq. for CF).
//
// A unit is (subdomain, row block, column block): 512 x 256 by default, or the
// shape the plan's autotuner measured fastest.  The CTA stages the
// coefficient block C(:, cols) and, per 128-row tile, the skeleton rows
// A(rows, J) in shared memory, then streams A once: lane l of warp w owns rows
// 4l..4l+3 of the tile and 4 columns at a time, so each k-step is two shared
// loads (one a broadcast) feeding 16 FMAs; A is read with 16-byte loads,
// 512 contiguous bytes per warp per column.
//
// Reductions keep FP64 off the per-element path (GB300 runs FP64 at 1/64 of
// FP32): each thread sums a tile's terms plainly (at most 128) and adds the
// tile sum to a Kahan-compensated running sum in the working precision, warps
// reduce in the working precision, and only the per-CTA, per-subdomain and
// window totals are FP64.  The last CTA of each subdomain (an atomic counter,
// after a device-wide fence) sums that subdomain's unit partials in a fixed
// order, and the last subdomain to finish sums the window totals; every
// counter is reset by the CTA that completes it, so results are deterministic
// and the plan is ready for the next call.
#include "error_fold.cuh"
#include "spid_internal.cuh"

namespace spid {

namespace {

template <typename T> struct V4;   // 4 consecutive elements
template <> struct V4<float> {
  static __device__ __forceinline__ void load(const float* p, float (&v)[4]) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  }
  static __device__ __forceinline__ void store(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
  static __device__ __forceinline__ void lds(const float* p, float (&v)[4]) {
    const float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  }
};
template <> struct V4<double> {
  static __device__ __forceinline__ void load(const double* p, double (&v)[4]) {
    const double2 x = __ldg(reinterpret_cast<const double2*>(p));
    const double2 y = __ldg(reinterpret_cast<const double2*>(p) + 1);
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
  }
  static __device__ __forceinline__ void store(double* p, const double (&v)[4]) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
  static __device__ __forceinline__ void lds(const double* p, double (&v)[4]) {
    const double2 x = reinterpret_cast<const double2*>(p)[0];
    const double2 y = reinterpret_cast<const double2*>(p)[1];
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
  }
};

// Kahan-compensated running sum.
template <typename T>
__device__ __forceinline__ void kahan_add(T& s, T& c, T x) {
  const T y = x - c;
  const T t = s + y;
  c = (t - s) - y;
  s = t;
}

template <typename T, bool WRITE, int CB>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) error_kernel(ErrArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[2][8];
  __shared__ int last_sub;
  __shared__ const T* colp[kErrMaxK];
  __shared__ int64_t roff_s[kErrTile];   // boxes: element offsets of the tile's rows
  const int u = blockIdx.x + a.unit_base;
  const int s = a.unit_sub[u];
  const int row0 = a.unit_row0[u], col0 = a.unit_col0[u];
  const int m = a.m[s], n = a.n[s];
  const int kk = a.k[s];
  constexpr int cb = CB;                          // columns per unit (== a.col_block)
  const int ncb = min(cb, n - col0);
  const int nrb = min(a.row_block, m - row0);
  T* Cs = reinterpret_cast<T*>(smem_raw);                 // [kk][cb]
  T* AJ = Cs + (size_t)a.k_max * cb;                       // [kk][kErrTile]
  const T* A = static_cast<const T*>(a.window) + a.off[s];
  const int64_t ld = a.ld[s];
  const T* Cg = static_cast<const T*>(a.C) + a.coff[s];
  const int32_t* Jg = a.J + (int64_t)s * a.k_max;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  // a box of a global field: row r at element row_offset(geo, r) of its column
  // (x-runs a multiple of 4 long, so a lane's 4 rows stay contiguous)
  const RowGeom geo = a.geo ? a.geo[s] : RowGeom{0, 0, 0, 0, 0, 0, 0};
  const bool boxed = geo.ex > 0;   // uniform over the CTA

  // skeleton column p: A(:, J[p]) of the window, or column p of the m x k
  // block the caller formed (floats; FP32 plans only)
  if (tid < kk)
    colp[tid] = a.skel ? reinterpret_cast<const T*>(a.skel + a.skel_off[s] + (int64_t)tid * m)
                       : A + (int64_t)Jg[tid] * ld;
  for (int e = tid; e < kk * cb; e += 256) {
    const int p = e / cb, jj = e % cb;
    Cs[e] = (jj < ncb) ? Cg[(int64_t)p * n + col0 + jj] : T(0);
  }
  T se = T(0), ce = T(0), sa = T(0), ca = T(0);   // Kahan sums of e^2 and a^2
  for (int t0 = 0; t0 < nrb; t0 += kErrTile) {
    const int rt = row0 + t0;                       // first row of the tile
    __syncthreads();
    if (boxed) {
      if (tid < kErrTile) roff_s[tid] = (rt + tid < m) ? row_offset(geo, rt + tid) : 0;
      __syncthreads();
    }
    for (int e = tid; e < kk * kErrTile; e += 256) {
      const int p = e / kErrTile, r = e % kErrTile;
      // the skeleton block of a coarse-grid plan (skel) has contiguous rows
      const int64_t ro = (boxed && !a.skel) ? roff_s[r] : (int64_t)(rt + r);
      AJ[e] = (rt + r < m) ? colp[p][ro] : T(0);
    }
    __syncthreads();
    const int r = rt + 4 * lane;                    // this lane's 4 rows
    const int64_t rofs = boxed ? roff_s[4 * lane] : (int64_t)r;   // their element offset
    const bool full_rows = (r + 4 <= m);
    // this tile's sums of e^2 and a^2, plain FP32 (at most 8 passes x 16
    // terms), added to the Kahan sums once per tile
    T te = T(0), ta = T(0);
    for (int cg = 4 * warp; cg < ncb; cg += 32) {   // 4 columns per warp per pass
      T av[4][4];   // A(r .. r+3, col0 + cg + y)
      const T* src0 = A + (int64_t)(col0 + cg) * ld + rofs;
      if (full_rows && cg + 4 <= ncb) {
#pragma unroll
        for (int y = 0; y < 4; ++y) V4<T>::load(src0 + y * ld, av[y]);
      } else {
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          const bool in = cg + y < ncb;
          const T* src = src0 + y * ld;
          if (in && full_rows) {
            V4<T>::load(src, av[y]);
          } else {
#pragma unroll
            for (int x = 0; x < 4; ++x) av[y][x] = (in && r + x < m) ? src[x] : T(0);
          }
        }
      }
      // k-step 0 starts the products (no zeroing pass), steps 1.. accumulate
      T acc[4][4];
      if (kk > 0) {
        T aj[4], cc[4];
        V4<T>::lds(AJ + 4 * lane, aj);
        V4<T>::lds(Cs + cg, cc);
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = aj[x] * cc[y];
      } else {
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = T(0);
      }
#pragma unroll 2
      for (int p = 1; p < kk; ++p) {
        T aj[4], cc[4];
        V4<T>::lds(AJ + p * kErrTile + 4 * lane, aj);
        V4<T>::lds(Cs + p * cb + cg, cc);
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = fma(aj[x], cc[y], acc[x][y]);
      }
      T le = te, la = ta;
#pragma unroll
      for (int y = 0; y < 4; ++y) {
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          const T d = av[y][x] - acc[x][y];
          le = fma(d, d, le);
          la = fma(av[y][x], av[y][x], la);
        }
        if (WRITE) {
          const int col = col0 + cg + y;
          if (col < n) {
            T* dst = static_cast<T*>(a.out) + a.off[s] + (int64_t)col * ld + rofs;
            T o[4] = {acc[0][y], acc[1][y], acc[2][y], acc[3][y]};
            if (full_rows) {
              V4<T>::store(dst, o);
            } else {
#pragma unroll
              for (int x = 0; x < 4; ++x)
                if (r + x < m) dst[x] = o[x];
            }
          }
        }
      }
      te = le;
      ta = la;
    }
    kahan_add(se, ce, te);
    kahan_add(sa, ca, ta);
  }
  // warp tree in the working precision, then FP64 across the 8 warps
  T we = se - ce, wa = sa - ca;
  for (int o = 16; o > 0; o >>= 1) {
    we += __shfl_xor_sync(0xffffffffu, we, o);
    wa += __shfl_xor_sync(0xffffffffu, wa, o);
  }
  if (lane == 0) { red[0][warp] = (double)we; red[1][warp] = (double)wa; }
  __syncthreads();
  if (tid == 0) {
    double te = 0.0, ta = 0.0;
    for (int w = 0; w < 8; ++w) { te += red[0][w]; ta += red[1][w]; }
    a.part[2 * (int64_t)u] = te;
    a.part[2 * (int64_t)u + 1] = ta;
    __threadfence();
    const int units_s = a.unit_ptr[s + 1] - a.unit_ptr[s];
    last_sub = (atomicAdd(&a.sub_cnt[s], 1) == units_s - 1);
  }
  __syncthreads();
  if (!last_sub || warp != 0) return;
  error_fold_subdomain(a, s, lane);
}

}  // namespace

size_t error_smem_bytes(int k_max, int col_block, bool fp64) {
  return (fp64 ? 8 : 4) * (size_t)k_max * (col_block + kErrTile) + 16;
}

cudaError_t launch_error(const ErrArgs& a, int units, bool fp64, cudaStream_t st) {
  if (units <= 0) return cudaSuccess;
  if (a.row_block < kErrTile || a.row_block % kErrTile ||
      (a.col_block != 64 && a.col_block != 128 && a.col_block != 256))
    return cudaErrorInvalidValue;
  const size_t smem = error_smem_bytes(a.k_max, a.col_block, fp64);
  cudaError_t e = cudaSuccess;
#define SPID_LAUNCH_ERR(T, W, CB)                                                           \
  do {                                                                                      \
    e = cudaFuncSetAttribute(error_kernel<T, W, CB>,                                        \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);       \
    if (e != cudaSuccess) return e;                                                         \
    error_kernel<T, W, CB><<<units, 256, smem, st>>>(a);                                    \
  } while (0)
  const bool w = a.out != nullptr;
#define SPID_LAUNCH_ERR_CB(T, W)                                   \
  do {                                                             \
    if (a.col_block == 256) SPID_LAUNCH_ERR(T, W, 256);            \
    else if (a.col_block == 128) SPID_LAUNCH_ERR(T, W, 128);       \
    else SPID_LAUNCH_ERR(T, W, 64);                                \
  } while (0)
  if (fp64) {
    if (w) SPID_LAUNCH_ERR_CB(double, true); else SPID_LAUNCH_ERR_CB(double, false);
  } else {
    if (w) SPID_LAUNCH_ERR_CB(float, true); else SPID_LAUNCH_ERR_CB(float, false);
  }
#undef SPID_LAUNCH_ERR_CB
#undef SPID_LAUNCH_ERR
  return cudaGetLastError();
}

}  // namespace spid
