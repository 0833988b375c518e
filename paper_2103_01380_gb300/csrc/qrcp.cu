// qrcp.cu -- batched column-pivoted QR of the sketches, rank decision and
// coefficients (Section 2: A Z = Q R, C = [I_k | R11^-1 R12] Z^T; Algorithm 1
// steps 3-6 applied to the sketch as in Algorithm 2; adaptive rank per
// Remark 2.1).
//
// One CTA per subdomain.  Thread t owns CPT columns of Y_s and keeps each of
// them (l_pad values) in registers for the whole factorization, so a
// Householder step costs one broadcast of the reflector through shared memory
// plus a dot product and an axpy per column.  Pivoting never moves data: the
// pivot column's owner publishes the reflector, and the column is retired.
//   - pivot = largest residual norm^2, ties to the lowest column index.  The
//     norms carry FP64-class precision without the FP64 pipe (GB300 runs FP64
//     at 1/64 of FP32): in FP32 modes each norm is an unevaluated sum of two
//     floats (hi + lo, ~48-bit significand) built from exact products
//     (fma) and error-free additions; it is downdated by the exact square of
//     the new R entry at every step and recomputed from the remaining rows
//     whenever it has lost two digits.  In FP64 mode the norms are doubles.
//     The argmax compares the (hi, lo) pairs exactly with integer redux.
//   - adaptive stop: smallest k with sum of residual norms^2 <= tol^2 ||Y||_F^2;
//   - rank guard: keep leading pivots with |R_jj| > 2 u |R_00|;
//   - T = R11^-1 R12 by back-substitution with FP64-class accuracy (double-
//     float on the FP32 pipe in FP32 modes, FP64 in FP64 mode), one thread per
//     column, in place; C(:, J) = I exactly.
#include "spid_internal.cuh"

namespace spid {

namespace {

constexpr int kMaxWarps = 16;

// ---------------------------------------------------------------------------
// Residual norms: a double-float in FP32 modes, a double in FP64 mode.
// ---------------------------------------------------------------------------
template <typename T> struct Norm;

template <> struct Norm<float> {
  float hi, lo;
  // error-free a + b = s + e (Knuth two-sum)
  static __device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
  }
  __device__ __forceinline__ void set_zero() { hi = 0.f; lo = 0.f; }
  // += y^2 with the product exact (fma) and the sum compensated
  __device__ __forceinline__ void add_square(float y) {
    const float p = y * y;
    const float pe = fmaf(y, y, -p);
    float s, e;
    two_sum(hi, p, s, e);
    e += lo + pe;
    hi = s + e;
    lo = e - (hi - s);
  }
  // -= y^2, exactly rounded to the pair
  __device__ __forceinline__ void sub_square(float y) {
    const float p = y * y;
    const float pe = fmaf(y, y, -p);
    float s, e;
    two_sum(hi, -p, s, e);
    e += lo - pe;
    hi = s + e;
    lo = e - (hi - s);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
  __device__ __forceinline__ bool below(const Norm& floor) const { return hi < floor.hi; }
  __device__ __forceinline__ Norm scaled(float f) const { return Norm{hi * f, lo * f}; }
  // order-preserving 64-bit key of a non-negative value (hi, then lo)
  static __device__ __forceinline__ uint32_t okey(float x) {
    const uint32_t b = __float_as_uint(x);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
  }
  __device__ __forceinline__ void key(uint32_t& k0, uint32_t& k1) const {
    if (!(hi > 0.f)) { k0 = 0u; k1 = 0u; return; }
    k0 = okey(hi);
    k1 = okey(lo);
  }
};

template <> struct Norm<double> {
  double hi;
  __device__ __forceinline__ void set_zero() { hi = 0.0; }
  __device__ __forceinline__ void add_square(double y) { hi = fma(y, y, hi); }
  __device__ __forceinline__ void sub_square(double y) { hi = fma(-y, y, hi); }
  __device__ __forceinline__ double value() const { return hi; }
  __device__ __forceinline__ bool below(const Norm& floor) const { return hi < floor.hi; }
  __device__ __forceinline__ Norm scaled(double f) const { return Norm{hi * f}; }
  __device__ __forceinline__ void key(uint32_t& k0, uint32_t& k1) const {
    if (!(hi > 0.0)) { k0 = 0u; k1 = 0u; return; }
    const unsigned long long b = (unsigned long long)__double_as_longlong(hi);
    k0 = (uint32_t)(b >> 32);
    k1 = (uint32_t)b;
  }
};

struct PivotKey {
  uint32_t k0, k1, col;
};

// Warp argmax of (k0, k1) with ties to the lowest column: three integer redux.
__device__ __forceinline__ PivotKey warp_pivot(uint32_t k0, uint32_t k1, uint32_t col) {
  const uint32_t m0 = __reduce_max_sync(0xffffffffu, k0);
  const uint32_t m1 = __reduce_max_sync(0xffffffffu, k0 == m0 ? k1 : 0u);
  const uint32_t mc = __reduce_min_sync(0xffffffffu, (k0 == m0 && k1 == m1) ? col : 0xffffffffu);
  return {m0, m1, mc};
}


// T = R11^-1 r in place over r[0 .. keff), FP64-class accuracy.
// FP32 data: every t_l is carried as an unevaluated pair (hi, lo), each product
// R_il t_l is split exactly with fma, and the running residual is an
// error-free double-float sum; the division is corrected by one residual
// step.  All on the FP32 pipe.  FP64 data: plain FP64.
// The loops run over keff only (usually a handful of pivots): the column is
// copied to a per-thread array indexed at run time, so the code stays small
// -- a fully unrolled LP x LP triangle is fetched almost entirely even when
// only its first rows execute, and instruction fetch then dominates the QR.
template <int LP>
__device__ __noinline__ void back_substitute(float (&r)[LP], const float (&R)[LP][LP], int keff) {
  float th[LP], tl[LP];
#pragma unroll
  for (int i = 0; i < LP; ++i) {
    th[i] = r[i];
    tl[i] = 0.f;
  }
  for (int ii = keff - 1; ii >= 0; --ii) {
    float hi = th[ii], lo = 0.f;
    for (int ll = ii + 1; ll < keff; ++ll) {
      const float Rv = R[ii][ll];
      const float p = Rv * th[ll];
      float pe = fmaf(Rv, th[ll], -p);
      pe = fmaf(Rv, tl[ll], pe);
      // (hi, lo) -= (p, pe)
      const float s = hi - p;
      const float bb = s - hi;
      float e = (hi - (s - bb)) + (-p - bb);
      e += lo - pe;
      hi = s + e;
      lo = e - (hi - s);
    }
    const float d = R[ii][ii];
    const float q = hi / d;
    const float res = fmaf(-q, d, hi) + lo;
    const float ql = res / d;
    th[ii] = q + ql;
    tl[ii] = ql - (th[ii] - q);
  }
#pragma unroll
  for (int i = 0; i < LP; ++i) r[i] = th[i];
}

template <int LP>
__device__ __noinline__ void back_substitute(double (&r)[LP], const double (&R)[LP][LP], int keff) {
  double t[LP];
#pragma unroll
  for (int i = 0; i < LP; ++i) t[i] = r[i];
  for (int ii = keff - 1; ii >= 0; --ii) {
    double acc = t[ii];
    for (int ll = ii + 1; ll < keff; ++ll) acc = fma(-R[ii][ll], t[ll], acc);
    t[ii] = acc / R[ii][ii];
  }
#pragma unroll
  for (int i = 0; i < LP; ++i) r[i] = t[i];
}

template <typename T, int LP, int CPT>
__global__ void __launch_bounds__(512) qrcp_kernel(QrcpArgs a) {
  __shared__ __align__(16) T vs[2][LP];   // Householder vector, double-buffered by step parity
  __shared__ T beta_s[2];
  __shared__ T R11[LP][LP];            // R11(i, p) = R(i, J[p])
  __shared__ int Js[LP];
  __shared__ uint4 red_key[2][kMaxWarps];
  __shared__ T guard_thr;              // 2 u |R_00|
  __shared__ int stop_s[2];            // the pivot of this step failed the rank guard
  __shared__ double red_rest[2][kMaxWarps];

  const int s = blockIdx.x + a.sub_base;
  const int n = a.n[s];
  const int NT = blockDim.x;
  const int tid = threadIdx.x;
  const int warp = tid / 32, lane = tid % 32, nwarps = NT / 32;
  int kcap = a.k_max;
  if (kcap > a.l) kcap = a.l;
  if (kcap > n) kcap = n;
  const bool adaptive = a.tol > 0.0;

  const T* Y = static_cast<const T*>(a.Y) + a.yoff[s];
  T y[CPT][LP];
  Norm<T> nu[CPT], nu_floor[CPT];
  int step_of[CPT];
  bool bad = false;
#pragma unroll
  for (int c = 0; c < CPT; ++c) {
    const int col = tid + c * NT;
    step_of[c] = (col < n) ? -1 : -2;   // -1 active, -2 no column, >= 0 pivot step
    nu[c].set_zero();
    // the column is LP contiguous values (16-byte aligned: LP is a multiple of 16)
    constexpr int VW = 16 / sizeof(T);
#pragma unroll
    for (int i4 = 0; i4 < LP; i4 += VW) {
      typename Vec16<T>::type v = Vec16<T>::zero();
      if (col < n)
        v = __ldg(reinterpret_cast<const typename Vec16<T>::type*>(Y + (int64_t)col * LP + i4));
      const T* vs_ = reinterpret_cast<const T*>(&v);
      // rows at and past l (a plan may sketch more rows of Omega than its QR reads)
#pragma unroll
      for (int u = 0; u < VW; ++u) y[c][i4 + u] = (i4 + u < a.l) ? vs_[u] : T(0);
    }
#pragma unroll
    for (int i = 0; i < LP; ++i) {
      if (!isfinite(y[c][i])) bad = true;
      nu[c].add_square(y[c][i]);
    }
    nu_floor[c] = nu[c].scaled(T(1e-2));
  }
  T* C = static_cast<T*>(a.C) + a.coff[s];
  if (__syncthreads_or(bad)) {
    if (tid == 0) {
      raise_status(a.status, kStatusNonfinite);
      a.k_out[s] = 0;
    }
    for (int i = tid; i < a.k_max; i += NT) a.J[(int64_t)s * a.k_max + i] = -1;
    for (int64_t e = tid; e < (int64_t)a.k_max * n; e += NT) C[e] = T(0);
    return;
  }
  // ||Y||_F^2, fixed-order block sum (adaptive mode only)
  double normY2 = 0.0;
  if (adaptive) {
    double t = 0.0;
#pragma unroll
    for (int c = 0; c < CPT; ++c)
      if (step_of[c] == -1) t += nu[c].value();
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red_rest[1][warp] = t;
    __syncthreads();
    for (int w = 0; w < nwarps; ++w) normY2 += red_rest[1][w];
  }
  const double tol2 = a.tol * a.tol;

  int k = 0;
  bool guard_stop = false;   // the guard ended the factorization before its target
  for (int j = 0; j < kcap; ++j) {
    const int par = j & 1;
    // ---- argmax of the residual norms^2 (exact on the pairs, ties -> lowest column)
    uint32_t b0 = 0u, b1 = 0u, bcol = 0xffffffffu;
    double rest = 0.0;
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      if (step_of[c] != -1) continue;
      uint32_t k0, k1;
      nu[c].key(k0, k1);
      if (adaptive) rest += nu[c].value();
      if (bcol == 0xffffffffu || k0 > b0 || (k0 == b0 && k1 > b1)) {
        b0 = k0; b1 = k1; bcol = (uint32_t)(tid + c * NT);
      }
    }
    const PivotKey wk = warp_pivot(b0, b1, bcol);
    if (adaptive)
      for (int o = 16; o > 0; o >>= 1) rest += __shfl_xor_sync(0xffffffffu, rest, o);
    if (lane == 0) {
      red_key[par][warp] = make_uint4(wk.k0, wk.k1, wk.col, 0u);
      red_rest[par][warp] = rest;
    }
    __syncthreads();
    // every warp reduces the per-warp winners itself (no second barrier)
    const uint4 q = (lane < nwarps) ? red_key[par][lane] : make_uint4(0u, 0u, 0xffffffffu, 0u);
    const PivotKey best = warp_pivot(q.x, q.y, q.z);
    if (adaptive) {
      double trest = 0.0;
      for (int w = 0; w < nwarps; ++w) trest += red_rest[par][w];
      if (trest <= tol2 * normY2) break;
    }
    if ((best.k0 | best.k1) == 0u || best.col == 0xffffffffu) break;   // residual is zero
    const int pcol = (int)best.col;
    // ---- the owner of the pivot column builds the reflector (working precision)
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      if (tid + c * NT != pcol) continue;
      T sp[4] = {T(0), T(0), T(0), T(0)}, xj = T(0);   // four chains: short latency
#pragma unroll
      for (int i = 0; i < LP; ++i) {
        if (i > j) sp[i & 3] = fma(y[c][i], y[c][i], sp[i & 3]);
        if (i == j) xj = y[c][i];
      }
      const T sig = (sp[0] + sp[1]) + (sp[2] + sp[3]);
      const T norm = sqrt(fma(xj, xj, sig));
      const T alpha = (xj >= T(0)) ? -norm : norm;
      // rank guard, applied as the pivots are produced: it keeps a leading
      // prefix, so the first R_jj at or below 2 u |R_00| ends the factorization
      if (j == 0) guard_thr = (T)(2.0 * a.u_mode) * abs(alpha);
      const bool stop = (j == 0) ? !(abs(alpha) > T(0)) : !(abs(alpha) > guard_thr);
      stop_s[par] = stop ? 1 : 0;
      if (stop) continue;
      const T vj = xj - alpha;
      const T vtv = fma(vj, vj, sig);
      beta_s[par] = (vtv > T(0)) ? T(2) / vtv : T(0);
#pragma unroll
      for (int i = 0; i < LP; ++i) {
        if (i < j) { vs[par][i] = T(0); R11[i][j] = y[c][i]; }
        else if (i == j) { vs[par][i] = vj; R11[j][j] = alpha; }
        else vs[par][i] = y[c][i];
      }
      Js[j] = pcol;
      step_of[c] = j;
    }
    __syncthreads();
    if (stop_s[par]) {
      guard_stop = j > 0;
      break;
    }
    // ---- apply H_j = I - beta v v^T to every remaining column (v is zero
    // above row j, so no row predicate is needed); downdate the norm by the
    // new R entry; recompute it from the remaining rows once it lost two digits
    const T beta = beta_s[par];
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      if (step_of[c] != -1) continue;
      T dp[4] = {T(0), T(0), T(0), T(0)};
      constexpr int VW = 16 / sizeof(T);
#pragma unroll
      for (int i4 = 0; i4 < LP; i4 += VW) {
        const typename Vec16<T>::type x = *reinterpret_cast<const typename Vec16<T>::type*>(&vs[par][i4]);
        const T* xs = reinterpret_cast<const T*>(&x);
#pragma unroll
        for (int u = 0; u < VW; ++u) dp[(i4 + u) & 3] = fma(xs[u], y[c][i4 + u], dp[(i4 + u) & 3]);
      }
      const T f = beta * ((dp[0] + dp[1]) + (dp[2] + dp[3]));
      T rj = T(0);
#pragma unroll
      for (int i = 0; i < LP; ++i) {
        y[c][i] = fma(-f, vs[par][i], y[c][i]);
        rj = (i == j) ? y[c][i] : rj;
      }
      nu[c].sub_square(rj);
      if (nu[c].below(nu_floor[c])) {
        // the downdate lost two digits: take the norm of the rows that remain
        // (four independent chains; the stored rows are what the next step sees)
        T sq[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
        for (int i = 0; i < LP; ++i)
          if (i > j) sq[i & 3] = fma(y[c][i], y[c][i], sq[i & 3]);
        nu[c].set_zero();
        nu[c].hi = (sq[0] + sq[1]) + (sq[2] + sq[3]);
        nu_floor[c] = nu[c].scaled(T(1e-2));
      }
    }
    k = j + 1;
  }
  __syncthreads();
  // ---- rank guard
  int keff = 0;
  if (k > 0) {
    const T thr = (T)(2.0 * a.u_mode) * abs(R11[0][0]);
    if (thr > T(0)) {
      for (int j = 0; j < k; ++j) {
        if (abs(R11[j][j]) > thr) keff = j + 1;
        else break;
      }
    }
  }
  if (tid == 0) {
    a.k_out[s] = keff;
    if (guard_stop || keff < k) raise_status(a.status, kStatusRankCut);
  }
  for (int i = tid; i < a.k_max; i += NT) a.J[(int64_t)s * a.k_max + i] = (i < keff) ? Js[i] : -1;
  // ---- coefficients: FP64 back-substitution R11 t = R(0:keff, col), in place
#pragma unroll
  for (int c = 0; c < CPT; ++c) {
    const int col = tid + c * NT;
    if (step_of[c] == -2) continue;
    if (step_of[c] >= 0 && step_of[c] < keff) {
      for (int i = 0; i < a.k_max; ++i) C[(int64_t)i * n + col] = (i == step_of[c]) ? T(1) : T(0);
      continue;
    }
    back_substitute(y[c], R11, keff);
#pragma unroll
    for (int i = 0; i < LP; ++i)
      if (i < a.k_max) C[(int64_t)i * n + col] = (i < keff) ? y[c][i] : T(0);
    for (int i = LP; i < a.k_max; ++i) C[(int64_t)i * n + col] = T(0);
  }
}

template <typename T, int LP, int CPT>
cudaError_t launch_qrcp_t(const QrcpArgs& a, int grid, int threads, cudaStream_t st) {
  qrcp_kernel<T, LP, CPT><<<grid, threads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

// Columns per thread the QR kernel needs for n_max columns (0: unsupported).
int qrcp_cols_per_thread(int n_max, int l_pad, bool fp64) {
  if (n_max <= 512) return 1;
  if (n_max <= 1024 && l_pad <= (fp64 ? 32 : 48)) return 2;
  return 0;
}

cudaError_t launch_qrcp(const QrcpArgs& a, int grid, int n_max, int l_pad, bool fp64,
                        cudaStream_t st) {
  if (grid <= 0) return cudaSuccess;
  const int cpt = qrcp_cols_per_thread(n_max, l_pad, fp64);
  if (cpt == 0) return cudaErrorInvalidValue;
  int threads = (n_max + cpt - 1) / cpt;
  threads = (threads + 31) / 32 * 32;
  if (fp64) {
    if (cpt == 1) {
      switch (l_pad) {
        case 16: return launch_qrcp_t<double, 16, 1>(a, grid, threads, st);
        case 32: return launch_qrcp_t<double, 32, 1>(a, grid, threads, st);
        case 48: return launch_qrcp_t<double, 48, 1>(a, grid, threads, st);
      }
    } else {
      switch (l_pad) {
        case 16: return launch_qrcp_t<double, 16, 2>(a, grid, threads, st);
        case 32: return launch_qrcp_t<double, 32, 2>(a, grid, threads, st);
      }
    }
  } else {
    if (cpt == 1) {
      switch (l_pad) {
        case 16: return launch_qrcp_t<float, 16, 1>(a, grid, threads, st);
        case 32: return launch_qrcp_t<float, 32, 1>(a, grid, threads, st);
        case 48: return launch_qrcp_t<float, 48, 1>(a, grid, threads, st);
        case 64: return launch_qrcp_t<float, 64, 1>(a, grid, threads, st);
      }
    } else {
      switch (l_pad) {
        case 16: return launch_qrcp_t<float, 16, 2>(a, grid, threads, st);
        case 32: return launch_qrcp_t<float, 32, 2>(a, grid, threads, st);
        case 48: return launch_qrcp_t<float, 48, 2>(a, grid, threads, st);
      }
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace spid
