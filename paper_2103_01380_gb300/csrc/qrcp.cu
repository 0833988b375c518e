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
//   - pivot = largest residual norm^2, kept in FP64 by downdating
//     (nu -= R(j,c)^2) and recomputed from the remaining rows (accumulated in
//     the working precision) whenever it has lost two digits; the argmax is
//     exact in FP64 with ties to the lowest column index;
//   - adaptive stop: smallest k with sum of residual norms^2 <= tol^2 ||Y||_F^2;
//   - rank guard: keep leading pivots with |R_jj| > 2 u |R_00|;
//   - T = R11^-1 R12 by FP64 back-substitution, one thread per column, in
//     place; C(:, J) = I exactly.
#include "spid_internal.cuh"

namespace spid {



namespace {

constexpr int kMaxWarps = 16;

// Exact FP64 argmax with ties to the lowest column: the bit pattern of a
// non-negative double orders like the value, so the warp reduces the high
// word, then the low word among the leaders, then the column among the exact
// winners, with three integer redux.sync operations.
struct PivotKey {
  uint32_t hi, lo, col;
};

__device__ __forceinline__ PivotKey warp_pivot(double nu, uint32_t col) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(nu);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const uint32_t mhi = __reduce_max_sync(0xffffffffu, hi);
  const uint32_t mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? lo : 0u);
  const uint32_t mcol = __reduce_min_sync(0xffffffffu, (hi == mhi && lo == mlo) ? col : 0xffffffffu);
  return {mhi, mlo, mcol};
}

__device__ __forceinline__ bool key_better(const PivotKey& a, const PivotKey& b) {
  if (a.hi != b.hi) return a.hi > b.hi;
  if (a.lo != b.lo) return a.lo > b.lo;
  return a.col < b.col;
}

template <typename T, int LP, int CPT>
__global__ void __launch_bounds__(512) qrcp_kernel(QrcpArgs a) {
  __shared__ T vs[2][LP];              // Householder vector, double-buffered by step parity
  __shared__ T beta_s[2];
  __shared__ double R11[LP][LP];       // R11(i, p) = R(i, J[p])
  __shared__ int Js[LP];
  __shared__ uint4 red_key[2][kMaxWarps];
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
  double nu[CPT], nu_floor[CPT];
  int step_of[CPT];
  bool bad = false;
#pragma unroll
  for (int c = 0; c < CPT; ++c) {
    const int col = tid + c * NT;
    step_of[c] = (col < n) ? -1 : -2;   // -1 active, -2 no column, >= 0 pivot step
    T acc = T(0);
#pragma unroll
    for (int i = 0; i < LP; ++i) {
      y[c][i] = (col < n) ? Y[(int64_t)col * LP + i] : T(0);
      if (!isfinite(y[c][i])) bad = true;
      acc = fma(y[c][i], y[c][i], acc);
    }
    nu[c] = (double)acc;
    nu_floor[c] = 1e-2 * nu[c];
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
      if (step_of[c] == -1) t += nu[c];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red_rest[1][warp] = t;
    __syncthreads();
    for (int w = 0; w < nwarps; ++w) normY2 += red_rest[1][w];
  }
  const double tol2 = a.tol * a.tol;

  int k = 0;
  for (int j = 0; j < kcap; ++j) {
    const int par = j & 1;
    // ---- argmax of the residual norms^2 (exact FP64, ties -> lowest column)
    double bnu = -1.0, rest = 0.0;
    uint32_t bcol = 0xffffffffu;
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      if (step_of[c] != -1) continue;
      rest += nu[c];
      if (nu[c] > bnu) { bnu = nu[c]; bcol = (uint32_t)(tid + c * NT); }
    }
    const PivotKey wk = warp_pivot(bnu > 0.0 ? bnu : 0.0, bcol);
    if (adaptive)
      for (int o = 16; o > 0; o >>= 1) rest += __shfl_xor_sync(0xffffffffu, rest, o);
    if (lane == 0) {
      red_key[par][warp] = make_uint4(wk.hi, wk.lo, wk.col, 0u);
      red_rest[par][warp] = rest;
    }
    __syncthreads();
    PivotKey best = {0u, 0u, 0xffffffffu};
    double trest = 0.0;
    for (int w = 0; w < nwarps; ++w) {
      const uint4 q = red_key[par][w];
      const PivotKey kq = {q.x, q.y, q.z};
      if (key_better(kq, best)) best = kq;
      if (adaptive) trest += red_rest[par][w];
    }
    if (adaptive && trest <= tol2 * normY2) break;
    if ((best.hi | best.lo) == 0u || best.col == 0xffffffffu) break;   // residual is zero
    const int pcol = (int)best.col;
    // ---- the owner of the pivot column builds the reflector
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      if (tid + c * NT != pcol) continue;
      double sig = 0.0, xj = 0.0;
#pragma unroll
      for (int i = 0; i < LP; ++i) {
        if (i > j) sig += (double)y[c][i] * (double)y[c][i];
        if (i == j) xj = (double)y[c][i];
      }
      const double norm = sqrt(xj * xj + sig);
      const double alpha = (xj >= 0.0) ? -norm : norm;
      const double vj = xj - alpha;
      const double vtv = vj * vj + sig;
      beta_s[par] = (T)((vtv > 0.0) ? 2.0 / vtv : 0.0);
#pragma unroll
      for (int i = 0; i < LP; ++i) {
        if (i < j) { vs[par][i] = T(0); R11[i][j] = (double)y[c][i]; }
        else if (i == j) { vs[par][i] = (T)vj; R11[j][j] = alpha; }
        else vs[par][i] = y[c][i];
      }
      Js[j] = pcol;
      step_of[c] = j;
    }
    __syncthreads();
    // ---- apply H_j = I - beta v v^T to every remaining column; downdate the
    // FP64 norm; recompute it from the remaining rows once it lost two digits
    const T beta = beta_s[par];
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      if (step_of[c] != -1) continue;
      T dot = T(0);
#pragma unroll
      for (int i = 0; i < LP; ++i)
        if (i >= j) dot = fma(vs[par][i], y[c][i], dot);
      const T f = beta * dot;
      T rj = T(0), tail = T(0);
#pragma unroll
      for (int i = 0; i < LP; ++i) {
        if (i >= j) y[c][i] = fma(-f, vs[par][i], y[c][i]);
        if (i == j) rj = y[c][i];
        if (i > j) tail = fma(y[c][i], y[c][i], tail);
      }
      nu[c] -= (double)(rj * rj);
      if (nu[c] < nu_floor[c]) {
        nu[c] = (double)tail;
        nu_floor[c] = 1e-2 * nu[c];
      }
    }
    k = j + 1;
  }
  __syncthreads();
  // ---- rank guard
  int keff = 0;
  if (k > 0) {
    const double r00 = fabs(R11[0][0]);
    if (r00 > 0.0) {
      for (int j = 0; j < k; ++j) {
        if (fabs(R11[j][j]) > 2.0 * a.u_mode * r00) keff = j + 1;
        else break;
      }
    }
  }
  if (tid == 0) a.k_out[s] = keff;
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
#pragma unroll
    for (int ii = LP - 1; ii >= 0; --ii) {
      if (ii < keff) {
        double acc = (double)y[c][ii];
#pragma unroll
        for (int ll = ii + 1; ll < LP; ++ll)
          if (ll < keff) acc -= R11[ii][ll] * (double)y[c][ll];
        y[c][ii] = (T)(acc / R11[ii][ii]);
      }
    }
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
