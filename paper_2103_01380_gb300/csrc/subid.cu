// subid.cu -- the coarse-grid column ID of Section 2 (SubID and SPID
// paragraphs, Algorithms 2 and 3) and the trilinear reconstruction of
// Section 5.2, FP32:
//   subsample    B = A(J, :), the rows of the coarse grid of every box
//   subid_qr     pivoted modified Gram-Schmidt QR of B (the paper's mgsqr),
//                rank decision, C_B = [I | R11^-1 R12] Z^T, skeleton B(:, I_B)
//   coarse_recon G = B(:, I_B) C_B on the coarse grid
//   spid_interp  A_hat = M G (trilinear) fused with ||A - A_hat||^2, ||A||^2
//
// The QR runs one CTA per subdomain with B's working copy in global memory
// (L2-resident at these sizes): every step picks the active column of largest
// residual norm (ties to the lowest index), turns it into q_j in shared
// memory, and one warp per remaining column computes R(j, c) = q_j . w_c,
// updates w_c -= R(j, c) q_j and recomputes ||w_c||^2 from the updated
// values -- the residual norms are therefore taken from the current columns
// at every step, as in the oracle, with no downdating.
#include "error_fold.cuh"
#include "subid_internal.cuh"

namespace spid {

namespace {

constexpr int kQrThreads = 512;
constexpr int kQrWarps = kQrThreads / 32;

__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int coarse_index(int a, int s, int e) { return min(a * s, e - 1); }

// ---------------------------------------------------------------- subsample
__global__ void __launch_bounds__(256) subsample_kernel(const SubArgs a, const float* window,
                                                        int col0, int ncols) {
  const int s = blockIdx.y;
  const int c1 = min(col0 + ncols, a.n[s]);
  if (c1 <= col0) return;
  const SubBox b = a.box[s];
  const int mc = a.mc[s];
  const int64_t work = (int64_t)mc * (c1 - col0);
  const float* A = window + a.off[s];
  const int64_t ld = a.ld[s];
  float* B = a.B + a.boff[s];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < work;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int j = col0 + (int)(e / mc);
    const int cr = (int)(e % mc);
    int t = cr;
    const int cx = t % b.cx;
    t /= b.cx;
    const int cy = t % b.cy;
    t /= b.cy;
    const int cz = t % b.cz;
    const int q = t / b.cz;
    const int64_t r = (((int64_t)q * b.ez + coarse_index(cz, b.sz, b.ez)) * b.ey +
                       coarse_index(cy, b.sy, b.ey)) * b.ex + coarse_index(cx, b.sx, b.ex);
    B[(int64_t)j * mc + cr] = A[(int64_t)j * ld + r];
  }
}

// ---------------------------------------------------------------- pivoted MGS QR
// Double-float back-substitution T = R11^-1 r for one column (FP64-class
// accuracy on the FP32 pipe): every t_i is an unevaluated pair (th, tl), the
// products R_ip t_p are split exactly with fma and summed error-free, and the
// division is corrected by one residual step.
__device__ void df_back_substitute(const float* R11, int k, float* th, float* tl,
                                   const float* rhs) {
  for (int i = k - 1; i >= 0; --i) {
    float hi = rhs[i], lo = 0.f;
    for (int p = i + 1; p < k; ++p) {
      const float Rv = R11[i * k + p];
      const float prod = Rv * th[p];
      const float perr = fmaf(Rv, th[p], -prod) + Rv * tl[p];
      const float sum = hi - prod;                      // two-sum of hi and -prod
      const float bb = sum - hi;
      float err = (hi - (sum - bb)) + (-prod - bb);
      err += lo - perr;
      hi = sum + err;
      lo = err - (hi - sum);
    }
    const float d = R11[i * k + i];
    const float q = hi / d;
    const float res = fmaf(-q, d, hi) + lo;
    const float ql = res / d;
    th[i] = q + ql;
    tl[i] = ql - (th[i] - q);
  }
}

__global__ void __launch_bounds__(kQrThreads, 1) subid_qr_kernel(const SubArgs a, int n_max,
                                                                 int qv_floats) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* qv = reinterpret_cast<float*>(smem_raw);          // q_j [mc], later R11 [k x k]
  float* nu = qv + qv_floats;                              // residual norms^2 [n]
  int32_t* step = reinterpret_cast<int32_t*>(nu + n_max);  // -1 active, >= 0 pivot step
  __shared__ unsigned long long wkey[kQrWarps];
  __shared__ double wrest[kQrWarps];
  __shared__ double normB2_s;
  __shared__ int32_t Js[kSubMaxK];

  const int s = blockIdx.x;
  const int n = a.n[s], mc = a.mc[s], k_max = a.k_max;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const float* B = a.B + a.boff[s];
  float* W = a.W + a.boff[s];
  float* R = a.R + (int64_t)k_max * a.coff[s];
  float* C = a.C + (int64_t)k_max * a.coff[s];
  float* Bsk = a.Bskel + (int64_t)k_max * a.sklo[s];
  int32_t* J = a.J + (int64_t)s * k_max;

  for (int64_t e = tid; e < (int64_t)k_max * n; e += kQrThreads) R[e] = 0.f;
  // W = B and the initial column norms; non-finite check
  bool bad = false;
  for (int c = warp; c < n; c += kQrWarps) {
    float acc = 0.f;
    for (int i = lane; i < mc; i += 32) {
      const float x = B[(int64_t)c * mc + i];
      W[(int64_t)c * mc + i] = x;
      acc = fmaf(x, x, acc);
      bad |= !isfinite(x);
    }
    acc = warp_sum(acc);
    if (lane == 0) {
      nu[c] = acc;
      step[c] = -1;
    }
  }
  if (__syncthreads_or(bad)) {
    if (tid == 0) {
      raise_status(a.status, kStatusNonfinite);
      a.k[s] = 0;
    }
    for (int p = tid; p < k_max; p += kQrThreads) J[p] = -1;
    for (int64_t e = tid; e < (int64_t)k_max * n; e += kQrThreads) C[e] = 0.f;
    for (int64_t e = tid; e < (int64_t)k_max * mc; e += kQrThreads) Bsk[e] = 0.f;
    return;
  }
  if (warp == 0) {   // ||B||_F^2 in a fixed order
    double t = 0.0;
    for (int c = lane; c < n; c += 32) t += (double)nu[c];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) normB2_s = t;
  }
  __syncthreads();
  const double normB2 = normB2_s;
  const double tol2 = a.tol * a.tol;
  int kcap = k_max;
  if (kcap > n) kcap = n;
  if (kcap > mc) kcap = mc;
  int k = 0;
  float r00 = 0.f;
  for (int j = 0; j < kcap; ++j) {
    // ---- pivot: largest residual norm^2 among active columns, lowest index on ties
    unsigned long long key = 0ull;
    double rest = 0.0;
    for (int c = tid; c < n; c += kQrThreads) {
      if (step[c] != -1) continue;
      rest += (double)nu[c];
      const unsigned long long kc =
          ((unsigned long long)__float_as_uint(nu[c]) << 32) | (0xffffffffu - (uint32_t)c);
      key = kc > key ? kc : key;
    }
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key, o);
      key = ok > key ? ok : key;
      rest += __shfl_xor_sync(0xffffffffu, rest, o);
    }
    if (lane == 0) { wkey[warp] = key; wrest[warp] = rest; }
    __syncthreads();
    key = 0ull;
    rest = 0.0;
    for (int w = 0; w < kQrWarps; ++w) {
      key = wkey[w] > key ? wkey[w] : key;
      rest += wrest[w];
    }
    // every thread takes the same decisions from the same shared values
    if (tol2 > 0.0 && rest <= tol2 * normB2) break;
    if (key == 0ull) break;
    const int p = (int)(0xffffffffu - (uint32_t)(key & 0xffffffffull));
    const float nu_p = __uint_as_float((uint32_t)(key >> 32));
    if (!(nu_p > 0.f)) break;
    const float rjj = sqrtf(nu_p);
    if (j == 0) r00 = rjj;
    else if (!(rjj > 0x1p-23f * r00)) break;   // rank guard |R_jj| > 2 u |R_00|, u = 2^-24
    // ---- q_j = w_p / R_jj
    for (int i = tid; i < mc; i += kQrThreads) qv[i] = W[(int64_t)p * mc + i] / rjj;
    if (tid == 0) {
      J[j] = p;
      Js[j] = p;
      R[(int64_t)j * n + p] = rjj;
      step[p] = j;
    }
    __syncthreads();
    // ---- modified Gram-Schmidt against q_j, norms from the updated columns
    for (int c = warp; c < n; c += kQrWarps) {
      if (step[c] != -1) continue;   // warp-uniform
      float* w = W + (int64_t)c * mc;
      float d = 0.f;
      for (int i = lane; i < mc; i += 32) d = fmaf(qv[i], w[i], d);
      d = warp_sum(d);
      float acc = 0.f;
      for (int i = lane; i < mc; i += 32) {
        const float v = fmaf(-d, qv[i], w[i]);
        w[i] = v;
        acc = fmaf(v, v, acc);
      }
      acc = warp_sum(acc);
      if (lane == 0) {
        R[(int64_t)j * n + c] = d;
        nu[c] = acc;
      }
    }
    __syncthreads();
    k = j + 1;
  }
  // ---- rank, pivots, coefficients
  if (tid == 0) a.k[s] = k;
  for (int p = k + tid; p < k_max; p += kQrThreads) J[p] = -1;
  float* R11 = qv;   // q_j is no longer needed
  for (int e = tid; e < k * k; e += kQrThreads) {
    const int i = e / k, p = e % k;
    R11[e] = R[(int64_t)i * n + Js[p]];
  }
  __syncthreads();
  for (int c = tid; c < n; c += kQrThreads) {
    const int st = step[c];
    if (st >= 0) {
      for (int i = 0; i < k_max; ++i) C[(int64_t)i * n + c] = (i == st) ? 1.f : 0.f;
      continue;
    }
    float rhs[kSubMaxK], th[kSubMaxK], tl[kSubMaxK];
    for (int i = 0; i < k; ++i) rhs[i] = R[(int64_t)i * n + c];
    df_back_substitute(R11, k, th, tl, rhs);
    for (int i = 0; i < k_max; ++i) C[(int64_t)i * n + c] = (i < k) ? th[i] : 0.f;
  }
  // ---- coarse skeleton B(:, I_B)
  for (int64_t e = tid; e < (int64_t)k_max * mc; e += kQrThreads) {
    const int p = (int)(e / mc), i = (int)(e % mc);
    Bsk[e] = (p < k) ? B[(int64_t)Js[p] * mc + i] : 0.f;
  }
}

// ---------------------------------------------------------------- coarse reconstruction
__global__ void __launch_bounds__(256) coarse_recon_kernel(const SubArgs a) {
  const int s = blockIdx.y;
  const int mc = a.mc[s], n = a.n[s], k = a.k[s], k_max = a.k_max;
  const float* Bsk = a.Bskel + (int64_t)k_max * a.sklo[s];
  const float* C = a.C + (int64_t)k_max * a.coff[s];
  float* G = a.W + a.boff[s];
  const int64_t work = (int64_t)mc * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < work;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / mc), cr = (int)(e % mc);
    float v = 0.f;
    for (int p = 0; p < k; ++p) v = fmaf(Bsk[(int64_t)p * mc + cr], C[(int64_t)p * n + j], v);
    G[e] = v;
  }
}

// ---------------------------------------------------------------- trilinear reconstruction + error
// Cell of fine coordinate x on an axis of e points, interval s, c coarse
// points: lower coarse index a (the last cell for the end point) and the
// upper node's weight.
__device__ __forceinline__ void axis_cell(int x, int e, int s, int c, int32_t& a, float& w) {
  if (c < 2) { a = 0; w = 0.f; return; }
  a = min(x / s, c - 2);
  const int x0 = coarse_index(a, s, e), x1 = coarse_index(a + 1, s, e);
  w = (float)(x - x0) / (float)(x1 - x0);
}

__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

template <bool WRITE>
__global__ void __launch_bounds__(256) spid_interp_kernel(const SubErrArgs args, int mc_max,
                                                          int e_max) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[2][8];
  __shared__ int last_sub;
  const SubArgs& a = args.a;
  const ErrArgs& e = args.e;
  float* g = reinterpret_cast<float*>(smem_raw);                  // G(:, j) [mc]
  int32_t* tab_a = reinterpret_cast<int32_t*>(g + mc_max);        // [3][e_max] cells z, y, x
  float* tab_w = reinterpret_cast<float*>(tab_a + 3 * e_max);     // [3][e_max] weights
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int u = blockIdx.x;
  // subdomain of unit u (binary search over the unit prefix)
  int lo = 0, hi = a.S;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (e.unit_ptr[mid] <= u) lo = mid; else hi = mid;
  }
  const int s = lo;
  const SubBox b = a.box[s];
  const int mc = a.mc[s];
  const int rel = u - e.unit_ptr[s];
  const int j = rel / b.zblocks;
  const int z0 = (rel % b.zblocks) * b.zc, z1 = min(b.ez, z0 + b.zc);
  const float* G = a.W + a.boff[s] + (int64_t)j * mc;
  for (int i = tid; i < mc; i += blockDim.x) g[i] = G[i];
  for (int x = tid; x < b.ez; x += blockDim.x) axis_cell(x, b.ez, b.sz, b.cz, tab_a[x], tab_w[x]);
  for (int x = tid; x < b.ey; x += blockDim.x)
    axis_cell(x, b.ey, b.sy, b.cy, tab_a[e_max + x], tab_w[e_max + x]);
  for (int x = tid; x < b.ex; x += blockDim.x)
    axis_cell(x, b.ex, b.sx, b.cx, tab_a[2 * e_max + x], tab_w[2 * e_max + x]);
  __syncthreads();
  const int64_t colbase = a.off[s] + (int64_t)j * a.ld[s];
  const bool have_a = args.window != nullptr;
  const float* A = have_a ? args.window + colbase : nullptr;
  const int plane = b.ey * b.ex;
  float se = 0.f, ce = 0.f, sa = 0.f, ca = 0.f;
  for (int pxy = tid; pxy < plane; pxy += blockDim.x) {
    const int y = pxy / b.ex, x = pxy - (pxy / b.ex) * b.ex;
    const int ay = tab_a[e_max + y], ax = tab_a[2 * e_max + x];
    const float wy = tab_w[e_max + y], wx = tab_w[2 * e_max + x];
    const int ay1 = min(ay + 1, b.cy - 1), ax1 = min(ax + 1, b.cx - 1);
    const float w00 = (1.f - wy) * (1.f - wx), w01 = (1.f - wy) * wx;
    const float w10 = wy * (1.f - wx), w11 = wy * wx;
    float le = 0.f, la = 0.f;
    for (int q = 0; q < b.nq; ++q) {
      for (int z = z0; z < z1; ++z) {
        const int az = tab_a[z], az1 = min(az + 1, b.cz - 1);
        const float wz = tab_w[z];
        const int p0 = (q * b.cz + az) * b.cy, p1 = (q * b.cz + az1) * b.cy;
        const float lo_z = w00 * g[(p0 + ay) * b.cx + ax] + w01 * g[(p0 + ay) * b.cx + ax1] +
                           w10 * g[(p0 + ay1) * b.cx + ax] + w11 * g[(p0 + ay1) * b.cx + ax1];
        const float hi_z = w00 * g[(p1 + ay) * b.cx + ax] + w01 * g[(p1 + ay) * b.cx + ax1] +
                           w10 * g[(p1 + ay1) * b.cx + ax] + w11 * g[(p1 + ay1) * b.cx + ax1];
        const float v = fmaf(wz, hi_z - lo_z, lo_z);
        const int64_t r = ((int64_t)q * b.ez + z) * plane + pxy;
        const float av = have_a ? __ldg(A + r) : 0.f;   // reconstruction alone needs no A
        const float d = av - v;
        le = fmaf(d, d, le);
        la = fmaf(av, av, la);
        if (WRITE) args.out[colbase + r] = v;
      }
    }
    kahan_add(se, ce, le);
    kahan_add(sa, ca, la);
  }
  // CTA partial: warp tree in FP32, FP64 across warps, then the fixed-order fold
  float we = se - ce, wa = sa - ca;
  for (int o = 16; o > 0; o >>= 1) {
    we += __shfl_xor_sync(0xffffffffu, we, o);
    wa += __shfl_xor_sync(0xffffffffu, wa, o);
  }
  if (lane == 0) { red[0][warp] = (double)we; red[1][warp] = (double)wa; }
  __syncthreads();
  if (tid == 0) {
    double te = 0.0, ta = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) { te += red[0][w]; ta += red[1][w]; }
    e.part[2 * (int64_t)u] = te;
    e.part[2 * (int64_t)u + 1] = ta;
    __threadfence();
    const int units_s = e.unit_ptr[s + 1] - e.unit_ptr[s];
    last_sub = (atomicAdd(&e.sub_cnt[s], 1) == units_s - 1);
  }
  __syncthreads();
  if (!last_sub || warp != 0) return;
  error_fold_subdomain(e, s, lane);
}

int grid_for(int64_t work) {
  const int64_t blocks = (work + 255) / 256;
  return (int)(blocks < 1 ? 1 : (blocks > 1024 ? 1024 : blocks));
}

}  // namespace

cudaError_t launch_subsample(const SubArgs& a, const float* window, int col0, int ncols,
                             int64_t max_work, cudaStream_t st) {
  if (max_work <= 0) return cudaSuccess;
  subsample_kernel<<<dim3(grid_for(max_work), a.S), 256, 0, st>>>(a, window, col0, ncols);
  return cudaGetLastError();
}

size_t subid_qr_smem_bytes(int mc_max, int n_max, int k_max) {
  const int qv = mc_max > k_max * k_max ? mc_max : k_max * k_max;
  return sizeof(float) * ((size_t)qv + n_max) + sizeof(int32_t) * (size_t)n_max;
}

cudaError_t launch_subid_qr(const SubArgs& a, int mc_max, int n_max, cudaStream_t st) {
  const int qv = mc_max > a.k_max * a.k_max ? mc_max : a.k_max * a.k_max;
  const size_t smem = subid_qr_smem_bytes(mc_max, n_max, a.k_max);
  cudaError_t e = cudaFuncSetAttribute(subid_qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  subid_qr_kernel<<<a.S, kQrThreads, smem, st>>>(a, n_max, qv);
  return cudaGetLastError();
}

cudaError_t launch_coarse_recon(const SubArgs& a, int64_t max_work, cudaStream_t st) {
  if (max_work <= 0) return cudaSuccess;
  coarse_recon_kernel<<<dim3(grid_for(max_work), a.S), 256, 0, st>>>(a);
  return cudaGetLastError();
}

size_t spid_interp_smem_bytes(int mc_max, int e_max) {
  return sizeof(float) * (size_t)mc_max + 3 * (sizeof(int32_t) + sizeof(float)) * (size_t)e_max;
}

cudaError_t launch_spid_interp(const SubErrArgs& a, int64_t units, int mc_max, int e_max,
                               cudaStream_t st) {
  if (units <= 0) return cudaSuccess;
  const size_t smem = spid_interp_smem_bytes(mc_max, e_max);
  cudaError_t e;
  if (a.out) {
    e = cudaFuncSetAttribute(spid_interp_kernel<true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    spid_interp_kernel<true><<<(unsigned)units, 256, smem, st>>>(a, mc_max, e_max);
  } else {
    e = cudaFuncSetAttribute(spid_interp_kernel<false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    spid_interp_kernel<false><<<(unsigned)units, 256, smem, st>>>(a, mc_max, e_max);
  }
  return cudaGetLastError();
}

}  // namespace spid
