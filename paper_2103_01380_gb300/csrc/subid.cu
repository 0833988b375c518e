// subid.cu -- the coarse-grid column ID of Section 2 (SubID and SPID
// paragraphs, Algorithms 2 and 3) and the trilinear reconstruction of
// Section 5.2, FP32:
//   subsample    B = A(J, :), the rows of the coarse grid of every box, with
//                each column's squared norm for the QR's first pivot
//   subid_qr     pivoted modified Gram-Schmidt QR of B (the paper's mgsqr),
//                rank decision, C_B = [I | R11^-1 R12] Z^T, skeleton B(:, I_B)
//   coarse_recon G = B(:, I_B) C_B on the coarse grid
//   spid_interp  A_hat = M G (trilinear) fused with ||A - A_hat||^2, ||A||^2
//   fine_skeleton F = M B(:, I_B), the interpolated skeleton (m x k), so that
//                the error pass is the rank-k product F C_B against A
//
// The QR runs one cluster of up to 8 CTAs per subdomain (the columns dealt
// out to the CTAs' warps) with B's working copy in global memory: every step
// picks the active column of largest residual norm (ties to the lowest
// index; the CTAs exchange their candidates through distributed shared
// memory and take the same decision), turns it into q_j in each CTA's shared
// memory, and one warp per remaining column computes R(j, c) = q_j . w_c,
// updates w_c -= R(j, c) q_j and recomputes ||w_c||^2 from the updated
// values -- the residual norms are therefore taken from the current columns
// at every step, as in the oracle, with no downdating.  W is rewritten only
// every few steps: in between, the pending updates are re-applied as each
// column is read (the same fma sequence, so the same values).
#include <algorithm>

#include <cooperative_groups.h>

#include "error_fold.cuh"
#include "subid_internal.cuh"

namespace cg = cooperative_groups;

namespace spid {

namespace {

constexpr int kQrThreads = 1024;
constexpr int kQrWarps = kQrThreads / 32;
// q_j slots: up to kQrMaxSlots - 1 MGS updates stay pending (re-applied from
// shared memory) before the working copy W is rewritten
constexpr int kQrMaxSlots = 4;
constexpr int kQrSlotBudgetFloats = 24 * 1024;
// the per-warp column buffers are used while the kernel's shared memory stays
// within this (m_c up to ~1400)
constexpr size_t kQrColumnSmemMax = 200 * 1024;

__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int coarse_index(int a, int s, int e) { return min(a * s, e - 1); }

// ---------------------------------------------------------------- subsample
// One warp per (column j, part t): B(rows of part t, j) = A(coarse rows, j)
// and the part's squared norm for the QR's first pivot (NaN when the part
// holds a non-finite entry).  A column's nrm_parts parts split its m_c rows
// evenly; the QR adds them in order.
constexpr int kSampleColsPerBlock = 8;

struct GatherPart {
  int j, t, r0, r1;
};

__device__ __forceinline__ bool gather_part(const SubArgs& a, int s, int col0, int ncols, int mc,
                                            GatherPart& g) {
  const int R = a.nrm_parts;
  const int wg = blockIdx.x * kSampleColsPerBlock + threadIdx.x / 32;
  g.j = col0 + wg / R;
  g.t = wg % R;
  if (g.j >= min(col0 + ncols, a.n[s])) return false;
  const int chunk = (mc + R - 1) / R;
  g.r0 = min(mc, g.t * chunk);
  g.r1 = min(mc, g.r0 + chunk);
  return true;
}

__device__ __forceinline__ void finish_part_norm(const SubArgs& a, int s, const GatherPart& g,
                                                 const float* acc, bool bad, int lane) {
  const float v = warp_sum((acc[0] + acc[1]) + (acc[2] + acc[3]));
  const bool any_bad = __any_sync(0xffffffffu, bad);
  if (lane == 0)
    a.nrm[(a.coff[s] + g.j) * a.nrm_parts + g.t] = any_bad ? __int_as_float(0x7fc00000) : v;
}

__global__ void __launch_bounds__(256) subsample_kernel(const SubArgs a, const float* window,
                                                        int col0, int ncols) {
  const int s = blockIdx.y;
  const int mc = a.mc[s];
  GatherPart g;
  if (!gather_part(a, s, col0, ncols, mc, g)) return;   // warp-uniform; no block barrier below
  const int lane = threadIdx.x % 32;
  const SubBox b = a.box[s];
  const float* Aj = window + a.off[s] + (int64_t)g.j * a.ld[s];
  float* Bj = a.B + a.boff[s] + (int64_t)g.j * coarse_ld(mc);
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  bool bad = false;
  // four independent gathers in flight per lane
  for (int i0 = g.r0 + lane; i0 < g.r1; i0 += 128) {
    float v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int cr = i0 + 32 * u;
      v[u] = 0.f;
      if (cr < g.r1) {
        const int t1 = (int)fdiv((uint32_t)cr, b.div_cx);
        const int cx = cr - t1 * b.cx;
        const int t2 = (int)fdiv((uint32_t)t1, b.div_cy);
        const int cy = t1 - t2 * b.cy;
        const int q = (int)fdiv((uint32_t)t2, b.div_cz);
        const int cz = t2 - q * b.cz;
        const int64_t r = (((int64_t)q * b.ez + coarse_index(cz, b.sz, b.ez)) * b.ey +
                           coarse_index(cy, b.sy, b.ey)) * b.ex + coarse_index(cx, b.sx, b.ex);
        v[u] = __ldg(Aj + r);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int cr = i0 + 32 * u;
      if (cr < g.r1) {
        Bj[cr] = v[u];
        acc[u] = fmaf(v[u], v[u], acc[u]);
        bad |= !isfinite(v[u]);
      }
    }
  }
  finish_part_norm(a, s, g, acc, bad, lane);
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

// Error-free sum of two double-float values (h, l) += (bh, bl): the residual
// norms are summed on the FP32 pipe (FP64 issue is a small fraction of it).
__device__ __forceinline__ void df_add(float& h, float& l, float bh, float bl) {
  const float s = h + bh;
  const float bb = s - h;
  const float e = ((h - (s - bb)) + (bh - bb)) + (l + bl);
  h = s + e;
  l = e - (h - s);
}

// One subdomain's QR runs on a cluster of G CTAs.  Column c belongs to rank
// (c / kQrWarps) % G and, there, to warp c % kQrWarps; o-th column of a rank:
__device__ __forceinline__ int owned_col(int o, int G, int rank) {
  return ((o / kQrWarps) * G + rank) * kQrWarps + o % kQrWarps;
}

__device__ __forceinline__ void fma4(float4& v, float c, const float4 q) {
  v.x = fmaf(c, q.x, v.x);
  v.y = fmaf(c, q.y, v.y);
  v.z = fmaf(c, q.z, v.z);
  v.w = fmaf(c, q.w, v.w);
}
__device__ __forceinline__ float dot4(const float4 q, const float4 v, float acc) {
  return fmaf(q.w, v.w, fmaf(q.z, v.z, fmaf(q.y, v.y, fmaf(q.x, v.x, acc))));
}

// One column's MGS step j with the updates of steps base..base+NP-1 still
// pending: the column is read as stored (B, or W as of step base), the pending
// updates w -= R(t, c) q_t are re-applied on the fly -- the same fma sequence
// as if every step had been stored, so the values are identical -- then
// d = q_j . w, and a second pass forms w - d q_j, its squared norm and, when
// wr, stores it as the new W.  Columns are ldb = m_c rounded up to 4 floats
// (16-byte aligned, zero past m_c, as are the q slots), so a lane moves four
// rows per access: nf = ldb / 4 float4 per column.  cb (the warp's shared
// buffer, or null) keeps the pass-1 values for the second pass.
template <int NP>
__device__ __forceinline__ void mgs_column(const float4* x, float4* w, const float* qv, int qs,
                                           int P, int base, int j, const float* Rc, int n,
                                           int nf, int lane, bool wr, float4* cb, float& d_out,
                                           float& nu_out) {
  constexpr int U = NP >= 3 ? 2 : 4;   // float4 loads in flight per lane
  float dc[NP > 0 ? NP : 1];
  const float4* qp[NP > 0 ? NP : 1];
#pragma unroll
  for (int t = 0; t < NP; ++t) {
    dc[t] = -Rc[(int64_t)(base + t) * n];
    qp[t] = reinterpret_cast<const float4*>(qv + ((base + t) % P) * qs);
  }
  const float4* qj = reinterpret_cast<const float4*>(qv + (j % P) * qs);
  float dd[4] = {0.f, 0.f, 0.f, 0.f};
  int f = lane;
  for (; f + 32 * (U - 1) < nf; f += 32 * U) {
    float4 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = x[f + 32 * u];
#pragma unroll
    for (int t = 0; t < NP; ++t)
#pragma unroll
      for (int u = 0; u < U; ++u) fma4(v[u], dc[t], qp[t][f + 32 * u]);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      dd[u] = dot4(qj[f + 32 * u], v[u], dd[u]);
      if (cb) cb[f + 32 * u] = v[u];
    }
  }
  for (; f < nf; f += 32) {
    float4 v = x[f];
#pragma unroll
    for (int t = 0; t < NP; ++t) fma4(v, dc[t], qp[t][f]);
    dd[0] = dot4(qj[f], v, dd[0]);
    if (cb) cb[f] = v;
  }
  const float d = warp_sum((dd[0] + dd[1]) + (dd[2] + dd[3]));
  const float nd = -d;
  float aa[4] = {0.f, 0.f, 0.f, 0.f};
  f = lane;
  for (; f + 32 * (U - 1) < nf; f += 32 * U) {
    float4 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (cb) {
        v[u] = cb[f + 32 * u];
      } else {
        v[u] = x[f + 32 * u];
#pragma unroll
        for (int t = 0; t < NP; ++t) fma4(v[u], dc[t], qp[t][f + 32 * u]);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      fma4(v[u], nd, qj[f + 32 * u]);
      if (wr) w[f + 32 * u] = v[u];
      aa[u] = dot4(v[u], v[u], aa[u]);
    }
  }
  for (; f < nf; f += 32) {
    float4 v;
    if (cb) {
      v = cb[f];
    } else {
      v = x[f];
#pragma unroll
      for (int t = 0; t < NP; ++t) fma4(v, dc[t], qp[t][f]);
    }
    fma4(v, nd, qj[f]);
    if (wr) w[f] = v;
    aa[0] = dot4(v, v, aa[0]);
  }
  d_out = d;
  nu_out = warp_sum((aa[0] + aa[1]) + (aa[2] + aa[3]));
}

// What a CTA publishes to the other CTAs of its cluster (double-buffered by
// pivot step: a slot is rewritten only after every rank has passed the
// cluster barrier that follows its last read).
struct QrXchg {
  unsigned long long key;   // largest (||w_c||^2 bits, ~c) among own active columns
  float rest_h, rest_l;     // sum of own active ||w_c||^2 (double-float)
  double nb;                // sum of own ||b_c||^2 (initial exchange only)
  int bad;                  // a non-finite entry in own columns (initial exchange only)
};

__global__ void __launch_bounds__(kQrThreads, 1) subid_qr_kernel(const SubArgs a, int n_max,
                                                                 int qv_floats, int qs, int P,
                                                                 int cb_floats) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // qv_floats and the n_max-long arrays are multiples of 4 (16-byte alignment)
  float* qv = reinterpret_cast<float*>(smem_raw);          // q_t in slot t % P (stride qs), later R11
  const int n_pad = (n_max + 3) & ~3;
  float* nu = qv + qv_floats;                              // residual norms^2 [n] (own columns)
  int32_t* step = reinterpret_cast<int32_t*>(nu + n_pad);  // -1 active, >= 0 pivot step
  // a warp's column values between its two MGS passes [kQrWarps][cb_floats], if
  // they fit (cb_floats > 0)
  float4* cbw = cb_floats > 0 ? reinterpret_cast<float4*>(reinterpret_cast<float*>(step + n_pad) +
                                                          (int64_t)(threadIdx.x / 32) * cb_floats)
                              : nullptr;
  __shared__ unsigned long long wkey[kQrWarps];
  __shared__ float wrest_h[kQrWarps], wrest_l[kQrWarps];
  __shared__ double wnb[kQrWarps];
  __shared__ QrXchg xs[2];
  __shared__ double normB2_s;
  __shared__ int dec_p;     // pivot column of this step, -1: stop
  __shared__ float dec_nu;  // its residual norm^2
  __shared__ int32_t Js[kSubMaxK];

  cg::cluster_group cluster = cg::this_cluster();
  const int G = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int s = blockIdx.x / G;
  const int n = a.n[s], mc = a.mc[s], k_max = a.k_max;
  const int ldb = coarse_ld(mc);   // column stride of B and W
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int cstride = G * kQrWarps;                 // a warp's column stride
  const int c_first = rank * kQrWarps + warp;       // a warp's first column
  const float* B = a.B + a.boff[s];
  float* W = a.W + a.boff[s];
  float* R = a.R + (int64_t)k_max * a.coff[s];
  float* C = a.C + (int64_t)k_max * a.coff[s];
  float* Bsk = a.Bskel + (int64_t)k_max * a.sklo[s];
  int32_t* J = a.J + (int64_t)s * k_max;

  // own columns of R start at zero; every rank tracks the pivot steps of all
  for (int o = tid;; o += kQrThreads) {
    const int c = owned_col(o, G, rank);
    if (c >= n) break;
    for (int i = 0; i < k_max; ++i) R[(int64_t)i * n + c] = 0.f;
  }
  for (int c = tid; c < n; c += kQrThreads) step[c] = -1;
  // initial column norms, from the gather (NaN: a non-finite entry); B stays
  // untouched, W is written only once updates are due
  bool bad = false;
  for (int c = c_first; c < n; c += cstride) {
    const float* parts = a.nrm + (a.coff[s] + c) * a.nrm_parts;
    float v = 0.f;
    for (int t = lane; t < a.nrm_parts; t += 32) v += parts[t];
    v = warp_sum(v);
    if (lane == 0) {
      bad |= isnan(v);
      nu[c] = v;
    }
  }
  // own part of ||B||_F^2 (FP64, fixed order), non-finite flag; exchanged
  {
    const int any_bad = __syncthreads_or(bad);
    double t = 0.0;
    for (int c = c_first; c < n; c += cstride)
      if (lane == 0) t += (double)nu[c];
    if (lane == 0) wnb[warp] = t;
    __syncthreads();
    if (tid == 0) {
      double u = 0.0;
      for (int w = 0; w < kQrWarps; ++w) u += wnb[w];
      xs[0].nb = u;
      xs[0].bad = any_bad;
    }
  }
  cluster.sync();
  if (tid == 0) {
    double u = 0.0;
    int any = 0;
    for (int r = 0; r < G; ++r) {
      const QrXchg* x = cluster.map_shared_rank(&xs[0], r);
      u += x->nb;
      any |= x->bad;
    }
    normB2_s = u;
    dec_p = any;
  }
  __syncthreads();
  if (dec_p) {   // the same decision on every rank
    if (tid == 0 && rank == 0) {
      raise_status(a.status, kStatusNonfinite);
      a.k[s] = 0;
    }
    if (rank == 0)
      for (int p = tid; p < k_max; p += kQrThreads) J[p] = -1;
    for (int o = tid;; o += kQrThreads) {   // own columns of C
      const int c = owned_col(o, G, rank);
      if (c >= n) break;
      for (int i = 0; i < k_max; ++i) C[(int64_t)i * n + c] = 0.f;
    }
    for (int64_t e = (int64_t)rank * kQrThreads + tid; e < (int64_t)k_max * mc;
         e += (int64_t)G * kQrThreads)
      Bsk[e] = 0.f;
    cluster.sync();   // no rank leaves while another may still read its slots
    return;
  }
  const double normB2 = normB2_s;
  const double tol2 = a.tol * a.tol;
  int kcap = k_max;
  if (kcap > n) kcap = n;
  if (kcap > mc) kcap = mc;
  int k = 0;
  int base = 0;   // W holds the columns as of step base (base 0: B itself)
  float r00 = 0.f;
  for (int j = 0; j < kcap; ++j) {
    // ---- pivot: largest residual norm^2 among active columns, lowest index on
    // ties; own columns first, then the ranks' results in rank order
    unsigned long long key = 0ull;
    float rh = 0.f, rl = 0.f;
    for (int o = tid;; o += kQrThreads) {
      const int c = owned_col(o, G, rank);
      if (c >= n) break;
      if (step[c] != -1) continue;
      df_add(rh, rl, nu[c], 0.f);
      const unsigned long long kc =
          ((unsigned long long)__float_as_uint(nu[c]) << 32) | (0xffffffffu - (uint32_t)c);
      key = kc > key ? kc : key;
    }
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key, o);
      key = ok > key ? ok : key;
      const float oh = __shfl_xor_sync(0xffffffffu, rh, o);
      const float ol = __shfl_xor_sync(0xffffffffu, rl, o);
      df_add(rh, rl, oh, ol);
    }
    if (lane == 0) { wkey[warp] = key; wrest_h[warp] = rh; wrest_l[warp] = rl; }
    __syncthreads();
    if (warp == 0) {   // kQrWarps == 32: one warp's value per lane
      key = wkey[lane];
      rh = wrest_h[lane];
      rl = wrest_l[lane];
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key, o);
        key = ok > key ? ok : key;
        const float oh = __shfl_xor_sync(0xffffffffu, rh, o);
        const float ol = __shfl_xor_sync(0xffffffffu, rl, o);
        df_add(rh, rl, oh, ol);
      }
      if (lane == 0) {
        xs[j & 1].key = key;
        xs[j & 1].rest_h = rh;
        xs[j & 1].rest_l = rl;
      }
    }
    cluster.sync();
    if (tid == 0) {   // every rank takes the same decision from the same values
      key = 0ull;
      rh = 0.f;
      rl = 0.f;
      for (int r = 0; r < G; ++r) {
        const QrXchg* x = cluster.map_shared_rank(&xs[j & 1], r);
        const unsigned long long kr = x->key;
        key = kr > key ? kr : key;
        df_add(rh, rl, x->rest_h, x->rest_l);
      }
      const double rest = (double)rh + (double)rl;
      const float nu_p = __uint_as_float((uint32_t)(key >> 32));
      int p = (int)(0xffffffffu - (uint32_t)(key & 0xffffffffull));
      if (tol2 > 0.0 && rest <= tol2 * normB2) p = -1;
      if (key == 0ull || !(nu_p > 0.f)) p = -1;
      // rank guard |R_jj| > 2 u |R_00|, u = 2^-24
      if (p >= 0 && j > 0 && !(sqrtf(nu_p) > 0x1p-23f * r00)) p = -1;
      dec_p = p;
      dec_nu = nu_p;
    }
    __syncthreads();
    const int p = dec_p;
    if (p < 0) break;
    const float rjj = sqrtf(dec_nu);
    if (j == 0) r00 = rjj;
    // ---- q_j = w_p / R_jj: w_p as stored (B until W is first written) with the
    // pending updates re-applied; w_p may come from another rank, hence L2 loads
    const int np = j - base;   // pending steps base..j-1, np < P
    const float* src = (base == 0) ? B : W;
    {
      float rp[kQrMaxSlots];
#pragma unroll
      for (int t = 0; t < kQrMaxSlots; ++t)
        rp[t] = t < np ? -__ldcg(R + (int64_t)(base + t) * n + p) : 0.f;
      float* qj = qv + (j % P) * qs;
      for (int i = tid; i < ldb; i += kQrThreads) {   // zero past m_c
        float v = 0.f;
        if (i < mc) {
          v = __ldcg(src + (int64_t)p * ldb + i);
#pragma unroll
          for (int t = 0; t < kQrMaxSlots; ++t)
            if (t < np) v = fmaf(rp[t], qv[((base + t) % P) * qs + i], v);
          v = v / rjj;
        }
        qj[i] = v;
      }
    }
    if (tid == 0) {
      if (rank == 0) J[j] = p;
      if ((p / kQrWarps) % G == rank) R[(int64_t)j * n + p] = rjj;
      Js[j] = p;
      step[p] = j;
    }
    __syncthreads();
    // ---- modified Gram-Schmidt against q_j, norms from the updated columns;
    // W is rewritten once P updates are pending
    const bool wr = j + 1 - base >= P;
    for (int c = c_first; c < n; c += cstride) {
      if (step[c] != -1) continue;   // warp-uniform
      const float4* x = reinterpret_cast<const float4*>(src + (int64_t)c * ldb);
      float4* w = reinterpret_cast<float4*>(W + (int64_t)c * ldb);
      const int nf = ldb / 4;
      float d = 0.f, acc = 0.f;
      switch (np) {
        case 0: mgs_column<0>(x, w, qv, qs, P, base, j, R + c, n, nf, lane, wr, cbw, d, acc); break;
        case 1: mgs_column<1>(x, w, qv, qs, P, base, j, R + c, n, nf, lane, wr, cbw, d, acc); break;
        case 2: mgs_column<2>(x, w, qv, qs, P, base, j, R + c, n, nf, lane, wr, cbw, d, acc); break;
        default: mgs_column<3>(x, w, qv, qs, P, base, j, R + c, n, nf, lane, wr, cbw, d, acc); break;
      }
      if (lane == 0) {
        R[(int64_t)j * n + c] = d;
        nu[c] = acc;
      }
    }
    if (wr) base = j + 1;
    __syncthreads();
    k = j + 1;
  }
  // every rank's R columns are written; after this barrier no rank reads
  // another's shared memory
  cluster.sync();
  // ---- rank, pivots, coefficients
  if (rank == 0) {
    if (tid == 0) a.k[s] = k;
    for (int p = k + tid; p < k_max; p += kQrThreads) J[p] = -1;
  }
  float* R11 = qv;   // q_j is no longer needed
  for (int e = tid; e < k * k; e += kQrThreads) {
    const int i = e / k, p = e % k;
    R11[e] = __ldcg(R + (int64_t)i * n + Js[p]);
  }
  __syncthreads();
  for (int o = tid;; o += kQrThreads) {   // own columns
    const int c = owned_col(o, G, rank);
    if (c >= n) break;
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
  // ---- coarse skeleton B(:, I_B), split over the ranks
  for (int64_t e = (int64_t)rank * kQrThreads + tid; e < (int64_t)k_max * mc;
       e += (int64_t)G * kQrThreads) {
    const int p = (int)(e / mc), i = (int)(e % mc);
    Bsk[e] = (p < k) ? B[(int64_t)Js[p] * ldb + i] : 0.f;
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

// A_hat = M G per unit (subdomain, column, z block), without intermediate
// stages: a task is one (y, x) position -- four consecutive x of one row when
// ex is a multiple of four, read as one 16-byte vector -- and a run of up to
// kZRun consecutive fine z planes.  The thread computes the position's
// bilinear (y, x) weights and corner offsets once, evaluates the bilinear
// value on each coarse z plane its run crosses (the upper plane of one cell
// is the lower plane of the next), and each fine element is then one lerp in
// z.  All of a task's A loads for one QoI are issued before any is used.
// One CTA walks a contiguous range of units; the subdomain lookup and its
// per-axis cell tables are refreshed only when the range crosses into the
// next subdomain, and the only barriers are around staging G(:, j).
constexpr int kZRun = 4;

template <bool WRITE>
__global__ void __launch_bounds__(256, 3) spid_interp_kernel(const SubErrArgs args, int mc_max,
                                                          int e_max, int units_per_cta,
                                                          int total_units) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[2][8];
  __shared__ int last_sub;
  const SubArgs& a = args.a;
  const ErrArgs& e = args.e;
  float* g = reinterpret_cast<float*>(smem_raw);                  // G(:, j) [mc]
  int32_t* tab_a = reinterpret_cast<int32_t*>(g + ((mc_max + 3) & ~3));   // [3][e_max]
  float* tab_w = reinterpret_cast<float*>(tab_a + 3 * e_max);             // [3][e_max]
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int nthr = blockDim.x;
  const int u0 = blockIdx.x * units_per_cta;
  const int u1 = min(u0 + units_per_cta, total_units);
  if (u0 >= u1) return;
  int lo = 0, hi = a.S;                   // subdomain of the first unit
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (e.unit_ptr[mid] <= u0) lo = mid; else hi = mid;
  }
  int s = lo;
  int s_tab = -1;
  int s_end = e.unit_ptr[s + 1];
  const bool have_a = args.window != nullptr;
  for (int u = u0; u < u1; ++u) {
    while (u >= s_end) s_end = e.unit_ptr[++s + 1];
    const SubBox b = a.box[s];
    const int mc = a.mc[s];
    const int rel = u - e.unit_ptr[s];
    const int j = rel / b.zblocks;
    const int z0 = (rel - j * b.zblocks) * b.zc, z1 = min(b.ez, z0 + b.zc);
    const int plane = b.ey * b.ex;
    const int cplane = b.cy * b.cx;
    __syncthreads();   // the previous unit is done with g and the tables
    const float* G = a.W + a.boff[s] + (int64_t)j * mc;
    for (int i = tid; i < mc; i += nthr) g[i] = G[i];
    if (s != s_tab) {
      for (int x = tid; x < b.ez; x += nthr) axis_cell(x, b.ez, b.sz, b.cz, tab_a[x], tab_w[x]);
      for (int x = tid; x < b.ey; x += nthr)
        axis_cell(x, b.ey, b.sy, b.cy, tab_a[e_max + x], tab_w[e_max + x]);
      for (int x = tid; x < b.ex; x += nthr)
        axis_cell(x, b.ex, b.sx, b.cx, tab_a[2 * e_max + x], tab_w[2 * e_max + x]);
      s_tab = s;
    }
    __syncthreads();
    const int64_t colbase = a.off[s] + (int64_t)j * a.ld[s];
    const bool vec = (b.ex & 3) == 0;               // four x of one row per 16-byte vector
    const int W = vec ? 4 : 1;                       // fine x points per task
    const int npos = plane / W;
    const int nzr = (z1 - z0 + kZRun - 1) / kZRun;   // z runs
    float se = 0.f, ce = 0.f, sa = 0.f, ca = 0.f;
    for (int task = tid; task < npos * nzr; task += nthr) {
      const int zr = task / npos, pos = task - zr * npos;
      const int yx = pos * W;
      const int y = (int)fdiv((uint32_t)yx, b.div_ex), x0 = yx - y * b.ex;
      const int ay = tab_a[e_max + y], ay1 = min(ay + 1, b.cy - 1);
      const float wy = tab_w[e_max + y];
      // per fine x of the task: the four (y, x) corners and their weights
      int o00[4], o01[4];
      float c00[4], c01[4], c10[4], c11[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int xx = min(x0 + t, b.ex - 1);
        const int ax = tab_a[2 * e_max + xx], ax1 = min(ax + 1, b.cx - 1);
        const float wx = tab_w[2 * e_max + xx];
        o00[t] = ay * b.cx + ax;
        o01[t] = ay * b.cx + ax1;
        c00[t] = (1.f - wy) * (1.f - wx);
        c01[t] = (1.f - wy) * wx;
        c10[t] = wy * (1.f - wx);
        c11[t] = wy * wx;
      }
      const int dy = (ay1 - ay) * b.cx;              // row offset to the y + 1 corners
      const int zs = z0 + zr * kZRun, ze = min(z1, zs + kZRun);
      for (int q = 0; q < b.nq; ++q) {
        // this task's A for QoI q: up to kZRun vectors, all in flight first
        float4 av[kZRun];
        const float* Aq = have_a ? args.window + colbase + ((int64_t)q * b.ez) * plane + yx
                                 : nullptr;
#pragma unroll
        for (int r = 0; r < kZRun; ++r) {
          const int z = zs + r;
          if (have_a && z < ze) {
            av[r] = vec ? __ldg(reinterpret_cast<const float4*>(Aq + (int64_t)z * plane))
                        : make_float4(__ldg(Aq + (int64_t)z * plane), 0.f, 0.f, 0.f);
          } else {
            av[r] = make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
        const float* gq = g + q * b.cz * cplane;
        float lo4[4], hi4[4];
        int cur = -1;
        float le = 0.f, la = 0.f;
#pragma unroll
        for (int r = 0; r < kZRun; ++r) {
          const int z = zs + r;
          if (z >= ze) break;
          const int az = tab_a[z];
          const float wz = tab_w[z];
          if (az != cur) {
            const int az1 = min(az + 1, b.cz - 1);
            const float* p1 = gq + az1 * cplane;
            if (az == cur + 1 && cur >= 0) {
#pragma unroll
              for (int t = 0; t < 4; ++t) lo4[t] = hi4[t];
            } else {
              const float* p0 = gq + az * cplane;
#pragma unroll
              for (int t = 0; t < 4; ++t)
                lo4[t] = c00[t] * p0[o00[t]] + c01[t] * p0[o01[t]] + c10[t] * p0[o00[t] + dy] +
                         c11[t] * p0[o01[t] + dy];
            }
#pragma unroll
            for (int t = 0; t < 4; ++t)
              hi4[t] = c00[t] * p1[o00[t]] + c01[t] * p1[o01[t]] + c10[t] * p1[o00[t] + dy] +
                       c11[t] * p1[o01[t] + dy];
            cur = az;
          }
          const float v0 = fmaf(wz, hi4[0] - lo4[0], lo4[0]);
          const float v1 = fmaf(wz, hi4[1] - lo4[1], lo4[1]);
          const float v2 = fmaf(wz, hi4[2] - lo4[2], lo4[2]);
          const float v3 = fmaf(wz, hi4[3] - lo4[3], lo4[3]);
          const float4 x = av[r];
          const float d0 = x.x - v0;
          le = fmaf(d0, d0, le);
          la = fmaf(x.x, x.x, la);
          if (vec) {
            const float d1 = x.y - v1, d2 = x.z - v2, d3 = x.w - v3;
            le = fmaf(d1, d1, fmaf(d2, d2, fmaf(d3, d3, le)));
            la = fmaf(x.y, x.y, fmaf(x.z, x.z, fmaf(x.w, x.w, la)));
          }
          if (WRITE) {
            float* o = args.out + colbase + ((int64_t)q * b.ez + z) * plane + yx;
            if (vec) *reinterpret_cast<float4*>(o) = make_float4(v0, v1, v2, v3);
            else *o = v0;
          }
        }
        kahan_add(se, ce, le);
        kahan_add(sa, ca, la);
      }
    }
    // unit partial: warp tree in FP32, FP64 across warps, then the fixed-order fold
    float we = se - ce, wa = sa - ca;
    for (int o = 16; o > 0; o >>= 1) {
      we += __shfl_xor_sync(0xffffffffu, we, o);
      wa += __shfl_xor_sync(0xffffffffu, wa, o);
    }
    if (lane == 0) { red[0][warp] = (double)we; red[1][warp] = (double)wa; }
    __syncthreads();
    if (tid == 0) {
      double te = 0.0, ta = 0.0;
      for (int w = 0; w < (int)(nthr / 32); ++w) { te += red[0][w]; ta += red[1][w]; }
      e.part[2 * (int64_t)u] = te;
      e.part[2 * (int64_t)u + 1] = ta;
      __threadfence();
      const int units_s = e.unit_ptr[s + 1] - e.unit_ptr[s];
      last_sub = (atomicAdd(&e.sub_cnt[s], 1) == units_s - 1);
    }
    __syncthreads();
    if (last_sub && warp == 0) error_fold_subdomain(e, s, lane);
  }
}

// ---------------------------------------------------------------- fine skeleton
// A_hat = M B(:, I_B) C_B is linear in both factors, so the interpolation can
// be applied to the k skeleton columns once instead of to all n reconstructed
// columns: F = M B(:, I_B) (m x k per subdomain, column p at p m_s of the
// subdomain's block) is the trilinear interpolation of each coarse skeleton
// column to the fine grid.  The error pass is then the rank-k product F C_B
// against A -- the same HBM-rate kernel as the column ID's error pass.
__global__ void __launch_bounds__(256, 4) fine_skeleton_kernel(const SubArgs a, float* F,
                                                               const int64_t* foff, int e_max) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int32_t* tab_a = reinterpret_cast<int32_t*>(smem_raw);   // [3][e_max] cell per z, y, x
  float* tab_w = reinterpret_cast<float*>(tab_a + 3 * e_max);   // [3][e_max] weight
  const int s = blockIdx.y;
  const SubBox b = a.box[s];
  const int m = a.m[s], mc = a.mc[s], k = a.k[s];
  for (int x = threadIdx.x; x < b.ez; x += blockDim.x) axis_cell(x, b.ez, b.sz, b.cz, tab_a[x], tab_w[x]);
  for (int x = threadIdx.x; x < b.ey; x += blockDim.x)
    axis_cell(x, b.ey, b.sy, b.cy, tab_a[e_max + x], tab_w[e_max + x]);
  for (int x = threadIdx.x; x < b.ex; x += blockDim.x)
    axis_cell(x, b.ex, b.sx, b.cx, tab_a[2 * e_max + x], tab_w[2 * e_max + x]);
  __syncthreads();
  const float* Bsk = a.Bskel + (int64_t)a.k_max * a.sklo[s];
  float* Fs = F + foff[s];
  const int plane = b.ey * b.ex;
  const int cplane = b.cy * b.cx;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
    const int qz = (int)fdiv((uint32_t)r, b.div_plane), yx = r - qz * plane;
    const int q = qz / b.ez, z = qz - q * b.ez;
    const int y = (int)fdiv((uint32_t)yx, b.div_ex), x = yx - y * b.ex;
    const int az = tab_a[z], ay = tab_a[e_max + y], ax = tab_a[2 * e_max + x];
    const float wz = tab_w[z], wy = tab_w[e_max + y], wx = tab_w[2 * e_max + x];
    const int az1 = min(az + 1, b.cz - 1), ay1 = min(ay + 1, b.cy - 1), ax1 = min(ax + 1, b.cx - 1);
    const int base = q * b.cz * cplane;
    const int i00 = base + az * cplane + ay * b.cx, i01 = base + az * cplane + ay1 * b.cx;
    const int i10 = base + az1 * cplane + ay * b.cx, i11 = base + az1 * cplane + ay1 * b.cx;
#pragma unroll 1
    for (int p = 0; p < k; ++p) {
      const float* c = Bsk + (int64_t)p * mc;
      const float v00 = fmaf(wx, c[i00 + ax1] - c[i00 + ax], c[i00 + ax]);
      const float v01 = fmaf(wx, c[i01 + ax1] - c[i01 + ax], c[i01 + ax]);
      const float v10 = fmaf(wx, c[i10 + ax1] - c[i10 + ax], c[i10 + ax]);
      const float v11 = fmaf(wx, c[i11 + ax1] - c[i11 + ax], c[i11 + ax]);
      const float v0 = fmaf(wy, v01 - v00, v00), v1 = fmaf(wy, v11 - v10, v10);
      Fs[(int64_t)p * m + r] = fmaf(wz, v1 - v0, v0);
    }
  }
}

// ---------------------------------------------------------------- point sets
// Coarse-grid ID on an arbitrary point set (an unstructured grid, rows in any
// order, Section 2): the coarse rows are an explicit list per subdomain and M
// is a fixed-width stencil (t coarse rows and weights per fine row).

// B_s(:, col0 + j) = A_s(crow_s, col0 + j).
__global__ void __launch_bounds__(256) subsample_rows_kernel(const SubArgs a, const float* window,
                                                             int col0, int ncols,
                                                             const int32_t* crow,
                                                             const int64_t* crow_off) {
  const int s = blockIdx.y;
  const int mc = a.mc[s];
  GatherPart g;
  if (!gather_part(a, s, col0, ncols, mc, g)) return;   // warp-uniform; no block barrier below
  const int lane = threadIdx.x % 32;
  const int32_t* rows = crow + crow_off[s];
  const float* Aj = window + a.off[s] + (int64_t)g.j * a.ld[s];
  float* Bj = a.B + a.boff[s] + (int64_t)g.j * coarse_ld(mc);
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  bool bad = false;
  for (int i0 = g.r0 + lane; i0 < g.r1; i0 += 128) {
    float v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + 32 * u;
      v[u] = i < g.r1 ? __ldg(Aj + rows[i]) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + 32 * u;
      if (i < g.r1) {
        Bj[i] = v[u];
        acc[u] = fmaf(v[u], v[u], acc[u]);
        bad |= !isfinite(v[u]);
      }
    }
  }
  finish_part_norm(a, s, g, acc, bad, lane);
}

// F_s(r, p) = sum_q w_s(r, q) B(:, I_B)(idx_s(r, q), p), p < k_s.
// TW > 0: the stencil width as a compile-time constant (the row's stencil in
// registers); TW == 0: any width t <= 16, read per skeleton column.
template <int TW>
__global__ void __launch_bounds__(256, 4) fine_skeleton_points_kernel(
    const SubArgs a, float* F, const int64_t* foff, const int32_t* iidx, const float* iw,
    const int64_t* ioff, int t) {
  const int s = blockIdx.y;
  const int m = a.m[s], mc = a.mc[s], k = a.k[s];
  const float* Bsk = a.Bskel + (int64_t)a.k_max * a.sklo[s];
  const int32_t* idx = iidx + ioff[s];
  const float* w = iw + ioff[s];
  float* Fs = F + foff[s];
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
    if (TW > 0) {
      int32_t ri[TW > 0 ? TW : 1];
      float rw[TW > 0 ? TW : 1];
#pragma unroll
      for (int q = 0; q < TW; ++q) {
        ri[q] = idx[(int64_t)r * TW + q];
        rw[q] = w[(int64_t)r * TW + q];
      }
#pragma unroll 1
      for (int p = 0; p < k; ++p) {
        const float* c = Bsk + (int64_t)p * mc;
        float v = 0.f;
#pragma unroll
        for (int q = 0; q < TW; ++q) v = fmaf(rw[q], c[ri[q]], v);
        Fs[(int64_t)p * m + r] = v;
      }
    } else {
      for (int p = 0; p < k; ++p) {
        const float* c = Bsk + (int64_t)p * mc;
        float v = 0.f;
        for (int q = 0; q < t; ++q) v = fmaf(w[(int64_t)r * t + q], c[idx[(int64_t)r * t + q]], v);
        Fs[(int64_t)p * m + r] = v;
      }
    }
  }
}

// out_s(:, j) = F_s C_s(:, j) (reconstruction without the window): one thread
// per (row, block of 32 columns), C's block staged in shared memory.
__global__ void __launch_bounds__(256) skeleton_product_kernel(const SubArgs a, const float* F,
                                                               const int64_t* foff, float* out) {
  __shared__ float cs[kSubMaxK][32];
  const int s = blockIdx.z;
  const int m = a.m[s], n = a.n[s], k = a.k[s];
  const int j0 = blockIdx.y * 32;
  if (j0 >= n) return;
  const int nc = min(32, n - j0);
  const float* C = a.C + (int64_t)a.k_max * a.coff[s];
  for (int e = threadIdx.x; e < k * 32; e += blockDim.x) {
    const int p = e / 32, jj = e % 32;
    cs[p][jj] = jj < nc ? C[(int64_t)p * n + j0 + jj] : 0.f;
  }
  __syncthreads();
  const float* Fs = F + foff[s];
  float* o = out + a.off[s];
  const int64_t ld = a.ld[s];
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
    float acc[32];
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) acc[jj] = 0.f;
    for (int p = 0; p < k; ++p) {
      const float f = Fs[(int64_t)p * m + r];
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) acc[jj] = fmaf(f, cs[p][jj], acc[jj]);
    }
#pragma unroll
    for (int jj = 0; jj < 32; ++jj)
      if (jj < nc) o[(int64_t)(j0 + jj) * ld + r] = acc[jj];
  }
}

int grid_for(int64_t work) {
  const int64_t blocks = (work + 255) / 256;
  return (int)(blocks < 1 ? 1 : (blocks > 1024 ? 1024 : blocks));
}

}  // namespace

cudaError_t launch_subsample(const SubArgs& a, const float* window, int col0, int ncols,
                             int64_t max_work, cudaStream_t st) {
  if (max_work <= 0) return cudaSuccess;
  const unsigned gx =
      (unsigned)(((int64_t)ncols * a.nrm_parts + kSampleColsPerBlock - 1) / kSampleColsPerBlock);
  subsample_kernel<<<dim3(gx, a.S), 32 * kSampleColsPerBlock, 0, st>>>(a, window, col0, ncols);
  return cudaGetLastError();
}

static int qr_slot_stride(int mc_max) { return (mc_max + 3) & ~3; }
static int qr_slots(int mc_max) {
  const int P = kQrSlotBudgetFloats / qr_slot_stride(mc_max);
  return P < 1 ? 1 : (P > kQrMaxSlots ? kQrMaxSlots : P);
}
static int qr_qv_floats(int mc_max, int k_max) {
  const int q = qr_slots(mc_max) * qr_slot_stride(mc_max);
  return ((q > k_max * k_max ? q : k_max * k_max) + 3) & ~3;
}

size_t subid_qr_smem_bytes(int mc_max, int n_max, int k_max) {
  const size_t n_pad = (size_t)((n_max + 3) & ~3);
  return sizeof(float) * ((size_t)qr_qv_floats(mc_max, k_max) + n_pad) + sizeof(int32_t) * n_pad;
}

// Cluster size for the QR: up to 8 CTAs per subdomain while the clusters of
// all subdomains still fit on the SMs at once, and no more CTAs than the
// columns give warps.
static int qr_cluster_size(int S, int n_max) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 1;
  const int col_groups = (n_max + kQrWarps - 1) / kQrWarps;
  int G = 8;
  while (G > 1 && ((int64_t)G * S > sms || G > col_groups)) G /= 2;
  return G;
}

cudaError_t launch_subid_qr(const SubArgs& a, int mc_max, int n_max, cudaStream_t st) {
  const int qv = qr_qv_floats(mc_max, a.k_max);
  const int qs = qr_slot_stride(mc_max), P = qr_slots(mc_max);
  const size_t smem0 = subid_qr_smem_bytes(mc_max, n_max, a.k_max);
  const int cbf = smem0 + sizeof(float) * (size_t)kQrWarps * qs <= kQrColumnSmemMax ? qs : 0;
  const size_t smem = smem0 + sizeof(float) * (size_t)kQrWarps * cbf;
  cudaError_t e = cudaFuncSetAttribute(subid_qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int G = qr_cluster_size(a.S, n_max);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.S * G));
  cfg.blockDim = dim3(kQrThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)G;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  while (G > 1) {   // a cluster shape the SMs cannot hold falls back to a smaller one
    int fit = 0;
    if (cudaOccupancyMaxActiveClusters(&fit, subid_qr_kernel, &cfg) == cudaSuccess && fit > 0)
      break;
    cudaGetLastError();
    G /= 2;
    cfg.gridDim = dim3((unsigned)(a.S * G));
    attr[0].val.clusterDim.x = (unsigned)G;
  }
  return cudaLaunchKernelEx(&cfg, subid_qr_kernel, a, n_max, qv, qs, P, cbf);
}

cudaError_t launch_coarse_recon(const SubArgs& a, int64_t max_work, cudaStream_t st) {
  if (max_work <= 0) return cudaSuccess;
  coarse_recon_kernel<<<dim3(grid_for(max_work), a.S), 256, 0, st>>>(a);
  return cudaGetLastError();
}

size_t spid_interp_smem_bytes(int mc_max, int e_max) {
  return sizeof(float) * (size_t)((mc_max + 3) & ~3) +
         3 * (sizeof(int32_t) + sizeof(float)) * (size_t)e_max;
}

cudaError_t launch_spid_interp(const SubErrArgs& a, int64_t units, int mc_max, int e_max,
                               cudaStream_t st) {
  if (units <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  // three resident CTAs per SM (register-bound), a few waves; each CTA walks a
  // contiguous range of units
  const int64_t target = (int64_t)sms * 6;
  const int per = (int)((units + target - 1) / target);
  const int grid = (int)((units + per - 1) / per);
  const size_t smem = spid_interp_smem_bytes(mc_max, e_max);
  if (a.out) {
    e = cudaFuncSetAttribute(spid_interp_kernel<true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    spid_interp_kernel<true><<<grid, 256, smem, st>>>(a, mc_max, e_max, per, (int)units);
  } else {
    e = cudaFuncSetAttribute(spid_interp_kernel<false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    spid_interp_kernel<false><<<grid, 256, smem, st>>>(a, mc_max, e_max, per, (int)units);
  }
  return cudaGetLastError();
}

// CTAs per subdomain for the fine-skeleton kernels: about two resident waves in
// all (four 256-thread CTAs per SM), each thread taking several rows (the box
// kernel builds its per-axis tables once per CTA)
static int fine_skeleton_blocks(int S, int m_max) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 1;
  return std::max(1, std::min(grid_for(m_max), (8 * sms + S - 1) / S));
}

cudaError_t launch_fine_skeleton(const SubArgs& a, float* F, const int64_t* foff, int m_max,
                                 int e_max, cudaStream_t st) {
  if (m_max <= 0) return cudaSuccess;
  const size_t smem = (sizeof(int32_t) + sizeof(float)) * 3 * (size_t)e_max;
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(
        fine_skeleton_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  fine_skeleton_kernel<<<dim3(fine_skeleton_blocks(a.S, m_max), a.S), 256, smem, st>>>(
      a, F, foff, e_max);
  return cudaGetLastError();
}

cudaError_t launch_subsample_rows(const SubArgs& a, const float* window, int col0, int ncols,
                                  const int32_t* crow, const int64_t* crow_off, int64_t max_work,
                                  cudaStream_t st) {
  if (max_work <= 0) return cudaSuccess;
  const unsigned gx =
      (unsigned)(((int64_t)ncols * a.nrm_parts + kSampleColsPerBlock - 1) / kSampleColsPerBlock);
  subsample_rows_kernel<<<dim3(gx, a.S), 32 * kSampleColsPerBlock, 0, st>>>(a, window, col0, ncols,
                                                                           crow, crow_off);
  return cudaGetLastError();
}

cudaError_t launch_fine_skeleton_points(const SubArgs& a, float* F, const int64_t* foff,
                                        const int32_t* iidx, const float* iw, const int64_t* ioff,
                                        int t, int m_max, cudaStream_t st) {
  if (m_max <= 0) return cudaSuccess;
  const dim3 grid(fine_skeleton_blocks(a.S, m_max), a.S);
  if (t == 3)
    fine_skeleton_points_kernel<3><<<grid, 256, 0, st>>>(a, F, foff, iidx, iw, ioff, t);
  else if (t == 4)
    fine_skeleton_points_kernel<4><<<grid, 256, 0, st>>>(a, F, foff, iidx, iw, ioff, t);
  else
    fine_skeleton_points_kernel<0><<<grid, 256, 0, st>>>(a, F, foff, iidx, iw, ioff, t);
  return cudaGetLastError();
}

cudaError_t launch_skeleton_product(const SubArgs& a, const float* F, const int64_t* foff,
                                    float* out, int m_max, int n_max, cudaStream_t st) {
  if (m_max <= 0 || n_max <= 0) return cudaSuccess;
  const int gx = std::min((m_max + 255) / 256, 64);
  skeleton_product_kernel<<<dim3(gx, (n_max + 31) / 32, a.S), 256, 0, st>>>(a, F, foff, out);
  return cudaGetLastError();
}

}  // namespace spid
