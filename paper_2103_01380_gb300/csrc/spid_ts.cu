// spid_ts.cu -- modified (two-stage) SPID, Section 3.3.2 and Algorithm 6, as
// a composition of batched sketched-ID plans:
//   stage 1   one plan per time block b over the columns b n/N .. (b+1) n/N - 1
//             of every subdomain (target rank k): A_b ~ A_b(:, I_b) C_b
//   stage 2   a sketched ID with the tolerance tol2 of the union of skeleton
//             columns A0' = [A_0(:, I_0) .. A_{N-1}(:, I_{N-1})]: A0' ~ A0'(:, J2) C1
//   compose   C1' = C1 C0' with C0' = blockdiag(C_b), J = I_U(J2): the index of
//             A0' column q = b k + p in the window is b n/N + I_b(p)
// Both stages draw the same rows of Omega (one key), and the sketch is linear
// in the columns, so stage 2's sketch Omega A0' is the stage-1 sketches'
// skeleton columns, Y_b(:, I_b): the block plans sketch l2 = k2_max + p rows
// (their QR still reads the first k + p), and stage 2 gathers those columns
// (slots past k_{b,s} are zero and never picked) instead of streaming A0'
// from the window again -- no second pass over the data, no A0' buffer.
// The final factors are written into a third plan over the whole window,
// whose error / reconstruction passes then serve as spid_ts_error /
// spid_ts_reconstruct.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/spid.h"
#include "spid_internal.cuh"

namespace spid {
PlanView plan_view(spid_plan_t P);
spid_status plan_create_sketch_rows(const spid_plan_desc* d, spid_stream_t stream, int l_sketch,
                                    spid_plan_t* out);
}

using namespace spid;

struct spid_ts_plan_s {
  int device = 0;
  int S = 0, N = 0, k = 0, k2_max = 0;
  size_t esz = 4;
  int32_t n_max = 0, m_max = 0;
  std::vector<spid_plan_t> blocks;
  spid_plan_t stage2 = nullptr;
  spid_plan_t full = nullptr;
  // device
  int32_t* d_nb = nullptr;          // [S] block length n_s / N
  const int32_t** d_Jb = nullptr;   // [N] block plans' J
  const int32_t** d_kb = nullptr;   // [N] block plans' k
  const void** d_Cb = nullptr;      // [N] block plans' C
  const int64_t** d_cboff = nullptr;   // [N] block plans' C offsets
  const void** d_Yb = nullptr;      // [N] block plans' stored sketches
  const int64_t** d_yboff = nullptr;   // [N] block plans' sketch offsets
  int32_t yb_pad = 0;               // row stride of the block plans' sketches
  std::vector<void*> allocs;
};

namespace {

spid_status tfail(spid_status st, const std::string& msg) {
  set_last_error(msg.c_str());
  return st;
}

#define TS_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return tfail(e_ == cudaErrorMemoryAllocation ? SPID_ERR_OOM : SPID_ERR_CUDA,         \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                    \
  } while (0)

// Stage 2's sketch of A0': column q = b k + p of subdomain s is column I_b(p)
// of block b's sketch (rows 0 .. l2 - 1; the rest of the stored rows zero), or
// zero past the block's rank k_{b,s}.  One CTA per subdomain.
template <typename T>
__global__ void __launch_bounds__(256) gather_sketch_kernel(PlanView s2, int k, int yb_pad,
                                                            const void* const* Yb,
                                                            const int64_t* const* yboff,
                                                            const int32_t* const* Jb,
                                                            const int32_t* const* kb) {
  const int s = blockIdx.x;
  const int lp = s2.l_pad, l2 = s2.l;
  const int nq = s2.n[s];                       // N k
  T* Y2 = static_cast<T*>(s2.Y) + s2.yoff[s];
  for (int64_t e = threadIdx.x; e < (int64_t)nq * lp; e += blockDim.x) {
    const int q = (int)(e / lp), i = (int)(e - (int64_t)q * lp);
    const int b = q / k, p = q - b * k;
    T v = T(0);
    if (i < l2 && p < kb[b][s]) {
      const int j = Jb[b][(int64_t)s * k + p];
      v = static_cast<const T*>(Yb[b])[yboff[b][s] + (int64_t)j * yb_pad + i];
    }
    Y2[e] = v;
  }
}

// C1'(i, t) = sum_p C1(i, b k + p) C_b(p, t - b nb), b = t / nb; J(i) = b nb + I_b(p)
// for J2(i) = b k + p; k = k2.  Written into the whole-window plan's factors.
template <typename T>
__global__ void __launch_bounds__(256) compose_kernel(PlanView s2, PlanView fin, int k,
                                                      const int32_t* nb,
                                                      const int32_t* const* Jb,
                                                      const void* const* Cb,
                                                      const int64_t* const* cboff) {
  const int s = blockIdx.x;
  const int n = fin.n[s];
  const int nbs = nb[s];
  const int k2 = s2.k[s];
  const int k2_max = fin.k_max;
  const int n2 = s2.n[s];                       // N k
  const T* C1 = static_cast<const T*>(s2.C) + s2.coff[s];
  T* Cf = static_cast<T*>(fin.C) + fin.coff[s];
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int b = t / nbs, tt = t - b * nbs;
    const T* Cbb = static_cast<const T*>(Cb[b]) + cboff[b][s];   // k x nbs row-major
    for (int i = 0; i < k2_max; ++i) {
      T acc = T(0);
      if (i < k2)
        for (int p = 0; p < k; ++p)
          acc += C1[(int64_t)i * n2 + b * k + p] * Cbb[(int64_t)p * nbs + tt];
      Cf[(int64_t)i * n + t] = acc;
    }
  }
  for (int i = threadIdx.x; i < k2_max; i += blockDim.x) {
    int32_t j = -1;
    if (i < k2) {
      const int q = s2.J[(int64_t)s * s2.k_max + i];
      const int b = q / k, p = q - b * k;
      j = b * nbs + Jb[b][(int64_t)s * k + p];
    }
    fin.J[(int64_t)s * k2_max + i] = j;
  }
  if (threadIdx.x == 0) fin.k[s] = k2;
}

}  // namespace

extern "C" {

spid_status spid_ts_plan_create(const spid_ts_desc* d, spid_ts_plan_t* out) {
  if (!d || !out) return tfail(SPID_ERR_INVALID_ARG, "desc/out is NULL");
  *out = nullptr;
  const spid_plan_desc& B = d->base;
  if (B.boxes)
    return tfail(SPID_ERR_UNSUPPORTED, "the two-stage plan takes the blocks layout (base.boxes = NULL)");
  if (B.num_sub < 1 || B.num_sub > 65535 || !B.m || !B.n || !B.off || !B.ld)
    return tfail(SPID_ERR_INVALID_ARG, "bad base descriptor");
  if (d->blocks < 1) return tfail(SPID_ERR_INVALID_ARG, "blocks must be >= 1");
  if (B.tol != 0.0 || B.flags != 0)
    return tfail(SPID_ERR_INVALID_ARG, "stage 1 uses a fixed target rank: base.tol and base.flags must be 0");
  if (!(d->tol2 > 0.0)) return tfail(SPID_ERR_INVALID_ARG, "tol2 must be > 0");
  if (d->k2_max < 1 || d->k2_max > d->blocks * B.k_max)
    return tfail(SPID_ERR_INVALID_ARG, "k2_max must be in [1, blocks * k_max]");
  const int N = d->blocks, k = B.k_max, S = B.num_sub;
  for (int s = 0; s < S; ++s)
    if (B.n[s] < N || B.n[s] % N != 0)
      return tfail(SPID_ERR_INVALID_ARG, "n of subdomain " + std::to_string(s) +
                                             " is not a positive multiple of blocks");
  spid_ts_plan_s* P = new spid_ts_plan_s();
  auto bail = [&](spid_status st) {
    spid_ts_plan_destroy(P);
    return st;
  };
  P->S = S;
  P->N = N;
  P->k = k;
  P->k2_max = d->k2_max;
  P->esz = B.precision == SPID_PREC_FP64 ? 8 : 4;
  if (cudaGetDevice(&P->device) != cudaSuccess) {
    delete P;
    return tfail(SPID_ERR_CUDA, "cudaGetDevice failed");
  }
  // ---- stage 1: one plan per time block, sketching the l2 rows stage 2 reads
  const int l2 = d->k2_max + B.p;
  std::vector<int32_t> nb(S), n2(S, N * k), m(B.m, B.m + S);
  std::vector<int64_t> off_b(S), goff(S, 0), gld(S);
  for (int s = 0; s < S; ++s) nb[s] = B.n[s] / N;
  for (int b = 0; b < N; ++b) {
    for (int s = 0; s < S; ++s) off_b[s] = B.off[s] + (int64_t)b * nb[s] * B.ld[s];
    spid_plan_desc db = B;
    db.n = nb.data();
    db.off = off_b.data();
    db.qoi = nullptr;   // per-QoI totals only for the final factors
    db.num_qoi = 0;
    spid_plan_t pb = nullptr;
    spid_status st = plan_create_sketch_rows(&db, nullptr, l2, &pb);
    if (st != SPID_OK) return bail(st);
    P->blocks.push_back(pb);
  }
  // ---- stage 2: a plan over A0' (N k columns per subdomain) whose sketch is
  // gathered from the blocks' sketches; it never reads a window, so its
  // offsets only need to be valid
  const int64_t align = 16 / (int64_t)P->esz;
  for (int s = 0; s < S; ++s) {
    gld[s] = ((int64_t)m[s] + align - 1) / align * align;
    P->m_max = std::max(P->m_max, m[s]);
    P->n_max = std::max(P->n_max, B.n[s]);
  }
  spid_plan_desc d2 = B;
  d2.n = n2.data();
  d2.off = goff.data();
  d2.ld = gld.data();
  d2.k_max = d->k2_max;
  d2.tol = d->tol2;
  d2.qoi = nullptr;
  d2.num_qoi = 0;
  spid_status st = spid_plan_create(&d2, nullptr, &P->stage2);
  if (st != SPID_OK) return bail(st);
  // ---- whole-window plan holding the final factors
  spid_plan_desc df = B;
  df.k_max = d->k2_max;
  st = spid_plan_create(&df, nullptr, &P->full);
  if (st != SPID_OK) return bail(st);
  // ---- device tables
  auto dalloc = [&](void** p, size_t bytes) -> cudaError_t {
    cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    if (e == cudaSuccess) P->allocs.push_back(*p);
    return e;
  };
  std::vector<const int32_t*> Jb(N), kb(N);
  std::vector<const void*> Cb(N), Yb(N);
  std::vector<const int64_t*> cboff(N), yboff(N);
  for (int b = 0; b < N; ++b) {
    const PlanView v = plan_view(P->blocks[b]);
    Jb[b] = v.J;
    kb[b] = v.k;
    Cb[b] = v.C;
    cboff[b] = v.coff;
    Yb[b] = v.Y;
    yboff[b] = v.yoff;
    P->yb_pad = v.l_pad;
  }
  struct Up { void** dst; const void* src; size_t bytes; };
  const Up ups[] = {
      {reinterpret_cast<void**>(&P->d_nb), nb.data(), sizeof(int32_t) * S},
      {reinterpret_cast<void**>(&P->d_Yb), Yb.data(), sizeof(void*) * N},
      {reinterpret_cast<void**>(&P->d_yboff), yboff.data(), sizeof(void*) * N},
      {reinterpret_cast<void**>(&P->d_Jb), Jb.data(), sizeof(void*) * N},
      {reinterpret_cast<void**>(&P->d_kb), kb.data(), sizeof(void*) * N},
      {reinterpret_cast<void**>(&P->d_Cb), Cb.data(), sizeof(void*) * N},
      {reinterpret_cast<void**>(&P->d_cboff), cboff.data(), sizeof(void*) * N},
  };
  for (const Up& u : ups) {
    if (dalloc(u.dst, u.bytes) != cudaSuccess ||
        cudaMemcpy(*u.dst, u.src, u.bytes, cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(tfail(SPID_ERR_CUDA, "two-stage table upload failed"));
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return bail(tfail(SPID_ERR_CUDA, "sync failed"));
  *out = P;
  return SPID_OK;
}

spid_status spid_ts_plan_destroy(spid_ts_plan_t P) {
  if (!P) return SPID_OK;
  cudaSetDevice(P->device);
  cudaDeviceSynchronize();
  for (spid_plan_t b : P->blocks) spid_plan_destroy(b);
  spid_plan_destroy(P->stage2);
  spid_plan_destroy(P->full);
  for (void* p : P->allocs) cudaFree(p);
  delete P;
  return SPID_OK;
}

spid_status spid_ts_block(spid_ts_plan_t P, const void* window, int32_t block,
                          spid_stream_t stream) {
  if (!P) return tfail(SPID_ERR_INVALID_ARG, "plan is NULL");
  if (block < 0 || block >= P->N) return tfail(SPID_ERR_INVALID_ARG, "block out of range");
  spid_status st = spid_sketch_accumulate(P->blocks[block], window, 0, P->n_max, stream);
  if (st != SPID_OK) return st;
  return spid_finalize(P->blocks[block], stream);
}

spid_status spid_ts_finalize(spid_ts_plan_t P, const void* window, spid_stream_t stream) {
  if (!P) return tfail(SPID_ERR_INVALID_ARG, "plan is NULL");
  if (!window || reinterpret_cast<uintptr_t>(window) % 16)
    return tfail(SPID_ERR_INVALID_ARG, "window must be non-NULL and 16-byte aligned");
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != P->device) TS_CUDA(cudaSetDevice(P->device));
  cudaStream_t cs = (cudaStream_t)stream;
  const PlanView v2 = plan_view(P->stage2);
  const PlanView vf = plan_view(P->full);
  if (P->esz == 8)
    gather_sketch_kernel<double><<<P->S, 256, 0, cs>>>(v2, P->k, P->yb_pad, P->d_Yb, P->d_yboff,
                                                       P->d_Jb, P->d_kb);
  else
    gather_sketch_kernel<float><<<P->S, 256, 0, cs>>>(v2, P->k, P->yb_pad, P->d_Yb, P->d_yboff,
                                                      P->d_Jb, P->d_kb);
  TS_CUDA(cudaGetLastError());
  spid_status st = spid_finalize(P->stage2, stream);
  if (st != SPID_OK) return st;
  if (P->esz == 8)
    compose_kernel<double><<<P->S, 256, 0, cs>>>(v2, vf, P->k, P->d_nb, P->d_Jb, P->d_Cb,
                                                 P->d_cboff);
  else
    compose_kernel<float><<<P->S, 256, 0, cs>>>(v2, vf, P->k, P->d_nb, P->d_Jb, P->d_Cb,
                                                P->d_cboff);
  TS_CUDA(cudaGetLastError());
  return SPID_OK;
}

spid_status spid_ts_error(spid_ts_plan_t P, const void* window, double* err_dev,
                          double* total_dev, spid_stream_t stream) {
  if (!P) return tfail(SPID_ERR_INVALID_ARG, "plan is NULL");
  return spid_error(P->full, window, err_dev, total_dev, stream);
}

spid_status spid_ts_reconstruct(spid_ts_plan_t P, const void* window, void* out,
                                spid_stream_t stream) {
  if (!P) return tfail(SPID_ERR_INVALID_ARG, "plan is NULL");
  return spid_reconstruct(P->full, window, out, stream);
}

spid_status spid_ts_get_factors(spid_ts_plan_t P, int32_t* k_host, int32_t* J_host,
                                void* C_host, spid_stream_t stream) {
  if (!P) return tfail(SPID_ERR_INVALID_ARG, "plan is NULL");
  return spid_get_factors(P->full, k_host, J_host, C_host, stream);
}

spid_status spid_ts_get_block_factors(spid_ts_plan_t P, int32_t block, int32_t* k_host,
                                      int32_t* J_host, void* C_host, spid_stream_t stream) {
  if (!P) return tfail(SPID_ERR_INVALID_ARG, "plan is NULL");
  if (block < 0 || block >= P->N) return tfail(SPID_ERR_INVALID_ARG, "block out of range");
  return spid_get_factors(P->blocks[block], k_host, J_host, C_host, stream);
}

spid_status spid_ts_device_status(spid_ts_plan_t P, spid_stream_t stream) {
  if (!P) return tfail(SPID_ERR_INVALID_ARG, "plan is NULL");
  // the first error wins; the informational rank-guard cut only if nothing failed
  spid_status worst = SPID_OK;
  auto take = [&](spid_status st) {
    if (st == SPID_OK) return;
    if (worst == SPID_OK || (worst == SPID_ERR_RANK && st != SPID_ERR_RANK)) worst = st;
  };
  for (spid_plan_t b : P->blocks) take(spid_device_status(b, stream));
  take(spid_device_status(P->stage2, stream));
  take(spid_device_status(P->full, stream));
  return worst;
}

}  // extern "C"
