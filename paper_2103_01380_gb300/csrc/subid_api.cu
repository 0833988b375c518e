// subid_api.cu -- C ABI of the coarse-grid column ID (include/spid.h,
// spid_sub_*): plan creation with all workspace, the subsample gather, the
// finalize (pivoted MGS QR + coefficients + coarse skeleton), and the SPID
// (trilinear) and SubID error / reconstruction passes.  Section 2 SubID and
// SPID paragraphs, Algorithms 2 and 3, Section 5.2.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/spid.h"
#include "subid_internal.cuh"

using namespace spid;

struct spid_sub_plan_s {
  int device = 0;
  int S = 0;
  std::vector<SubBox> box;
  std::vector<int32_t> m, n, mc;
  std::vector<int64_t> off, ld, boff, coff, sklo;
  int k_max = 0;
  double tol = 0.0;
  int mc_max = 0, n_max = 0, e_max = 0, m_max = 0;
  std::vector<int64_t> foff;   // F_s at foff[s] = k_max sum_{s'<s} m_s'
  int64_t b_elems = 0, c_elems = 0, sk_elems = 0;
  // SPID error units (per subdomain: n_s columns x zblocks)
  std::vector<int32_t> uptr;
  int64_t spid_units = 0;
  int64_t f_elems = 0;     // fine skeleton F = M B(:, I_B): sum m_s k_max
  // point-set plans (arbitrary grids): coarse rows and interpolation stencils
  bool points = false;
  int32_t t = 0;                              // stencil width
  std::vector<int32_t> crow, iidx;            // concatenated coarse rows / stencil indices
  std::vector<float> iw;                      // stencil weights
  std::vector<int64_t> crow_off, ioff;        // per subdomain: sum m_c, sum m t
  int32_t* d_crow = nullptr;
  int64_t* d_crow_off = nullptr;
  int32_t* d_iidx = nullptr;
  float* d_iw = nullptr;
  int64_t* d_ioff = nullptr;
  // SubID error units (512-row x 256-column blocks, as the main error pass)
  std::vector<int32_t> usub, urow, ucol, uptr_subid;
  // device
  SubBox* d_box = nullptr;
  int32_t *d_m = nullptr, *d_n = nullptr, *d_mc = nullptr;
  int64_t *d_off = nullptr, *d_ld = nullptr, *d_boff = nullptr, *d_coff = nullptr,
          *d_sklo = nullptr, *d_ccoff = nullptr;   // d_ccoff = k_max * coff (C in elements)
  float *d_B = nullptr, *d_W = nullptr, *d_R = nullptr, *d_C = nullptr, *d_Bsk = nullptr;
  float* d_nrm = nullptr;       // squared column norms of B in nrm_parts parts, from the gather
  int nrm_parts = 1;
  float* d_F = nullptr;         // fine skeleton M B(:, I_B)
  int64_t* d_foff = nullptr;
  int32_t *d_J = nullptr, *d_k = nullptr;
  int* d_status = nullptr;
  int32_t* d_uptr = nullptr;
  double* d_part_spid = nullptr;
  int32_t *d_usub = nullptr, *d_urow = nullptr, *d_ucol = nullptr, *d_uptr_subid = nullptr;
  double* d_part_subid = nullptr;
  double* d_sub_err = nullptr;
  int* d_cnt = nullptr;   // [S + 1]
  std::vector<void*> allocs;
  int64_t workspace = 0;

  cudaError_t alloc(void** p, size_t bytes) {
    bytes = std::max<size_t>(bytes, 16);
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) {
      allocs.push_back(*p);
      workspace += (int64_t)bytes;
    }
    return e;
  }
  SubArgs args() const {
    SubArgs a;
    a.box = d_box;
    a.m = d_m;
    a.n = d_n;
    a.mc = d_mc;
    a.off = d_off;
    a.ld = d_ld;
    a.boff = d_boff;
    a.coff = d_coff;
    a.sklo = d_sklo;
    a.B = d_B;
    a.nrm = d_nrm;
    a.nrm_parts = nrm_parts;
    a.W = d_W;
    a.R = d_R;
    a.C = d_C;
    a.Bskel = d_Bsk;
    a.J = d_J;
    a.k = d_k;
    a.k_max = k_max;
    a.S = S;
    a.tol = tol;
    a.status = d_status;
    return a;
  }
  ErrArgs fold_args(const float* window, float* out, double* err, double* total) const {
    ErrArgs e;
    e.window = window;
    e.out = out;
    e.m = d_m;
    e.n = d_n;
    e.off = d_off;
    e.ld = d_ld;
    e.C = d_C;
    e.coff = nullptr;
    e.J = d_J;
    e.k = d_k;
    e.k_max = k_max;
    e.unit_sub = nullptr;
    e.unit_row0 = nullptr;
    e.unit_col0 = nullptr;
    e.part = nullptr;
    e.unit_base = 0;
    e.unit_ptr = nullptr;
    e.sub_cnt = d_cnt;
    e.all_cnt = d_cnt + S;
    e.err = err;
    e.sub_err = d_sub_err;
    e.total = total;
    e.S = S;
    e.srows = nullptr;
    return e;
  }
};

namespace {

spid_status sfail(spid_status st, const std::string& msg) {
  set_last_error(msg.c_str());
  return st;
}

#define SUB_CUDA(call)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return sfail(e_ == cudaErrorMemoryAllocation ? SPID_ERR_OOM : SPID_ERR_CUDA,         \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                    \
  } while (0)

int coarse_count(int e, int s) { return (e - 1) / s + 1 + ((e - 1) % s != 0 ? 1 : 0); }



spid_status check(spid_sub_plan_t P) {
  if (!P) return sfail(SPID_ERR_INVALID_ARG, "plan is NULL");
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != P->device) SUB_CUDA(cudaSetDevice(P->device));
  return SPID_OK;
}

spid_status check_window(const void* w, const char* what) {
  if (!w) return sfail(SPID_ERR_INVALID_ARG, std::string(what) + " is NULL");
  if (reinterpret_cast<uintptr_t>(w) % 16)
    return sfail(SPID_ERR_INVALID_ARG, std::string(what) + " must be 16-byte aligned");
  return SPID_OK;
}

// Device workspace and uploads shared by both plan kinds (the host tables
// of P are filled).  Takes ownership of P.
spid_status finish_plan(spid_sub_plan_s* P, spid_sub_plan_t* out) {
  if (cudaGetDevice(&P->device) != cudaSuccess) {
    delete P;
    return sfail(SPID_ERR_CUDA, "cudaGetDevice failed");
  }
  // The gathers read scattered sectors (a coarse line's 64 bytes, or single
  // points); filling whole 128-byte lines from DRAM doubled their reads.
  // 32-byte fetches: coarse gather 176 -> 155 us, point-set gather 339 ->
  // 247 us on the bench windows.  A hint of the current context; a refusal
  // changes nothing else, so its status is dropped.
  if (cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, 32) != cudaSuccess) cudaGetLastError();
  auto bail = [&](spid_status st) {
    spid_sub_plan_destroy(P);
    return st;
  };
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->device);
  if (subid_qr_smem_bytes(P->mc_max, P->n_max, P->k_max) + 1024 > (size_t)optin ||
      (!P->points && spid_interp_smem_bytes(P->mc_max, P->e_max) + 1024 > (size_t)optin)) {
    delete P;
    return sfail(SPID_ERR_UNSUPPORTED, "coarse grid too large for shared memory");
  }
#define SUB_ALLOC(ptr, bytes)                                                              \
  do {                                                                                     \
    cudaError_t e_ = P->alloc(reinterpret_cast<void**>(&(ptr)), (bytes));                  \
    if (e_ != cudaSuccess)                                                                 \
      return bail(sfail(e_ == cudaErrorMemoryAllocation ? SPID_ERR_OOM : SPID_ERR_CUDA,    \
                        std::string("cudaMalloc: ") + cudaGetErrorString(e_)));            \
  } while (0)
  const size_t S = (size_t)P->S;
  // the gather splits each column over nrm_parts warps when the window has
  // too few columns to fill the GPU (parts of >= 128 coarse rows)
  {
    const int64_t cols = (int64_t)P->S * P->n_max;
    int64_t parts = cols >= kGatherWarps ? 1 : (kGatherWarps + cols - 1) / cols;
    parts = std::min<int64_t>(parts, std::max<int64_t>(1, (P->mc_max + 127) / 128));
    P->nrm_parts = (int)parts;
  }
  SUB_ALLOC(P->d_box, sizeof(SubBox) * S);
  SUB_ALLOC(P->d_m, sizeof(int32_t) * S);
  SUB_ALLOC(P->d_n, sizeof(int32_t) * S);
  SUB_ALLOC(P->d_mc, sizeof(int32_t) * S);
  SUB_ALLOC(P->d_off, sizeof(int64_t) * S);
  SUB_ALLOC(P->d_ld, sizeof(int64_t) * S);
  SUB_ALLOC(P->d_boff, sizeof(int64_t) * S);
  SUB_ALLOC(P->d_coff, sizeof(int64_t) * S);
  SUB_ALLOC(P->d_sklo, sizeof(int64_t) * S);
  SUB_ALLOC(P->d_ccoff, sizeof(int64_t) * S);
  SUB_ALLOC(P->d_B, sizeof(float) * P->b_elems);
  SUB_ALLOC(P->d_nrm, sizeof(float) * (P->c_elems / P->k_max) * P->nrm_parts);
  SUB_ALLOC(P->d_W, sizeof(float) * P->b_elems);
  SUB_ALLOC(P->d_R, sizeof(float) * P->c_elems);
  SUB_ALLOC(P->d_C, sizeof(float) * P->c_elems);
  SUB_ALLOC(P->d_Bsk, sizeof(float) * P->sk_elems);
  SUB_ALLOC(P->d_F, sizeof(float) * P->f_elems);
  SUB_ALLOC(P->d_foff, sizeof(int64_t) * S);
  SUB_ALLOC(P->d_J, sizeof(int32_t) * S * P->k_max);
  SUB_ALLOC(P->d_k, sizeof(int32_t) * S);
  SUB_ALLOC(P->d_status, sizeof(int));
  SUB_ALLOC(P->d_uptr, sizeof(int32_t) * (S + 1));
  SUB_ALLOC(P->d_part_spid, sizeof(double) * 2 * (size_t)P->spid_units);
  SUB_ALLOC(P->d_usub, sizeof(int32_t) * P->usub.size());
  SUB_ALLOC(P->d_urow, sizeof(int32_t) * P->usub.size());
  SUB_ALLOC(P->d_ucol, sizeof(int32_t) * P->usub.size());
  SUB_ALLOC(P->d_uptr_subid, sizeof(int32_t) * (S + 1));
  SUB_ALLOC(P->d_part_subid, sizeof(double) * 2 * P->usub.size());
  SUB_ALLOC(P->d_sub_err, sizeof(double) * 2 * S);
  SUB_ALLOC(P->d_cnt, sizeof(int) * (S + 1));
  if (P->points) {
    SUB_ALLOC(P->d_crow, sizeof(int32_t) * P->crow.size());
    SUB_ALLOC(P->d_crow_off, sizeof(int64_t) * S);
    SUB_ALLOC(P->d_iidx, sizeof(int32_t) * P->iidx.size());
    SUB_ALLOC(P->d_iw, sizeof(float) * P->iw.size());
    SUB_ALLOC(P->d_ioff, sizeof(int64_t) * S);
  }
#undef SUB_ALLOC
  std::vector<int64_t> ccoff(S);
  for (size_t i = 0; i < S; ++i) ccoff[i] = (int64_t)P->k_max * P->coff[i];
  struct Up { void* dst; const void* src; size_t bytes; };
  const Up ups[] = {
      {P->d_box, P->box.data(), sizeof(SubBox) * P->box.size()},   // empty for point sets
      {P->d_m, P->m.data(), sizeof(int32_t) * S},
      {P->d_n, P->n.data(), sizeof(int32_t) * S},
      {P->d_mc, P->mc.data(), sizeof(int32_t) * S},
      {P->d_off, P->off.data(), sizeof(int64_t) * S},
      {P->d_ld, P->ld.data(), sizeof(int64_t) * S},
      {P->d_boff, P->boff.data(), sizeof(int64_t) * S},
      {P->d_coff, P->coff.data(), sizeof(int64_t) * S},
      {P->d_sklo, P->sklo.data(), sizeof(int64_t) * S},
      {P->d_foff, P->foff.data(), sizeof(int64_t) * S},
      {P->d_ccoff, ccoff.data(), sizeof(int64_t) * S},
      {P->d_uptr, P->uptr.data(), sizeof(int32_t) * (S + 1)},
      {P->d_usub, P->usub.data(), sizeof(int32_t) * P->usub.size()},
      {P->d_urow, P->urow.data(), sizeof(int32_t) * P->usub.size()},
      {P->d_ucol, P->ucol.data(), sizeof(int32_t) * P->usub.size()},
      {P->d_uptr_subid, P->uptr_subid.data(), sizeof(int32_t) * (S + 1)},
  };
  for (const Up& u : ups)
    if (u.bytes && cudaMemcpy(u.dst, u.src, u.bytes, cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(sfail(SPID_ERR_CUDA, "cudaMemcpy failed"));
  if (P->points) {
    const Up pts[] = {
        {P->d_crow, P->crow.data(), sizeof(int32_t) * P->crow.size()},
        {P->d_crow_off, P->crow_off.data(), sizeof(int64_t) * S},
        {P->d_iidx, P->iidx.data(), sizeof(int32_t) * P->iidx.size()},
        {P->d_iw, P->iw.data(), sizeof(float) * P->iw.size()},
        {P->d_ioff, P->ioff.data(), sizeof(int64_t) * S},
    };
    for (const Up& u : pts)
      if (cudaMemcpy(u.dst, u.src, u.bytes, cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(sfail(SPID_ERR_CUDA, "cudaMemcpy failed"));
  }
  if (cudaMemset(P->d_B, 0, sizeof(float) * P->b_elems) != cudaSuccess ||
      cudaMemset(P->d_nrm, 0, sizeof(float) * (P->c_elems / P->k_max) * P->nrm_parts) != cudaSuccess ||
      cudaMemset(P->d_k, 0, sizeof(int32_t) * S) != cudaSuccess ||
      cudaMemset(P->d_status, 0, sizeof(int)) != cudaSuccess ||
      cudaMemset(P->d_cnt, 0, sizeof(int) * (S + 1)) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess)
    return bail(sfail(SPID_ERR_CUDA, "cudaMemset failed"));
  *out = P;
  return SPID_OK;
}

}  // namespace

extern "C" {

spid_status spid_sub_plan_create(const spid_sub_desc* d, spid_sub_plan_t* out) {
  if (!d || !out) return sfail(SPID_ERR_INVALID_ARG, "desc/out is NULL");
  *out = nullptr;
  if (d->num_sub < 1 || d->num_sub > 65535)
    return sfail(SPID_ERR_INVALID_ARG, "num_sub must be in [1, 65535]");
  if (!d->box || !d->n || !d->off || !d->ld) return sfail(SPID_ERR_INVALID_ARG, "NULL array");
  if (d->k_max < 1 || d->k_max > kSubMaxK)
    return sfail(SPID_ERR_INVALID_ARG, "k_max must be in [1, 64]");
  if (!(d->tol >= 0.0)) return sfail(SPID_ERR_INVALID_ARG, "tol must be >= 0");
  for (int i = 0; i < 3; ++i)
    if (d->stride[i] < 1) return sfail(SPID_ERR_INVALID_ARG, "stride must be >= 1");
  if (d->flags != 0) return sfail(SPID_ERR_INVALID_ARG, "flags must be 0");
  spid_sub_plan_s* P = new spid_sub_plan_s();
  auto bail = [&](spid_status st) {
    spid_sub_plan_destroy(P);
    return st;
  };
  P->S = d->num_sub;
  P->k_max = d->k_max;
  P->tol = d->tol;
  int64_t bsum = 0, csum = 0, ssum = 0, units = 0;
  P->uptr.assign(P->S + 1, 0);
  P->uptr_subid.assign(P->S + 1, 0);
  for (int s = 0; s < P->S; ++s) {
    SubBox b;
    b.nq = d->box[4 * s];
    b.ez = d->box[4 * s + 1];
    b.ey = d->box[4 * s + 2];
    b.ex = d->box[4 * s + 3];
    if (b.nq < 1 || b.ez < 1 || b.ey < 1 || b.ex < 1) {
      delete P;
      return sfail(SPID_ERR_INVALID_ARG, "box extents must be >= 1 (subdomain " +
                                             std::to_string(s) + ")");
    }
    b.sz = d->stride[0];
    b.sy = d->stride[1];
    b.sx = d->stride[2];
    b.cz = coarse_count(b.ez, b.sz);
    b.cy = coarse_count(b.ey, b.sy);
    b.cx = coarse_count(b.ex, b.sx);
    const int64_t m = (int64_t)b.nq * b.ez * b.ey * b.ex;
    const int64_t mc = (int64_t)b.nq * b.cz * b.cy * b.cx;
    const int ns = d->n[s];
    if (m > INT32_MAX || ns < 1 || ns > kSubMaxN || d->ld[s] < m || d->off[s] < 0 ||
        d->off[s] % 4 || d->ld[s] % 4) {
      delete P;
      return sfail(SPID_ERR_INVALID_ARG, "bad n/off/ld for subdomain " + std::to_string(s));
    }
    if (mc > kSubMaxCoarse) {
      delete P;
      return sfail(SPID_ERR_UNSUPPORTED, "coarse grid of subdomain " + std::to_string(s) +
                                             " exceeds 40960 rows");
    }
    // SPID error units: columns x z blocks of about kSubUnitElems fine elements
    const int64_t per_col = std::max<int64_t>(1, (m + kSubUnitElems - 1) / kSubUnitElems);
    b.zc = (int)std::max<int64_t>(1, (b.ez + per_col - 1) / per_col);
    b.zblocks = (b.ez + b.zc - 1) / b.zc;
    b.div_ex = make_fastdiv((uint32_t)b.ex);
    b.div_plane = make_fastdiv((uint32_t)((int64_t)b.ey * b.ex));
    b.div_cx = make_fastdiv((uint32_t)b.cx);
    b.div_cy = make_fastdiv((uint32_t)b.cy);
    b.div_cz = make_fastdiv((uint32_t)b.cz);
    b.div_mc = make_fastdiv((uint32_t)mc);
    P->box.push_back(b);
    P->m.push_back((int32_t)m);
    P->n.push_back(ns);
    P->mc.push_back((int32_t)mc);
    P->off.push_back(d->off[s]);
    P->ld.push_back(d->ld[s]);
    P->boff.push_back(bsum);
    P->coff.push_back(csum);
    P->sklo.push_back(ssum);
    bsum += (int64_t)coarse_ld((int)mc) * ns;
    csum += ns;
    ssum += mc;
    P->uptr[s] = (int32_t)units;
    units += (int64_t)ns * b.zblocks;
    P->mc_max = std::max<int>(P->mc_max, (int)mc);
    P->m_max = std::max<int>(P->m_max, (int)m);
    P->foff.push_back(P->f_elems);
    P->f_elems += m * d->k_max;
    P->n_max = std::max(P->n_max, ns);
    P->e_max = std::max({P->e_max, b.ez, b.ey, b.ex});
    P->uptr_subid[s] = (int32_t)P->usub.size();
    for (int64_t r = 0; r < m; r += kErrRowBlock)
      for (int c = 0; c < ns; c += kErrColBlock) {
        P->usub.push_back(s);
        P->urow.push_back((int32_t)r);
        P->ucol.push_back(c);
      }
  }
  if (units > INT32_MAX) {
    delete P;
    return sfail(SPID_ERR_UNSUPPORTED, "too many error units");
  }
  P->uptr[P->S] = (int32_t)units;
  P->uptr_subid[P->S] = (int32_t)P->usub.size();
  P->spid_units = units;
  P->b_elems = bsum;
  P->c_elems = csum * P->k_max;
  P->sk_elems = ssum * P->k_max;
  return finish_plan(P, out);
}

spid_status spid_sub_plan_create_points(const spid_sub_points_desc* d, spid_sub_plan_t* out) {
  if (!d || !out) return sfail(SPID_ERR_INVALID_ARG, "desc/out is NULL");
  *out = nullptr;
  if (d->num_sub < 1 || d->num_sub > 65535)
    return sfail(SPID_ERR_INVALID_ARG, "num_sub must be in [1, 65535]");
  if (!d->m || !d->n || !d->off || !d->ld || !d->mc || !d->coarse_rows || !d->interp_idx ||
      !d->interp_w)
    return sfail(SPID_ERR_INVALID_ARG, "NULL array");
  if (d->k_max < 1 || d->k_max > kSubMaxK)
    return sfail(SPID_ERR_INVALID_ARG, "k_max must be in [1, 64]");
  if (!(d->tol >= 0.0)) return sfail(SPID_ERR_INVALID_ARG, "tol must be >= 0");
  if (d->stencil < 1 || d->stencil > kSubMaxStencil)
    return sfail(SPID_ERR_INVALID_ARG, "stencil must be in [1, 16]");
  if (d->flags != 0) return sfail(SPID_ERR_INVALID_ARG, "flags must be 0");
  spid_sub_plan_s* P = new spid_sub_plan_s();
  P->S = d->num_sub;
  P->k_max = d->k_max;
  P->tol = d->tol;
  P->points = true;
  P->t = d->stencil;
  const int t = d->stencil;
  int64_t bsum = 0, csum = 0, ssum = 0, rsum = 0, isum = 0;
  P->uptr.assign(P->S + 1, 0);
  P->uptr_subid.assign(P->S + 1, 0);
  for (int s = 0; s < P->S; ++s) {
    const int32_t m = d->m[s], ns = d->n[s], mc = d->mc[s];
    if (m < 1 || ns < 1 || ns > kSubMaxN || mc < 1 || mc > m || d->ld[s] < m || d->off[s] < 0 ||
        d->off[s] % 4 || d->ld[s] % 4) {
      delete P;
      return sfail(SPID_ERR_INVALID_ARG, "bad m/n/mc/off/ld for subdomain " + std::to_string(s));
    }
    if (mc > kSubMaxCoarse) {
      delete P;
      return sfail(SPID_ERR_UNSUPPORTED, "coarse set of subdomain " + std::to_string(s) +
                                             " exceeds 40960 rows");
    }
    for (int i = 0; i < mc; ++i) {
      const int32_t r = d->coarse_rows[ssum + i];
      if (r < 0 || r >= m) {
        delete P;
        return sfail(SPID_ERR_INVALID_ARG, "coarse row out of range in subdomain " + std::to_string(s));
      }
      P->crow.push_back(r);
    }
    for (int64_t e = 0; e < (int64_t)m * t; ++e) {
      const int32_t q = d->interp_idx[isum + e];
      const float w = d->interp_w[isum + e];
      if (q < 0 || q >= mc || !std::isfinite(w)) {
        delete P;
        return sfail(SPID_ERR_INVALID_ARG, "stencil index/weight invalid in subdomain " +
                                               std::to_string(s));
      }
      P->iidx.push_back(q);
      P->iw.push_back(w);
    }
    P->m.push_back(m);
    P->n.push_back(ns);
    P->mc.push_back(mc);
    P->off.push_back(d->off[s]);
    P->ld.push_back(d->ld[s]);
    P->boff.push_back(bsum);
    P->coff.push_back(csum);
    P->sklo.push_back(ssum);
    P->crow_off.push_back(ssum);
    P->ioff.push_back(isum);
    P->foff.push_back(P->f_elems);
    P->f_elems += (int64_t)m * d->k_max;
    bsum += (int64_t)coarse_ld(mc) * ns;
    csum += ns;
    ssum += mc;
    rsum += m;
    isum += (int64_t)m * t;
    P->mc_max = std::max<int>(P->mc_max, mc);
    P->m_max = std::max<int>(P->m_max, m);
    P->n_max = std::max(P->n_max, ns);
    P->uptr_subid[s] = (int32_t)P->usub.size();
    for (int64_t r = 0; r < m; r += kErrRowBlock)
      for (int c = 0; c < ns; c += kErrColBlock) {
        P->usub.push_back(s);
        P->urow.push_back((int32_t)r);
        P->ucol.push_back(c);
      }
  }
  P->uptr_subid[P->S] = (int32_t)P->usub.size();
  P->spid_units = 0;
  P->b_elems = bsum;
  P->c_elems = csum * P->k_max;
  P->sk_elems = ssum * P->k_max;
  return finish_plan(P, out);
}

spid_status spid_sub_plan_destroy(spid_sub_plan_t P) {
  if (!P) return SPID_OK;
  cudaSetDevice(P->device);
  cudaDeviceSynchronize();
  for (void* p : P->allocs) cudaFree(p);
  delete P;
  return SPID_OK;
}

spid_status spid_sub_plan_info(spid_sub_plan_t P, int64_t* mc_host, int64_t* workspace) {
  if (!P) return sfail(SPID_ERR_INVALID_ARG, "plan is NULL");
  if (mc_host)
    for (int s = 0; s < P->S; ++s) mc_host[s] = P->mc[s];
  if (workspace) *workspace = P->workspace;
  return SPID_OK;
}

spid_status spid_sub_sample(spid_sub_plan_t P, const float* window, int32_t col0, int32_t ncols,
                            spid_stream_t stream) {
  spid_status st = check(P);
  if (st != SPID_OK) return st;
  st = check_window(window, "window");
  if (st != SPID_OK) return st;
  if (col0 < 0 || ncols < 0) return sfail(SPID_ERR_INVALID_ARG, "negative column range");
  if (ncols == 0 || col0 >= P->n_max) return SPID_OK;
  ncols = std::min(ncols, P->n_max - col0);
  const int64_t max_work = (int64_t)P->mc_max * ncols;
  if (P->points)
    SUB_CUDA(launch_subsample_rows(P->args(), window, col0, ncols, P->d_crow, P->d_crow_off,
                                   max_work, (cudaStream_t)stream));
  else
    SUB_CUDA(launch_subsample(P->args(), window, col0, ncols, max_work, (cudaStream_t)stream));
  return SPID_OK;
}

spid_status spid_sub_finalize(spid_sub_plan_t P, spid_stream_t stream) {
  spid_status st = check(P);
  if (st != SPID_OK) return st;
  SUB_CUDA(launch_subid_qr(P->args(), P->mc_max, P->n_max, (cudaStream_t)stream));
  return SPID_OK;
}

static spid_status run_sub_error(spid_sub_plan_t P, const float* window, int32_t form,
                                 float* out, double* err_dev, double* total_dev,
                                 cudaStream_t cs) {
  if (form == SPID_FORM_SPID) {
    SubErrArgs a;
    a.a = P->args();
    a.e = P->fold_args(window, out, err_dev, total_dev);
    a.e.part = P->d_part_spid;
    a.e.unit_ptr = P->d_uptr;
    a.e.srows = P->d_mc;
    a.window = window;
    a.out = out;
    if (P->points) {
      SUB_CUDA(launch_fine_skeleton_points(P->args(), P->d_F, P->d_foff, P->d_iidx, P->d_iw,
                                           P->d_ioff, P->t, P->m_max, cs));
      if (!window) {   // reconstruction only: out = F C_B
        SUB_CUDA(launch_skeleton_product(P->args(), P->d_F, P->d_foff, out, P->m_max, P->n_max, cs));
        return SPID_OK;
      }
    } else if (window) {
      SUB_CUDA(launch_fine_skeleton(P->args(), P->d_F, P->d_foff, P->m_max, P->e_max, cs));
    }
    if (window) {
      // F = M B(:, I_B) once, then the rank-k error pass F C_B against A
      ErrArgs f = P->fold_args(window, out, err_dev, total_dev);
      f.coff = P->d_ccoff;
      f.unit_sub = P->d_usub;
      f.unit_row0 = P->d_urow;
      f.unit_col0 = P->d_ucol;
      f.part = P->d_part_subid;
      f.unit_ptr = P->d_uptr_subid;
      f.srows = P->d_mc;
      f.skel = P->d_F;
      f.skel_off = P->d_foff;
      SUB_CUDA(launch_error(f, (int)P->usub.size(), false, cs));
    } else {
      // reconstruction without the window: G = B(:, I_B) C_B, then M G
      SUB_CUDA(launch_coarse_recon(P->args(), (int64_t)P->mc_max * P->n_max, cs));
      SUB_CUDA(launch_spid_interp(a, P->spid_units, P->mc_max, P->e_max, cs));
    }
    return SPID_OK;
  }
  if (form == SPID_FORM_SUBID) {
    // A(:, I_B) C_B: the CUDA-core error pass of the sketched ID on these factors
    ErrArgs e = P->fold_args(window, out, err_dev, total_dev);
    e.coff = P->d_ccoff;
    e.unit_sub = P->d_usub;
    e.unit_row0 = P->d_urow;
    e.unit_col0 = P->d_ucol;
    e.part = P->d_part_subid;
    e.unit_ptr = P->d_uptr_subid;
    SUB_CUDA(launch_error(e, (int)P->usub.size(), false, cs));
    return SPID_OK;
  }
  return sfail(SPID_ERR_INVALID_ARG, "form must be SPID_FORM_SPID or SPID_FORM_SUBID");
}

spid_status spid_sub_error(spid_sub_plan_t P, const float* window, int32_t form,
                           double* err_dev, double* total_dev, spid_stream_t stream) {
  spid_status st = check(P);
  if (st != SPID_OK) return st;
  st = check_window(window, "window");
  if (st != SPID_OK) return st;
  return run_sub_error(P, window, form, nullptr, err_dev, total_dev, (cudaStream_t)stream);
}

spid_status spid_sub_reconstruct(spid_sub_plan_t P, const float* window, int32_t form, float* out,
                                 spid_stream_t stream) {
  spid_status st = check(P);
  if (st != SPID_OK) return st;
  st = check_window(out, "out");
  if (st != SPID_OK) return st;
  if (form == SPID_FORM_SUBID) {
    st = check_window(window, "window");
    if (st != SPID_OK) return st;
  } else if (window) {
    st = check_window(window, "window");
    if (st != SPID_OK) return st;
  }
  return run_sub_error(P, window, form, out, nullptr, nullptr, (cudaStream_t)stream);
}

spid_status spid_sub_get_factors(spid_sub_plan_t P, int32_t* k_host, int32_t* J_host,
                                 float* C_host, float* Bskel_host, spid_stream_t stream) {
  spid_status st = check(P);
  if (st != SPID_OK) return st;
  SUB_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  if (k_host) SUB_CUDA(cudaMemcpy(k_host, P->d_k, sizeof(int32_t) * P->S, cudaMemcpyDeviceToHost));
  if (J_host)
    SUB_CUDA(cudaMemcpy(J_host, P->d_J, sizeof(int32_t) * P->S * P->k_max, cudaMemcpyDeviceToHost));
  if (C_host) SUB_CUDA(cudaMemcpy(C_host, P->d_C, sizeof(float) * P->c_elems, cudaMemcpyDeviceToHost));
  if (Bskel_host)
    SUB_CUDA(cudaMemcpy(Bskel_host, P->d_Bsk, sizeof(float) * P->sk_elems, cudaMemcpyDeviceToHost));
  return SPID_OK;
}

spid_status spid_sub_get_coarse(spid_sub_plan_t P, float* B_host, spid_stream_t stream) {
  spid_status st = check(P);
  if (st != SPID_OK) return st;
  if (!B_host) return sfail(SPID_ERR_INVALID_ARG, "B_host is NULL");
  SUB_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  // the device columns are padded to coarse_ld(m_c) rows; the host gets m_c
  int64_t hoff = 0;
  for (int s = 0; s < P->S; ++s) {
    const size_t mc = (size_t)P->mc[s];
    SUB_CUDA(cudaMemcpy2D(B_host + hoff, sizeof(float) * mc, P->d_B + P->boff[s],
                          sizeof(float) * (size_t)coarse_ld((int)mc), sizeof(float) * mc,
                          (size_t)P->n[s], cudaMemcpyDeviceToHost));
    hoff += (int64_t)mc * P->n[s];
  }
  return SPID_OK;
}

spid_status spid_sub_device_status(spid_sub_plan_t P, spid_stream_t stream) {
  spid_status st = check(P);
  if (st != SPID_OK) return st;
  SUB_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  int v = 0;
  SUB_CUDA(cudaMemcpy(&v, P->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  SUB_CUDA(cudaMemset(P->d_status, 0, sizeof(int)));
  if (v & kStatusNonfinite) return sfail(SPID_ERR_NONFINITE, "non-finite value in a coarse matrix");
  return SPID_OK;
}

}  // extern "C"
