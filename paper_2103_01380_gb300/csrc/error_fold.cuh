// error_fold.cuh -- the deterministic end of both error passes (Section 5.1
// relative Frobenius error, Section 2 compression-factor sums): once the last
// work unit of subdomain s has stored its {e2, a2} partial, one warp sums the
// subdomain's partials in unit order, and the last subdomain to finish sums
// the window totals {sum e2, sum a2, sum m n, sum k (r + n)} in subdomain
// order, r = the rows stored per skeleton column (m, or m_c for a coarse-grid
// skeleton, Section 5.2), and, when the plan labels its subdomains by QoI, the
// per-QoI sums of e2 and a2.  Every counter is reset by the warp that
// completes it.
#pragma once

#include "spid_internal.cuh"

namespace spid {

// Called by the 32 lanes of one warp after a device-wide fence, by the CTA
// whose unit completed subdomain s (its atomic on sub_cnt[s] returned the
// last count).  Units of s are a.unit_ptr[s] .. a.unit_ptr[s + 1] of a.part.
__device__ __forceinline__ void error_fold_subdomain(const ErrArgs& a, int s, int lane) {
  __threadfence();
  const int u0 = a.unit_ptr[s], u1 = a.unit_ptr[s + 1];
  double es = 0.0, as = 0.0;
  for (int q = u0 + lane; q < u1; q += 32) {
    es += __ldcg(a.part + 2 * (int64_t)q);
    as += __ldcg(a.part + 2 * (int64_t)q + 1);
  }
  for (int o = 16; o > 0; o >>= 1) {
    es += __shfl_xor_sync(0xffffffffu, es, o);
    as += __shfl_xor_sync(0xffffffffu, as, o);
  }
  int last_all = 0;
  if (lane == 0) {
    a.sub_err[2 * s] = es;
    a.sub_err[2 * s + 1] = as;
    if (a.err) { a.err[2 * s] = es; a.err[2 * s + 1] = as; }
    a.sub_cnt[s] = 0;
    __threadfence();
    last_all = (atomicAdd(a.all_cnt, 1) == a.S - 1);
  }
  last_all = __shfl_sync(0xffffffffu, last_all, 0);
  if (!last_all) return;
  // ---- last subdomain of the window: fixed-order window totals
  __threadfence();
  double te = 0.0, ta = 0.0, mn = 0.0, kd = 0.0;
  for (int q = lane; q < a.S; q += 32) {
    te += __ldcg(a.sub_err + 2 * (int64_t)q);
    ta += __ldcg(a.sub_err + 2 * (int64_t)q + 1);
    const double mq = (double)a.m[q], nq = (double)a.n[q];
    const double sq = a.srows ? (double)a.srows[q] : mq;   // coarse skeleton: m_c rows
    mn += mq * nq;
    kd += (double)a.k[q] * (sq + nq);
  }
  for (int o = 16; o > 0; o >>= 1) {
    te += __shfl_xor_sync(0xffffffffu, te, o);
    ta += __shfl_xor_sync(0xffffffffu, ta, o);
    mn += __shfl_xor_sync(0xffffffffu, mn, o);
    kd += __shfl_xor_sync(0xffffffffu, kd, o);
  }
  if (lane == 0 && a.total) { a.total[0] = te; a.total[1] = ta; a.total[2] = mn; a.total[3] = kd; }
  // per-QoI totals (Section 5.1 reports each QoI's error): the subdomains of
  // QoI g, lane-strided in subdomain order, then the same fixed tree
  for (int g = 0; g < a.num_qoi && a.total; ++g) {
    double ge = 0.0, ga = 0.0;
    for (int q = lane; q < a.S; q += 32) {
      if (a.qoi[q] != g) continue;
      ge += __ldcg(a.sub_err + 2 * (int64_t)q);
      ga += __ldcg(a.sub_err + 2 * (int64_t)q + 1);
    }
    for (int o = 16; o > 0; o >>= 1) {
      ge += __shfl_xor_sync(0xffffffffu, ge, o);
      ga += __shfl_xor_sync(0xffffffffu, ga, o);
    }
    if (lane == 0) { a.total[4 + 2 * g] = ge; a.total[5 + 2 * g] = ga; }
  }
  if (lane == 0) *a.all_cnt = 0;
}

}  // namespace spid
