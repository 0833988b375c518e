// spid_api.cu -- the C ABI of libspid (include/spid.h): plan creation, the
// per-call work schedules and the kernel launches of the hot path
//   sketch (a1-a2) -> finalize (a3-a5) -> error / reconstruct (a6), CF (a7).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/spid.h"
#include "spid_internal.cuh"


using namespace spid;

namespace {

thread_local std::string g_last_error;

spid_status fail(spid_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

#define SPID_CUDA(call)                                                                    \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(e_ == cudaErrorMemoryAllocation ? SPID_ERR_OOM : SPID_ERR_CUDA,          \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                     \
  } while (0)

// One sketch launch plan for a window column range.
struct Schedule {
  int grid = 0;            // CTAs per launch (per subdomain in per-subdomain mode)
  int nprob = 0;
  int max_tiles = 1;       // 128-column tiles of the widest problem (TF32)
  int stages = 1;          // TF32 pipeline depth
  int simt_tj = 1;         // CUDA-core sketch: columns per thread (64 tj >= widest problem or pack)
  bool packed = false;     // the tables hold pack segments (tensor-core, or batched CUDA-core)
  std::vector<int> cta_base_of_sub, prob_base_of_sub, nprob_of_sub;
  void* dev = nullptr;     // one device block holding every table below
  const Problem* probs = nullptr;
  const Segment* segs = nullptr;
  const int32_t* seg_ptr = nullptr;
  const int64_t* slot_off = nullptr;
  const int32_t* pslot_ptr = nullptr;
  const int32_t* pslots = nullptr;
  int* prob_cnt = nullptr;   // per-problem completed-segment counters
  const Slice* slices = nullptr;
  const Pack* packs = nullptr;
  const PackSegment* psegs = nullptr;
  int64_t partial_elems = 0;
};

}  // namespace

void spid::set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

namespace spid {
PlanView plan_view(spid_plan_t P);
// A plan whose sketch draws l_sketch >= k_max + p rows of Omega while its QR
// reads the first k_max + p (the two-stage driver's block plans).
spid_status plan_create_sketch_rows(const spid_plan_desc* d, spid_stream_t stream, int l_sketch,
                                    spid_plan_t* out);
}

// Tile shapes and schedules of one plan (spid_tuning without the timings).
struct TuneCfg {
  int pack_slices = kPackSlices;   // 64-column slices per Omega chunk (CUDA-core plans: 2)
  int slice_major = 0;             // tensor-core sketch: packs cut slice index major
  int slice_cols = kSliceCols;     // tensor-core sketch: columns per slice (TMA box width)
  int stages = 0;                  // tensor-core sketch pipeline depth, 0 = as many as fit
  int ctas_per_sm = 0;             // CUDA-core sketch CTAs per SM, 0 = by register budget
  int err_path = 0;                // 0 CUDA cores, 1 tensor cores
  int err_rows = kErrRowBlock;     // error-pass unit rows
  int err_cols = kErrColBlock;     // error-pass unit columns
};

struct spid_plan_s {
  int device = 0;
  int num_sms = 0;
  size_t smem_optin = 0;
  int S = 0;
  std::vector<int32_t> m, n;
  std::vector<int64_t> off, ld;
  int n_max = 0;
  int k_max = 0, p = 0, l = 0, l_pad = 0;
  int l_sk = 0;                 // rows of Omega the sketch draws (>= l; the QR reads the first l)
  double tol = 0.0;
  int prec = SPID_PREC_FP32;
  uint32_t flags = 0;
  uint64_t seed = 0;
  size_t esz = 4;
  // layout: boxes of a global field (geo[s].ex > 0) or contiguous blocks
  bool boxes = false;
  std::vector<RowGeom> geo;
  int64_t window_extent = 0;    // elements of the window any call reads, from its base
  // per-QoI error totals (num_qoi = 0: none)
  std::vector<int32_t> qoi;
  int num_qoi = 0;
  // Tensor maps of the window (tensor-core plans): map s < S covers subdomain
  // s alone; map S + g is shared by every subdomain with tma_group[s] == g,
  // which sits at origin tma_org[4 s .. 4 s + 3] of it.  A pack whose slices
  // read through one shared map touches one descriptor instead of one per
  // subdomain.
  struct TmaGroup {
    int64_t base;        // element offset of the map's origin in the window
    int rank;            // 2 (rows, columns) or 5 (x, y, z, q, columns)
    int64_t dims[5];     // extents, innermost first
    int64_t strides[4];  // element strides of dims 1 ..
  };
  std::vector<TmaGroup> tma_groups;
  std::vector<int32_t> tma_group;
  std::vector<int32_t> tma_org;
  int num_tmaps() const { return S + (int)tma_groups.size(); }
  bool fp64() const { return prec == SPID_PREC_FP64; }
  bool per_sub() const { return (flags & SPID_FLAG_PER_SUBDOMAIN) != 0; }
  bool tensor_core() const { return prec >= SPID_PREC_TF32; }
  bool bf16() const { return prec == SPID_PREC_BF16 || prec == SPID_PREC_BF16X3; }
  bool err_tc_possible() const {
    return tensor_core() && !per_sub() && !boxes && k_max <= kErrTcKMax &&
           smem_optin >= error_tc_smem_bytes();
  }
  double u_mode() const {
    switch (prec) {
      case SPID_PREC_FP64: return std::ldexp(1.0, -53);
      case SPID_PREC_TF32: return std::ldexp(1.0, -11);
      case SPID_PREC_BF16: return std::ldexp(1.0, -9);
      case SPID_PREC_BF16X3: return std::ldexp(1.0, -16);
      default: return std::ldexp(1.0, -24);
    }
  }

  // device state
  int32_t* d_m = nullptr;
  int32_t* d_n = nullptr;
  RowGeom* d_geo = nullptr;     // boxes layout only
  int32_t* d_qoi = nullptr;     // num_qoi > 0 only
  int64_t* d_off = nullptr;
  int64_t* d_ld = nullptr;
  int64_t* d_yoff = nullptr;
  int64_t* d_coff = nullptr;
  void* d_Y = nullptr;
  void* d_C = nullptr;
  int32_t* d_J = nullptr;
  int32_t* d_k = nullptr;
  int* d_status = nullptr;
  int32_t* d_unit_sub = nullptr;
  int32_t* d_unit_row0 = nullptr;
  int32_t* d_unit_col0 = nullptr;
  int32_t* d_unit_ptr = nullptr;
  double* d_err_part = nullptr;
  double* d_sub_err = nullptr;
  int* d_err_cnt = nullptr;     // [S + 1] error-pass completion counters
  // tensor-core error pass: segments of 128-row tiles over one CTA per SM
  int err_tc_grid = 0;          // > 0 once the tensor-core error schedule exists
  ErrSeg* d_err_segs = nullptr;
  int32_t* d_err_seg_ptr = nullptr;   // [grid + 1]
  int32_t* d_err_tc_ptr = nullptr;    // [S + 1] segments of each subdomain
  double* d_err_tc_part = nullptr;    // [segments][2]
  void* d_tmaps = nullptr;
  void* d_partial = nullptr;
  int64_t partial_cap = 0;
  int units = 0;
  int units_cap = 0;            // unit arrays are sized for the smallest unit shape
  std::vector<int32_t> unit_ptr;
  TuneCfg tune;
  float tuned_sketch_ms = 0.f, tuned_error_ms = 0.f;
  int64_t y_elems = 0, c_elems = 0;
  int64_t workspace = 0;

  const void* bound_window = nullptr;
  int live_graphs = 0;          // graphs captured from this plan and not yet destroyed
  std::map<std::pair<int, int>, Schedule> schedules;
  std::vector<void*> allocs;
  std::mutex mu;                // schedule cache
  std::mutex tune_mu;           // set_tuning / autotune

  cudaError_t alloc(void** p, size_t bytes) {
    bytes = std::max<size_t>(bytes, 16);
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) {
      allocs.push_back(*p);
      workspace += (int64_t)bytes;
    }
    return e;
  }
  int group_cols() const {
    return tensor_core() ? tune.pack_slices * kSliceCols : sketch_simt_group_cols(fp64());
  }
  int group_cols_max() const {
    return tensor_core() ? kPackSlices * kSliceCols : sketch_simt_group_cols(fp64());
  }
  int sketch_grid() const {
    if (tensor_core()) return num_sms;
    if (tune.ctas_per_sm > 0) return tune.ctas_per_sm * num_sms;
    return (!fp64() && l_pad <= 32) || (fp64() && l_pad <= 16) ? 2 * num_sms : num_sms;
  }
};

namespace {

// One launch per subdomain (SPID_FLAG_PER_SUBDOMAIN) keeps at most this many
// CUDA-core CTAs per SM: its partial-sum workspace holds a slot per CTA per
// subdomain.
constexpr int kPerSubMaxCtasPerSm = 2;
// default pack width of the batched CUDA-core sketch
constexpr int kSimtPackSlices = 2;
constexpr int kPerSubMinChunks = 8;

// Build the sketch schedule for window columns [col0, col0 + ncols).
//
// Problems: every subdomain restricted to groups of up to group_cols()
// columns of the range.  Work units: a problem (CUDA-core kernels) or a pack
// of problems with equal m cut into 64-column slices (tensor-core kernels,
// which regenerate Omega once per chunk for the whole pack).  The chunks of all
// units are partitioned over the CTAs, balanced by bytes; consecutive chunks of
// one unit on one CTA form a segment, which writes one partial slot per
// problem it touches.
spid_status build_schedule(spid_plan_t P, int col0, int ncols, Schedule& sc) {
  const int CG = P->group_cols();
  int G = P->sketch_grid();
  const bool tc = P->tensor_core();
  const int W = tc ? P->tune.slice_cols : kSliceCols;                 // slice width
  // slices per pack; CUDA-core packs stay within the kernel's widest column tile
  const int pack_cap = tc ? P->tune.pack_slices * kSliceCols / W
                          : std::min(P->tune.pack_slices, sketch_simt_group_cols(P->fp64()) / kSliceCols);
  // ---- problems, subdomain by subdomain; with packing, ordered by m
  std::vector<int> subs(P->S);
  for (int s = 0; s < P->S; ++s) subs[s] = s;
  // packs share one Omega chunk and one chunk decode: group equal m and box
  // shape; inside a class, order by position in the window, so that a pack's
  // subdomains are neighbours in memory (for one-QoI boxes of a global field:
  // boxes adjacent along x with the same QoI, whose x-runs form one contiguous
  // row of each snapshot)
  auto shape = [&](int s) {
    const RowGeom& g = P->geo[s];
    return std::make_tuple(P->m[s], g.ex, g.ey, g.ez);
  };
  if (!P->per_sub())
    std::stable_sort(subs.begin(), subs.end(), [&](int x, int y) {
      return std::make_tuple(shape(x), P->off[x]) < std::make_tuple(shape(y), P->off[y]);
    });
  std::vector<Problem> probs;
  std::vector<int> prob_sub_first(P->S + 1, 0);   // per-subdomain mode: problems of s
  struct Unit { int nch; double w; int prob0; int nprob; int pack; };
  std::vector<Unit> units;
  std::vector<Slice> slices;
  std::vector<Pack> packs;
  // The map a slice's TMA box reads: the subdomain's shared map when the whole
  // box lies inside its columns, else its own map, whose column extent
  // zero-fills the box past the subdomain's last column.
  auto place = [&](Slice& sl) {
    const int s = sl.sub;
    const int g = tc && !P->tma_group.empty() ? P->tma_group[s] : -1;
    if (g >= 0 && sl.col0 + W <= P->n[s]) {
      sl.map = P->S + g;
      sl.tx = P->tma_org[4 * s + 0];
      sl.ty = P->tma_org[4 * s + 1];
      sl.tz = P->tma_org[4 * s + 2];
      sl.tq = P->tma_org[4 * s + 3];
    } else {
      sl.map = s;
      sl.tx = sl.ty = sl.tz = sl.tq = 0;
    }
  };
  // Batched tensor-core plans: the 64-column slices of every subdomain of one m
  // form a stream that is cut into packs of pack_slices slices, so every pack
  // but the last of an m-class is full whatever the window lengths; a problem
  // (the fold unit) is a subdomain's run of consecutive slices inside one pack.
  // A chunk's weight counts its columns plus a fixed share for the Omega chunk
  // it regenerates.
  const bool streamed = !P->per_sub();
  const bool packed = tc || streamed;   // pack segments (else one problem per segment)
  if (streamed) {
    // Packs are cut from the stream of 64-column slices of one shape class,
    // either subdomain major (all slices of one subdomain, then the next: a
    // pack holds up to 512 consecutive columns of one subdomain; the default)
    // or slice index major (slice j of every subdomain, then slice j + 1: a
    // pack holds 8 subdomains at the same columns); the tuner measures both.
    // A chunk's weight counts its columns, a share for the Omega chunk it
    // regenerates, and the pack's epilogue (TMEM drain and fold) spread over
    // the pack's chunks, so CTAs that get many short packs (small m) get fewer
    // chunks.
    Pack pk{};
    int cols = 0;
    auto close_pack = [&]() {
      if (pk.nslices == 0) return;
      const int nch = (pk.m + kChunkRows - 1) / kChunkRows;
      units.push_back({nch, (double)(cols + kSliceCols / 2) * (1.0 + kPackOverheadChunks / nch),
                       pk.prob0, pk.nprob, (int)packs.size()});
      packs.push_back(pk);
      pk = Pack{};
      cols = 0;
    };
    auto add_slice = [&](int s, int c, int end) {
      if (pk.nslices == pack_cap) close_pack();
      if (pk.nslices == 0) {
        pk.slice0 = (int)slices.size();
        pk.m = P->m[s];
        pk.prob0 = (int)probs.size();
        pk.nprob = 0;
        pk.ex = P->geo[s].ex;
        pk.ey = P->geo[s].ey;
        pk.ez = P->geo[s].ez;
      }
      const int nc = std::min(W, end - c);
      // consecutive slices of one subdomain in a pack share a problem
      if (pk.nprob == 0 || probs.back().sub != s || probs.back().col0 + probs.back().ncols != c) {
        Problem pb;
        pb.sub = s;
        pb.col0 = c;
        pb.ncols = 0;
        pb.m = P->m[s];
        pb.off = P->off[s];
        pb.ld = P->ld[s];
        pb.geo = P->geo[s];
        probs.push_back(pb);
        ++pk.nprob;
      }
      Slice sl;
      sl.prob = (int)probs.size() - 1;
      sl.sub = s;
      sl.col0 = c;
      sl.ncols = nc;
      sl.out_col = c - probs.back().col0;
      sl.member = pk.nprob - 1;
      place(sl);
      slices.push_back(sl);
      probs.back().ncols += nc;
      ++pk.nslices;
      cols += nc;
    };
    for (size_t q0 = 0; q0 < subs.size();) {
      // one shape class: subs[q0 .. q1)
      size_t q1 = q0 + 1;
      while (q1 < subs.size() && shape(subs[q1]) == shape(subs[q0])) ++q1;
      close_pack();
      int jmax = 0;
      for (size_t q = q0; q < q1; ++q) {
        const int end = std::min<int64_t>((int64_t)col0 + ncols, P->n[subs[q]]);
        jmax = std::max(jmax, end > col0 ? (end - col0 + W - 1) / W : 0);
      }
      if (P->tune.slice_major) {
        for (int j = 0; j < jmax; ++j)
          for (size_t q = q0; q < q1; ++q) {
            const int s = subs[q];
            const int end = std::min<int64_t>((int64_t)col0 + ncols, P->n[s]);
            const int c = col0 + j * W;
            if (c < end) add_slice(s, c, end);
          }
      } else {
        for (size_t q = q0; q < q1; ++q) {
          const int s = subs[q];
          const int end = std::min<int64_t>((int64_t)col0 + ncols, P->n[s]);
          for (int c = col0; c < end; c += W) add_slice(s, c, end);
        }
      }
      q0 = q1;
    }
    close_pack();
  }
  for (int s : subs) {
    if (streamed) break;
    prob_sub_first[s] = (int)probs.size();
    const int end = std::min<int64_t>((int64_t)col0 + ncols, P->n[s]);
    for (int c = col0; c < end; c += CG) {
      Problem pb;
      pb.sub = s;
      pb.col0 = c;
      pb.ncols = std::min(CG, end - c);
      pb.m = P->m[s];
      pb.off = P->off[s];
      pb.ld = P->ld[s];
      pb.geo = P->geo[s];
      probs.push_back(pb);
    }
  }
  std::vector<int> prob_sub_last(P->S, 0);
  for (int s : subs) {
    const int end = std::min<int64_t>((int64_t)col0 + ncols, P->n[s]);
    prob_sub_last[s] = prob_sub_first[s] + (end > col0 ? (end - col0 + CG - 1) / CG : 0);
  }
  // CUDA-core kernels: the register tile fits the widest problem of this
  // column range, and the grid holds as many CTAs per SM as that tile allows
  if (!tc) {
    if (streamed) {
      // packed: one 64-column group per slice, the tile fits the widest pack
      int mx = 1;
      for (const Pack& pk : packs) mx = std::max(mx, pk.nslices);
      int tj = 1;
      while (tj < mx) tj *= 2;
      sc.simt_tj = tj;
    } else {
      int max_cols = 1;
      for (const Problem& pb : probs) max_cols = std::max(max_cols, pb.ncols);
      sc.simt_tj = sketch_simt_tj(P->fp64(), max_cols);
    }
    int cps = P->tune.ctas_per_sm > 0 ? P->tune.ctas_per_sm
                                      : sketch_simt_ctas_per_sm(P->fp64(), P->l_pad, sc.simt_tj);
    if (P->per_sub()) cps = std::min(cps, kPerSubMaxCtasPerSm);
    G = cps * P->num_sms;
  }
  // ---- work units
  auto make_units = [&](int p0, int p1) {
    if (!tc) {
      for (int p = p0; p < p1; ++p)
        units.push_back({(probs[p].m + kChunkRows - 1) / kChunkRows, (double)probs[p].ncols, p, 1, -1});
      return;
    }
    int p = p0;
    while (p < p1) {
      Pack pk;
      pk.slice0 = (int)slices.size();
      pk.nslices = 0;
      pk.m = probs[p].m;
      pk.prob0 = p;
      pk.nprob = 0;
      pk.ex = probs[p].geo.ex;
      pk.ey = probs[p].geo.ey;
      pk.ez = probs[p].geo.ez;
      int cols = 0;
      while (p < p1 && probs[p].m == pk.m && probs[p].geo.ex == pk.ex &&
             probs[p].geo.ey == pk.ey && probs[p].geo.ez == pk.ez &&
             pk.nslices + (probs[p].ncols + W - 1) / W <= pack_cap) {
        for (int c = 0; c < probs[p].ncols; c += W) {
          Slice sl;
          sl.prob = p;
          sl.sub = probs[p].sub;
          sl.col0 = probs[p].col0 + c;
          sl.ncols = std::min(W, probs[p].ncols - c);
          sl.out_col = c;
          sl.member = pk.nprob;
          place(sl);
          slices.push_back(sl);
          ++pk.nslices;
        }
        cols += probs[p].ncols;
        ++pk.nprob;
        ++p;
      }
      units.push_back({(pk.m + kChunkRows - 1) / kChunkRows, (double)cols, pk.prob0, pk.nprob,
                       (int)packs.size()});
      packs.push_back(pk);
    }
  };
  std::vector<Segment> segs;
  std::vector<PackSegment> psegs;
  std::vector<int32_t> seg_ptr;
  std::vector<int64_t> slot_off;
  int64_t slot_total = 0;
  std::vector<std::vector<int32_t>> slots_of_prob(probs.size());
  // chunk i of the units [u0, u1) goes to the CTA whose equal share of the
  // total weight contains the chunk's midpoint; appends G + 1 entries to
  // seg_ptr.  A CUDA-core launch for one subdomain spreads its chunks over only
  // as many CTAs as keep kPerSubMinChunks each (the rest find no work): every
  // CTA that works writes a partial slot, and one CTA folds them all.
  auto partition = [&](int u0, int u1) {
    double W = 0.0;
    int nch_all = 0;
    for (int u = u0; u < u1; ++u) {
      W += units[u].nch * units[u].w;
      nch_all += units[u].nch;
    }
    const int Gw = (!tc && P->per_sub()) ? std::max(1, std::min(G, nch_all / kPerSubMinChunks)) : G;
    struct Run { int unit, chunk0, chunk1; };
    std::vector<std::vector<Run>> per_cta(G);
    double acc = 0.0;
    for (int u = u0; u < u1; ++u) {
      const double w = units[u].w;
      for (int ch = 0; ch < units[u].nch; ++ch) {
        int c = W > 0 ? (int)((acc + 0.5 * w) * Gw / W) : 0;
        c = std::min(std::max(c, 0), Gw - 1);
        std::vector<Run>& v = per_cta[c];
        if (!v.empty() && v.back().unit == u && v.back().chunk1 == ch) v.back().chunk1 = ch + 1;
        else v.push_back({u, ch, ch + 1});
        acc += w;
      }
    }
    for (int c = 0; c < G; ++c) {
      seg_ptr.push_back((int32_t)(packed ? psegs.size() : segs.size()));
      for (const Run& r : per_cta[c]) {
        const Unit& un = units[r.unit];
        const int32_t first_slot = (int32_t)slot_off.size();
        for (int q = 0; q < un.nprob; ++q) {
          const int p = un.prob0 + q;
          slots_of_prob[p].push_back((int32_t)slot_off.size());
          slot_off.push_back(slot_total);
          slot_total += (int64_t)probs[p].ncols * P->l_pad;
        }
        if (packed) psegs.push_back({un.pack, r.chunk0, r.chunk1, first_slot});
        else segs.push_back({un.prob0, r.chunk0, r.chunk1, first_slot});
      }
    }
    seg_ptr.push_back((int32_t)(packed ? psegs.size() : segs.size()));
  };
  sc.cta_base_of_sub.assign(P->S, 0);
  sc.prob_base_of_sub.assign(P->S, 0);
  sc.nprob_of_sub.assign(P->S, 0);
  if (P->per_sub()) {
    // one launch of G CTAs per subdomain: seg_ptr has S blocks of G + 1 entries
    for (int s = 0; s < P->S; ++s) {
      sc.cta_base_of_sub[s] = (int)seg_ptr.size();
      sc.prob_base_of_sub[s] = prob_sub_first[s];
      sc.nprob_of_sub[s] = prob_sub_last[s] - prob_sub_first[s];
      const int u0 = (int)units.size();
      make_units(prob_sub_first[s], prob_sub_last[s]);
      partition(u0, (int)units.size());
    }
  } else {
    if (!streamed) make_units(0, (int)probs.size());
    partition(0, (int)units.size());
  }
  std::vector<int32_t> pslot_ptr(probs.size() + 1, 0), pslots;
  for (size_t p = 0; p < probs.size(); ++p) {
    pslot_ptr[p] = (int32_t)pslots.size();
    for (int32_t q : slots_of_prob[p]) pslots.push_back(q);
  }
  pslot_ptr[probs.size()] = (int32_t)pslots.size();
  int max_slices = 1;
  for (const Pack& pk : packs) max_slices = std::max(max_slices, pk.nslices);

  sc.grid = G;
  sc.packed = packed;
  sc.nprob = (int)probs.size();
  sc.max_tiles = tc ? (max_slices * W + 127) / 128 : 1;
  sc.partial_elems = slot_total;
  if (slot_total > P->partial_cap)
    return fail(SPID_ERR_INVALID_ARG, "sketch schedule exceeds the partial workspace");
  if (tc) {
    const bool split = P->prec == SPID_PREC_BF16X3;
    const int mt = sc.max_tiles;
    const size_t fixed = P->bf16() ? sketch_bf16_smem_bytes(0, mt, P->l_pad, split)
                                   : sketch_tc_smem_bytes(0, mt, P->l_pad);
    const size_t per_stage = (P->bf16() ? sketch_bf16_smem_bytes(1, mt, P->l_pad, split)
                                        : sketch_tc_smem_bytes(1, mt, P->l_pad)) - fixed;
    int stages = (int)((P->smem_optin - fixed) / per_stage);
    stages = std::min(stages, sketch_tc_max_stages());
    if (P->tune.stages > 0) stages = std::min(stages, P->tune.stages);
    if (stages < 2) return fail(SPID_ERR_UNSUPPORTED, "not enough shared memory for the sketch pipeline");
    sc.stages = stages;
  }
  // one device block for all tables (16-byte aligned pieces)
  std::vector<unsigned char> host;
  std::vector<size_t> at;
  auto put = [&](const void* src, size_t bytes) {
    at.push_back(host.size());
    const size_t span = (std::max<size_t>(bytes, 16) + 15) / 16 * 16;
    host.resize(host.size() + span, 0);
    if (bytes && src) std::memcpy(host.data() + at.back(), src, bytes);
  };
  put(probs.data(), sizeof(Problem) * probs.size());                 // 0
  put(segs.data(), sizeof(Segment) * segs.size());                   // 1
  put(seg_ptr.data(), sizeof(int32_t) * seg_ptr.size());             // 2
  put(slot_off.data(), sizeof(int64_t) * slot_off.size());           // 3
  put(pslot_ptr.data(), sizeof(int32_t) * pslot_ptr.size());         // 4
  put(pslots.data(), sizeof(int32_t) * pslots.size());               // 5
  put(nullptr, sizeof(int) * probs.size());                          // 6: counters start at zero
  put(slices.data(), sizeof(Slice) * slices.size());                 // 7
  put(packs.data(), sizeof(Pack) * packs.size());                    // 8
  put(psegs.data(), sizeof(PackSegment) * psegs.size());             // 9
  SPID_CUDA(P->alloc(&sc.dev, host.size()));
  SPID_CUDA(cudaMemcpy(sc.dev, host.data(), host.size(), cudaMemcpyHostToDevice));
  unsigned char* d = static_cast<unsigned char*>(sc.dev);
  sc.probs = reinterpret_cast<const Problem*>(d + at[0]);
  sc.segs = reinterpret_cast<const Segment*>(d + at[1]);
  sc.seg_ptr = reinterpret_cast<const int32_t*>(d + at[2]);
  sc.slot_off = reinterpret_cast<const int64_t*>(d + at[3]);
  sc.pslot_ptr = reinterpret_cast<const int32_t*>(d + at[4]);
  sc.pslots = reinterpret_cast<const int32_t*>(d + at[5]);
  sc.prob_cnt = reinterpret_cast<int*>(d + at[6]);
  sc.slices = reinterpret_cast<const Slice*>(d + at[7]);
  sc.packs = reinterpret_cast<const Pack*>(d + at[8]);
  sc.psegs = reinterpret_cast<const PackSegment*>(d + at[9]);
  return SPID_OK;
}

// Tensor-core error schedule: the 128-row tiles of every (subdomain, column
// block of <= 256 columns), in that order, cut into G contiguous ranges of
// equal bytes (a tile goes to the CTA whose share holds its midpoint); a run of
// one (subdomain, block) on one CTA is a segment.  Segments come out grouped
// by subdomain, so each subdomain's partials are a contiguous range.
void build_error_tc_schedule(spid_plan_t P, int G, std::vector<ErrSeg>& segs,
                             std::vector<int32_t>& seg_ptr, std::vector<int32_t>& sub_ptr) {
  double W = 0.0;
  for (int s = 0; s < P->S; ++s) W += (double)P->m[s] * P->n[s];
  segs.clear();
  seg_ptr.assign(G + 1, 0);
  sub_ptr.assign(P->S + 1, 0);
  std::vector<std::vector<ErrSeg>> per_cta(G);
  double acc = 0.0;
  for (int s = 0; s < P->S; ++s) {
    const int tiles = (P->m[s] + kErrTcRows - 1) / kErrTcRows;
    for (int c0 = 0; c0 < P->n[s]; c0 += kErrTcCols) {
      const int nc = std::min(kErrTcCols, P->n[s] - c0);
      for (int t = 0; t < tiles; ++t) {
        const double w = (double)std::min(kErrTcRows, P->m[s] - t * kErrTcRows) * nc;
        int c = W > 0 ? (int)((acc + 0.5 * w) * G / W) : 0;
        c = std::min(std::max(c, 0), G - 1);
        std::vector<ErrSeg>& v = per_cta[c];
        if (!v.empty() && v.back().sub == s && v.back().col0 == c0 && v.back().tile1 == t)
          v.back().tile1 = t + 1;
        else
          v.push_back({s, c0, nc, t, t + 1});
        acc += w;
      }
    }
  }
  for (int c = 0; c < G; ++c) {
    seg_ptr[c] = (int32_t)segs.size();
    segs.insert(segs.end(), per_cta[c].begin(), per_cta[c].end());
  }
  seg_ptr[G] = (int32_t)segs.size();
  // subdomain ranges (CTA ranges are consecutive, so s is non-decreasing)
  int q = 0;
  for (int s = 0; s <= P->S; ++s) {
    while (q < (int)segs.size() && segs[q].sub < s) ++q;
    sub_ptr[s] = q;
  }
}

spid_status get_schedule(spid_plan_t P, int col0, int ncols, Schedule** out) {
  std::lock_guard<std::mutex> g(P->mu);
  auto key = std::make_pair(col0, ncols);
  auto it = P->schedules.find(key);
  if (it == P->schedules.end()) {
    Schedule sc;
    spid_status st = build_schedule(P, col0, ncols, sc);
    if (st != SPID_OK) return st;
    it = P->schedules.emplace(key, sc).first;
  }
  *out = &it->second;
  return SPID_OK;
}

// Unit shapes the tuner may choose for the CUDA-core error pass.
constexpr int kTuneErrRows[] = {256, 512, 1024};
constexpr int kTuneErrCols[] = {64, 128, 256};
constexpr int kTuneMaxCtasPerSm = 4;

int count_error_units(spid_plan_t P, int rows, int cols) {
  int64_t u = 0;
  for (int s = 0; s < P->S; ++s)
    u += (int64_t)((P->m[s] + rows - 1) / rows) * ((P->n[s] + cols - 1) / cols);
  return (int)std::min<int64_t>(u, INT32_MAX);
}

// Error-pass units (subdomain, row block, column block) for the plan's unit
// shape, copied into the arrays sized at plan creation (synchronous).
spid_status upload_error_units(spid_plan_t P) {
  const int rows = P->tune.err_rows, cols = P->tune.err_cols;
  std::vector<int32_t> usub, urow, ucol, uptr(P->S + 1, 0);
  for (int s = 0; s < P->S; ++s) {
    uptr[s] = (int32_t)usub.size();
    for (int r = 0; r < P->m[s]; r += rows)
      for (int c = 0; c < P->n[s]; c += cols) {
        usub.push_back(s);
        urow.push_back(r);
        ucol.push_back(c);
      }
  }
  uptr[P->S] = (int32_t)usub.size();
  if ((int64_t)usub.size() > P->units_cap)
    return fail(SPID_ERR_INVALID_ARG, "error-pass unit shape below the smallest supported one");
  SPID_CUDA(cudaMemcpy(P->d_unit_sub, usub.data(), sizeof(int32_t) * usub.size(),
                       cudaMemcpyHostToDevice));
  SPID_CUDA(cudaMemcpy(P->d_unit_row0, urow.data(), sizeof(int32_t) * urow.size(),
                       cudaMemcpyHostToDevice));
  SPID_CUDA(cudaMemcpy(P->d_unit_col0, ucol.data(), sizeof(int32_t) * ucol.size(),
                       cudaMemcpyHostToDevice));
  SPID_CUDA(cudaMemcpy(P->d_unit_ptr, uptr.data(), sizeof(int32_t) * uptr.size(),
                       cudaMemcpyHostToDevice));
  P->unit_ptr = uptr;
  P->units = (int)usub.size();
  return SPID_OK;
}

// The tensor-core error schedule, built (and its tables allocated) the first
// time a tuning selects that path.
spid_status ensure_error_tc(spid_plan_t P) {
  if (P->err_tc_grid > 0) return SPID_OK;
  if (!P->err_tc_possible())
    return fail(SPID_ERR_UNSUPPORTED, "the tensor-core error pass needs a batched TF32/BF16/3xBF16 "
                                      "plan with k_max <= 32");
  std::vector<ErrSeg> esegs;
  std::vector<int32_t> eseg_ptr, esub_ptr;
  const int G = P->num_sms;
  build_error_tc_schedule(P, G, esegs, eseg_ptr, esub_ptr);
  SPID_CUDA(P->alloc(reinterpret_cast<void**>(&P->d_err_segs), sizeof(ErrSeg) * esegs.size()));
  SPID_CUDA(P->alloc(reinterpret_cast<void**>(&P->d_err_seg_ptr), sizeof(int32_t) * eseg_ptr.size()));
  SPID_CUDA(P->alloc(reinterpret_cast<void**>(&P->d_err_tc_ptr), sizeof(int32_t) * esub_ptr.size()));
  SPID_CUDA(P->alloc(reinterpret_cast<void**>(&P->d_err_tc_part), sizeof(double) * 2 * esegs.size()));
  SPID_CUDA(cudaMemcpy(P->d_err_segs, esegs.data(), sizeof(ErrSeg) * esegs.size(),
                       cudaMemcpyHostToDevice));
  SPID_CUDA(cudaMemcpy(P->d_err_seg_ptr, eseg_ptr.data(), sizeof(int32_t) * eseg_ptr.size(),
                       cudaMemcpyHostToDevice));
  SPID_CUDA(cudaMemcpy(P->d_err_tc_ptr, esub_ptr.data(), sizeof(int32_t) * esub_ptr.size(),
                       cudaMemcpyHostToDevice));
  P->err_tc_grid = G;
  return SPID_OK;
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// One tensor map per subdomain over the window, 128-byte swizzle, zero fill
// outside the subdomain.  Blocks: 2-D, dim0 = rows (contiguous), dim1 =
// window columns, box = 32 rows x 64 columns.  Boxes of a global field: 5-D,
// (x, y, z, q, column) over the box's own extents with the field's strides,
// box = 32 points along x x 64 columns, so a 32-row chunk of the data matrix
// (ex a multiple of 32) is one tile -- the same 8 KB [64][32] shared-memory
// image either way.
spid_status encode_window_maps(spid_plan_t P, const void* window, std::vector<CUtensorMap>& maps) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return fail(SPID_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
  maps.resize(P->num_tmaps());
  for (int s = 0; s < P->S; ++s) {
    void* base = const_cast<char*>(static_cast<const char*>(window)) + P->off[s] * P->esz;
    const RowGeom& g = P->geo[s];
    CUresult r;
    if (g.ex > 0) {
      const int64_t nqs = (int64_t)P->m[s] / ((int64_t)g.ex * g.ey * g.ez);
      cuuint64_t dims[5] = {(cuuint64_t)g.ex, (cuuint64_t)g.ey, (cuuint64_t)g.ez,
                            (cuuint64_t)nqs, (cuuint64_t)P->n[s]};
      cuuint64_t strides[4] = {(cuuint64_t)g.sy * P->esz, (cuuint64_t)g.sz * P->esz,
                               (cuuint64_t)g.sq * P->esz, (cuuint64_t)P->ld[s] * P->esz};
      cuuint32_t box[5] = {32, 1, 1, 1, (cuuint32_t)P->tune.slice_cols};
      cuuint32_t estr[5] = {1, 1, 1, 1, 1};
      r = enc(&maps[s], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, base, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
      cuuint64_t dims[2] = {(cuuint64_t)P->m[s], (cuuint64_t)P->n[s]};
      cuuint64_t strides[1] = {(cuuint64_t)P->ld[s] * P->esz};
      cuuint32_t box[2] = {32, (cuuint32_t)P->tune.slice_cols};
      cuuint32_t estr[2] = {1, 1};
      r = enc(&maps[s], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (r != CUDA_SUCCESS)
      return fail(SPID_ERR_INVALID_ARG, "cuTensorMapEncodeTiled failed for subdomain " +
                                            std::to_string(s) + " (code " + std::to_string((int)r) + ")");
  }
  // shared maps: the same box over a whole field or a run of equally strided blocks
  for (size_t gi = 0; gi < P->tma_groups.size(); ++gi) {
    const spid_plan_s::TmaGroup& g = P->tma_groups[gi];
    void* base = const_cast<char*>(static_cast<const char*>(window)) + g.base * P->esz;
    cuuint64_t dims[5], strides[4];
    cuuint32_t box[5] = {32, 1, 1, 1, 1};
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    for (int i = 0; i < g.rank; ++i) dims[i] = (cuuint64_t)g.dims[i];
    for (int i = 0; i + 1 < g.rank; ++i) strides[i] = (cuuint64_t)g.strides[i] * P->esz;
    box[g.rank - 1] = (cuuint32_t)P->tune.slice_cols;
    CUresult r = enc(&maps[P->S + gi], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, g.rank, base, dims, strides,
                     box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
      return fail(SPID_ERR_INVALID_ARG, "cuTensorMapEncodeTiled failed for shared map " +
                                            std::to_string(gi) + " (code " + std::to_string((int)r) + ")");
  }
  return SPID_OK;
}

// Point the plan's own tensor maps at `window` (synchronizes the stream when
// the window changes: work in flight may still read the previous maps).
spid_status bind_window(spid_plan_t P, const void* window, cudaStream_t st) {
  if (P->bound_window == window) return SPID_OK;
  std::vector<CUtensorMap> maps;
  spid_status rc = encode_window_maps(P, window, maps);
  if (rc != SPID_OK) return rc;
  SPID_CUDA(cudaStreamSynchronize(st));
  SPID_CUDA(cudaMemcpy(P->d_tmaps, maps.data(), sizeof(CUtensorMap) * maps.size(),
                       cudaMemcpyHostToDevice));
  P->bound_window = window;
  return SPID_OK;
}

// Launch the sketch of window columns [col0, col0 + ncols) with a schedule
// already built; tmaps: device tensor maps of `window` (tensor-core plans).
spid_status launch_sketch_range(spid_plan_t P, const Schedule* sc, const void* window,
                                const void* tmaps, cudaStream_t cs) {
  SketchArgs a;
  a.probs = sc->probs;
  a.segs = sc->segs;
  a.seg_ptr = sc->seg_ptr;
  a.slot_off = sc->slot_off;
  a.partial = P->d_partial;
  a.window = window;
  a.tmaps = tmaps;
  a.cta_base = 0;
  a.l = P->l_sk;
  a.l_pad = P->l_pad;
  a.seed = P->seed;
  a.status = P->d_status;
  a.pslot_ptr = sc->pslot_ptr;
  a.pslots = sc->pslots;
  a.prob_cnt = sc->prob_cnt;
  a.Y = P->d_Y;
  a.yoff = P->d_yoff;
  a.slices = sc->slices;
  a.packs = sc->packs;
  a.psegs = sc->psegs;
  a.slice_cols = P->tune.slice_cols;
  const int nlaunch = P->per_sub() ? P->S : 1;
  for (int q = 0; q < nlaunch; ++q) {
    a.cta_base = P->per_sub() ? sc->cta_base_of_sub[q] : 0;
    cudaError_t e =
        P->bf16() ? launch_sketch_bf16(a, sc->grid, sc->stages, sc->max_tiles,
                                       P->prec == SPID_PREC_BF16X3, cs)
        : P->tensor_core() ? launch_sketch_tc(a, sc->grid, sc->stages, sc->max_tiles, cs)
        : sc->packed       ? launch_sketch_simt_packed(a, sc->grid, P->fp64(), sc->simt_tj, cs)
                           : launch_sketch_simt(a, sc->grid, P->fp64(), sc->simt_tj, cs);
    if (e != cudaSuccess) return fail(SPID_ERR_CUDA, std::string("sketch launch: ") + cudaGetErrorString(e));
  }
  return SPID_OK;
}

// Free every cached sketch schedule (their tables encode the tuning).
// The caller has synchronized the device.
void drop_schedules(spid_plan_t P) {
  for (auto& kv : P->schedules) {
    void* d = kv.second.dev;
    cudaFree(d);
    P->allocs.erase(std::remove(P->allocs.begin(), P->allocs.end(), d), P->allocs.end());
  }
  P->schedules.clear();
}

// Zero every completion counter (schedules and error pass).  Needed only after
// a kernel gave up on a timeout and left a counter part-way.
cudaError_t reset_counters(spid_plan_t P, cudaStream_t st) {
  for (auto& kv : P->schedules) {
    cudaError_t e = cudaMemsetAsync(kv.second.prob_cnt, 0,
                                    sizeof(int) * std::max(kv.second.nprob, 1), st);
    if (e != cudaSuccess) return e;
  }
  return cudaMemsetAsync(P->d_err_cnt, 0, sizeof(int) * (P->S + 1), st);
}

spid_status check_plan(spid_plan_t P) {
  if (!P) return fail(SPID_ERR_INVALID_ARG, "plan is NULL");
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != P->device) {
    SPID_CUDA(cudaSetDevice(P->device));
  }
  return SPID_OK;
}

}  // namespace

spid::PlanView spid::plan_view(spid_plan_t P) {
  PlanView v;
  v.S = P->S;
  v.k_max = P->k_max;
  v.esz = P->esz;
  v.m = P->d_m;
  v.n = P->d_n;
  v.k = P->d_k;
  v.J = P->d_J;
  v.C = P->d_C;
  v.coff = P->d_coff;
  v.status = P->d_status;
  v.Y = P->d_Y;
  v.yoff = P->d_yoff;
  v.l = P->l;
  v.l_pad = P->l_pad;
  return v;
}

extern "C" {

const char* spid_status_string(spid_status s) {
  switch (s) {
    case SPID_OK: return "SPID_OK";
    case SPID_ERR_INVALID_ARG: return "SPID_ERR_INVALID_ARG";
    case SPID_ERR_CUDA: return "SPID_ERR_CUDA";
    case SPID_ERR_OOM: return "SPID_ERR_OOM";
    case SPID_ERR_STATE: return "SPID_ERR_STATE";
    case SPID_ERR_TIMEOUT: return "SPID_ERR_TIMEOUT";
    case SPID_ERR_NONFINITE: return "SPID_ERR_NONFINITE";
    case SPID_ERR_UNSUPPORTED: return "SPID_ERR_UNSUPPORTED";
    case SPID_ERR_RANK: return "SPID_ERR_RANK";
  }
  return "SPID_ERR_UNKNOWN";
}

const char* spid_last_error(void) { return g_last_error.c_str(); }

double spid_compression_factor(int32_t num_sub, const int32_t* m, const int32_t* n,
                               const int32_t* k) {
  double num = 0.0, den = 0.0;
  for (int32_t s = 0; s < num_sub; ++s) {
    num += (double)m[s] * (double)n[s];
    den += (double)k[s] * ((double)m[s] + (double)n[s]);
  }
  return den > 0.0 ? num / den : INFINITY;
}

// Subdomains of a plan descriptor: rows, element offset of row 0 at column
// 0, column stride and row placement, from the blocks arrays or from the boxes
// of a global field.  Validates everything; on success fills the vectors.
static spid_status parse_layout(const spid_plan_desc* d, size_t esz, std::vector<int32_t>& m,
                                std::vector<int64_t>& off, std::vector<int64_t>& ld,
                                std::vector<RowGeom>& geo, std::vector<int32_t>& qoi,
                                int& num_qoi) {
  const int S = d->num_sub;
  const int64_t align = (int64_t)(16 / esz);
  m.assign(S, 0);
  off.assign(S, 0);
  ld.assign(S, 0);
  geo.assign(S, RowGeom{0, 0, 0, 0, 0, 0, 0});
  const spid_box_layout* L = d->boxes;
  if (!L) {
    if (!d->m || !d->off || !d->ld) return fail(SPID_ERR_INVALID_ARG, "a descriptor array is NULL");
    for (int s = 0; s < S; ++s) {
      if (d->m[s] < 1 || d->ld[s] < d->m[s] || d->off[s] < 0)
        return fail(SPID_ERR_INVALID_ARG, "bad size for subdomain " + std::to_string(s));
      if (d->off[s] % align || d->ld[s] % align)
        return fail(SPID_ERR_INVALID_ARG, "off/ld of subdomain " + std::to_string(s) +
                                              " not a multiple of 16 bytes");
      m[s] = d->m[s];
      off[s] = d->off[s];
      ld[s] = d->ld[s];
    }
  } else {
    if (L->nq < 1 || L->X < 1 || L->Y < 1 || L->Z < 1 || L->num_box < 1 || !L->org3 || !L->ext3 ||
        (L->split_qoi != 0 && L->split_qoi != 1))
      return fail(SPID_ERR_INVALID_ARG, "bad box layout (nq, X, Y, Z, num_box, org3, ext3, split_qoi)");
    const int64_t plane = L->X * L->Y, field = plane * L->Z;
    if (L->X % align || L->snap_stride % align || L->snap_stride < (int64_t)L->nq * field)
      return fail(SPID_ERR_INVALID_ARG, "box layout: X and snap_stride must be multiples of 16 bytes "
                                        "and snap_stride >= nq X Y Z");
    const int per_box = L->split_qoi ? L->nq : 1;
    if ((int64_t)L->num_box * per_box != S)
      return fail(SPID_ERR_INVALID_ARG, "num_sub must be num_box (or num_box nq with split_qoi)");
    for (int b = 0; b < L->num_box; ++b) {
      const int32_t* o = L->org3 + 3 * b;
      const int32_t* e = L->ext3 + 3 * b;
      if (o[0] < 0 || o[1] < 0 || o[2] < 0 || e[0] < 1 || e[1] < 1 || e[2] < 1 ||
          o[0] + (int64_t)e[0] > L->X || o[1] + (int64_t)e[1] > L->Y || o[2] + (int64_t)e[2] > L->Z)
        return fail(SPID_ERR_INVALID_ARG, "box " + std::to_string(b) + " is empty or leaves the field");
      if (o[0] % align || e[0] % align)
        return fail(SPID_ERR_INVALID_ARG, "box " + std::to_string(b) +
                                              ": x origin and x extent must be multiples of 16 bytes");
      const int64_t pts = (int64_t)e[0] * e[1] * e[2];
      const int64_t rows = pts * (L->split_qoi ? 1 : L->nq);
      if (rows > INT32_MAX) return fail(SPID_ERR_INVALID_ARG, "box " + std::to_string(b) + " has too many rows");
      for (int q = 0; q < per_box; ++q) {
        const int s = b * per_box + q;
        m[s] = (int32_t)rows;
        off[s] = (int64_t)q * field + (int64_t)o[2] * plane + (int64_t)o[1] * L->X + o[0];
        ld[s] = L->snap_stride;
        geo[s] = RowGeom{e[0], e[1], e[2], 0, L->X, plane, field};
      }
    }
  }
  // per-QoI labels
  qoi.clear();
  num_qoi = 0;
  if (d->qoi) {
    if (d->num_qoi < 1 || d->num_qoi > 64)
      return fail(SPID_ERR_INVALID_ARG, "num_qoi must be 1..64 when qoi is given");
    for (int s = 0; s < S; ++s)
      if (d->qoi[s] < 0 || d->qoi[s] >= d->num_qoi)
        return fail(SPID_ERR_INVALID_ARG, "qoi of subdomain " + std::to_string(s) + " out of range");
    qoi.assign(d->qoi, d->qoi + S);
    num_qoi = d->num_qoi;
  } else if (L && L->split_qoi) {
    if (d->num_qoi != 0 && d->num_qoi != L->nq)
      return fail(SPID_ERR_INVALID_ARG, "num_qoi must be 0 or nq for split boxes without qoi");
    if (L->nq > 64) return fail(SPID_ERR_INVALID_ARG, "at most 64 QoIs for per-QoI totals");
    qoi.resize(S);
    for (int s = 0; s < S; ++s) qoi[s] = s % L->nq;
    num_qoi = L->nq;
  } else if (d->num_qoi != 0) {
    return fail(SPID_ERR_INVALID_ARG, "num_qoi > 0 needs the qoi array");
  }
  return SPID_OK;
}

// Shared tensor maps of a tensor-core plan.  Boxes of a global field: one
// 5-D map over the whole field [t][q][Z][Y][X]; a box is placed by its origin
// (and its QoI when QoIs are split).  Blocks: the subdomains with equal ld,
// equal m and equal offset modulo ld form a 2-D map of m rows whose columns are
// the window's runs of ld elements from that residue; subdomain s starts at
// column off / ld.  Subdomains of whole 32-row chunks that fit inside one run
// share a map of whole runs of every residue instead.  A group of one keeps
// only its own map.
static void build_tma_groups(spid_plan_s* P, const spid_box_layout* L) {
  P->tma_groups.clear();
  P->tma_group.assign(P->S, -1);
  P->tma_org.assign(4 * (size_t)P->S, 0);
  if (!P->tensor_core() || P->S < 2) return;
  if (L) {
    spid_plan_s::TmaGroup g{};
    g.base = 0;
    g.rank = 5;
    const int64_t plane = (int64_t)L->X * L->Y;
    const int64_t d[5] = {L->X, L->Y, L->Z, L->nq, P->n_max};
    const int64_t st[4] = {L->X, plane, plane * L->Z, L->snap_stride};
    std::copy(d, d + 5, g.dims);
    std::copy(st, st + 4, g.strides);
    P->tma_groups.push_back(g);
    const int per_box = L->split_qoi ? L->nq : 1;
    for (int s = 0; s < P->S; ++s) {
      const int32_t* o = L->org3 + 3 * (s / per_box);
      P->tma_group[s] = 0;
      P->tma_org[4 * s + 0] = o[0];
      P->tma_org[4 * s + 1] = o[1];
      P->tma_org[4 * s + 2] = o[2];
      P->tma_org[4 * s + 3] = L->split_qoi ? s % per_box : 0;
    }
    return;
  }
  // key (ld, r, m): a map of m rows from residue r; key (ld, -1, 0): a map of
  // whole ld-runs that places each subdomain at x = r, for subdomains whose
  // rows are whole 32-row chunks inside one run (no chunk reads past them)
  std::map<std::tuple<int64_t, int64_t, int32_t>, std::vector<int>> runs;
  for (int s = 0; s < P->S; ++s) {
    const int64_t c0 = P->off[s] / P->ld[s], r = P->off[s] % P->ld[s];
    if (c0 + P->n[s] > INT32_MAX) continue;   // the column coordinate is 32-bit
    const bool whole = P->m[s] % kChunkRows == 0 && r + P->m[s] <= P->ld[s] && P->ld[s] <= INT32_MAX;
    runs[whole ? std::make_tuple(P->ld[s], (int64_t)-1, 0) : std::make_tuple(P->ld[s], r, P->m[s])]
        .push_back(s);
  }
  for (const auto& kv : runs) {
    if (kv.second.size() < 2) continue;
    const bool whole = std::get<1>(kv.first) < 0;
    spid_plan_s::TmaGroup g{};
    g.base = whole ? 0 : std::get<1>(kv.first);
    g.rank = 2;
    g.dims[0] = whole ? std::get<0>(kv.first) : std::get<2>(kv.first);
    g.dims[1] = 0;
    g.strides[0] = std::get<0>(kv.first);
    const int gi = (int)P->tma_groups.size();
    for (int s : kv.second) {
      const int64_t c0 = P->off[s] / P->ld[s];
      g.dims[1] = std::max<int64_t>(g.dims[1], c0 + P->n[s]);
      P->tma_group[s] = gi;
      P->tma_org[4 * s + 0] = whole ? (int32_t)(P->off[s] % P->ld[s]) : 0;
      P->tma_org[4 * s + 1] = (int32_t)c0;
    }
    P->tma_groups.push_back(g);
  }
}

static spid_status plan_create(const spid_plan_desc* d, spid_stream_t stream, int l_sketch,
                               spid_plan_t* out);

spid_status spid_plan_create(const spid_plan_desc* d, spid_stream_t stream, spid_plan_t* out) {
  return plan_create(d, stream, 0, out);
}

}  // extern "C"

spid_status spid::plan_create_sketch_rows(const spid_plan_desc* d, spid_stream_t stream,
                                          int l_sketch, spid_plan_t* out) {
  return plan_create(d, stream, l_sketch, out);
}

extern "C" {

static spid_status plan_create(const spid_plan_desc* d, spid_stream_t stream, int l_sketch,
                               spid_plan_t* out) {
  g_last_error.clear();
  if (!d || !out) return fail(SPID_ERR_INVALID_ARG, "desc/out is NULL");
  *out = nullptr;
  if (d->num_sub < 1 || !d->n) return fail(SPID_ERR_INVALID_ARG, "num_sub < 1 or n is NULL");
  if (d->precision < SPID_PREC_FP64 || d->precision > SPID_PREC_BF16X3)
    return fail(SPID_ERR_INVALID_ARG, "unknown precision");
  if (d->k_max < 1 || d->p < 0 || d->k_max + d->p > 64)
    return fail(SPID_ERR_INVALID_ARG, "need k_max >= 1, p >= 0, k_max + p <= 64");
  if (!(d->tol >= 0.0) || !std::isfinite(d->tol)) return fail(SPID_ERR_INVALID_ARG, "tol must be >= 0");
  const size_t esz = d->precision == SPID_PREC_FP64 ? 8 : 4;
  std::vector<int32_t> lm, lqoi;
  std::vector<int64_t> loff, lld;
  std::vector<RowGeom> lgeo;
  int lnq = 0;
  {
    spid_status st = parse_layout(d, esz, lm, loff, lld, lgeo, lqoi, lnq);
    if (st != SPID_OK) return st;
  }
  int n_max = 0;
  for (int s = 0; s < d->num_sub; ++s) {
    if (d->n[s] < 1 || d->n[s] > (1 << 20))
      return fail(SPID_ERR_INVALID_ARG, "bad window length for subdomain " + std::to_string(s));
    n_max = std::max(n_max, d->n[s]);
  }
  if (d->boxes && d->precision >= SPID_PREC_TF32)
    for (int s = 0; s < d->num_sub; ++s)
      if (lgeo[s].ex % 32)
        return fail(SPID_ERR_UNSUPPORTED, "the tensor-core sketches read boxes whose x extent is a "
                                          "multiple of 32 points (subdomain " + std::to_string(s) + ")");
  spid_plan_s* P = new spid_plan_s();
  auto bail = [&](spid_status st) {
    spid_plan_destroy(P);
    return st;
  };
  P->S = d->num_sub;
  P->m = lm;
  P->n.assign(d->n, d->n + P->S);
  P->off = loff;
  P->ld = lld;
  P->geo = lgeo;
  P->boxes = d->boxes != nullptr;
  P->qoi = lqoi;
  P->num_qoi = lnq;
  for (int s = 0; s < P->S; ++s)
    P->window_extent = std::max<int64_t>(P->window_extent, P->off[s] + P->ld[s] * (P->n[s] - 1) +
                                                               row_offset(P->geo[s], P->m[s] - 1) + 1);
  P->n_max = n_max;
  P->k_max = d->k_max;
  P->p = d->p;
  P->l = d->k_max + d->p;
  P->l_sk = std::max(P->l, l_sketch);
  if (P->l_sk > 64) {
    delete P;
    return fail(SPID_ERR_INVALID_ARG, "at most 64 sketch rows");
  }
  P->l_pad = (P->l_sk + 15) / 16 * 16;
  P->tol = d->tol;
  P->prec = d->precision;
  P->flags = d->flags;
  P->seed = d->seed;
  P->esz = esz;
  build_tma_groups(P, d->boxes);
  if (qrcp_cols_per_thread(n_max, P->l_pad, P->fp64()) == 0) {
    delete P;
    return fail(SPID_ERR_UNSUPPORTED, "window length / oversampled rank beyond the QR kernel's range");
  }
  cudaError_t e = cudaGetDevice(&P->device);
  if (e != cudaSuccess) { delete P; return fail(SPID_ERR_CUDA, cudaGetErrorString(e)); }
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, P->device);
  if (e != cudaSuccess) { delete P; return fail(SPID_ERR_CUDA, cudaGetErrorString(e)); }
  P->num_sms = prop.multiProcessorCount;
  P->smem_optin = prop.sharedMemPerBlockOptin;
  if (P->tensor_core() && prop.major < 10) {
    delete P;
    return fail(SPID_ERR_UNSUPPORTED, "the tensor-core sketch needs sm_100 or newer");
  }

  // offsets of Y and C
  std::vector<int64_t> yoff(P->S), coff(P->S);
  int64_t ysum = 0, csum = 0;
  for (int s = 0; s < P->S; ++s) {
    yoff[s] = ysum;
    coff[s] = csum;
    ysum += (int64_t)P->n[s] * P->l_pad;
    csum += (int64_t)P->n[s] * P->k_max;
  }
  P->y_elems = ysum;
  P->c_elems = csum;
  // error units: the arrays hold the unit list of the smallest unit shape the
  // tuner may pick (kTuneErrRows[0] x kTuneErrCols[0])
  P->units_cap = count_error_units(P, kTuneErrRows[0], kTuneErrCols[0]);
  // partial workspace bound: (CTAs + problems) slots of one column group each,
  // for the widest column group and the largest grid any tuning may use
  // (narrower groups divide the widest, so they need no more)
  const int CG = P->group_cols_max();
  int64_t nprob_full = 0;
  for (int s = 0; s < P->S; ++s) nprob_full += (P->n[s] + CG - 1) / CG;
  const int64_t ctas =
      P->per_sub() ? (int64_t)std::max(P->sketch_grid(), kPerSubMaxCtasPerSm * P->num_sms) * P->S
                   : (int64_t)std::max(P->sketch_grid(), kTuneMaxCtasPerSm * P->num_sms);
  P->partial_cap = (ctas + nprob_full) * (int64_t)CG * P->l_pad;
  if (P->flags & SPID_FLAG_TC_ERROR) P->tune.err_path = P->err_tc_possible() ? 1 : 0;
  // the CUDA-core sketch keeps a register tile of 64 columns per pack slice:
  // 2 slices leave room for 3 CTAs per SM (8 allow 1)
  if (!P->tensor_core()) P->tune.pack_slices = kSimtPackSlices;

#define SPID_ALLOC(ptr, bytes)                                                            \
  do {                                                                                    \
    cudaError_t e_ = P->alloc(reinterpret_cast<void**>(&(ptr)), (bytes));                 \
    if (e_ != cudaSuccess) {                                                              \
      g_last_error = std::string("cudaMalloc: ") + cudaGetErrorString(e_);                \
      return bail(e_ == cudaErrorMemoryAllocation ? SPID_ERR_OOM : SPID_ERR_CUDA);        \
    }                                                                                     \
  } while (0)
  SPID_ALLOC(P->d_m, sizeof(int32_t) * P->S);
  SPID_ALLOC(P->d_n, sizeof(int32_t) * P->S);
  SPID_ALLOC(P->d_off, sizeof(int64_t) * P->S);
  SPID_ALLOC(P->d_ld, sizeof(int64_t) * P->S);
  SPID_ALLOC(P->d_yoff, sizeof(int64_t) * P->S);
  SPID_ALLOC(P->d_coff, sizeof(int64_t) * P->S);
  SPID_ALLOC(P->d_Y, esz * P->y_elems);
  SPID_ALLOC(P->d_C, esz * P->c_elems);
  SPID_ALLOC(P->d_J, sizeof(int32_t) * P->S * P->k_max);
  SPID_ALLOC(P->d_k, sizeof(int32_t) * P->S);
  SPID_ALLOC(P->d_status, sizeof(int));
  SPID_ALLOC(P->d_unit_sub, sizeof(int32_t) * P->units_cap);
  SPID_ALLOC(P->d_unit_row0, sizeof(int32_t) * P->units_cap);
  SPID_ALLOC(P->d_unit_col0, sizeof(int32_t) * P->units_cap);
  SPID_ALLOC(P->d_unit_ptr, sizeof(int32_t) * (P->S + 1));
  SPID_ALLOC(P->d_err_part, sizeof(double) * 2 * P->units_cap);
  SPID_ALLOC(P->d_sub_err, sizeof(double) * 2 * P->S);
  SPID_ALLOC(P->d_err_cnt, sizeof(int) * (P->S + 1));
  SPID_ALLOC(P->d_partial, esz * P->partial_cap);
  if (P->tensor_core()) SPID_ALLOC(P->d_tmaps, sizeof(CUtensorMap) * P->num_tmaps());
  if (P->boxes) SPID_ALLOC(P->d_geo, sizeof(RowGeom) * P->S);
  if (P->num_qoi > 0) SPID_ALLOC(P->d_qoi, sizeof(int32_t) * P->S);
#undef SPID_ALLOC
#define SPID_H2D(dst, src, bytes)                                                          \
  do {                                                                                     \
    cudaError_t e_ = cudaMemcpy((dst), (src), (bytes), cudaMemcpyHostToDevice);            \
    if (e_ != cudaSuccess) {                                                               \
      g_last_error = std::string("cudaMemcpy: ") + cudaGetErrorString(e_);                 \
      return bail(SPID_ERR_CUDA);                                                          \
    }                                                                                      \
  } while (0)
  SPID_H2D(P->d_m, P->m.data(), sizeof(int32_t) * P->S);
  SPID_H2D(P->d_n, P->n.data(), sizeof(int32_t) * P->S);
  SPID_H2D(P->d_off, P->off.data(), sizeof(int64_t) * P->S);
  SPID_H2D(P->d_ld, P->ld.data(), sizeof(int64_t) * P->S);
  SPID_H2D(P->d_yoff, yoff.data(), sizeof(int64_t) * P->S);
  SPID_H2D(P->d_coff, coff.data(), sizeof(int64_t) * P->S);
  if (P->boxes) SPID_H2D(P->d_geo, P->geo.data(), sizeof(RowGeom) * P->S);
  if (P->num_qoi > 0) SPID_H2D(P->d_qoi, P->qoi.data(), sizeof(int32_t) * P->S);
#undef SPID_H2D
  {
    spid_status st = upload_error_units(P);
    if (st == SPID_OK && P->tune.err_path == 1) st = ensure_error_tc(P);
    if (st != SPID_OK) return bail(st);
  }
  {
    cudaStream_t cs = (cudaStream_t)stream;
    if (cudaMemsetAsync(P->d_Y, 0, esz * P->y_elems, cs) != cudaSuccess ||
        cudaMemsetAsync(P->d_status, 0, sizeof(int), cs) != cudaSuccess ||
        cudaMemsetAsync(P->d_err_cnt, 0, sizeof(int) * (P->S + 1), cs) != cudaSuccess ||
        cudaMemsetAsync(P->d_k, 0, sizeof(int32_t) * P->S, cs) != cudaSuccess)
      return bail(fail(SPID_ERR_CUDA, "cudaMemsetAsync failed"));
    // the whole-window schedule is built now so that steady-state calls allocate nothing
    Schedule* sc = nullptr;
    spid_status st = get_schedule(P, 0, n_max, &sc);
    if (st != SPID_OK) return bail(st);
    if (cudaStreamSynchronize(cs) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
      return bail(fail(SPID_ERR_CUDA, "sync failed"));
  }
  *out = P;
  return SPID_OK;
}

spid_status spid_plan_destroy(spid_plan_t P) {
  if (!P) return SPID_OK;
  if (P->live_graphs > 0)
    return fail(SPID_ERR_STATE, "destroy the plan's graphs (spid_graph_destroy) first");
  cudaSetDevice(P->device);
  cudaDeviceSynchronize();
  for (void* p : P->allocs) cudaFree(p);
  delete P;
  return SPID_OK;
}

spid_status spid_plan_info(spid_plan_t P, int32_t* l, int32_t* l_pad, int64_t* ws) {
  if (!P) return fail(SPID_ERR_INVALID_ARG, "plan is NULL");
  if (l) *l = P->l;
  if (l_pad) *l_pad = P->l_pad;
  if (ws) *ws = P->workspace;
  return SPID_OK;
}

spid_status spid_reset(spid_plan_t P, spid_stream_t stream) {
  spid_status st = check_plan(P);
  if (st != SPID_OK) return st;
  SPID_CUDA(cudaMemsetAsync(P->d_Y, 0, P->esz * P->y_elems, (cudaStream_t)stream));
  SPID_CUDA(reset_counters(P, (cudaStream_t)stream));
  return SPID_OK;
}

spid_status spid_sketch_accumulate(spid_plan_t P, const void* window, int32_t col0,
                                   int32_t ncols, spid_stream_t stream) {
  spid_status st = check_plan(P);
  if (st != SPID_OK) return st;
  if (!window) return fail(SPID_ERR_INVALID_ARG, "window is NULL");
  if (reinterpret_cast<uintptr_t>(window) % 16)
    return fail(SPID_ERR_INVALID_ARG, "window must be 16-byte aligned");
  if (col0 < 0 || ncols < 0) return fail(SPID_ERR_INVALID_ARG, "negative column range");
  if (ncols == 0 || col0 >= P->n_max) return SPID_OK;
  ncols = std::min(ncols, P->n_max - col0);
  cudaStream_t cs = (cudaStream_t)stream;
  Schedule* sc = nullptr;
  st = get_schedule(P, col0, ncols, &sc);
  if (st != SPID_OK) return st;
  if (P->tensor_core()) {
    st = bind_window(P, window, cs);
    if (st != SPID_OK) return st;
  }
  return launch_sketch_range(P, sc, window, P->d_tmaps, cs);
}

static spid_status run_finalize(spid_plan_t P, cudaStream_t cs) {
  QrcpArgs a;
  a.Y = P->d_Y;
  a.yoff = P->d_yoff;
  a.n = P->d_n;
  a.C = P->d_C;
  a.coff = P->d_coff;
  a.J = P->d_J;
  a.k_out = P->d_k;
  a.l = P->l;
  a.k_max = P->k_max;
  a.tol = P->tol;
  a.u_mode = P->u_mode();
  a.sub_base = 0;
  a.status = P->d_status;
  if (P->per_sub()) {
    for (int s = 0; s < P->S; ++s) {
      a.sub_base = s;
      cudaError_t e = launch_qrcp(a, 1, P->n[s], P->l_pad, P->fp64(), cs);
      if (e != cudaSuccess) return fail(SPID_ERR_CUDA, std::string("qrcp launch: ") + cudaGetErrorString(e));
    }
  } else {
    cudaError_t e = launch_qrcp(a, P->S, P->n_max, P->l_pad, P->fp64(), cs);
    if (e != cudaSuccess) return fail(SPID_ERR_CUDA, std::string("qrcp launch: ") + cudaGetErrorString(e));
  }
  return SPID_OK;
}

spid_status spid_finalize(spid_plan_t P, spid_stream_t stream) {
  spid_status st = check_plan(P);
  if (st != SPID_OK) return st;
  return run_finalize(P, (cudaStream_t)stream);
}

static spid_status run_error(spid_plan_t P, const void* window, void* out, double* err_dev,
                             double* total_dev, cudaStream_t cs) {
  if (!window) return fail(SPID_ERR_INVALID_ARG, "window is NULL");
  if (reinterpret_cast<uintptr_t>(window) % 16 || (out && reinterpret_cast<uintptr_t>(out) % 16))
    return fail(SPID_ERR_INVALID_ARG, "window/out must be 16-byte aligned");
  ErrArgs a;
  a.window = window;
  a.out = out;
  a.m = P->d_m;
  a.n = P->d_n;
  a.off = P->d_off;
  a.ld = P->d_ld;
  a.C = P->d_C;
  a.coff = P->d_coff;
  a.J = P->d_J;
  a.k = P->d_k;
  a.k_max = P->k_max;
  a.unit_sub = P->d_unit_sub;
  a.unit_row0 = P->d_unit_row0;
  a.unit_col0 = P->d_unit_col0;
  a.part = P->d_err_part;
  a.unit_base = 0;
  a.unit_ptr = P->d_unit_ptr;
  a.sub_cnt = P->d_err_cnt;
  a.all_cnt = P->d_err_cnt + P->S;
  a.err = err_dev;
  a.sub_err = P->d_sub_err;
  a.total = total_dev;
  a.S = P->S;
  a.row_block = P->tune.err_rows;
  a.col_block = P->tune.err_cols;
  a.geo = P->boxes ? P->d_geo : nullptr;
  a.qoi = P->d_qoi;
  a.num_qoi = P->num_qoi;
  if (P->tune.err_path == 1 && P->err_tc_grid > 0) {
    ErrTcArgs t;
    t.e = a;
    t.e.part = P->d_err_tc_part;
    t.e.unit_ptr = P->d_err_tc_ptr;
    t.segs = P->d_err_segs;
    t.seg_ptr = P->d_err_seg_ptr;
    t.status = P->d_status;
    cudaError_t e = launch_error_tc(t, P->err_tc_grid, cs);
    if (e != cudaSuccess) return fail(SPID_ERR_CUDA, std::string("error launch: ") + cudaGetErrorString(e));
    return SPID_OK;
  }
  if (P->per_sub()) {
    for (int s = 0; s < P->S; ++s) {
      a.unit_base = P->unit_ptr[s];
      cudaError_t e = launch_error(a, P->unit_ptr[s + 1] - P->unit_ptr[s], P->fp64(), cs);
      if (e != cudaSuccess) return fail(SPID_ERR_CUDA, std::string("error launch: ") + cudaGetErrorString(e));
    }
  } else {
    cudaError_t e = launch_error(a, P->units, P->fp64(), cs);
    if (e != cudaSuccess) return fail(SPID_ERR_CUDA, std::string("error launch: ") + cudaGetErrorString(e));
  }
  return SPID_OK;
}

spid_status spid_error(spid_plan_t P, const void* window, double* err_dev, double* total_dev,
                       spid_stream_t stream) {
  spid_status st = check_plan(P);
  if (st != SPID_OK) return st;
  return run_error(P, window, nullptr, err_dev, total_dev, (cudaStream_t)stream);
}

spid_status spid_reconstruct(spid_plan_t P, const void* window, void* out, spid_stream_t stream) {
  spid_status st = check_plan(P);
  if (st != SPID_OK) return st;
  if (!out) return fail(SPID_ERR_INVALID_ARG, "out is NULL");
  return run_error(P, window, out, nullptr, nullptr, (cudaStream_t)stream);
}

spid_status spid_get_factors(spid_plan_t P, int32_t* k_host, int32_t* J_host, void* C_host,
                             spid_stream_t stream) {
  spid_status st = check_plan(P);
  if (st != SPID_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  SPID_CUDA(cudaStreamSynchronize(cs));
  if (k_host) SPID_CUDA(cudaMemcpy(k_host, P->d_k, sizeof(int32_t) * P->S, cudaMemcpyDeviceToHost));
  if (J_host)
    SPID_CUDA(cudaMemcpy(J_host, P->d_J, sizeof(int32_t) * P->S * P->k_max, cudaMemcpyDeviceToHost));
  if (C_host) SPID_CUDA(cudaMemcpy(C_host, P->d_C, P->esz * P->c_elems, cudaMemcpyDeviceToHost));
  return SPID_OK;
}

spid_status spid_get_sketch(spid_plan_t P, void* Y_host, spid_stream_t stream) {
  spid_status st = check_plan(P);
  if (st != SPID_OK) return st;
  if (!Y_host) return fail(SPID_ERR_INVALID_ARG, "Y_host is NULL");
  SPID_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  SPID_CUDA(cudaMemcpy(Y_host, P->d_Y, P->esz * P->y_elems, cudaMemcpyDeviceToHost));
  return SPID_OK;
}

spid_status spid_device_status(spid_plan_t P, spid_stream_t stream) {
  spid_status st = check_plan(P);
  if (st != SPID_OK) return st;
  SPID_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  int v = 0;
  SPID_CUDA(cudaMemcpy(&v, P->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  SPID_CUDA(cudaMemset(P->d_status, 0, sizeof(int)));
  if (v & kStatusTimeout) {
    SPID_CUDA(reset_counters(P, (cudaStream_t)stream));
    SPID_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return fail(SPID_ERR_TIMEOUT, "a bounded device wait timed out");
  }
  if (v & kStatusNonfinite) return fail(SPID_ERR_NONFINITE, "non-finite values reached a sketch");
  if (v & kStatusRankCut)
    return fail(SPID_ERR_RANK, "the rank guard stopped a factorization before its target");
  return SPID_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Omega and Philox exposed for checking
// ---------------------------------------------------------------------------
namespace {

template <typename T>
__global__ void omega_kernel(uint64_t seed, int64_t r0, int32_t nrows, int32_t l, T* out) {
  const uint2 key = philox_key(seed);
  const int groups = (l + 3) / 4;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)nrows * groups;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / groups;
    const int g = (int)(t % groups);
    T w[4];
    omega_group<T>(key, (uint32_t)(r0 + c), (uint32_t)g, w);
    for (int u = 0; u < 4; ++u)
      if (4 * g + u < l) out[c * l + 4 * g + u] = w[u];
  }
}

__global__ void philox_kernel(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out,
                              int64_t count) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x) {
    const uint4 c = make_uint4(ctr[4 * t], ctr[4 * t + 1], ctr[4 * t + 2], ctr[4 * t + 3]);
    const uint4 x = philox4x32_10(c, make_uint2(k0, k1));
    out[4 * t] = x.x;
    out[4 * t + 1] = x.y;
    out[4 * t + 2] = x.z;
    out[4 * t + 3] = x.w;
  }
}

}  // namespace

extern "C" spid_status spid_omega(uint64_t seed, int64_t r0, int32_t nrows, int32_t l,
                                  int32_t precision, void* out_dev, spid_stream_t stream) {
  if (!out_dev || nrows < 0 || l < 1 || r0 < 0 || r0 + nrows > ((int64_t)1 << 32))
    return fail(SPID_ERR_INVALID_ARG, "bad omega arguments");
  if (nrows == 0) return SPID_OK;
  const int64_t work = (int64_t)nrows * ((l + 3) / 4);
  const int grid = (int)std::min<int64_t>((work + 255) / 256, 4096);
  if (precision == SPID_PREC_FP64)
    omega_kernel<double><<<grid, 256, 0, (cudaStream_t)stream>>>(seed, r0, nrows, l, (double*)out_dev);
  else
    omega_kernel<float><<<grid, 256, 0, (cudaStream_t)stream>>>(seed, r0, nrows, l, (float*)out_dev);
  SPID_CUDA(cudaGetLastError());
  return SPID_OK;
}

extern "C" spid_status spid_philox(const uint32_t* ctr_dev, uint32_t key0, uint32_t key1,
                                   uint32_t* out_dev, int64_t count, spid_stream_t stream) {
  if (!ctr_dev || !out_dev || count < 0) return fail(SPID_ERR_INVALID_ARG, "bad philox arguments");
  if (count == 0) return SPID_OK;
  const int grid = (int)std::min<int64_t>((count + 255) / 256, 4096);
  philox_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(ctr_dev, key0, key1, out_dev, count);
  SPID_CUDA(cudaGetLastError());
  return SPID_OK;
}

// ---------------------------------------------------------------------------
// Tuning: candidate tile shapes and schedules, measured on the caller's window
// ---------------------------------------------------------------------------
namespace {

bool valid_tuning(const spid_tuning& t) {
  auto in = [](int v, std::initializer_list<int> set) {
    return std::find(set.begin(), set.end(), v) != set.end();
  };
  return in(t.sketch_pack_slices, {1, 2, 4, 8}) && (t.sketch_stages == 0 ||
         (t.sketch_stages >= 2 && t.sketch_stages <= 8)) &&
         in(t.sketch_ctas_per_sm, {0, 1, 2, 3, 4}) && in(t.error_path, {0, 1}) &&
         in(t.error_rows, {256, 512, 1024}) && in(t.error_cols, {64, 128, 256}) &&
         in(t.sketch_slice_major, {0, 1}) && in(t.sketch_slice_cols, {0, 16, 32, 64});
}

TuneCfg cfg_of(const spid_tuning& t) {
  TuneCfg c;
  c.pack_slices = t.sketch_pack_slices;
  c.slice_major = t.sketch_slice_major;
  c.slice_cols = t.sketch_slice_cols ? t.sketch_slice_cols : kSliceCols;
  c.stages = t.sketch_stages;
  c.ctas_per_sm = t.sketch_ctas_per_sm;
  c.err_path = t.error_path;
  c.err_rows = t.error_rows;
  c.err_cols = t.error_cols;
  return c;
}

spid_tuning tuning_of(const TuneCfg& c, float sk, float er) {
  spid_tuning t;
  t.sketch_pack_slices = c.pack_slices;
  t.sketch_slice_major = c.slice_major;
  t.sketch_slice_cols = c.slice_cols;
  t.sketch_stages = c.stages;
  t.sketch_ctas_per_sm = c.ctas_per_sm;
  t.error_path = c.err_path;
  t.error_rows = c.err_rows;
  t.error_cols = c.err_cols;
  t.sketch_ms = sk;
  t.error_ms = er;
  return t;
}

// Install a sketch configuration: drop the cached schedules and rebuild the
// whole-window one.  The device is idle.
spid_status apply_sketch_cfg(spid_plan_t P, const TuneCfg& c) {
  P->tune.pack_slices = c.pack_slices;
  P->tune.slice_major = c.slice_major;
  if (P->tune.slice_cols != c.slice_cols) P->bound_window = nullptr;   // maps carry the box width
  P->tune.slice_cols = c.slice_cols;
  P->tune.stages = c.stages;
  P->tune.ctas_per_sm = c.ctas_per_sm;
  drop_schedules(P);
  Schedule* sc = nullptr;
  return get_schedule(P, 0, P->n_max, &sc);
}

spid_status apply_error_cfg(spid_plan_t P, const TuneCfg& c) {
  if (c.err_path == 1) {
    spid_status st = ensure_error_tc(P);
    if (st != SPID_OK) return st;
  }
  P->tune.err_path = c.err_path;
  P->tune.err_rows = c.err_rows;
  P->tune.err_cols = c.err_cols;
  return upload_error_units(P);
}

// Median of `reps` timed runs of fn after one warm-up, CUDA events on cs.
template <typename F>
spid_status time_median(cudaStream_t cs, int reps, F fn, float* ms) {
  spid_status st = fn();
  if (st != SPID_OK) return st;
  std::vector<float> t;
  cudaEvent_t e0, e1;
  SPID_CUDA(cudaEventCreate(&e0));
  SPID_CUDA(cudaEventCreate(&e1));
  for (int r = 0; r < reps && st == SPID_OK; ++r) {
    cudaEventRecord(e0, cs);
    st = fn();
    cudaEventRecord(e1, cs);
    cudaError_t e = cudaEventSynchronize(e1);
    float x = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&x, e0, e1);
    if (e != cudaSuccess && st == SPID_OK)
      st = fail(SPID_ERR_CUDA, std::string("tuning timer: ") + cudaGetErrorString(e));
    t.push_back(x);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != SPID_OK) return st;
  std::sort(t.begin(), t.end());
  *ms = t[t.size() / 2];
  return SPID_OK;
}

}  // namespace

extern "C" spid_status spid_plan_get_tuning(spid_plan_t P, spid_tuning* out) {
  if (!P || !out) return fail(SPID_ERR_INVALID_ARG, "plan/out is NULL");
  *out = tuning_of(P->tune, P->tuned_sketch_ms, P->tuned_error_ms);
  return SPID_OK;
}

extern "C" spid_status spid_plan_set_tuning(spid_plan_t P, const spid_tuning* t) {
  spid_status st = check_plan(P);
  if (st != SPID_OK) return st;
  if (!t || !valid_tuning(*t)) return fail(SPID_ERR_INVALID_ARG, "tuning value out of range");
  if (P->live_graphs > 0) return fail(SPID_ERR_STATE, "graphs captured from the plan exist");
  if (t->error_path == 1 && !P->err_tc_possible())
    return fail(SPID_ERR_UNSUPPORTED, "the tensor-core error pass needs a batched TF32/BF16/3xBF16 "
                                      "plan with k_max <= 32");
  if (t->sketch_slice_cols && t->sketch_slice_cols != kSliceCols && P->prec != SPID_PREC_TF32)
    return fail(SPID_ERR_UNSUPPORTED, "slices narrower than 64 columns: TF32 plans only");
  std::lock_guard<std::mutex> g(P->tune_mu);
  SPID_CUDA(cudaDeviceSynchronize());
  const TuneCfg c = cfg_of(*t);
  st = apply_sketch_cfg(P, c);
  if (st == SPID_OK) st = apply_error_cfg(P, c);
  P->tuned_sketch_ms = P->tuned_error_ms = 0.f;
  return st;
}

extern "C" spid_status spid_plan_autotune(spid_plan_t P, const void* window, spid_stream_t stream,
                                          spid_tuning* best) {
  return spid_plan_autotune_calls(P, window, 0, stream, best);
}

extern "C" spid_status spid_plan_autotune_calls(spid_plan_t P, const void* window,
                                                int32_t microbatch, spid_stream_t stream,
                                                spid_tuning* best) {
  spid_status st = check_plan(P);
  if (st != SPID_OK) return st;
  if (!window || reinterpret_cast<uintptr_t>(window) % 16)
    return fail(SPID_ERR_INVALID_ARG, "window is NULL or not 16-byte aligned");
  if (microbatch < 0) return fail(SPID_ERR_INVALID_ARG, "microbatch must be >= 0");
  // the column ranges the caller sketches: the whole window, or runs of
  // `microbatch` columns
  std::vector<std::pair<int, int>> calls;
  if (microbatch == 0 || microbatch >= P->n_max) calls.push_back({0, P->n_max});
  else
    for (int c = 0; c < P->n_max; c += microbatch) calls.push_back({c, std::min(microbatch, P->n_max - c)});
  auto sketch_calls = [&]() -> spid_status {
    for (const auto& cr : calls) {
      Schedule* sc = nullptr;
      spid_status s2 = get_schedule(P, cr.first, cr.second, &sc);
      if (s2 == SPID_OK) s2 = launch_sketch_range(P, sc, window, P->d_tmaps, (cudaStream_t)stream);
      if (s2 != SPID_OK) return s2;
    }
    return SPID_OK;
  };
  if (P->live_graphs > 0) return fail(SPID_ERR_STATE, "graphs captured from the plan exist");
  std::lock_guard<std::mutex> g(P->tune_mu);
  cudaStream_t cs = (cudaStream_t)stream;
  SPID_CUDA(cudaDeviceSynchronize());
  if (P->tensor_core()) {
    st = bind_window(P, window, cs);
    if (st != SPID_OK) return st;
  }
  constexpr int kReps = 5;
  constexpr float kTuneMargin = 0.02f;
  // ---- sketch candidates
  std::vector<TuneCfg> cands;
  if (P->tensor_core()) {
    for (int order : {0, 1})
      for (int ps : {8, 4, 2, 1})
        for (int stg : {0, 4, 2}) {
          if (order == 1 && ps < 4) continue;   // small packs: the order hardly matters
          TuneCfg c = P->tune;
          c.slice_major = order;
          c.pack_slices = ps;
          c.stages = stg;
          c.slice_cols = kSliceCols;
          cands.push_back(c);
        }
    // narrower slices (fewer window columns per chunk), full 512-column packs
    if (P->prec == SPID_PREC_TF32)
      for (int order : {0, 1})
        for (int w : {32, 16}) {
          TuneCfg c = P->tune;
          c.slice_major = order;
          c.pack_slices = kPackSlices;
          c.stages = 0;
          c.slice_cols = w;
          cands.push_back(c);
        }
  } else {
    // the default first (2-slice packs, CTAs per SM by the register budget of
    // each call's variant), then other pack widths and CTA counts
    for (int ps : {kSimtPackSlices, 4, 8, 1}) {
      TuneCfg c = P->tune;
      c.pack_slices = ps;
      c.ctas_per_sm = 0;
      cands.push_back(c);
    }
    for (int cps : {1, 2, 3, 4}) {
      TuneCfg c = P->tune;
      c.pack_slices = kSimtPackSlices;
      c.ctas_per_sm = cps;
      cands.push_back(c);
    }
  }
  TuneCfg best_cfg = P->tune;
  float best_sk = 0.f;
  int seen_stages = -1, seen_pack = -1, seen_order = -1, seen_width = -1;
  for (const TuneCfg& c : cands) {
    st = apply_sketch_cfg(P, c);
    if (st == SPID_ERR_UNSUPPORTED) continue;   // e.g. too few stages fit
    if (st != SPID_OK) return st;
    // the tensor maps carry the slice width: re-encode them for this candidate
    if (P->tensor_core()) {
      st = bind_window(P, window, cs);
      if (st != SPID_OK) return st;
    }
    Schedule* sc = nullptr;
    st = get_schedule(P, calls[0].first, calls[0].second, &sc);
    if (st != SPID_OK) return st;
    // stage counts above what fits collapse onto the same launch: skip repeats
    if (P->tensor_core() && sc->stages == seen_stages && c.pack_slices == seen_pack &&
        c.slice_major == seen_order && c.slice_cols == seen_width)
      continue;
    seen_stages = sc->stages;
    seen_pack = c.pack_slices;
    seen_order = c.slice_major;
    seen_width = c.slice_cols;
    float ms = 0.f;
    st = time_median(cs, kReps, sketch_calls, &ms);
    if (st != SPID_OK) return st;
    // the first candidate is the default; another must beat the best so far
    // by kTuneMargin to replace it (run-to-run noise is a few percent)
    if (best_sk == 0.f || ms < best_sk * (1.f - kTuneMargin)) {
      best_sk = ms;
      best_cfg.pack_slices = c.pack_slices;
      best_cfg.slice_major = c.slice_major;
      best_cfg.slice_cols = c.slice_cols;
      best_cfg.stages = c.stages;
      best_cfg.ctas_per_sm = c.ctas_per_sm;
    }
  }
  st = apply_sketch_cfg(P, best_cfg);
  if (st == SPID_OK && P->tensor_core()) st = bind_window(P, window, cs);
  if (st != SPID_OK) return st;
  st = sketch_calls();
  if (st == SPID_OK) st = run_finalize(P, cs);
  if (st != SPID_OK) return st;
  // ---- error-pass candidates
  std::vector<TuneCfg> ecands;
  {
    TuneCfg t = best_cfg;   // the default shape first
    t.err_path = 0;
    t.err_rows = kErrRowBlock;
    t.err_cols = kErrColBlock;
    ecands.push_back(t);
  }
  for (int r : kTuneErrRows)
    for (int c : kTuneErrCols) {
      if (r == kErrRowBlock && c == kErrColBlock) continue;
      TuneCfg t = best_cfg;
      t.err_path = 0;
      t.err_rows = r;
      t.err_cols = c;
      ecands.push_back(t);
    }
  if (P->err_tc_possible()) {
    TuneCfg t = best_cfg;
    t.err_path = 1;
    t.err_rows = kErrRowBlock;
    t.err_cols = kErrColBlock;
    ecands.push_back(t);
  }
  float best_er = 0.f;
  TuneCfg best_e = best_cfg;
  for (const TuneCfg& c : ecands) {
    st = apply_error_cfg(P, c);
    if (st != SPID_OK) return st;
    float ms = 0.f;
    st = time_median(cs, kReps, [&] { return run_error(P, window, nullptr, nullptr, nullptr, cs); },
                     &ms);
    if (st != SPID_OK) return st;
    if (best_er == 0.f || ms < best_er * (1.f - kTuneMargin)) {
      best_er = ms;
      best_e = c;
    }
  }
  st = apply_error_cfg(P, best_e);
  if (st != SPID_OK) return st;
  SPID_CUDA(cudaStreamSynchronize(cs));
  P->tuned_sketch_ms = best_sk;
  P->tuned_error_ms = best_er;
  if (best) *best = tuning_of(P->tune, best_sk, best_er);
  return SPID_OK;
}

extern "C" spid_status spid_plan_tuning_key(spid_plan_t P, char* buf, int32_t len) {
  spid_status st = check_plan(P);
  if (st != SPID_OK) return st;
  if (!buf || len <= 0) return fail(SPID_ERR_INVALID_ARG, "buf is NULL or len <= 0");
  cudaDeviceProp prop;
  SPID_CUDA(cudaGetDeviceProperties(&prop, P->device));
  double msum = 0.0, nsum = 0.0;
  for (int s = 0; s < P->S; ++s) {
    msum += P->m[s];
    nsum += P->n[s];
  }
  auto lg = [](double x) { return x >= 1.0 ? (int)std::floor(std::log2(x)) : 0; };
  const int w = std::snprintf(buf, (size_t)len,
                              "spid-tune-2;cc=%d.%d;sms=%d;prec=%d;flags=%u;l_pad=%d;k_max=%d;"
                              "log2S=%d;log2m=%d;log2n=%d",
                              prop.major, prop.minor, P->num_sms, P->prec, P->flags, P->l_pad,
                              P->k_max, lg(P->S), lg(msum / P->S), lg(nsum / P->S));
  if (w < 0 || w >= len) return fail(SPID_ERR_INVALID_ARG, "key buffer too small");
  return SPID_OK;
}

// ---------------------------------------------------------------------------
// CUDA graphs of one step
// ---------------------------------------------------------------------------
struct spid_graph_s {
  spid_plan_t plan = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  void* d_tmaps = nullptr;
  // host-window launches: the device window, its extent, the error sums and
  // the events that order the copy against this graph's previous launch
  void* window = nullptr;
  size_t window_bytes = 0;
  double* total_dev = nullptr;
  cudaEvent_t ev_uploaded = nullptr, ev_done = nullptr;
  bool launched = false;
};

extern "C" spid_status spid_graph_destroy(spid_graph_t G) {
  if (!G) return SPID_OK;
  if (G->plan) cudaSetDevice(G->plan->device);
  cudaDeviceSynchronize();
  if (G->exec) cudaGraphExecDestroy(G->exec);
  if (G->graph) cudaGraphDestroy(G->graph);
  if (G->d_tmaps) cudaFree(G->d_tmaps);
  if (G->ev_uploaded) cudaEventDestroy(G->ev_uploaded);
  if (G->ev_done) cudaEventDestroy(G->ev_done);
  if (G->plan) G->plan->live_graphs--;
  delete G;
  return SPID_OK;
}

extern "C" spid_status spid_graph_create(spid_plan_t P, const void* window, int32_t col0,
                                         int32_t ncols, int32_t microbatch, uint32_t what,
                                         double* err_dev, double* total_dev,
                                         spid_graph_t* out) {
  spid_status st = check_plan(P);
  if (st != SPID_OK) return st;
  if (!out) return fail(SPID_ERR_INVALID_ARG, "graph_out is NULL");
  *out = nullptr;
  if (what == 0 || (what & ~7u)) return fail(SPID_ERR_INVALID_ARG, "what must be a non-empty OR of SPID_GRAPH_*");
  const bool sketch = what & SPID_GRAPH_SKETCH, finalize = what & SPID_GRAPH_FINALIZE,
             error = what & SPID_GRAPH_ERROR;
  if ((sketch || error) && (!window || reinterpret_cast<uintptr_t>(window) % 16))
    return fail(SPID_ERR_INVALID_ARG, "window is NULL or not 16-byte aligned");
  if (col0 < 0 || ncols < 0 || microbatch < 0)
    return fail(SPID_ERR_INVALID_ARG, "negative column range or micro-batch");
  // schedules of every sketch call, built before capture (they may allocate)
  std::vector<Schedule*> scheds;
  if (sketch && ncols > 0 && col0 < P->n_max) {
    ncols = std::min(ncols, P->n_max - col0);
    const int mb = microbatch > 0 ? microbatch : ncols;
    for (int c = col0; c < col0 + ncols; c += mb) {
      Schedule* sc = nullptr;
      st = get_schedule(P, c, std::min(mb, col0 + ncols - c), &sc);
      if (st != SPID_OK) return st;
      scheds.push_back(sc);
    }
  }
  spid_graph_s* G = new spid_graph_s();
  G->plan = P;
  P->live_graphs++;
  auto bail = [&](spid_status s2) {
    spid_graph_destroy(G);
    return s2;
  };
  if (!scheds.empty() && P->tensor_core()) {
    std::vector<CUtensorMap> maps;
    st = encode_window_maps(P, window, maps);
    if (st != SPID_OK) return bail(st);
    cudaError_t e = cudaMalloc(&G->d_tmaps, sizeof(CUtensorMap) * maps.size());
    if (e == cudaSuccess)
      e = cudaMemcpy(G->d_tmaps, maps.data(), sizeof(CUtensorMap) * maps.size(),
                     cudaMemcpyHostToDevice);
    if (e != cudaSuccess)
      return bail(fail(e == cudaErrorMemoryAllocation ? SPID_ERR_OOM : SPID_ERR_CUDA,
                       std::string("graph tensor maps: ") + cudaGetErrorString(e)));
  }
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return bail(fail(SPID_ERR_CUDA, cudaGetErrorString(e)));
  e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return bail(fail(SPID_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e)));
  }
  spid_status cap = SPID_OK;
  for (Schedule* sc : scheds)
    if (cap == SPID_OK) cap = launch_sketch_range(P, sc, window, G->d_tmaps, cs);
  if (cap == SPID_OK && finalize) cap = run_finalize(P, cs);
  if (cap == SPID_OK && error) cap = run_error(P, window, nullptr, err_dev, total_dev, cs);
  e = cudaStreamEndCapture(cs, &G->graph);
  cudaStreamDestroy(cs);
  if (cap != SPID_OK) return bail(cap);
  if (e != cudaSuccess)
    return bail(fail(SPID_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e)));
  e = cudaGraphInstantiate(&G->exec, G->graph, 0);
  if (e != cudaSuccess)
    return bail(fail(SPID_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e)));
  if (sketch || error) {
    G->window = const_cast<void*>(window);
    G->window_bytes = (size_t)P->window_extent * P->esz;
  }
  G->total_dev = total_dev;
  e = cudaEventCreateWithFlags(&G->ev_uploaded, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&G->ev_done, cudaEventDisableTiming);
  if (e != cudaSuccess)
    return bail(fail(SPID_ERR_CUDA, std::string("graph events: ") + cudaGetErrorString(e)));
  *out = G;
  return SPID_OK;
}

extern "C" spid_status spid_graph_launch_host(spid_graph_t G, const void* window_host,
                                              double* total_host, int32_t* k_host,
                                              int32_t* J_host, void* C_host,
                                              spid_stream_t copy_stream, spid_stream_t stream) {
  if (!G || !G->exec) return fail(SPID_ERR_INVALID_ARG, "graph is NULL");
  if (!window_host) return fail(SPID_ERR_INVALID_ARG, "window_host is NULL");
  if (!G->window) return fail(SPID_ERR_INVALID_ARG, "graph has no window (finalize only)");
  if (total_host && !G->total_dev)
    return fail(SPID_ERR_INVALID_ARG, "total_host given but the graph has no total_dev");
  spid_status st = check_plan(G->plan);
  if (st != SPID_OK) return st;
  cudaStream_t cps = (cudaStream_t)copy_stream, cs = (cudaStream_t)stream;
  const bool split = cps != cs;
  if (split && G->launched) SPID_CUDA(cudaStreamWaitEvent(cps, G->ev_done, 0));
  SPID_CUDA(cudaMemcpyAsync(G->window, window_host, G->window_bytes, cudaMemcpyHostToDevice, cps));
  if (split) {
    SPID_CUDA(cudaEventRecord(G->ev_uploaded, cps));
    SPID_CUDA(cudaStreamWaitEvent(cs, G->ev_uploaded, 0));
  }
  SPID_CUDA(cudaGraphLaunch(G->exec, cs));
  if (split) {
    SPID_CUDA(cudaEventRecord(G->ev_done, cs));
    G->launched = true;
  }
  spid_plan_t P = G->plan;
  if (total_host)
    SPID_CUDA(cudaMemcpyAsync(total_host, G->total_dev, (4 + 2 * (size_t)P->num_qoi) * sizeof(double),
                              cudaMemcpyDeviceToHost, cs));
  // the compressed representation of the step (Algorithms 2-3 output)
  if (k_host)
    SPID_CUDA(cudaMemcpyAsync(k_host, P->d_k, sizeof(int32_t) * P->S, cudaMemcpyDeviceToHost, cs));
  if (J_host)
    SPID_CUDA(cudaMemcpyAsync(J_host, P->d_J, sizeof(int32_t) * P->S * P->k_max,
                              cudaMemcpyDeviceToHost, cs));
  if (C_host)
    SPID_CUDA(cudaMemcpyAsync(C_host, P->d_C, P->esz * P->c_elems, cudaMemcpyDeviceToHost, cs));
  return SPID_OK;
}

extern "C" spid_status spid_graph_launch(spid_graph_t G, spid_stream_t stream) {
  if (!G || !G->exec) return fail(SPID_ERR_INVALID_ARG, "graph is NULL");
  spid_status st = check_plan(G->plan);
  if (st != SPID_OK) return st;
  SPID_CUDA(cudaGraphLaunch(G->exec, (cudaStream_t)stream));
  return SPID_OK;
}
