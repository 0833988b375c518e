// producer.cu -- an in-situ snapshot producer for measuring compression
// alongside a running solver (Section 5.2 and Algorithms 4-6: the flow solver
// updates the state every time step and the compression consumes the
// snapshots).  It is a stand-in for the paper's compressible Navier-Stokes
// solver, not part of the decomposition: one explicit step of
//   f_t + (u . grad) f = nu lap f
// for every QoI f of the state, velocity u = QoIs 1..3, on a periodic grid^3
// grid of spacing h = 2 pi / grid; first-order upwind advection and the
// 7-point Laplacian, forward Euler.  Stable for dt (3 max|u| / h + 6 nu / h^2)
// <= 1.
//
// State layout = one snapshot of a box-major window: box b's [q][z][y][x]
// block (nq edge^3 floats) starts at element b * box_stride, box index
// (bz nb + by) nb + bx with nb = grid/edge -- box_stride = nq edge^3 for a
// snapshot-major window ([j][box][rows]), = nq edge^3 n for a subdomain-major
// one ([box][j][rows], the pointer at column j).
// One thread per grid point computes the 7 neighbour offsets once (periodic
// wrap across boxes) and updates every QoI; each point is read 7 times per
// QoI, mostly from L1/L2, and written once.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "../../include/spid.h"
#include "spid_internal.cuh"

namespace spid {
namespace {

struct ProducerArgs {
  const float* in;
  float* out;
  int32_t grid, edge, nb, nq;
  int64_t in_stride, out_stride;   // elements between consecutive boxes
  int64_t field;                   // edge^3
  float dt, nu, inv_h, inv_h2;
};

// (box, offset inside the box) of grid point (X, Y, Z)
__device__ __forceinline__ void point_at(const ProducerArgs& a, int X, int Y, int Z, int64_t& box,
                                         int64_t& local) {
  const int bx = X / a.edge, by = Y / a.edge, bz = Z / a.edge;
  const int x = X - bx * a.edge, y = Y - by * a.edge, z = Z - bz * a.edge;
  box = ((int64_t)bz * a.nb + by) * a.nb + bx;
  local = ((int64_t)z * a.edge + y) * a.edge + x;
}

__device__ __forceinline__ int64_t in_offset(const ProducerArgs& a, int X, int Y, int Z) {
  int64_t box, local;
  point_at(a, X, Y, Z, box, local);
  return box * a.in_stride + local;
}

__global__ void __launch_bounds__(256) producer_step_kernel(const ProducerArgs a) {
  const int64_t npts = (int64_t)a.grid * a.grid * a.grid;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npts;
       p += (int64_t)gridDim.x * blockDim.x) {
    // p enumerates the state in storage order: box, then (z, y, x) inside it
    const int64_t box = p / a.field;
    const int64_t rem = p - box * a.field;
    const int z = (int)(rem / ((int64_t)a.edge * a.edge));
    const int y = (int)((rem / a.edge) % a.edge);
    const int x = (int)(rem % a.edge);
    const int bx = (int)(box % a.nb), by = (int)((box / a.nb) % a.nb), bz = (int)(box / ((int64_t)a.nb * a.nb));
    const int X = bx * a.edge + x, Y = by * a.edge + y, Z = bz * a.edge + z;
    const int G = a.grid;
    const int64_t o0 = box * a.in_stride + rem;
    const int64_t oo = box * a.out_stride + rem;
    const int64_t oxm = in_offset(a, (X + G - 1) % G, Y, Z), oxp = in_offset(a, (X + 1) % G, Y, Z);
    const int64_t oym = in_offset(a, X, (Y + G - 1) % G, Z), oyp = in_offset(a, X, (Y + 1) % G, Z);
    const int64_t ozm = in_offset(a, X, Y, (Z + G - 1) % G), ozp = in_offset(a, X, Y, (Z + 1) % G);
    const float u = __ldg(a.in + o0 + 1 * a.field);
    const float v = __ldg(a.in + o0 + 2 * a.field);
    const float w = __ldg(a.in + o0 + 3 * a.field);
    for (int q = 0; q < a.nq; ++q) {
      const float* f = a.in + (int64_t)q * a.field;
      const float f0 = __ldg(f + o0);
      const float fxm = __ldg(f + oxm), fxp = __ldg(f + oxp);
      const float fym = __ldg(f + oym), fyp = __ldg(f + oyp);
      const float fzm = __ldg(f + ozm), fzp = __ldg(f + ozp);
      const float adv = (u > 0.f ? u * (f0 - fxm) : u * (fxp - f0)) +
                        (v > 0.f ? v * (f0 - fym) : v * (fyp - f0)) +
                        (w > 0.f ? w * (f0 - fzm) : w * (fzp - f0));
      const float lap = (fxm + fxp) + (fym + fyp) + (fzm + fzp) - 6.f * f0;
      a.out[(int64_t)q * a.field + oo] = f0 - a.dt * a.inv_h * adv + a.nu * a.dt * a.inv_h2 * lap;
    }
  }
}

}  // namespace
}  // namespace spid

extern "C" spid_status spid_producer_step(const float* state_in, int64_t in_box_stride,
                                          float* state_out, int64_t out_box_stride, int32_t grid,
                                          int32_t edge, int32_t nq, float dt, float nu,
                                          spid_stream_t stream) {
  using namespace spid;
  const int64_t box_elems = (int64_t)nq * edge * edge * edge;
  if (!state_in || !state_out || state_in == state_out || grid < 2 || edge < 1 ||
      grid % edge || nq < 4 || !(dt > 0.f) || !(nu >= 0.f) || in_box_stride < box_elems ||
      out_box_stride < box_elems) {
    set_last_error("spid_producer_step: need distinct buffers, grid % edge == 0, nq >= 4, "
                   "dt > 0, nu >= 0, box strides >= nq edge^3");
    return SPID_ERR_INVALID_ARG;
  }
  ProducerArgs a;
  a.in = state_in;
  a.out = state_out;
  a.grid = grid;
  a.edge = edge;
  a.nb = grid / edge;
  a.nq = nq;
  a.field = (int64_t)edge * edge * edge;
  a.in_stride = in_box_stride;
  a.out_stride = out_box_stride;
  const float h = 6.283185307179586f / (float)grid;
  a.inv_h = 1.f / h;
  a.inv_h2 = 1.f / (h * h);
  a.dt = dt;
  a.nu = nu;
  // per-box QoI planes are a.field apart: QoI q of a point is at offset q field
  // from its QoI-0 element inside the same box
  const int64_t npts = (int64_t)grid * grid * grid;
  const int blocks = (int)std::min<int64_t>((npts + 255) / 256, 152 * 16);
  producer_step_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error((std::string("spid_producer_step: ") + cudaGetErrorString(e)).c_str());
    return SPID_ERR_CUDA;
  }
  return SPID_OK;
}
