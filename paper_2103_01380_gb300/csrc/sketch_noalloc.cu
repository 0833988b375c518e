// sketch_noalloc.cu -- an FP32 sketch of one subdomain that allocates nothing.
//
// Who needs it: an in-situ caller -- a simulation that reserves nearly all of
// the GPU's memory for its own fields through its own pool at start-up, or
// that runs its time loop with no allocation and no implicit device
// synchronization (cudaMalloc / cudaFree may synchronize the device) -- cannot
// create a plan (spid_plan_create allocates its workspace) in the middle of a
// run.  This entry point takes the caller's input and output pointers and keeps
// its split-K partial sums in one fixed, file-scope device array instead.
//
// The paper has no counterpart: it is a deployment convenience, not part of
// the method.  The arithmetic is the FP32 SIMT sketch (Y = Omega A with the same
// Omega as every other entry point); only where the partial sums live differs.
//
// Shared-state rules: the static array is held by every GPU that loads this
// library until the process exits; every call uses the same array and leaves
// its contents behind; calls that overlap on the GPU (different streams, or
// different host threads without ordering) race on it.
#include <mutex>

#include "../../include/spid.h"
#include "spid_internal.cuh"

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaJGroups = 64;
constexpr int kNaMaxDevices = 64;

// The scratch: SPID_NOALLOC_SCRATCH_FLOATS FP32 partial sums (8 MiB).
static __device__ __align__(256) float g_noalloc_scratch[SPID_NOALLOC_SCRATCH_FLOATS];

struct NaArgs {
  const float* A;
  int32_t m, n;
  int64_t ld;
  int32_t l;
  int32_t ctas;         // CTAs per column group (split of the rows)
  int32_t chunks;       // 32-row chunks of A
  uint64_t seed;
  float* scratch;       // device address of g_noalloc_scratch
  float* Y;
  int32_t ldy;
};

// Grid: (ctas, column groups of up to 64 TJ columns).  CTA (c, g) sketches the
// rows of chunks [c chunks / ctas, (c+1) chunks / ctas) for the columns of
// group g and writes its partial to slot (g, c) of the scratch.
template <int TI, int TJ>
__global__ void __launch_bounds__(kNaThreads, (TI * TJ <= 64) ? 2 : 1)
sketch_noalloc_kernel(NaArgs a) {
  constexpr int LP = 4 * TI;
  constexpr int CG = kNaJGroups * TJ;
  constexpr int CGP = CG + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* As = reinterpret_cast<float*>(smem_raw);      // [32][CGP]
  float* Om = As + spid::kChunkRows * CGP;               // [32][LP], 16-byte aligned (CGP*32*4 % 16 == 0)

  const int tid = threadIdx.x;
  const int ig = tid / kNaJGroups, jg = tid % kNaJGroups;
  const int c = blockIdx.x, g = blockIdx.y;
  const int col0 = g * CG;
  const int nc = min(CG, a.n - col0);
  const int ch0 = (int)((int64_t)c * a.chunks / a.ctas);
  const int ch1 = (int)((int64_t)(c + 1) * a.chunks / a.ctas);
  const uint2 key = spid::philox_key(a.seed);
  const float* A = a.A + (int64_t)col0 * a.ld;

  float acc[TJ][TI];
#pragma unroll
  for (int u = 0; u < TJ; ++u)
#pragma unroll
    for (int v = 0; v < TI; ++v) acc[u][v] = 0.f;

  for (int ch = ch0; ch < ch1; ++ch) {
    const int r0 = ch * spid::kChunkRows;
    for (int v = tid; v < nc * 8; v += kNaThreads) {
      const int cc = v / 8, q = v % 8;
      const int r = r0 + 4 * q;
      const float* src = A + (int64_t)cc * a.ld + r;
      float x[4];
      if (r + 4 <= a.m) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(src));
        x[0] = t.x; x[1] = t.y; x[2] = t.z; x[3] = t.w;
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = (r + u < a.m) ? src[u] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) As[(4 * q + u) * CGP + cc] = x[u];
    }
    for (int task = tid; task < spid::kChunkRows * (LP / 4); task += kNaThreads) {
      const int k = task % spid::kChunkRows, gg = task / spid::kChunkRows;
      float w[4] = {0.f, 0.f, 0.f, 0.f};
      if (4 * gg < a.l && r0 + k < a.m) {
        spid::omega_group<float>(key, (uint32_t)(r0 + k), (uint32_t)gg, w);
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (4 * gg + u >= a.l) w[u] = 0.f;
      }
      *reinterpret_cast<float4*>(Om + k * LP + 4 * gg) = make_float4(w[0], w[1], w[2], w[3]);
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < spid::kChunkRows; ++k) {
      float av[TJ], wv[TI];
#pragma unroll
      for (int u = 0; u < TJ; ++u) av[u] = As[k * CGP + jg + kNaJGroups * u];
#pragma unroll
      for (int v = 0; v < TI; v += 4) {
        const float4 t = *reinterpret_cast<const float4*>(Om + k * LP + ig * TI + v);
        wv[v] = t.x; wv[v + 1] = t.y; wv[v + 2] = t.z; wv[v + 3] = t.w;
      }
#pragma unroll
      for (int u = 0; u < TJ; ++u)
#pragma unroll
        for (int v = 0; v < TI; ++v) acc[u][v] = fmaf(av[u], wv[v], acc[u][v]);
    }
    __syncthreads();
  }
  // slot (g, c): [column in group][LP]; a CTA with no rows writes zeros
  float* slot = a.scratch + ((int64_t)g * a.ctas + c) * CG * LP;
#pragma unroll
  for (int u = 0; u < TJ; ++u) {
    const int j = jg + kNaJGroups * u;
    if (j < nc) {
#pragma unroll
      for (int v = 0; v < TI; v += 4)
        *reinterpret_cast<float4*>(slot + (int64_t)j * LP + ig * TI + v) =
            make_float4(acc[u][v], acc[u][v + 1], acc[u][v + 2], acc[u][v + 3]);
    }
  }
}

// Y(i, j) = sum over c of slot (g, c) in increasing c (fixed order).
template <int LP, int CG>
__global__ void __launch_bounds__(256) reduce_noalloc_kernel(NaArgs a) {
  const int64_t total = (int64_t)a.n * a.l;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / a.l), i = (int)(e % a.l);
    const int g = j / CG, jj = j % CG;
    const float* base = a.scratch + (int64_t)g * a.ctas * CG * LP + (int64_t)jj * LP + i;
    float s = 0.f;
    for (int c = 0; c < a.ctas; ++c) s += base[(int64_t)c * CG * LP];
    a.Y[(int64_t)j * a.ldy + i] = s;
  }
}

std::mutex g_setup_mu;
float* g_scratch_ptr[kNaMaxDevices] = {};
int g_num_sms[kNaMaxDevices] = {};

spid_status na_fail(spid_status s, const char* what) {
  spid::set_last_error(what);
  return s;
}

template <int TI, int TJ>
cudaError_t launch_na(const NaArgs& a, int groups, cudaStream_t st) {
  constexpr int LP = 4 * TI;
  constexpr int CGP = kNaJGroups * TJ + 1;
  const size_t smem = sizeof(float) * (size_t)spid::kChunkRows * (CGP + LP);
  auto k = sketch_noalloc_kernel<TI, TJ>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<dim3(a.ctas, groups), kNaThreads, smem, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int64_t total = (int64_t)a.n * a.l;
  const int rgrid = (int)((total + 255) / 256 < 1024 ? (total + 255) / 256 : 1024);
  reduce_noalloc_kernel<LP, kNaJGroups * TJ><<<rgrid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

extern "C" spid_status spid_sketch_fp32_noalloc(const float* A, int32_t m, int32_t n, int64_t ld,
                                                int32_t l, uint64_t seed, float* Y, int32_t ldy,
                                                spid_stream_t stream) {
  if (!A || !Y) return na_fail(SPID_ERR_INVALID_ARG, "A and Y must be device pointers");
  if (m < 1 || n < 1 || l < 1 || l > 64 || ld < m || ldy < l)
    return na_fail(SPID_ERR_INVALID_ARG, "need m, n >= 1, 1 <= l <= 64, ld >= m, ldy >= l");
  if ((reinterpret_cast<uintptr_t>(A) % 16) || (ld % 4))
    return na_fail(SPID_ERR_INVALID_ARG, "A must be 16-byte aligned with ld a multiple of 4");
  const int l_pad = (l + 15) / 16 * 16;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return na_fail(SPID_ERR_CUDA, "cudaGetDevice failed");
  if (dev < 0 || dev >= kNaMaxDevices)
    return na_fail(SPID_ERR_UNSUPPORTED, "device ordinal beyond the 64 devices whose scratch "
                                         "address this entry point caches");
  {
    // one-time set-up per device, with that device current: the device
    // address of the static array (host code cannot use the symbol itself)
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) return na_fail(SPID_ERR_CUDA, cudaGetErrorString(e));
      int sms = 0;
      e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return na_fail(SPID_ERR_CUDA, cudaGetErrorString(e));
      g_num_sms[dev] = sms;
      g_scratch_ptr[dev] = static_cast<float*>(p);
    }
  }
  const int TJ = 8;
  const int CG = kNaJGroups * TJ;
  const int groups = (n + CG - 1) / CG;
  const int64_t chunks = ((int64_t)m + spid::kChunkRows - 1) / spid::kChunkRows;
  // every CTA owns one slot of CG x l_pad floats in each column group
  int64_t ctas = (int64_t)SPID_NOALLOC_SCRATCH_FLOATS / ((int64_t)groups * CG * l_pad);
  const int64_t want = 2 * (int64_t)g_num_sms[dev];
  if (ctas > want) ctas = want;
  if (ctas > chunks) ctas = chunks;
  if (ctas < 1)
    return na_fail(SPID_ERR_INVALID_ARG,
                   "column groups x l_pad exceed the static scratch (SPID_NOALLOC_SCRATCH_FLOATS floats)");
  NaArgs a;
  a.A = A;
  a.m = m;
  a.n = n;
  a.ld = ld;
  a.l = l;
  a.ctas = (int32_t)ctas;
  a.chunks = (int32_t)chunks;
  a.seed = seed;
  a.scratch = g_scratch_ptr[dev];
  a.Y = Y;
  a.ldy = ldy;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaErrorInvalidValue;
  switch (l_pad) {
    case 16: e = launch_na<4, 8>(a, groups, st); break;
    case 32: e = launch_na<8, 8>(a, groups, st); break;
    case 48: e = launch_na<12, 8>(a, groups, st); break;
    case 64: e = launch_na<16, 8>(a, groups, st); break;
  }
  if (e != cudaSuccess) return na_fail(SPID_ERR_CUDA, cudaGetErrorString(e));
  return SPID_OK;
}
