// ph_noalloc.cu -- conserved totals for callers that cannot allocate device
// memory.
//
// Who needs it: callers that may not call cudaMalloc at all -- a plugin whose
// host application owns every byte of device memory, a solver embedded in a
// code that reserves its whole memory budget up front, or a time-critical
// loop that must not enter the CUDA allocator (it can block and synchronise).
// ph_totals needs a per-block scratch buffer that its mesh allocated; this
// variant takes the state from the caller and keeps its scratch in a fixed
// file-scope __device__ array instead.
//
// The array holds PH_TOTALS_NOALLOC_MAX_BLOCKS x 7 doubles (896 KiB: up to
// 5 conserved variables plus 2 passive scalars per block) on every GPU that
// loads the library, for the life of the process.  In host code the array's
// name is only a host-side stand-in, so its device address is looked up once
// per device with cudaGetSymbolAddress (on the first call made while that
// device is current) and passed to the kernels.
#include <mutex>

#include "../../include/ph_hydro.h"
#include "ph_internal.h"

namespace {

constexpr int kMaxBlocks = PH_TOTALS_NOALLOC_MAX_BLOCKS;
constexpr int kMaxVar = ph::NV + ph::MAXS;
constexpr int kMaxLevels = ph::MAXLEV + 1;
constexpr int kMaxDevices = 64;

// Per-block partial sums, kMaxVar entries per block: every call overwrites
// entries [0, nblocks * nvar) and reads only those, so nothing has to start
// at zero.  Shared by all calls.
static __device__ __align__(256) double g_partial[kMaxBlocks * kMaxVar];

std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

struct Vols {
  double v[kMaxLevels];
  int nlevels;
};

// One CTA per block: FP64 sums of every variable over the block's interior
// cells, times the cell volume of the block's level.  A level outside
// [0, nlevels) has no volume: its sums become NaN, and so do the totals.
template <class T>
__global__ void noalloc_block_sums(const T* __restrict__ U, int3 nx, int nvar,
                                   const int8_t* __restrict__ level, Vols vol, double* partial) {
  __shared__ double red[kMaxVar][256];
  const int b = blockIdx.x;
  const int cells = nx.x * nx.y * nx.z;
  const T* Ub = U + (size_t)b * nvar * cells;
  double acc[kMaxVar];
#pragma unroll
  for (int v = 0; v < kMaxVar; ++v) acc[v] = 0.0;
  for (int c = threadIdx.x; c < cells; c += blockDim.x)
#pragma unroll
    for (int v = 0; v < kMaxVar; ++v)
      if (v < nvar) acc[v] += (double)Ub[(size_t)v * cells + c];
#pragma unroll
  for (int v = 0; v < kMaxVar; ++v) red[v][threadIdx.x] = acc[v];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int v = 0; v < kMaxVar; ++v) red[v][threadIdx.x] += red[v][threadIdx.x + w];
    __syncthreads();
  }
  if ((int)threadIdx.x < nvar) {
    const int l = level ? (int)level[b] : 0;
    const double dv = (l >= 0 && l < vol.nlevels) ? vol.v[l] : __longlong_as_double(0x7ff8000000000000ll);
    partial[(size_t)b * nvar + threadIdx.x] = red[threadIdx.x][0] * dv;
  }
}

__global__ void noalloc_final(const double* __restrict__ partial, int nblocks, int nvar, double* out) {
  const int v = threadIdx.x;
  if (v >= nvar) return;
  double s = 0.0, comp = 0.0;  // Neumaier compensated sum over blocks in order
  for (int b = 0; b < nblocks; ++b) {
    const double x = partial[(size_t)b * nvar + v];
    const double t = s + x;
    if (fabs(s) >= fabs(x))
      comp += (s - t) + x;
    else
      comp += (x - t) + s;
    s = t;
  }
  out[v] = s + comp;
}

int reject(int code, const char* msg) {
  ph::set_error_message(msg);  // readable through ph_last_error()
  return code;
}

}  // namespace

extern "C" int ph_totals_noalloc(const void* U, int32_t precision, const int32_t nx[3], int32_t nvar,
                                 int32_t nblocks, const int8_t* level, const double* vol,
                                 int32_t nlevels, double* out, void* stream) {
  if (!U || !nx || !out || !vol) return reject(PH_ERR_INVALID, "ph_totals_noalloc: null argument");
  if (precision != PH_FP64 && precision != PH_FP32)
    return reject(PH_ERR_INVALID, "ph_totals_noalloc: precision must be PH_FP64 or PH_FP32");
  if (nx[0] < 1 || nx[1] < 1 || nx[2] < 1)
    return reject(PH_ERR_INVALID, "ph_totals_noalloc: nx must be positive");
  if (nvar < ph::NV || nvar > kMaxVar)
    return reject(PH_ERR_INVALID, "ph_totals_noalloc: nvar must be 5, 6 or 7 (5 + passive scalars)");
  if (nlevels < 1 || nlevels > kMaxLevels)
    return reject(PH_ERR_INVALID, "ph_totals_noalloc: nlevels must be 1 .. 5");
  if (!level && nlevels != 1)
    return reject(PH_ERR_INVALID, "ph_totals_noalloc: level is NULL but nlevels > 1");
  if (nblocks < 0 || nblocks > kMaxBlocks)
    return reject(PH_ERR_INVALID,
                  "ph_totals_noalloc: nblocks exceeds PH_TOTALS_NOALLOC_MAX_BLOCKS (16384)");
  Vols vols{};
  vols.nlevels = nlevels;
  for (int l = 0; l < nlevels; ++l) vols.v[l] = vol[l];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return reject(PH_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return reject(PH_ERR_INVALID, "ph_totals_noalloc: device index above 63");
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_partial);
      if (e != cudaSuccess) return reject(PH_ERR_CUDA, cudaGetErrorString(e));
      g_addr[dev] = (double*)p;
    }
    scratch = g_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int3 n3 = make_int3(nx[0], nx[1], nx[2]);
  if (nblocks > 0) {
    if (precision == PH_FP64)
      noalloc_block_sums<double><<<nblocks, 256, 0, s>>>((const double*)U, n3, nvar, level, vols, scratch);
    else
      noalloc_block_sums<float><<<nblocks, 256, 0, s>>>((const float*)U, n3, nvar, level, vols, scratch);
  }
  noalloc_final<<<1, 32, 0, s>>>(scratch, nblocks, nvar, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return reject(PH_ERR_CUDA, cudaGetErrorString(e));
  return PH_OK;
}
