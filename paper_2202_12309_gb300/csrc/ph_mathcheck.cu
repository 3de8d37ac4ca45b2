// ph_mathcheck.cu -- evaluates the stage kernels' reciprocal and root
// routines on caller data, so that their accuracy can be tested against the
// correctly rounded CUDA operations.
#include "../../include/ph_hydro.h"
#include "ph_device.cuh"
#include "ph_internal.h"

namespace {

template <class T>
__global__ void math_kernel(int fn, const T* __restrict__ x, T* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const T v = x[i];
    T r;
    switch (fn) {
      case PH_MATH_RCP: r = ph::rcp(v); break;
      case PH_MATH_RSQRT: r = ph::rsq(v); break;
      default: r = ph::sq(v); break;
    }
    y[i] = r;
  }
}

__global__ void math_approx_kernel(int fn, const double* __restrict__ x, double* __restrict__ y,
                                   long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = fn == PH_MATH_RCP_APPROX ? ph::rcp_approx(x[i]) : ph::rsqrt_approx(x[i]);
}

int mfail(int code, const char* msg) {
  ph::set_error_message(msg);
  return code;
}

}  // namespace

extern "C" int ph_debug_math(int32_t fn, int32_t precision, const void* x, void* y, int64_t n,
                             void* stream) {
  if (fn < PH_MATH_RCP || fn > PH_MATH_RSQRT_APPROX || (precision != PH_FP64 && precision != PH_FP32) ||
      n < 0 || (n > 0 && (!x || !y)))
    return mfail(PH_ERR_INVALID, "ph_debug_math: bad argument");
  if (fn >= PH_MATH_RCP_APPROX && precision != PH_FP64)
    return mfail(PH_ERR_INVALID, "ph_debug_math: the raw approximations are FP64 only");
  if (n == 0) return PH_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  if (fn >= PH_MATH_RCP_APPROX)
    math_approx_kernel<<<grid, 256, 0, s>>>(fn, (const double*)x, (double*)y, n);
  else if (precision == PH_FP64)
    math_kernel<double><<<grid, 256, 0, s>>>(fn, (const double*)x, (double*)y, n);
  else
    math_kernel<float><<<grid, 256, 0, s>>>(fn, (const float*)x, (float*)y, n);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return mfail(PH_ERR_CUDA, cudaGetErrorString(e));
  return PH_OK;
}

// ---------------------------------------------------------------------------
// Fused multiply-add throughput probe: every thread runs `iters` rounds of 8
// independent multiply-add chains (no memory traffic inside the loop), so the
// launch is bound by the FP64 pipe (kind 0), the FP32 pipe (kind 1) or the
// FP32 pipe with paired fma.rn.f32x2 (kind 2).  The caller times the launch;
// flops = ctas * 256 * iters * 8 * 2 (x 2 lanes for kind 2).
namespace {

template <class T>
__global__ void __launch_bounds__(256) fma_rate_kernel(long long iters, T b, T c, T* __restrict__ out) {
  T a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = T(threadIdx.x + j);
  for (long long it = 0; it < iters; ++it)
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = fma(a[j], b, c);
  T s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j];
  out[blockIdx.x * 256 + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) fma_rate_pair_kernel(long long iters, float b, float c,
                                                              float* __restrict__ out) {
  unsigned long long a[8], bb, cc;
  asm("mov.b64 %0, {%1, %1};" : "=l"(bb) : "f"(b));
  asm("mov.b64 %0, {%1, %1};" : "=l"(cc) : "f"(c));
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float x = (float)(threadIdx.x + j), y = x + 0.5f;
    asm("mov.b64 %0, {%1, %2};" : "=l"(a[j]) : "f"(x), "f"(y));
  }
  for (long long it = 0; it < iters; ++it)
#pragma unroll
    for (int j = 0; j < 8; ++j) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[j]) : "l"(bb), "l"(cc));
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float x, y;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a[j]));
    s += x + y;
  }
  out[blockIdx.x * 256 + threadIdx.x] = s;
}

}  // namespace

extern "C" int ph_debug_fma_rate(int32_t kind, int32_t ctas, int64_t iters, void* out, void* stream) {
  if (kind < 0 || kind > 2 || ctas < 1 || ctas > (1 << 20) || iters < 1 || iters > (1ll << 32) || !out)
    return mfail(PH_ERR_INVALID, "ph_debug_fma_rate: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  if (kind == 0)
    fma_rate_kernel<double><<<ctas, 256, 0, s>>>(iters, 0.9999999999, 1e-10, (double*)out);
  else if (kind == 1)
    fma_rate_kernel<float><<<ctas, 256, 0, s>>>(iters, 0.9999f, 1e-5f, (float*)out);
  else
    fma_rate_pair_kernel<<<ctas, 256, 0, s>>>(iters, 0.9999f, 1e-5f, (float*)out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return mfail(PH_ERR_CUDA, cudaGetErrorString(e));
  return PH_OK;
}
