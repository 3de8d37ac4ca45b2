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
