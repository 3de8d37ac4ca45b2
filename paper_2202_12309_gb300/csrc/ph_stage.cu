// ph_stage.cu -- instantiations and launcher of the fused stage kernel (K3).
#include "ph_internal.h"
#include "ph_stage.cuh"

namespace ph {

bool stage_tile_supported(int TX, int TY) {
  return (TX == 8 && TY == 8) || (TX == 16 && TY == 8) || (TX == 16 && TY == 16) ||
         (TX == 32 && TY == 8);
}

template <class T>
size_t stage_smem_bytes(int TX, int TY) {
  if (TX == 8 && TY == 8) return StageSmem<T, 8, 8>::bytes;
  if (TX == 16 && TY == 8) return StageSmem<T, 16, 8>::bytes;
  if (TX == 16 && TY == 16) return StageSmem<T, 16, 16>::bytes;
  if (TX == 32 && TY == 8) return StageSmem<T, 32, 8>::bytes;
  return 0;
}

template <class T, int TX, int TY>
static cudaError_t configure_tile() {
  return cudaFuncSetAttribute(stage_kernel<T, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)StageSmem<T, TX, TY>::bytes);
}

// Opt every instantiation into its dynamic shared memory once per device,
// outside any stream capture.
cudaError_t configure_stage_kernels() {
  cudaError_t e;
  if ((e = configure_tile<double, 8, 8>()) != cudaSuccess) return e;
  if ((e = configure_tile<double, 16, 8>()) != cudaSuccess) return e;
  if ((e = configure_tile<double, 16, 16>()) != cudaSuccess) return e;
  if ((e = configure_tile<double, 32, 8>()) != cudaSuccess) return e;
  if ((e = configure_tile<float, 8, 8>()) != cudaSuccess) return e;
  if ((e = configure_tile<float, 16, 8>()) != cudaSuccess) return e;
  if ((e = configure_tile<float, 16, 16>()) != cudaSuccess) return e;
  if ((e = configure_tile<float, 32, 8>()) != cudaSuccess) return e;
  return cudaSuccess;
}

template <class T, int TX, int TY>
static cudaError_t launch_tile(const StageArgs<T>& a, cudaStream_t s) {
  const size_t smem = StageSmem<T, TX, TY>::bytes;
  const unsigned grid = (unsigned)a.nleaf * a.ntile[0] * a.ntile[1] * a.ntile[2];
  if (grid == 0) return cudaSuccess;
  stage_kernel<T, TX, TY><<<grid, TX * TY, smem, s>>>(a);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_stage(const StageArgs<T>& a, int TX, int TY, cudaStream_t s) {
  if (TX == 8 && TY == 8) return launch_tile<T, 8, 8>(a, s);
  if (TX == 16 && TY == 8) return launch_tile<T, 16, 8>(a, s);
  if (TX == 16 && TY == 16) return launch_tile<T, 16, 16>(a, s);
  if (TX == 32 && TY == 8) return launch_tile<T, 32, 8>(a, s);
  return cudaErrorInvalidValue;
}

template cudaError_t launch_stage<double>(const StageArgs<double>&, int, int, cudaStream_t);
template cudaError_t launch_stage<float>(const StageArgs<float>&, int, int, cudaStream_t);
template size_t stage_smem_bytes<double>(int, int);
template size_t stage_smem_bytes<float>(int, int);

}  // namespace ph
