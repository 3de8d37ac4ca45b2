// ph_stage.cu -- instantiations and launchers of the fused stage kernel (K3),
// and the tensor maps its TMA variant copies planes with.
#include <cuda.h>

#include <cstdlib>
#include <cstring>
#include <mutex>

#include "ph_nvtx.h"
#include "ph_internal.h"
#include "ph_stage.cuh"
#include "ph_stage_pair.cuh"

namespace ph {

bool stage_tile_supported(int TX, int TY) {
  return (TX == 8 && TY == 8) || (TX == 16 && TY == 8) || (TX == 16 && TY == 16) ||
         (TX == 32 && TY == 8);
}

bool stage_pair_tile(int TX, int TY) { return TX == PairSmem::TX && TY == PairSmem::TY; }

bool stage_pair_kernel(bool fp32, bool tma, int nvar, bool multi_level, const int tile[3], const int nx[3]) {
  if (!fp32 || !tma || nvar != NV || multi_level || tile[1] != 16) return false;
  if (tile[0] != 32 && tile[0] != 16) return false;
  return nx[0] % tile[0] == 0 && nx[1] % tile[1] == 0;
}

template <class T>
size_t stage_smem_bytes(int TX, int TY) {
  if (sizeof(T) == 4 && stage_pair_tile(TX, TY)) return PairSmem::bytes;
  if (TX == 8 && TY == 8) return StageSmem<T, 8, 8>::bytes;
  if (TX == 16 && TY == 8) return StageSmem<T, 16, 8>::bytes;
  if (TX == 16 && TY == 16) return StageSmem<T, 16, 16>::bytes;
  if (TX == 32 && TY == 8) return StageSmem<T, 32, 8>::bytes;
  return 0;
}

template <class T, int TX, int TY, int NVT = NV>
static cudaError_t configure_tile() {
  cudaError_t e = cudaFuncSetAttribute(stage_kernel<T, TX, TY, NVT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)StageSmem<T, TX, TY, NVT>::bytes);
  if (e != cudaSuccess) return e;
  for (int st = 0; st < 3; ++st) {
    if (NVT != NV && st > 0) break;  // per-stage instances: hydro variables only
    auto* k = st == 0 ? stage_kernel_tma<T, TX, TY, NVT, 0>
                      : (st == 1 ? stage_kernel_tma<T, TX, TY, NVT, 1> : stage_kernel_tma<T, TX, TY, NVT, 2>);
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)StageSmem<T, TX, TY, NVT>::bytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Meshes with passive scalars: tiles 16 x 16 and 8 x 8, one or two scalars.
bool stage_scalar_tile(int TX, int TY) { return (TX == 16 && TY == 16) || (TX == 8 && TY == 8); }

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
  if ((e = configure_tile<double, 16, 16, NV + 1>()) != cudaSuccess) return e;
  if ((e = configure_tile<double, 16, 16, NV + 2>()) != cudaSuccess) return e;
  if ((e = configure_tile<double, 8, 8, NV + 1>()) != cudaSuccess) return e;
  if ((e = configure_tile<double, 8, 8, NV + 2>()) != cudaSuccess) return e;
  if ((e = configure_tile<float, 16, 16, NV + 1>()) != cudaSuccess) return e;
  if ((e = configure_tile<float, 16, 16, NV + 2>()) != cudaSuccess) return e;
  if ((e = configure_tile<float, 8, 8, NV + 1>()) != cudaSuccess) return e;
  if ((e = configure_tile<float, 8, 8, NV + 2>()) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(stage_kernel_pair<32, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)PairSmem::bytes)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(stage_kernel_pair<32, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)PairSmem::bytes)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(stage_kernel_pair<16, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)PairSmem16::bytes)) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(stage_kernel_pair<16, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)PairSmem16::bytes);
}

template <class T, int TX, int TY, int NVT = NV>
static cudaError_t launch_tile(const StageArgs<T>& a, const CUtensorMap* tmap, cudaStream_t s) {
  using SM = StageSmem<T, TX, TY, NVT>;
  const unsigned grid = (unsigned)a.nleaf * a.ntile[0] * a.ntile[1] * a.ntile[2];
  if (grid == 0) return cudaSuccess;
  if (tmap)
    if (NVT != NV)
      stage_kernel_tma<T, TX, TY, NVT, 0><<<grid, SM::NT, SM::bytes, s>>>(a, *tmap);
    else if (a.stage == 1)
      stage_kernel_tma<T, TX, TY, NVT, 1><<<grid, SM::NT, SM::bytes, s>>>(a, *tmap);
    else
      stage_kernel_tma<T, TX, TY, NVT, 2><<<grid, SM::NT, SM::bytes, s>>>(a, *tmap);
  else
    stage_kernel<T, TX, TY, NVT><<<grid, SM::NT, SM::bytes, s>>>(a);
  return cudaGetLastError();
}

template <class T, int NVT>
static cudaError_t launch_scalar_tiles(const StageArgs<T>& a, int TX, int TY, cudaStream_t s,
                                       const CUtensorMap* tmap) {
  if (TX == 16 && TY == 16) return launch_tile<T, 16, 16, NVT>(a, tmap, s);
  if (TX == 8 && TY == 8) return launch_tile<T, 8, 8, NVT>(a, tmap, s);
  return cudaErrorInvalidValue;
}

// The paired FP32 kernel (TXP x 16 tiles, TMA staging, uniform meshes).
template <int TXP>
static cudaError_t launch_pair(const StageArgs<float>& a, const CUtensorMap* tmap, cudaStream_t s) {
  using SM = PairSmemT<TXP>;
  if (!tmap || a.face_rec || a.nx[0] % TXP || a.nx[1] % SM::TY) return cudaErrorInvalidValue;
  const unsigned grid = (unsigned)a.nleaf * a.ntile[0] * a.ntile[1] * a.ntile[2];
  if (grid == 0) return cudaSuccess;
  if (a.stage == 1)
    stage_kernel_pair<TXP, 1><<<grid, SM::NT, SM::bytes, s>>>(a, *tmap);
  else
    stage_kernel_pair<TXP, 2><<<grid, SM::NT, SM::bytes, s>>>(a, *tmap);
  return cudaGetLastError();
}

// Resident CTAs per SM of the stage-2 kernel a launch would run (0 if the
// query fails); stage 1 has the same shape.
template <class K>
static int occupancy_of(K kernel, int nt, size_t smem) {
  int n = 0;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, nt, smem) == cudaSuccess ? n : 0;
}

template <class T, int TX, int TY, int NVT = NV>
static int tile_occupancy(bool tma) {
  using SM = StageSmem<T, TX, TY, NVT>;
  if (!tma) return occupancy_of(stage_kernel<T, TX, TY, NVT>, SM::NT, SM::bytes);
  if (NVT != NV) return occupancy_of(stage_kernel_tma<T, TX, TY, NVT, 0>, SM::NT, SM::bytes);
  return occupancy_of(stage_kernel_tma<T, TX, TY, NVT, 2>, SM::NT, SM::bytes);
}

template <class T>
int stage_ctas_per_sm(int TX, int TY, int nvar, bool pair, bool tma) {
  if constexpr (sizeof(T) == 4) {
    if (pair && TX == 32 && TY == 16) return occupancy_of(stage_kernel_pair<32, 2>, PairSmem::NT, PairSmem::bytes);
    if (pair && TX == 16 && TY == 16)
      return occupancy_of(stage_kernel_pair<16, 2>, PairSmem16::NT, PairSmem16::bytes);
  }
  if (pair) return 0;
  if (nvar == NV + 1 || nvar == NV + 2) {
    const bool one = nvar == NV + 1;
    if (TX == 16 && TY == 16) return one ? tile_occupancy<T, 16, 16, NV + 1>(tma) : tile_occupancy<T, 16, 16, NV + 2>(tma);
    if (TX == 8 && TY == 8) return one ? tile_occupancy<T, 8, 8, NV + 1>(tma) : tile_occupancy<T, 8, 8, NV + 2>(tma);
    return 0;
  }
  if (TX == 8 && TY == 8) return tile_occupancy<T, 8, 8>(tma);
  if (TX == 16 && TY == 8) return tile_occupancy<T, 16, 8>(tma);
  if (TX == 16 && TY == 16) return tile_occupancy<T, 16, 16>(tma);
  if (TX == 32 && TY == 8) return tile_occupancy<T, 32, 8>(tma);
  return 0;
}

template <class T>
cudaError_t launch_stage(const StageArgs<T>& a, int TX, int TY, cudaStream_t s, const CUtensorMap* tmap) {
  PH_RANGE("ph stage");
  if (a.nvar == NV + 1) return launch_scalar_tiles<T, NV + 1>(a, TX, TY, s, tmap);
  if (a.nvar == NV + 2) return launch_scalar_tiles<T, NV + 2>(a, TX, TY, s, tmap);
  if (a.nvar != NV) return cudaErrorInvalidValue;
  if (a.pair || stage_pair_tile(TX, TY)) {
    if constexpr (sizeof(T) == 4) {
      if (a.pair && TX == 32 && TY == 16) return launch_pair<32>(a, tmap, s);
      if (a.pair && TX == 16 && TY == 16) return launch_pair<16>(a, tmap, s);
    }
    return cudaErrorInvalidValue;
  }
  if (TX == 8 && TY == 8) return launch_tile<T, 8, 8>(a, tmap, s);
  if (TX == 16 && TY == 8) return launch_tile<T, 16, 8>(a, tmap, s);
  if (TX == 16 && TY == 16) return launch_tile<T, 16, 16>(a, tmap, s);
  if (TX == 32 && TY == 8) return launch_tile<T, 32, 8>(a, tmap, s);
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- tensor maps

namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}
}  // namespace

bool stage_tma_wanted() {
  const char* e = std::getenv("PH_STAGE_LOADS");
  return !(e && std::strcmp(e, "plain") == 0);
}

// Tensor map over a pool of padded blocks [leaf][v][k][j][i] seen as a 4-D
// tensor (S1, S2, S3, nvar * nleaf) with box (TX+4, TY+4, 1, nvar).  Returns false
// (and the stage kernel keeps its plain loads) when the layout breaks a TMA
// rule: rows of S1 elements must be a multiple of 16 bytes, as must the box
// rows and the base address.
bool make_stage_tmap(CUtensorMap* out, const void* base, size_t esize, const int S[3], int nleaf, int TX,
                     int TY, int nvar) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || !base || nleaf <= 0) return false;
  if (((size_t)S[0] * esize) % 16 || ((size_t)(TX + 4) * esize) % 16) return false;
  if (reinterpret_cast<uintptr_t>(base) % 16) return false;
  if (TY + 4 > 256 || TX + 4 > 256) return false;
  cuuint64_t dims[4] = {(cuuint64_t)S[0], (cuuint64_t)S[1], (cuuint64_t)S[2], (cuuint64_t)nvar * nleaf};
  cuuint64_t strides[3] = {(cuuint64_t)S[0] * esize, (cuuint64_t)S[0] * S[1] * esize,
                           (cuuint64_t)S[0] * S[1] * S[2] * esize};
  cuuint32_t box[4] = {(cuuint32_t)(TX + 4), (cuuint32_t)(TY + 4), 1, (cuuint32_t)nvar};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  std::memset(out, 0, sizeof(*out));
  CUresult r = fn(out, esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4,
                  const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template cudaError_t launch_stage<double>(const StageArgs<double>&, int, int, cudaStream_t,
                                          const CUtensorMap*);
template cudaError_t launch_stage<float>(const StageArgs<float>&, int, int, cudaStream_t,
                                         const CUtensorMap*);
template int stage_ctas_per_sm<double>(int, int, int, bool, bool);
template int stage_ctas_per_sm<float>(int, int, int, bool, bool);
template size_t stage_smem_bytes<double>(int, int);
template size_t stage_smem_bytes<float>(int, int);

}  // namespace ph
