// ph_batch.cu -- many independent uniform meshes advanced by one persistent
// launch per cycle, captured in a CUDA graph.
//
// Each member is a periodic uniform mesh with its own block size, block count,
// problem and dt.  One cooperative kernel runs the whole cycle for all
// members: stage 1 over a work list of (leaf, tile) items, ghost exchange,
// stage 2 (folding each member's signal-speed max), ghost exchange, and the
// per-member dt update, separated by four grid barriers.  The paper's point
// that kernel-launch latency dominates small blocks (Sec. 5.1) is taken to its
// end: one launch per cycle however many meshes and blocks there are.
//
// Grid barriers spin on a generation counter with an iteration limit; a CTA
// that gives up sets an error word and every CTA returns, so a stalled
// barrier can never hang the GPU (the host reads PH_ERR_TIMEOUT).
#include <algorithm>
#include <array>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ph_hydro.h"
#include "ph_nvtx.h"
#include "ph_internal.h"
#include "ph_stage.cuh"
#include "ph_stage_pair.cuh"

namespace ph {

struct GridBar {
  unsigned int count;
  unsigned int gen;
  int error;
  int pad;
};

struct Member {
  long long off;  // element offset of the member's first block in each pool
  int nx[3], S[3], nb[3];
  int ntile[3];
  int tile[2];    // the member's tile (TX, TY)
  int KC;
  int nleaf, leaf0;
  double idx[3];
  double cfl;
  double gamma, dfloor, pfloor;
};

template <class T>
struct BatchArgs {
  T* U0;
  T* U1;
  const Member* mem;
  const int* leaf_member;   // global leaf -> member
  const int* nbr;           // 27 member-local neighbour leaves per global leaf
  const int2* items;        // (global leaf, tile) in cost order
  int nitems, nleaf, nsim;
  DevScalars* sc;           // one per member
  GridBar* bar;
  unsigned long long spin_limit;
  // TMA plane staging: per member, the tensor maps of the U0 and U1 pools
  // (2 m and 2 m + 1), in device memory
  const CUtensorMap* tmaps;
  // the stages write the ghost zones of their output (push exchange), so the
  // cycle has no ghost phases
  int push;
};

// Bounded grid barrier.  Returns false (in every thread of the CTA) if this
// CTA gave up or another CTA reported an error.
__device__ __forceinline__ bool grid_barrier(GridBar* gb, unsigned long long spin_limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = &gb->gen;
    volatile int* verr = &gb->error;
    const unsigned int g = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&gb->count, 1u);
    int ok = 1;
    if (arrived == gridDim.x - 1) {
      gb->count = 0u;
      __threadfence();
      atomicAdd(&gb->gen, 1u);
    } else {
      unsigned long long it = 0;
      while (*vgen == g) {
        if (*verr) { ok = 0; break; }
        if (++it > spin_limit) {
          atomicExch(&gb->error, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok && !*verr;
  }
  __syncthreads();
  return s_ok != 0;
}

template <class T>
__device__ __forceinline__ Phys<T> member_phys(const Member& M) {
  Phys<T> P;
  P.gamma = (T)M.gamma;
  P.gm1 = (T)(M.gamma - 1.0);
  P.igm1 = (T)(1.0 / (M.gamma - 1.0));
  P.dfloor = (T)M.dfloor;
  P.pfloor = (T)M.pfloor;
  return P;
}

// Threads, shared memory and CTAs per SM (register budget) of the batch
// kernel for a launch choice.  Pair mode (FP32 with TMA staging, launch
// choice 32 x 16 or 16 x 16): every member runs the paired tile of
// ph_stage_pair.cuh of that width (its blocks must tile into it); other
// choices run the one-cell tile.
template <class T, int TX, int TY, bool TMA>
struct BatchTile {
  static constexpr bool PAIR = sizeof(T) == 4 && TMA && TY == 16 && (TX == 32 || TX == 16);
  using PS = PairSmemT<(TX == 16 ? 16 : 32)>;
  using One = StageSmem<T, (PAIR ? 16 : TX), (PAIR ? 16 : TY)>;
  static constexpr int NT = PAIR ? PS::NT : One::NT;
  static constexpr size_t bytes = PAIR ? PS::bytes : One::bytes;
  static constexpr size_t red_off = PAIR ? PS::red_off : One::red_off;
  static constexpr size_t bar_off = PAIR ? PS::bar_off : One::bar_off;
  // FP64: registers capped for 512 threads per SM (2 CTAs of a 16 x 16 tile),
  // as the single-mesh stage kernels compile; the cycle kernel holds both
  // stages and would otherwise take 150 registers (one CTA per SM)
  static constexpr int MINB = PAIR ? PS::MINB : (sizeof(T) == 4 ? 3 : (512 / NT > 0 ? 512 / NT : 1));
};

// The tile job of work item `it` in the given stage; returns the member.
template <class T>
__device__ __forceinline__ int batch_job(const BatchArgs<T>& a, int it, int stage, TileJob<T>& J) {
  const int2 item = a.items[it];
  const int g = item.x;
  const int m = a.leaf_member[g];
  const Member& M = a.mem[m];
  const size_t bsize = (size_t)NV * M.S[0] * M.S[1] * M.S[2];
  const size_t boff = (size_t)M.off + (size_t)(g - M.leaf0) * bsize;
  int t = item.y;
  const int tk = t / (M.ntile[0] * M.ntile[1]);
  t -= tk * M.ntile[0] * M.ntile[1];
  const int tj = t / M.ntile[0];
  const int ti = t - tj * M.ntile[0];
  J.Ub = (stage == 1 ? a.U0 : a.U1) + boff;
  J.U0b = a.U0 + boff;
  J.Uoutb = (stage == 1 ? a.U1 : a.U0) + boff;
  for (int d = 0; d < 3; ++d) {
    J.nx[d] = M.nx[d];
    J.S[d] = M.S[d];
  }
  J.i0 = ti * M.tile[0];
  J.j0 = tj * M.tile[1];
  J.k0 = tk * M.KC;
  J.k1 = min(J.k0 + M.KC, M.nx[2]);
  J.idx1 = (T)M.idx[0];
  J.idx2 = (T)M.idx[1];
  J.idx3 = (T)M.idx[2];
  J.dt = (T)a.sc[m].dt_next;
  J.stage = stage;
  J.want_rate = stage == 2;
  J.leaf = g;
  J.nbr27 = a.push ? a.nbr + 27 * g : nullptr;
  J.pool = (stage == 1 ? a.U1 : a.U0) + M.off;
  J.bsize = bsize;
  return m;
}

template <class T, int TX, int TY, bool TMA, int STAGE>
__device__ bool batch_stage_phase(const BatchArgs<T>& a, const StageArgs<T>& nocap, unsigned char* smem,
                                  double* red, unsigned& floors, uint64_t* bars, int* failed,
                                  unsigned* parity) {
  for (int it = blockIdx.x; it < a.nitems; it += gridDim.x) {
    TileJob<T> J;
    const int m = batch_job<T>(a, it, STAGE, J);
    const Member& M = a.mem[m];
    const int vz0 = (J.leaf - M.leaf0) * NV;
    const CUtensorMap* tm = TMA ? a.tmaps + 2 * m + (STAGE == 1 ? 0 : 1) : nullptr;
    double rate;
    if constexpr (BatchTile<T, TX, TY, TMA>::PAIR) {
      rate = stage_tile_pair<TX, STAGE, true>(J, member_phys<float>(M), smem, floors, tm, vz0, bars, failed, parity);
    } else {
      rate = stage_tile<T, TX, TY, TMA>(J, member_phys<T>(M), nocap, smem, floors, tm, vz0, bars, failed, parity);
    }
    if (TMA && *(volatile int*)failed) return false;  // every thread saw it after a barrier
    if (STAGE == 2) block_max_to(&a.sc[m].wmax_bits, rate, red);
    __syncthreads();  // the next item's priming overwrites the ring
  }
  return true;
}

template <class T>
__device__ void batch_ghost_phase(const BatchArgs<T>& a, T* U) {
  for (int g = blockIdx.x; g < a.nleaf; g += gridDim.x) {
    const Member& M = a.mem[a.leaf_member[g]];
    const Shell sh(M.nx);
    const size_t vs = (size_t)M.S[0] * M.S[1] * M.S[2];
    const size_t bsize = (size_t)NV * vs;
    T* base = U + M.off;
    T* dstb = base + (size_t)(g - M.leaf0) * bsize;
    const int* nb = a.nbr + 27 * g;
    const int total = sh.count();
    for (int c = threadIdx.x; c < total; c += blockDim.x) {
      int i, j, k;
      sh.cell(c, i, j, k);
      const int ox = i < NG ? -1 : (i >= NG + M.nx[0] ? 1 : 0);
      const int oy = j < NG ? -1 : (j >= NG + M.nx[1] ? 1 : 0);
      const int oz = k < NG ? -1 : (k >= NG + M.nx[2] ? 1 : 0);
      const T* srcb = base + (size_t)nb[(oz + 1) * 9 + (oy + 1) * 3 + (ox + 1)] * bsize;
      const size_t so =
          ((size_t)(k - oz * M.nx[2]) * M.S[1] + (j - oy * M.nx[1])) * M.S[0] + (i - ox * M.nx[0]);
      const size_t dofs = ((size_t)k * M.S[1] + j) * M.S[0] + i;
#pragma unroll
      for (int v = 0; v < NV; ++v) dstb[v * vs + dofs] = srcb[v * vs + so];
    }
  }
}

template <class T, int TX, int TY, bool TMA>
__global__ void __launch_bounds__(BatchTile<T, TX, TY, TMA>::NT, BatchTile<T, TX, TY, TMA>::MINB)
batch_cycle_kernel(const BatchArgs<T> a) {
  using SM = BatchTile<T, TX, TY, TMA>;
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  unsigned char* smem_raw = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_dyn) + 127) & ~uintptr_t(127));
  double* red = reinterpret_cast<double*>(smem_raw + SM::red_off);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + SM::bar_off);
  __shared__ int failed;
  unsigned parity = 0;
  if (TMA) {
    if (threadIdx.x == 0) {
      failed = 0;
      for (int s = 0; s < 4; ++s) mbar_init(bars + s, 1);
      mbar_fence_init();
    }
    __syncthreads();
  }
  StageArgs<T> nocap = {};
  unsigned floors = 0;
  // a failed barrier leaves a sticky error in the first member's scalars
#define PH_BARRIER_OR_RETURN                                         \
  if (!grid_barrier(a.bar, a.spin_limit)) {                          \
    if (threadIdx.x == 0) atomicExch(&a.sc[0].error, 1);             \
    return;                                                          \
  }
  // a CTA whose plane wait gave up reports it and leaves; the others give
  // up at the next grid barrier (bounded), so nothing hangs
#define PH_STAGE_OR_RETURN(st)                                                                \
  if (!batch_stage_phase<T, TX, TY, TMA, st>(a, nocap, smem_raw, red, floors, bars, &failed,   \
                                             &parity)) {                                      \
    if (threadIdx.x == 0) atomicExch(&a.sc[0].error, 1);                                      \
    return;                                                                                   \
  }
  // stage 1's interior writes and the ghost writes to U1 are read by stage
  // 2's TMA copies (async proxy) in other CTAs: proxy fence before the barrier
  PH_STAGE_OR_RETURN(1)
  if (TMA) fence_proxy_async_global();
  PH_BARRIER_OR_RETURN
  if (!a.push) {
    batch_ghost_phase<T>(a, a.U1);
    if (TMA) fence_proxy_async_global();
    PH_BARRIER_OR_RETURN
  }
  PH_STAGE_OR_RETURN(2)
  PH_BARRIER_OR_RETURN
  if (!a.push) {
    batch_ghost_phase<T>(a, a.U0);
    PH_BARRIER_OR_RETURN
  }
  if (floors) atomicAdd(&a.sc[0].floor_hits, (unsigned long long)floors);
#undef PH_BARRIER_OR_RETURN
#undef PH_STAGE_OR_RETURN
  if (blockIdx.x == 0) {
    for (int m = threadIdx.x; m < a.nsim; m += blockDim.x) {
      DevScalars& s = a.sc[m];
      s.dt_last = s.dt_next;
      s.time += s.dt_next;
      s.cycle += 1;
      const double w = __longlong_as_double((long long)s.wmax_bits);
      const double dt = a.mem[m].cfl / w;
      s.dt_next = dt;
      if (!isfinite(dt) || !(dt > 0.0)) s.nonfinite = 1;
      s.wmax_bits = 0ull;
    }
  }
}

// A barrier that cannot complete (it waits for one CTA more than the grid
// has): every CTA gives up after spin_limit iterations and reports it.
__global__ void barrier_timeout_kernel(GridBar* gb, unsigned long long spin_limit, int* out) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = &gb->gen;
    const unsigned int g = *vgen;
    atomicAdd(&gb->count, 1u);  // never reaches gridDim.x + 1
    unsigned long long it = 0;
    int ok = 1;
    while (*vgen == g) {
      if (++it > spin_limit) {
        atomicExch(&gb->error, 1);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    s_ok = ok;
  }
  __syncthreads();
  if (threadIdx.x == 0 && !s_ok) atomicAdd(out, 1);
}

template <class T, int TX, int TY, bool TMA>
size_t batch_smem() {
  return BatchTile<T, TX, TY, TMA>::bytes;
}

}  // namespace ph

using ph::BatchArgs;
using ph::DevScalars;
using ph::GridBar;
using ph::Member;

namespace {

int bfail(int code, const std::string& msg) {
  ph::set_error_message(msg.c_str());
  return code;
}
#define PB_CUDA(expr)                                                              \
  do {                                                                             \
    cudaError_t _e = (expr);                                                       \
    if (_e != cudaSuccess) return bfail(PH_ERR_CUDA, std::string(#expr) + ": " +   \
                                                         cudaGetErrorString(_e)); \
  } while (0)

// autotuner candidates; 16 x 16 is the 16-wide paired tile in pair mode,
// 32 x 16 exists only there
const int kTiles[5][2] = {{8, 8}, {16, 8}, {16, 16}, {32, 8}, {32, 16}};

}  // namespace

struct ph_batch {
  int nsim = 0;
  int precision = PH_FP64;
  size_t esize = 8;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  std::vector<ph_config> cfg;
  std::vector<Member> mem;
  int nleaf = 0;
  long long pool_elems = 0;
  // device
  void* U0 = nullptr;
  void* U1 = nullptr;
  Member* d_mem = nullptr;
  int* d_leaf_member = nullptr;
  int* d_nbr = nullptr;
  int2* d_items = nullptr;
  int nitems = 0;
  DevScalars* d_sc = nullptr;
  GridBar* d_bar = nullptr;
  CUtensorMap* d_tmaps = nullptr;  // 2 per member (U0, U1 pools), for TMA staging
  bool tma = false;
  bool push = true;  // stages fill the ghost zones (PH_GHOSTS=launch: ghost phases)
  void* staging = nullptr;
  size_t staging_bytes = 0;
  // launch choice
  int TX = 16, TY = 16, KC = 32, ctas_per_sm = 1;
  int grid = 0;
  unsigned long long spin_limit = 1ull << 24;
  cudaGraphExec_t gexec = nullptr;
  std::vector<void*> owned;

  void* dalloc(size_t bytes) {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) return nullptr;
    owned.push_back(p);
    return p;
  }
};

namespace {

template <class T, int TX, int TY, bool TMA>
cudaError_t set_attr() {
  return cudaFuncSetAttribute(ph::batch_cycle_kernel<T, TX, TY, TMA>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)ph::batch_smem<T, TX, TY, TMA>());
}

template <class T, int TX, int TY, bool TMA>
int occupancy(int* per_sm) {
  cudaError_t e = set_attr<T, TX, TY, TMA>();
  if (e != cudaSuccess) return bfail(PH_ERR_CUDA, cudaGetErrorString(e));
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, ph::batch_cycle_kernel<T, TX, TY, TMA>,
                                                    ph::BatchTile<T, TX, TY, TMA>::NT,
                                                    ph::batch_smem<T, TX, TY, TMA>());
  if (e != cudaSuccess) return bfail(PH_ERR_CUDA, cudaGetErrorString(e));
  return PH_OK;
}

template <class T, bool TMA>
int occupancy_t(int TX, int TY, int* per_sm) {
  if constexpr (sizeof(T) == 4 && TMA)
    if (TX == 32 && TY == 16) return occupancy<T, 32, 16, TMA>(per_sm);
  if (TX == 8 && TY == 8) return occupancy<T, 8, 8, TMA>(per_sm);
  if (TX == 16 && TY == 8) return occupancy<T, 16, 8, TMA>(per_sm);
  if (TX == 16 && TY == 16) return occupancy<T, 16, 16, TMA>(per_sm);
  if (TX == 32 && TY == 8) return occupancy<T, 32, 8, TMA>(per_sm);
  return bfail(PH_ERR_INVALID, "unsupported tile");
}

template <class T, int TX, int TY, bool TMA>
cudaError_t launch_cycle(ph_batch* b, cudaStream_t s) {
  PH_RANGE("ph batch cycle");
  BatchArgs<T> a;
  a.U0 = (T*)b->U0;
  a.U1 = (T*)b->U1;
  a.mem = b->d_mem;
  a.leaf_member = b->d_leaf_member;
  a.nbr = b->d_nbr;
  a.items = b->d_items;
  a.nitems = b->nitems;
  a.nleaf = b->nleaf;
  a.nsim = b->nsim;
  a.sc = b->d_sc;
  a.bar = b->d_bar;
  a.spin_limit = b->spin_limit;
  a.tmaps = b->d_tmaps;
  a.push = b->push ? 1 : 0;
  cudaLaunchConfig_t lc;
  std::memset(&lc, 0, sizeof(lc));
  lc.gridDim = dim3(b->grid);
  lc.blockDim = dim3(ph::BatchTile<T, TX, TY, TMA>::NT);
  lc.dynamicSmemBytes = ph::batch_smem<T, TX, TY, TMA>();
  lc.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  return cudaLaunchKernelEx(&lc, ph::batch_cycle_kernel<T, TX, TY, TMA>, a);
}

template <class T, bool TMA>
cudaError_t launch_cycle_tt(ph_batch* b, cudaStream_t s) {
  if constexpr (sizeof(T) == 4 && TMA)
    if (b->TX == 32 && b->TY == 16) return launch_cycle<T, 32, 16, TMA>(b, s);
  if (b->TX == 8 && b->TY == 8) return launch_cycle<T, 8, 8, TMA>(b, s);
  if (b->TX == 16 && b->TY == 8) return launch_cycle<T, 16, 8, TMA>(b, s);
  if (b->TX == 16 && b->TY == 16) return launch_cycle<T, 16, 16, TMA>(b, s);
  if (b->TX == 32 && b->TY == 8) return launch_cycle<T, 32, 8, TMA>(b, s);
  return cudaErrorInvalidValue;
}

template <class T>
cudaError_t launch_cycle_t(ph_batch* b, cudaStream_t s) {
  return b->tma ? launch_cycle_tt<T, true>(b, s) : launch_cycle_tt<T, false>(b, s);
}

// Tensor maps of every member's blocks in both pools for the member's tile;
// false if any member's geometry does not admit one (then plain loads).
bool build_tmaps(ph_batch* b) {
  if (!ph::stage_tma_wanted() || !b->d_tmaps) return false;
  std::vector<CUtensorMap> maps(2 * (size_t)b->nsim);
  for (int m = 0; m < b->nsim; ++m) {
    const Member& M = b->mem[m];
    const char* u0 = (const char*)b->U0 + (size_t)M.off * b->esize;
    const char* u1 = (const char*)b->U1 + (size_t)M.off * b->esize;
    if (!ph::make_stage_tmap(&maps[2 * m], u0, b->esize, M.S, M.nleaf, M.tile[0], M.tile[1]) ||
        !ph::make_stage_tmap(&maps[2 * m + 1], u1, b->esize, M.S, M.nleaf, M.tile[0], M.tile[1]))
      return false;
  }
  return cudaMemcpy(b->d_tmaps, maps.data(), sizeof(CUtensorMap) * maps.size(),
                    cudaMemcpyHostToDevice) == cudaSuccess;
}

// One cycle: reset the barrier word, then the persistent kernel.
cudaError_t launch_one(ph_batch* b, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b->d_bar, 0, sizeof(GridBar), s);
  if (e != cudaSuccess) return e;
  return b->precision == PH_FP32 ? launch_cycle_t<float>(b, s) : launch_cycle_t<double>(b, s);
}

void drop_graph(ph_batch* b) {
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
}

// Pair mode: FP32 with TMA staging and the launch choice 32 x 16 or 16 x 16;
// every member's blocks must tile into the choice (the paired tile of that
// width runs on all of them).
bool pair_choice(const ph_batch* b, int TX, int TY) {
  return b->precision == PH_FP32 && ph::stage_tma_wanted() && TY == 16 && (TX == 32 || TX == 16);
}
bool pair_possible(const ph_batch* b, int TX) {
  if (b->precision != PH_FP32 || !ph::stage_tma_wanted()) return false;
  for (const Member& M : b->mem)
    if (M.nx[0] % TX || M.nx[1] % 16) return false;
  return true;
}

// Apply a launch choice: tiles per member, the cost-ordered work list, grid.
int configure(ph_batch* b, int TX, int TY, int KC, int ctas) {
  const bool pair = pair_choice(b, TX, TY);
  if (pair && !pair_possible(b, TX))
    return bfail(PH_ERR_INVALID, "batch: FP32 tiles of 32 x 16 and 16 x 16 are paired and need TMA staging "
                                 "and blocks that tile into them");
  if (TX == 32 && TY == 16 && !pair)
    return bfail(PH_ERR_INVALID, "batch: the 32 x 16 tile is the paired FP32 tile");
  for (Member& M : b->mem) {
    M.tile[0] = TX;
    M.tile[1] = TY;
  }
  const bool tma = build_tmaps(b);
  if (pair && !tma) return bfail(PH_ERR_INVALID, "batch: the paired tile needs TMA staging");
  int per_sm = 0;
  int rc = b->precision == PH_FP32
               ? (tma ? occupancy_t<float, true>(TX, TY, &per_sm) : occupancy_t<float, false>(TX, TY, &per_sm))
               : (tma ? occupancy_t<double, true>(TX, TY, &per_sm) : occupancy_t<double, false>(TX, TY, &per_sm));
  if (rc) return rc;
  b->tma = tma;
  if (per_sm < 1) return bfail(PH_ERR_INVALID, "batch kernel does not fit on an SM");
  int dev = 0, nsm = 0;
  PB_CUDA(cudaGetDevice(&dev));
  PB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  if (ctas < 1) ctas = per_sm;
  ctas = std::min(ctas, per_sm);
  b->TX = TX;
  b->TY = TY;
  b->KC = KC;
  b->ctas_per_sm = ctas;
  b->grid = ctas * nsm;
  // tiles and items; cost of an item = planes it marches x tile area
  std::vector<std::pair<long long, int2>> items;
  for (int m = 0; m < b->nsim; ++m) {
    Member& M = b->mem[m];
    M.ntile[0] = (M.nx[0] + M.tile[0] - 1) / M.tile[0];
    M.ntile[1] = (M.nx[1] + M.tile[1] - 1) / M.tile[1];
    M.KC = std::min(KC, M.nx[2]);
    M.ntile[2] = (M.nx[2] + M.KC - 1) / M.KC;
    const int per = M.ntile[0] * M.ntile[1] * M.ntile[2];
    for (int l = 0; l < M.nleaf; ++l)
      for (int t = 0; t < per; ++t) {
        const int tk = t / (M.ntile[0] * M.ntile[1]);
        const long long planes = std::min(M.KC, M.nx[2] - tk * M.KC) + 3;
        items.push_back({planes, make_int2(M.leaf0 + l, t)});
      }
  }
  std::stable_sort(items.begin(), items.end(),
                   [](const std::pair<long long, int2>& x, const std::pair<long long, int2>& y) {
                     return x.first > y.first;
                   });
  std::vector<int2> flat(items.size());
  for (size_t i = 0; i < items.size(); ++i) flat[i] = items[i].second;
  if (b->d_items) {
    cudaFree(b->d_items);
    b->owned.erase(std::find(b->owned.begin(), b->owned.end(), (void*)b->d_items));
  }
  b->d_items = (int2*)b->dalloc(sizeof(int2) * std::max<size_t>(flat.size(), 1));
  if (!b->d_items) return bfail(PH_ERR_OOM, "device allocation failed (work list)");
  b->nitems = (int)flat.size();
  PB_CUDA(cudaMemcpyAsync(b->d_items, flat.data(), sizeof(int2) * flat.size(),
                          cudaMemcpyHostToDevice, b->stream));
  PB_CUDA(cudaMemcpyAsync(b->d_mem, b->mem.data(), sizeof(Member) * b->nsim,
                          cudaMemcpyHostToDevice, b->stream));
  PB_CUDA(cudaStreamSynchronize(b->stream));
  drop_graph(b);
  return PH_OK;
}

int capture(ph_batch* b) {
  drop_graph(b);
  PB_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t le = launch_one(b, b->cap);
  cudaGraph_t g = nullptr;
  cudaError_t ee = cudaStreamEndCapture(b->cap, &g);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return bfail(PH_ERR_CUDA, std::string("batch launch (capture): ") + cudaGetErrorString(le));
  }
  if (ee != cudaSuccess) return bfail(PH_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(ee));
  cudaError_t ie = cudaGraphInstantiate(&b->gexec, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    b->gexec = nullptr;
    return bfail(PH_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
  }
  return PH_OK;
}

int check_error_word(ph_batch* b) {
  DevScalars s0;
  PB_CUDA(cudaMemcpyAsync(&s0, b->d_sc, sizeof(s0), cudaMemcpyDeviceToHost, b->stream));
  PB_CUDA(cudaStreamSynchronize(b->stream));
  if (s0.error) return bfail(PH_ERR_TIMEOUT, "batch grid barrier gave up");
  return PH_OK;
}

int member_count(const ph_batch* b, int sim) {
  const Member& M = b->mem[sim];
  return M.nleaf * 5 * M.nx[0] * M.nx[1] * M.nx[2];
}

template <class T>
ph::Phys<T> phys_of(const Member& M) {
  ph::Phys<T> P;
  P.gamma = (T)M.gamma;
  P.gm1 = (T)(M.gamma - 1.0);
  P.igm1 = (T)(1.0 / (M.gamma - 1.0));
  P.dfloor = (T)M.dfloor;
  P.pfloor = (T)M.pfloor;
  return P;
}

template <class T>
int set_state_member(ph_batch* b, int sim, const void* U, int on_device) {
  Member& M = b->mem[sim];
  const size_t count = (size_t)member_count(b, sim);
  T* packed;
  if (on_device) {
    packed = (T*)U;
  } else {
    if (count * sizeof(T) > b->staging_bytes) {
      if (b->staging) {
        cudaFree(b->staging);
        b->owned.erase(std::find(b->owned.begin(), b->owned.end(), b->staging));
      }
      b->staging = b->dalloc(count * sizeof(T));
      if (!b->staging) {
        b->staging_bytes = 0;
        return bfail(PH_ERR_OOM, "device allocation failed (staging)");
      }
      b->staging_bytes = count * sizeof(T);
    }
    packed = (T*)b->staging;
    PB_CUDA(cudaMemcpyAsync(packed, U, count * sizeof(T), cudaMemcpyHostToDevice, b->stream));
  }
  T* base = (T*)b->U0 + M.off;
  PB_CUDA(ph::launch_pack<T>(base, packed, M.nx, M.nleaf, 0, b->stream));
  PB_CUDA(ph::launch_ghost_uniform<T>(base, b->d_nbr + 27 * M.leaf0, M.nx, M.nleaf, b->stream));
  DevScalars zero;
  PB_CUDA(cudaMemcpyAsync(&zero, b->d_sc + sim, sizeof(zero), cudaMemcpyDeviceToHost, b->stream));
  PB_CUDA(cudaStreamSynchronize(b->stream));
  const int sticky = zero.error;
  std::memset(&zero, 0, sizeof(zero));
  zero.error = sticky;
  PB_CUDA(cudaMemcpyAsync(b->d_sc + sim, &zero, sizeof(zero), cudaMemcpyHostToDevice, b->stream));
  ph::LevelGeom g;
  std::memset(&g, 0, sizeof(g));
  for (int d = 0; d < 3; ++d) g.idx[0][d] = M.idx[d];
  PB_CUDA(ph::launch_rate<T>(base, nullptr, g, M.nx, M.nleaf, phys_of<T>(M), b->d_sc + sim,
                             b->stream));
  PB_CUDA(ph::launch_advance(b->d_sc + sim, M.cfl, 2, b->stream));
  DevScalars hs;
  PB_CUDA(cudaMemcpyAsync(&hs, b->d_sc + sim, sizeof(hs), cudaMemcpyDeviceToHost, b->stream));
  PB_CUDA(cudaStreamSynchronize(b->stream));
  hs.dt_last = hs.dt_next;
  PB_CUDA(cudaMemcpy(b->d_sc + sim, &hs, sizeof(hs), cudaMemcpyHostToDevice));
  return PH_OK;
}

template <class T>
int get_state_member(ph_batch* b, int sim, void* U, int on_device) {
  Member& M = b->mem[sim];
  const size_t count = (size_t)member_count(b, sim);
  T* packed;
  if (on_device) {
    packed = (T*)U;
  } else {
    if (count * sizeof(T) > b->staging_bytes) {
      if (b->staging) {
        cudaFree(b->staging);
        b->owned.erase(std::find(b->owned.begin(), b->owned.end(), b->staging));
      }
      b->staging = b->dalloc(count * sizeof(T));
      if (!b->staging) {
        b->staging_bytes = 0;
        return bfail(PH_ERR_OOM, "device allocation failed (staging)");
      }
      b->staging_bytes = count * sizeof(T);
    }
    packed = (T*)b->staging;
  }
  T* base = (T*)b->U0 + M.off;
  PB_CUDA(ph::launch_pack<T>(base, packed, M.nx, M.nleaf, 1, b->stream));
  if (!on_device)
    PB_CUDA(cudaMemcpyAsync(U, packed, count * sizeof(T), cudaMemcpyDeviceToHost, b->stream));
  PB_CUDA(cudaStreamSynchronize(b->stream));
  return PH_OK;
}

}  // namespace

extern "C" {

int ph_batch_create(const ph_config* cfgs, int32_t nsim, void* stream, ph_batch** out) {
  if (!cfgs || !out || nsim < 1) return bfail(PH_ERR_INVALID, "ph_batch_create: bad argument");
  *out = nullptr;
  const int prec = cfgs[0].precision;
  for (int s = 0; s < nsim; ++s) {
    const ph_config& c = cfgs[s];
    if (c.precision != prec) return bfail(PH_ERR_INVALID, "ph_batch_create: mixed precisions");
    if (c.max_level != 0) return bfail(PH_ERR_INVALID, "ph_batch_create: members must be uniform");
    for (int f = 0; f < 6; ++f)
      if (c.bc[f] != PH_BC_PERIODIC) return bfail(PH_ERR_INVALID, "ph_batch_create: members must be periodic");
    if (c.nscalars != 0) return bfail(PH_ERR_INVALID, "ph_batch_create: members without passive scalars only");
    for (int d = 0; d < 3; ++d) {
      if (c.nx[d] < 4 || c.nb[d] < 1 || !(c.xmax[d] > c.xmin[d]))
        return bfail(PH_ERR_INVALID, "ph_batch_create: bad member geometry");
    }
    if (!(c.gamma > 1.0) || !(c.cfl > 0.0)) return bfail(PH_ERR_INVALID, "ph_batch_create: gamma/cfl");
  }
  if (prec != PH_FP64 && prec != PH_FP32) return bfail(PH_ERR_INVALID, "ph_batch_create: precision");
  ph_batch* b = new ph_batch();
  b->nsim = nsim;
  b->precision = prec;
  b->esize = prec == PH_FP32 ? 4 : 8;
  b->stream = (cudaStream_t)stream;
  {
    const char* g = std::getenv("PH_GHOSTS");
    b->push = !(g && std::strcmp(g, "launch") == 0);
  }
  b->cfg.assign(cfgs, cfgs + nsim);
  std::vector<int> leaf_member, nbr;
  long long off = 0;
  for (int s = 0; s < nsim; ++s) {
    const ph_config& c = cfgs[s];
    Member M;
    std::memset(&M, 0, sizeof(M));
    M.off = off;
    for (int d = 0; d < 3; ++d) {
      M.nx[d] = c.nx[d];
      M.S[d] = c.nx[d] + 2 * ph::NG;
      M.nb[d] = c.nb[d];
      M.idx[d] = (double)((int64_t)c.nb[d] * c.nx[d]) / (c.xmax[d] - c.xmin[d]);
    }
    M.nleaf = c.nb[0] * c.nb[1] * c.nb[2];
    M.leaf0 = b->nleaf;
    M.cfl = c.cfl;
    M.gamma = c.gamma;
    M.dfloor = c.dfloor;
    M.pfloor = c.pfloor;
    // Z-order of the member's root grid (single level): the leaf order of ph_mesh
    std::vector<std::pair<uint64_t, std::array<int, 3>>> lv;
    for (int k = 0; k < c.nb[2]; ++k)
      for (int j = 0; j < c.nb[1]; ++j)
        for (int i = 0; i < c.nb[0]; ++i) {
          uint64_t key = 0;
          const int loc[3] = {i, j, k};
          for (int d = 0; d < 3; ++d)
            for (int bb = 0; bb < 21; ++bb) key |= ((uint64_t)((loc[d] >> bb) & 1)) << (3 * bb + d);
          lv.push_back({key, {i, j, k}});
        }
    std::stable_sort(lv.begin(), lv.end(),
                     [](const std::pair<uint64_t, std::array<int, 3>>& x,
                        const std::pair<uint64_t, std::array<int, 3>>& y) { return x.first < y.first; });
    std::vector<int> slot_of((size_t)M.nleaf);
    for (int l = 0; l < M.nleaf; ++l) {
      const auto& p = lv[l].second;
      slot_of[(p[2] * c.nb[1] + p[1]) * c.nb[0] + p[0]] = l;
    }
    for (int l = 0; l < M.nleaf; ++l) {
      const auto& p = lv[l].second;
      leaf_member.push_back(s);
      for (int oz = -1; oz <= 1; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
          for (int ox = -1; ox <= 1; ++ox) {
            const int a = (p[0] + ox + c.nb[0]) % c.nb[0];
            const int bq = (p[1] + oy + c.nb[1]) % c.nb[1];
            const int cq = (p[2] + oz + c.nb[2]) % c.nb[2];
            nbr.push_back(slot_of[(cq * c.nb[1] + bq) * c.nb[0] + a]);
          }
    }
    b->nleaf += M.nleaf;
    off += (long long)M.nleaf * 5 * M.S[0] * M.S[1] * M.S[2];
    b->mem.push_back(M);
  }
  b->pool_elems = off;
  int rc = PH_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) rc = bfail(PH_ERR_CUDA, cudaGetErrorString(e));
  if (!rc) {
    b->U0 = b->dalloc(b->esize * (size_t)off);
    b->U1 = b->dalloc(b->esize * (size_t)off);
    b->d_mem = (Member*)b->dalloc(sizeof(Member) * nsim);
    b->d_leaf_member = (int*)b->dalloc(sizeof(int) * leaf_member.size());
    b->d_nbr = (int*)b->dalloc(sizeof(int) * nbr.size());
    b->d_sc = (DevScalars*)b->dalloc(sizeof(DevScalars) * nsim);
    b->d_bar = (GridBar*)b->dalloc(sizeof(GridBar));
    b->d_tmaps = (CUtensorMap*)b->dalloc(sizeof(CUtensorMap) * 2 * (size_t)nsim);  // 256-B aligned
    if (!b->U0 || !b->U1 || !b->d_mem || !b->d_leaf_member || !b->d_nbr || !b->d_sc || !b->d_bar ||
        !b->d_tmaps)
      rc = bfail(PH_ERR_OOM, "device allocation failed (batch)");
  }
  if (!rc) {
    e = cudaMemsetAsync(b->U0, 0, b->esize * (size_t)off, b->stream);
    if (!e) e = cudaMemsetAsync(b->U1, 0, b->esize * (size_t)off, b->stream);
    if (!e) e = cudaMemsetAsync(b->d_sc, 0, sizeof(DevScalars) * nsim, b->stream);
    if (!e) e = cudaMemsetAsync(b->d_bar, 0, sizeof(GridBar), b->stream);
    if (!e) e = cudaMemcpyAsync(b->d_leaf_member, leaf_member.data(), sizeof(int) * leaf_member.size(),
                                cudaMemcpyHostToDevice, b->stream);
    if (!e) e = cudaMemcpyAsync(b->d_nbr, nbr.data(), sizeof(int) * nbr.size(),
                                cudaMemcpyHostToDevice, b->stream);
    if (e) rc = bfail(PH_ERR_CUDA, cudaGetErrorString(e));
  }
  if (!rc) {
    // FP32: the widest paired tile every member's blocks tile into; else the
    // one-cell 16 x 16 (FP64, or FP32 without TMA), 16 x 8 or 8 x 8 tile
    int minn = 1 << 30;
    for (const Member& M : b->mem) minn = std::min(minn, std::min(M.nx[0], M.nx[1]));
    int TX = minn >= 16 ? 16 : 8, TY = minn >= 16 ? 16 : 8;
    if (pair_possible(b, 32)) {
      TX = 32;
    } else if (!pair_possible(b, 16) && TY == 16 && pair_choice(b, 16, 16)) {
      TY = 8;  // FP32 with TMA: 16 x 16 is paired, and these blocks do not tile into it
    }
    rc = configure(b, TX, TY, 32, 0);
  }
  if (rc) {
    ph_batch_destroy(b);
    return rc;
  }
  *out = b;
  return PH_OK;
}

int ph_batch_destroy(ph_batch* b) {
  if (!b) return PH_OK;
  cudaStreamSynchronize(b->stream);
  drop_graph(b);
  for (void* p : b->owned) cudaFree(p);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
  return PH_OK;
}

int ph_batch_num_blocks(const ph_batch* b, int32_t sim, int32_t* n) {
  if (!b || !n || sim < 0 || sim >= b->nsim) return bfail(PH_ERR_INVALID, "ph_batch_num_blocks: bad argument");
  *n = b->mem[sim].nleaf;
  return PH_OK;
}

int ph_batch_set_state(ph_batch* b, int32_t sim, const void* U, int64_t count, int32_t on_device) {
  if (!b || !U || sim < 0 || sim >= b->nsim) return bfail(PH_ERR_INVALID, "ph_batch_set_state: bad argument");
  if (count != member_count(b, sim)) return bfail(PH_ERR_INVALID, "ph_batch_set_state: count mismatch");
  return b->precision == PH_FP32 ? set_state_member<float>(b, sim, U, on_device)
                                 : set_state_member<double>(b, sim, U, on_device);
}

int ph_batch_get_state(ph_batch* b, int32_t sim, void* U, int64_t count, int32_t on_device) {
  if (!b || !U || sim < 0 || sim >= b->nsim) return bfail(PH_ERR_INVALID, "ph_batch_get_state: bad argument");
  if (count != member_count(b, sim)) return bfail(PH_ERR_INVALID, "ph_batch_get_state: count mismatch");
  return b->precision == PH_FP32 ? get_state_member<float>(b, sim, U, on_device)
                                 : get_state_member<double>(b, sim, U, on_device);
}

int ph_batch_step(ph_batch* b, int32_t ncycles) {
  PH_RANGE("ph_batch_step");
  if (!b || ncycles < 0) return bfail(PH_ERR_INVALID, "ph_batch_step: bad argument");
  if (ncycles == 0) return PH_OK;
  if (!b->gexec) {
    int rc = capture(b);
    if (rc) return rc;
  }
  for (int c = 0; c < ncycles; ++c) PB_CUDA(cudaGraphLaunch(b->gexec, b->stream));
  return PH_OK;
}

int ph_batch_get_dt(ph_batch* b, double* dt) {
  if (!b || !dt) return bfail(PH_ERR_INVALID, "ph_batch_get_dt: null argument");
  std::vector<DevScalars> hs(b->nsim);
  PB_CUDA(cudaMemcpyAsync(hs.data(), b->d_sc, sizeof(DevScalars) * b->nsim, cudaMemcpyDeviceToHost,
                          b->stream));
  PB_CUDA(cudaStreamSynchronize(b->stream));
  for (int s = 0; s < b->nsim; ++s) dt[s] = hs[s].dt_last;
  return check_error_word(b);
}

int ph_batch_get_time(ph_batch* b, double* time, int64_t* cycle) {
  if (!b) return bfail(PH_ERR_INVALID, "ph_batch_get_time: null batch");
  std::vector<DevScalars> hs(b->nsim);
  PB_CUDA(cudaMemcpyAsync(hs.data(), b->d_sc, sizeof(DevScalars) * b->nsim, cudaMemcpyDeviceToHost,
                          b->stream));
  PB_CUDA(cudaStreamSynchronize(b->stream));
  for (int s = 0; s < b->nsim; ++s) {
    if (time) time[s] = hs[s].time;
    if (cycle) cycle[s] = hs[s].cycle;
  }
  return check_error_word(b);
}

int ph_batch_status(ph_batch* b, int64_t* floor_hits, int32_t* nonfinite) {
  if (!b) return bfail(PH_ERR_INVALID, "ph_batch_status: null batch");
  std::vector<DevScalars> hs(b->nsim);
  PB_CUDA(cudaMemcpyAsync(hs.data(), b->d_sc, sizeof(DevScalars) * b->nsim, cudaMemcpyDeviceToHost,
                          b->stream));
  PB_CUDA(cudaStreamSynchronize(b->stream));
  long long fh = 0;
  int nf = 0;
  for (int s = 0; s < b->nsim; ++s) {
    fh += (long long)hs[s].floor_hits;
    nf |= hs[s].nonfinite;
  }
  if (floor_hits) *floor_hits = fh;
  if (nonfinite) *nonfinite = nf;
  int rc = check_error_word(b);
  if (rc) return rc;
  if (fh || nf) return bfail(PH_ERR_NONPHYSICAL, "floors applied or non-finite dt");
  return PH_OK;
}

int ph_batch_get_launch(const ph_batch* b, int32_t choice[4]) {
  if (!b || !choice) return bfail(PH_ERR_INVALID, "ph_batch_get_launch: null argument");
  choice[0] = b->TX;
  choice[1] = b->TY;
  choice[2] = b->KC;
  choice[3] = b->ctas_per_sm;
  return PH_OK;
}

int ph_batch_set_launch(ph_batch* b, const int32_t choice[4]) {
  if (!b || !choice) return bfail(PH_ERR_INVALID, "ph_batch_set_launch: null argument");
  if (!(ph::stage_tile_supported(choice[0], choice[1]) || pair_choice(b, choice[0], choice[1])) ||
      choice[2] < 1)
    return bfail(PH_ERR_INVALID, "ph_batch_set_launch: unsupported tile");
  return configure(b, choice[0], choice[1], choice[2], choice[3]);
}

// Autotuner: time `trial_cycles` cycles of every candidate (tile shape, chunk
// depth, CTAs per SM) on the current state, keep the fastest, restore the
// state and clocks of the simulation.  chosen[4] receives the choice.
int ph_batch_autotune(ph_batch* b, int32_t trial_cycles, int32_t chosen[4]) {
  if (!b || trial_cycles < 1) return bfail(PH_ERR_INVALID, "ph_batch_autotune: bad argument");
  int minn = 1 << 30;
  for (const Member& M : b->mem) minn = std::min(minn, std::min(M.nx[0], M.nx[1]));
  const size_t bytes = b->esize * (size_t)b->pool_elems;
  void* save = nullptr;
  PB_CUDA(cudaMalloc(&save, bytes));
  std::vector<DevScalars> hs(b->nsim);
  cudaError_t e = cudaMemcpyAsync(save, b->U0, bytes, cudaMemcpyDeviceToDevice, b->stream);
  if (!e) e = cudaMemcpyAsync(hs.data(), b->d_sc, sizeof(DevScalars) * b->nsim, cudaMemcpyDeviceToHost,
                              b->stream);
  if (!e) e = cudaStreamSynchronize(b->stream);
  if (e) {
    cudaFree(save);
    return bfail(PH_ERR_CUDA, cudaGetErrorString(e));
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int bc[4] = {b->TX, b->TY, b->KC, b->ctas_per_sm};
  int rc = PH_OK;
  for (int t = 0; t < 5 && !rc; ++t) {
    const int TX = kTiles[t][0], TY = kTiles[t][1];
    const bool pair = pair_choice(b, TX, TY);
    if (pair ? !pair_possible(b, TX) : (t == 4 || TX > 2 * minn || TY > minn)) continue;
    int per_sm = 0;
    // an upper bound for the CTA count; configure() clamps to the variant it picks
    rc = b->precision == PH_FP32 ? (pair ? occupancy_t<float, true>(TX, TY, &per_sm)
                                         : occupancy_t<float, false>(TX, TY, &per_sm))
                                 : occupancy_t<double, false>(TX, TY, &per_sm);
    if (rc) break;
    const int kcs[3] = {8, 16, 32};
    for (int kci = 0; kci < 3 && !rc; ++kci) {
      for (int ctas = 1; ctas <= per_sm && !rc; ++ctas) {
        rc = configure(b, TX, TY, kcs[kci], ctas);
        if (rc) break;
        e = launch_one(b, b->stream);  // warm-up
        if (!e) e = cudaEventRecord(e0, b->stream);
        for (int c = 0; c < trial_cycles && !e; ++c) e = launch_one(b, b->stream);
        if (!e) e = cudaEventRecord(e1, b->stream);
        if (!e) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e) {
          rc = bfail(PH_ERR_CUDA, cudaGetErrorString(e));
          break;
        }
        rc = check_error_word(b);
        if (!rc && ms < best) {
          best = ms;
          bc[0] = TX;
          bc[1] = TY;
          bc[2] = kcs[kci];
          bc[3] = ctas;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  e = cudaMemcpyAsync(b->U0, save, bytes, cudaMemcpyDeviceToDevice, b->stream);
  if (!e) e = cudaMemcpyAsync(b->d_sc, hs.data(), sizeof(DevScalars) * b->nsim, cudaMemcpyHostToDevice,
                              b->stream);
  if (!e) e = cudaStreamSynchronize(b->stream);
  cudaFree(save);
  if (rc) return rc;
  if (e) return bfail(PH_ERR_CUDA, cudaGetErrorString(e));
  rc = configure(b, bc[0], bc[1], bc[2], bc[3]);
  if (rc) return rc;
  if (chosen)
    for (int i = 0; i < 4; ++i) chosen[i] = bc[i];
  return PH_OK;
}

// Failure-detection self test: a cooperative launch of `nctas` CTAs whose
// barrier waits for one CTA more than exist; every CTA must give up after
// spin_limit polls.  *gave_up receives the number of CTAs that reported it.
int ph_debug_barrier_timeout(void* stream, int32_t nctas, int64_t spin_limit, int32_t* gave_up) {
  if (!gave_up || nctas < 1 || nctas > 64 || spin_limit < 0 || spin_limit > (1ll << 26))
    return bfail(PH_ERR_INVALID, "ph_debug_barrier_timeout: bad argument");
  GridBar* bar = nullptr;
  int* out = nullptr;
  PB_CUDA(cudaMalloc(&bar, sizeof(GridBar)));
  cudaError_t e = cudaMalloc(&out, sizeof(int));
  cudaStream_t s = (cudaStream_t)stream;
  if (!e) e = cudaMemsetAsync(bar, 0, sizeof(GridBar), s);
  if (!e) e = cudaMemsetAsync(out, 0, sizeof(int), s);
  if (!e) {
    ph::barrier_timeout_kernel<<<nctas, 32, 0, s>>>(bar, (unsigned long long)spin_limit, out);
    e = cudaGetLastError();
  }
  int h = 0;
  if (!e) e = cudaMemcpyAsync(&h, out, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (!e) e = cudaStreamSynchronize(s);
  cudaFree(bar);
  cudaFree(out);
  if (e) return bfail(PH_ERR_CUDA, cudaGetErrorString(e));
  *gave_up = h;
  return h ? PH_ERR_TIMEOUT : PH_OK;
}

}  // extern "C"
