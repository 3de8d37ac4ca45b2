// ph_internal.h -- host-side declarations shared by the library's translation
// units (not part of the public ABI).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <string>
#include <vector>

#include "../../include/ph_hydro.h"

#include "ph_device.cuh"

struct ph_mesh;

namespace ph {

// What the adjoint needs of a uniform mesh (filled by ph_api.cu).
struct MeshAccess {
  void* U0;
  void* U1;
  const int* nbr;
  DevScalars* sc;
  cudaStream_t stream;
  int nx[3];
  int nleaf;
  size_t block_elems;
  int precision;
  double gamma, dfloor, pfloor;
  double idx[3];
};
int mesh_access(ph_mesh* m, MeshAccess* out);
int mesh_set_state(ph_mesh* m, const void* U, int on_device);
int mesh_cycle_fixed_dt(ph_mesh* m, double dt);   // one cycle with a prescribed dt
int mesh_cycle_read_dt(ph_mesh* m, double* dt);   // one CFL cycle, returns its dt
// Stream-ordered forms without host synchronisation: one cycle with the dt
// at device address d_dt; one CFL cycle whose dt is stored at d_dt.
int mesh_cycle_device_dt(ph_mesh* m, const double* d_dt);
int mesh_cycle_record_dt(ph_mesh* m, double* d_dt);
// Device memory from the mesh's allocator (NULL on failure); mesh_free
// returns it (stream-ordered on the mesh's stream, as the allocator is).
void* mesh_alloc(ph_mesh* m, size_t bytes);
void mesh_free(ph_mesh* m, void* p);


// Record the message that ph_last_error() returns on this thread.
void set_error_message(const char* msg);

// Cell geometry per level: 1/dx per direction and the cell volume.
struct LevelGeom {
  double idx[MAXLEV + 1][3];
  double vol[MAXLEV + 1];
};

// Octree node table of a mesh (Sec. 2.1: an oct-tree of blocks in which one
// leaf covers each location).  Entries 0 .. nroot-1 are the root-grid slots
// (x1 fastest); an entry >= 0 is the index of the leaf at that node, and an
// entry v <= -2 marks a refined node whose 8 children are the entries
// (-2 - v) + c, c = c1 + 2 c2 + 4 c3.
constexpr int NODE_UNSET = -1;
__host__ __device__ inline int node_children(int v) { return -2 - v; }

// Device view of the tree, used by the ghost exchange and remesh kernels to
// evaluate the composite field anywhere.
struct TreeView {
  const int* node;
  int nb[3];
  int nx[3];
  int S[3];
  int bc[6];        // physical boundary per face (PH_BC_*)
  int* error;       // set if an evaluation needs more nesting than supported
};

template <class T>
struct StageArgs;

// K3: fused stage over all leaves.  Returns the launch error.
// tmap: tensor map of the stencil input pool (TMA plane staging), or null
// for plain loads.
template <class T>
cudaError_t launch_stage(const StageArgs<T>& a, int TX, int TY, cudaStream_t s,
                         const CUtensorMap* tmap = nullptr);
bool make_stage_tmap(CUtensorMap* out, const void* base, size_t esize, const int S[3], int nleaf, int TX,
                     int TY, int nvar = NV);
bool stage_tma_wanted();  // false when PH_STAGE_LOADS=plain
template <class T>
size_t stage_smem_bytes(int TX, int TY);
bool stage_tile_supported(int TX, int TY);
// 32 x 16: the paired FP32 kernel (FP32 uniform meshes with TMA staging,
// nx1 a multiple of 32 and nx2 of 16), the only kernel of that tile
bool stage_pair_tile(int TX, int TY);
// Whether a mesh's stages run the paired FP32 kernel: FP32, TMA staging,
// hydro variables only, one level, and tiles 32 x 16 or 16 x 16 that divide
// the block (16 x 16 tiles of other meshes run the one-cell kernel).
bool stage_pair_kernel(bool fp32, bool tma, int nvar, bool multi_level, const int tile[3], const int nx[3]);
// Resident CTAs per SM of the stage kernel for a tile (0 if unknown); the
// stage kernels' shared-memory attributes must be set (configure_stage_kernels).
template <class T>
int stage_ctas_per_sm(int TX, int TY, int nvar, bool pair, bool tma);
// tiles that meshes with passive scalars can use
bool stage_scalar_tile(int TX, int TY);
cudaError_t configure_stage_kernels();

// K1 (uniform mesh): every ghost cell of every leaf copied from the
// same-level neighbour given by nbr[27 * leaf + region] (-1: a neighbour on
// another shard, whose cells the shard unpack writes), or, across a
// physical boundary face (bcm: 2 bits per face, x1 inner first; leaf_id and
// nb give the leaf's place in the root grid), from its image in the block.
template <class T>
cudaError_t launch_ghost_uniform(T* U, const int* nbr, const int nx[3], int nleaf, cudaStream_t s,
                                 const int* leaf_id = nullptr, const int nb[3] = nullptr,
                                 int bcm = 0, int nvar = NV);

// K1 (multi-level mesh): every ghost cell of every leaf takes the composite
// field of the mesh (copy / restriction / prolongation).
// nbr[27 * leaf + region]: the same-level leaf covering that neighbour
// region (its ghost cells are copied directly, one CTA per leaf), or -1;
// the cells of regions with -1 are eval[0 .. neval) = (leaf, shell index),
// evaluated in a second launch, one thread per cell, from recipe[0 .. neval)
// (launch_ghost_recipes: source offsets resolved once per tree).
template <class T>
cudaError_t launch_ghost_composite(T* U, const TreeView& tv, const int* leaf_id, const int* nbr,
                                   int nleaf, const int2* eval, const void* recipe, int neval, cudaStream_t s,
                                   int nvar = NV);
// Resolve the evaluation list of a tree into recipes (ghost_recipe_bytes()
// each): for cells that are one prolongation, restriction or copy of cells in
// leaves of their own level, the source offsets and sign flips.
size_t ghost_recipe_bytes();
cudaError_t launch_ghost_recipes(const TreeView& tv, const int* leaf_id, const int2* eval, int neval,
                                 void* out, cudaStream_t s, int nvar);

// K7: interior of every new leaf from the old mesh's composite field.
template <class T>
cudaError_t launch_remesh(T* Unew, const int* new_leaf_id, int nnew, const T* Uold,
                          const TreeView& old_tv, cudaStream_t s, int nvar = NV);

// K5: max over interior cells of (|v_d|+c)/dx_d into sc->wmax_bits.
template <class T>
cudaError_t launch_rate(const T* U, const int8_t* level, const LevelGeom& g, const int nx[3],
                        int nleaf, Phys<T> P, DevScalars* sc, cudaStream_t s, int nvar = NV);

// dt bookkeeping: mode bit 1 commits the cycle (time += dt, cycle++),
// bit 2 computes the next dt = cfl / wmax and clears wmax, bit 4 copies the
// next dt into the last (a fresh state).
cudaError_t launch_advance(DevScalars* sc, double cfl, int mode, cudaStream_t s);

// Interior <-> padded copies.  dir 0: packed -> padded, 1: padded -> packed.
template <class T>
cudaError_t launch_pack(T* padded, T* packed, const int nx[3], int nleaf, int dir, cudaStream_t s,
                        int nvar = NV);

// Conserved totals: per-leaf FP64 sums into partial[nleaf*5], then one
// ordered compensated sum into out[5].
template <class T>
cudaError_t launch_totals(const T* U, const int8_t* level, const LevelGeom& g, const int nx[3],
                          int nleaf, double* partial, double* out, cudaStream_t s, int nvar = NV);

// K6: refinement indicator per leaf (FP64).
template <class T>
cudaError_t launch_indicator(const T* U, const int nx[3], int nleaf, double* mb, cudaStream_t s,
                             int nvar = NV);

// K4: flux correction at fine-coarse faces, applied after the stage update.
// One CTA per coarse leaf corr_leaf[c] with records rec_beg[c] .. rec_beg[c+1].
// want_rate (stage 2): also fold the signal rate of every corrected cell
// into sc->wmax_bits (the stage skips those cells).
template <class T>
cudaError_t launch_flux_correct(T* U, const int* corr_leaf, const int* rec_beg, int ncorr,
                                const int* rec_face, const T* fc_coarse, const T* fc_fine,
                                const int nx[3], const int8_t* level, const LevelGeom& g,
                                double beta, DevScalars* sc, cudaStream_t s, int nvar, Phys<T> P,
                                int want_rate);

// Domain decomposition of a uniform mesh (ph_shard.cu).  Shard `shard` of
// `nshards` owns the global leaves [lo, hi) of the Z-ordered root grid; the
// halo plan lists, per peer (peers in order, offsets in *_off), the ghost
// cells it receives (destination: local leaf * padded cells + cell, flips of
// the normal momentum across reflecting walls) and the interior cells it
// sends (source: local leaf * padded cells + cell), both in the order of
// the receiving ghost cell's (global leaf, padded cell) key.  Local
// positions are element offsets into the state pool (local leaf times
// nvar x padded cells, plus the padded cell); variable v is v x padded cells
// further.
struct ShardPlan {
  int nshards = 1, shard = 0;
  long long lo = 0, hi = 0;
  std::vector<long long> first;            // per shard, its first global leaf (size nshards + 1)
  std::vector<int> owner;                  // per global leaf
  std::vector<std::array<int, 3>> loc;     // per global leaf, root-grid location
  std::vector<int64_t> send_off, recv_off; // per peer, entry offsets (size nshards + 1)
  std::vector<int64_t> send_key, send_src;
  std::vector<int64_t> recv_key, recv_dst;
  std::vector<int8_t> recv_flip;
};
int shard_plan(const ph_config& cfg, int nshards, int shard, ShardPlan* out, std::string* err);
template <class T>
cudaError_t launch_shard_pack(const T* U, const long long* src, long long n, long long vs, int nvar, T* buf,
                              cudaStream_t s);
template <class T>
cudaError_t launch_shard_unpack(T* U, const long long* dst, const int8_t* flip, long long n, long long vs,
                                int nvar, const T* buf, cudaStream_t s);
cudaError_t launch_shard_wmax(const unsigned long long* src, int n, unsigned long long* dst, cudaStream_t s);

}  // namespace ph
