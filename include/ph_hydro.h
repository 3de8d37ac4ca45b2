/* ph_hydro.h -- C ABI of the GB300 Parthenon-hydro hot path (libphhydro.so).
 *
 * The library advances the 3-D Euler equations of an ideal gas on a mesh of
 * equal-sized MeshBlocks with ghost zones, one GPU, all work in hand-written
 * CUDA kernels for sm_103a (arXiv:2202.12309; the method is that of its
 * Parthenon-hydro miniapp, Sec. 4.1: two-stage Runge-Kutta, piecewise-linear
 * reconstruction, HLLE Riemann solver; the mesh and its boundary
 * communication are Sec. 2.1, 3.6 and 3.7; the time step is a global
 * min-reduction, Sec. 3.10; the call sequence follows the driver pattern of
 * Sec. 3.11: create a mesh, refine, set the state, step, read state and dt).
 *
 * Conventions for every entry point:
 *  - Return value: PH_OK (0) or a negative PH_ERR_* code.  The message of the
 *    last failure on the calling thread is ph_last_error().  No C++ exception
 *    crosses this ABI.
 *  - Work is enqueued on the stream given at creation; calls that return data
 *    to host memory synchronise that stream.  ph_step does not synchronise
 *    (except on multi-level meshes, where it reads refinement flags each cycle).
 *  - Caller buffers are borrowed for the duration of the call only.
 *  - State arrays are in the mesh's precision (double for PH_FP64, float for
 *    PH_FP32), conserved variables (rho, m1, m2, m3, E, then any passive
 *    scalars rho r_s), interior cells only,
 *    layout U[block][var][k][j][i] with i fastest, blocks in the order of
 *    ph_tree (Z-order).
 *  - Device memory of a mesh is owned by the library and comes from the
 *    allocator installed with ph_set_allocator (cudaMalloc by default).
 */
#ifndef PH_HYDRO_H
#define PH_HYDRO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PH_OK 0
#define PH_ERR_INVALID (-1)     /* bad argument or configuration */
#define PH_ERR_OOM (-2)         /* device allocation failed */
#define PH_ERR_NONPHYSICAL (-3) /* non-finite state or density/pressure floor hit */
#define PH_ERR_TIMEOUT (-4)     /* a bounded device-side wait gave up */
#define PH_ERR_CUDA (-5)        /* a CUDA runtime call failed */
#define PH_ERR_STATE (-6)       /* call not valid in the object's current state */
#define PH_ERR_IO (-7)          /* a file could not be opened, read or written */

#define PH_FP64 0
#define PH_FP32 1

/* Mesh configuration (Sec. 2.1: equal-sized blocks, an integer number of
 * blocks per dimension; Sec. 4.1: ideal gas).  All fields are read once by
 * ph_create.
 *   nx[3]          interior cells per block along x1, x2, x3 (each >= 4)
 *   nb[3]          root-grid blocks along x1, x2, x3 (each >= 1)
 *   xmin/xmax      domain extent; boundaries as in bc[] (periodic by default)
 *   max_level      0 (uniform) .. 4: finest level of the block tree; blocks
 *                  that touch (face, edge or corner) differ by one level at
 *                  most (a refinement splits coarser touching blocks first;
 *                  siblings do not merge next to blocks two levels finer)
 *   adaptive       1: tag and remesh after every cycle (max_level >= 1)
 *   gamma          adiabatic index; cfl: Courant number
 *   dfloor/pfloor  density and pressure floors applied when converting to
 *                  primitive variables (every application is counted)
 *   refine_tol     refine a block below max_level whose indicator exceeds it
 *   derefine_tol   merge 8 sibling blocks whose indicators are all below it
 *   derefine_count siblings must be at least this many cycles old to merge
 *   static_region  1: level-0 blocks overlapping the open box
 *                  (static_lo, static_hi) are refined at creation and pinned
 *   precision      PH_FP64 or PH_FP32 (state and fluxes; dt and totals stay FP64)
 *   tile[3]        fused-stage tile (TX, TY, KC); 0,0,0 = pick a default
 *                  (KC then follows the leaf count).  TX x TY: 8x8, 16x8,
 *                  16x16, 32x8, and for FP32 uniform meshes 32x16; on FP32
 *                  uniform meshes with TMA staging and no passive scalars
 *                  whose blocks tile into them, 32x16 and 16x16 run the
 *                  paired kernel (two cells per thread; both widths give the
 *                  same bits), other tiles the one-cell kernel
 *   bc[6]          physical boundary of each face (PH_BC_*, below); all zero
 *                  = periodic everywhere
 *   nscalars       passive scalars, 0 .. 2 (Sec. 3.4: the hydro package
 *                  advects every variable flagged as advected): conserved
 *                  rho r_s stored after the energy (state arrays then hold
 *                  5 + nscalars variables per cell); the concentration r_s
 *                  is reconstructed like the primitives and its flux is the
 *                  HLLE formula with the hydro wave speeds.  Tiles 16x16 or
 *                  8x8; not with ph_batch_* or ph_adjoint.
 *   pad            unused
 */
typedef struct ph_config {
  int32_t nx[3];
  int32_t nb[3];
  double xmin[3];
  double xmax[3];
  int32_t max_level;
  int32_t adaptive;
  double gamma;
  double cfl;
  double dfloor;
  double pfloor;
  double refine_tol;
  double derefine_tol;
  int32_t derefine_count;
  int32_t static_region;
  double static_lo[3];
  double static_hi[3];
  int32_t precision;
  int32_t tile[3];
  int32_t bc[6];
  int32_t nscalars;
  int32_t pad;
} ph_config;

/* Physical boundary conditions, per face in ph_config.bc (x1 inner, x1 outer,
 * x2 inner, x2 outer, x3 inner, x3 outer).  A ghost location outside the
 * domain takes the value of its image inside, at the same level:
 *   PH_BC_PERIODIC  shifted by the domain length (both faces of an axis
 *                   periodic or neither);
 *   PH_BC_OUTFLOW   the nearest interior cell (zero-gradient copy);
 *   PH_BC_REFLECT   mirrored about the face (ghost layer g takes interior
 *                   layer g) with the momentum component normal to the face
 *                   negated (the paper's reflective boundaries, Sec. 3.4).
 * Batched meshes and the adjoint are periodic only. */
#define PH_BC_PERIODIC 0
#define PH_BC_OUTFLOW 1
#define PH_BC_REFLECT 2

typedef struct ph_mesh ph_mesh;

/* Device allocator hook: alloc(bytes, stream, ctx) returns a device pointer
 * or NULL; release(ptr, stream, ctx) returns it.  Installed process-wide;
 * NULL, NULL restores cudaMalloc/cudaFree.  Meshes created before the call
 * keep the allocator they were created with. */
typedef void* (*ph_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*ph_free_fn)(void* ptr, void* stream, void* ctx);
int ph_set_allocator(ph_alloc_fn alloc, ph_free_fn release, void* ctx);

/* Message of the last failure on this thread ("" if none). */
const char* ph_last_error(void);

/* Create a mesh (Sec. 2.1): root grid, oct-tree, Z-order, static refinement
 * (Sec. 3.8).  `stream` is a cudaStream_t (NULL = legacy default stream).
 * The state is zero until ph_set_state.  *out receives the handle.
 * Errors: PH_ERR_INVALID (nx < 4, nb < 1, bad level/precision/tile/bc),
 * PH_ERR_OOM, PH_ERR_CUDA. */
int ph_create(const ph_config* cfg, void* stream, ph_mesh** out);

/* Release the mesh and its device memory (synchronises its stream). */
int ph_destroy(ph_mesh* mesh);

/* Number of leaf blocks. */
int ph_num_blocks(const ph_mesh* mesh, int32_t* n);

/* Leaves in Z-order (Sec. 2.1), 4 int64 per leaf: level, lx1, lx2, lx3.
 * `n` is the capacity in leaves; PH_ERR_INVALID if smaller than the count. */
int ph_tree(const ph_mesh* mesh, int64_t* out, int32_t n);

/* Copy the interior state in (count = blocks*5*nx1*nx2*nx3 elements) and
 * fill ghosts; computes the first dt.  on_device: 1 if U is a device pointer,
 * 0 for host memory.  PH_ERR_INVALID if count does not match. */
int ph_set_state(ph_mesh* mesh, const void* U, int64_t count, int32_t on_device);

/* Copy the interior state out (same layout and count rule). */
int ph_get_state(ph_mesh* mesh, void* U, int64_t count, int32_t on_device);

/* Stream-ordered forms of ph_set_state / ph_get_state: the copies, ghost
 * fill and first dt are queued on the mesh's stream and the call returns
 * without waiting for them, so that transfers of one mesh overlap the cycles
 * of another on another stream.  A host buffer must stay valid and unchanged
 * (set) or unread (get) until the stream has passed the copy; page-locked
 * host memory is needed for the copy to overlap anything (a pageable source
 * or destination makes the driver copy synchronously).  Errors as the
 * synchronous forms; ph_get_state_async also PH_ERR_STATE before a state was
 * set. */
int ph_set_state_async(ph_mesh* mesh, const void* U, int64_t count, int32_t on_device);
int ph_get_state_async(ph_mesh* mesh, void* U, int64_t count, int32_t on_device);

/* Copy whole blocks out, ghosts included: layout U[block][var][k][j][i] over
 * (nx+4)^3 cells (count = blocks*5*(nx1+4)*(nx2+4)*(nx3+4)). */
int ph_get_full(ph_mesh* mesh, void* U, int64_t count, int32_t on_device);

/* Advance `ncycles` cycles (Sec. 3.11 MultiStageDriver): per cycle, two RK
 * stages each followed by the ghost exchange (Sec. 3.7) and, on multi-level
 * meshes, flux correction; then dt for the next cycle (Sec. 3.10) and, when
 * adaptive, tagging and remesh (Sec. 3.8).  Uniform meshes replay a captured
 * CUDA graph of one cycle and return without synchronising. */
int ph_step(ph_mesh* mesh, int32_t ncycles);

/* dt used by the last cycle (the first dt before any cycle); synchronises. */
int ph_get_dt(ph_mesh* mesh, double* dt);
/* dt the next cycle will use; synchronises. */
int ph_get_next_dt(ph_mesh* mesh, double* dt);

/* Simulation time and cycle count; synchronises. */
int ph_get_time(ph_mesh* mesh, double* time, int64_t* cycle);

/* Conserved totals: sum over interior cells of all leaves of U_v dV, in FP64;
 * out receives 5 + nscalars values. */
int ph_totals(ph_mesh* mesh, double* out);

/* Refinement indicator of every leaf (reading of the unspecified criterion:
 * max over interior cells and directions of |rho_{+1} - rho_{-1}| / (2 rho))
 * and the flags it implies (+1 refine, -1 derefine, 0 keep) under the
 * configured tolerances.  Arrays of n entries (n >= ph_num_blocks). */
int ph_tag(ph_mesh* mesh, int8_t* flags, double* indicator, int32_t n);

/* Rebuild the tree from explicit flags (+1 refine a level-0 leaf, -1 merge
 * 8 level-1 siblings that are all -1, 0 keep; Sec. 2.1/3.8) and move the data
 * (prolongation for new children, restriction for merged parents).
 * check_age: also require derefine_count cycles of age to merge.
 * *changed (may be NULL) is set to 1 if the tree changed. */
int ph_refine_where(ph_mesh* mesh, const int8_t* flags, int32_t n, int32_t check_age,
                    int32_t* changed);

/* One tag + remesh pass on the current state (initial refinement). */
int ph_refine_by_density(ph_mesh* mesh, int32_t* changed);

/* Health of the state since creation: number of floor applications and 1 if
 * a non-finite dt was produced.  The dt comes from the max signal rate over
 * every interior cell (after a state is set or loaded, after a remesh and
 * after each cycle's stage 2); a NaN rate in any cell wins that max, so one
 * non-finite cell makes the dt non-finite.  Returns PH_ERR_NONPHYSICAL when
 * either is non-zero (outputs are still written). */
int ph_status(ph_mesh* mesh, int64_t* floor_hits, int32_t* nonfinite);

/* Kernel-level entry points used by tests and benchmarks ------------------ */

/* Ghost exchange alone on the current state (Sec. 3.7). */
int ph_fill_ghosts(ph_mesh* mesh);

/* Number of kernel launches one uniform-mesh cycle enqueues: 3 on periodic
 * meshes (the stages write the ghost zones of their output themselves), 5
 * with physical boundaries or with the environment variable PH_GHOSTS=launch
 * at ph_create (a separate exchange launch after each stage). */
int ph_launches_per_cycle(const ph_mesh* mesh, int32_t* n);

/* Fused-stage tile in use (TX, TY, KC). */
int ph_get_tile(const ph_mesh* mesh, int32_t tile[3]);

/* Run `ncycles` uniform-mesh cycles with the same launches as ph_step but
 * without the graph, recording a CUDA event on the mesh's stream between
 * launches; ms_out[s] (s < nslots, nslots <= 5) receives the summed device
 * time of launch slot s of the cycle: 0 stage 1, 1 ghost exchange, 2 stage 2,
 * 3 ghost exchange, 4 dt bookkeeping (slots 1 and 3 are empty, about zero,
 * where the stages write the ghost zones themselves).  Synchronises.  Uniform meshes only
 * (PH_ERR_INVALID otherwise). */
int ph_profile_cycles(ph_mesh* mesh, int32_t ncycles, double* ms_out, int32_t nslots);

/* Advance a uniform mesh by ncycles with a prescribed dt per cycle (host
 * array dts[ncycles]) instead of the CFL dt; synchronises every cycle. */
int ph_step_dt(ph_mesh* mesh, int32_t ncycles, const double* dts);

/* Gradient of a loss of the final state with respect to the initial
 * conserved state and the adiabatic index (uniform meshes).  The paper has
 * no adjoint; this is the reverse of the cycle described above (Sec. 4.1),
 * with the dt schedule held fixed and the limiter / wave-speed / floor
 * branches frozen at their forward values.
 *   U0       initial interior state (layout of ph_set_state)
 *   ncycles  cycles of the forward run; ckpt_every: keep every k-th state
 *            and recompute the k cycles in between (memory ~ ncycles/k + 4k
 *            states: two sets of a segment's stage inputs, one read by the
 *            reverse sweep while the segment before is recomputed into the
 *            other; the last k cycles' stage inputs are kept from the
 *            forward run, so those are not recomputed)
 *   dts      host array of ncycles dts, or NULL to use (and freeze) the CFL
 *            dts of the forward run
 *   dLdU     dL/dU_final (interior layout); dLdU0 receives dL/dU0
 *   dLdgamma receives dL/dgamma (may be NULL)
 *   on_device: 1 if U0, dLdU and dLdU0 are device pointers
 * The mesh is left at the final state of the forward run.  Periodic uniform
 * meshes only (PH_ERR_INVALID otherwise). */
int ph_adjoint(ph_mesh* mesh, const void* U0, int32_t ncycles, int32_t ckpt_every,
               const double* dts, const void* dLdU, void* dLdU0, double* dLdgamma,
               int32_t on_device);

/* ---------------------------------------------------------------------------
 * Batched independent meshes (one persistent launch per cycle).
 *
 * `nsim` uniform periodic meshes (max_level 0), each with its own block size,
 * block count, state and dt, all in one precision, advanced together: one
 * cooperative kernel per cycle runs stage 1, the ghost exchange, stage 2 and
 * the ghost exchange for every block of every member (a work list of
 * (block, tile) items, four grid barriers with bounded spins) and updates each
 * member's dt; the cycle is captured in a CUDA graph.  This is the paper's
 * "all blocks in one kernel" (Sec. 3.6, 5.1) taken to one launch per cycle
 * across independent problems.  Member s's state uses the layout of
 * ph_get_state for its own mesh (blocks in Z-order).
 * ------------------------------------------------------------------------- */
typedef struct ph_batch ph_batch;

/* Create from nsim configurations (uniform, periodic, same precision; tile
 * ignored); PH_ERR_INVALID otherwise. */
int ph_batch_create(const ph_config* cfgs, int32_t nsim, void* stream, ph_batch** out);
int ph_batch_destroy(ph_batch* batch);
int ph_batch_num_blocks(const ph_batch* batch, int32_t sim, int32_t* n);
/* Copy member `sim`'s interior state in (fills its ghosts, computes its dt)
 * or out; count = its blocks * 5 * nx1 * nx2 * nx3. */
int ph_batch_set_state(ph_batch* batch, int32_t sim, const void* U, int64_t count,
                       int32_t on_device);
int ph_batch_get_state(ph_batch* batch, int32_t sim, void* U, int64_t count,
                       int32_t on_device);
/* Advance every member by ncycles (graph replays; does not synchronise). */
int ph_batch_step(ph_batch* batch, int32_t ncycles);
/* Per-member dt of the last cycle, time and cycle count (arrays of nsim);
 * synchronise; PH_ERR_TIMEOUT if a grid barrier gave up. */
int ph_batch_get_dt(ph_batch* batch, double* dt);
int ph_batch_get_time(ph_batch* batch, double* time, int64_t* cycle);
int ph_batch_status(ph_batch* batch, int64_t* floor_hits, int32_t* nonfinite);
/* Launch choice {TX, TY, KC, CTAs per SM}: read, set, or pick by timing
 * trial_cycles cycles of every candidate (tile 8x8/16x8/16x16/32x8, chunk
 * 8/16/32 planes, 1..max CTAs per SM) on the current state, which is restored
 * afterwards. */
int ph_batch_get_launch(const ph_batch* batch, int32_t choice[4]);
int ph_batch_set_launch(ph_batch* batch, const int32_t choice[4]);
int ph_batch_autotune(ph_batch* batch, int32_t trial_cycles, int32_t chosen[4]);

/* Failure-detection self test of the bounded grid barrier: launches nctas
 * (1..64) CTAs whose barrier can never complete; each gives up after
 * spin_limit polls (<= 2^26).  *gave_up = CTAs that reported it; returns
 * PH_ERR_TIMEOUT when any did (the expected outcome), with the GPU context
 * still usable. */
int ph_debug_barrier_timeout(void* stream, int32_t nctas, int64_t spin_limit, int32_t* gave_up);

/* ---------------------------------------------------------------------------
 * Domain decomposition (Sec. 2.1: MeshBlocks are distributed over ranks as
 * contiguous ranges of the Z-ordered block list; Sec. 3.7: ghost zones of
 * blocks whose neighbours live elsewhere are filled by packing buffers on the
 * sender, sending them and unpacking on the receiver; Sec. 3.10: dt is a
 * global min-reduction).  Uniform meshes (max_level 0), any boundaries.
 *
 * A shard is a mesh holding shard s of nshards: the global leaves
 * [s N / P, (s + 1) N / P) of the Z-ordered root grid (N blocks, P shards),
 * in that order.  Its state calls (ph_set_state, ph_get_state, ph_totals,
 * ph_tree) cover its own leaves only.  Its ghost cells whose source lies on
 * another shard come from the halo exchange: a per-cell plan, ordered by the
 * receiving cell's (global leaf, padded cell index) on both sides, so a
 * sender's slab for a peer and the peer's slab from it list the same cells
 * in the same order.  Messages hold nvar values per entry (entries x nvar
 * elements of the mesh's precision).  ph_step, ph_step_dt, ph_adjoint,
 * ph_save and ph_profile_cycles refuse shards (PH_ERR_STATE / _INVALID).
 *
 * One cycle of every shard, as ph_shards_step runs it for shards of one
 * process and as a caller with its own transport (one process per GPU)
 * writes it:
 *   ph_shard_stage(m, 1); ph_shard_pack(m, 1, send); exchange; ph_shard_unpack(m, 1, recv);
 *   ph_shard_stage(m, 2); ph_shard_pack(m, 0, send); exchange; ph_shard_unpack(m, 0, recv);
 *   ph_shard_rate(m, 0, r); r = max over shards; ph_shard_finish(m, 0, r);
 * and after ph_set_state on every shard (whose dt is then its own shard's):
 *   ph_shard_pack(m, 0, ...); exchange; ph_shard_unpack(m, 0, ...);
 *   ph_shard_rate(m, 1, r); r = max over shards; ph_shard_finish(m, 1, r).
 * Every call is stream-ordered on the shard's stream and returns without
 * waiting; buffers are device pointers.
 * ------------------------------------------------------------------------- */

/* Create shard `shard` of `nshards` (1 <= nshards <= blocks) of the uniform
 * mesh `cfg`, on `stream`.  nshards = 1 is ph_create.  Errors as ph_create;
 * PH_ERR_INVALID for max_level > 0 or a bad shard. */
int ph_create_shard(const ph_config* cfg, int32_t nshards, int32_t shard, void* stream, ph_mesh** out);

/* Halo of a shard with one peer: entries it sends to / receives from `peer`
 * and their offsets (in entries) in its send / receive buffers, which hold
 * every peer's slab in peer order; leaf_range (may be NULL) receives the
 * shard's global leaves [first, last).  Any output may be NULL. */
int ph_shard_halo(const ph_mesh* m, int32_t peer, int64_t* send_entries, int64_t* send_offset,
                  int64_t* recv_entries, int64_t* recv_offset, int64_t leaf_range[2]);

/* Stage `stage` (1 or 2) of the cycle on the shard's leaves, followed by the
 * ghost cells whose sources are its own leaves (and physical boundaries). */
int ph_shard_stage(ph_mesh* m, int32_t stage);

/* One launch packing every outgoing halo value of pool (0: the state U0,
 * after stage 2 or ph_set_state; 1: the stage-1 result) into sendbuf; one
 * launch unpacking every incoming value from recvbuf into that pool's ghost
 * cells (the normal momentum negated where the image crossed a reflecting
 * wall).  Buffers: device, layout of ph_shard_halo. */
int ph_shard_pack(ph_mesh* m, int32_t pool, void* sendbuf);
int ph_shard_unpack(ph_mesh* m, int32_t pool, const void* recvbuf);

/* The shard's largest signal rate max (|v_d| + c)/dx_d, as one double at
 * device address d_rate: recompute = 0 takes the one the last stage 2 folded
 * in, 1 computes it from the state (after ph_set_state and its exchange). */
int ph_shard_rate(ph_mesh* m, int32_t recompute, double* d_rate);

/* Time-step bookkeeping with the global rate at device address d_rate (the
 * max over shards of ph_shard_rate): first = 0 commits the cycle (time, cycle
 * count) and sets the next dt = cfl / rate; first = 1 sets the first dt of a
 * fresh state. */
int ph_shard_finish(ph_mesh* m, int32_t first, const double* d_rate);

/* All shards of one mesh in this process (shards[s] is shard s of n; they
 * may live on different devices, each on its own stream): the exchange is a
 * device copy (cudaMemcpyPeerAsync) into each receiver's own buffer and the
 * dt reduction runs on shard 0's device.  ph_shards_sync after ph_set_state
 * on every shard (ghost exchange and the global first dt); ph_shards_step
 * advances ncycles.  Neither waits for the GPU.
 * Errors: PH_ERR_INVALID (not the n shards of one mesh), PH_ERR_STATE (a
 * shard without a state), PH_ERR_CUDA. */
int ph_shards_sync(ph_mesh* const* shards, int32_t n);
int ph_shards_step(ph_mesh* const* shards, int32_t n, int32_t ncycles);

/* The halo plan of shard `shard` with `peer`, from the configuration alone
 * (host computation, no device work): the keys (global leaf x padded cells +
 * padded cell index of the receiving ghost cell) it sends to and receives
 * from the peer, in message order.  *nsend / *nrecv hold the capacities of
 * send_keys / recv_keys (either array may be NULL to query the counts) and
 * receive the counts; leaf_range (may be NULL) the shard's global leaves.
 * Errors: PH_ERR_INVALID (bad shard or peer, capacity too small). */
int ph_shard_plan(const ph_config* cfg, int32_t nshards, int32_t shard, int32_t peer, int64_t* send_keys,
                  int64_t* nsend, int64_t* recv_keys, int64_t* nrecv, int64_t leaf_range[2]);

/* Outputs and restarts (Sec. 3.9: outputs of single or double precision, and
 * a restart type from which a run continues bitwise identically).
 *
 * ph_save writes the mesh to the file `path` (created or truncated): its
 * configuration, block tree (levels, locations and the per-leaf ages that set
 * the derefinement cadence), time, cycle, current and next dt, status
 * counters, and the interior state in the layout of ph_get_state, stored in
 * `precision` (PH_FP64 or PH_FP32).  A file whose precision is at least the
 * mesh's is a restart file: ph_load of it followed by ph_step(n) gives the
 * state, dt, time and tree that n more cycles of the saved mesh give, bit for
 * bit.  An FP64 mesh saved as PH_FP32 is an output (each value rounded to
 * nearest); it loads, but the continuation is not bitwise.  Synchronises the
 * mesh's stream.  Errors: PH_ERR_INVALID (bad argument), PH_ERR_STATE (no
 * state yet), PH_ERR_IO (the file could not be written).
 *
 * ph_load reads such a file and creates a new mesh on `stream` (as
 * ph_create), owned by the caller (ph_destroy).  The file is validated before
 * any device work: PH_ERR_IO if it cannot be opened or is truncated,
 * PH_ERR_INVALID if it is not a file of this format or its tree does not tile
 * the domain; *out is NULL on any error.  The file's format is native byte
 * order, not portable across machines of different endianness. */
int ph_save(ph_mesh* m, const char* path, int32_t precision);
int ph_load(const char* path, void* stream, ph_mesh** out);

/* Accuracy check of the stage kernels' reciprocal and root routines.  The
 * paper has no counterpart: the kernels compute 1/x, 1/sqrt(x) and sqrt(x)
 * (Sec. 4.1's HLLE wave speeds and Roe weights, the primitive variables, the
 * limiter) from the hardware approximation plus one Newton-Raphson step
 * instead of the correctly rounded operations; this entry evaluates those
 * routines on caller data so that tests can bound their error.
 *   fn         PH_MATH_RCP, PH_MATH_RSQRT or PH_MATH_SQRT (the routines),
 *              PH_MATH_RCP_APPROX or PH_MATH_RSQRT_APPROX (the raw hardware
 *              approximations they start from; PH_FP64 only)
 *   precision  PH_FP64 (x, y double) or PH_FP32 (float)
 *   x, y       device pointers to n elements; y[i] = fn(x[i]); may not overlap
 *   stream     cudaStream_t the kernel is queued on (asynchronous)
 * Returns PH_ERR_INVALID for a bad argument, PH_ERR_CUDA if the launch fails. */
#define PH_MATH_RCP 0
#define PH_MATH_RSQRT 1
#define PH_MATH_SQRT 2
#define PH_MATH_RCP_APPROX 3
#define PH_MATH_RSQRT_APPROX 4
int ph_debug_math(int32_t fn, int32_t precision, const void* x, void* y, int64_t n, void* stream);

/* Multiply-add throughput probe (the paper has no counterpart): measures the
 * peak rate of the arithmetic pipe that bounds the FP64 stage kernel, so that
 * its roofline fraction is taken against a measured rather than a nominal
 * peak.  Launches `ctas` CTAs of 256 threads on `stream` (a cudaStream_t,
 * asynchronous); every thread runs `iters` rounds of 8 independent
 * multiply-add chains with no memory traffic and writes one value to
 * out[cta * 256 + thread] (a device array of ctas * 256 doubles for kind
 * PH_FMA_FP64, floats otherwise).  The caller times the launch on the stream;
 * it performs ctas * 256 * iters * 16 flops (twice that for
 * PH_FMA_FP32X2, whose instructions work on two lanes).
 * Errors: PH_ERR_INVALID (kind, ctas outside 1 .. 2^20, iters outside
 * 1 .. 2^32, null out), PH_ERR_CUDA (launch). */
#define PH_FMA_FP64 0
#define PH_FMA_FP32 1
#define PH_FMA_FP32X2 2
int ph_debug_fma_rate(int32_t kind, int32_t ctas, int64_t iters, void* out, void* stream);

/* Conserved totals of a caller-owned state without any device allocation.
 * The paper has no counterpart: this exists for callers that may not call
 * cudaMalloc at all (a plugin whose host application owns every byte of
 * device memory, a solver embedded in a code that reserves its whole memory
 * budget up front, a time-critical loop that must not enter the CUDA
 * allocator, which can block and synchronise).  It computes what ph_totals
 * computes, from the state alone:
 *   U       device pointer, interior state in the layout of ph_get_state
 *           (U[block][var][k][j][i] over nx cells), double for PH_FP64 or
 *           float for PH_FP32
 *   nx[3]   host array, interior cells per block
 *   nvar    variables per cell: 5 + the mesh's passive scalars (5, 6 or 7);
 *           it sets the block stride and the number of totals
 *   nblocks 0 .. PH_TOTALS_NOALLOC_MAX_BLOCKS; more is rejected with
 *           PH_ERR_INVALID
 *   level   device pointer to nblocks levels, or NULL for all level 0
 *   vol     host array of nlevels cell volumes, vol[l] for level l
 *           (1 <= nlevels <= 5, nlevels = 1 when level is NULL); a block whose
 *           level is outside [0, nlevels) makes every total NaN
 *   out     device pointer to nvar doubles, written asynchronously on `stream`
 *           (a cudaStream_t; NULL = legacy default stream)
 * Its scratch (per-block partial sums) is a fixed device array of
 * PH_TOTALS_NOALLOC_MAX_BLOCKS x 7 doubles (896 KiB) that every GPU which
 * loads the library holds until the process exits.  The first call on a
 * device, made with that device current, looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the array: calls whose work overlaps on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * Each call overwrites the entries it reads, so nothing needs clearing. */
#define PH_TOTALS_NOALLOC_MAX_BLOCKS 16384
int ph_totals_noalloc(const void* U, int32_t precision, const int32_t nx[3], int32_t nvar,
                      int32_t nblocks, const int8_t* level, const double* vol, int32_t nlevels,
                      double* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PH_HYDRO_H */
