// ph_stage.cuh -- the fused per-block stage kernel (K3).
//
// One launch covers every leaf block of the mesh ("pack all blocks into one
// kernel", arXiv:2202.12309 Sec. 3.6/5.1).  A CTA owns a TX x TY column tile
// of one block and marches along x3 over KC planes, holding four planes of
// primitives (tile + 2 ghost cells in x1, x2) in a shared-memory ring.  For
// plane k it:
//   (C) computes van Leer half-slopes: x1 and x2 for the plane, x3 for its own
//       column (x3 slopes roll through registers, each computed once), and
//       the HLLE flux on the x3 face above its cell;
//   (E) computes HLLE fluxes on all x1 and x2 faces of the plane into shared
//       memory;
//   (F) converts plane k+3, staged in the ring slot of plane k-1 while (C)
//       and (E) ran, to primitives, and stages plane k+4 into the slot of
//       plane k;
//   (G) forms the flux divergence and the SSPRK2 combination and writes the
//       new conserved state (stage 2 also folds the cell's signal speed into
//       the block-wide max that becomes the next dt, Sec. 3.10); on periodic
//       uniform meshes it also writes each new value within two cells of a
//       block face into the ghost zones of the neighbours it fills, which is
//       the whole ghost exchange of the stage (Sec. 3.7).
// Every face flux is computed once per tile (twice only on tile borders),
// every slope once per tile (plus one halo column/row), every primitive
// once per tile plus halo.
#pragma once
#include "ph_device.cuh"
#include "ph_tma.cuh"

namespace ph {

template <class T>
struct StageArgs {
  const T* Uin;        // stencil input, padded blocks [slot][v][k][j][i]
  const T* U0;         // stage 2: state at the start of the cycle (pointwise)
  T* Uout;             // stage 1: U1; stage 2: U0 (in place)
  const int8_t* level; // per leaf (null: all level 0)
  double idx[MAXLEV + 1][3];  // 1/dx per level and direction
  int nx[3];           // interior cells per block
  int S[3];            // padded extents nx + 4
  int ntile[3];        // tiles per block along x1, x2 and k-chunks along x3
  int KC;              // planes per chunk
  int nleaf;
  int stage;           // 1 or 2
  int want_rate;       // stage 2 on uniform meshes: fold the next dt's max
  Phys<T> P;
  DevScalars* sc;
  // flux-correction capture (multi-level meshes): per leaf and face,
  // 2 rec + 1 on the fine side of record rec, 2 rec on the coarse side, -1 none
  const int* face_rec;
  T* fc_coarse;        // [rec][v][n_t2][n_t1] flux of the coarse block on the face
  T* fc_fine;          // [rec][v][2 n_t2][2 n_t1] fluxes of the fine blocks on the face
  const int* fine_off; // per leaf 6 x 2: offset of the fine block's quadrant (t1, t2)
  int nvar;            // conserved variables per cell: NV + passive scalars
  // Uniform periodic meshes: the 27 neighbours of every leaf (as the ghost
  // exchange uses them).  When set, the stage also writes each new interior
  // value into the ghost zones of Uout that it fills (push exchange), and the
  // separate exchange launch is not needed.
  const int* nbr;
  // FP32 uniform meshes with TMA staging whose blocks tile into the launch's
  // 32 x 16 or 16 x 16 tiles: the paired kernel (ph_stage_pair.cuh) runs
  int pair;
};

// Store one face flux of a leaf on a fine-coarse face (Sec. 3.7 flux
// correction).  face = 2 d + side; (a1, a2) are the cell's indices along
// t1 = d+1 and t2 = d+2 (mod 3).  The coarse leaf of the record writes its
// coarse flux; each of the 4 fine leaves writes its quadrant (q1, q2) of the
// record's fine fluxes, which are 2 n_t1 x 2 n_t2 per variable.
template <class T>
__device__ __forceinline__ void capture(const StageArgs<T>& a, int leaf, int face, int a1, int a2,
                                        int v, T val) {
  const int fr = a.face_rec[6 * leaf + face];
  const int rec = fr >> 1;
  const int d = face >> 1;
  const int m1 = a.nx[(d + 1) % 3], m2 = a.nx[(d + 2) % 3];
  if ((fr & 1) == 0) {
    a.fc_coarse[(((size_t)rec * a.nvar + v) * m2 + a2) * m1 + a1] = val;
  } else {
    const int q1 = a.fine_off[12 * leaf + 2 * face], q2 = a.fine_off[12 * leaf + 2 * face + 1];
    a.fc_fine[(((size_t)rec * a.nvar + v) * (2 * m2) + q2 * m2 + a2) * (2 * m1) + q1 * m1 + a1] = val;
  }
}

// NTO: thread count of the CTA when the tile runs inside a kernel of another
// size (0: the tile's own choice below).
// Cell (i, j, k) of a leaf lies on a face whose flux-correction record has
// the leaf on its coarse side (fr: the leaf's 6 records, 2 rec on the coarse
// side, 2 rec + 1 on the fine side, -1 none): the correction changes it.
__device__ __forceinline__ bool coarse_face_cell(const int* fr, int i, int j, int k, int n1, int n2, int n3) {
  auto coarse = [](int r) { return r >= 0 && (r & 1) == 0; };
  return (i == 0 && coarse(fr[0])) || (i == n1 - 1 && coarse(fr[1])) || (j == 0 && coarse(fr[2])) ||
         (j == n2 - 1 && coarse(fr[3])) || (k == 0 && coarse(fr[4])) || (k == n3 - 1 && coarse(fr[5]));
}

template <class T, int TX, int TY, int NVT = NV, int NTO = 0>
struct StageSmem {
  static constexpr int WX = TX + 4, WY = TY + 4;
  // threads.  FP32 (issue-bound): enough for the largest per-plane work list
  // (x1 or x2 slopes) in one round, so no warp works a second round while the
  // others wait at the barrier, with registers capped for 3 CTAs per SM.
  // FP64 (bound by the FP64 pipe): one thread per cell, no cap (the extra warp
  // and the cap cost more FP64 pipe time in spills than the balance saves).
  static constexpr int NT0 = (TX + 2) * TY > TX * (TY + 2) ? (TX + 2) * TY : TX * (TY + 2);
  static constexpr int NT = NTO ? NTO : (sizeof(T) == 4 ? (NT0 + 31) / 32 * 32 : TX * TY);
  // resident CTAs per SM the registers are allocated for (FP32: 3; FP64: left
  // to the compiler, which keeps 2 CTAs of 256 threads without spills)
  static constexpr int MINB = sizeof(T) == 4 ? 3 : 0;
  static constexpr int PLANE = NVT * WX * WY;         // one plane of every variable with halo
  static constexpr int SLOT = (PLANE * (int)sizeof(T) + 127) / 128 * 128 / (int)sizeof(T);
  static constexpr unsigned PLANE_BYTES = PLANE * sizeof(T);  // one TMA box
  // row pitch of the face-flux arrays: TX+4 keeps the FP32 warps of own_cell
  // on distinct banks; FP64 keeps the dense TX+1
  static constexpr int FP = sizeof(T) == 4 ? TX + 4 : TX + 1;
  static constexpr int DXN = NVT * TY * (TX + 2);     // x1 slopes
  static constexpr int DYN = NVT * (TY + 2) * TX;     // x2 slopes
  static constexpr int FXN = NVT * TY * FP;           // x1 face fluxes (TX+1 used per row)
  static constexpr int FYN = NVT * (TY + 1) * FP;     // x2 face fluxes (TX used per row)
  static constexpr size_t body = sizeof(T) * (size_t)(4 * SLOT + DXN + DYN + FXN + FYN);
  static constexpr size_t red_off = (body + 15) / 16 * 16;
  static constexpr size_t bar_off = red_off + 32 * sizeof(double);
  // + 4 mbarriers, + slack to align the base to 128 bytes (TMA destinations)
  static constexpr size_t bytes = bar_off + 4 * sizeof(uint64_t) + 128;
};

// Cell owned by thread tid < TX*TY.  The rows a warp touches are chosen so
// that its 32 lanes hit distinct shared-memory banks for 4-byte data with row
// pitch TX+4: a 16-wide warp covers rows r and r+4 (4 (16+4) = 16 mod 32), an
// 8-wide warp rows r, r+2, r+4, r+6, a 32-wide warp one row.
template <class T, int TX, int TY>
__device__ __forceinline__ void own_cell(int tid, int& tx, int& ty) {
  if (sizeof(T) == 8) {  // a half-warp of doubles already fills all 32 banks
    tx = tid % TX;
    ty = tid / TX;
  } else if (TX == 16 && TY % 8 == 0) {
    const int w = tid >> 5, h = (tid >> 4) & 1;
    tx = tid & 15;
    ty = (w & 3) + 8 * (w >> 2) + 4 * h;
  } else if (TX == 8 && TY % 8 == 0) {
    const int w = tid >> 5, q = (tid >> 3) & 3;
    tx = tid & 7;
    ty = (w & 1) + 8 * (w >> 1) + 2 * q;
  } else {
    tx = tid % TX;
    ty = tid / TX;
  }
}

// One tile of one block for one stage.  J holds the block's data pointers,
// geometry, the tile's origin and the k-range; returns the max over the
// tile's own cells of the signal rate (|v_d|+c)/dx_d of the new state when
// J.want_rate (else 0).  Uses the whole CTA; smem as laid out by StageSmem.
template <class T>
struct TileJob {
  const T* Ub;     // stencil input block (padded)
  const T* U0b;    // stage 2: the block at the start of the cycle
  T* Uoutb;        // output block
  int nx[3], S[3];
  int i0, j0, k0, k1;
  T idx1, idx2, idx3;
  T dt;
  int stage;
  int want_rate;
  int leaf;        // leaf index for flux capture (multi-level meshes)
  const int* nbr27;  // push exchange: the leaf's 27 neighbours (null: none)
  T* pool;           // push exchange: the output pool (block b at b * bsize)
  size_t bsize;
};

// Push form of the same-level ghost exchange (uniform periodic meshes): the
// new value u of interior cell (i, j, k) of a block is also the ghost value
// of every neighbour whose ghost region holds the cell's periodic image.  A
// cell within NG cells of the low (high) face along x_d lies in the high
// (low) ghost layer of the neighbour on that side, at index i_d + n_d
// (i_d - n_d); a cell near faces along several axes also fills the edge and
// corner regions of the neighbours across them (up to 7 writes).  Writes the
// same values as the pull exchange (ph_kernels.cu), into ghost cells only, so
// concurrent tiles never write a cell twice or a cell another tile reads.
template <class T, int W, int NVT>
__device__ __forceinline__ void push_ghosts(const TileJob<T>& J, int i, int j, int k, const T* u,
                                            size_t vstride) {
  // W = 1: one cell; W = 2: cells (i, i+1) as one 2-wide store, i even
  const int n1 = J.nx[0], n2 = J.nx[1], n3 = J.nx[2];
  const int s1 = i < NG ? -1 : (i + W > n1 - NG ? 1 : 0);
  const int s2 = j < NG ? -1 : (j >= n2 - NG ? 1 : 0);
  const int s3 = k < NG ? -1 : (k >= n3 - NG ? 1 : 0);
  if ((s1 | s2 | s3) == 0) return;
  const int S1 = J.S[0], S2 = J.S[1];
#pragma unroll
  for (int m = 1; m < 8; ++m) {
    const int o1 = (m & 1) ? s1 : 0, o2 = (m & 2) ? s2 : 0, o3 = (m & 4) ? s3 : 0;
    if (((m & 1) && !s1) || ((m & 2) && !s2) || ((m & 4) && !s3)) continue;
    const int nb = J.nbr27[(o3 + 1) * 9 + (o2 + 1) * 3 + (o1 + 1)];
    T* dst = J.pool + (size_t)nb * J.bsize +
             ((size_t)(k - o3 * n3 + NG) * S2 + (j - o2 * n2 + NG)) * S1 + (i - o1 * n1 + NG);
    if constexpr (W == 1) {
#pragma unroll
      for (int v = 0; v < NVT; ++v) dst[v * vstride] = u[v];
    } else {
      static_assert(W == 1 || sizeof(T) == 4, "paired pushes are FP32");
#pragma unroll
      for (int v = 0; v < NVT; ++v) {
        float2 p;
        p.x = u[2 * v];
        p.y = u[2 * v + 1];
        *reinterpret_cast<float2*>(dst + v * vstride) = p;
      }
    }
  }
}

// TMA = true: planes arrive by one tensor copy each (tmap over the stencil
// input pool, box (TX+4, TY+4, 1, 5) at (i0, j0, plane, vz0)), issued one plane
// ahead on the slot's mbarrier, and are converted to primitives in place.
// Returns with *failed set (and every thread leaving) if a wait gave up.
// Half slopes of every variable: the five hydro ones batched, the passive
// scalars one by one.
template <class T, int NVT>
__device__ __forceinline__ void vanleer_all(const T wm[NVT], const T w0[NVT], const T wp[NVT], T h[NVT]) {
  vanleer_half5(wm, w0, wp, h);
#pragma unroll
  for (int v = NV; v < NVT; ++v) h[v] = vanleer_half_rcp(wm[v], w0[v], wp[v]);
}


// STAGE: 1 or 2 fixes the stage at compile time (its own register
// allocation); 0 takes it from J.stage.  NTO: see StageSmem.
template <class T, int TX, int TY, bool TMA, int NVT = NV, int STAGE = 0, int NTO = 0>
__device__ __forceinline__ double stage_tile(const TileJob<T>& J, const Phys<T>& P,
                                             const StageArgs<T>& a, unsigned char* smem_raw,
                                             unsigned& floors, const CUtensorMap* tmap = nullptr,
                                             int vz0 = 0, uint64_t* bars = nullptr,
                                             int* failed = nullptr,
                                             unsigned* parity_io = nullptr) {
  using SM = StageSmem<T, TX, TY, NVT, NTO>;
  constexpr int NT = SM::NT;        // threads of the CTA
  constexpr int NC = TX * TY;       // threads that own a cell of the tile
  constexpr int FP = SM::FP;
  constexpr int WX = SM::WX, WY = SM::WY;
  T* ring = reinterpret_cast<T*>(smem_raw);
  T* sdx = ring + 4 * SM::SLOT;
  T* sdy = sdx + SM::DXN;
  T* sfx = sdy + SM::DYN;
  T* sfy = sfx + SM::FXN;

  const int tid = threadIdx.x;
  // The x2 work lists are walked from warp 1 on: when a list leaves a second,
  // partial round, the x1 list's falls to warp 0 and the x2 list's to warp 1,
  // which run on different SM sub-partitions, instead of both to warp 0.
  const int trot = (tid + NT - 32) % NT;
  const bool has_cell = (NT == NC) || tid < NC;  // compile-time true when every thread owns one
  int tx = 0, ty = 0;
  if (has_cell) own_cell<T, TX, TY>(tid, tx, ty);
  const int n1 = J.nx[0], n2 = J.nx[1], n3 = J.nx[2];
  const int S1 = J.S[0], S2 = J.S[1], S3 = J.S[2];
  const int i0 = J.i0, j0 = J.j0, k0 = J.k0, k1 = J.k1;
  const T idx1 = J.idx1, idx2 = J.idx2, idx3 = J.idx3;
  const size_t vstride = (size_t)S1 * S2 * S3;
  const T* __restrict__ Ub = J.Ub;
  const int leaf = J.leaf;

  // Stage plane p (interior index, -2..n3+1) into its ring slot as primitives.
  // Cells past a ragged block edge are clamped to the edge (never used).
  auto load_plane = [&](int p) {
    T* dst = ring + ((p + 4) & 3) * SM::SLOT;
    const size_t kofs = (size_t)(p + NG) * S2 * S1;
    for (int c = tid; c < WX * WY; c += NT) {
      const int jj = c / WX, ii = c - jj * WX;
      const int jp = min(j0 + jj, S2 - 1), ip = min(i0 + ii, S1 - 1);
      const T* src = Ub + kofs + (size_t)jp * S1 + ip;
      T w[NVT];
#pragma unroll
      for (int v = 0; v < NVT; ++v) w[v] = __ldg(src + v * vstride);
      cons_to_prim<T, NVT>(w, P, floors);
#pragma unroll
      for (int v = 0; v < NVT; ++v) dst[(v * WY + jj) * WX + ii] = w[v];
    }
  };
  // TMA path: issue the copy of plane p (one thread), then convert it in
  // place once its barrier completes (all threads).  Cells of a ragged tile
  // outside the padded block arrive as zeros and are left alone (no valid
  // cell's stencil reaches them).
  // bit s: parity of the next completion of slot s (carried across calls by
  // a CTA that runs several tiles on the same barriers)
  unsigned parity = parity_io ? *parity_io : 0u;
  auto issue = [&](int p) {
    if (TMA && tid == 0) {
      const int sl = (p + 4) & 3;
      mbar_expect_tx(bars + sl, SM::PLANE_BYTES);
      tma_load_4d(ring + sl * SM::SLOT, tmap, bars + sl, J.i0, J.j0, p + NG, vz0);
    }
  };
  // The conversion list is walked from warp 2 on, so that its partial second
  // round falls on other warps than the x1 / x2 face lists' (warps 0 and 1)
  // in the same barrier interval.
  // The four 2 x 2 corners of a staged plane are read by no stencil.  FP64
  // does not convert them: the list is rows 0-1 (columns 2..TX+1), rows
  // 2..TY+1 (every column), rows TY+2..TY+3 (columns 2..TX+1).  FP32, bound
  // by instruction issue, converts the whole plane (the mapping costs more
  // than the 16 conversions it saves).
  const int crot = (tid + NT - (64 % NT)) % NT;
  constexpr int NCV = sizeof(T) == 4 ? WX * WY : WX * WY - 16;
  auto convert = [&](int p) -> bool {
    const int sl = (p + 4) & 3;
    const bool ok = mbar_wait(bars + sl, (parity >> sl) & 1u, 1u << 22);
    parity ^= 1u << sl;
    T* dst = ring + sl * SM::SLOT;
    const int vi = min(WX, S1 - i0), vj = min(WY, S2 - j0);
    for (int c = crot; c < NCV; c += NT) {
      int jj, ii;
      if (sizeof(T) == 4) {
        jj = c / WX;
        ii = c - jj * WX;
      } else if (c < 2 * TX) {
        jj = c / TX;
        ii = 2 + c - jj * TX;
      } else if (c < 2 * TX + TY * WX) {
        const int q = c - 2 * TX;
        jj = q / WX;
        ii = q - jj * WX;
        jj += 2;
      } else {
        const int q = c - 2 * TX - TY * WX;
        jj = q / TX;
        ii = 2 + q - jj * TX;
        jj += TY + 2;
      }
      if (ii >= vi || jj >= vj) continue;
      T w[NVT];
#pragma unroll
      for (int v = 0; v < NVT; ++v) w[v] = dst[(v * WY + jj) * WX + ii];
      cons_to_prim<T, NVT>(w, P, floors);
#pragma unroll
      for (int v = 0; v < NVT; ++v) dst[(v * WY + jj) * WX + ii] = w[v];
    }
    return ok;
  };
  // every thread reports a failed wait; all leave together after a barrier
  auto check_failed = [&](bool ok) -> bool {
    if (!ok) atomicExch(failed, 1);
    __syncthreads();
    return *(volatile int*)failed != 0;
  };
  auto col = [&](int p, T w[NVT]) {  // own column's primitive at plane p
    const T* s = ring + ((p + 4) & 3) * SM::SLOT;
#pragma unroll
    for (int v = 0; v < NVT; ++v) w[v] = s[(v * WY + ty + 2) * WX + tx + 2];
  };

  // Priming: planes k0-2 .. k0+1 give the x3 slope at k0 and the flux at k0-1/2.
  if (TMA) {
    for (int p = k0 - 2; p <= k0 + 1; ++p) issue(p);
    bool ok = true;
    for (int p = k0 - 2; p <= k0 + 1; ++p) ok = convert(p) && ok;
    fence_proxy_async_smem();
    if (check_failed(ok)) return 0.0;
  } else {
    load_plane(k0 - 2);
    load_plane(k0 - 1);
    load_plane(k0);
    load_plane(k0 + 1);
    __syncthreads();
  }
  // (the x3 differences are recomputed per plane rather than carried: a
  // carried difference costs more registers than the subtraction it saves)
  T dz[NVT], fzm[NVT];
  if (has_cell) {  // x3 work is per owned column
    T wa[NVT], wb[NVT], wc[NVT], wd[NVT], wl[NVT], wr[NVT];
    col(k0 - 2, wa);
    col(k0 - 1, wb);
    col(k0, wc);
    col(k0 + 1, wd);
    T d0[NVT];
    vanleer_all<T, NVT>(wa, wb, wc, d0);
    vanleer_all<T, NVT>(wb, wc, wd, dz);
#pragma unroll
    for (int v = 0; v < NVT; ++v) {
      wl[v] = wb[v] + d0[v];
      wr[v] = wc[v] - dz[v];
    }
    hlle<T, 2, NVT>(wl, wr, P, fzm);
  }
  __syncthreads();
  // Plane k0+2 into the slot of plane k0-2 (read above); the loop's step k
  // then brings in plane k+3 while it computes the fluxes of plane k.
  if (TMA) {
    issue(k0 + 2);
    const bool ok = convert(k0 + 2);
    fence_proxy_async_smem();
    if (check_failed(ok)) return 0.0;
    if (k0 + 3 <= k1 + 1) issue(k0 + 3);  // slot of plane k0-1, read above
  } else {
    load_plane(k0 + 2);
    __syncthreads();
  }

  const int i = i0 + tx, j = j0 + ty;
  const bool own = has_cell && (i < n1) && (j < n2);
  // dt / dx_d (stage 2: half of it, the SSPRK2 weight of dt L)
  const int stg = STAGE ? STAGE : J.stage;
  const T hs = stg == 1 ? T(1) : T(0.5);
  const T c1 = hs * J.dt * idx1, c2 = hs * J.dt * idx2, c3 = hs * J.dt * idx3;
  // running max in the data precision (FP32: no FP64 conversion or compare
  // per cell; widening is exact and monotonic, so the max is the same)
  T rate = T(0);

  for (int k = k0; k < k1; ++k) {
    // (C) slopes; own x3 flux (planes k, k+1, k+2 are in the ring)
    T fzlo[NVT];  // x3 flux below the cell; fzm becomes the flux above it
    if (has_cell) {
      T wa[NVT], wb[NVT], wc[NVT], wl[NVT], wr[NVT], f[NVT];
      col(k, wa);
      col(k + 1, wb);
      col(k + 2, wc);
      T d1[NVT];
      vanleer_all<T, NVT>(wa, wb, wc, d1);
#pragma unroll
      for (int v = 0; v < NVT; ++v) {
        wl[v] = wa[v] + dz[v];
        wr[v] = wb[v] - d1[v];
        dz[v] = d1[v];
      }
      hlle<T, 2, NVT>(wl, wr, P, f);
#pragma unroll
      for (int v = 0; v < NVT; ++v) {
        fzlo[v] = fzm[v];
        fzm[v] = f[v];
      }
    }
    // FP64: the warps that take the lists' partial rounds move by two every
    // other plane, to the other two SM sub-partitions (warp w runs on
    // sub-partition w % 4), so that the two CTAs on an SM less often load
    // the same sub-partition's FP64 unit with their extra rounds.
    const int sh = (sizeof(T) == 8 && NT >= 128) ? 64 * (k & 1) : 0;
    {
      const T* W = ring + ((k + 4) & 3) * SM::SLOT;
      for (int c = (tid + NT - sh) % NT; c < (TX + 2) * TY; c += NT) {   // x1 slopes, cells -1..TX
        const int jj = c / (TX + 2), ii = c - jj * (TX + 2);
        T a[NVT], b[NVT], q[NVT], h[NVT];
#pragma unroll
        for (int v = 0; v < NVT; ++v) {
          const T* r = W + (v * WY + jj + 2) * WX + ii;
          a[v] = r[0];
          b[v] = r[1];
          q[v] = r[2];
        }
        vanleer_all<T, NVT>(a, b, q, h);
#pragma unroll
        for (int v = 0; v < NVT; ++v) sdx[(v * TY + jj) * (TX + 2) + ii] = h[v];
      }
      for (int c = (trot + NT - sh) % NT; c < TX * (TY + 2); c += NT) {  // x2 slopes, rows -1..TY
        const int jj = c / TX, ii = c - jj * TX;
        T a[NVT], b[NVT], q[NVT], h[NVT];
#pragma unroll
        for (int v = 0; v < NVT; ++v) {
          const T* r = W + (v * WY + jj) * WX + ii + 2;
          a[v] = r[0];
          b[v] = r[WX];
          q[v] = r[2 * WX];
        }
        vanleer_all<T, NVT>(a, b, q, h);
#pragma unroll
        for (int v = 0; v < NVT; ++v) sdy[(v * (TY + 2) + jj) * TX + ii] = h[v];
      }
    }
    __syncthreads();
    // (E) x1 and x2 face fluxes of the plane.  FP64: when both lists leave a
    // partial second round that together fit one warp, the last warp takes
    // both remainders at once, x2 faces with their velocity components
    // rotated so that the normal one comes first (the flux is then the same
    // to the last bit), instead of two half-empty warps each issuing the whole
    // flux on the FP64 pipe.
    {
      constexpr int NF1 = (TX + 1) * TY, NF2 = TX * (TY + 1);
      constexpr int E1 = NF1 - NT, E2 = NF2 - NT;
      constexpr bool MERGE = sizeof(T) == 8 && E1 > 0 && E2 > 0 && E1 + E2 <= 32;
      const T* W = ring + ((k + 4) & 3) * SM::SLOT;
      for (int c = tid; c < (MERGE ? NT : NF1); c += NT) {
        const int jj = c / (TX + 1), f = c - jj * (TX + 1);  // face between cells f-1, f
        T wl[NVT], wr[NVT], fl[NVT];
#pragma unroll
        for (int v = 0; v < NVT; ++v) {
          const T* r = W + (v * WY + jj + 2) * WX + f + 1;
          const T* s = sdx + (v * TY + jj) * (TX + 2) + f;
          wl[v] = r[0] + s[0];
          wr[v] = r[1] - s[1];
        }
        hlle<T, 0, NVT>(wl, wr, P, fl);
#pragma unroll
        for (int v = 0; v < NVT; ++v) sfx[(v * TY + jj) * FP + f] = fl[v];
      }
      for (int c = MERGE ? tid : trot; c < (MERGE ? NT : NF2); c += NT) {
        const int g = c / TX, ii = c - g * TX;   // face between rows g-1, g
        T wl[NVT], wr[NVT], fl[NVT];
#pragma unroll
        for (int v = 0; v < NVT; ++v) {
          const T* r = W + (v * WY + g + 1) * WX + ii + 2;
          const T* s = sdy + (v * (TY + 2) + g) * TX + ii;
          wl[v] = r[0] + s[0];
          wr[v] = r[WX] - s[TX];
        }
        hlle<T, 1, NVT>(wl, wr, P, fl);
#pragma unroll
        for (int v = 0; v < NVT; ++v) sfy[(v * (TY + 1) + g) * FP + ii] = fl[v];
      }
      if (MERGE && tid >= NT - 32 - sh && tid < NT - 32 - sh + E1 + E2) {
        const int l = tid - (NT - 32 - sh);
        const bool y = l >= E1;              // lanes E1.. take x2 faces
        const int c = NT + (y ? l - E1 : l);
        const int jj = c / (TX + 1), f = c - jj * (TX + 1);
        const int g = c / TX, ii = c - g * TX;
        const T* r = y ? W + (g + 1) * WX + ii + 2 : W + (jj + 2) * WX + f + 1;
        const T* sp = y ? sdy + g * TX + ii : sdx + jj * (TX + 2) + f;
        const int rs = y ? WX : 1, ss = y ? TX : 1;
        const int svs = y ? (TY + 2) * TX : TY * (TX + 2);
        T* o = y ? sfy + g * FP + ii : sfx + jj * FP + f;
        const int ovs = y ? (TY + 1) * FP : TY * FP;
        T wl[NVT], wr[NVT], fl[NVT];
#pragma unroll
        for (int v = 0; v < NVT; ++v) {
          wl[v] = r[v * WY * WX] + sp[v * svs];
          wr[v] = r[v * WY * WX + rs] - sp[v * svs + ss];
        }
        // x2 faces: (v1, v2, v3) -> (v2, v3, v1)
        const T l1 = wl[1], r1 = wr[1];
        wl[1] = y ? wl[2] : wl[1];
        wl[2] = y ? wl[3] : wl[2];
        wl[3] = y ? l1 : wl[3];
        wr[1] = y ? wr[2] : wr[1];
        wr[2] = y ? wr[3] : wr[2];
        wr[3] = y ? r1 : wr[3];
        hlle<T, 0, NVT>(wl, wr, P, fl);
        const T f3 = fl[3];
        fl[3] = y ? fl[2] : fl[3];
        fl[2] = y ? fl[1] : fl[2];
        fl[1] = y ? f3 : fl[1];
#pragma unroll
        for (int v = 0; v < NVT; ++v) o[v * ovs] = fl[v];
      }
    }
    // (F) plane k+3 into the slot of plane k-1, which step k does not read
    if (TMA) {
      const bool ok = k + 3 <= k1 + 1 ? convert(k + 3) : true;
      fence_proxy_async_smem();  // this thread's reads of plane k before its slot is refilled
      if (check_failed(ok)) return 0.0;
      // plane k+4 into the slot of plane k, read for the last time above
      if (k + 4 <= k1 + 1) issue(k + 4);
    } else {
      if (k + 3 <= k1 + 1) load_plane(k + 3);
      __syncthreads();
    }
    // (G) flux divergence + SSPRK2 combination
    if (own) {
      const size_t cell = (size_t)(k + NG) * S2 * S1 + (size_t)(j + NG) * S1 + (i + NG);
      T unew[NVT];
#pragma unroll
      for (int v = 0; v < NVT; ++v) {
        // stage 1: U + dt L; stage 2: (U0 + U1)/2 + (dt/2) L, with
        // dt L = -sum_d (F_d+ - F_d-) dt/dx_d
        const T dfx = sfx[(v * TY + ty) * FP + tx + 1] - sfx[(v * TY + ty) * FP + tx];
        const T dfy = sfy[(v * (TY + 1) + ty + 1) * FP + tx] - sfy[(v * (TY + 1) + ty) * FP + tx];
        const T dfz = fzm[v] - fzlo[v];
        const T ucur = Ub[cell + v * vstride];
        const T base = stg == 1 ? ucur : T(0.5) * (J.U0b[cell + v * vstride] + ucur);
        unew[v] = fma(-dfx, c1, fma(-dfy, c2, fma(-dfz, c3, base)));
        J.Uoutb[cell + v * vstride] = unew[v];
      }
      if (J.nbr27) push_ghosts<T, 1, NVT>(J, i, j, k, unew, vstride);
      if (a.face_rec) {  // multi-level mesh: keep fluxes on fine-coarse faces
        const int* fr = a.face_rec + 6 * leaf;
        if (i == 0 && fr[0] >= 0)
          for (int v = 0; v < NVT; ++v) capture(a, leaf, 0, j, k, v, sfx[(v * TY + ty) * FP + tx]);
        if (i == n1 - 1 && fr[1] >= 0)
          for (int v = 0; v < NVT; ++v) capture(a, leaf, 1, j, k, v, sfx[(v * TY + ty) * FP + tx + 1]);
        if (j == 0 && fr[2] >= 0)
          for (int v = 0; v < NVT; ++v) capture(a, leaf, 2, k, i, v, sfy[(v * (TY + 1) + ty) * FP + tx]);
        if (j == n2 - 1 && fr[3] >= 0)
          for (int v = 0; v < NVT; ++v) capture(a, leaf, 3, k, i, v, sfy[(v * (TY + 1) + ty + 1) * FP + tx]);
        if (k == 0 && fr[4] >= 0)
          for (int v = 0; v < NVT; ++v) capture(a, leaf, 4, i, j, v, fzlo[v]);
        if (k == n3 - 1 && fr[5] >= 0)
          for (int v = 0; v < NVT; ++v) capture(a, leaf, 5, i, j, v, fzm[v]);
      }
      // the signal rate of the new state for the next dt; on multi-level
      // meshes, cells next to a fine-coarse face on the coarse side are
      // skipped here and rated by the flux correction that changes them
      if (J.want_rate && !(a.face_rec && coarse_face_cell(a.face_rec + 6 * leaf, i, j, k, n1, n2, n3))) {
        cons_to_prim<T, NVT>(unew, P, floors);
        rate = rate_max(rate, wave_rate(unew, P, idx1, idx2, idx3));
      }
    }
  }
  if (parity_io) *parity_io = parity;
  return (double)rate;
}

template <class T, int TX, int TY, int NVT = NV>
__device__ __forceinline__ bool make_job(const StageArgs<T>& a, TileJob<T>& J) {
  const int tiles_per_block = a.ntile[0] * a.ntile[1] * a.ntile[2];
  const int leaf = blockIdx.x / tiles_per_block;
  if (leaf >= a.nleaf) return false;
  int t = blockIdx.x - leaf * tiles_per_block;
  const int tk = t / (a.ntile[0] * a.ntile[1]);
  t -= tk * a.ntile[0] * a.ntile[1];
  const int tj = t / a.ntile[0];
  const int ti = t - tj * a.ntile[0];
  const size_t bsize = (size_t)NVT * a.S[0] * a.S[1] * a.S[2];
  J.Ub = a.Uin + (size_t)leaf * bsize;
  J.U0b = a.U0 + (size_t)leaf * bsize;
  J.Uoutb = a.Uout + (size_t)leaf * bsize;
  for (int d = 0; d < 3; ++d) {
    J.nx[d] = a.nx[d];
    J.S[d] = a.S[d];
  }
  J.i0 = ti * TX;
  J.j0 = tj * TY;
  J.k0 = tk * a.KC;
  J.k1 = min(J.k0 + a.KC, a.nx[2]);
  const int lev = a.level ? (int)a.level[leaf] : 0;
  J.idx1 = (T)a.idx[lev][0];
  J.idx2 = (T)a.idx[lev][1];
  J.idx3 = (T)a.idx[lev][2];
  J.dt = (T)a.sc->dt_next;
  J.stage = a.stage;
  J.want_rate = a.want_rate;
  J.leaf = leaf;
  J.nbr27 = a.nbr ? a.nbr + 27 * leaf : nullptr;
  J.pool = a.Uout;
  J.bsize = bsize;
  return true;
}

template <class T, int TX, int TY, int NVT = NV>
__global__ void __launch_bounds__(StageSmem<T, TX, TY, NVT>::NT, StageSmem<T, TX, TY, NVT>::MINB)
stage_kernel(const StageArgs<T> a) {
  using SM = StageSmem<T, TX, TY, NVT>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* red = reinterpret_cast<double*>(smem_raw + SM::red_off);
  TileJob<T> J;
  if (!make_job<T, TX, TY, NVT>(a, J)) return;
  unsigned floors = 0;
  const double rate = stage_tile<T, TX, TY, false, NVT>(J, a.P, a, smem_raw, floors);
  if (a.want_rate) block_max_to(&a.sc->wmax_bits, rate, red);
  if (floors) atomicAdd(&a.sc->floor_hits, (unsigned long long)floors);
}

// The same stage with planes staged by TMA from the tensor map of the stencil
// input pool.
template <class T, int TX, int TY, int NVT = NV, int STAGE = 0>
__global__ void __launch_bounds__(StageSmem<T, TX, TY, NVT>::NT, StageSmem<T, TX, TY, NVT>::MINB)
stage_kernel_tma(const __grid_constant__ StageArgs<T> a, const __grid_constant__ CUtensorMap tmap) {
  using SM = StageSmem<T, TX, TY, NVT>;
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  unsigned char* smem_raw = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_dyn) + 127) & ~uintptr_t(127));
  double* red = reinterpret_cast<double*>(smem_raw + SM::red_off);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + SM::bar_off);
  __shared__ int failed;
  TileJob<T> J;
  if (!make_job<T, TX, TY, NVT>(a, J)) return;
  if (threadIdx.x == 0) {
    failed = 0;
    for (int s = 0; s < 4; ++s) mbar_init(bars + s, 1);
    mbar_fence_init();
  }
  __syncthreads();
  unsigned floors = 0;
  const double rate =
      stage_tile<T, TX, TY, true, NVT, STAGE>(J, a.P, a, smem_raw, floors, &tmap, J.leaf * NVT, bars,
                                              &failed);
  if (failed) {
    if (threadIdx.x == 0) atomicExch(&a.sc->error, 1);
    return;
  }
  if (a.want_rate) block_max_to(&a.sc->wmax_bits, rate, red);
  if (floors) atomicAdd(&a.sc->floor_hits, (unsigned long long)floors);
}

}  // namespace ph
