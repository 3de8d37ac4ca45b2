// ph_kernels.cu -- mesh-level kernels: ghost exchange (K1), remesh data
// movement (K7), signal-speed max for dt (K5), dt bookkeeping, refinement
// indicator (K6), interior <-> padded copies and conserved totals.
//
// Ghost exchange (arXiv:2202.12309 Sec. 3.7, "fill-in-one"): the paper packs
// every buffer of every block into one kernel, sends, and unpacks with
// restriction/prolongation.  On one GPU there is nothing to send, so K1 is a
// single pull: each ghost cell reads the data it needs straight from the
// interior of the leaf that covers it.  It reads interior cells only and
// writes ghost cells only, so one launch has no ordering hazard.
#include <algorithm>

#include "ph_nvtx.h"
#include "ph_internal.h"

namespace ph {

// Physical boundaries (PH_BC_*): a ghost index g outside the domain along
// one axis maps to its image inside, in the same block: outflow takes the
// first interior layer, reflecting mirrors about the face (and the caller
// negates the normal momentum).  lo/hi: the block touches the inner / outer
// face of the domain; bc_lo/bc_hi: the faces' boundary kinds.  Returns true
// if the index was mapped (the offset along the axis becomes 0).
__device__ __forceinline__ bool bc_image(int& g, int o, int n, bool lo, bool hi, int bc_lo,
                                         int bc_hi, bool& reflect) {
  if (o < 0 && lo && bc_lo != 0) {
    g = bc_lo == 1 ? NG : 2 * NG - 1 - g;
    reflect = bc_lo == 2;
    return true;
  }
  if (o > 0 && hi && bc_hi != 0) {
    g = bc_hi == 1 ? NG + n - 1 : 2 * (NG + n) - 1 - g;
    reflect = bc_hi == 2;
    return true;
  }
  return false;
}

// blockIdx.x = leaf, blockIdx.y = chunk of the leaf's ghost shell (each CTA
// copies about 1024 ghost cells, so that small meshes of large blocks still
// fill the GPU).  bcm packs the six faces' boundary kinds (2 bits each, x1
// inner first); 0 = periodic everywhere, where leaf_id and nbl are unused.
template <class T, int NVT = NV>
__global__ void ghost_uniform_kernel(T* U, const int* __restrict__ nbr, int3 nx,
                                     const int* __restrict__ leaf_id, int3 nbl, int bcm) {
  const int nxa[3] = {nx.x, nx.y, nx.z};
  const Shell sh(nxa);
  const int b = blockIdx.x;
  const int S1 = sh.S1, S2 = sh.S2, S3 = nx.z + 2 * NG;
  const size_t vs = (size_t)S1 * S2 * S3;
  T* dstb = U + (size_t)b * NVT * vs;
  const int* nb = nbr + 27 * b;
  const int total = sh.count();
  const int per = (total + gridDim.y - 1) / gridDim.y;
  const int c0 = blockIdx.y * per, c1 = min(total, c0 + per);
  int lx[3] = {0, 0, 0};
  if (bcm) {
    lx[0] = leaf_id[4 * b + 1];
    lx[1] = leaf_id[4 * b + 2];
    lx[2] = leaf_id[4 * b + 3];
  }
  for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    int i, j, k;
    sh.cell(c, i, j, k);
    int ox = i < NG ? -1 : (i >= NG + nx.x ? 1 : 0);
    int oy = j < NG ? -1 : (j >= NG + nx.y ? 1 : 0);
    int oz = k < NG ? -1 : (k >= NG + nx.z ? 1 : 0);
    int si = i, sj = j, sk = k;
    bool f1 = false, f2 = false, f3 = false;
    if (bcm) {
      if (bc_image(si, ox, nx.x, lx[0] == 0, lx[0] == nbl.x - 1, bcm & 3, (bcm >> 2) & 3, f1)) ox = 0;
      if (bc_image(sj, oy, nx.y, lx[1] == 0, lx[1] == nbl.y - 1, (bcm >> 4) & 3, (bcm >> 6) & 3, f2)) oy = 0;
      if (bc_image(sk, oz, nx.z, lx[2] == 0, lx[2] == nbl.z - 1, (bcm >> 8) & 3, (bcm >> 10) & 3, f3)) oz = 0;
    }
    const int src = nb[(oz + 1) * 9 + (oy + 1) * 3 + (ox + 1)];
    if (src < 0) continue;  // source on another shard: filled by the shard unpack
    const T* srcb = U + (size_t)src * NVT * vs;
    const size_t so = ((size_t)(sk - oz * nx.z) * S2 + (sj - oy * nx.y)) * S1 + (si - ox * nx.x);
    const size_t dofs = ((size_t)k * S2 + j) * S1 + i;
    T w[NVT];
#pragma unroll
    for (int v = 0; v < NVT; ++v) w[v] = srcb[v * vs + so];
    if (f1) w[1] = -w[1];
    if (f2) w[2] = -w[2];
    if (f3) w[3] = -w[3];
#pragma unroll
    for (int v = 0; v < NVT; ++v) dstb[v * vs + dofs] = w[v];
  }
}

// Periodic meshes with an even nx1: the ghost shell's rows split into
// aligned pairs of x1-adjacent cells (the x1-ghost layers are 2 wide and the
// interior starts at an even index), and both cells of a pair come from the
// same neighbour, contiguous and in order.  Each thread moves one pair of
// every variable with one 2-element load and store (8 bytes in FP32, 16 in
// FP64): half the threads and memory instructions of the per-cell copy.
template <class T>
struct Pair;
template <>
struct Pair<float> {
  using V = float2;
};
template <>
struct Pair<double> {
  using V = double2;
};

template <class T, int NVT = NV>
__global__ void ghost_uniform_pairs_kernel(T* U, const int* __restrict__ nbr, int3 nx) {
  using V = typename Pair<T>::V;
  const int nxa[3] = {nx.x, nx.y, nx.z};
  const Shell sh(nxa);
  const int b = blockIdx.x;
  const int S1 = sh.S1, S2 = sh.S2, S3 = nx.z + 2 * NG;
  const size_t vs = (size_t)S1 * S2 * S3;
  T* dstb = U + (size_t)b * NVT * vs;
  const int* nb = nbr + 27 * b;
  const int total = sh.count() / 2;
  const int per = (total + gridDim.y - 1) / gridDim.y;
  const int c0 = blockIdx.y * per, c1 = min(total, c0 + per);
  for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    int i, j, k;
    sh.cell(2 * c, i, j, k);  // the pair's first cell; its partner is (i + 1, j, k)
    const int ox = i < NG ? -1 : (i >= NG + nx.x ? 1 : 0);
    const int oy = j < NG ? -1 : (j >= NG + nx.y ? 1 : 0);
    const int oz = k < NG ? -1 : (k >= NG + nx.z ? 1 : 0);
    const int src = nb[(oz + 1) * 9 + (oy + 1) * 3 + (ox + 1)];
    if (src < 0) continue;  // source on another shard: filled by the shard unpack
    const T* srcb = U + (size_t)src * NVT * vs;
    const size_t so = ((size_t)(k - oz * nx.z) * S2 + (j - oy * nx.y)) * S1 + (i - ox * nx.x);
    const size_t dofs = ((size_t)k * S2 + j) * S1 + i;
    V w[NVT];
#pragma unroll
    for (int v = 0; v < NVT; ++v) w[v] = *reinterpret_cast<const V*>(srcb + v * vs + so);
#pragma unroll
    for (int v = 0; v < NVT; ++v) *reinterpret_cast<V*>(dstb + v * vs + dofs) = w[v];
  }
}

template <class T, int NVT>
static cudaError_t launch_ghost_uniform_n(T* U, const int* nbr, const int nx[3], int nleaf, cudaStream_t s,
                                          const int* leaf_id, const int nb[3], int bcm) {
  const long long S1 = nx[0] + 2 * NG, S2 = nx[1] + 2 * NG, S3 = nx[2] + 2 * NG;
  const long long shell = S1 * S2 * S3 - (long long)nx[0] * nx[1] * nx[2];
  if (bcm == 0 && nx[0] % 2 == 0) {
    const long long pairs = shell / 2;
    const int chunks = (int)std::min<long long>(64, std::max<long long>(1, (pairs + 1023) / 1024));
    ghost_uniform_pairs_kernel<T, NVT><<<dim3(nleaf, chunks), 256, 0, s>>>(
        U, nbr, make_int3(nx[0], nx[1], nx[2]));
    return cudaGetLastError();
  }
  const int chunks = (int)std::min<long long>(64, std::max<long long>(1, (shell + 1023) / 1024));
  const int3 nbl = nb ? make_int3(nb[0], nb[1], nb[2]) : make_int3(1, 1, 1);
  ghost_uniform_kernel<T, NVT><<<dim3(nleaf, chunks), 256, 0, s>>>(
      U, nbr, make_int3(nx[0], nx[1], nx[2]), leaf_id, nbl, bcm);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_ghost_uniform(T* U, const int* nbr, const int nx[3], int nleaf, cudaStream_t s,
                                 const int* leaf_id, const int nb[3], int bcm, int nvar) {
  PH_RANGE("ph ghost exchange (uniform)");
  if (nleaf <= 0) return cudaSuccess;
  if (nvar == NV + 1) return launch_ghost_uniform_n<T, NV + 1>(U, nbr, nx, nleaf, s, leaf_id, nb, bcm);
  if (nvar == NV + 2) return launch_ghost_uniform_n<T, NV + 2>(U, nbr, nx, nleaf, s, leaf_id, nb, bcm);
  return launch_ghost_uniform_n<T, NV>(U, nbr, nx, nleaf, s, leaf_id, nb, bcm);
}

// --------------------------------------------------------------------------
// Composite field of a multi-level mesh (Sec. 2.1 + Sec. 3.7).  The value of
// cell (I,J,K) of level L, built from leaf interiors only:
//   covered by a leaf of level L:  that leaf's value;
//   covered by finer leaves:       mean of the 8 cells of level L+1
//                                  (restriction; summed c3 outer, c1 inner,
//                                  then x 1/8);
//   covered by a coarser leaf:     the level-(L-1) value plus +-1/4 of the
//                                  minmod-limited level-(L-1) differences in
//                                  x1, x2, x3 in that order (prolongation).
// Locations outside the domain first map to their image inside (PH_BC_*).
// Every add/multiply is an unfused round-to-nearest operation so that the
// result is reproducible operation by operation.
//
// The evaluation nests (a prolongation needs values of the next coarser
// level, which may themselves be prolonged or restricted); it is written as
// a chain of D non-inlined functions rather than a recursion, so that its
// stack is sized statically.  In a tree whose touching leaves differ by one
// level and whose blocks have at least 4 cells per axis, ghost cells need 2
// nested evaluations and new leaves at a remesh 3; the chain allows 4 and
// records an error instead of going deeper.
// --------------------------------------------------------------------------
constexpr int COMPOSITE_DEPTH = 4;

__device__ __forceinline__ long long wrapi(long long i, long long n) {
  long long r = i % n;
  return r < 0 ? r + n : r;
}

// Map a global cell index of a level whose axis has N cells into the domain
// (PH_BC_*: periodic shift, outflow clamp, reflecting mirror); returns true
// if the normal momentum must be negated.
__device__ __forceinline__ bool domain_image(long long& X, long long N, int bc_lo, int bc_hi) {
  if (X >= 0 && X < N) return false;
  const int bc = X < 0 ? bc_lo : bc_hi;
  if (bc == 0) {
    X = wrapi(X, N);
    return false;
  }
  if (bc == 1) {
    X = X < 0 ? 0 : N - 1;
    return false;
  }
  X = X < 0 ? -1 - X : 2 * N - 1 - X;
  return true;
}

template <class T>
__device__ __forceinline__ void negate_momenta(T* out, bool f1, bool f2, bool f3) {
  if (f1) out[1] = -out[1];
  if (f2) out[2] = -out[2];
  if (f3) out[3] = -out[3];
}

// Leaf covering block (b1,b2,b3) of level L (coordinates inside the domain):
// its index with its level in *lev, or -1 when finer leaves cover it.
__device__ __forceinline__ int tree_cover(const TreeView& tv, int L, long long b1, long long b2,
                                          long long b3, int* lev) {
  int node = (int)(((b3 >> L) * tv.nb[1] + (b2 >> L)) * tv.nb[0] + (b1 >> L));
  for (int d = 0;; ++d) {
    const int v = tv.node[node];
    if (v >= 0) {
      *lev = d;
      return v;
    }
    if (d == L || v == NODE_UNSET) return -1;
    const int s = L - d - 1;
    node = node_children(v) + (int)(((b1 >> s) & 1) + 2 * ((b2 >> s) & 1) + 4 * ((b3 >> s) & 1));
  }
}

template <class T, int NVT>
__device__ __forceinline__ void read_cell(const T* U, const TreeView& tv, int leaf, int li, int lj,
                                          int lk, T out[NVT]) {
  const size_t vs = (size_t)tv.S[0] * tv.S[1] * tv.S[2];
  const T* p = U + (size_t)leaf * NVT * vs + ((size_t)(lk + NG) * tv.S[1] + (lj + NG)) * tv.S[0] + (li + NG);
#pragma unroll
  for (int v = 0; v < NVT; ++v) out[v] = p[v * vs];
}

template <class T>
__device__ __forceinline__ T minmod_dev(T a, T b) {
  if (mul_rn(a, b) > T(0)) return fabs(a) < fabs(b) ? a : b;
  return T(0);
}

template <class T, int D, int NVT>
__device__ __noinline__ void composite_value(const T* U, const TreeView& tv, int L, long long I,
                                             long long J, long long K, T* out) {
  const long long N1 = (long long)tv.nb[0] * tv.nx[0] << L, N2 = (long long)tv.nb[1] * tv.nx[1] << L,
                  N3 = (long long)tv.nb[2] * tv.nx[2] << L;
  const bool f1 = domain_image(I, N1, tv.bc[0], tv.bc[1]);
  const bool f2 = domain_image(J, N2, tv.bc[2], tv.bc[3]);
  const bool f3 = domain_image(K, N3, tv.bc[4], tv.bc[5]);
  const long long b1 = I / tv.nx[0], b2 = J / tv.nx[1], b3 = K / tv.nx[2];
  int lev = 0;
  const int lf = tree_cover(tv, L, b1, b2, b3, &lev);
  if (lf >= 0 && lev == L) {
    read_cell<T, NVT>(U, tv, lf, (int)(I - b1 * tv.nx[0]), (int)(J - b2 * tv.nx[1]), (int)(K - b3 * tv.nx[2]),
              out);
    negate_momenta(out, f1, f2, f3);
    return;
  }
  if constexpr (D == 0) {
    atomicExch(tv.error, 1);
#pragma unroll
    for (int v = 0; v < NVT; ++v) out[v] = T(0);
    return;
  } else {
    if (lf >= 0) {  // coarser leaf: prolongation from level L-1
      const long long C[3] = {I >> 1, J >> 1, K >> 1};
      const long long F[3] = {I, J, K};
      T uc[NVT], acc[NVT];
      composite_value<T, D - 1, NVT>(U, tv, L - 1, C[0], C[1], C[2], uc);
#pragma unroll
      for (int v = 0; v < NVT; ++v) acc[v] = uc[v];
      for (int d = 0; d < 3; ++d) {
        long long cm[3] = {C[0], C[1], C[2]}, cp[3] = {C[0], C[1], C[2]};
        cm[d] -= 1;
        cp[d] += 1;
        T um[NVT], up[NVT];
        composite_value<T, D - 1, NVT>(U, tv, L - 1, cm[0], cm[1], cm[2], um);
        composite_value<T, D - 1, NVT>(U, tv, L - 1, cp[0], cp[1], cp[2], up);
        const T sg = (F[d] & 1) ? T(0.25) : T(-0.25);
#pragma unroll
        for (int v = 0; v < NVT; ++v)
          acc[v] = add_rn(acc[v], mul_rn(sg, minmod_dev(sub_rn(uc[v], um[v]), sub_rn(up[v], uc[v]))));
      }
#pragma unroll
      for (int v = 0; v < NVT; ++v) out[v] = acc[v];
    } else {  // finer leaves: restriction from level L+1
      T sum[NVT];
#pragma unroll
      for (int v = 0; v < NVT; ++v) sum[v] = T(0);
      for (int c3 = 0; c3 < 2; ++c3)
        for (int c2 = 0; c2 < 2; ++c2)
          for (int c1 = 0; c1 < 2; ++c1) {
            T f[NVT];
            composite_value<T, D - 1, NVT>(U, tv, L + 1, 2 * I + c1, 2 * J + c2, 2 * K + c3, f);
#pragma unroll
            for (int v = 0; v < NVT; ++v) sum[v] = add_rn(sum[v], f[v]);
          }
#pragma unroll
      for (int v = 0; v < NVT; ++v) out[v] = mul_rn(T(0.125), sum[v]);
    }
    negate_momenta(out, f1, f2, f3);
  }
}

// nbr[27 b + region]: the leaf of the same level that covers the block
// location next to leaf b in that neighbour region, or -1 (finer or coarser
// leaves, or a physical boundary).  Ghost cells of such a region are plain
// copies of that leaf's interior, the value the composite evaluation gives
// there, read directly instead of through the tree; this kernel (one CTA per
// leaf) does those copies.  The other ghost cells are listed per tree
// (leaf, shell index) and evaluated by ghost_composite_eval_kernel, one
// thread each over the whole list, so that the few leaves next to a level
// jump do not serialise their evaluations in a handful of CTAs.
template <class T, int NVT>
__global__ void ghost_composite_kernel(T* U, const TreeView tv, const int* __restrict__ leaf_id,
                                       const int* __restrict__ nbr) {
  const Shell sh(tv.nx);
  const int b = blockIdx.x;
  const int lev = leaf_id[4 * b];
  const long long o1 = (long long)leaf_id[4 * b + 1] * tv.nx[0] - NG;
  const long long o2 = (long long)leaf_id[4 * b + 2] * tv.nx[1] - NG;
  const long long o3 = (long long)leaf_id[4 * b + 3] * tv.nx[2] - NG;
  const size_t vs = (size_t)tv.S[0] * tv.S[1] * tv.S[2];
  T* dst = U + (size_t)b * NVT * vs;
  const int* nb = nbr + 27 * b;
  const int total = sh.count();
  for (int c = threadIdx.x; c < total; c += blockDim.x) {
    int i, j, k;
    sh.cell(c, i, j, k);
    const int ox = i < NG ? -1 : (i >= NG + tv.nx[0] ? 1 : 0);
    const int oy = j < NG ? -1 : (j >= NG + tv.nx[1] ? 1 : 0);
    const int oz = k < NG ? -1 : (k >= NG + tv.nx[2] ? 1 : 0);
    const int src = nb[(oz + 1) * 9 + (oy + 1) * 3 + (ox + 1)];
    if (src < 0) continue;  // evaluated through the tree (the evaluation list)
    T val[NVT];
    const T* s = U + (size_t)src * NVT * vs +
                 ((size_t)(k - oz * tv.nx[2]) * tv.S[1] + (j - oy * tv.nx[1])) * tv.S[0] + (i - ox * tv.nx[0]);
#pragma unroll
    for (int v = 0; v < NVT; ++v) val[v] = s[v * vs];
    const size_t d = ((size_t)k * tv.S[1] + j) * tv.S[0] + i;
#pragma unroll
    for (int v = 0; v < NVT; ++v) dst[v * vs + d] = val[v];
  }
}

// Ghost cells of regions without a same-level leaf: list[e] = (leaf, shell
// index), one thread each.  Most of them are one prolongation from 7 cells
// of level L-1 or one restriction of 8 cells of level L+1, every source cell
// in a leaf of its own level (or a copy of a cell of level L through a
// physical boundary).  For those the tree walks depend on the tree only, so
// they are done once per tree (ghost_recipe_kernel): the element offsets of
// the source cells and the momentum sign flips of every image.  Each
// exchange then reads the sources and combines them with the operations of
// composite_value(), in its order (ghost_composite_eval_kernel); the other
// cells take the recursive evaluation through the tree in a second launch
// (ghost_composite_tree_kernel), which keeps the recursion's stack and
// registers (212 a thread) out of the first one.
struct GhostRecipe {
  long long src[8];  // element offset of variable 0 of each source cell
  // bits 0-1 kind (0: through the tree, 1: copy, 2: prolongation,
  // 3: restriction); 2-4 parity of the cell along x1..x3 (prolongation);
  // 5-7 momentum flips of the ghost cell's own image; 8 + 3 s: flips of
  // source s
  unsigned meta;
  // bit s: source s of a prolongation is covered by finer leaves, its value
  // the mean of its 8 children (src[s] is the offset of child (0, 0, 0))
  unsigned mean;
};

template <int NVT>
__device__ __forceinline__ bool direct_source(const TreeView& tv, int L, long long I, long long J, long long K,
                                              long long& off, unsigned& flips) {
  const long long N1 = (long long)tv.nb[0] * tv.nx[0] << L, N2 = (long long)tv.nb[1] * tv.nx[1] << L,
                  N3 = (long long)tv.nb[2] * tv.nx[2] << L;
  const bool f1 = domain_image(I, N1, tv.bc[0], tv.bc[1]);
  const bool f2 = domain_image(J, N2, tv.bc[2], tv.bc[3]);
  const bool f3 = domain_image(K, N3, tv.bc[4], tv.bc[5]);
  const long long b1 = I / tv.nx[0], b2 = J / tv.nx[1], b3 = K / tv.nx[2];
  int lev = 0;
  const int lf = tree_cover(tv, L, b1, b2, b3, &lev);
  if (lf < 0 || lev != L) return false;
  const size_t vs = (size_t)tv.S[0] * tv.S[1] * tv.S[2];
  off = (long long)((size_t)lf * NVT * vs +
                    ((size_t)(K - b3 * tv.nx[2] + NG) * tv.S[1] + (J - b2 * tv.nx[1] + NG)) * tv.S[0] +
                    (I - b1 * tv.nx[0] + NG));
  flips = (f1 ? 1u : 0u) | (f2 ? 2u : 0u) | (f3 ? 4u : 0u);
  return true;
}

// A prolongation source: a cell of a leaf of its level, or (mean = true) a
// cell covered by finer leaves whose 8 children lie in one leaf of the next
// level (the restriction composite_value() takes there).
template <int NVT>
__device__ __forceinline__ bool prolong_source(const TreeView& tv, int L, long long I, long long J, long long K,
                                               long long& off, unsigned& flips, bool& mean) {
  mean = false;
  if (direct_source<NVT>(tv, L, I, J, K, off, flips)) return true;
  const long long N1 = (long long)tv.nb[0] * tv.nx[0] << L, N2 = (long long)tv.nb[1] * tv.nx[1] << L,
                  N3 = (long long)tv.nb[2] * tv.nx[2] << L;
  const bool f1 = domain_image(I, N1, tv.bc[0], tv.bc[1]);
  const bool f2 = domain_image(J, N2, tv.bc[2], tv.bc[3]);
  const bool f3 = domain_image(K, N3, tv.bc[4], tv.bc[5]);
  int lev = 0;
  if (tree_cover(tv, L, I / tv.nx[0], J / tv.nx[1], K / tv.nx[2], &lev) >= 0) return false;  // coarser
  const long long c1 = 2 * I, c2 = 2 * J, c3 = 2 * K;  // first child; the 8 share a block (nx even)
  const long long b1 = c1 / tv.nx[0], b2 = c2 / tv.nx[1], b3 = c3 / tv.nx[2];
  const int lf = tree_cover(tv, L + 1, b1, b2, b3, &lev);
  if (lf < 0 || lev != L + 1) return false;
  const size_t vs = (size_t)tv.S[0] * tv.S[1] * tv.S[2];
  off = (long long)((size_t)lf * NVT * vs +
                    ((size_t)(c3 - b3 * tv.nx[2] + NG) * tv.S[1] + (c2 - b2 * tv.nx[1] + NG)) * tv.S[0] +
                    (c1 - b1 * tv.nx[0] + NG));
  flips = (f1 ? 1u : 0u) | (f2 ? 2u : 0u) | (f3 ? 4u : 0u);
  mean = true;
  return true;
}

template <int NVT>
__global__ void ghost_recipe_kernel(const TreeView tv, const int* __restrict__ leaf_id,
                                    const int2* __restrict__ list, int n, GhostRecipe* __restrict__ out) {
  const Shell sh(tv.nx);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int2 it = list[e];
    const int b = it.x;
    int i, j, k;
    sh.cell(it.y, i, j, k);
    const int L = leaf_id[4 * b];
    long long I = (long long)leaf_id[4 * b + 1] * tv.nx[0] - NG + i;
    long long J = (long long)leaf_id[4 * b + 2] * tv.nx[1] - NG + j;
    long long K = (long long)leaf_id[4 * b + 3] * tv.nx[2] - NG + k;
    GhostRecipe R;
#pragma unroll
    for (int q = 0; q < 8; ++q) R.src[q] = 0;
    R.mean = 0u;
    bool mn = false;
    const long long N1 = (long long)tv.nb[0] * tv.nx[0] << L, N2 = (long long)tv.nb[1] * tv.nx[1] << L,
                    N3 = (long long)tv.nb[2] * tv.nx[2] << L;
    const bool f1 = domain_image(I, N1, tv.bc[0], tv.bc[1]);
    const bool f2 = domain_image(J, N2, tv.bc[2], tv.bc[3]);
    const bool f3 = domain_image(K, N3, tv.bc[4], tv.bc[5]);
    unsigned meta = ((f1 ? 1u : 0u) | (f2 ? 2u : 0u) | (f3 ? 4u : 0u)) << 5;
    const long long b1 = I / tv.nx[0], b2 = J / tv.nx[1], b3 = K / tv.nx[2];
    int lev = 0;
    const int lf = tree_cover(tv, L, b1, b2, b3, &lev);
    bool ok = true;
    unsigned fl = 0;
    if (lf >= 0 && lev == L) {  // a cell of this level (an image through a boundary)
      const size_t vs = (size_t)tv.S[0] * tv.S[1] * tv.S[2];
      R.src[0] = (long long)((size_t)lf * NVT * vs +
                             ((size_t)(K - b3 * tv.nx[2] + NG) * tv.S[1] + (J - b2 * tv.nx[1] + NG)) * tv.S[0] +
                             (I - b1 * tv.nx[0] + NG));
      meta |= 1u;
    } else if (lf >= 0) {  // prolongation: C, then C -+ e_d for d = 1, 2, 3
      const long long C[3] = {I >> 1, J >> 1, K >> 1};
      ok = direct_source<NVT>(tv, L - 1, C[0], C[1], C[2], R.src[0], fl);
      meta |= fl << 8;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        long long cm[3] = {C[0], C[1], C[2]}, cp[3] = {C[0], C[1], C[2]};
        cm[d] -= 1;
        cp[d] += 1;
        ok = ok && prolong_source<NVT>(tv, L - 1, cm[0], cm[1], cm[2], R.src[1 + 2 * d], fl, mn);
        meta |= ok ? fl << (8 + 3 * (1 + 2 * d)) : 0u;
        R.mean |= ok && mn ? 1u << (1 + 2 * d) : 0u;
        ok = ok && prolong_source<NVT>(tv, L - 1, cp[0], cp[1], cp[2], R.src[2 + 2 * d], fl, mn);
        meta |= ok ? fl << (8 + 3 * (2 + 2 * d)) : 0u;
        R.mean |= ok && mn ? 1u << (2 + 2 * d) : 0u;
      }
      meta |= 2u | (unsigned)(I & 1) << 2 | (unsigned)(J & 1) << 3 | (unsigned)(K & 1) << 4;
    } else {  // restriction of the 8 children, x1 fastest
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        ok = ok && direct_source<NVT>(tv, L + 1, 2 * I + (c & 1), 2 * J + ((c >> 1) & 1), 2 * K + (c >> 2),
                                      R.src[c], fl);
        meta |= ok ? fl << (8 + 3 * c) : 0u;
      }
      meta |= 3u;
    }
    R.meta = ok ? meta : 0u;
    out[e] = R;
  }
}

template <class T, int NVT>
__device__ __forceinline__ void recipe_source(const T* U, const TreeView& tv, size_t vs, const GhostRecipe& R,
                                              int s, T out[NVT]) {
  if ((R.mean >> s) & 1u) {  // restriction of the 8 children, x1 fastest
    const size_t p1 = 1, p2 = tv.S[0], p3 = (size_t)tv.S[0] * tv.S[1];
#pragma unroll
    for (int v = 0; v < NVT; ++v) out[v] = T(0);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const T* q = U + R.src[s] + (c & 1) * p1 + ((c >> 1) & 1) * p2 + (c >> 2) * p3;
#pragma unroll
      for (int v = 0; v < NVT; ++v) out[v] = add_rn(out[v], q[v * vs]);
    }
#pragma unroll
    for (int v = 0; v < NVT; ++v) out[v] = mul_rn(T(0.125), out[v]);
  } else {
#pragma unroll
    for (int v = 0; v < NVT; ++v) out[v] = U[R.src[s] + v * vs];
  }
  const unsigned f = R.meta >> (8 + 3 * s);
  negate_momenta(out, f & 1u, (f & 2u) != 0, (f & 4u) != 0);
}

template <class T, int NVT>
__global__ void ghost_composite_eval_kernel(T* U, const TreeView tv, const int* __restrict__ leaf_id,
                                            const int2* __restrict__ list, const GhostRecipe* __restrict__ rec,
                                            int n) {
  const Shell sh(tv.nx);
  const size_t vs = (size_t)tv.S[0] * tv.S[1] * tv.S[2];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int2 it = list[e];
    const int b = it.x;
    int i, j, k;
    sh.cell(it.y, i, j, k);
    const GhostRecipe R = rec[e];
    const unsigned kind = R.meta & 3u;
    T val[NVT];
    if (kind == 0u) continue;  // ghost_composite_tree_kernel
    {
      if (kind == 1u) {
#pragma unroll
        for (int v = 0; v < NVT; ++v) val[v] = U[R.src[0] + v * vs];
      } else if (kind == 2u) {
        T uc[NVT];
        recipe_source<T, NVT>(U, tv, vs, R, 0, uc);
#pragma unroll
        for (int v = 0; v < NVT; ++v) val[v] = uc[v];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          T um[NVT], up[NVT];
          recipe_source<T, NVT>(U, tv, vs, R, 1 + 2 * d, um);
          recipe_source<T, NVT>(U, tv, vs, R, 2 + 2 * d, up);
          const T sg = ((R.meta >> (2 + d)) & 1u) ? T(0.25) : T(-0.25);
#pragma unroll
          for (int v = 0; v < NVT; ++v)
            val[v] = add_rn(val[v], mul_rn(sg, minmod_dev(sub_rn(uc[v], um[v]), sub_rn(up[v], uc[v]))));
        }
      } else {
        T sum[NVT];
#pragma unroll
        for (int v = 0; v < NVT; ++v) sum[v] = T(0);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          T f[NVT];
          recipe_source<T, NVT>(U, tv, vs, R, c, f);
#pragma unroll
          for (int v = 0; v < NVT; ++v) sum[v] = add_rn(sum[v], f[v]);
        }
#pragma unroll
        for (int v = 0; v < NVT; ++v) val[v] = mul_rn(T(0.125), sum[v]);
      }
      const unsigned f = R.meta >> 5;
      negate_momenta(val, f & 1u, (f & 2u) != 0, (f & 4u) != 0);
    }
    T* dst = U + (size_t)b * NVT * vs + ((size_t)k * tv.S[1] + j) * tv.S[0] + i;
#pragma unroll
    for (int v = 0; v < NVT; ++v) dst[v * vs] = val[v];
  }
}

template <class T, int NVT>
__global__ void ghost_composite_tree_kernel(T* U, const TreeView tv, const int* __restrict__ leaf_id,
                                            const int2* __restrict__ list, const GhostRecipe* __restrict__ rec,
                                            int n) {
  const Shell sh(tv.nx);
  const size_t vs = (size_t)tv.S[0] * tv.S[1] * tv.S[2];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    if (rec[e].meta & 3u) continue;
    const int2 it = list[e];
    const int b = it.x;
    int i, j, k;
    sh.cell(it.y, i, j, k);
    const int lev = leaf_id[4 * b];
    const long long o1 = (long long)leaf_id[4 * b + 1] * tv.nx[0] - NG;
    const long long o2 = (long long)leaf_id[4 * b + 2] * tv.nx[1] - NG;
    const long long o3 = (long long)leaf_id[4 * b + 3] * tv.nx[2] - NG;
    T val[NVT];
    composite_value<T, COMPOSITE_DEPTH, NVT>(U, tv, lev, o1 + i, o2 + j, o3 + k, val);
    T* dst = U + (size_t)b * NVT * vs + ((size_t)k * tv.S[1] + j) * tv.S[0] + i;
#pragma unroll
    for (int v = 0; v < NVT; ++v) dst[v * vs] = val[v];
  }
}

template <class T, int NVT>
static cudaError_t launch_ghost_composite_n(T* U, const TreeView& tv, const int* leaf_id, const int* nbr,
                                           int nleaf, const int2* eval, const void* recipe, int neval,
                                           cudaStream_t s) {
  ghost_composite_kernel<T, NVT><<<nleaf, 256, 0, s>>>(U, tv, leaf_id, nbr);
  if (neval > 0) {
    const int grid = std::min((neval + 127) / 128, 152 * 16);
    ghost_composite_eval_kernel<T, NVT><<<grid, 128, 0, s>>>(U, tv, leaf_id, eval,
                                                             (const GhostRecipe*)recipe, neval);
    ghost_composite_tree_kernel<T, NVT><<<grid, 128, 0, s>>>(U, tv, leaf_id, eval,
                                                             (const GhostRecipe*)recipe, neval);
  }
  return cudaGetLastError();
}

size_t ghost_recipe_bytes() { return sizeof(GhostRecipe); }

cudaError_t launch_ghost_recipes(const TreeView& tv, const int* leaf_id, const int2* eval, int neval,
                                 void* out, cudaStream_t s, int nvar) {
  if (neval <= 0) return cudaSuccess;
  const int grid = std::min((neval + 127) / 128, 152 * 16);
  GhostRecipe* r = (GhostRecipe*)out;
  if (nvar == NV + 1)
    ghost_recipe_kernel<NV + 1><<<grid, 128, 0, s>>>(tv, leaf_id, eval, neval, r);
  else if (nvar == NV + 2)
    ghost_recipe_kernel<NV + 2><<<grid, 128, 0, s>>>(tv, leaf_id, eval, neval, r);
  else
    ghost_recipe_kernel<NV><<<grid, 128, 0, s>>>(tv, leaf_id, eval, neval, r);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_ghost_composite(T* U, const TreeView& tv, const int* leaf_id, const int* nbr,
                                   int nleaf, const int2* eval, const void* recipe, int neval, cudaStream_t s,
                                   int nvar) {
  PH_RANGE("ph ghost exchange (composite)");
  if (nleaf <= 0) return cudaSuccess;
  if (nvar == NV + 1)
    return launch_ghost_composite_n<T, NV + 1>(U, tv, leaf_id, nbr, nleaf, eval, recipe, neval, s);
  if (nvar == NV + 2)
    return launch_ghost_composite_n<T, NV + 2>(U, tv, leaf_id, nbr, nleaf, eval, recipe, neval, s);
  return launch_ghost_composite_n<T, NV>(U, tv, leaf_id, nbr, nleaf, eval, recipe, neval, s);
}

template <class T, int NVT>
__global__ void remesh_kernel(T* Unew, const int* __restrict__ leaf_id, const T* Uold,
                              const TreeView tv) {
  const int b = blockIdx.x;
  const int lev = leaf_id[4 * b];
  const int n1 = tv.nx[0], n2 = tv.nx[1], n3 = tv.nx[2];
  const long long o1 = (long long)leaf_id[4 * b + 1] * n1;
  const long long o2 = (long long)leaf_id[4 * b + 2] * n2;
  const long long o3 = (long long)leaf_id[4 * b + 3] * n3;
  const size_t vs = (size_t)tv.S[0] * tv.S[1] * tv.S[2];
  T* dst = Unew + (size_t)b * NVT * vs;
  const int total = n1 * n2 * n3;
  for (int c = threadIdx.x; c < total; c += blockDim.x) {
    const int k = c / (n1 * n2), r = c - k * n1 * n2, j = r / n1, i = r - j * n1;
    T val[NVT];
    composite_value<T, COMPOSITE_DEPTH, NVT>(Uold, tv, lev, o1 + i, o2 + j, o3 + k, val);
    const size_t d = ((size_t)(k + NG) * tv.S[1] + (j + NG)) * tv.S[0] + (i + NG);
#pragma unroll
    for (int v = 0; v < NVT; ++v) dst[v * vs + d] = val[v];
  }
}

template <class T>
cudaError_t launch_remesh(T* Unew, const int* new_leaf_id, int nnew, const T* Uold,
                          const TreeView& old_tv, cudaStream_t s, int nvar) {
  PH_RANGE("ph remesh");
  if (nnew <= 0) return cudaSuccess;
  if (nvar == NV + 1)
    remesh_kernel<T, NV + 1><<<nnew, 256, 0, s>>>(Unew, new_leaf_id, Uold, old_tv);
  else if (nvar == NV + 2)
    remesh_kernel<T, NV + 2><<<nnew, 256, 0, s>>>(Unew, new_leaf_id, Uold, old_tv);
  else
    remesh_kernel<T, NV><<<nnew, 256, 0, s>>>(Unew, new_leaf_id, Uold, old_tv);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// K5: signal-speed max for the CFL dt (Sec. 3.10), from interior cells.
// --------------------------------------------------------------------------
// SMs of the current device (read once; 1 if the query fails), for grid sizes.
static int device_sms() {
  static int nsm = 0;
  if (nsm <= 0) {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
      nsm = n;
    else
      return 1;
  }
  return nsm;
}

// One CTA per (leaf, slab of kper planes): the (j, i) cells of a plane in
// steps of the block size (positions advanced without a division per cell).
template <class T>
__global__ void __launch_bounds__(256) rate_kernel(const T* __restrict__ U, const int8_t* __restrict__ level,
                                                   const LevelGeom g, int3 nx, Phys<T> P, DevScalars* sc,
                                                   int nvar, int nsplit, int kper) {
  __shared__ double red[32];
  const int b = blockIdx.x / nsplit;
  const int ka = (blockIdx.x - b * nsplit) * kper, kb = min(nx.z, ka + kper);
  const int S1 = nx.x + 2 * NG, S2 = nx.y + 2 * NG, S3 = nx.z + 2 * NG;
  const size_t vs = (size_t)S1 * S2 * S3;
  const T* Ub = U + (size_t)b * nvar * vs;
  const int lev = level ? (int)level[b] : 0;
  const T i1 = (T)g.idx[lev][0], i2 = (T)g.idx[lev][1], i3 = (T)g.idx[lev][2];
  unsigned floors = 0;
  T m = T(0);  // running max in the data precision (widening is exact and monotonic)
  const int plane = nx.x * nx.y;
  const int dj = blockDim.x / nx.x, di = blockDim.x - dj * nx.x;
  const int jt = threadIdx.x / nx.x, it = threadIdx.x - jt * nx.x;
  for (int k = ka; k < kb; ++k) {
    int i = it, j = jt;
    for (int c = threadIdx.x; c < plane; c += blockDim.x) {
      const size_t o = ((size_t)(k + NG) * S2 + (j + NG)) * S1 + (i + NG);
      T w[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) w[v] = Ub[v * vs + o];
      cons_to_prim(w, P, floors);
      m = rate_max(m, wave_rate(w, P, i1, i2, i3));
      i += di;
      j += dj;
      if (i >= nx.x) {
        i -= nx.x;
        ++j;
      }
    }
  }
  block_max_to(&sc->wmax_bits, (double)m, red);
  if (floors) atomicAdd(&sc->floor_hits, (unsigned long long)floors);
}

template <class T>
cudaError_t launch_rate(const T* U, const int8_t* level, const LevelGeom& g, const int nx[3],
                        int nleaf, Phys<T> P, DevScalars* sc, cudaStream_t s, int nvar) {
  PH_RANGE("ph dt rate");
  if (nleaf <= 0) return cudaSuccess;
  // at least ~4 CTAs per SM: split the leaves' planes into slabs when there
  // are few leaves
  const long long want = 4LL * device_sms();
  int nsplit = (int)std::min<long long>(nx[2], std::max<long long>(1, (want + nleaf - 1) / nleaf));
  const int kper = (nx[2] + nsplit - 1) / nsplit;
  nsplit = (nx[2] + kper - 1) / kper;
  rate_kernel<T><<<(unsigned)((long long)nleaf * nsplit), 256, 0, s>>>(
      U, level, g, make_int3(nx[0], nx[1], nx[2]), P, sc, nvar, nsplit, kper);
  return cudaGetLastError();
}

__global__ void advance_kernel(DevScalars* sc, double cfl, int mode) {
  if (mode & 1) {
    sc->dt_last = sc->dt_next;
    sc->time += sc->dt_next;
    sc->cycle += 1;
  }
  if (mode & 2) {
    const double w = __longlong_as_double((long long)sc->wmax_bits);
    const double dt = cfl / w;
    sc->dt_next = dt;
    if (!isfinite(dt) || !(dt > 0.0)) sc->nonfinite = 1;
    sc->wmax_bits = 0ull;
  }
  if (mode & 4) sc->dt_last = sc->dt_next;  // a fresh state reports its first dt as the last
}

cudaError_t launch_advance(DevScalars* sc, double cfl, int mode, cudaStream_t s) {
  PH_RANGE("ph dt advance");
  advance_kernel<<<1, 1, 0, s>>>(sc, cfl, mode);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Interior <-> padded copies
// --------------------------------------------------------------------------
// One CTA per (leaf, variable, slab of kper planes): a plane is contiguous in
// the packed layout; its padded position advances without a division per cell.
template <class T>
__global__ void __launch_bounds__(256) pack_kernel(T* padded, T* packed, int3 nx, int dir, int nvar,
                                                   int nsplit, int kper) {
  const int bv = blockIdx.x / nsplit;          // leaf * nvar + variable
  const int ka = (blockIdx.x - bv * nsplit) * kper, kb = min(nx.z, ka + kper);
  const int S1 = nx.x + 2 * NG, S2 = nx.y + 2 * NG, S3 = nx.z + 2 * NG;
  const int plane = nx.x * nx.y;
  T* pv = padded + (size_t)bv * S1 * S2 * S3;  // variables of a leaf are consecutive in both layouts
  T* qv = packed + (size_t)bv * plane * nx.z;
  const int dj = blockDim.x / nx.x, di = blockDim.x - dj * nx.x;
  const int jt = threadIdx.x / nx.x, it = threadIdx.x - jt * nx.x;
  for (int k = ka; k < kb; ++k) {
    T* pk = pv + ((size_t)(k + NG) * S2 + NG) * S1 + NG;
    T* qk = qv + (size_t)k * plane;
    int i = it, j = jt;
    for (int c = threadIdx.x; c < plane; c += blockDim.x) {
      T* pp = pk + (size_t)j * S1 + i;
      if (dir == 0)
        *pp = qk[c];
      else
        qk[c] = *pp;
      i += di;
      j += dj;
      if (i >= nx.x) {
        i -= nx.x;
        ++j;
      }
    }
  }
}

template <class T>
cudaError_t launch_pack(T* padded, T* packed, const int nx[3], int nleaf, int dir, cudaStream_t s,
                        int nvar) {
  PH_RANGE("ph pack");
  if (nleaf <= 0) return cudaSuccess;
  // at least ~8 CTAs per SM: split the planes into slabs when there are
  // few leaves
  const long long units = (long long)nleaf * nvar;
  const long long want = 8LL * device_sms();
  int nsplit = (int)std::min<long long>(nx[2], std::max<long long>(1, (want + units - 1) / units));
  const int kper = (nx[2] + nsplit - 1) / nsplit;
  nsplit = (nx[2] + kper - 1) / kper;
  pack_kernel<T><<<(unsigned)(units * nsplit), 256, 0, s>>>(padded, packed, make_int3(nx[0], nx[1], nx[2]),
                                                             dir, nvar, nsplit, kper);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Conserved totals in FP64
// --------------------------------------------------------------------------
template <class T, int NVT>
__global__ void totals_block_kernel(const T* __restrict__ U, const int8_t* __restrict__ level,
                                    const LevelGeom g, int3 nx, double* partial) {
  __shared__ double red[NVT][256];
  const int b = blockIdx.x;
  const int S1 = nx.x + 2 * NG, S2 = nx.y + 2 * NG, S3 = nx.z + 2 * NG;
  const size_t vs = (size_t)S1 * S2 * S3;
  const T* Ub = U + (size_t)b * NVT * vs;
  double acc[NVT];
#pragma unroll
  for (int v = 0; v < NVT; ++v) acc[v] = 0.0;
  const int total = nx.x * nx.y * nx.z;
  for (int c = threadIdx.x; c < total; c += blockDim.x) {
    const int k = c / (nx.x * nx.y), r = c - k * nx.x * nx.y, j = r / nx.x, i = r - j * nx.x;
    const size_t o = ((size_t)(k + NG) * S2 + (j + NG)) * S1 + (i + NG);
#pragma unroll
    for (int v = 0; v < NVT; ++v) acc[v] += (double)Ub[v * vs + o];
  }
#pragma unroll
  for (int v = 0; v < NVT; ++v) red[v][threadIdx.x] = acc[v];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
#pragma unroll
      for (int v = 0; v < NVT; ++v) red[v][threadIdx.x] += red[v][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < NVT) {
    const double dv = g.vol[level ? (int)level[b] : 0];
    partial[(size_t)b * NVT + threadIdx.x] = red[threadIdx.x][0] * dv;
  }
}

__global__ void totals_final_kernel(const double* __restrict__ partial, int nleaf, double* out,
                                    int nvar) {
  const int v = threadIdx.x;
  if (v >= nvar) return;
  double s = 0.0, comp = 0.0;  // Neumaier compensated sum over leaves in order
  for (int b = 0; b < nleaf; ++b) {
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

template <class T>
cudaError_t launch_totals(const T* U, const int8_t* level, const LevelGeom& g, const int nx[3],
                          int nleaf, double* partial, double* out, cudaStream_t s, int nvar) {
  PH_RANGE("ph totals");
  const int3 n = make_int3(nx[0], nx[1], nx[2]);
  if (nleaf > 0) {
    if (nvar == NV + 1)
      totals_block_kernel<T, NV + 1><<<nleaf, 256, 0, s>>>(U, level, g, n, partial);
    else if (nvar == NV + 2)
      totals_block_kernel<T, NV + 2><<<nleaf, 256, 0, s>>>(U, level, g, n, partial);
    else
      totals_block_kernel<T, NV><<<nleaf, 256, 0, s>>>(U, level, g, n, partial);
  }
  totals_final_kernel<<<1, 32, 0, s>>>(partial, nleaf, out, nvar);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// K6: refinement indicator, max over interior cells and d of
// |rho_{+e_d} - rho_{-e_d}| / (2 rho), in FP64 (IEEE division).
// Correctly rounded division by the same positive number is monotonic, so the
// largest of a cell's three rounded quotients is the rounded quotient of its
// largest difference: one division per cell, the same bits.  (A NaN
// difference is skipped, as the comparison with the running max skips a NaN
// quotient; a non-positive denominator gives no quotient above 0 either way.)
// --------------------------------------------------------------------------
template <class T>
__global__ void indicator_kernel(const T* __restrict__ U, int3 nx, double* mb, int nvar) {
  __shared__ unsigned long long red[32];
  const int b = blockIdx.x;
  const int S1 = nx.x + 2 * NG, S2 = nx.y + 2 * NG, S3 = nx.z + 2 * NG;
  const T* r = U + (size_t)b * nvar * S1 * S2 * S3;  // density is variable 0
  double m = 0.0;
  const int total = nx.x * nx.y * nx.z;
  for (int c = threadIdx.x; c < total; c += blockDim.x) {
    const int k = c / (nx.x * nx.y), q = c - k * nx.x * nx.y, j = q / nx.x, i = q - j * nx.x;
    const size_t o = ((size_t)(k + NG) * S2 + (j + NG)) * S1 + (i + NG);
    const double den = __dmul_rn(2.0, (double)r[o]);
    const double a1 = fabs(__dsub_rn((double)r[o + 1], (double)r[o - 1]));
    const double a2 = fabs(__dsub_rn((double)r[o + S1], (double)r[o - S1]));
    const double a3 = fabs(__dsub_rn((double)r[o + (size_t)S1 * S2], (double)r[o - (size_t)S1 * S2]));
    const double g = __ddiv_rn(fmax(fmax(a1, a2), a3), den);
    if (g > m) m = g;
  }
  unsigned long long bits = (unsigned long long)__double_as_longlong(m);
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ob = __shfl_xor_sync(0xffffffffu, bits, o);
    bits = ob > bits ? ob : bits;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = bits;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long best = 0ull;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) best = red[w] > best ? red[w] : best;
    mb[b] = __longlong_as_double((long long)best);
  }
}

template <class T>
cudaError_t launch_indicator(const T* U, const int nx[3], int nleaf, double* mb, cudaStream_t s,
                             int nvar) {
  PH_RANGE("ph refinement indicator");
  if (nleaf <= 0) return cudaSuccess;
  indicator_kernel<T><<<nleaf, 256, 0, s>>>(U, make_int3(nx[0], nx[1], nx[2]), mb, nvar);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// K4: flux correction (Sec. 3.7).  A record is one face of one level-0 leaf
// whose neighbour across the face is refined.  During the stage the coarse
// leaf stored its own face flux Fc and the 4 fine leaves stored theirs; the
// coarse cell next to the face is corrected by the difference between Fc and
// the mean of the 4 fine fluxes over it, which equals replacing the flux
// before the update:  U += beta dt (Fc - <Ff>) / dx  on a high face,
//                     U -= beta dt (Fc - <Ff>) / dx  on a low face.
// One CTA per corrected coarse leaf walks its records in order (faces x1-,
// x1+, x2-, ...), so a cell on an edge of the block is corrected face by
// face, deterministically and without atomics.
// rec_face: 2*d + side (side 1 = high face).
// --------------------------------------------------------------------------
// want_rate (stage 2): afterwards, fold the signal rate of every corrected
// cell into sc->wmax_bits (the stage skipped those cells).
template <class T>
__global__ void flux_correct_kernel(T* U, const int* __restrict__ corr_leaf,
                                    const int* __restrict__ rec_beg,
                                    const int* __restrict__ rec_face, const T* __restrict__ fcc,
                                    const T* __restrict__ fcf, int3 nx,
                                    const int8_t* __restrict__ level, const LevelGeom g,
                                    double beta, DevScalars* sc, int nvar, Phys<T> P, int want_rate) {
  __shared__ double red[32];
  const int leaf = corr_leaf[blockIdx.x];
  const int lev = level[leaf];
  const int n[3] = {nx.x, nx.y, nx.z};
  const int S[3] = {nx.x + 2 * NG, nx.y + 2 * NG, nx.z + 2 * NG};
  const size_t vs = (size_t)S[0] * S[1] * S[2];
  T* Ub = U + (size_t)leaf * nvar * vs;
  for (int r = rec_beg[blockIdx.x]; r < rec_beg[blockIdx.x + 1]; ++r) {
    const int face = rec_face[r];
    const int d = face >> 1, side = face & 1;
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const int m1 = n[t1], m2 = n[t2];
    const double id = g.idx[lev][d];
    const T coef = (T)(beta * sc->dt_next * id) * (side ? T(1) : T(-1));
    const T* Fc = fcc + (size_t)r * nvar * m1 * m2;
    const T* Ff = fcf + (size_t)r * nvar * 4 * m1 * m2;
    for (int c = threadIdx.x; c < m1 * m2; c += blockDim.x) {
      const int a2 = c / m1, a1 = c - a2 * m1;
      int l[3];
      l[d] = side ? n[d] - 1 : 0;
      l[t1] = a1;
      l[t2] = a2;
      const size_t o = ((size_t)(l[2] + NG) * S[1] + (l[1] + NG)) * S[0] + (l[0] + NG);
      const int w = 2 * m1;
      for (int v = 0; v < nvar; ++v) {
        const T* f = Ff + (size_t)v * 4 * m1 * m2;
        const T fmean = T(0.25) * (f[(2 * a2) * w + 2 * a1] + f[(2 * a2) * w + 2 * a1 + 1] +
                                   f[(2 * a2 + 1) * w + 2 * a1] + f[(2 * a2 + 1) * w + 2 * a1 + 1]);
        const T fc = Fc[(size_t)v * m1 * m2 + c];
        Ub[v * vs + o] += coef * (fc - fmean);
      }
    }
    __syncthreads();
  }
  if (!want_rate) return;
  const T i1 = (T)g.idx[lev][0], i2 = (T)g.idx[lev][1], i3 = (T)g.idx[lev][2];
  unsigned floors = 0;
  double m = 0.0;
  for (int r = rec_beg[blockIdx.x]; r < rec_beg[blockIdx.x + 1]; ++r) {
    const int face = rec_face[r];
    const int d = face >> 1, side = face & 1;
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const int m1 = n[t1], m2 = n[t2];
    for (int c = threadIdx.x; c < m1 * m2; c += blockDim.x) {
      const int a2 = c / m1, a1 = c - a2 * m1;
      int l[3];
      l[d] = side ? n[d] - 1 : 0;
      l[t1] = a1;
      l[t2] = a2;
      const size_t o = ((size_t)(l[2] + NG) * S[1] + (l[1] + NG)) * S[0] + (l[0] + NG);
      T w[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) w[v] = Ub[v * vs + o];
      cons_to_prim(w, P, floors);
      m = rate_max(m, (double)wave_rate(w, P, i1, i2, i3));
    }
  }
  block_max_to(&sc->wmax_bits, m, red);
  if (floors) atomicAdd(&sc->floor_hits, (unsigned long long)floors);
}

template <class T>
cudaError_t launch_flux_correct(T* U, const int* corr_leaf, const int* rec_beg, int ncorr,
                                const int* rec_face, const T* fc_coarse, const T* fc_fine,
                                const int nx[3], const int8_t* level, const LevelGeom& g,
                                double beta, DevScalars* sc, cudaStream_t s, int nvar, Phys<T> P,
                                int want_rate) {
  PH_RANGE("ph flux correction");
  if (ncorr <= 0) return cudaSuccess;
  flux_correct_kernel<T><<<ncorr, 256, 0, s>>>(U, corr_leaf, rec_beg, rec_face, fc_coarse, fc_fine,
                                                make_int3(nx[0], nx[1], nx[2]), level, g, beta, sc,
                                                nvar, P, want_rate);
  return cudaGetLastError();
}

// explicit instantiations
#define PH_INST(T)                                                                              \
  template cudaError_t launch_ghost_uniform<T>(T*, const int*, const int*, int, cudaStream_t, \
                                              const int*, const int*, int, int);              \
  template cudaError_t launch_ghost_composite<T>(T*, const TreeView&, const int*, const int*,  \
                                                 int, const int2*, const void*, int, cudaStream_t, \
                                                 int);                                          \
  template cudaError_t launch_remesh<T>(T*, const int*, int, const T*, const TreeView&,        \
                                        cudaStream_t, int);                                     \
  template cudaError_t launch_rate<T>(const T*, const int8_t*, const LevelGeom&, const int*,   \
                                      int, Phys<T>, DevScalars*, cudaStream_t, int);            \
  template cudaError_t launch_pack<T>(T*, T*, const int*, int, int, cudaStream_t, int);         \
  template cudaError_t launch_totals<T>(const T*, const int8_t*, const LevelGeom&, const int*,  \
                                        int, double*, double*, cudaStream_t, int);              \
  template cudaError_t launch_indicator<T>(const T*, const int*, int, double*, cudaStream_t,    \
                                           int);                                                \
  template cudaError_t launch_flux_correct<T>(T*, const int*, const int*, int, const int*,      \
                                              const T*, const T*, const int*, const int8_t*,    \
                                              const LevelGeom&, double, DevScalars*,            \
                                              cudaStream_t, int, Phys<T>, int);
PH_INST(double)
PH_INST(float)
#undef PH_INST

}  // namespace ph
