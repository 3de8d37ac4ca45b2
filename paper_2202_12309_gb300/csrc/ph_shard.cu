// ph_shard.cu -- domain decomposition of a uniform mesh over shards: the
// partition, the halo plan, and the pack / unpack kernels of the exchange.
//
// The paper distributes MeshBlocks over ranks as contiguous ranges of the
// Z-ordered block list (Sec. 2.1) and fills the ghost zones of blocks whose
// neighbours live on another rank by packing buffers on the sender, sending
// them, and unpacking on the receiver (Sec. 3.7).  Here the partition is
// the same (shard s owns global leaves [s N / P, (s + 1) N / P) of the
// Z-ordered root grid), and the halo plan is resolved per ghost cell: every
// ghost cell of a shard's leaf whose source (the neighbour's interior cell
// the same-level exchange would copy, after mapping through physical
// boundaries) lies on another shard is one entry.  Entries are ordered by
// (global leaf, padded cell index) of the receiving ghost cell, on both
// sides, so a sender's list for a peer and that peer's list from the sender
// enumerate the same cells in the same order without any handshake.  One
// pack launch gathers every outgoing value of every peer into one buffer
// (peers in order, nvar values per entry), one unpack launch scatters every
// incoming value (negating the momentum component normal to a reflecting
// wall where the mapping crossed one).
#include <algorithm>
#include <array>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ph_hydro.h"
#include "ph_internal.h"
#include "ph_nvtx.h"

namespace ph {

namespace {

uint64_t morton3(int64_t a, int64_t b, int64_t c) {
  uint64_t key = 0;
  const int64_t v[3] = {a, b, c};
  for (int d = 0; d < 3; ++d)
    for (int bit = 0; bit < 21; ++bit) key |= ((uint64_t)((v[d] >> bit) & 1)) << (3 * bit + d);
  return key;
}

// Image of a ghost index along one axis across a physical boundary (the
// mapping of the exchange kernels): true if mapped.
bool bc_map(int& g, int o, int n, bool lo, bool hi, int bc_lo, int bc_hi, bool& reflect) {
  if (o < 0 && lo && bc_lo != PH_BC_PERIODIC) {
    g = bc_lo == PH_BC_OUTFLOW ? NG : 2 * NG - 1 - g;
    reflect = bc_lo == PH_BC_REFLECT;
    return true;
  }
  if (o > 0 && hi && bc_hi != PH_BC_PERIODIC) {
    g = bc_hi == PH_BC_OUTFLOW ? NG + n - 1 : 2 * (NG + n) - 1 - g;
    reflect = bc_hi == PH_BC_REFLECT;
    return true;
  }
  return false;
}

}  // namespace

int shard_plan(const ph_config& cfg, int nshards, int shard, ShardPlan* out, std::string* err) {
  if (cfg.max_level != 0) {
    *err = "sharded meshes are uniform (max_level 0)";
    return PH_ERR_INVALID;
  }
  const int nb[3] = {cfg.nb[0], cfg.nb[1], cfg.nb[2]};
  const int n[3] = {cfg.nx[0], cfg.nx[1], cfg.nx[2]};
  const long long nleaf = (long long)nb[0] * nb[1] * nb[2];
  if (nshards < 1 || shard < 0 || shard >= nshards || nshards > nleaf) {
    *err = "need 1 <= nshards <= number of blocks and 0 <= shard < nshards";
    return PH_ERR_INVALID;
  }
  ShardPlan& P = *out;
  P = ShardPlan();
  P.nshards = nshards;
  P.shard = shard;
  // global Z-order of the root grid
  std::vector<std::pair<uint64_t, int>> keys;
  keys.reserve(nleaf);
  for (int k = 0; k < nb[2]; ++k)
    for (int j = 0; j < nb[1]; ++j)
      for (int i = 0; i < nb[0]; ++i) keys.push_back({morton3(i, j, k), (k * nb[1] + j) * nb[0] + i});
  std::stable_sort(keys.begin(), keys.end());
  std::vector<int> slot_leaf(nleaf);  // root slot -> global leaf
  P.loc.resize(nleaf);
  for (long long g = 0; g < nleaf; ++g) {
    const int slot = keys[g].second;
    slot_leaf[slot] = (int)g;
    P.loc[g] = {slot % nb[0], (slot / nb[0]) % nb[1], slot / (nb[0] * nb[1])};
  }
  P.owner.resize(nleaf);
  P.first.resize(nshards + 1);
  for (int s = 0; s <= nshards; ++s) P.first[s] = (long long)s * nleaf / nshards;
  for (int s = 0; s < nshards; ++s)
    for (long long g = P.first[s]; g < P.first[s + 1]; ++g) P.owner[g] = s;
  const long long lo = P.first[shard], hi = P.first[shard + 1];
  const int S1 = n[0] + 2 * NG, S2 = n[1] + 2 * NG, S3 = n[2] + 2 * NG;
  const long long cells = (long long)S1 * S2 * S3;
  const long long bstride = (long long)(NV + cfg.nscalars) * cells;  // one padded block, every variable
  std::vector<std::vector<int64_t>> skey(nshards), ssrc(nshards), rkey(nshards), rdst(nshards);
  std::vector<std::vector<int8_t>> rflip(nshards);
  auto nbr_leaf = [&](const std::array<int, 3>& l, const int o[3]) {
    int a[3];
    for (int d = 0; d < 3; ++d) a[d] = ((l[d] + o[d]) % nb[d] + nb[d]) % nb[d];
    return slot_leaf[(a[2] * nb[1] + a[1]) * nb[0] + a[0]];
  };
  for (long long g = 0; g < nleaf; ++g) {
    const int og = P.owner[g];
    // only leaves of this shard (receiving) or touching it (sending)
    bool touch = og == shard;
    for (int t = 0; t < 27 && !touch; ++t) {
      const int o[3] = {t % 3 - 1, (t / 3) % 3 - 1, t / 9 - 1};
      touch = P.owner[nbr_leaf(P.loc[g], o)] == shard;
    }
    if (!touch) continue;
    const auto& l = P.loc[g];
    for (int k = 0; k < S3; ++k)
      for (int j = 0; j < S2; ++j)
        for (int i = 0; i < S1; ++i) {
          int o[3] = {i < NG ? -1 : (i >= NG + n[0] ? 1 : 0), j < NG ? -1 : (j >= NG + n[1] ? 1 : 0),
                      k < NG ? -1 : (k >= NG + n[2] ? 1 : 0)};
          if (o[0] == 0 && o[1] == 0 && o[2] == 0) continue;  // interior
          int s[3] = {i, j, k};
          bool f[3] = {false, false, false};
          for (int d = 0; d < 3; ++d)
            if (bc_map(s[d], o[d], n[d], l[d] == 0, l[d] == nb[d] - 1, cfg.bc[2 * d], cfg.bc[2 * d + 1], f[d]))
              o[d] = 0;
          const int src = nbr_leaf(l, o);
          const int os = P.owner[src];
          if (os == og) continue;  // filled by the owner's own exchange
          const long long dcell = ((long long)k * S2 + j) * S1 + i;
          const long long scell = ((long long)(s[2] - o[2] * n[2]) * S2 + (s[1] - o[1] * n[1])) * S1 +
                                  (s[0] - o[0] * n[0]);
          const int64_t key = (int64_t)g * cells + dcell;
          if (og == shard) {  // I receive it from os
            rkey[os].push_back(key);
            rdst[os].push_back((int64_t)(g - lo) * bstride + dcell);
            rflip[os].push_back((int8_t)((f[0] ? 1 : 0) | (f[1] ? 2 : 0) | (f[2] ? 4 : 0)));
          } else if (os == shard) {  // I send it to og
            skey[og].push_back(key);
            ssrc[og].push_back((int64_t)(src - lo) * bstride + scell);
          }
        }
  }
  P.send_off.assign(nshards + 1, 0);
  P.recv_off.assign(nshards + 1, 0);
  for (int p = 0; p < nshards; ++p) {
    P.send_off[p + 1] = P.send_off[p] + (int64_t)skey[p].size();
    P.recv_off[p + 1] = P.recv_off[p] + (int64_t)rkey[p].size();
    P.send_key.insert(P.send_key.end(), skey[p].begin(), skey[p].end());
    P.send_src.insert(P.send_src.end(), ssrc[p].begin(), ssrc[p].end());
    P.recv_key.insert(P.recv_key.end(), rkey[p].begin(), rkey[p].end());
    P.recv_dst.insert(P.recv_dst.end(), rdst[p].begin(), rdst[p].end());
    P.recv_flip.insert(P.recv_flip.end(), rflip[p].begin(), rflip[p].end());
  }
  P.lo = lo;
  P.hi = hi;
  return PH_OK;
}

// Pack: buf[e * nvar + v] = U[src[e] + v * vs] (every outgoing entry of every
// peer, peers in order).  Unpack: U[dst[e] + v * vs] = buf[e * nvar + v],
// with the momentum components named by flip[e] negated.
template <class T>
__global__ void shard_pack_kernel(const T* __restrict__ U, const long long* __restrict__ src, long long n,
                                  long long vs, int nvar, T* __restrict__ buf) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long a = src[e];
    for (int v = 0; v < nvar; ++v) buf[e * nvar + v] = U[a + v * vs];
  }
}

template <class T>
__global__ void shard_unpack_kernel(T* __restrict__ U, const long long* __restrict__ dst,
                                    const int8_t* __restrict__ flip, long long n, long long vs, int nvar,
                                    const T* __restrict__ buf) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long a = dst[e];
    const int f = flip[e];
    for (int v = 0; v < nvar; ++v) {
      T x = buf[e * nvar + v];
      if (v >= 1 && v <= 3 && ((f >> (v - 1)) & 1)) x = -x;
      U[a + v * vs] = x;
    }
  }
}

static int grid_of(long long n) {
  long long g = (n + 255) / 256;
  return (int)std::min<long long>(std::max<long long>(g, 1), 152 * 8);
}

template <class T>
cudaError_t launch_shard_pack(const T* U, const long long* src, long long n, long long vs, int nvar, T* buf,
                              cudaStream_t s) {
  PH_RANGE("ph shard pack");
  if (n <= 0) return cudaSuccess;
  shard_pack_kernel<T><<<grid_of(n), 256, 0, s>>>(U, src, n, vs, nvar, buf);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_shard_unpack(T* U, const long long* dst, const int8_t* flip, long long n, long long vs,
                                int nvar, const T* buf, cudaStream_t s) {
  PH_RANGE("ph shard unpack");
  if (n <= 0) return cudaSuccess;
  shard_unpack_kernel<T><<<grid_of(n), 256, 0, s>>>(U, dst, flip, n, vs, nvar, buf);
  return cudaGetLastError();
}

// dst[0] = max over src[0 .. n) of non-negative doubles stored as bits (the
// order of their bit patterns is the numeric order; NaN above +inf).
__global__ void shard_wmax_kernel(const unsigned long long* __restrict__ src, int n, unsigned long long* dst) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    unsigned long long m = 0;
    for (int i = 0; i < n; ++i) m = src[i] > m ? src[i] : m;
    dst[0] = m;
  }
}

cudaError_t launch_shard_wmax(const unsigned long long* src, int n, unsigned long long* dst, cudaStream_t s) {
  shard_wmax_kernel<<<1, 32, 0, s>>>(src, n, dst);
  return cudaGetLastError();
}

template cudaError_t launch_shard_pack<double>(const double*, const long long*, long long, long long, int,
                                               double*, cudaStream_t);
template cudaError_t launch_shard_pack<float>(const float*, const long long*, long long, long long, int, float*,
                                              cudaStream_t);
template cudaError_t launch_shard_unpack<double>(double*, const long long*, const int8_t*, long long, long long,
                                                 int, const double*, cudaStream_t);
template cudaError_t launch_shard_unpack<float>(float*, const long long*, const int8_t*, long long, long long,
                                                int, const float*, cudaStream_t);

}  // namespace ph

// Host-only query of the halo plan (no device work): lets a caller, or a
// test on a machine without a GPU, check what shard `shard` sends to and
// receives from `peer`.
extern "C" int ph_shard_plan(const ph_config* cfg, int32_t nshards, int32_t shard, int32_t peer,
                             int64_t* send_keys, int64_t* nsend, int64_t* recv_keys, int64_t* nrecv,
                             int64_t leaf_range[2]) {
  if (!cfg || !nsend || !nrecv) {
    ph::set_error_message("ph_shard_plan: null argument");
    return PH_ERR_INVALID;
  }
  ph::ShardPlan P;
  std::string err;
  const int rc = ph::shard_plan(*cfg, nshards, shard, &P, &err);
  if (rc) {
    ph::set_error_message(("ph_shard_plan: " + err).c_str());
    return rc;
  }
  if (peer < 0 || peer >= nshards) {
    ph::set_error_message("ph_shard_plan: peer out of range");
    return PH_ERR_INVALID;
  }
  const int64_t ns = P.send_off[peer + 1] - P.send_off[peer];
  const int64_t nr = P.recv_off[peer + 1] - P.recv_off[peer];
  const int64_t cap_s = *nsend, cap_r = *nrecv;
  *nsend = ns;
  *nrecv = nr;
  if (leaf_range) {
    leaf_range[0] = P.lo;
    leaf_range[1] = P.hi;
  }
  if (send_keys) {
    if (cap_s < ns) {
      ph::set_error_message("ph_shard_plan: send_keys too small");
      return PH_ERR_INVALID;
    }
    std::copy(P.send_key.begin() + P.send_off[peer], P.send_key.begin() + P.send_off[peer + 1], send_keys);
  }
  if (recv_keys) {
    if (cap_r < nr) {
      ph::set_error_message("ph_shard_plan: recv_keys too small");
      return PH_ERR_INVALID;
    }
    std::copy(P.recv_key.begin() + P.recv_off[peer], P.recv_key.begin() + P.recv_off[peer + 1], recv_keys);
  }
  return PH_OK;
}
