// ph_api.cu -- the C ABI (include/ph_hydro.h): mesh object, host block tree,
// device tables, the per-cycle launch sequence and its CUDA-graph capture.
//
// Host tree (arXiv:2202.12309 Sec. 2.1): root grid of nb1 x nb2 x nb3 blocks,
// each of which may split into 2^3 children, recursively up to max_level;
// leaves that touch differ by one level at most; leaves are kept in Z-order
// of their location scaled to the finest level (x1 in the lowest bit).  Leaf b's data lives in slot b of the device pools, so a remesh
// rebuilds the pool in the new order (Sec. 3.8: the tree is rebuilt first,
// then populated).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ph_hydro.h"
#include "ph_nvtx.h"
#include "ph_internal.h"
#include "ph_stage.cuh"

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(PH_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define PH_CUDA(expr)                                       \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) return cuda_fail(_e, #expr);     \
  } while (0)

struct Allocator {
  ph_alloc_fn alloc = nullptr;
  ph_free_fn release = nullptr;
  void* ctx = nullptr;
};
std::mutex g_alloc_mu;
Allocator g_alloc;

struct Leaf {
  int level;
  int64_t lx[3];
  int age;
};

// Z-order key: interleave the location scaled to level 1 (x1 lowest bit).
uint64_t zkey(const Leaf& l, int max_level) {
  uint64_t key = 0;
  for (int d = 0; d < 3; ++d) {
    const uint64_t c = (uint64_t)l.lx[d] << (max_level - l.level);
    for (int b = 0; b < 21; ++b) key |= ((c >> b) & 1ull) << (3 * b + d);
  }
  return key;
}

}  // namespace

void ph::set_error_message(const char* msg) { g_err = msg ? msg : ""; }

struct ph_mesh {
  ph_config cfg;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;  // private stream used only for graph capture
  Allocator alloc;
  int nx[3], S[3], nb[3];
  int nvar = ph::NV;        // conserved variables per cell: NV + passive scalars
  size_t block_elems = 0;  // nvar * S1 * S2 * S3
  size_t esize = 8;
  bool multi_level = false;
  // uniform periodic mesh: the stage kernels write the ghost zones of their
  // output themselves (push exchange), no separate exchange launch per stage
  bool push = false;

  std::vector<Leaf> leaf;
  std::vector<int> node;  // octree node table (ph_internal.h), host copy

  // device memory
  void* U0 = nullptr;
  void* U1 = nullptr;
  size_t pool_cap = 0;  // leaves the pools can hold
  ph::DevScalars* sc = nullptr;
  int* d_nbr = nullptr;
  int8_t* d_level = nullptr;
  int* d_node = nullptr;
  int* d_leaf_id = nullptr;
  double* d_partial = nullptr;
  double* d_totals = nullptr;
  double* d_mb = nullptr;
  size_t table_cap = 0;
  // flux correction
  int* d_face_rec = nullptr;
  int* d_fine_off = nullptr;
  int* d_corr_leaf = nullptr;
  int* d_rec_beg = nullptr;
  int* d_rec_face = nullptr;
  void* d_fcc = nullptr;
  void* d_fcf = nullptr;
  int nrec = 0, ncorr = 0;
  // multi-level: ghost cells evaluated through the tree, (leaf, shell index)
  int2* d_eval = nullptr;
  void* d_recipe = nullptr;  // per evaluated cell: source offsets resolved once per tree
  int neval = 0;
  // staging for host copies and packed device copies
  void* staging = nullptr;
  size_t staging_bytes = 0;

  cudaGraphExec_t gexec = nullptr;
  int tile[3] = {0, 0, 0};
  bool default_tile = false;  // tile[2] follows the leaf count (choose_chunk)
  bool state_set = false;
  // tensor maps of the U0 and U1 pools for TMA plane staging (tma: usable)
  CUtensorMap tm[2];
  bool tma = false;

  // domain decomposition (ph_create_shard): this mesh holds the global
  // leaves [plan.lo, plan.hi) of a uniform mesh split into plan.nshards
  int nshards = 1;
  ph::ShardPlan plan;
  int device = 0;
  long long* d_send_src = nullptr;
  long long* d_recv_dst = nullptr;
  int8_t* d_recv_flip = nullptr;
  void* d_sendbuf = nullptr;   // in-process exchange (ph_shards_step / sync)
  void* d_recvbuf = nullptr;
  unsigned long long* d_wscratch = nullptr;  // per shard + 1: the dt reduction (shard 0)
  cudaEvent_t ev = nullptr;       // the shard's pack (or its wmax copy) is done
  cudaEvent_t ev_done = nullptr;  // the shard's unpack (or dt reduction) is done

  std::vector<void*> owned;  // every device allocation, for destroy

  void* dalloc(size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (alloc.alloc) {
      p = alloc.alloc(bytes, (void*)stream, alloc.ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
      p = nullptr;
    }
    if (p) owned.push_back(p);
    return p;
  }
  void dfree(void* p) {
    if (!p) return;
    auto it = std::find(owned.begin(), owned.end(), p);
    if (it != owned.end()) owned.erase(it);
    if (alloc.release)
      alloc.release(p, (void*)stream, alloc.ctx);
    else
      cudaFree(p);
  }
  int nleaf() const { return (int)leaf.size(); }
  double dx(int d, int level) const {
    return (cfg.xmax[d] - cfg.xmin[d]) / (double)(((int64_t)nb[d] * nx[d]) << level);
  }
};

namespace {

// ---------------------------------------------------------------- tree logic

bool overlaps_static(const ph_mesh* m, const Leaf& l) {
  if (!m->cfg.static_region) return false;
  for (int d = 0; d < 3; ++d) {
    const double w = (m->cfg.xmax[d] - m->cfg.xmin[d]) / (double)((int64_t)m->nb[d] << l.level);
    const double lo = m->cfg.xmin[d] + (double)l.lx[d] * w;
    const double hi = m->cfg.xmin[d] + (double)(l.lx[d] + 1) * w;
    if (!(lo < m->cfg.static_hi[d] && hi > m->cfg.static_lo[d])) return false;
  }
  return true;
}

int root_slot(const ph_mesh* m, int64_t a, int64_t b, int64_t c) {
  return (int)((c * m->nb[1] + b) * m->nb[0] + a);
}

// Octree node table of a leaf list (entries as in ph_internal.h): false if
// the leaves overlap or leave a gap.
bool build_nodes(const std::vector<Leaf>& leaves, const int nb[3], std::vector<int>& node) {
  const size_t nroot = (size_t)nb[0] * nb[1] * nb[2];
  node.assign(nroot, ph::NODE_UNSET);
  for (size_t b = 0; b < leaves.size(); ++b) {
    const Leaf& l = leaves[b];
    const int L = l.level;
    int n = (int)((((l.lx[2] >> L) * nb[1]) + (l.lx[1] >> L)) * nb[0] + (l.lx[0] >> L));
    for (int d = 0; d < L; ++d) {
      if (node[n] >= 0) return false;  // a coarser leaf already covers it
      if (node[n] == ph::NODE_UNSET) {
        const int base = (int)node.size();
        node.resize(node.size() + 8, ph::NODE_UNSET);
        node[n] = -2 - base;
      }
      const int s = L - d - 1;
      n = ph::node_children(node[n]) +
          (int)(((l.lx[0] >> s) & 1) + 2 * ((l.lx[1] >> s) & 1) + 4 * ((l.lx[2] >> s) & 1));
    }
    if (node[n] != ph::NODE_UNSET) return false;  // overlap
    node[n] = (int)b;
  }
  for (int v : node)
    if (v == ph::NODE_UNSET) return false;  // gap
  return true;
}

// Sort leaves in Z-order and rebuild the node table.
void index_tree(ph_mesh* m) {
  const int ml = m->cfg.max_level;
  std::stable_sort(m->leaf.begin(), m->leaf.end(), [ml](const Leaf& a, const Leaf& b) {
    const uint64_t ka = zkey(a, ml), kb = zkey(b, ml);
    return ka != kb ? ka < kb : a.level < b.level;
  });
  build_nodes(m->leaf, m->nb, m->node);
}

// Leaf covering block location blk of level L (inside the domain), with its
// level in *lev; -1 when finer leaves cover it.
int cover(const ph_mesh* m, int L, const int64_t blk[3], int* lev) {
  int n = root_slot(m, blk[0] >> L, blk[1] >> L, blk[2] >> L);
  for (int d = 0;; ++d) {
    const int v = m->node[n];
    if (v >= 0) {
      *lev = d;
      return v;
    }
    if (d == L || v == ph::NODE_UNSET) return -1;
    const int s = L - d - 1;
    n = ph::node_children(v) + (int)(((blk[0] >> s) & 1) + 2 * ((blk[1] >> s) & 1) + 4 * ((blk[2] >> s) & 1));
  }
}

// Block location of level l next to blk in direction o: false across a
// physical boundary face, otherwise wrapped periodically.
bool neighbour(const ph_mesh* m, int l, const int64_t blk[3], const int o[3], int64_t out[3]) {
  for (int d = 0; d < 3; ++d) {
    int64_t x = blk[d] + o[d];
    const int64_t n = (int64_t)m->nb[d] << l;
    if (x < 0 || x >= n) {
      if (m->cfg.bc[2 * d + (x < 0 ? 0 : 1)] != PH_BC_PERIODIC) return false;
      x = (x + n) % n;
    }
    out[d] = x;
  }
  return true;
}

// New leaf list from flags (Sec. 2.1/3.8; the one-level rule of Athena++,
// which the paper defers to): +1 splits a leaf below max_level, and every
// leaf touching a splitting leaf (face, edge or corner) that is coarser than
// it splits too, repeatedly; a complete set of 8 sibling leaves all flagged
// -1 (old enough when check_age, none pinned by the static region, none
// splitting) merges unless a leaf touching their parent would then be two
// levels finer.  Returns false if nothing changes.
bool next_tree(const ph_mesh* m, const std::vector<int8_t>& flags, bool check_age,
               std::vector<Leaf>& out) {
  out.clear();
  const int n = m->nleaf();
  std::vector<char> split(n, 0), keep(n, 1);
  std::vector<int> todo;
  for (int b = 0; b < n; ++b)
    if (flags[b] == 1 && m->leaf[b].level < m->cfg.max_level) {
      split[b] = 1;
      todo.push_back(b);
    }
  while (!todo.empty()) {
    const Leaf& a = m->leaf[todo.back()];
    todo.pop_back();
    for (int q = 0; q < 27; ++q) {
      const int o[3] = {q % 3 - 1, (q / 3) % 3 - 1, q / 9 - 1};
      if (!o[0] && !o[1] && !o[2]) continue;
      int64_t nbk[3];
      if (!neighbour(m, a.level, a.lx, o, nbk)) continue;
      int lev = 0;
      const int c = cover(m, a.level, nbk, &lev);
      if (c >= 0 && lev < a.level && !split[c]) {
        split[c] = 1;
        todo.push_back(c);
      }
    }
  }
  bool changed = false;
  for (int b = 0; b < n; ++b) {
    if (!split[b]) continue;
    changed = true;
    keep[b] = 0;
    const Leaf& l = m->leaf[b];
    for (int c = 0; c < 8; ++c)
      out.push_back(Leaf{l.level + 1, {2 * l.lx[0] + (c & 1), 2 * l.lx[1] + ((c >> 1) & 1),
                                       2 * l.lx[2] + ((c >> 2) & 1)}, 0});
  }
  // merges: visit each parent once, from its first child (child index 0)
  for (int b = 0; b < n; ++b) {
    const Leaf& k = m->leaf[b];
    if (k.level == 0 || (k.lx[0] & 1) || (k.lx[1] & 1) || (k.lx[2] & 1)) continue;
    const int pl = k.level - 1;
    const int64_t P[3] = {k.lx[0] >> 1, k.lx[1] >> 1, k.lx[2] >> 1};
    int sib[8];
    bool ok = true;
    for (int c = 0; c < 8 && ok; ++c) {
      const int64_t cb[3] = {2 * P[0] + (c & 1), 2 * P[1] + ((c >> 1) & 1), 2 * P[2] + ((c >> 2) & 1)};
      int lev = 0;
      const int s = cover(m, k.level, cb, &lev);
      if (s < 0 || lev != k.level) {
        ok = false;
        break;
      }
      sib[c] = s;
      if (flags[s] != -1 || split[s] || (check_age && m->leaf[s].age < m->cfg.derefine_count) ||
          overlaps_static(m, m->leaf[s]))
        ok = false;
    }
    for (int q = 0; q < 27 && ok; ++q) {
      const int o[3] = {q % 3 - 1, (q / 3) % 3 - 1, q / 9 - 1};
      if (!o[0] && !o[1] && !o[2]) continue;
      int64_t nbk[3];
      if (!neighbour(m, pl, P, o, nbk)) continue;
      int lev = 0;
      if (cover(m, pl, nbk, &lev) >= 0) continue;  // the parent's level or coarser
      for (int c = 0; c < 8 && ok; ++c) {          // finer: the blocks touching the parent
        const int cb[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
        bool touches = true;
        for (int d = 0; d < 3; ++d)
          if ((o[d] == 1 && cb[d] != 0) || (o[d] == -1 && cb[d] != 1)) touches = false;
        if (!touches) continue;
        const int64_t fb[3] = {2 * nbk[0] + cb[0], 2 * nbk[1] + cb[1], 2 * nbk[2] + cb[2]};
        const int f = cover(m, pl + 1, fb, &lev);
        if (f < 0 || split[f]) ok = false;
      }
    }
    if (!ok) continue;
    changed = true;
    for (int c = 0; c < 8; ++c) keep[sib[c]] = 0;
    out.push_back(Leaf{pl, {P[0], P[1], P[2]}, 0});
  }
  if (!changed) return false;
  for (int b = 0; b < n; ++b)
    if (keep[b]) out.push_back(m->leaf[b]);
  return true;
}

// ---------------------------------------------------------------- device tables

// The device tables of a mesh (rebuilt whenever the tree changes).
constexpr int kTableSlots = 15;
void table_slots(ph_mesh* m, void** (&slot)[kTableSlots]) {
  void** ptrs[kTableSlots] = {(void**)&m->d_nbr, (void**)&m->d_level, (void**)&m->d_node,
                              (void**)&m->d_leaf_id, (void**)&m->d_partial, (void**)&m->d_mb,
                              (void**)&m->d_face_rec, (void**)&m->d_fine_off, (void**)&m->d_corr_leaf,
                              (void**)&m->d_rec_beg, (void**)&m->d_rec_face, (void**)&m->d_fcc,
                              (void**)&m->d_fcf, (void**)&m->d_eval, (void**)&m->d_recipe};
  for (int i = 0; i < kTableSlots; ++i) slot[i] = ptrs[i];
}

void free_tables(ph_mesh* m) {
  void** slot[kTableSlots];
  table_slots(m, slot);
  for (void** p : slot) {
    m->dfree(*p);
    *p = nullptr;
  }
}

template <class V>
int upload(ph_mesh* m, V** dst, const std::vector<V>& src) {
  *dst = (V*)m->dalloc(sizeof(V) * std::max<size_t>(src.size(), 1));
  if (!*dst) return fail(PH_ERR_OOM, "device allocation failed (tables)");
  if (!src.empty())
    PH_CUDA(cudaMemcpyAsync(*dst, src.data(), sizeof(V) * src.size(), cudaMemcpyHostToDevice,
                            m->stream));
  return PH_OK;
}

int build_tables_fresh(ph_mesh* m);
ph::TreeView tree_view(const ph_mesh* m);

// Build and upload every per-leaf table for the current tree.  The new
// tables are made beside the old ones, which are released only when every
// new one exists: on a failure (PH_ERR_OOM) the mesh keeps its old tables.
int build_tables(ph_mesh* m) {
  void** slot[kTableSlots];
  table_slots(m, slot);
  void* keep[kTableSlots];
  for (int i = 0; i < kTableSlots; ++i) {
    keep[i] = *slot[i];
    *slot[i] = nullptr;
  }
  const int nrec = m->nrec, ncorr = m->ncorr, neval = m->neval;
  const int rc = build_tables_fresh(m);
  if (rc) {
    free_tables(m);
    for (int i = 0; i < kTableSlots; ++i) *slot[i] = keep[i];
    m->nrec = nrec;
    m->ncorr = ncorr;
    m->neval = neval;
    return rc;
  }
  for (int i = 0; i < kTableSlots; ++i) m->dfree(keep[i]);
  return PH_OK;
}

int build_tables_fresh(ph_mesh* m) {
  const int n = m->nleaf();
  std::vector<int8_t> level(n);
  std::vector<int> leaf_id(4 * n), nbr(27 * n, -1);
  for (int b = 0; b < n; ++b) {
    const Leaf& l = m->leaf[b];
    level[b] = (int8_t)l.level;
    leaf_id[4 * b] = l.level;
    for (int d = 0; d < 3; ++d) leaf_id[4 * b + 1 + d] = (int)l.lx[d];
    if (!m->multi_level) {
      for (int oz = -1; oz <= 1; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
          for (int ox = -1; ox <= 1; ++ox) {
            const int64_t a = (l.lx[0] + ox + m->nb[0]) % m->nb[0];
            const int64_t bb = (l.lx[1] + oy + m->nb[1]) % m->nb[1];
            const int64_t c = (l.lx[2] + oz + m->nb[2]) % m->nb[2];
            nbr[27 * b + (oz + 1) * 9 + (oy + 1) * 3 + (ox + 1)] = m->node[root_slot(m, a, bb, c)];
          }
    } else {
      // the same-level leaf across each neighbour region, where there is one
      // (the composite ghost exchange copies those regions directly)
      for (int oz = -1; oz <= 1; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
          for (int ox = -1; ox <= 1; ++ox) {
            const int o[3] = {ox, oy, oz};
            int64_t nbk[3];
            int lev = -1;
            if (!neighbour(m, l.level, l.lx, o, nbk)) continue;  // physical boundary
            const int v = cover(m, l.level, nbk, &lev);
            if (v >= 0 && lev == l.level) nbr[27 * b + (oz + 1) * 9 + (oy + 1) * 3 + (ox + 1)] = v;
          }
    }
  }
  int rc;
  if ((rc = upload(m, &m->d_level, level))) return rc;
  if ((rc = upload(m, &m->d_leaf_id, leaf_id))) return rc;
  if ((rc = upload(m, &m->d_nbr, nbr))) return rc;
  // multi-level: the ghost cells of regions without a same-level leaf, which
  // the exchange evaluates through the tree
  m->neval = 0;
  if (m->multi_level) {
    const ph::Shell sh(m->nx);
    std::vector<int2> ev;
    for (int b = 0; b < n; ++b)
      for (int c = 0; c < sh.count(); ++c) {
        int i, j, k;
        sh.cell(c, i, j, k);
        const int ox = i < ph::NG ? -1 : (i >= ph::NG + m->nx[0] ? 1 : 0);
        const int oy = j < ph::NG ? -1 : (j >= ph::NG + m->nx[1] ? 1 : 0);
        const int oz = k < ph::NG ? -1 : (k >= ph::NG + m->nx[2] ? 1 : 0);
        if (nbr[27 * b + (oz + 1) * 9 + (oy + 1) * 3 + (ox + 1)] < 0) ev.push_back(make_int2(b, c));
      }
    if ((rc = upload(m, &m->d_eval, ev))) return rc;
    m->neval = (int)ev.size();
  }
  if ((rc = upload(m, &m->d_node, m->node))) return rc;
  if (m->multi_level) {
    m->d_recipe = m->dalloc(ph::ghost_recipe_bytes() * (size_t)std::max(m->neval, 1));
    if (!m->d_recipe) return fail(PH_ERR_OOM, "device allocation failed (tables)");
    PH_CUDA(ph::launch_ghost_recipes(tree_view(m), m->d_leaf_id, m->d_eval, m->neval, m->d_recipe, m->stream,
                                     m->nvar));
  }
  m->d_partial = (double*)m->dalloc(sizeof(double) * m->nvar * std::max(n, 1));
  m->d_mb = (double*)m->dalloc(sizeof(double) * std::max(n, 1));
  if (!m->d_partial || !m->d_mb) return fail(PH_ERR_OOM, "device allocation failed (tables)");

  // flux-correction records: one per (leaf, face) whose neighbour across the
  // face is refined one level further; face_rec holds 2 rec on the coarse
  // side and 2 rec + 1 on each of the 4 fine leaves across it
  m->nrec = 0;
  m->ncorr = 0;
  if (m->multi_level) {
    std::vector<int> face_rec(6 * n, -1), fine_off(12 * n, 0), corr_leaf, rec_beg, rec_face;
    for (int b = 0; b < n; ++b) {
      const Leaf& l = m->leaf[b];
      if (l.level >= m->cfg.max_level) continue;
      bool any = false;
      for (int d = 0; d < 3; ++d)
        for (int side = 0; side < 2; ++side) {
          int o[3] = {0, 0, 0};
          o[d] = side ? 1 : -1;
          int64_t nbk[3];
          if (!neighbour(m, l.level, l.lx, o, nbk)) continue;  // physical boundary
          int lev = 0;
          if (cover(m, l.level, nbk, &lev) >= 0) continue;    // same level or coarser
          if (!any) {
            corr_leaf.push_back(b);
            rec_beg.push_back(m->nrec);
            any = true;
          }
          const int rec = m->nrec++;
          const int face = 2 * d + side;
          face_rec[6 * b + face] = 2 * rec;
          rec_face.push_back(face);
          // the 4 finer leaves adjacent to this face, on their opposite face
          const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
          for (int c = 0; c < 8; ++c) {
            const int cb[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
            if (cb[d] != (side ? 0 : 1)) continue;
            const int64_t fb[3] = {2 * nbk[0] + cb[0], 2 * nbk[1] + cb[1], 2 * nbk[2] + cb[2]};
            int fl = 0;
            const int kid = cover(m, l.level + 1, fb, &fl);
            if (kid < 0 || fl != l.level + 1)
              return fail(PH_ERR_STATE, "build_tables: leaves more than one level apart touch");
            const int kface = 2 * d + (1 - side);
            face_rec[6 * kid + kface] = 2 * rec + 1;
            fine_off[12 * kid + 2 * kface] = cb[t1];
            fine_off[12 * kid + 2 * kface + 1] = cb[t2];
          }
        }
    }
    rec_beg.push_back(m->nrec);
    m->ncorr = (int)corr_leaf.size();
    if ((rc = upload(m, &m->d_face_rec, face_rec))) return rc;
    if ((rc = upload(m, &m->d_fine_off, fine_off))) return rc;
    if ((rc = upload(m, &m->d_corr_leaf, corr_leaf))) return rc;
    if ((rc = upload(m, &m->d_rec_beg, rec_beg))) return rc;
    if ((rc = upload(m, &m->d_rec_face, rec_face))) return rc;
    const int nmax = std::max(m->nx[0], std::max(m->nx[1], m->nx[2]));
    const size_t face_elems = (size_t)m->nvar * nmax * nmax;
    m->d_fcc = m->dalloc(m->esize * face_elems * std::max(m->nrec, 1));
    m->d_fcf = m->dalloc(m->esize * face_elems * 4 * std::max(m->nrec, 1));
    if (!m->d_fcc || !m->d_fcf) return fail(PH_ERR_OOM, "device allocation failed (flux records)");
  }
  return PH_OK;
}

// (Re)build the tensor maps after the pools change.
void build_tmaps(ph_mesh* m) {
  m->tma = ph::stage_tma_wanted() &&
           ph::make_stage_tmap(&m->tm[0], m->U0, m->esize, m->S, (int)m->pool_cap, m->tile[0], m->tile[1],
                               m->nvar) &&
           ph::make_stage_tmap(&m->tm[1], m->U1, m->esize, m->S, (int)m->pool_cap, m->tile[0], m->tile[1],
                               m->nvar);
  if (!m->tma && ph::stage_pair_tile(m->tile[0], m->tile[1])) {
    // the paired kernel needs TMA staging: fall back to the 16 x 16 tile
    m->tile[0] = 16;
    m->tile[1] = 16;
    build_tmaps(m);
  }
}

const CUtensorMap* tmap_for(const ph_mesh* m, int stage) {
  return m->tma ? &m->tm[stage == 1 ? 0 : 1] : nullptr;
}

int ensure_pools(ph_mesh* m, int n) {
  if ((size_t)n <= m->pool_cap && m->U0) return PH_OK;
  m->dfree(m->U0);
  m->dfree(m->U1);
  m->U0 = m->U1 = nullptr;
  const size_t bytes = m->esize * m->block_elems * (size_t)std::max(n, 1);
  m->U0 = m->dalloc(bytes);
  m->U1 = m->dalloc(bytes);
  if (!m->U0 || !m->U1) return fail(PH_ERR_OOM, "device allocation failed (state pools)");
  PH_CUDA(cudaMemsetAsync(m->U0, 0, bytes, m->stream));
  PH_CUDA(cudaMemsetAsync(m->U1, 0, bytes, m->stream));
  m->pool_cap = (size_t)std::max(n, 1);
  build_tmaps(m);
  return PH_OK;
}

int ensure_staging(ph_mesh* m, size_t bytes) {
  if (bytes <= m->staging_bytes) return PH_OK;
  m->dfree(m->staging);
  m->staging = m->dalloc(bytes);
  if (!m->staging) {
    m->staging_bytes = 0;
    return fail(PH_ERR_OOM, "device allocation failed (staging)");
  }
  m->staging_bytes = bytes;
  return PH_OK;
}

ph::TreeView tree_view(const ph_mesh* m) {
  ph::TreeView tv;
  tv.node = m->d_node;
  tv.error = m->sc ? &m->sc->tree_error : nullptr;
  for (int d = 0; d < 3; ++d) {
    tv.nb[d] = m->nb[d];
    tv.nx[d] = m->nx[d];
    tv.S[d] = m->S[d];
  }
  for (int f = 0; f < 6; ++f) tv.bc[f] = m->cfg.bc[f];
  return tv;
}

// The six faces' boundary kinds packed 2 bits each (0: periodic everywhere).
int bc_mask(const ph_mesh* m) {
  int b = 0;
  for (int f = 0; f < 6; ++f) b |= (m->cfg.bc[f] & 3) << (2 * f);
  return b;
}

template <class T>
ph::Phys<T> phys(const ph_mesh* m) {
  ph::Phys<T> P;
  P.gamma = (T)m->cfg.gamma;
  P.gm1 = (T)(m->cfg.gamma - 1.0);
  P.igm1 = (T)(1.0 / (m->cfg.gamma - 1.0));
  P.dfloor = (T)m->cfg.dfloor;
  P.pfloor = (T)m->cfg.pfloor;
  return P;
}

void inv_dx(const ph_mesh* m, double idx[ph::MAXLEV + 1][3]) {
  for (int l = 0; l <= ph::MAXLEV; ++l)
    for (int d = 0; d < 3; ++d) idx[l][d] = 1.0 / m->dx(d, l);
}

ph::LevelGeom level_geom(const ph_mesh* m) {
  ph::LevelGeom g;
  inv_dx(m, g.idx);
  for (int l = 0; l <= ph::MAXLEV; ++l) g.vol[l] = m->dx(0, l) * m->dx(1, l) * m->dx(2, l);
  return g;
}

template <class T>
int fill_ghosts_t(ph_mesh* m, T* U) {
  if (m->multi_level) {
    PH_CUDA(ph::launch_ghost_composite<T>(U, tree_view(m), m->d_leaf_id, m->d_nbr, m->nleaf(), m->d_eval,
                                          m->d_recipe, m->neval, m->stream, m->nvar));
  } else {
    PH_CUDA(ph::launch_ghost_uniform<T>(U, m->d_nbr, m->nx, m->nleaf(), m->stream,
                                        m->d_leaf_id, m->nb, bc_mask(m), m->nvar));
  }
  return PH_OK;
}

template <class T>
ph::StageArgs<T> stage_args(ph_mesh* m, int stage) {
  ph::StageArgs<T> a;
  std::memset(&a, 0, sizeof(a));
  a.Uin = (const T*)(stage == 1 ? m->U0 : m->U1);
  a.U0 = (const T*)m->U0;
  a.Uout = (T*)(stage == 1 ? m->U1 : m->U0);
  a.level = m->d_level;
  inv_dx(m, a.idx);
  for (int d = 0; d < 3; ++d) {
    a.nx[d] = m->nx[d];
    a.S[d] = m->S[d];
  }
  a.ntile[0] = (m->nx[0] + m->tile[0] - 1) / m->tile[0];
  a.ntile[1] = (m->nx[1] + m->tile[1] - 1) / m->tile[1];
  a.ntile[2] = (m->nx[2] + m->tile[2] - 1) / m->tile[2];
  a.KC = m->tile[2];
  a.nleaf = m->nleaf();
  a.stage = stage;
  a.want_rate = stage == 2 ? 1 : 0;
  a.P = phys<T>(m);
  a.sc = m->sc;
  a.nvar = m->nvar;
  a.nbr = m->push ? m->d_nbr : nullptr;
  a.pair = ph::stage_pair_kernel(sizeof(T) == 4, m->tma, m->nvar, m->multi_level, m->tile, m->nx) ? 1 : 0;
  if (m->multi_level && m->nrec > 0) {
    a.face_rec = m->d_face_rec;
    a.fc_coarse = (T*)m->d_fcc;
    a.fc_fine = (T*)m->d_fcf;
    a.fine_off = m->d_fine_off;
  }
  return a;
}

// New dt from the current state (K5 + bookkeeping), without committing a cycle.
template <class T>
int refresh_dt_t(ph_mesh* m) {
  PH_CUDA(ph::launch_rate<T>((const T*)m->U0, m->d_level, level_geom(m), m->nx, m->nleaf(), phys<T>(m), m->sc,
                             m->stream, m->nvar));
  PH_CUDA(ph::launch_advance(m->sc, m->cfg.cfl, 2, m->stream));
  return PH_OK;
}

// Enqueue one uniform-mesh cycle: stage, exchange, stage, exchange, dt
// (the exchanges are part of the stages on periodic meshes: 3 launches).
template <class T>
int enqueue_uniform_cycle(ph_mesh* m, cudaStream_t s) {
  const ph::StageArgs<T> a1 = stage_args<T>(m, 1);
  PH_CUDA(ph::launch_stage<T>(a1, m->tile[0], m->tile[1], s, tmap_for(m, 1)));
  if (!m->push)
    PH_CUDA(ph::launch_ghost_uniform<T>((T*)m->U1, m->d_nbr, m->nx, m->nleaf(), s,
                                        m->d_leaf_id, m->nb, bc_mask(m), m->nvar));
  const ph::StageArgs<T> a2 = stage_args<T>(m, 2);
  PH_CUDA(ph::launch_stage<T>(a2, m->tile[0], m->tile[1], s, tmap_for(m, 2)));
  if (!m->push)
    PH_CUDA(ph::launch_ghost_uniform<T>((T*)m->U0, m->d_nbr, m->nx, m->nleaf(), s,
                                        m->d_leaf_id, m->nb, bc_mask(m), m->nvar));
  PH_CUDA(ph::launch_advance(m->sc, m->cfg.cfl, 3, s));
  return PH_OK;
}

void drop_graph(ph_mesh* m) {
  if (m->gexec) {
    cudaGraphExecDestroy(m->gexec);
    m->gexec = nullptr;
  }
}

template <class T>
int capture_graph(ph_mesh* m) {
  drop_graph(m);
  PH_CUDA(cudaStreamBeginCapture(m->cap, cudaStreamCaptureModeThreadLocal));
  int rc = enqueue_uniform_cycle<T>(m, m->cap);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(m->cap, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&m->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    m->gexec = nullptr;
    return cuda_fail(e, "cudaGraphInstantiate");
  }
  return PH_OK;
}

// Default tiles: the x3 chunk depth (the planes one CTA marches: 16, 8 or 4
// of them) that minimises a model of the stage time, the number of whole
// waves of resident CTAs times (planes + 1.5): besides its planes a chunk
// stages and converts 4 halo planes and computes the x3 slope and flux below
// its first plane, about one and a half planes of work.  A shorter chunk is
// taken only when the model gains 3% or more.  Measured cases it reproduces:
// 960 leaves of 16^3 (two-level blast) 5% faster per cycle in 8-plane chunks,
// 2368 leaves of 16^3 (three-level Kelvin-Helmholtz) 2% slower in them,
// 64^3 zones in 32^3 blocks fastest in 4-plane chunks, 16 planes on the 256^3
// meshes.  Re-evaluated when a remesh changes the leaf count.
void choose_chunk(ph_mesh* m) {
  const int full = m->nx[2] >= 32 ? 16 : m->nx[2];
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
    nsm = 152;
  const bool fp32 = m->esize == 4, tma = ph::stage_tma_wanted();
  const bool pair = ph::stage_pair_kernel(fp32, tma, m->nvar, m->multi_level, m->tile, m->nx);
  int per_sm = fp32 ? ph::stage_ctas_per_sm<float>(m->tile[0], m->tile[1], m->nvar, pair, tma)
                    : ph::stage_ctas_per_sm<double>(m->tile[0], m->tile[1], m->nvar, pair, tma);
  const long long slots = (long long)std::max(per_sm, 1) * nsm;
  const long long cols = (long long)std::max(m->nleaf(), 1) * ((m->nx[0] + m->tile[0] - 1) / m->tile[0]) *
                         ((m->nx[1] + m->tile[1] - 1) / m->tile[1]);
  int best_kc = full;
  double best = 0.0;
  for (int kc = full; kc >= 4 || kc == full; kc = (kc + 1) / 2) {
    const long long n = cols * ((m->nx[2] + kc - 1) / kc);
    const double cost = (double)((n + slots - 1) / slots) * (std::min(kc, m->nx[2]) + 1.5);
    if (kc == full || cost < 0.97 * best) {
      best = cost;
      best_kc = kc;
    }
    if (kc <= 1) break;
  }
  m->tile[2] = best_kc;
}

template <class T>
int remesh_t(ph_mesh* m, std::vector<Leaf>& nl);

// One multi-level cycle (host-driven; flux correction after each stage).
template <class T>
int multi_level_cycle(ph_mesh* m) {
  // dt of this cycle: set by set_state, a refinement, a load, the previous
  // cycle's stage 2 (folded signal rates) or the remesh after it
  int rc;
  const ph::LevelGeom geom = level_geom(m);
  for (int stage = 1; stage <= 2; ++stage) {
    const ph::StageArgs<T> a = stage_args<T>(m, stage);
    PH_CUDA(ph::launch_stage<T>(a, m->tile[0], m->tile[1], m->stream, tmap_for(m, stage)));
    T* out = (T*)(stage == 1 ? m->U1 : m->U0);
    PH_CUDA(ph::launch_flux_correct<T>(out, m->d_corr_leaf, m->d_rec_beg, m->ncorr, m->d_rec_face,
                                       (const T*)m->d_fcc, (const T*)m->d_fcf, m->nx, m->d_level, geom,
                                       stage == 1 ? 1.0 : 0.5, m->sc, m->stream, m->nvar, phys<T>(m),
                                       stage == 2 ? 1 : 0));
    if ((rc = fill_ghosts_t<T>(m, out))) return rc;
  }
  // commit the cycle; the next dt from the rates stage 2 and the correction
  // folded (recomputed below on the new mesh if the tree changes)
  PH_CUDA(ph::launch_advance(m->sc, m->cfg.cfl, 3, m->stream));
  for (auto& l : m->leaf) l.age += 1;
  if (m->cfg.adaptive) {
    std::vector<int8_t> flags;
    std::vector<double> mb;
    PH_CUDA(ph::launch_indicator<T>((const T*)m->U0, m->nx, m->nleaf(), m->d_mb, m->stream, m->nvar));
    mb.resize(m->nleaf());
    PH_CUDA(cudaMemcpyAsync(mb.data(), m->d_mb, sizeof(double) * mb.size(), cudaMemcpyDeviceToHost,
                            m->stream));
    PH_CUDA(cudaStreamSynchronize(m->stream));
    flags.assign(m->nleaf(), 0);
    for (int b = 0; b < m->nleaf(); ++b) {
      const Leaf& l = m->leaf[b];
      if (mb[b] > m->cfg.refine_tol && l.level < m->cfg.max_level)
        flags[b] = 1;
      else if (mb[b] < m->cfg.derefine_tol && l.level > 0 && !overlaps_static(m, l))
        flags[b] = -1;
    }
    std::vector<Leaf> nl;
    if (next_tree(m, flags, true, nl)) {
      if ((rc = remesh_t<T>(m, nl))) return rc;
      if ((rc = refresh_dt_t<T>(m))) return rc;
    }
  }
  return PH_OK;
}

// Replace the tree by `nl` and move the data: each new leaf's interior is the
// old mesh's composite field (prolongation for new children, restriction for
// merged parents, copy otherwise), then ghosts are refilled.
template <class T>
int remesh_t(ph_mesh* m, std::vector<Leaf>& nl) {
  PH_RANGE("ph remesh (tree and data)");
  int rc;
  std::vector<Leaf> old = m->leaf;
  m->leaf = nl;
  index_tree(m);  // sorts the new leaves; host tables now describe the new tree
  const int nnew = m->nleaf();
  std::vector<int> leaf_id(4 * nnew);
  for (int b = 0; b < nnew; ++b) {
    leaf_id[4 * b] = m->leaf[b].level;
    for (int d = 0; d < 3; ++d) leaf_id[4 * b + 1 + d] = (int)m->leaf[b].lx[d];
  }
  // the old device tables and pool stay valid until the copy is enqueued
  ph::TreeView old_tv = tree_view(m);
  int* d_new_id = nullptr;
  const size_t bytes = m->esize * m->block_elems * (size_t)std::max(nnew, 1);
  void* U0n = nullptr;
  void* U1n = nullptr;
  rc = upload(m, &d_new_id, leaf_id);
  if (!rc) {
    U0n = m->dalloc(bytes);
    U1n = U0n ? m->dalloc(bytes) : nullptr;
    if (!U1n) rc = fail(PH_ERR_OOM, "device allocation failed (remesh)");
  }
  if (rc) {  // nothing has moved yet: give back what was taken, keep the old tree
    m->dfree(U0n);
    m->dfree(U1n);
    m->dfree(d_new_id);
    m->leaf = old;
    index_tree(m);
    return rc;
  }
  PH_CUDA(cudaMemsetAsync(U0n, 0, bytes, m->stream));
  PH_CUDA(cudaMemsetAsync(U1n, 0, bytes, m->stream));
  PH_CUDA(ph::launch_remesh<T>((T*)U0n, d_new_id, nnew, (const T*)m->U0, old_tv, m->stream, m->nvar));
  PH_CUDA(cudaStreamSynchronize(m->stream));
  m->dfree(d_new_id);
  if ((rc = build_tables(m))) {  // the old tables, pools and tree stay as they were
    m->dfree(U0n);
    m->dfree(U1n);
    m->leaf = old;
    index_tree(m);
    return rc;
  }
  m->dfree(m->U0);
  m->dfree(m->U1);
  m->U0 = U0n;
  m->U1 = U1n;
  m->pool_cap = (size_t)std::max(nnew, 1);
  build_tmaps(m);
  if (m->default_tile) choose_chunk(m);
  if ((rc = fill_ghosts_t<T>(m, (T*)m->U0))) return rc;
  drop_graph(m);
  return PH_OK;
}

template <class T>
int step_t(ph_mesh* m, int n) {
  int rc;
  if (m->multi_level) {
    for (int c = 0; c < n; ++c)
      if ((rc = multi_level_cycle<T>(m))) return rc;
    return PH_OK;
  }
  if (!m->gexec)
    if ((rc = capture_graph<T>(m))) return rc;
  PH_RANGE("ph cycle graph replays");
  for (int c = 0; c < n; ++c) PH_CUDA(cudaGraphLaunch(m->gexec, m->stream));
  return PH_OK;
}

template <class T>
int profile_t(ph_mesh* m, int n, double* ms, int nslots) {
  cudaEvent_t ev[6];
  for (int e = 0; e < 6; ++e) PH_CUDA(cudaEventCreate(&ev[e]));
  double acc[5] = {0, 0, 0, 0, 0};
  int rc = PH_OK;
  for (int c = 0; c < n && !rc; ++c) {
    const ph::StageArgs<T> a1 = stage_args<T>(m, 1);
    const ph::StageArgs<T> a2 = stage_args<T>(m, 2);
    cudaError_t e = cudaEventRecord(ev[0], m->stream);
    if (!e) e = ph::launch_stage<T>(a1, m->tile[0], m->tile[1], m->stream, tmap_for(m, 1));
    if (!e) e = cudaEventRecord(ev[1], m->stream);
    if (!e && !m->push) e = ph::launch_ghost_uniform<T>((T*)m->U1, m->d_nbr, m->nx, m->nleaf(), m->stream, m->d_leaf_id, m->nb, bc_mask(m), m->nvar);
    if (!e) e = cudaEventRecord(ev[2], m->stream);
    if (!e) e = ph::launch_stage<T>(a2, m->tile[0], m->tile[1], m->stream, tmap_for(m, 2));
    if (!e) e = cudaEventRecord(ev[3], m->stream);
    if (!e && !m->push) e = ph::launch_ghost_uniform<T>((T*)m->U0, m->d_nbr, m->nx, m->nleaf(), m->stream, m->d_leaf_id, m->nb, bc_mask(m), m->nvar);
    if (!e) e = cudaEventRecord(ev[4], m->stream);
    if (!e) e = ph::launch_advance(m->sc, m->cfg.cfl, 3, m->stream);
    if (!e) e = cudaEventRecord(ev[5], m->stream);
    if (!e) e = cudaEventSynchronize(ev[5]);
    for (int s = 0; s < 5 && !e; ++s) {
      float t = 0.f;
      e = cudaEventElapsedTime(&t, ev[s], ev[s + 1]);
      acc[s] += t;
    }
    if (e) rc = cuda_fail(e, "profile_cycles");
  }
  for (int e = 0; e < 6; ++e) cudaEventDestroy(ev[e]);
  for (int s = 0; s < nslots && s < 5; ++s) ms[s] = acc[s];
  return rc;
}

template <class T>
int set_state_t(ph_mesh* m, const void* U, int on_device, int async = 0) {
  int rc;
  const size_t count = (size_t)m->nleaf() * m->nvar * m->nx[0] * m->nx[1] * m->nx[2];
  T* packed;
  if (on_device) {
    packed = (T*)U;
  } else {
    if ((rc = ensure_staging(m, count * sizeof(T)))) return rc;
    packed = (T*)m->staging;
    PH_CUDA(cudaMemcpyAsync(packed, U, count * sizeof(T), cudaMemcpyHostToDevice, m->stream));
  }
  PH_CUDA(ph::launch_pack<T>((T*)m->U0, packed, m->nx, m->nleaf(), 0, m->stream, m->nvar));
  if ((rc = fill_ghosts_t<T>(m, (T*)m->U0))) return rc;
  PH_CUDA(cudaMemsetAsync(m->sc, 0, sizeof(ph::DevScalars), m->stream));
  if ((rc = refresh_dt_t<T>(m))) return rc;
  // the first dt is reported as the "last" dt until a cycle runs
  PH_CUDA(ph::launch_advance(m->sc, m->cfg.cfl, 4, m->stream));
  if (!async) PH_CUDA(cudaStreamSynchronize(m->stream));
  m->state_set = true;
  return PH_OK;
}

template <class T>
int get_state_t(ph_mesh* m, void* U, int on_device, int async = 0) {
  int rc;
  const size_t count = (size_t)m->nleaf() * m->nvar * m->nx[0] * m->nx[1] * m->nx[2];
  T* packed;
  if (on_device) {
    packed = (T*)U;
  } else {
    if ((rc = ensure_staging(m, count * sizeof(T)))) return rc;
    packed = (T*)m->staging;
  }
  PH_CUDA(ph::launch_pack<T>((T*)m->U0, packed, m->nx, m->nleaf(), 1, m->stream, m->nvar));
  if (!on_device)
    PH_CUDA(cudaMemcpyAsync(U, packed, count * sizeof(T), cudaMemcpyDeviceToHost, m->stream));
  if (!async) PH_CUDA(cudaStreamSynchronize(m->stream));
  return PH_OK;
}

template <class T>
int totals_t(ph_mesh* m, double* out) {
  PH_CUDA(ph::launch_totals<T>((const T*)m->U0, m->d_level, level_geom(m), m->nx, m->nleaf(), m->d_partial,
                               m->d_totals, m->stream, m->nvar));
  PH_CUDA(cudaMemcpyAsync(out, m->d_totals, m->nvar * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  PH_CUDA(cudaStreamSynchronize(m->stream));
  return PH_OK;
}

template <class T>
int tag_t(ph_mesh* m, int8_t* flags, double* mb) {
  PH_CUDA(ph::launch_indicator<T>((const T*)m->U0, m->nx, m->nleaf(), m->d_mb, m->stream, m->nvar));
  std::vector<double> h(m->nleaf());
  PH_CUDA(cudaMemcpyAsync(h.data(), m->d_mb, sizeof(double) * h.size(), cudaMemcpyDeviceToHost,
                          m->stream));
  PH_CUDA(cudaStreamSynchronize(m->stream));
  for (int b = 0; b < m->nleaf(); ++b) {
    const Leaf& l = m->leaf[b];
    int8_t f = 0;
    if (h[b] > m->cfg.refine_tol && l.level < m->cfg.max_level)
      f = 1;
    else if (h[b] < m->cfg.derefine_tol && l.level > 0 && !overlaps_static(m, l))
      f = -1;
    if (flags) flags[b] = f;
    if (mb) mb[b] = h[b];
  }
  return PH_OK;
}

// One uniform-mesh cycle with a prescribed dt (written into the device
// scalars before the captured cycle runs).
template <class T>
int cycle_fixed_dt_t(ph_mesh* m, double dt) {
  int rc;
  if (!m->gexec)
    if ((rc = capture_graph<T>(m))) return rc;
  PH_CUDA(cudaMemcpyAsync(&m->sc->dt_next, &dt, sizeof(double), cudaMemcpyHostToDevice, m->stream));
  PH_CUDA(cudaGraphLaunch(m->gexec, m->stream));
  PH_CUDA(cudaStreamSynchronize(m->stream));  // dt lives on this stack frame
  return PH_OK;
}

#define DISPATCH(m, fn, ...) \
  ((m)->cfg.precision == PH_FP32 ? fn<float>(__VA_ARGS__) : fn<double>(__VA_ARGS__))

bool valid_tile(const ph_config* c, const int t[3]) {
  if (t[2] < 1 || t[2] > c->nx[2]) return false;
  if (c->nscalars > 0) return ph::stage_scalar_tile(t[0], t[1]);
  if (ph::stage_pair_tile(t[0], t[1]))
    return c->precision == PH_FP32 && c->max_level == 0 && c->nx[0] % t[0] == 0 &&
           c->nx[1] % t[1] == 0;
  return ph::stage_tile_supported(t[0], t[1]);
}

}  // namespace

// ============================================================== adjoint access

namespace ph {


void* mesh_alloc(ph_mesh* m, size_t bytes) { return m->dalloc(bytes); }
void mesh_free(ph_mesh* m, void* p) { m->dfree(p); }

int mesh_access(ph_mesh* m, MeshAccess* out) {
  if (m->multi_level) return fail(PH_ERR_INVALID, "adjoint: uniform meshes only");
  if (m->nshards > 1) return fail(PH_ERR_INVALID, "adjoint: not on a shard of a decomposed mesh");
  if (bc_mask(m)) return fail(PH_ERR_INVALID, "adjoint: periodic meshes only");
  if (m->nvar != ph::NV) return fail(PH_ERR_INVALID, "adjoint: meshes without passive scalars only");
  out->U0 = m->U0;
  out->U1 = m->U1;
  out->nbr = m->d_nbr;
  out->sc = m->sc;
  out->stream = m->stream;
  for (int d = 0; d < 3; ++d) {
    out->nx[d] = m->nx[d];
    out->idx[d] = 1.0 / m->dx(d, 0);
  }
  out->nleaf = m->nleaf();
  out->block_elems = m->block_elems;
  out->precision = m->cfg.precision;
  out->gamma = m->cfg.gamma;
  out->dfloor = m->cfg.dfloor;
  out->pfloor = m->cfg.pfloor;
  return PH_OK;
}

int mesh_set_state(ph_mesh* m, const void* U, int on_device) {
  return DISPATCH(m, set_state_t, m, U, on_device);
}

int mesh_cycle_fixed_dt(ph_mesh* m, double dt) { return DISPATCH(m, cycle_fixed_dt_t, m, dt); }

// One cycle with the dt read from device memory (stream-ordered, no host
// synchronisation): the cycle graph runs on the dt the copy leaves in place.
int mesh_cycle_device_dt(ph_mesh* m, const double* d_dt) {
  if (!m->gexec) {
    const int rc = DISPATCH(m, capture_graph, m);
    if (rc) return rc;
  }
  PH_CUDA(cudaMemcpyAsync(&m->sc->dt_next, d_dt, sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
  PH_CUDA(cudaGraphLaunch(m->gexec, m->stream));
  return PH_OK;
}

// One CFL cycle; its dt is copied to device memory d_dt (stream-ordered).
int mesh_cycle_record_dt(ph_mesh* m, double* d_dt) {
  const int rc = DISPATCH(m, step_t, m, 1);
  if (rc) return rc;
  PH_CUDA(cudaMemcpyAsync(d_dt, &m->sc->dt_last, sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
  return PH_OK;
}

int mesh_cycle_read_dt(ph_mesh* m, double* dt) {
  int rc = DISPATCH(m, step_t, m, 1);
  if (rc) return rc;
  DevScalars hs;
  PH_CUDA(cudaMemcpyAsync(&hs, m->sc, sizeof(hs), cudaMemcpyDeviceToHost, m->stream));
  PH_CUDA(cudaStreamSynchronize(m->stream));
  *dt = hs.dt_last;
  return PH_OK;
}

}  // namespace ph

// ============================================================== C ABI

extern "C" {

int ph_step_dt(ph_mesh* m, int32_t ncycles, const double* dts) {
  PH_RANGE("ph_step_dt");
  if (!m || (!dts && ncycles > 0) || ncycles < 0) return fail(PH_ERR_INVALID, "ph_step_dt: bad argument");
  if (m->multi_level) return fail(PH_ERR_INVALID, "ph_step_dt: uniform meshes only");
  if (m->nshards > 1) return fail(PH_ERR_INVALID, "ph_step_dt: not on a shard of a decomposed mesh");
  if (!m->state_set) return fail(PH_ERR_STATE, "ph_step_dt: set the state first");
  for (int c = 0; c < ncycles; ++c) {
    int rc = ph::mesh_cycle_fixed_dt(m, dts[c]);
    if (rc) return rc;
  }
  return PH_OK;
}

int ph_set_allocator(ph_alloc_fn alloc, ph_free_fn release, void* ctx) {
  if ((alloc == nullptr) != (release == nullptr))
    return fail(PH_ERR_INVALID, "ph_set_allocator: give both functions or neither");
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc.alloc = alloc;
  g_alloc.release = release;
  g_alloc.ctx = ctx;
  return PH_OK;
}

const char* ph_last_error(void) { return g_err.c_str(); }

static int create_mesh(const ph_config* cfg, void* stream, int nshards, int shard, ph_mesh** out);

int ph_create(const ph_config* cfg, void* stream, ph_mesh** out) {
  return create_mesh(cfg, stream, 1, 0, out);
}

// Device side of a shard's halo plan: the index lists of the pack and unpack
// launches, exchange buffers for in-process shards, the dt reduction
// scratch and an event for cross-stream ordering.
static int setup_shard(ph_mesh* m) {
  const ph::ShardPlan& P = m->plan;
  PH_CUDA(cudaGetDevice(&m->device));
  const size_t ns = P.send_src.size(), nr = P.recv_dst.size();
  m->d_send_src = (long long*)m->dalloc(sizeof(long long) * std::max<size_t>(ns, 1));
  m->d_recv_dst = (long long*)m->dalloc(sizeof(long long) * std::max<size_t>(nr, 1));
  m->d_recv_flip = (int8_t*)m->dalloc(std::max<size_t>(nr, 1));
  m->d_sendbuf = m->dalloc(m->esize * m->nvar * std::max<size_t>(ns, 1));
  m->d_recvbuf = m->dalloc(m->esize * m->nvar * std::max<size_t>(nr, 1));
  m->d_wscratch = (unsigned long long*)m->dalloc(sizeof(unsigned long long) * (P.nshards + 1));
  if (!m->d_send_src || !m->d_recv_dst || !m->d_recv_flip || !m->d_sendbuf || !m->d_recvbuf || !m->d_wscratch)
    return fail(PH_ERR_OOM, "device allocation failed (shard halo plan)");
  if (ns)
    PH_CUDA(cudaMemcpyAsync(m->d_send_src, P.send_src.data(), sizeof(long long) * ns, cudaMemcpyHostToDevice,
                            m->stream));
  if (nr) {
    PH_CUDA(cudaMemcpyAsync(m->d_recv_dst, P.recv_dst.data(), sizeof(long long) * nr, cudaMemcpyHostToDevice,
                            m->stream));
    PH_CUDA(cudaMemcpyAsync(m->d_recv_flip, P.recv_flip.data(), nr, cudaMemcpyHostToDevice, m->stream));
  }
  PH_CUDA(cudaEventCreateWithFlags(&m->ev, cudaEventDisableTiming));
  PH_CUDA(cudaEventCreateWithFlags(&m->ev_done, cudaEventDisableTiming));
  return PH_OK;
}

static int create_mesh(const ph_config* cfg, void* stream, int nshards, int shard, ph_mesh** out) {
  if (!cfg || !out) return fail(PH_ERR_INVALID, "ph_create: null argument");
  *out = nullptr;
  ph::ShardPlan plan;
  if (nshards > 1) {
    std::string err;
    const int prc = ph::shard_plan(*cfg, nshards, shard, &plan, &err);
    if (prc) return fail(prc, "ph_create_shard: " + err);
  }
  for (int d = 0; d < 3; ++d) {
    if (cfg->nx[d] < 2 * ph::NG) return fail(PH_ERR_INVALID, "ph_create: nx must be >= 4");
    if (cfg->nb[d] < 1) return fail(PH_ERR_INVALID, "ph_create: nb must be >= 1");
    if (!(cfg->xmax[d] > cfg->xmin[d])) return fail(PH_ERR_INVALID, "ph_create: empty domain");
  }
  if (cfg->max_level < 0 || cfg->max_level > ph::MAXLEV)
    return fail(PH_ERR_INVALID, "ph_create: max_level must be 0 .. 4");
  if (cfg->max_level >= 1 && (cfg->nx[0] % 2 || cfg->nx[1] % 2 || cfg->nx[2] % 2))
    return fail(PH_ERR_INVALID, "ph_create: multi-level meshes need even nx");
  for (int d = 0; d < 3; ++d)
    if (((int64_t)cfg->nb[d] << cfg->max_level) > (1 << 20))
      return fail(PH_ERR_INVALID, "ph_create: too many blocks along an axis at the finest level");
  if (cfg->precision != PH_FP64 && cfg->precision != PH_FP32)
    return fail(PH_ERR_INVALID, "ph_create: precision must be PH_FP64 or PH_FP32");
  if (!(cfg->gamma > 1.0) || !(cfg->cfl > 0.0))
    return fail(PH_ERR_INVALID, "ph_create: need gamma > 1 and cfl > 0");
  if (cfg->nscalars < 0 || cfg->nscalars > ph::MAXS)
    return fail(PH_ERR_INVALID, "ph_create: nscalars must be 0 .. 2");
  for (int d = 0; d < 3; ++d) {
    const int lo = cfg->bc[2 * d], hi = cfg->bc[2 * d + 1];
    if (lo < PH_BC_PERIODIC || lo > PH_BC_REFLECT || hi < PH_BC_PERIODIC || hi > PH_BC_REFLECT)
      return fail(PH_ERR_INVALID, "ph_create: bc entries must be PH_BC_PERIODIC, _OUTFLOW or _REFLECT");
    if ((lo == PH_BC_PERIODIC) != (hi == PH_BC_PERIODIC))
      return fail(PH_ERR_INVALID, "ph_create: both faces of an axis periodic or neither");
  }
  ph_mesh* m = new ph_mesh();
  m->cfg = *cfg;
  m->stream = (cudaStream_t)stream;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    m->alloc = g_alloc;
  }
  for (int d = 0; d < 3; ++d) {
    m->nx[d] = cfg->nx[d];
    m->nb[d] = cfg->nb[d];
    m->S[d] = cfg->nx[d] + 2 * ph::NG;
  }
  m->esize = cfg->precision == PH_FP32 ? 4 : 8;
  m->nvar = ph::NV + cfg->nscalars;
  m->block_elems = (size_t)m->nvar * m->S[0] * m->S[1] * m->S[2];
  m->multi_level = cfg->max_level >= 1;
  {
    const char* g = std::getenv("PH_GHOSTS");  // "launch": keep the separate exchange launch
    bool periodic = true;
    for (int f = 0; f < 6; ++f) periodic = periodic && cfg->bc[f] == PH_BC_PERIODIC;
    // shards exchange ghosts between stages (pack / copy / unpack), never by push
    m->push = !m->multi_level && periodic && nshards == 1 && !(g && std::strcmp(g, "launch") == 0);
  }
  int t[3] = {cfg->tile[0], cfg->tile[1], cfg->tile[2]};
  const bool default_tile = t[0] == 0 && t[1] == 0 && t[2] == 0;
  if (default_tile) {
    // tiles march 16 planes (measured on 256^3 meshes: more, shorter tiles
    // leave a smaller last wave than whole-block columns, 2-7% faster)
    t[0] = cfg->nx[0] >= 16 ? 16 : 8;
    t[1] = (cfg->nx[1] >= 16 && t[0] == 16) ? 16 : 8;
    t[2] = cfg->nx[2] >= 32 ? 16 : cfg->nx[2];
    if (cfg->nscalars > 0 && !(t[0] == 16 && t[1] == 16)) t[0] = t[1] = 8;
    // FP32 uniform meshes: the 32 x 16 paired tile where the blocks tile into
    // it (16 x 16, paired as well where the blocks tile into that, otherwise)
    const int pt[3] = {32, 16, t[2]};
    if (ph::stage_tma_wanted() && valid_tile(cfg, pt)) {
      t[0] = pt[0];
      t[1] = pt[1];
    }
  }
  if (!valid_tile(cfg, t)) {
    delete m;
    return fail(PH_ERR_INVALID, "ph_create: unsupported tile");
  }
  for (int d = 0; d < 3; ++d) m->tile[d] = t[d];
  cudaError_t e = ph::configure_stage_kernels();
  if (e != cudaSuccess) {
    delete m;
    return cuda_fail(e, "configure_stage_kernels");
  }
  e = cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete m;
    return cuda_fail(e, "cudaStreamCreateWithFlags");
  }
  // root grid, then static refinement (Sec. 3.8) before any data exists
  if (nshards > 1) {  // this shard's range of the Z-ordered root grid
    m->nshards = nshards;
    m->plan = plan;
    for (long long g = plan.lo; g < plan.hi; ++g)
      m->leaf.push_back(Leaf{0, {plan.loc[g][0], plan.loc[g][1], plan.loc[g][2]}, 0});
  } else {
    for (int64_t k = 0; k < cfg->nb[2]; ++k)
      for (int64_t j = 0; j < cfg->nb[1]; ++j)
        for (int64_t i = 0; i < cfg->nb[0]; ++i) m->leaf.push_back(Leaf{0, {i, j, k}, 0});
  }
  index_tree(m);
  // the static region is refined to the finest level, one level at a time
  for (int l = 0; l < cfg->max_level && cfg->static_region; ++l) {
    std::vector<int8_t> flags(m->nleaf(), 0);
    for (int b = 0; b < m->nleaf(); ++b)
      if (m->leaf[b].level == l && overlaps_static(m, m->leaf[b])) flags[b] = 1;
    std::vector<Leaf> nl;
    if (next_tree(m, flags, false, nl)) {
      m->leaf = nl;
      index_tree(m);
    }
  }
  m->default_tile = default_tile;
  if (default_tile) choose_chunk(m);
  int rc = PH_OK;
  m->sc = (ph::DevScalars*)m->dalloc(sizeof(ph::DevScalars));
  m->d_totals = (double*)m->dalloc(8 * sizeof(double));
  if (!m->sc || !m->d_totals) rc = fail(PH_ERR_OOM, "device allocation failed");
  if (!rc) rc = ensure_pools(m, m->nleaf());
  if (!rc) rc = build_tables(m);
  if (!rc && nshards > 1) rc = setup_shard(m);
  if (!rc) {
    e = cudaMemsetAsync(m->sc, 0, sizeof(ph::DevScalars), m->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemsetAsync");
  }
  if (!rc) {
    e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize");
  }
  if (rc) {
    ph_destroy(m);
    return rc;
  }
  *out = m;
  return PH_OK;
}

int ph_destroy(ph_mesh* m) {
  if (!m) return PH_OK;
  cudaStreamSynchronize(m->stream);
  drop_graph(m);
  if (m->ev) cudaEventDestroy(m->ev);
  if (m->ev_done) cudaEventDestroy(m->ev_done);
  std::vector<void*> all = m->owned;
  for (void* p : all) m->dfree(p);
  if (m->cap) cudaStreamDestroy(m->cap);
  delete m;
  return PH_OK;
}

int ph_num_blocks(const ph_mesh* m, int32_t* n) {
  if (!m || !n) return fail(PH_ERR_INVALID, "ph_num_blocks: null argument");
  *n = m->nleaf();
  return PH_OK;
}

int ph_tree(const ph_mesh* m, int64_t* out, int32_t n) {
  if (!m || !out) return fail(PH_ERR_INVALID, "ph_tree: null argument");
  if (n < m->nleaf()) return fail(PH_ERR_INVALID, "ph_tree: output too small");
  for (int b = 0; b < m->nleaf(); ++b) {
    out[4 * b] = m->leaf[b].level;
    for (int d = 0; d < 3; ++d) out[4 * b + 1 + d] = m->leaf[b].lx[d];
  }
  return PH_OK;
}

static int64_t interior_count(const ph_mesh* m) {
  return (int64_t)m->nleaf() * m->nvar * m->nx[0] * m->nx[1] * m->nx[2];
}

int ph_set_state(ph_mesh* m, const void* U, int64_t count, int32_t on_device) {
  PH_RANGE("ph_set_state");
  if (!m || !U) return fail(PH_ERR_INVALID, "ph_set_state: null argument");
  if (count != interior_count(m)) return fail(PH_ERR_INVALID, "ph_set_state: count mismatch");
  return DISPATCH(m, set_state_t, m, U, on_device);
}

int ph_get_state(ph_mesh* m, void* U, int64_t count, int32_t on_device) {
  PH_RANGE("ph_get_state");
  if (!m || !U) return fail(PH_ERR_INVALID, "ph_get_state: null argument");
  if (count != interior_count(m)) return fail(PH_ERR_INVALID, "ph_get_state: count mismatch");
  return DISPATCH(m, get_state_t, m, U, on_device);
}

int ph_set_state_async(ph_mesh* m, const void* U, int64_t count, int32_t on_device) {
  PH_RANGE("ph_set_state_async");
  if (!m || !U) return fail(PH_ERR_INVALID, "ph_set_state_async: null argument");
  if (count != interior_count(m)) return fail(PH_ERR_INVALID, "ph_set_state_async: count mismatch");
  return DISPATCH(m, set_state_t, m, U, on_device, 1);
}

int ph_get_state_async(ph_mesh* m, void* U, int64_t count, int32_t on_device) {
  PH_RANGE("ph_get_state_async");
  if (!m || !U) return fail(PH_ERR_INVALID, "ph_get_state_async: null argument");
  if (count != interior_count(m)) return fail(PH_ERR_INVALID, "ph_get_state_async: count mismatch");
  if (!m->state_set) return fail(PH_ERR_STATE, "ph_get_state_async: set the state first");
  return DISPATCH(m, get_state_t, m, U, on_device, 1);
}

int ph_get_full(ph_mesh* m, void* U, int64_t count, int32_t on_device) {
  if (!m || !U) return fail(PH_ERR_INVALID, "ph_get_full: null argument");
  if (count != (int64_t)(m->nleaf() * m->block_elems))
    return fail(PH_ERR_INVALID, "ph_get_full: count mismatch");
  PH_CUDA(cudaMemcpyAsync(U, m->U0, count * m->esize,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->stream));
  PH_CUDA(cudaStreamSynchronize(m->stream));
  return PH_OK;
}

// ============================================================== shards

int ph_create_shard(const ph_config* cfg, int32_t nshards, int32_t shard, void* stream, ph_mesh** out) {
  if (nshards < 1) return fail(PH_ERR_INVALID, "ph_create_shard: nshards must be >= 1");
  return create_mesh(cfg, stream, nshards, shard, out);
}

int ph_shard_halo(const ph_mesh* m, int32_t peer, int64_t* send_entries, int64_t* send_offset,
                  int64_t* recv_entries, int64_t* recv_offset, int64_t leaf_range[2]) {
  if (!m) return fail(PH_ERR_INVALID, "ph_shard_halo: null mesh");
  if (m->nshards < 2) return fail(PH_ERR_INVALID, "ph_shard_halo: not a shard of a decomposed mesh");
  if (peer < 0 || peer >= m->nshards) return fail(PH_ERR_INVALID, "ph_shard_halo: peer out of range");
  const ph::ShardPlan& P = m->plan;
  if (send_entries) *send_entries = P.send_off[peer + 1] - P.send_off[peer];
  if (send_offset) *send_offset = P.send_off[peer];
  if (recv_entries) *recv_entries = P.recv_off[peer + 1] - P.recv_off[peer];
  if (recv_offset) *recv_offset = P.recv_off[peer];
  if (leaf_range) {
    leaf_range[0] = P.lo;
    leaf_range[1] = P.hi;
  }
  return PH_OK;
}

}  // extern "C"

namespace {

template <class T>
int shard_stage_t(ph_mesh* m, int stage, cudaStream_t s) {
  const ph::StageArgs<T> a = stage_args<T>(m, stage);
  PH_CUDA(ph::launch_stage<T>(a, m->tile[0], m->tile[1], s, tmap_for(m, stage)));
  T* out = (T*)(stage == 1 ? m->U1 : m->U0);
  PH_CUDA(ph::launch_ghost_uniform<T>(out, m->d_nbr, m->nx, m->nleaf(), s, m->d_leaf_id, m->nb, bc_mask(m),
                                      m->nvar));
  return PH_OK;
}

template <class T>
int shard_pack_t(ph_mesh* m, int pool, void* buf) {
  const long long vs = (long long)m->S[0] * m->S[1] * m->S[2];
  PH_CUDA(ph::launch_shard_pack<T>((const T*)(pool ? m->U1 : m->U0), m->d_send_src,
                                   (long long)m->plan.send_src.size(), vs, m->nvar, (T*)buf, m->stream));
  return PH_OK;
}

template <class T>
int shard_unpack_t(ph_mesh* m, int pool, const void* buf) {
  const long long vs = (long long)m->S[0] * m->S[1] * m->S[2];
  PH_CUDA(ph::launch_shard_unpack<T>((T*)(pool ? m->U1 : m->U0), m->d_recv_dst, m->d_recv_flip,
                                     (long long)m->plan.recv_dst.size(), vs, m->nvar, (const T*)buf, m->stream));
  return PH_OK;
}

int check_shard_set(ph_mesh* const* sh, int n, const char* who) {
  if (!sh || n < 2) return fail(PH_ERR_INVALID, std::string(who) + ": need the shards of one mesh");
  for (int s = 0; s < n; ++s) {
    if (!sh[s] || sh[s]->nshards != n || sh[s]->plan.shard != s)
      return fail(PH_ERR_INVALID, std::string(who) + ": shards[s] must be shard s of n");
    if (std::memcmp(&sh[s]->cfg, &sh[0]->cfg, sizeof(ph_config)) != 0)
      return fail(PH_ERR_INVALID, std::string(who) + ": shards of different meshes");
    if (!sh[s]->state_set) return fail(PH_ERR_STATE, std::string(who) + ": set every shard's state first");
  }
  return PH_OK;
}

// Ghost exchange of pool (0: U0, 1: U1) between the shards of one process:
// pack on every shard, copy each peer's slab into the receiver's buffer (a
// peer copy when the shards live on different devices), unpack.  Events
// order the streams: a receiver copies after the sender packed, a sender
// packs again only after every receiver has finished with its buffer.
template <class T>
int shards_exchange(ph_mesh* const* sh, int n, int pool) {
  int rc;
  for (int s = 0; s < n; ++s) {
    for (int p = 0; p < n; ++p)
      if (p != s) PH_CUDA(cudaStreamWaitEvent(sh[s]->stream, sh[p]->ev_done, 0));
    if ((rc = shard_pack_t<T>(sh[s], pool, sh[s]->d_sendbuf))) return rc;
    PH_CUDA(cudaEventRecord(sh[s]->ev, sh[s]->stream));
  }
  for (int p = 0; p < n; ++p) {
    ph_mesh* r = sh[p];
    const size_t per = r->esize * r->nvar;
    for (int s = 0; s < n; ++s) {
      if (s == p) continue;
      const int64_t cnt = r->plan.recv_off[s + 1] - r->plan.recv_off[s];
      const int64_t scnt = sh[s]->plan.send_off[p + 1] - sh[s]->plan.send_off[p];
      if (cnt != scnt) return fail(PH_ERR_STATE, "shard exchange: halo plans disagree");
      if (cnt == 0) continue;
      PH_CUDA(cudaStreamWaitEvent(r->stream, sh[s]->ev, 0));
      PH_CUDA(cudaMemcpyPeerAsync((char*)r->d_recvbuf + per * r->plan.recv_off[s], r->device,
                                  (const char*)sh[s]->d_sendbuf + per * sh[s]->plan.send_off[p], sh[s]->device,
                                  per * cnt, r->stream));
    }
    if ((rc = shard_unpack_t<T>(r, pool, r->d_recvbuf))) return rc;
    PH_CUDA(cudaEventRecord(r->ev_done, r->stream));
  }
  return PH_OK;
}

// One dt for all shards: the max signal rate over shards (recompute: from
// U0, else the one the last stage 2 folded), then each shard's bookkeeping
// (first: the first dt of a fresh state; else commit the cycle and the next dt).
int shards_dt(ph_mesh* const* sh, int n, int recompute, int first) {
  ph_mesh* z = sh[0];
  for (int s = 0; s < n; ++s) {
    ph_mesh* m = sh[s];
    if (recompute) {
      const int rc = m->cfg.precision == PH_FP32
                         ? (ph::launch_rate<float>((const float*)m->U0, m->d_level, level_geom(m), m->nx, m->nleaf(),
                                                   phys<float>(m), m->sc, m->stream, m->nvar) == cudaSuccess ? 0 : 1)
                         : (ph::launch_rate<double>((const double*)m->U0, m->d_level, level_geom(m), m->nx, m->nleaf(),
                                                    phys<double>(m), m->sc, m->stream, m->nvar) == cudaSuccess ? 0 : 1);
      if (rc) return fail(PH_ERR_CUDA, "shard dt: rate launch failed");
    }
    PH_CUDA(cudaStreamWaitEvent(m->stream, z->ev_done, 0));  // shard 0 read the previous cycle's values
    PH_CUDA(cudaMemcpyPeerAsync(z->d_wscratch + s, z->device, &m->sc->wmax_bits, m->device, sizeof(unsigned long long),
                                m->stream));
    PH_CUDA(cudaEventRecord(m->ev, m->stream));
  }
  for (int s = 1; s < n; ++s) PH_CUDA(cudaStreamWaitEvent(z->stream, sh[s]->ev, 0));
  PH_CUDA(ph::launch_shard_wmax(z->d_wscratch, n, z->d_wscratch + n, z->stream));
  PH_CUDA(cudaEventRecord(z->ev_done, z->stream));
  for (int s = 0; s < n; ++s) {
    ph_mesh* m = sh[s];
    PH_CUDA(cudaStreamWaitEvent(m->stream, z->ev_done, 0));
    PH_CUDA(cudaMemcpyPeerAsync(&m->sc->wmax_bits, m->device, z->d_wscratch + n, z->device, sizeof(unsigned long long),
                                m->stream));
    if (first) {
      PH_CUDA(ph::launch_advance(m->sc, m->cfg.cfl, 2, m->stream));
      PH_CUDA(ph::launch_advance(m->sc, m->cfg.cfl, 4, m->stream));
    } else {
      PH_CUDA(ph::launch_advance(m->sc, m->cfg.cfl, 3, m->stream));
    }
  }
  // the next exchange's packs wait for every shard's ev_done: make them
  // cover the copies above
  for (int s = 0; s < n; ++s) PH_CUDA(cudaEventRecord(sh[s]->ev_done, sh[s]->stream));
  return PH_OK;
}

template <class T>
int shards_step_t(ph_mesh* const* sh, int n, int ncycles) {
  int rc;
  for (int c = 0; c < ncycles; ++c) {
    for (int stage = 1; stage <= 2; ++stage) {
      for (int s = 0; s < n; ++s)
        if ((rc = shard_stage_t<T>(sh[s], stage, sh[s]->stream))) return rc;
      if ((rc = shards_exchange<T>(sh, n, stage == 1 ? 1 : 0))) return rc;
    }
    if ((rc = shards_dt(sh, n, 0, 0))) return rc;
  }
  return PH_OK;
}

}  // namespace

extern "C" {

int ph_shard_stage(ph_mesh* m, int32_t stage) {
  if (!m || (stage != 1 && stage != 2)) return fail(PH_ERR_INVALID, "ph_shard_stage: bad argument");
  if (m->nshards < 2) return fail(PH_ERR_INVALID, "ph_shard_stage: not a shard of a decomposed mesh");
  if (!m->state_set) return fail(PH_ERR_STATE, "ph_shard_stage: set the state first");
  return DISPATCH(m, shard_stage_t, m, stage, m->stream);
}

int ph_shard_pack(ph_mesh* m, int32_t pool, void* sendbuf) {
  if (!m || (pool != 0 && pool != 1) || !sendbuf) return fail(PH_ERR_INVALID, "ph_shard_pack: bad argument");
  if (m->nshards < 2) return fail(PH_ERR_INVALID, "ph_shard_pack: not a shard of a decomposed mesh");
  return DISPATCH(m, shard_pack_t, m, pool, sendbuf);
}

int ph_shard_unpack(ph_mesh* m, int32_t pool, const void* recvbuf) {
  if (!m || (pool != 0 && pool != 1) || !recvbuf) return fail(PH_ERR_INVALID, "ph_shard_unpack: bad argument");
  if (m->nshards < 2) return fail(PH_ERR_INVALID, "ph_shard_unpack: not a shard of a decomposed mesh");
  return DISPATCH(m, shard_unpack_t, m, pool, recvbuf);
}

int ph_shard_rate(ph_mesh* m, int32_t recompute, double* d_rate) {
  if (!m || !d_rate) return fail(PH_ERR_INVALID, "ph_shard_rate: bad argument");
  if (m->nshards < 2) return fail(PH_ERR_INVALID, "ph_shard_rate: not a shard of a decomposed mesh");
  if (recompute) {
    const cudaError_t e =
        m->cfg.precision == PH_FP32
            ? ph::launch_rate<float>((const float*)m->U0, m->d_level, level_geom(m), m->nx, m->nleaf(),
                                     phys<float>(m), m->sc, m->stream, m->nvar)
            : ph::launch_rate<double>((const double*)m->U0, m->d_level, level_geom(m), m->nx, m->nleaf(),
                                      phys<double>(m), m->sc, m->stream, m->nvar);
    if (e != cudaSuccess) return cuda_fail(e, "ph_shard_rate");
  }
  PH_CUDA(cudaMemcpyAsync(d_rate, &m->sc->wmax_bits, sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
  return PH_OK;
}

int ph_shard_finish(ph_mesh* m, int32_t first, const double* d_rate) {
  if (!m || !d_rate) return fail(PH_ERR_INVALID, "ph_shard_finish: bad argument");
  if (m->nshards < 2) return fail(PH_ERR_INVALID, "ph_shard_finish: not a shard of a decomposed mesh");
  PH_CUDA(cudaMemcpyAsync(&m->sc->wmax_bits, d_rate, sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
  if (first) {
    PH_CUDA(ph::launch_advance(m->sc, m->cfg.cfl, 2, m->stream));
    PH_CUDA(ph::launch_advance(m->sc, m->cfg.cfl, 4, m->stream));
  } else {
    PH_CUDA(ph::launch_advance(m->sc, m->cfg.cfl, 3, m->stream));
  }
  return PH_OK;
}

int ph_shards_sync(ph_mesh* const* shards, int32_t n) {
  PH_RANGE("ph_shards_sync");
  int rc = check_shard_set(shards, n, "ph_shards_sync");
  if (rc) return rc;
  rc = shards[0]->cfg.precision == PH_FP32 ? shards_exchange<float>(shards, n, 0)
                                           : shards_exchange<double>(shards, n, 0);
  if (rc) return rc;
  return shards_dt(shards, n, 1, 1);
}

int ph_shards_step(ph_mesh* const* shards, int32_t n, int32_t ncycles) {
  PH_RANGE("ph_shards_step");
  if (ncycles < 0) return fail(PH_ERR_INVALID, "ph_shards_step: negative cycle count");
  int rc = check_shard_set(shards, n, "ph_shards_step");
  if (rc) return rc;
  return shards[0]->cfg.precision == PH_FP32 ? shards_step_t<float>(shards, n, ncycles)
                                             : shards_step_t<double>(shards, n, ncycles);
}

int ph_step(ph_mesh* m, int32_t ncycles) {
  PH_RANGE("ph_step");
  if (!m) return fail(PH_ERR_INVALID, "ph_step: null mesh");
  if (ncycles < 0) return fail(PH_ERR_INVALID, "ph_step: negative cycle count");
  if (!m->state_set) return fail(PH_ERR_STATE, "ph_step: set the state first");
  if (m->nshards > 1)
    return fail(PH_ERR_STATE, "ph_step: a shard steps with ph_shards_step or the ph_shard_* phases");
  if (ncycles == 0) return PH_OK;
  return DISPATCH(m, step_t, m, ncycles);
}

static int read_scalars(ph_mesh* m, ph::DevScalars* hs) {
  PH_CUDA(cudaMemcpyAsync(hs, m->sc, sizeof(*hs), cudaMemcpyDeviceToHost, m->stream));
  PH_CUDA(cudaStreamSynchronize(m->stream));
  return PH_OK;
}

int ph_get_dt(ph_mesh* m, double* dt) {
  if (!m || !dt) return fail(PH_ERR_INVALID, "ph_get_dt: null argument");
  ph::DevScalars hs;
  int rc = read_scalars(m, &hs);
  if (rc) return rc;
  *dt = hs.dt_last;
  return PH_OK;
}

int ph_get_next_dt(ph_mesh* m, double* dt) {
  if (!m || !dt) return fail(PH_ERR_INVALID, "ph_get_next_dt: null argument");
  ph::DevScalars hs;
  int rc = read_scalars(m, &hs);
  if (rc) return rc;
  *dt = hs.dt_next;
  return PH_OK;
}

int ph_get_time(ph_mesh* m, double* time, int64_t* cycle) {
  if (!m) return fail(PH_ERR_INVALID, "ph_get_time: null mesh");
  ph::DevScalars hs;
  int rc = read_scalars(m, &hs);
  if (rc) return rc;
  if (time) *time = hs.time;
  if (cycle) *cycle = hs.cycle;
  return PH_OK;
}

int ph_totals(ph_mesh* m, double* out) {
  PH_RANGE("ph_totals");
  if (!m || !out) return fail(PH_ERR_INVALID, "ph_totals: null argument");
  return DISPATCH(m, totals_t, m, out);
}

int ph_tag(ph_mesh* m, int8_t* flags, double* indicator, int32_t n) {
  if (!m) return fail(PH_ERR_INVALID, "ph_tag: null mesh");
  if (n < m->nleaf()) return fail(PH_ERR_INVALID, "ph_tag: output too small");
  return DISPATCH(m, tag_t, m, flags, indicator);
}

int ph_refine_where(ph_mesh* m, const int8_t* flags, int32_t n, int32_t check_age,
                    int32_t* changed) {
  PH_RANGE("ph_refine_where");
  if (!m || !flags) return fail(PH_ERR_INVALID, "ph_refine_where: null argument");
  if (n != m->nleaf()) return fail(PH_ERR_INVALID, "ph_refine_where: flag count mismatch");
  if (!m->multi_level) return fail(PH_ERR_INVALID, "ph_refine_where: mesh has max_level 0");
  std::vector<int8_t> f(flags, flags + n);
  std::vector<Leaf> nl;
  const bool ch = next_tree(m, f, check_age != 0, nl);
  if (changed) *changed = ch ? 1 : 0;
  if (!ch) return PH_OK;
  int rc = DISPATCH(m, remesh_t, m, nl);
  if (rc) return rc;
  if (m->state_set) {
    rc = m->cfg.precision == PH_FP32 ? refresh_dt_t<float>(m) : refresh_dt_t<double>(m);
  }
  return rc;
}

int ph_refine_by_density(ph_mesh* m, int32_t* changed) {
  if (!m) return fail(PH_ERR_INVALID, "ph_refine_by_density: null mesh");
  std::vector<int8_t> flags(m->nleaf());
  int rc = ph_tag(m, flags.data(), nullptr, m->nleaf());
  if (rc) return rc;
  return ph_refine_where(m, flags.data(), m->nleaf(), 1, changed);
}

int ph_status(ph_mesh* m, int64_t* floor_hits, int32_t* nonfinite) {
  if (!m) return fail(PH_ERR_INVALID, "ph_status: null mesh");
  ph::DevScalars hs;
  int rc = read_scalars(m, &hs);
  if (rc) return rc;
  if (floor_hits) *floor_hits = (int64_t)hs.floor_hits;
  if (nonfinite) *nonfinite = hs.nonfinite;
  if (hs.error) return fail(PH_ERR_TIMEOUT, "a bounded device wait gave up");
  if (hs.tree_error) return fail(PH_ERR_STATE, "a composite-field evaluation nested too deep");
  if (hs.floor_hits || hs.nonfinite)
    return fail(PH_ERR_NONPHYSICAL, "floors applied or non-finite dt");
  return PH_OK;
}

int ph_fill_ghosts(ph_mesh* m) {
  if (!m) return fail(PH_ERR_INVALID, "ph_fill_ghosts: null mesh");
  int rc = m->cfg.precision == PH_FP32 ? fill_ghosts_t<float>(m, (float*)m->U0)
                                       : fill_ghosts_t<double>(m, (double*)m->U0);
  if (rc) return rc;
  PH_CUDA(cudaStreamSynchronize(m->stream));
  return PH_OK;
}

int ph_launches_per_cycle(const ph_mesh* m, int32_t* n) {
  if (!m || !n) return fail(PH_ERR_INVALID, "ph_launches_per_cycle: null argument");
  *n = m->multi_level ? 0 : (m->push ? 3 : 5);
  return PH_OK;
}

int ph_profile_cycles(ph_mesh* m, int32_t ncycles, double* ms_out, int32_t nslots) {
  if (!m || !ms_out || nslots < 0 || nslots > 5 || ncycles < 0)
    return fail(PH_ERR_INVALID, "ph_profile_cycles: bad argument");
  if (m->multi_level) return fail(PH_ERR_INVALID, "ph_profile_cycles: uniform meshes only");
  if (m->nshards > 1) return fail(PH_ERR_INVALID, "ph_profile_cycles: not on a shard of a decomposed mesh");
  if (!m->state_set) return fail(PH_ERR_STATE, "ph_profile_cycles: set the state first");
  return DISPATCH(m, profile_t, m, ncycles, ms_out, nslots);
}

int ph_get_tile(const ph_mesh* m, int32_t tile[3]) {
  if (!m || !tile) return fail(PH_ERR_INVALID, "ph_get_tile: null argument");
  for (int d = 0; d < 3; ++d) tile[d] = m->tile[d];
  return PH_OK;
}

// ------------------------------------------------------------ restart files
// Sec. 3.9: outputs of selectable precision, and a restart type from which a
// run continues bitwise identically.  Layout (native byte order):
//   char magic[8] "PHYDRST1"; int32 version (1); int32 data precision;
//   ph_config; int32 nleaf; int32 pad; double time, dt_next, dt_last;
//   int64 cycle; uint64 floor_hits; int32 nonfinite, error;
//   per leaf: int32 level, int32 age, int64 lx[3];
//   interior state in the layout of ph_get_state, in the data precision.
namespace {

constexpr char kMagic[8] = {'P', 'H', 'Y', 'D', 'R', 'S', 'T', '1'};

struct FileHead {
  char magic[8];
  int32_t version;
  int32_t data_precision;
  ph_config cfg;
  int32_t nleaf;
  int32_t pad;
  double time, dt_next, dt_last;
  int64_t cycle;
  uint64_t floor_hits;
  int32_t nonfinite, error;
};

struct FileLeaf {
  int32_t level, age;
  int64_t lx[3];
};

struct FileCloser {
  FILE* f;
  ~FileCloser() {
    if (f) fclose(f);
  }
};

}  // namespace

int ph_save(ph_mesh* m, const char* path, int32_t precision) {
  if (!m || !path) return fail(PH_ERR_INVALID, "ph_save: null argument");
  if (precision != PH_FP64 && precision != PH_FP32)
    return fail(PH_ERR_INVALID, "ph_save: precision must be PH_FP64 or PH_FP32");
  if (!m->state_set) return fail(PH_ERR_STATE, "ph_save: set the state first");
  if (m->nshards > 1) return fail(PH_ERR_INVALID, "ph_save: not on a shard of a decomposed mesh");
  ph::DevScalars hs;
  int rc = read_scalars(m, &hs);
  if (rc) return rc;
  const int64_t count = interior_count(m);
  std::vector<unsigned char> buf((size_t)count * m->esize);
  if ((rc = ph_get_state(m, buf.data(), count, 0))) return rc;
  FileHead h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, kMagic, 8);
  h.version = 1;
  h.data_precision = precision;
  h.cfg = m->cfg;
  h.nleaf = m->nleaf();
  h.time = hs.time;
  h.dt_next = hs.dt_next;
  h.dt_last = hs.dt_last;
  h.cycle = hs.cycle;
  h.floor_hits = hs.floor_hits;
  h.nonfinite = hs.nonfinite;
  h.error = hs.error;
  std::vector<FileLeaf> lv(m->nleaf());
  for (int b = 0; b < m->nleaf(); ++b) {
    lv[b].level = m->leaf[b].level;
    lv[b].age = m->leaf[b].age;
    for (int d = 0; d < 3; ++d) lv[b].lx[d] = m->leaf[b].lx[d];
  }
  // data in the requested precision (a narrowing conversion rounds to nearest)
  std::vector<unsigned char> out;
  const unsigned char* data = buf.data();
  size_t data_bytes = buf.size();
  const int mp = m->cfg.precision;
  if (precision != mp) {
    out.resize((size_t)count * (precision == PH_FP32 ? 4 : 8));
    if (precision == PH_FP32) {
      const double* src = (const double*)buf.data();
      float* dst = (float*)out.data();
      for (int64_t i = 0; i < count; ++i) dst[i] = (float)src[i];
    } else {
      const float* src = (const float*)buf.data();
      double* dst = (double*)out.data();
      for (int64_t i = 0; i < count; ++i) dst[i] = (double)src[i];
    }
    data = out.data();
    data_bytes = out.size();
  }
  FileCloser fc{fopen(path, "wb")};
  if (!fc.f) return fail(PH_ERR_IO, std::string("ph_save: cannot open ") + path);
  bool ok = fwrite(&h, sizeof(h), 1, fc.f) == 1;
  if (ok && !lv.empty()) ok = fwrite(lv.data(), sizeof(FileLeaf), lv.size(), fc.f) == lv.size();
  if (ok && data_bytes) ok = fwrite(data, 1, data_bytes, fc.f) == data_bytes;
  if (fclose(fc.f) != 0) ok = false;
  fc.f = nullptr;
  if (!ok) return fail(PH_ERR_IO, std::string("ph_save: write failed: ") + path);
  return PH_OK;
}

int ph_load(const char* path, void* stream, ph_mesh** out) {
  if (!path || !out) return fail(PH_ERR_INVALID, "ph_load: null argument");
  *out = nullptr;
  FileCloser fc{fopen(path, "rb")};
  if (!fc.f) return fail(PH_ERR_IO, std::string("ph_load: cannot open ") + path);
  FileHead h;
  if (fread(&h, sizeof(h), 1, fc.f) != 1) return fail(PH_ERR_IO, "ph_load: truncated header");
  if (std::memcmp(h.magic, kMagic, 8) != 0 || h.version != 1)
    return fail(PH_ERR_INVALID, "ph_load: not a restart file of this library");
  if (h.data_precision != PH_FP64 && h.data_precision != PH_FP32)
    return fail(PH_ERR_INVALID, "ph_load: bad data precision");
  for (int d = 0; d < 3; ++d)
    if (h.cfg.nx[d] < 1 || h.cfg.nx[d] > (1 << 16) || h.cfg.nb[d] < 1 || h.cfg.nb[d] > (1 << 16))
      return fail(PH_ERR_INVALID, "ph_load: bad block or grid size");
  if (h.cfg.nscalars < 0 || h.cfg.nscalars > ph::MAXS)
    return fail(PH_ERR_INVALID, "ph_load: bad scalar count");
  const int64_t nroot = (int64_t)h.cfg.nb[0] * h.cfg.nb[1] * h.cfg.nb[2];
  const int64_t cells = (int64_t)h.cfg.nx[0] * h.cfg.nx[1] * h.cfg.nx[2];
  if (h.cfg.max_level < 0 || h.cfg.max_level > ph::MAXLEV)
    return fail(PH_ERR_INVALID, "ph_load: bad max_level");
  if (nroot > (1 << 24) || cells > (1 << 30) || h.nleaf < 1 ||
      (int64_t)h.nleaf > (nroot << (3 * h.cfg.max_level)) || h.nleaf > (1 << 26))
    return fail(PH_ERR_INVALID, "ph_load: bad leaf count");
  {  // the file must hold exactly the tree and the state its header announces
    const int64_t want = (int64_t)sizeof(FileHead) + (int64_t)h.nleaf * sizeof(FileLeaf) +
                         (int64_t)h.nleaf * (ph::NV + h.cfg.nscalars) * cells *
                             (h.data_precision == PH_FP32 ? 4 : 8);
    if (fseek(fc.f, 0, SEEK_END) != 0) return fail(PH_ERR_IO, "ph_load: cannot seek");
    const long have = ftell(fc.f);
    if (have < 0 || (int64_t)have != want)
      return fail(PH_ERR_IO, "ph_load: file size does not match its header (truncated?)");
    if (fseek(fc.f, (long)sizeof(FileHead), SEEK_SET) != 0)
      return fail(PH_ERR_IO, "ph_load: cannot seek");
  }
  std::vector<FileLeaf> lv(h.nleaf);
  if (fread(lv.data(), sizeof(FileLeaf), lv.size(), fc.f) != lv.size())
    return fail(PH_ERR_IO, "ph_load: truncated tree");
  // the tree must tile the root grid
  {
    std::vector<Leaf> tl;
    for (const FileLeaf& l : lv) {
      if (l.level < 0 || l.level > h.cfg.max_level)
        return fail(PH_ERR_INVALID, "ph_load: bad leaf level");
      for (int d = 0; d < 3; ++d)
        if (l.lx[d] < 0 || l.lx[d] >= ((int64_t)h.cfg.nb[d] << l.level))
          return fail(PH_ERR_INVALID, "ph_load: leaf outside the domain");
      tl.push_back(Leaf{l.level, {l.lx[0], l.lx[1], l.lx[2]}, l.age});
    }
    std::vector<int> nodes;
    if (!build_nodes(tl, h.cfg.nb, nodes))
      return fail(PH_ERR_INVALID, "ph_load: leaves do not tile the domain");
  }
  const int64_t count = (int64_t)h.nleaf * (ph::NV + h.cfg.nscalars) * h.cfg.nx[0] * h.cfg.nx[1] * h.cfg.nx[2];
  const size_t fbytes = (size_t)count * (h.data_precision == PH_FP32 ? 4 : 8);
  std::vector<unsigned char> data(fbytes);
  if (fbytes && fread(data.data(), 1, fbytes, fc.f) != fbytes)
    return fail(PH_ERR_IO, "ph_load: truncated state");
  ph_mesh* m = nullptr;
  int rc = ph_create(&h.cfg, stream, &m);
  if (rc) return rc;
  // install the saved tree (ages included: they set the derefinement cadence)
  m->leaf.clear();
  for (const FileLeaf& l : lv) m->leaf.push_back(Leaf{l.level, {l.lx[0], l.lx[1], l.lx[2]}, l.age});
  index_tree(m);
  drop_graph(m);
  if (!rc) rc = ensure_pools(m, m->nleaf());
  if (!rc) rc = build_tables(m);
  if (!rc && m->default_tile) choose_chunk(m);
  // state in the mesh's precision (widening is exact)
  std::vector<unsigned char> conv;
  const void* U = data.data();
  if (!rc && h.data_precision != h.cfg.precision) {
    conv.resize((size_t)count * (h.cfg.precision == PH_FP32 ? 4 : 8));
    if (h.cfg.precision == PH_FP32) {
      const double* src = (const double*)data.data();
      float* dst = (float*)conv.data();
      for (int64_t i = 0; i < count; ++i) dst[i] = (float)src[i];
    } else {
      const float* src = (const float*)data.data();
      double* dst = (double*)conv.data();
      for (int64_t i = 0; i < count; ++i) dst[i] = (double)src[i];
    }
    U = conv.data();
  }
  if (!rc) rc = ph_set_state(m, U, count, 0);
  if (!rc) {
    ph::DevScalars hs;
    std::memset(&hs, 0, sizeof(hs));
    hs.time = h.time;
    hs.dt_next = h.dt_next;
    hs.dt_last = h.dt_last;
    hs.cycle = h.cycle;
    hs.floor_hits = h.floor_hits;
    hs.nonfinite = h.nonfinite;
    hs.error = h.error;
    cudaError_t e = cudaMemcpyAsync(m->sc, &hs, sizeof(hs), cudaMemcpyHostToDevice, m->stream);
    if (!e) e = cudaStreamSynchronize(m->stream);
    if (e) rc = cuda_fail(e, "ph_load");
  }
  if (rc) {
    ph_destroy(m);
    return rc;
  }
  *out = m;
  return PH_OK;
}

}  // extern "C"

