// hydro_oracle.hpp -- plain, slow, FP64 CPU oracle for the Parthenon-hydro cycle.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
// call this code: only tests/, __graft_entry__.smoke() and bench.py's CPU
// baseline leg use it.  It shares no code, header, table or constant with the
// CUDA library; the two meet only through the seeded input generators.
//
// What it computes (arXiv:2202.12309, Sec. 4.1 "Parthenon-hydro"): the 3-D
// Euler equations of an ideal gas, advanced with a two-stage Runge-Kutta
// integrator, piecewise-linear reconstruction and the HLLE Riemann solver, on
// a mesh of equal-sized MeshBlocks arranged in an oct-tree (Sec. 2.1), with
// ghost cells filled from neighbours, restriction/prolongation at level
// boundaries and flux correction (Sec. 3.7), and a global CFL time step from a
// min-reduction (Sec. 3.10).  The paper names the methods only; every choice it
// leaves open is fixed here as one "reading", listed in the comments below and
// in the design notes.  Everything is written in the order the method defines
// it, one cell / one face at a time, with no blocking or fusion.
//
// The scalar type R is double, or std::complex<double> for complex-step
// derivatives (Squire & Trapp 1998): every branch (limiter, wave-speed max/min,
// floors, |x|) is decided on the real part, which freezes branches exactly as
// the adjoint does.
//
// Parity status per function (pins live in tests/test_oracle_*.py):
//   cons_to_prim, vanleer, hlle_flux, stage update, dt, ghost fill (uniform),
//   restriction/prolongation, flux correction, tree order, tagging: pinned by
//   closed forms, invariants, exact Riemann solutions and brute force.
#pragma once
#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <map>
#include <set>
#include <vector>

namespace ho {

using cplx = std::complex<double>;
inline double re(double x) { return x; }
inline double re(const cplx& x) { return x.real(); }
using std::sqrt;

// |x|, max, min with branches taken on the real part (identity for double).
template <class R> inline R rabs(const R& x) { return re(x) < 0.0 ? R(-x) : x; }
template <class R> inline R rmax(const R& a, const R& b) { return re(a) >= re(b) ? a : b; }
template <class R> inline R rmin(const R& a, const R& b) { return re(a) <= re(b) ? a : b; }

enum { IDN = 0, IM1 = 1, IM2 = 2, IM3 = 3, IEN = 4, NVAR = 5 };
// Passive scalars (Sec. 3.4: the hydro package advects every variable flagged
// as advected): up to MAXS extra conserved variables rho r_s after the energy,
// advected with the flow.  Arrays are sized for the maximum.
constexpr int MAXS = 2;
constexpr int NMAX = NVAR + MAXS;
constexpr int NG = 2;  // ghost width (PLM needs two cells on each side)

// Mesh / physics configuration.  Plain POD, mirrored field by field by the
// ctypes wrapper in oracle/__init__.py.
struct Config {
  int32_t nx[3];          // interior cells per block along x1,x2,x3
  int32_t nb[3];          // root-grid blocks along x1,x2,x3
  double xmin[3], xmax[3];
  int32_t max_level;      // 0 = uniform; finest level of the tree (at most 4)
  int32_t adaptive;       // tag + remesh after every cycle
  double gamma, cfl, dfloor, pfloor;
  double refine_tol, derefine_tol;
  int32_t derefine_count;
  int32_t static_region;  // 1: blocks overlapping [static_lo, static_hi] refined and pinned
  double static_lo[3], static_hi[3];
  int32_t bc[6];          // physical boundary per face (x1 inner, x1 outer, x2 ..., x3 ...):
                          // BC_PERIODIC, BC_OUTFLOW or BC_REFLECT; both faces of an axis
                          // periodic or neither
  int32_t nscalars;       // passive scalars, 0 .. MAXS
  int32_t pad;
};

// Physical boundary conditions.  Reading (the paper's reflective boundaries
// mirror the vector component normal to the boundary, Sec. 3.4; outflow is the
// usual zero-gradient copy): a location outside the domain along axis d takes
// the value at its image inside the domain at the same level --
//   periodic:   shifted by the domain length;
//   outflow:    the nearest cell inside (the first interior layer);
//   reflecting: mirrored about the boundary face (ghost layer g takes interior
//               layer g), with the momentum component along d negated.
constexpr int BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_REFLECT = 2;

// ---------------------------------------------------------------------------
// Pointwise physics (Sec. 4.1: Euler equations, ideal gas)
// ---------------------------------------------------------------------------

// Conserved U = (rho, m1, m2, m3, E) -> primitive W = (rho, v1, v2, v3, p).
// Reading: E = p/(gamma-1) + rho |v|^2 / 2; density and pressure floors are
// applied here and only here, and every hit is counted.
// Passive scalars: the concentration r = (rho r) / rho (after the floor).
template <class R>
inline void cons_to_prim(const R u[NMAX], R w[NMAX], const R& gamma, double dfloor,
                         double pfloor, long* floors, int ns = 0) {
  R rho = u[IDN];
  if (re(rho) < dfloor) { rho = R(dfloor); ++*floors; }
  w[IDN] = rho;
  w[IM1] = u[IM1] / rho;
  w[IM2] = u[IM2] / rho;
  w[IM3] = u[IM3] / rho;
  R ke = 0.5 * (u[IM1] * w[IM1] + u[IM2] * w[IM2] + u[IM3] * w[IM3]);
  R p = (gamma - 1.0) * (u[IEN] - ke);
  if (re(p) < pfloor) { p = R(pfloor); ++*floors; }
  w[IEN] = p;
  for (int s = 0; s < ns; ++s) w[NVAR + s] = u[NVAR + s] / rho;
}

// Piecewise-linear reconstruction slope (Sec. 4.1 "piecewise linear
// reconstruction").  Reading: van Leer's harmonic limiter applied to each
// primitive variable: delta = 2 dL dR / (dL + dR) where dL dR > 0, else 0.
template <class R>
inline R vanleer(const R& wm, const R& w0, const R& wp) {
  R dl = w0 - wm;
  R dr = wp - w0;
  R prod = dl * dr;
  // branch on the real parts (for doubles this is prod > 0): with complex
  // arguments Re(dl dr) would also carry -Im(dl) Im(dr)
  if (re(dl) * re(dr) > 0.0) return 2.0 * prod / (dl + dr);
  return R(0.0);
}

// HLLE flux through a face with normal along `dir` (0,1,2) from the left and
// right primitive states (Sec. 4.1 "HLLE Riemann solver").  Reading: Einfeldt's
// wave-speed bounds with Roe-averaged velocity and enthalpy:
//   b+ = max(0, vR + cR, v~ + c~),  b- = min(0, vL - cL, v~ - c~),
//   F  = (b+ FL - b- FR + b+ b- (UR - UL)) / (b+ - b-).
// A passive scalar is one more conserved variable U = rho r with physical flux
// rho v_n r, through the same formula with the same bounds.
template <class R>
inline void hlle_flux(const R wl[NMAX], const R wr[NMAX], int dir, const R& gamma,
                      R flux[NMAX], int ns = 0) {
  const int ivn = IM1 + dir;
  const R gm1 = gamma - 1.0;
  // left and right conserved states and physical fluxes
  R ul[NMAX], ur[NMAX], fl[NMAX], fr[NMAX];
  R v2l = wl[IM1] * wl[IM1] + wl[IM2] * wl[IM2] + wl[IM3] * wl[IM3];
  R v2r = wr[IM1] * wr[IM1] + wr[IM2] * wr[IM2] + wr[IM3] * wr[IM3];
  R el = wl[IEN] / gm1 + 0.5 * wl[IDN] * v2l;
  R er = wr[IEN] / gm1 + 0.5 * wr[IDN] * v2r;
  ul[IDN] = wl[IDN];
  ur[IDN] = wr[IDN];
  for (int a = 0; a < 3; ++a) {
    ul[IM1 + a] = wl[IDN] * wl[IM1 + a];
    ur[IM1 + a] = wr[IDN] * wr[IM1 + a];
  }
  ul[IEN] = el;
  ur[IEN] = er;
  R vnl = wl[ivn], vnr = wr[ivn];
  fl[IDN] = wl[IDN] * vnl;
  fr[IDN] = wr[IDN] * vnr;
  for (int a = 0; a < 3; ++a) {
    fl[IM1 + a] = wl[IDN] * vnl * wl[IM1 + a];
    fr[IM1 + a] = wr[IDN] * vnr * wr[IM1 + a];
  }
  fl[ivn] = fl[ivn] + wl[IEN];
  fr[ivn] = fr[ivn] + wr[IEN];
  fl[IEN] = (el + wl[IEN]) * vnl;
  fr[IEN] = (er + wr[IEN]) * vnr;
  for (int s = NVAR; s < NVAR + ns; ++s) {
    ul[s] = wl[IDN] * wl[s];
    ur[s] = wr[IDN] * wr[s];
    fl[s] = wl[IDN] * vnl * wl[s];
    fr[s] = wr[IDN] * vnr * wr[s];
  }

  // sound speeds and Roe averages
  R cl = sqrt(gamma * wl[IEN] / wl[IDN]);
  R cr = sqrt(gamma * wr[IEN] / wr[IDN]);
  R sl = sqrt(wl[IDN]);
  R sr = sqrt(wr[IDN]);
  R hl = (el + wl[IEN]) / wl[IDN];
  R hr = (er + wr[IEN]) / wr[IDN];
  R vroe[3];
  for (int a = 0; a < 3; ++a) vroe[a] = (sl * wl[IM1 + a] + sr * wr[IM1 + a]) / (sl + sr);
  R hroe = (sl * hl + sr * hr) / (sl + sr);
  R v2roe = vroe[0] * vroe[0] + vroe[1] * vroe[1] + vroe[2] * vroe[2];
  R a2roe = rmax(R(0.0), R(gm1 * (hroe - 0.5 * v2roe)));
  R croe = sqrt(a2roe);

  R bp = rmax(R(0.0), rmax(R(vnr + cr), R(vroe[dir] + croe)));
  R bm = rmin(R(0.0), rmin(R(vnl - cl), R(vroe[dir] - croe)));
  for (int v = 0; v < NVAR + ns; ++v)
    flux[v] = (bp * fl[v] - bm * fr[v] + bp * bm * (ur[v] - ul[v])) / (bp - bm);
}

// minmod of two one-sided differences (used by prolongation).
template <class R>
inline R minmod(const R& a, const R& b) {
  if (re(a) * re(b) > 0.0) return re(rabs(a)) < re(rabs(b)) ? a : b;
  return R(0.0);
}

// ---------------------------------------------------------------------------
// Block tree (Sec. 2.1: oct-tree of MeshBlocks, Z-ordering)
// ---------------------------------------------------------------------------

struct LeafId {
  int32_t level;
  int64_t lx[3];
};

// Morton (Z-order) key of a block's logical location scaled to the finest
// level; bit b of x1 goes to bit 3b, x2 to 3b+1, x3 to 3b+2.
inline uint64_t morton_key(const LeafId& id, int max_level) {
  uint64_t key = 0;
  int sh = max_level - id.level;
  for (int d = 0; d < 3; ++d) {
    uint64_t c = (uint64_t)id.lx[d] << sh;
    for (int b = 0; b < 21; ++b) key |= ((c >> b) & 1ull) << (3 * b + d);
  }
  return key;
}

inline bool leaf_less(const LeafId& a, const LeafId& b, int max_level) {
  uint64_t ka = morton_key(a, max_level), kb = morton_key(b, max_level);
  if (ka != kb) return ka < kb;
  return a.level < b.level;
}

// ---------------------------------------------------------------------------
// Mesh of leaf blocks with ghost zones
// ---------------------------------------------------------------------------

template <class R>
struct Mesh {
  Config cfg;
  R gamma;
  std::vector<LeafId> leaf;
  std::vector<int32_t> age;            // cycles since the leaf was created
  std::vector<std::vector<R>> U;       // per leaf: nv() x S3 x S2 x S1 (ghosts included)
  std::vector<int32_t> root;           // root-grid slot -> level-0 leaf index, or -1 when refined
  std::map<std::array<int64_t, 4>, int32_t> leaf_at;  // (level, lx1, lx2, lx3) -> leaf index
  double time = 0.0, dt = 0.0;
  int64_t cycle = 0;
  long floors = 0;

  int S(int d) const { return cfg.nx[d] + 2 * NG; }
  int nv() const { return NVAR + cfg.nscalars; }  // conserved variables per cell
  size_t block_len() const { return (size_t)nv() * S(0) * S(1) * S(2); }
  size_t idx(int v, int k, int j, int i) const {
    return (((size_t)v * S(2) + k) * S(1) + j) * S(0) + i;
  }
  int64_t ncell(int d, int level) const { return ((int64_t)cfg.nb[d] * cfg.nx[d]) << level; }
  double dx(int d, int level) const {
    return (cfg.xmax[d] - cfg.xmin[d]) / (double)ncell(d, level);
  }

  explicit Mesh(const Config& c) : cfg(c), gamma(c.gamma) {
    for (int64_t k = 0; k < cfg.nb[2]; ++k)
      for (int64_t j = 0; j < cfg.nb[1]; ++j)
        for (int64_t i = 0; i < cfg.nb[0]; ++i) leaf.push_back(LeafId{0, {i, j, k}});
    age.assign(leaf.size(), 0);
    U.assign(leaf.size(), std::vector<R>(block_len(), R(0.0)));
    sort_and_index();
    // static refinement, one level at a time up to max_level (reading: the
    // static region is refined to the finest level)
    for (int l = 0; l < cfg.max_level && cfg.static_region; ++l) {
      std::vector<int8_t> flags(leaf.size(), 0);
      for (size_t b = 0; b < leaf.size(); ++b)
        if (leaf[b].level == l && in_static_region(leaf[b])) flags[b] = 1;
      remesh(flags);
    }
  }

  // Block extent along d: xmin + l * (width of one block at that level).
  void block_extent(const LeafId& id, int d, double* lo, double* hi) const {
    double w = (cfg.xmax[d] - cfg.xmin[d]) / (double)((int64_t)cfg.nb[d] << id.level);
    *lo = cfg.xmin[d] + (double)id.lx[d] * w;
    *hi = cfg.xmin[d] + (double)(id.lx[d] + 1) * w;
  }
  // Reading of "static + adaptive": a block overlapping the open box is refined
  // at start and never derefined.
  bool in_static_region(const LeafId& id) const {
    if (!cfg.static_region) return false;
    for (int d = 0; d < 3; ++d) {
      double lo, hi;
      block_extent(id, d, &lo, &hi);
      if (!(lo < cfg.static_hi[d] && hi > cfg.static_lo[d])) return false;
    }
    return true;
  }

  int root_slot(int64_t r0, int64_t r1, int64_t r2) const {
    return (int)((r2 * cfg.nb[1] + r1) * cfg.nb[0] + r0);
  }

  // Sort leaves in Z-order and rebuild the lookup tables.
  void sort_and_index() {
    std::vector<size_t> order(leaf.size());
    for (size_t b = 0; b < order.size(); ++b) order[b] = b;
    int ml = cfg.max_level;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
      return leaf_less(leaf[a], leaf[b], ml);
    });
    std::vector<LeafId> l2;
    std::vector<int32_t> a2;
    std::vector<std::vector<R>> u2;
    for (size_t b : order) {
      l2.push_back(leaf[b]);
      a2.push_back(age[b]);
      u2.push_back(std::move(U[b]));
    }
    leaf.swap(l2);
    age.swap(a2);
    U.swap(u2);
    size_t nroot = (size_t)cfg.nb[0] * cfg.nb[1] * cfg.nb[2];
    root.assign(nroot, -1);
    leaf_at.clear();
    for (size_t b = 0; b < leaf.size(); ++b) {
      const LeafId& id = leaf[b];
      if (id.level == 0) root[root_slot(id.lx[0], id.lx[1], id.lx[2])] = (int32_t)b;
      leaf_at[{id.level, id.lx[0], id.lx[1], id.lx[2]}] = (int32_t)b;
    }
  }

  // Number of blocks along d at level l.
  int64_t nblk(int d, int l) const { return (int64_t)cfg.nb[d] << l; }

  // The leaf covering block location blk of level L (Sec. 2.1: every
  // location is covered by exactly one leaf): its index, with its level in
  // *lev (<= L), or -1 when finer leaves cover it.
  int cover(int L, const int64_t blk[3], int* lev) const {
    for (int d = 0; d <= L; ++d) {
      const int sh = L - d;
      if (d == 0) {
        const int b = root[root_slot(blk[0] >> sh, blk[1] >> sh, blk[2] >> sh)];
        if (b >= 0) { *lev = 0; return b; }
        continue;
      }
      auto it = leaf_at.find({d, blk[0] >> sh, blk[1] >> sh, blk[2] >> sh});
      if (it != leaf_at.end()) { *lev = d; return it->second; }
    }
    return -1;
  }

  // Block location of level l adjacent to blk in direction o (each -1, 0, +1):
  // false across a physical (non-periodic) boundary, else wrapped.
  bool neighbour(int l, const int64_t blk[3], const int o[3], int64_t out[3]) const {
    for (int d = 0; d < 3; ++d) {
      int64_t x = blk[d] + o[d];
      const int64_t n = nblk(d, l);
      if (x < 0 || x >= n) {
        if (cfg.bc[2 * d + (x < 0 ? 0 : 1)] != BC_PERIODIC) return false;
        x = wrap(x, n);
      }
      out[d] = x;
    }
    return true;
  }

  static int64_t wrap(int64_t i, int64_t n) { return ((i % n) + n) % n; }

  // Interior value of leaf b at global cell (I,J,K) of the leaf's own level.
  void leaf_value(int b, int64_t I, int64_t J, int64_t K, R out[NMAX]) const {
    const LeafId& id = leaf[b];
    int i = (int)(I - id.lx[0] * cfg.nx[0]) + NG;
    int j = (int)(J - id.lx[1] * cfg.nx[1]) + NG;
    int k = (int)(K - id.lx[2] * cfg.nx[2]) + NG;
    for (int v = 0; v < nv(); ++v) out[v] = U[b][idx(v, k, j, i)];
  }

  // The composite field: the value of cell (I,J,K) of level L built from the
  // interior data of the leaves only, level by level.  Covered by a leaf of
  // level L: copy.  Covered by finer leaves: restriction = mean of the 8 cells
  // of level L+1 (Sec. 3.7, "restricted first").  Covered by a coarser leaf:
  // prolongation from level L-1 (Sec. 3.7, "interpolated (prolongated)");
  // reading: u_f = u_c + sum_d s_d minmod(u_c - u_{c-e_d}, u_{c+e_d} - u_c),
  // s_d = +-1/4, evaluated d = 1,2,3 in order, with the coarse values taken
  // from the composite field of level L-1 (itself prolonged or restricted
  // where no level-(L-1) leaf covers them).
  void composite(int L, int64_t I, int64_t J, int64_t K, R out[NMAX]) const {
    int64_t X[3] = {I, J, K};
    bool flip[3] = {false, false, false};
    bool outside = false;
    for (int d = 0; d < 3; ++d) {
      const int64_t n = ncell(d, L);
      if (X[d] >= 0 && X[d] < n) continue;
      const int side = X[d] < 0 ? 0 : 1;
      const int bc = cfg.bc[2 * d + side];
      if (bc == BC_PERIODIC) {
        X[d] = wrap(X[d], n);
      } else if (bc == BC_OUTFLOW) {
        X[d] = side ? n - 1 : 0;
        outside = true;
      } else {
        X[d] = side ? 2 * n - 1 - X[d] : -1 - X[d];
        flip[d] = true;
        outside = true;
      }
    }
    if (outside) {  // the image inside the domain, then the mirrored momenta
      composite(L, X[0], X[1], X[2], out);
      for (int d = 0; d < 3; ++d)
        if (flip[d]) out[IM1 + d] = -out[IM1 + d];
      return;
    }
    I = X[0];
    J = X[1];
    K = X[2];
    const int64_t blk[3] = {I / cfg.nx[0], J / cfg.nx[1], K / cfg.nx[2]};
    int lev = 0;
    const int b = cover(L, blk, &lev);
    if (b >= 0 && lev == L) {  // a leaf of this level covers it
      leaf_value(b, I, J, K, out);
      return;
    }
    if (b >= 0) {  // a coarser leaf covers it: prolongation from level L-1
      int64_t C[3] = {I >> 1, J >> 1, K >> 1};
      int64_t F[3] = {I, J, K};
      R uc[NMAX];
      composite(L - 1, C[0], C[1], C[2], uc);
      R acc[NMAX];
      for (int v = 0; v < nv(); ++v) acc[v] = uc[v];
      for (int d = 0; d < 3; ++d) {
        int64_t cm[3] = {C[0], C[1], C[2]}, cp[3] = {C[0], C[1], C[2]};
        cm[d] -= 1;
        cp[d] += 1;
        R um[NMAX], up[NMAX];
        composite(L - 1, cm[0], cm[1], cm[2], um);
        composite(L - 1, cp[0], cp[1], cp[2], up);
        double sgn = (F[d] & 1) ? 0.25 : -0.25;
        for (int v = 0; v < nv(); ++v)
          acc[v] = acc[v] + sgn * minmod(R(uc[v] - um[v]), R(up[v] - uc[v]));
      }
      for (int v = 0; v < nv(); ++v) out[v] = acc[v];
      return;
    }
    // finer leaves cover it: restriction = mean of the 8 cells of level L+1,
    // summed c3 outer, c1 inner
    R sum[NMAX];
    for (int v = 0; v < nv(); ++v) sum[v] = R(0.0);
    for (int c3 = 0; c3 < 2; ++c3)
      for (int c2 = 0; c2 < 2; ++c2)
        for (int c1 = 0; c1 < 2; ++c1) {
          R f[NMAX];
          composite(L + 1, 2 * I + c1, 2 * J + c2, 2 * K + c3, f);
          for (int v = 0; v < nv(); ++v) sum[v] = sum[v] + f[v];
        }
    for (int v = 0; v < nv(); ++v) out[v] = 0.125 * sum[v];
  }

  bool is_interior(int i, int j, int k) const {
    return i >= NG && i < NG + cfg.nx[0] && j >= NG && j < NG + cfg.nx[1] && k >= NG &&
           k < NG + cfg.nx[2];
  }

  // Ghost exchange (Sec. 3.7): every ghost cell of every leaf (faces, edges and
  // corners, all 26 neighbour regions) takes the composite-field value there.
  void fill_ghosts() {
    for (size_t b = 0; b < leaf.size(); ++b) {
      const LeafId& id = leaf[b];
      for (int k = 0; k < S(2); ++k)
        for (int j = 0; j < S(1); ++j)
          for (int i = 0; i < S(0); ++i) {
            if (is_interior(i, j, k)) continue;
            R val[NMAX];
            composite(id.level, id.lx[0] * cfg.nx[0] + i - NG, id.lx[1] * cfg.nx[1] + j - NG,
                      id.lx[2] * cfg.nx[2] + k - NG, val);
            for (int v = 0; v < nv(); ++v) U[b][idx(v, k, j, i)] = val[v];
          }
    }
  }

  void prim_at(const std::vector<R>& u, int k, int j, int i, R w[NMAX]) {
    R c[NMAX];
    for (int v = 0; v < nv(); ++v) c[v] = u[idx(v, k, j, i)];
    cons_to_prim(c, w, gamma, cfg.dfloor, cfg.pfloor, &floors, cfg.nscalars);
  }

  // Face fluxes of one leaf along direction d.  Face f lies between interior
  // cells f-1 and f (0 <= f <= n_d); its left state is reconstructed in cell
  // f-1 and its right state in cell f.
  // Layout: flux[((v * n3' + k) * n2' + j) * n1' + i] with n_d' = n_d + (d==dir).
  struct Fluxes {
    int n[3];
    std::vector<R> f;
    R& at(int v, int k, int j, int i) {
      return f[(((size_t)v * n[2] + k) * n[1] + j) * n[0] + i];
    }
  };

  Fluxes face_fluxes(int b, int dir) {
    Fluxes F;
    for (int d = 0; d < 3; ++d) F.n[d] = cfg.nx[d] + (d == dir ? 1 : 0);
    F.f.assign((size_t)nv() * F.n[0] * F.n[1] * F.n[2], R(0.0));
    const std::vector<R>& u = U[b];
    int e[3] = {dir == 0, dir == 1, dir == 2};
    for (int k = 0; k < F.n[2]; ++k)
      for (int j = 0; j < F.n[1]; ++j)
        for (int i = 0; i < F.n[0]; ++i) {
          // array indices of cell f (right of the face)
          int ci = i + NG, cj = j + NG, ck = k + NG;
          R w[4][NMAX];  // cells f-2, f-1, f, f+1 along dir
          for (int s = 0; s < 4; ++s)
            prim_at(u, ck + (s - 2) * e[2], cj + (s - 2) * e[1], ci + (s - 2) * e[0], w[s]);
          R wl[NMAX], wr[NMAX];
          for (int v = 0; v < nv(); ++v) {
            R dl = vanleer(w[0][v], w[1][v], w[2][v]);
            R dr = vanleer(w[1][v], w[2][v], w[3][v]);
            wl[v] = w[1][v] + 0.5 * dl;
            wr[v] = w[2][v] - 0.5 * dr;
          }
          R fl[NMAX];
          hlle_flux(wl, wr, dir, gamma, fl, cfg.nscalars);
          for (int v = 0; v < nv(); ++v) F.at(v, k, j, i) = fl[v];
        }
    return F;
  }

  // Flux correction (Sec. 3.7): at a face shared by a leaf of level l and
  // leaves of level l+1, the coarse flux is replaced by the mean of the 4 fine
  // fluxes over it (summed t1 inner, t2 outer).
  void flux_correct(std::vector<std::array<Fluxes, 3>>& F) {
    if (cfg.max_level < 1) return;
    for (size_t b = 0; b < leaf.size(); ++b) {
      const LeafId& id = leaf[b];
      const int l = id.level;
      if (l >= cfg.max_level) continue;
      for (int d = 0; d < 3; ++d) {
        int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
        for (int side = 0; side < 2; ++side) {
          int o[3] = {0, 0, 0};
          o[d] = side ? 1 : -1;
          int64_t nb_[3];
          if (!neighbour(l, id.lx, o, nb_)) continue;  // physical boundary: nothing to correct
          int lev = 0;
          if (cover(l, nb_, &lev) >= 0) continue;      // same-level or coarser neighbour
          int cface = side ? cfg.nx[d] : 0;  // coarse face index along d
          int fface = side ? 0 : cfg.nx[d];  // fine face index along d in the fine block
          int childd = side ? 0 : 1;         // child offset along d adjacent to the face
          for (int a2 = 0; a2 < cfg.nx[t2]; ++a2)
            for (int a1 = 0; a1 < cfg.nx[t1]; ++a1) {
              R sum[NMAX];
              for (int v = 0; v < nv(); ++v) sum[v] = R(0.0);
              for (int q2 = 0; q2 < 2; ++q2)
                for (int q1 = 0; q1 < 2; ++q1) {
                  int64_t g1 = 2 * (id.lx[t1] * cfg.nx[t1] + a1) + q1;  // fine global index
                  int64_t g2 = 2 * (id.lx[t2] * cfg.nx[t2] + a2) + q2;
                  int64_t fblk[3];
                  fblk[d] = 2 * nb_[d] + childd;
                  fblk[t1] = g1 / cfg.nx[t1];
                  fblk[t2] = g2 / cfg.nx[t2];
                  auto it = leaf_at.find({l + 1, fblk[0], fblk[1], fblk[2]});
                  const int fb = it->second;  // exists: neighbours differ by one level at most
                  int lc[3];
                  lc[d] = fface;
                  lc[t1] = (int)(g1 % cfg.nx[t1]);
                  lc[t2] = (int)(g2 % cfg.nx[t2]);
                  for (int v = 0; v < nv(); ++v)
                    sum[v] = sum[v] + F[fb][d].at(v, lc[2], lc[1], lc[0]);
                }
              int lc[3];
              lc[d] = cface;
              lc[t1] = a1;
              lc[t2] = a2;
              for (int v = 0; v < nv(); ++v) F[b][d].at(v, lc[2], lc[1], lc[0]) = 0.25 * sum[v];
            }
        }
      }
    }
  }

  // One stage of the two-stage Runge-Kutta integrator (Sec. 4.1).  Reading:
  // SSPRK2 (Heun) in the form
  //   stage 1: U1 = U0 + dt L(U0)
  //   stage 2: U  = 0.5 U0 + 0.5 (U1 + dt L(U1))
  // with L(U) = -[(F1_{i+1/2}-F1_{i-1/2})/dx1 + (F2..)/dx2 + (F3..)/dx3],
  // summed x1, then x2, then x3 (flux divergence, Sec. 3.7).
  void stage(int which, const std::vector<std::vector<R>>& U0, double dtv) {
    std::vector<std::array<Fluxes, 3>> F(leaf.size());
    for (size_t b = 0; b < leaf.size(); ++b)
      for (int d = 0; d < 3; ++d) F[b][d] = face_fluxes((int)b, d);
    flux_correct(F);
    for (size_t b = 0; b < leaf.size(); ++b) {
      int lev = leaf[b].level;
      double h1 = dx(0, lev), h2 = dx(1, lev), h3 = dx(2, lev);
      for (int k = 0; k < cfg.nx[2]; ++k)
        for (int j = 0; j < cfg.nx[1]; ++j)
          for (int i = 0; i < cfg.nx[0]; ++i)
            for (int v = 0; v < nv(); ++v) {
              R L = -((F[b][0].at(v, k, j, i + 1) - F[b][0].at(v, k, j, i)) / h1 +
                      (F[b][1].at(v, k, j + 1, i) - F[b][1].at(v, k, j, i)) / h2 +
                      (F[b][2].at(v, k + 1, j, i) - F[b][2].at(v, k, j, i)) / h3);
              size_t c = idx(v, k + NG, j + NG, i + NG);
              if (which == 1)
                U[b][c] = U0[b][c] + dtv * L;
              else
                U[b][c] = 0.5 * U0[b][c] + 0.5 * (U[b][c] + dtv * L);
            }
    }
  }

  // CFL time step (Sec. 3.10, global min-reduction).  Reading:
  // dt = cfl * min over interior cells of all leaves and d of dx_d/(|v_d|+c_s),
  // c_s = sqrt(gamma p / rho), in FP64, from the real part of the state.
  double compute_dt() {
    double m = INFINITY;
    for (size_t b = 0; b < leaf.size(); ++b) {
      int lev = leaf[b].level;
      for (int k = NG; k < NG + cfg.nx[2]; ++k)
        for (int j = NG; j < NG + cfg.nx[1]; ++j)
          for (int i = NG; i < NG + cfg.nx[0]; ++i) {
            double u[NMAX], w[NMAX];
            for (int v = 0; v < nv(); ++v) u[v] = re(U[b][idx(v, k, j, i)]);
            long dummy = 0;
            cons_to_prim(u, w, re(gamma), cfg.dfloor, cfg.pfloor, &dummy);
            double cs = std::sqrt(re(gamma) * w[IEN] / w[IDN]);
            for (int d = 0; d < 3; ++d) {
              double c = dx(d, lev) / (std::fabs(w[IM1 + d]) + cs);
              if (c < m) m = c;
            }
          }
    }
    return cfg.cfl * m;
  }

  // One full cycle with a given dt: two stages, each followed by ghost exchange.
  void cycle_with_dt(double dtv) {
    std::vector<std::vector<R>> U0 = U;
    stage(1, U0, dtv);
    fill_ghosts();
    stage(2, U0, dtv);
    fill_ghosts();
    time += dtv;
    cycle += 1;
    dt = dtv;
    for (auto& a : age) a += 1;
  }

  // Refinement indicator (reading): m_b = max over interior cells and d of
  // |rho_{i+e_d} - rho_{i-e_d}| / (2 rho_i), using the ghost-filled density.
  double indicator(int b) const {
    double m = 0.0;
    const std::vector<R>& u = U[b];
    for (int k = NG; k < NG + cfg.nx[2]; ++k)
      for (int j = NG; j < NG + cfg.nx[1]; ++j)
        for (int i = NG; i < NG + cfg.nx[0]; ++i) {
          double r0 = re(u[idx(IDN, k, j, i)]);
          double g[3] = {
              std::fabs(re(u[idx(IDN, k, j, i + 1)]) - re(u[idx(IDN, k, j, i - 1)])) / (2.0 * r0),
              std::fabs(re(u[idx(IDN, k, j + 1, i)]) - re(u[idx(IDN, k, j - 1, i)])) / (2.0 * r0),
              std::fabs(re(u[idx(IDN, k + 1, j, i)]) - re(u[idx(IDN, k - 1, j, i)])) / (2.0 * r0)};
          for (int d = 0; d < 3; ++d)
            if (g[d] > m) m = g[d];
        }
    return m;
  }

  // Flags: +1 refine when m_b > refine_tol and level < max_level; -1 derefine
  // when m_b < derefine_tol and level > 0 and the block is not pinned by the
  // static region; 0 otherwise.
  void tag(std::vector<int8_t>& flags, std::vector<double>* mb) const {
    flags.assign(leaf.size(), 0);
    if (mb) mb->assign(leaf.size(), 0.0);
    for (size_t b = 0; b < leaf.size(); ++b) {
      double m = indicator((int)b);
      if (mb) (*mb)[b] = m;
      if (m > cfg.refine_tol && leaf[b].level < cfg.max_level)
        flags[b] = 1;
      else if (m < cfg.derefine_tol && leaf[b].level > 0 && !in_static_region(leaf[b]))
        flags[b] = -1;
    }
  }

  // Rebuild the tree (Sec. 2.1/3.8): refine every +1 leaf into 8 children;
  // merge 8 siblings that are all -1 and at least derefine_count cycles old
  // ("derefinement only allowed periodically").  Reading (the Athena++ rule
  // the paper defers to): leaves that touch -- across a face, an edge or a
  // corner -- differ by one level at most, so refining a leaf first refines
  // every touching leaf that is coarser than it (repeated until nothing more
  // changes), and 8 siblings do not merge if a leaf touching their parent
  // would then be two levels finer.  New data is the composite field of the
  // old mesh at the new leaf's level: prolongation for new children,
  // restriction for merged parents.  Returns true if the tree changed.
  bool remesh(const std::vector<int8_t>& flags, bool check_age = true) {
    static const int kDirs = 27;
    auto dir = [](int q, int o[3]) {
      o[0] = q % 3 - 1;
      o[1] = (q / 3) % 3 - 1;
      o[2] = q / 9 - 1;
    };
    // 1. refinement set, closed under the one-level rule
    std::set<int> refine;
    for (size_t b = 0; b < leaf.size(); ++b)
      if (flags[b] == 1 && leaf[b].level < cfg.max_level) refine.insert((int)b);
    std::vector<int> work(refine.begin(), refine.end());
    while (!work.empty()) {
      const int a = work.back();
      work.pop_back();
      const LeafId& A = leaf[a];
      for (int q = 0; q < kDirs; ++q) {
        int o[3];
        dir(q, o);
        if (o[0] == 0 && o[1] == 0 && o[2] == 0) continue;
        int64_t nbk[3];
        if (!neighbour(A.level, A.lx, o, nbk)) continue;
        int lev = 0;
        const int c = cover(A.level, nbk, &lev);
        if (c >= 0 && lev < A.level && !refine.count(c)) {
          refine.insert(c);
          work.push_back(c);
        }
      }
    }
    // 2. merges: complete sibling sets, all -1, old enough, not static, none
    //    refined now, and no leaf touching the parent left two levels finer
    std::vector<LeafId> nl;
    std::vector<int32_t> na;
    std::vector<bool> keep_old(leaf.size(), true);
    bool changed = !refine.empty();
    for (int b : refine) {
      keep_old[b] = false;
      const LeafId& P = leaf[b];
      for (int c = 0; c < 8; ++c) {
        nl.push_back(LeafId{P.level + 1, {2 * P.lx[0] + (c & 1), 2 * P.lx[1] + ((c >> 1) & 1),
                                          2 * P.lx[2] + ((c >> 2) & 1)}});
        na.push_back(0);
      }
    }
    std::set<std::array<int64_t, 4>> parents_done;
    for (size_t b = 0; b < leaf.size(); ++b) {
      const LeafId& K = leaf[b];
      if (K.level == 0) continue;
      const int pl = K.level - 1;
      const int64_t P[3] = {K.lx[0] >> 1, K.lx[1] >> 1, K.lx[2] >> 1};
      if (!parents_done.insert({pl, P[0], P[1], P[2]}).second) continue;
      int sib[8];
      bool ok = true;
      for (int c = 0; c < 8 && ok; ++c) {
        auto it = leaf_at.find({K.level, 2 * P[0] + (c & 1), 2 * P[1] + ((c >> 1) & 1),
                                2 * P[2] + ((c >> 2) & 1)});
        if (it == leaf_at.end()) { ok = false; break; }
        const int sb = it->second;
        sib[c] = sb;
        if (flags[sb] != -1 || (check_age && age[sb] < cfg.derefine_count) ||
            in_static_region(leaf[sb]) || refine.count(sb))
          ok = false;
      }
      for (int q = 0; q < kDirs && ok; ++q) {
        int o[3];
        dir(q, o);
        if (o[0] == 0 && o[1] == 0 && o[2] == 0) continue;
        int64_t nbk[3];
        if (!neighbour(pl, P, o, nbk)) continue;
        int lev = 0;
        const int c = cover(pl, nbk, &lev);
        if (c >= 0) continue;  // covered at the parent's level or coarser
        // finer: every child block of the neighbour that touches the parent
        // must be a leaf of level pl+1 that is not being refined
        for (int cc = 0; cc < 8 && ok; ++cc) {
          const int cb[3] = {cc & 1, (cc >> 1) & 1, (cc >> 2) & 1};
          bool touches = true;
          for (int d = 0; d < 3; ++d)
            if ((o[d] == 1 && cb[d] != 0) || (o[d] == -1 && cb[d] != 1)) touches = false;
          if (!touches) continue;
          auto it = leaf_at.find({pl + 1, 2 * nbk[0] + cb[0], 2 * nbk[1] + cb[1], 2 * nbk[2] + cb[2]});
          if (it == leaf_at.end() || refine.count(it->second)) ok = false;
        }
      }
      if (!ok) continue;
      changed = true;
      for (int c = 0; c < 8; ++c) keep_old[sib[c]] = false;
      nl.push_back(LeafId{pl, {P[0], P[1], P[2]}});
      na.push_back(0);
    }
    if (!changed) return false;
    for (size_t b = 0; b < leaf.size(); ++b)
      if (keep_old[b]) { nl.push_back(leaf[b]); na.push_back(age[b]); }
    // new data from the old mesh's composite field
    std::vector<std::vector<R>> nu(nl.size(), std::vector<R>(block_len(), R(0.0)));
    for (size_t b = 0; b < nl.size(); ++b) {
      const LeafId& id = nl[b];
      for (int k = NG; k < NG + cfg.nx[2]; ++k)
        for (int j = NG; j < NG + cfg.nx[1]; ++j)
          for (int i = NG; i < NG + cfg.nx[0]; ++i) {
            R val[NMAX];
            composite(id.level, id.lx[0] * cfg.nx[0] + i - NG, id.lx[1] * cfg.nx[1] + j - NG,
                      id.lx[2] * cfg.nx[2] + k - NG, val);
            for (int v = 0; v < nv(); ++v) nu[b][idx(v, k, j, i)] = val[v];
          }
    }
    leaf.swap(nl);
    age.swap(na);
    U.swap(nu);
    sort_and_index();
    fill_ghosts();
    return true;
  }

  // One driver cycle (Sec. 3.11 EvolutionDriver/MultiStageDriver): dt from the
  // current state, the two stages, then tagging and remesh when adaptive.
  void step_one() {
    double dtv = compute_dt();
    cycle_with_dt(dtv);
    if (cfg.adaptive && cfg.max_level >= 1) {
      std::vector<int8_t> flags;
      tag(flags, nullptr);
      remesh(flags);
    }
  }

  // Conserved totals: sum over interior cells of all leaves of U_v dV, with
  // Neumaier's compensated summation so that the sum itself adds no
  // round-off that a conservation check could mistake for a flux error.
  void totals(double out[NMAX]) const {
    for (int v = 0; v < nv(); ++v) {
      double s = 0.0, comp = 0.0;
      for (size_t b = 0; b < leaf.size(); ++b) {
        int lev = leaf[b].level;
        double dv = dx(0, lev) * dx(1, lev) * dx(2, lev);
        for (int k = NG; k < NG + cfg.nx[2]; ++k)
          for (int j = NG; j < NG + cfg.nx[1]; ++j)
            for (int i = NG; i < NG + cfg.nx[0]; ++i) {
              double x = re(U[b][idx(v, k, j, i)]) * dv;
              double t = s + x;
              if (std::fabs(s) >= std::fabs(x))
                comp += (s - t) + x;
              else
                comp += (x - t) + s;
              s = t;
            }
      }
      out[v] = s + comp;
    }
  }
};

}  // namespace ho
