// hydro_oracle.cpp -- extern "C" entry points of the FP64 CPU oracle.
//
// TEST INFRASTRUCTURE ONLY (see hydro_oracle.hpp).  Built into
// oracle/liboracle.so with -O2 -ffp-contract=off so that every expression is
// evaluated exactly as written, one IEEE operation at a time.
#include "hydro_oracle.hpp"

#include <type_traits>

using ho::cplx;
using ho::Config;
using ho::Mesh;
using ho::NG;
using ho::NVAR;

namespace {

template <class R>
void copy_interior_in(Mesh<R>& m, const double* U, const double* V, double h) {
  size_t n1 = m.cfg.nx[0], n2 = m.cfg.nx[1], n3 = m.cfg.nx[2];
  size_t per = (size_t)m.nv() * n1 * n2 * n3;
  for (size_t b = 0; b < m.leaf.size(); ++b)
    for (int v = 0; v < m.nv(); ++v)
      for (size_t k = 0; k < n3; ++k)
        for (size_t j = 0; j < n2; ++j)
          for (size_t i = 0; i < n1; ++i) {
            size_t s = b * per + ((v * n3 + k) * n2 + j) * n1 + i;
            R val = R(U[s]);
            if constexpr (std::is_same<R, cplx>::value) {
              if (V) val = cplx(U[s], h * V[s]);
            }
            m.U[b][m.idx(v, (int)k + NG, (int)j + NG, (int)i + NG)] = val;
          }
  m.fill_ghosts();
}

}  // namespace

extern "C" {

void* or_create(const Config* cfg) { return new Mesh<double>(*cfg); }
void or_destroy(void* h) { delete static_cast<Mesh<double>*>(h); }
int or_num_blocks(void* h) { return (int)static_cast<Mesh<double>*>(h)->leaf.size(); }

// Leaves in Z-order: 4 int64 per leaf (level, lx1, lx2, lx3).
void or_tree(void* h, int64_t* out) {
  auto* m = static_cast<Mesh<double>*>(h);
  for (size_t b = 0; b < m->leaf.size(); ++b) {
    out[4 * b + 0] = m->leaf[b].level;
    for (int d = 0; d < 3; ++d) out[4 * b + 1 + d] = m->leaf[b].lx[d];
  }
}

// Interior state, layout [b][v][k][j][i]; ghosts are filled afterwards.
void or_set_state(void* h, const double* U) {
  copy_interior_in(*static_cast<Mesh<double>*>(h), U, nullptr, 0.0);
}

void or_get_state(void* h, double* U) {
  auto* m = static_cast<Mesh<double>*>(h);
  size_t n1 = m->cfg.nx[0], n2 = m->cfg.nx[1], n3 = m->cfg.nx[2];
  size_t per = (size_t)m->nv() * n1 * n2 * n3;
  for (size_t b = 0; b < m->leaf.size(); ++b)
    for (int v = 0; v < m->nv(); ++v)
      for (size_t k = 0; k < n3; ++k)
        for (size_t j = 0; j < n2; ++j)
          for (size_t i = 0; i < n1; ++i)
            U[b * per + ((v * n3 + k) * n2 + j) * n1 + i] =
                m->U[b][m->idx(v, (int)k + NG, (int)j + NG, (int)i + NG)];
}

// Whole blocks including ghosts, layout [b][v][k][j][i] over (n+2g)^3.
void or_get_full(void* h, double* U) {
  auto* m = static_cast<Mesh<double>*>(h);
  size_t len = m->block_len();
  for (size_t b = 0; b < m->leaf.size(); ++b)
    for (size_t c = 0; c < len; ++c) U[b * len + c] = m->U[b][c];
}

void or_fill_ghosts(void* h) { static_cast<Mesh<double>*>(h)->fill_ghosts(); }
double or_compute_dt(void* h) { return static_cast<Mesh<double>*>(h)->compute_dt(); }

// n driver cycles; dt of each cycle written to dts_out when not null.
void or_step(void* h, int n, double* dts_out) {
  auto* m = static_cast<Mesh<double>*>(h);
  for (int c = 0; c < n; ++c) {
    m->step_one();
    if (dts_out) dts_out[c] = m->dt;
  }
}

// n cycles with a prescribed dt schedule (no tagging).
void or_step_dt(void* h, int n, const double* dts) {
  auto* m = static_cast<Mesh<double>*>(h);
  for (int c = 0; c < n; ++c) m->cycle_with_dt(dts[c]);
}

// One stage only, for per-stage parity (which = 1 or 2; U0 = state before stage 1).
void or_stage(void* h, int which, const double* U0_interior, double dt) {
  auto* m = static_cast<Mesh<double>*>(h);
  Mesh<double> tmp(*m);
  copy_interior_in(tmp, U0_interior, nullptr, 0.0);
  m->stage(which, tmp.U, dt);
  m->fill_ghosts();
}

void or_get_time(void* h, double* t, double* dt, int64_t* cycle) {
  auto* m = static_cast<Mesh<double>*>(h);
  *t = m->time;
  *dt = m->dt;
  *cycle = m->cycle;
}

void or_totals(void* h, double* out) { static_cast<Mesh<double>*>(h)->totals(out); }
long or_floor_hits(void* h) { return static_cast<Mesh<double>*>(h)->floors; }

void or_tag(void* h, int8_t* flags, double* mb) {
  auto* m = static_cast<Mesh<double>*>(h);
  std::vector<int8_t> f;
  std::vector<double> v;
  m->tag(f, &v);
  for (size_t b = 0; b < f.size(); ++b) {
    flags[b] = f[b];
    if (mb) mb[b] = v[b];
  }
}

int or_remesh(void* h, const int8_t* flags, int check_age) {
  auto* m = static_cast<Mesh<double>*>(h);
  std::vector<int8_t> f(flags, flags + m->leaf.size());
  return m->remesh(f, check_age != 0) ? 1 : 0;
}

void or_composite(void* h, int L, int64_t I, int64_t J, int64_t K, double* out) {
  static_cast<Mesh<double>*>(h)->composite(L, I, J, K, out);
}

// Pointwise pieces, for unit pins.
void or_cons_to_prim(const double* u, double* w, double gamma, double dfloor, double pfloor) {
  long f = 0;
  ho::cons_to_prim(u, w, gamma, dfloor, pfloor, &f);
}
double or_vanleer(double a, double b, double c) { return ho::vanleer(a, b, c); }
double or_minmod(double a, double b) { return ho::minmod(a, b); }
void or_hlle(const double* wl, const double* wr, int dir, double gamma, double* f) {
  ho::hlle_flux(wl, wr, dir, gamma, f);
}
uint64_t or_morton(int level, int64_t l1, int64_t l2, int64_t l3, int max_level) {
  ho::LeafId id{level, {l1, l2, l3}};
  return ho::morton_key(id, max_level);
}

// Complex-step directional derivative (Squire & Trapp 1998) of
//   J(U0, gamma) = sum over interior cells (rho_final - rho_target)^2
// along (V, dgamma): runs the uniform mesh for ncycles with the dt schedule
// `dts` (frozen, as the adjoint uses it), perturbing U0 by i h V and gamma by
// i h dgamma.  Writes J and dJ = Im(J(U0 + i h V, gamma + i h dgamma)) / h.
void or_jvp(const Config* cfg, const double* U0, const double* V, double dgamma,
            const double* rho_target, int ncycles, const double* dts, double h, double* J,
            double* dJ) {
  Mesh<cplx> m(*cfg);
  m.gamma = cplx(cfg->gamma, h * dgamma);
  copy_interior_in(m, U0, V, h);
  for (int c = 0; c < ncycles; ++c) m.cycle_with_dt(dts[c]);
  size_t n1 = cfg->nx[0], n2 = cfg->nx[1], n3 = cfg->nx[2];
  cplx acc(0.0, 0.0);
  for (size_t b = 0; b < m.leaf.size(); ++b)
    for (size_t k = 0; k < n3; ++k)
      for (size_t j = 0; j < n2; ++j)
        for (size_t i = 0; i < n1; ++i) {
          cplx d = m.U[b][m.idx(ho::IDN, (int)k + NG, (int)j + NG, (int)i + NG)] -
                   rho_target[b * (n1 * n2 * n3) + (k * n2 + j) * n1 + i];
          acc += d * d;
        }
  *J = acc.real();
  *dJ = acc.imag() / h;
}

// Complex-step tangent of the whole final state: runs the uniform mesh for
// ncycles with the frozen dt schedule from U0 + i h V (gamma + i h dgamma)
// and writes the final interior state (real part) and J V (imaginary / h),
// both in the interior layout [b][v][k][j][i].
void or_jvp_state(const Config* cfg, const double* U0, const double* V, double dgamma,
                  int ncycles, const double* dts, double h, double* U_out, double* JV_out) {
  Mesh<cplx> m(*cfg);
  m.gamma = cplx(cfg->gamma, h * dgamma);
  copy_interior_in(m, U0, V, h);
  for (int c = 0; c < ncycles; ++c) m.cycle_with_dt(dts[c]);
  size_t n1 = cfg->nx[0], n2 = cfg->nx[1], n3 = cfg->nx[2];
  size_t per = (size_t)m.nv() * n1 * n2 * n3;
  for (size_t b = 0; b < m.leaf.size(); ++b)
    for (int v = 0; v < m.nv(); ++v)
      for (size_t k = 0; k < n3; ++k)
        for (size_t j = 0; j < n2; ++j)
          for (size_t i = 0; i < n1; ++i) {
            const cplx z = m.U[b][m.idx(v, (int)k + NG, (int)j + NG, (int)i + NG)];
            const size_t s = b * per + ((v * n3 + k) * n2 + j) * n1 + i;
            U_out[s] = z.real();
            JV_out[s] = z.imag() / h;
          }
}

}  // extern "C"
