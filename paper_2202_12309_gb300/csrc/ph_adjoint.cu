// ph_adjoint.cu -- reverse mode of the uniform-mesh cycle: hand-written
// adjoints of the fused stage (cons->prim, PLM, HLLE, divergence, SSPRK2) and
// of the ghost exchange, with checkpoint-every-k recomputation.
//
// The paper has no adjoint; this follows the forward method of Sec. 4.1 line
// by line in reverse.  Readings: the dt schedule of the forward run is held
// fixed (not differentiated); limiter, wave-speed and floor branches are
// frozen at their forward values (decided on the forward state exactly as
// the forward decides them).
//
// For a stage  U_out = a U0 + b (U + dt L(U))  the reverse needs the
// vector-Jacobian product of L.  L_i = -sum_d (F_{i+1/2} - F_{i-1/2}) / dx_d,
// so the adjoint of the face flux F_f between cells a (left) and b (right) is
//   Fbar_f = (mu_b - mu_a) / dx_d,
// which flows back through HLLE to the face states, through
// W_L = W_a + h_a, W_R = W_b - h_b to the cells and their half-slopes h, and
// through each half-slope h_k = vl(W_{k-1}, W_k, W_{k+1}) to three cells;
// finally W -> U by the transpose of the primitive Jacobian.  Per stage: the
// primitives of the stage input once; per direction the faces (HLLE
// reverse), the slopes (each cell's half-slope differentiated once; FP32
// fuses this into the gather) and the gather per cell; then the primitives
// (W -> U).  The transpose of the ghost exchange
// is a gather: an interior cell next to a block face receives the adjoint of
// the face-ghost cell that copied it in the neighbouring block.  Everything
// is a gather with one writer per output, so results are reproducible run to
// run except for the gamma derivative, which is summed with atomics.
#include <algorithm>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/ph_hydro.h"
#include "ph_nvtx.h"
#include "ph_internal.h"

namespace ph {

// ---------------------------------------------------------------------------
// pointwise reverses
// ---------------------------------------------------------------------------

// Forward cons->prim with the branch flags the reverse needs; returns 1/rho.
// Reciprocals, square roots and their inverses in this file are the stage
// kernels' Newton-refined routines (within an ulp or two of the correctly
// rounded ones): the reverse differentiates the same formulas, and a
// derivative needs no more than that.
template <class T>
__device__ __forceinline__ T prim_fwd(const T u[NV], const Phys<T>& P, T w[NV], bool& rf, bool& pf) {
  T rho = u[0];
  rf = rho < P.dfloor;
  if (rf) rho = P.dfloor;
  const T ir = rcp(rho);
  w[0] = rho;
  w[1] = u[1] * ir;
  w[2] = u[2] * ir;
  w[3] = u[3] * ir;
  // the stage kernels' conversion, fma for fma (cons_to_prim)
  T p = P.gm1 * fma(T(-0.5), fma(u[3], w[3], fma(u[2], w[2], u[1] * w[1])), u[4]);
  pf = p < P.pfloor;
  if (pf) p = P.pfloor;
  w[4] = p;
  return ir;
}

// Ubar = (dW/dU)^T Wbar; gamma adjoint of p = (gamma-1)(E - |m|^2/(2 rho)).
template <class T>
__device__ __forceinline__ void prim_rev(const T u[NV], const Phys<T>& P, const T wb[NV], T ub[NV],
                                         double& gbar) {
  bool rf, pf;
  T w[NV];
  const T ir = prim_fwd(u, P, w, rf, pf);
  const T rho = w[0];
  const T pb = pf ? T(0) : wb[4];
  const T v2 = w[1] * w[1] + w[2] * w[2] + w[3] * w[3];
  // p = gm1 * (E - 0.5 rho_u |v|^2) with v = m / rho_used
  T rb = rf ? T(0) : wb[0];
  T mb[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    // dv_a/dm_a = 1/rho ; dp/dm_a = -gm1 v_a
    mb[a] = wb[1 + a] * ir - pb * P.gm1 * w[1 + a];
    // dv_a/drho = -v_a/rho ; only if rho is not floored
    if (!rf) rb -= wb[1 + a] * w[1 + a] * ir;
  }
  if (!rf) rb += pb * P.gm1 * T(0.5) * v2;  // dp/drho = gm1 |v|^2 / 2
  ub[0] = rb;
  ub[1] = mb[0];
  ub[2] = mb[1];
  ub[3] = mb[2];
  ub[4] = pb * P.gm1;
  if (!pf) gbar += (double)pb * (double)(u[4] - T(0.5) * rho * v2);
}

// Half-slope and its partial derivatives (frozen branch dL dR > 0).
template <class T>
__device__ __forceinline__ T vl_half_d(T wm, T w0, T wp, T& dm, T& d0, T& dp) {
  const T dl = w0 - wm, dr = wp - w0, prod = dl * dr;
  if (!(prod > T(0))) {
    dm = d0 = dp = T(0);
    return T(0);
  }
  const T s = dl + dr, is = rcp(s), is2 = is * is;
  const T ddl = dr * dr * is2, ddr = dl * dl * is2;
  dm = -ddl;
  d0 = ddl - ddr;
  dp = ddr;
  return prod * is;
}

// Reverse of the HLLE flux in the factored form of the stage kernels' hlle()
// (ph_device.cuh), with the same forward arithmetic:
//   F = cL F_L + cR F_R + cD (U_R - U_L),  cL = b+/(b+ - b-), cR = -b-/(b+ - b-),
//   cD = b+ b-/(b+ - b-),  alL = cL v_nL - cD,  alR = cR v_nR + cD,
//   aL = alL rho_L, aR = alR rho_R:  F_rho = aL + aR,
//   F_v = aL v_L + aR v_R (+ cL p_L + cR p_R on the normal component),
//   F_E = alL (rho h)_L + alR (rho h)_R - cD (p_R - p_L).
// Einfeldt's max / min and the Roe sound-speed clip are frozen at their
// forward choices.  Accumulates wlb, wrb (primitive adjoints) and gbar
// (d/d gamma: gamma enters through 1/(gamma-1) in rho h, gamma - 1 in the
// Roe sound speed and gamma p in the sound speeds).
template <class T, int DIR>
__device__ void hlle_rev(const T wl[NV], const T wr[NV], const Phys<T>& P, const T fb[NV], T wlb[NV],
                         T wrb[NV], double& gbar) {
  constexpr int IN = 1 + DIR;
  constexpr int IB = 1 + (DIR + 1) % 3, IC = 1 + (DIR + 2) % 3;
  // ---- forward
  const T rl = wl[0], pl = wl[4], rr = wr[0], pr = wr[4];
  const T vnl = wl[IN], vnr = wr[IN];
  const T kl = fma(wl[IN], wl[IN], fma(wl[IB], wl[IB], wl[IC] * wl[IC]));
  const T kr = fma(wr[IN], wr[IN], fma(wr[IB], wr[IB], wr[IC] * wr[IC]));
  const T hl = fma(pl, P.igm1, fma(T(0.5) * rl, kl, pl));  // rho h
  const T hr = fma(pr, P.igm1, fma(T(0.5) * rr, kr, pr));
  const T ql = rsq(rl), qr = rsq(rr);                      // 1/sqrt(rho)
  const T sl = rl * ql, sr = rr * qr;                      // sqrt(rho)
  const T gl = sq(P.gamma * pl), gr = sq(P.gamma * pr);    // c = g / sqrt(rho)
  const T isum = rcp(sl + sr);
  const T wsl = sl * isum, wsr = sr * isum;
  T u[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) u[a] = fma(wsl, wl[1 + a], wsr * wr[1 + a]);
  const T t = fma(hl, ql, hr * qr);
  const T hroe = t * isum;
  const T usq = fma(u[IN - 1], u[IN - 1], fma(u[IB - 1], u[IB - 1], u[IC - 1] * u[IC - 1]));
  const T a2 = P.gm1 * fma(T(-0.5), usq, hroe);
  const bool a2pos = positive(a2);
  const T croe = a2pos ? sq(a2) : T(0);
  const T un = u[IN - 1];
  const T A = fma(gr, qr, vnr), B = un + croe;
  const T C = fma(-gl, ql, vnl), D = un - croe;
  const T bp = max0(A, B), bm = min0(C, D);
  const T idb = rcp(bp - bm);
  const T cL = bp * idb, cR = -bm * idb, cD = (bp * bm) * idb;
  const T alL = fma(cL, vnl, -cD), alR = fma(cR, vnr, cD);
  const T aL = alL * rl, aR = alR * rr;
  // ---- reverse
  T aLb = fb[0], aRb = fb[0];
#pragma unroll
  for (int a = 1; a <= 3; ++a) {
    aLb = fma(fb[a], wl[a], aLb);
    aRb = fma(fb[a], wr[a], aRb);
    wlb[a] += fb[a] * aL;
    wrb[a] += fb[a] * aR;
  }
  T cLb = fb[IN] * pl, cRb = fb[IN] * pr;
  T plb = fma(fb[IN], cL, fb[4] * cD), prb = fma(fb[IN], cR, -fb[4] * cD);
  T cDb = -fb[4] * (pr - pl);
  T hlb = fb[4] * alL, hrb = fb[4] * alR;
  const T alLb = fma(fb[4], hl, aLb * rl), alRb = fma(fb[4], hr, aRb * rr);
  T rlb = aLb * alL, rrb = aRb * alR;
  cLb = fma(alLb, vnl, cLb);
  cRb = fma(alRb, vnr, cRb);
  cDb += alRb - alLb;
  T vnlb = alLb * cL, vnrb = alRb * cR;
  T bpb = fma(cDb, bm, cLb) * idb, bmb = fma(cDb, bp, -cRb) * idb;
  {
    const T idbb = fma(cLb, bp, fma(-cRb, bm, cDb * (bp * bm)));
    const T db = -idb * idb * idbb;  // idb = 1/(b+ - b-)
    bpb += db;
    bmb -= db;
  }
  T Ab = T(0), Bb = T(0), Cb = T(0), Db = T(0);
  if (bp > T(0)) {
    if (A >= B) Ab = bpb; else Bb = bpb;
  }
  if (bm < T(0)) {
    if (C <= D) Cb = bmb; else Db = bmb;
  }
  T grb = Ab * qr, qrb = Ab * gr;
  T glb = -Cb * ql, qlb = -Cb * gl;
  vnrb += Ab;
  vnlb += Cb;
  const T unb = Bb + Db, croeb = Bb - Db;
  // Roe sound speed croe = sqrt(a2), a2 = (gamma - 1)(hroe - |u|^2 / 2)
  const T a2b = (a2pos && croe > T(0)) ? croeb * (T(0.5) * rcp(croe)) : T(0);
  const T hroeb = a2b * P.gm1;
  const T usqb = T(-0.5) * P.gm1 * a2b;
  gbar += (double)a2b * (double)fma(T(-0.5), usq, hroe);
  T ub[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) ub[a] = T(2) * usqb * u[a];
  ub[IN - 1] += unb;
  T wslb = T(0), wsrb = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    wslb = fma(ub[a], wl[1 + a], wslb);
    wsrb = fma(ub[a], wr[1 + a], wsrb);
    wlb[1 + a] += ub[a] * wsl;
    wrb[1 + a] += ub[a] * wsr;
  }
  // hroe = (hl ql + hr qr) isum, wsl = sl isum, wsr = sr isum
  const T tb = hroeb * isum;
  const T isumb = fma(hroeb, t, fma(wslb, sl, wsrb * sr));
  hlb = fma(tb, ql, hlb);
  hrb = fma(tb, qr, hrb);
  qlb = fma(tb, hl, qlb);
  qrb = fma(tb, hr, qrb);
  T slb = wslb * isum, srb = wsrb * isum;
  {
    const T sb = -isum * isum * isumb;  // isum = 1/(sl + sr)
    slb += sb;
    srb += sb;
  }
  rlb = fma(slb, ql, rlb);
  qlb = fma(slb, rl, qlb);
  rrb = fma(srb, qr, rrb);
  qrb = fma(srb, rr, qrb);
  // g = sqrt(gamma p)
  const T xlb = gl > T(0) ? glb * (T(0.5) * rcp(gl)) : T(0);
  const T xrb = gr > T(0) ? grb * (T(0.5) * rcp(gr)) : T(0);
  plb = fma(xlb, P.gamma, plb);
  prb = fma(xrb, P.gamma, prb);
  gbar += (double)xlb * (double)pl + (double)xrb * (double)pr;
  // q = rho^(-1/2)
  rlb = fma(qlb, T(-0.5) * ql * ql * ql, rlb);
  rrb = fma(qrb, T(-0.5) * qr * qr * qr, rrb);
  // rho h = p / (gamma - 1) + rho |v|^2 / 2 + p
  plb = fma(hlb, P.igm1 + T(1), plb);
  prb = fma(hrb, P.igm1 + T(1), prb);
  rlb = fma(hlb, T(0.5) * kl, rlb);
  rrb = fma(hrb, T(0.5) * kr, rrb);
  gbar -= ((double)hlb * (double)pl + (double)hrb * (double)pr) * (double)(P.igm1 * P.igm1);
  const T klb = hlb * (T(0.5) * rl), krb = hrb * (T(0.5) * rr);
#pragma unroll
  for (int a = 1; a <= 3; ++a) {
    wlb[a] = fma(T(2) * klb, wl[a], wlb[a]);
    wrb[a] = fma(T(2) * krb, wr[a], wrb[a]);
  }
  wlb[IN] += vnlb;
  wrb[IN] += vnrb;
  wlb[0] += rlb;
  wrb[0] += rrb;
  wlb[4] += plb;
  wrb[4] += prb;
}

// ---------------------------------------------------------------------------
// kernels (uniform mesh, padded layout [leaf][v][k][j][i])
// ---------------------------------------------------------------------------

struct AdjGeom {
  int nx[3], S[3];
  int nleaf;
  double idx[3];
};

__device__ __forceinline__ size_t cell_index(const AdjGeom& g, int k, int j, int i) {
  return ((size_t)k * g.S[1] + j) * g.S[0] + i;
}

template <class T>
__device__ __forceinline__ void load_u(const T* Ub, size_t vs, size_t c, T u[NV]) {
#pragma unroll
  for (int v = 0; v < NV; ++v) u[v] = Ub[v * vs + c];
}

__device__ __forceinline__ void block_sum_add(double v, double* dst) {
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) s += red[w];
    if (s != 0.0) atomicAdd(dst, s);
  }
}

// Faces along DIR: one thread per face (f in 0..n_d, other axes interior).
// Writes the adjoints of the face's left and right primitive states at the
// padded index of the right cell.
template <class T, int DIR>
__global__ void adj_faces_kernel(const T* __restrict__ Wp, const T* __restrict__ H, const T* __restrict__ mu,
                                 T* FLb, T* FRb, AdjGeom g, Phys<T> P, double* gbar_out) {
  constexpr int t1 = (DIR + 1) % 3, t2 = (DIR + 2) % 3;
  const size_t per_leaf = (size_t)(g.nx[DIR] + 1) * g.nx[t1] * g.nx[t2];
  const size_t vs = (size_t)g.S[0] * g.S[1] * g.S[2];
  double gbar = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < per_leaf * g.nleaf;
       e += (size_t)gridDim.x * blockDim.x) {
    const int leaf = (int)(e / per_leaf);
    size_t r = e - (size_t)leaf * per_leaf;
    // face box: n_d + 1 faces along DIR, interior cells along the others, x1 fastest
    int dims[3] = {g.nx[0], g.nx[1], g.nx[2]};
    dims[DIR] += 1;
    int bx[3];
    bx[0] = (int)(r % dims[0]);
    r /= dims[0];
    bx[1] = (int)(r % dims[1]);
    bx[2] = (int)(r / dims[1]);
    const int f = bx[DIR];
    int pos[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) pos[d] = (d == DIR) ? f : bx[d] + NG;  // along DIR: padded start of the stencil
    const T* Wb = Wp + (size_t)leaf * NV * vs;
    const T* mub = mu + (size_t)leaf * NV * vs;
    size_t c[4];
    for (int s = 0; s < 4; ++s) {
      int q[3] = {pos[0], pos[1], pos[2]};
      q[DIR] = f + s;
      c[s] = cell_index(g, q[2], q[1], q[0]);
    }
    // c[1] = left cell a, c[2] = right cell b
    T fb[NV];
    bool any = false;
    const T idx = (T)g.idx[DIR];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      fb[v] = (mub[v * vs + c[2]] - mub[v * vs + c[1]]) * idx;
      any |= fb[v] != T(0);
    }
    T wlb[NV] = {0, 0, 0, 0, 0}, wrb[NV] = {0, 0, 0, 0, 0};
    if (any) {
      // face states from the cells' half-slopes along DIR (adj_hslope_kernel)
      const T* Hb = H + (size_t)leaf * NV * vs;
      T wl[NV], wr[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        wl[v] = Wb[v * vs + c[1]] + Hb[v * vs + c[1]];
        wr[v] = Wb[v * vs + c[2]] - Hb[v * vs + c[2]];
      }
      hlle_rev<T, DIR>(wl, wr, P, fb, wlb, wrb, gbar);
    }
    T* FLo = FLb + (size_t)leaf * NV * vs;
    T* FRo = FRb + (size_t)leaf * NV * vs;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      FLo[v * vs + c[2]] = wlb[v];
      FRo[v * vs + c[2]] = wrb[v];
    }
  }
  block_sum_add(gbar, gbar_out);
}

// Cells along DIR (padded 0..S-1, other axes interior).  Face k+1/2 lives at
// padded index k+1 when 2 <= k+1 <= n+2.  Two kernels per direction:
//   adj_slope: for every cell k with both neighbours (1 <= k <= S-2), the
//     adjoint of its half-slope, hb = FL(face k+1/2) - FR(face k-1/2), times
//     the slope's partial derivatives: Gm = hb dh/dW_{k-1}, G0 = hb dh/dW_k,
//     Gp = hb dh/dW_{k+1} (zero elsewhere), each slope differentiated once;
//   adj_gather: Wbar_p += FL(face p+1/2) + FR(face p-1/2) + Gp_{p-1} + G0_p
//     + Gm_{p+1}, one writer per cell.
template <int DIR>
__device__ __forceinline__ void adj_line_cell(const AdjGeom& g, size_t e, size_t per_leaf, int& leaf, int pos[3]) {
  leaf = (int)(e / per_leaf);
  size_t r = e - (size_t)leaf * per_leaf;
  int dims[3] = {g.nx[0], g.nx[1], g.nx[2]};
  dims[DIR] = g.S[DIR];
  int bx[3];
  bx[0] = (int)(r % dims[0]);
  r /= dims[0];
  bx[1] = (int)(r % dims[1]);
  bx[2] = (int)(r / dims[1]);
#pragma unroll
  for (int d = 0; d < 3; ++d) pos[d] = (d == DIR) ? bx[d] : bx[d] + NG;
}

template <int DIR>
__device__ __forceinline__ size_t adj_at(const AdjGeom& g, const int pos[3], int q) {
  int qq[3] = {pos[0], pos[1], pos[2]};
  qq[DIR] = q;
  return cell_index(g, qq[2], qq[1], qq[0]);
}

template <class T, int DIR>
__global__ void adj_slope_kernel(const T* __restrict__ Wp, const T* __restrict__ FLb,
                                 const T* __restrict__ FRb, T* __restrict__ Gm, T* __restrict__ G0,
                                 T* __restrict__ Gp, AdjGeom g) {
  constexpr int t1 = (DIR + 1) % 3, t2 = (DIR + 2) % 3;
  const int Sd = g.S[DIR], n = g.nx[DIR];
  const size_t per_leaf = (size_t)Sd * g.nx[t1] * g.nx[t2];
  const size_t vs = (size_t)g.S[0] * g.S[1] * g.S[2];
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < per_leaf * g.nleaf;
       e += (size_t)gridDim.x * blockDim.x) {
    int leaf, pos[3];
    adj_line_cell<DIR>(g, e, per_leaf, leaf, pos);
    const int k = pos[DIR];
    const size_t lo = (size_t)leaf * NV * vs;
    const size_t ck = adj_at<DIR>(g, pos, k);
    T hb[NV] = {0, 0, 0, 0, 0};
    bool nz = false;
    if (k >= 1 && k <= Sd - 2) {
      const bool up = k + 1 >= NG && k + 1 <= n + NG, dn = k >= NG && k <= n + NG;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        hb[v] = (up ? FLb[lo + v * vs + adj_at<DIR>(g, pos, k + 1)] : T(0)) - (dn ? FRb[lo + v * vs + ck] : T(0));
        nz |= hb[v] != T(0);
      }
    }
    T m[NV] = {0, 0, 0, 0, 0}, z[NV] = {0, 0, 0, 0, 0}, q[NV] = {0, 0, 0, 0, 0};
    if (nz) {
      T wa[NV], wb[NV], wc[NV];
      load_u(Wp + lo, vs, adj_at<DIR>(g, pos, k - 1), wa);
      load_u(Wp + lo, vs, ck, wb);
      load_u(Wp + lo, vs, adj_at<DIR>(g, pos, k + 1), wc);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        T dm, d0, dp;
        vl_half_d(wa[v], wb[v], wc[v], dm, d0, dp);
        m[v] = hb[v] * dm;
        z[v] = hb[v] * d0;
        q[v] = hb[v] * dp;
      }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      Gm[lo + v * vs + ck] = m[v];
      G0[lo + v * vs + ck] = z[v];
      Gp[lo + v * vs + ck] = q[v];
    }
  }
}

template <class T, int DIR>
__global__ void adj_gather_kernel(const T* __restrict__ FLb, const T* __restrict__ FRb,
                                  const T* __restrict__ Gm, const T* __restrict__ G0,
                                  const T* __restrict__ Gp, T* Wbar, AdjGeom g) {
  constexpr int t1 = (DIR + 1) % 3, t2 = (DIR + 2) % 3;
  const int Sd = g.S[DIR], n = g.nx[DIR];
  const size_t per_leaf = (size_t)Sd * g.nx[t1] * g.nx[t2];
  const size_t vs = (size_t)g.S[0] * g.S[1] * g.S[2];
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < per_leaf * g.nleaf;
       e += (size_t)gridDim.x * blockDim.x) {
    int leaf, pos[3];
    adj_line_cell<DIR>(g, e, per_leaf, leaf, pos);
    const int p = pos[DIR];
    const size_t lo = (size_t)leaf * NV * vs;
    const size_t cp = adj_at<DIR>(g, pos, p);
    const bool up = p + 1 >= NG && p + 1 <= n + NG, dn = p >= NG && p <= n + NG;
    const size_t cu = adj_at<DIR>(g, pos, p + 1 < Sd ? p + 1 : p);  // read only if p + 1 < S
    const size_t cd = adj_at<DIR>(g, pos, p >= 1 ? p - 1 : p);       // read only if p >= 1
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const size_t o = lo + v * vs;
      T acc = T(0);
      if (up) acc += FLb[o + cu];  // left state of face p+1/2
      if (dn) acc += FRb[o + cp];  // right state of face p-1/2
      if (p >= 1) acc += Gp[o + cd];
      acc += G0[o + cp];
      if (p + 1 < Sd) acc += Gm[o + cu];
      Wbar[o + cp] += acc;
    }
  }
}

// FP32: the same gather in one kernel, each thread differentiating the three
// half-slopes its cell enters (FP32 arithmetic is cheap here; one launch and
// no intermediate arrays are not): the sum of the same terms in the same
// order as adj_slope + adj_gather.
template <class T, int DIR>
__global__ void adj_cells_kernel(const T* __restrict__ Wp, const T* __restrict__ FLb,
                                 const T* __restrict__ FRb, T* Wbar, AdjGeom g) {
  constexpr int t1 = (DIR + 1) % 3, t2 = (DIR + 2) % 3;
  const int Sd = g.S[DIR], n = g.nx[DIR];
  const size_t per_leaf = (size_t)Sd * g.nx[t1] * g.nx[t2];
  const size_t vs = (size_t)g.S[0] * g.S[1] * g.S[2];
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < per_leaf * g.nleaf;
       e += (size_t)gridDim.x * blockDim.x) {
    const int leaf = (int)(e / per_leaf);
    size_t r = e - (size_t)leaf * per_leaf;
    // cell box: the S_d padded cells along DIR, interior cells along the others
    int dims[3] = {g.nx[0], g.nx[1], g.nx[2]};
    dims[DIR] = Sd;
    int bx[3];
    bx[0] = (int)(r % dims[0]);
    r /= dims[0];
    bx[1] = (int)(r % dims[1]);
    bx[2] = (int)(r / dims[1]);
    const int p = bx[DIR];
    int pos[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) pos[d] = (d == DIR) ? p : bx[d] + NG;
    auto at = [&](int q) {
      int qq[3] = {pos[0], pos[1], pos[2]};
      qq[DIR] = q;
      return cell_index(g, qq[2], qq[1], qq[0]);
    };
    const T* Wsrc = Wp + (size_t)leaf * NV * vs;
    const T* FL = FLb + (size_t)leaf * NV * vs;
    const T* FR = FRb + (size_t)leaf * NV * vs;
    auto face_ok = [&](int q) { return q >= NG && q <= n + NG; };  // face stored at q
    // primitives of cells p-2 .. p+2 that exist
    T w[5][NV];
    for (int s = 0; s < 5; ++s) {
      const int q = p - 2 + s;
      if (q < 0 || q >= Sd) continue;
      load_u(Wsrc, vs, at(q), w[s]);
    }
    T acc[NV] = {0, 0, 0, 0, 0};
    // direct: left state of face p+1/2, right state of face p-1/2
    if (face_ok(p + 1))
      for (int v = 0; v < NV; ++v) acc[v] += FL[v * vs + at(p + 1)];
    if (face_ok(p))
      for (int v = 0; v < NV; ++v) acc[v] += FR[v * vs + at(p)];
    // slopes of cells k = p-1, p, p+1 (each needs k-1 and k+1 in range)
    for (int dk = -1; dk <= 1; ++dk) {
      const int k = p + dk;
      if (k < 1 || k > Sd - 2) continue;
      T hb[NV];
      bool nz = false;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        hb[v] = (face_ok(k + 1) ? FL[v * vs + at(k + 1)] : T(0)) - (face_ok(k) ? FR[v * vs + at(k)] : T(0));
        nz |= hb[v] != T(0);
      }
      if (!nz) continue;
      const int s = dk + 2;  // index of cell k in w[]
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        T dm, d0, dp;
        vl_half_d(w[s - 1][v], w[s][v], w[s + 1][v], dm, d0, dp);
        // cell p is k+1 (dk=-1), k (dk=0) or k-1 (dk=+1) relative to slope k
        acc[v] += hb[v] * (dk == -1 ? dp : (dk == 0 ? d0 : dm));
      }
    }
    T* Wb = Wbar + (size_t)leaf * NV * vs;
    const size_t cp = at(p);
#pragma unroll
    for (int v = 0; v < NV; ++v) Wb[v * vs + cp] += acc[v];
  }
}

// Primitive variables of every padded cell of a stage's input, once per
// stage: the face and cell kernels read them instead of converting their
// 4- and 5-cell stencils along each direction.
template <class T>
__global__ void adj_wprim_kernel(const T* __restrict__ U, T* __restrict__ Wp, AdjGeom g, Phys<T> P) {
  const size_t vs = (size_t)g.S[0] * g.S[1] * g.S[2];
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < vs * g.nleaf;
       e += (size_t)gridDim.x * blockDim.x) {
    const int leaf = (int)(e / vs);
    const size_t base = (size_t)leaf * NV * vs + (e - (size_t)leaf * vs);
    T u[NV], w[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) u[v] = U[base + v * vs];
    bool rf, pf;
    prim_fwd(u, P, w, rf, pf);
#pragma unroll
    for (int v = 0; v < NV; ++v) Wp[base + v * vs] = w[v];
  }
}

// Half van Leer slopes along DIR of the cells the face kernel reads: each
// cell's once per stage, where the face kernel would compute each twice (one
// per face of the cell).
template <class T, int DIR>
__global__ void adj_hslope_kernel(const T* __restrict__ Wp, T* __restrict__ H, AdjGeom g) {
  // the cells the face kernel reads: padded 1 .. S-2 along DIR, interior
  // along the other two axes
  constexpr int t1 = (DIR + 1) % 3, t2 = (DIR + 2) % 3;
  const size_t per_leaf = (size_t)g.S[DIR] * g.nx[t1] * g.nx[t2];
  const size_t vs = (size_t)g.S[0] * g.S[1] * g.S[2];
  const size_t stride = DIR == 0 ? 1 : (DIR == 1 ? (size_t)g.S[0] : (size_t)g.S[0] * g.S[1]);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < per_leaf * g.nleaf;
       e += (size_t)gridDim.x * blockDim.x) {
    int leaf, pos[3];
    adj_line_cell<DIR>(g, e, per_leaf, leaf, pos);
    const int q = pos[DIR];
    if (q < 1 || q > g.S[DIR] - 2) continue;
    const size_t base = (size_t)leaf * NV * vs + cell_index(g, pos[2], pos[1], pos[0]);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T dm, d0, dp;
      H[base + v * vs] = vl_half_d(Wp[base + v * vs - stride], Wp[base + v * vs], Wp[base + v * vs + stride], dm,
                                   d0, dp);
    }
  }
}

// W -> U for every padded cell: acc += J^T Wbar; Wbar cleared.
template <class T>
__global__ void adj_prim_kernel(const T* __restrict__ U, T* Wbar, T* acc, AdjGeom g, Phys<T> P,
                                double* gbar_out) {
  const size_t vs = (size_t)g.S[0] * g.S[1] * g.S[2];
  double gbar = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < vs * g.nleaf;
       e += (size_t)gridDim.x * blockDim.x) {
    const int leaf = (int)(e / vs);
    const size_t c = e - (size_t)leaf * vs;
    const size_t base = (size_t)leaf * NV * vs + c;
    T wb[NV];
    bool nz = false;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      wb[v] = Wbar[base + v * vs];
      nz |= wb[v] != T(0);
    }
    if (!nz) continue;
    T u[NV], ub[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) u[v] = U[base + v * vs];
    prim_rev(u, P, wb, ub, gbar);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      acc[base + v * vs] += ub[v];
      Wbar[base + v * vs] = T(0);
    }
  }
  block_sum_add(gbar, gbar_out);
}

// Transpose of the uniform ghost exchange: out = in on interior cells plus the
// adjoints of the face-ghost images in the neighbouring blocks; 0 on ghosts.
// ACC (after the reverse of stage 2): instead of storing the result s,
// acc += s and mu = dt s (the stage-1 seeds), 0 into mu on ghost cells.
template <class T, bool ACC = false>
__global__ void adj_ghost_t_kernel(const T* __restrict__ in, T* out, const int* __restrict__ nbr,
                                   AdjGeom g, T* acc = nullptr, T dt = T(0)) {
  const size_t vs = (size_t)g.S[0] * g.S[1] * g.S[2];
  const int n1 = g.nx[0], n2 = g.nx[1], n3 = g.nx[2];
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < vs * g.nleaf;
       e += (size_t)gridDim.x * blockDim.x) {
    const int leaf = (int)(e / vs);
    const size_t c = e - (size_t)leaf * vs;
    const int i = (int)(c % g.S[0]);
    const int j = (int)((c / g.S[0]) % g.S[1]);
    const int k = (int)(c / ((size_t)g.S[0] * g.S[1]));
    const bool interior = i >= NG && i < NG + n1 && j >= NG && j < NG + n2 && k >= NG && k < NG + n3;
    T* o = out + (size_t)leaf * NV * vs + c;
    if (!interior) {
#pragma unroll
      for (int v = 0; v < NV; ++v) o[v * vs] = T(0);  // ACC: mu
      continue;
    }
    const T* ib = in + (size_t)leaf * NV * vs + c;
    T s[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) s[v] = ib[v * vs];
    const int* nb = nbr + 27 * leaf;
    // (offset to the neighbour, index of the image cell there) per axis
    auto add = [&](int region, int ii, int jj, int kk) {
      const T* src = in + (size_t)nb[region] * NV * vs + ((size_t)kk * g.S[1] + jj) * g.S[0] + ii;
#pragma unroll
      for (int v = 0; v < NV; ++v) s[v] += src[v * vs];
    };
    // region index (oz+1)*9 + (oy+1)*3 + (ox+1)
    if (i < NG + 2) add(1 * 9 + 1 * 3 + 0, i + n1, j, k);            // -x neighbour's high ghosts
    if (i >= n1) add(1 * 9 + 1 * 3 + 2, i - n1, j, k);               // +x neighbour's low ghosts
    if (j < NG + 2) add(1 * 9 + 0 * 3 + 1, i, j + n2, k);
    if (j >= n2) add(1 * 9 + 2 * 3 + 1, i, j - n2, k);
    if (k < NG + 2) add(0 * 9 + 1 * 3 + 1, i, j, k + n3);
    if (k >= n3) add(2 * 9 + 1 * 3 + 1, i, j, k - n3);
    if (ACC) {
      T* a = acc + (size_t)leaf * NV * vs + c;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        a[v * vs] = a[v * vs] + s[v];
        o[v * vs] = dt * s[v];
      }
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) o[v * vs] = s[v];
    }
  }
}

// Stage-2 seeds of a reverse cycle from the state adjoint lam:
// acc0 = lam / 2, acc1 = lam / 2, mu = (dt / 2) lam.
template <class T>
__global__ void adj_seed_kernel(const T* __restrict__ lam, T* __restrict__ acc0, T* __restrict__ acc1,
                                T* __restrict__ mu, T hdt, size_t n) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const T l = lam[e];
    acc0[e] = T(0.5) * l;
    acc1[e] = T(0.5) * l;
    mu[e] = hdt * l;
  }
}

}  // namespace ph

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

namespace {

int afail(int code, const std::string& msg) {
  ph::set_error_message(msg.c_str());
  return code;
}
#define PA_CUDA(expr)                                                              \
  do {                                                                             \
    cudaError_t _e = (expr);                                                       \
    if (_e != cudaSuccess) return afail(PH_ERR_CUDA, std::string(#expr) + ": " +   \
                                                         cudaGetErrorString(_e)); \
  } while (0)

int grid_for(size_t n) {
  size_t g = (n + 255) / 256;
  return (int)std::min<size_t>(std::max<size_t>(g, 1), 152 * 16);
}

}  // namespace

namespace ph {


template <class T>
int vjp_L(const MeshAccess& A, const T* U, const T* mu, T* acc, T* FLb, T* FRb, T* Wbar, T* Wp,
          T* Gm, T* G0, T* Gp, T* H, double* gbar) {
  AdjGeom g;
  for (int d = 0; d < 3; ++d) {
    g.nx[d] = A.nx[d];
    g.S[d] = A.nx[d] + 2 * NG;
    g.idx[d] = A.idx[d];
  }
  g.nleaf = A.nleaf;
  Phys<T> P;
  P.gamma = (T)A.gamma;
  P.gm1 = (T)(A.gamma - 1.0);
  P.igm1 = (T)(1.0 / (A.gamma - 1.0));
  P.dfloor = (T)A.dfloor;
  P.pfloor = (T)A.pfloor;
  cudaStream_t s = A.stream;
  const size_t nfaces0 = (size_t)(A.nx[0] + 1) * A.nx[1] * A.nx[2] * A.nleaf;
  const size_t ncell = (size_t)(A.nx[0] + 4) * A.nx[1] * A.nx[2] * A.nleaf;
  const size_t all = A.block_elems / NV * A.nleaf;
  adj_wprim_kernel<T><<<grid_for(all), 256, 0, s>>>(U, Wp, g, P);
  // FP64 (bound by the FP64 pipe): every half-slope differentiated once
  // (adj_slope), then the gather; FP32: one fused gather (adj_cells)
  auto cells = [&](auto dir) {
    constexpr int D = decltype(dir)::value;
    if constexpr (sizeof(T) == 4) {
      adj_cells_kernel<T, D><<<grid_for(ncell), 256, 0, s>>>(Wp, FLb, FRb, Wbar, g);
    } else {
      adj_slope_kernel<T, D><<<grid_for(ncell), 256, 0, s>>>(Wp, FLb, FRb, Gm, G0, Gp, g);
      adj_gather_kernel<T, D><<<grid_for(ncell), 256, 0, s>>>(FLb, FRb, Gm, G0, Gp, Wbar, g);
    }
  };
  adj_hslope_kernel<T, 0><<<grid_for(ncell), 256, 0, s>>>(Wp, H, g);
  adj_faces_kernel<T, 0><<<grid_for(nfaces0), 256, 0, s>>>(Wp, H, mu, FLb, FRb, g, P, gbar);
  cells(std::integral_constant<int, 0>());
  adj_hslope_kernel<T, 1><<<grid_for(ncell), 256, 0, s>>>(Wp, H, g);
  adj_faces_kernel<T, 1><<<grid_for(nfaces0), 256, 0, s>>>(Wp, H, mu, FLb, FRb, g, P, gbar);
  cells(std::integral_constant<int, 1>());
  adj_hslope_kernel<T, 2><<<grid_for(ncell), 256, 0, s>>>(Wp, H, g);
  adj_faces_kernel<T, 2><<<grid_for(nfaces0), 256, 0, s>>>(Wp, H, mu, FLb, FRb, g, P, gbar);
  cells(std::integral_constant<int, 2>());
  adj_prim_kernel<T><<<grid_for(all), 256, 0, s>>>(U, Wbar, acc, g, P, gbar);
  PA_CUDA(cudaGetLastError());
  return PH_OK;
}

template <class T>
int adjoint_t(ph_mesh* m, const void* U0, int ncycles, int ckpt, const double* dts_in,
              const void* dLdU, void* dLdU0, double* dLdgamma, int on_device) {
  MeshAccess A;
  int rc = mesh_access(m, &A);
  if (rc) return rc;
  cudaStream_t s = A.stream;
  const size_t elems = A.block_elems * A.nleaf;  // padded state
  const size_t bytes = elems * sizeof(T);
  const int nseg = (ncycles + ckpt - 1) / ckpt;
  // workspaces come from the mesh's allocator (PyTorch's caching allocator
  // when installed), so repeated gradients do not enter cudaMalloc/cudaFree
  std::vector<void*> bufs;
  auto alloc = [&](size_t b) -> T* {
    void* p = mesh_alloc(m, b ? b : 16);
    bufs.push_back(p);
    return (T*)p;
  };
  // the reverse sweep runs on its own stream, so that the recomputation of
  // the segment before (on the mesh's stream) overlaps it
  cudaStream_t rs = nullptr;
  cudaEvent_t ev_init = nullptr, ev_rec[2] = {nullptr, nullptr}, ev_rev[2] = {nullptr, nullptr};
  auto cleanup = [&]() {
    cudaStreamSynchronize(s);
    if (rs) cudaStreamSynchronize(rs);
    for (void* p : bufs) mesh_free(m, p);
    for (cudaEvent_t e : {ev_init, ev_rec[0], ev_rec[1], ev_rev[0], ev_rev[1]})
      if (e) cudaEventDestroy(e);
    if (rs) cudaStreamDestroy(rs);
  };
  T* lam = alloc(bytes);
  T* acc0 = alloc(bytes);
  T* acc1 = alloc(bytes);
  T* mu = alloc(bytes);
  T* FLb = alloc(bytes);
  T* FRb = alloc(bytes);
  T* Wbar = alloc(bytes);
  T* ufinal = alloc(bytes);
  T* Wp = alloc(bytes);
  T* Gm = alloc(bytes);
  T* G0 = alloc(bytes);
  T* Gp = alloc(bytes);
  T* H = alloc(bytes);
  T* ck = alloc(bytes * nseg);
  // stage inputs of one segment (U^n, U^1 per cycle), two sets: the reverse
  // sweep reads one while the recomputation fills the other
  T* segs[2][2] = {{alloc(bytes * ckpt), alloc(bytes * ckpt)}, {alloc(bytes * ckpt), alloc(bytes * ckpt)}};
  double* gbar = (double*)alloc(sizeof(double) * 2);
  double* d_dts = (double*)alloc(sizeof(double) * ncycles);
  DevScalars* sc_final = (DevScalars*)alloc(sizeof(DevScalars));
  T* packed = alloc(sizeof(T) * (size_t)A.nleaf * NV * A.nx[0] * A.nx[1] * A.nx[2]);
  for (void* p : bufs)
    if (!p) {
      cleanup();
      return afail(PH_ERR_OOM, "device allocation failed (adjoint)");
    }
  if (bufs.size() != 22) {
    cleanup();
    return afail(PH_ERR_OOM, "device allocation failed (adjoint)");
  }
  const size_t count = (size_t)A.nleaf * NV * A.nx[0] * A.nx[1] * A.nx[2];
  {
    cudaError_t e = cudaStreamCreateWithFlags(&rs, cudaStreamNonBlocking);
    for (cudaEvent_t* ev : {&ev_init, &ev_rec[0], &ev_rec[1], &ev_rev[0], &ev_rev[1]})
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      cleanup();
      return afail(PH_ERR_CUDA, cudaGetErrorString(e));
    }
  }
  auto fail_clean = [&](int code) {
    cleanup();
    return code;
  };
  // ---- forward with checkpoints; the dt schedule (given, or recorded from
  // the CFL dts) lives in device memory, so no cycle waits for the host
  if ((rc = mesh_set_state(m, U0, on_device))) return fail_clean(rc);
  std::vector<double> dts(ncycles);
  if (dts_in) {
    for (int c = 0; c < ncycles; ++c) dts[c] = dts_in[c];
    PA_CUDA(cudaMemcpyAsync(d_dts, dts.data(), sizeof(double) * ncycles, cudaMemcpyHostToDevice, s));
  }
  // the last segment's stage inputs are kept as the forward pass makes them,
  // so the backward pass starts without recomputing it
  const int clast = (nseg - 1) * ckpt;
  for (int c = 0; c < ncycles; ++c) {
    if (c % ckpt == 0)
      PA_CUDA(cudaMemcpyAsync(ck + (size_t)(c / ckpt) * elems, A.U0, bytes, cudaMemcpyDeviceToDevice, s));
    T* const* last = segs[(nseg - 1) % 2];
    if (c >= clast)
      PA_CUDA(cudaMemcpyAsync(last[0] + (size_t)(c - clast) * elems, A.U0, bytes, cudaMemcpyDeviceToDevice, s));
    rc = dts_in ? mesh_cycle_device_dt(m, d_dts + c) : mesh_cycle_record_dt(m, d_dts + c);
    if (rc) return fail_clean(rc);
    if (c >= clast)
      PA_CUDA(cudaMemcpyAsync(last[1] + (size_t)(c - clast) * elems, A.U1, bytes, cudaMemcpyDeviceToDevice, s));
  }
  if (!dts_in) {
    PA_CUDA(cudaMemcpyAsync(dts.data(), d_dts, sizeof(double) * ncycles, cudaMemcpyDeviceToHost, s));
    PA_CUDA(cudaStreamSynchronize(s));
  }
  PA_CUDA(cudaMemcpyAsync(ufinal, A.U0, bytes, cudaMemcpyDeviceToDevice, s));
  // the recomputation below advances the mesh's clock again: keep the
  // forward run's time, cycle count and dts to restore at the end
  PA_CUDA(cudaMemcpyAsync(sc_final, A.sc, sizeof(DevScalars), cudaMemcpyDeviceToDevice, s));
  // ---- seed: dL/dU_final on interior cells, zero ghosts
  PA_CUDA(cudaMemsetAsync(lam, 0, bytes, s));
  if (on_device) {
    PA_CUDA(launch_pack<T>(lam, (T*)dLdU, A.nx, A.nleaf, 0, s));
  } else {
    PA_CUDA(cudaMemcpyAsync(packed, dLdU, count * sizeof(T), cudaMemcpyHostToDevice, s));
    PA_CUDA(launch_pack<T>(lam, packed, A.nx, A.nleaf, 0, s));
  }
  PA_CUDA(cudaMemsetAsync(gbar, 0, 2 * sizeof(double), s));
  PA_CUDA(cudaMemsetAsync(FLb, 0, bytes, s));
  PA_CUDA(cudaMemsetAsync(FRb, 0, bytes, s));
  PA_CUDA(cudaMemsetAsync(Wbar, 0, bytes, s));
  const int gE = grid_for(elems);
  AdjGeom g;
  for (int d = 0; d < 3; ++d) {
    g.nx[d] = A.nx[d];
    g.S[d] = A.nx[d] + 2 * NG;
    g.idx[d] = A.idx[d];
  }
  g.nleaf = A.nleaf;
  // ---- backward, segment by segment: the reverse sweep of segment sg (on
  // rs) overlaps the recomputation of segment sg - 1 (on the mesh's stream)
  // into the other set of stage inputs
  PA_CUDA(cudaEventRecord(ev_init, s));  // seeds, the last segment's inputs, checkpoints
  PA_CUDA(cudaStreamWaitEvent(rs, ev_init, 0));
  MeshAccess AR = A;
  AR.stream = rs;
  auto recompute = [&](int sgr) -> int {
    const int r0 = sgr * ckpt, r1 = std::min(r0 + ckpt, ncycles);
    T* const* set = segs[sgr % 2];
    // the set's last reader is the reverse sweep of segment sgr + 2
    if (sgr + 2 <= nseg - 1) PA_CUDA(cudaStreamWaitEvent(s, ev_rev[sgr % 2], 0));
    PA_CUDA(cudaMemcpyAsync(A.U0, ck + (size_t)sgr * elems, bytes, cudaMemcpyDeviceToDevice, s));
    for (int c = r0; c < r1; ++c) {
      PA_CUDA(cudaMemcpyAsync(set[0] + (size_t)(c - r0) * elems, A.U0, bytes, cudaMemcpyDeviceToDevice, s));
      int rr = mesh_cycle_device_dt(m, d_dts + c);
      if (rr) return rr;
      PA_CUDA(cudaMemcpyAsync(set[1] + (size_t)(c - r0) * elems, A.U1, bytes, cudaMemcpyDeviceToDevice, s));
    }
    PA_CUDA(cudaEventRecord(ev_rec[sgr % 2], s));
    return PH_OK;
  };
  // (the last segment's inputs were kept by the forward pass: ev_init covers them)
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int c0 = sg * ckpt, c1 = std::min(c0 + ckpt, ncycles);
    if (sg >= 1 && (rc = recompute(sg - 1))) return fail_clean(rc);
    if (sg != nseg - 1) PA_CUDA(cudaStreamWaitEvent(rs, ev_rec[sg % 2], 0));
    T* const* set = segs[sg % 2];
    for (int c = c1 - 1; c >= c0; --c) {
      const T* Un = set[0] + (size_t)(c - c0) * elems;
      const T* U1n = set[1] + (size_t)(c - c0) * elems;
      const T dt = (T)dts[c];
      // stage 2: U = 1/2 U0 + 1/2 (U1 + dt L(U1))
      adj_seed_kernel<T><<<gE, 256, 0, rs>>>(lam, acc0, acc1, mu, T(0.5) * dt, elems);
      if ((rc = vjp_L<T>(AR, U1n, mu, acc1, FLb, FRb, Wbar, Wp, Gm, G0, Gp, H, gbar))) return fail_clean(rc);
      // stage 1: U1 = U0 + dt L(U0); its seeds acc0 += G^T acc1, mu = dt G^T acc1
      adj_ghost_t_kernel<T, true><<<gE, 256, 0, rs>>>(acc1, mu, A.nbr, g, acc0, dt);
      if ((rc = vjp_L<T>(AR, Un, mu, acc0, FLb, FRb, Wbar, Wp, Gm, G0, Gp, H, gbar))) return fail_clean(rc);
      adj_ghost_t_kernel<T><<<gE, 256, 0, rs>>>(acc0, lam, A.nbr, g);
      PA_CUDA(cudaGetLastError());
    }
    PA_CUDA(cudaEventRecord(ev_rev[sg % 2], rs));
  }
  // ---- outputs; leave the mesh at the final state of the forward run
  if (on_device) {
    PA_CUDA(launch_pack<T>(lam, (T*)dLdU0, A.nx, A.nleaf, 1, rs));
  } else {
    PA_CUDA(launch_pack<T>(lam, packed, A.nx, A.nleaf, 1, rs));
    PA_CUDA(cudaMemcpyAsync(dLdU0, packed, count * sizeof(T), cudaMemcpyDeviceToHost, rs));
  }
  double hg = 0.0;
  PA_CUDA(cudaMemcpyAsync(&hg, gbar, sizeof(double), cudaMemcpyDeviceToHost, rs));
  PA_CUDA(cudaStreamSynchronize(rs));
  PA_CUDA(cudaMemcpyAsync(A.U0, ufinal, bytes, cudaMemcpyDeviceToDevice, s));
  PA_CUDA(cudaMemcpyAsync(A.sc, sc_final, sizeof(DevScalars), cudaMemcpyDeviceToDevice, s));
  PA_CUDA(cudaStreamSynchronize(s));
  if (dLdgamma) *dLdgamma = hg;
  cleanup();
  return PH_OK;
}

}  // namespace ph

extern "C" int ph_adjoint(ph_mesh* m, const void* U0, int32_t ncycles, int32_t ckpt_every,
                          const double* dts, const void* dLdU, void* dLdU0, double* dLdgamma,
                          int32_t on_device) {
  PH_RANGE("ph_adjoint");
  if (!m || !U0 || !dLdU || !dLdU0 || ncycles < 1 || ckpt_every < 1)
    return afail(PH_ERR_INVALID, "ph_adjoint: bad argument");
  ph::MeshAccess A;
  int rc = ph::mesh_access(m, &A);
  if (rc) return rc;
  return A.precision == PH_FP32
             ? ph::adjoint_t<float>(m, U0, ncycles, ckpt_every, dts, dLdU, dLdU0, dLdgamma, on_device)
             : ph::adjoint_t<double>(m, U0, ncycles, ckpt_every, dts, dLdU, dLdU0, dLdgamma, on_device);
}
