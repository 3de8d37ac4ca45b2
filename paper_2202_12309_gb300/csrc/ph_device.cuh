// ph_device.cuh -- device-side building blocks shared by the library's kernels.
//
// Pointwise physics of the Parthenon-hydro method (arXiv:2202.12309 Sec. 4.1:
// ideal-gas Euler equations, piecewise-linear reconstruction, HLLE fluxes)
// written for throughput on sm_103a: one reciprocal square root gives both
// sqrt(rho) and 1/rho, Roe weights are formed once, and every division that
// shares a denominator is a multiplication by one reciprocal.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ph {

constexpr int NV = 5;   // conserved variables: rho, m1, m2, m3, E
constexpr int MAXS = 2; // passive scalars rho r_s stored after E (variables NV .. NV+MAXS-1)
constexpr int NG = 2;   // ghost width: PLM needs two cells on each side
constexpr int MAXLEV = 4;  // finest level a mesh tree may have

// Device-resident scalars of one mesh.  The cycle's dt never leaves the GPU.
struct DevScalars {
  double dt_next;               // dt the next cycle uses
  double dt_last;               // dt the last cycle used
  double time;
  long long cycle;
  unsigned long long wmax_bits; // max over cells of (|v_d| + c)/dx_d, as bits (>= 0)
  unsigned long long floor_hits;
  int nonfinite;                // a non-finite dt was produced
  int error;                    // bounded device wait gave up
  int tree_error;               // composite evaluation needed more nesting than supported
  int pad;
};

template <class T>
struct Phys {
  T gamma, gm1, igm1, dfloor, pfloor;
};

// Round-to-nearest add/mul that the compiler may not fuse into an FMA: used
// wherever results must be reproducible operation by operation
// (restriction, prolongation).
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }

// --------------------------------------------------------------------------
// Reciprocal, reciprocal square root and square root for the stage kernels.
// GB300 retires two FP64 FMAs per clock per SM, and a correctly rounded FP64
// division or square root costs about ten of them.  These routines start from
// the hardware's approximate value (PTX rcp.approx.ftz / rsqrt.approx.ftz, on
// the special-function unit) and take one higher-order Newton-Raphson
// (Householder) step in FP64:
//   reciprocal:  e = 1 - x y,   y' = y (1 + e + e^2)        error e^3
//   rsqrt:       e = 1 - x y^2, y' = y (1 + e/2 + 3e^2/8)   error 5e^3/16
//   sqrt:        s = x y, e = 1 - s y, s' = s (1 + e/2 + 3e^2/8)
// (the truncated binomial series of (1-e)^-1 and (1-e)^-1/2).  With the
// approximation good to ~2^-20 the truncation error is below 2^-56, so the
// reciprocal and rsqrt are within one ulp of the exact values and the
// square root within two (tested against them).  Arguments outside [2^-1000, 2^1000] in magnitude (zero,
// subnormals, infinities, NaN; negative ones for the roots) take the
// correctly rounded path instead.  FP32: the hardware approximations alone
// (rcp / rsqrt / sqrt .approx.ftz.f32, one special-function instruction
// each, within 2 ulp of the exact values: tested); the FP32 kernels call
// them on normal positive numbers well inside the float range (densities
// and pressures at or above their floors, sums of same-signed slopes), and
// sq(0) = 0.
// --------------------------------------------------------------------------
__device__ __forceinline__ bool nr_range(double x) {  // 2^-1000 <= |x| <= 2^1000
  const unsigned hi = (unsigned)__double2hiint(x) & 0x7fffffffu;
  return hi - (23u << 20) < (2001u << 20);
}
__device__ __forceinline__ bool nr_range_pos(double x) {  // 2^-1000 <= x <= 2^1000
  return (unsigned)__double2hiint(x) - (23u << 20) < (2001u << 20);
}
__device__ __forceinline__ double rcp_approx(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  return y;
}
__device__ __forceinline__ double rsqrt_approx(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  return y;
}
__device__ __forceinline__ double rcp(double x) {
  if (!nr_range(x)) return 1.0 / x;
  const double y = rcp_approx(x);
  const double e = fma(-x, y, 1.0);
  return fma(y, fma(e, e, e), y);
}
__device__ __forceinline__ float rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ double rsq(double x) {
  if (!nr_range_pos(x)) return rsqrt(x);
  const double y = rsqrt_approx(x);
  const double e = fma(-(x * y), y, 1.0);
  return fma(y * e, fma(0.375, e, 0.5), y);
}
__device__ __forceinline__ float rsq(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ double sq(double x) {
  if (!nr_range_pos(x)) return sqrt(x);
  const double y = rsqrt_approx(x);
  const double s = x * y;
  const double e = fma(-s, y, 1.0);
  return fma(s * e, fma(0.375, e, 0.5), s);
}
__device__ __forceinline__ float sq(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// HLLE wave-speed bounds max(0, a, b) and min(0, a, b).  For doubles with
// integer instructions: the bit patterns of non-negative doubles order like
// signed 64-bit integers and every negative double is below them, so the
// integer max of (0, a, b) is the numeric max(0, a, b) (a positive NaN
// propagates); min(0, a, b) = -max(0, -a, -b) with the sign bit flipped.
__device__ __forceinline__ double max0(double a, double b) {
  const long long m = max(__double_as_longlong(a), __double_as_longlong(b));
  return __longlong_as_double(max(m, 0ll));
}
// FP32: one three-input max / min (NaN inputs are skipped, as fmaxf does).
__device__ __forceinline__ float max0(float a, float b) {
  float y;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(y) : "f"(a), "f"(b), "f"(0.f));
  return y;
}
__device__ __forceinline__ double min0(double a, double b) {
  constexpr long long S = (long long)0x8000000000000000ull;
  const long long m = max(__double_as_longlong(a) ^ S, __double_as_longlong(b) ^ S);
  return __longlong_as_double(max(m, 0ll) ^ S);
}
__device__ __forceinline__ float min0(float a, float b) {
  float y;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(y) : "f"(a), "f"(b), "f"(0.f));
  return y;
}
// x > 0 (integer test for doubles; NaN with the sign bit clear counts as > 0).
__device__ __forceinline__ bool positive(double x) { return __double_as_longlong(x) > 0; }
__device__ __forceinline__ bool positive(float x) { return x > 0.f; }

// Branch tests on FP64 values done with integer instructions: on GB300 an
// FP64 compare occupies the FP64 pipe (1/64 of the FP32 rate), an integer
// compare the ALU pipe.
//   below_floor(x, f): x < f for a positive floor f (the bit patterns of
//     doubles order like signed integers for f > 0; NaN is never below).
//   same_sign_nonzero(a, b): a b > 0 (up to underflow of the product).
__device__ __forceinline__ bool below_floor(double x, double f) {
  return __double_as_longlong(x) < __double_as_longlong(f);
}
__device__ __forceinline__ bool below_floor(float x, float f) { return x < f; }
__device__ __forceinline__ bool same_sign_nonzero(double a, double b) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  return ((ia ^ ib) >= 0) && ((ia << 1) != 0) && ((ib << 1) != 0);
}
__device__ __forceinline__ bool same_sign_nonzero(float a, float b) { return a * b > 0.f; }
// |x| within [2^-150, 2^150] (so that a product of five such values is a
// normal number); integer test on the exponent field.
__device__ __forceinline__ bool mid_range(double x) {
  const int e = (__double2hiint(x) >> 20) & 0x7ff;
  return e >= 1023 - 150 && e <= 1023 + 150;
}
__device__ __forceinline__ bool mid_range(float x) {
  const int e = (__float_as_int(x) >> 23) & 0xff;
  return e >= 127 - 20 && e <= 127 + 20;
}

// Conserved -> primitive in place: (rho, m1, m2, m3, E) -> (rho, v1, v2, v3, p),
// with density and pressure floors (each application counted).
// Passive scalars (variables NV .. NVT-1) become concentrations r = (rho r) / rho.
template <class T, int NVT = NV>
__device__ __forceinline__ void cons_to_prim(T w[NVT], const Phys<T>& P, unsigned& floors) {
  T rho = w[0];
  if (below_floor(rho, P.dfloor)) { rho = P.dfloor; ++floors; }
  const T ir = rcp(rho);
  const T v1 = w[1] * ir, v2 = w[2] * ir, v3 = w[3] * ir;
  // explicit fmas in a fixed order (the paired FP32 conversion uses the
  // same), so that every kernel converts a state to the same bits
  const T ke = fma(w[3], v3, fma(w[2], v2, w[1] * v1));
  T p = P.gm1 * fma(T(-0.5), ke, w[4]);
  if (below_floor(p, P.pfloor)) { p = P.pfloor; ++floors; }
  w[0] = rho;
  w[1] = v1;
  w[2] = v2;
  w[3] = v3;
  w[4] = p;
#pragma unroll
  for (int v = NV; v < NVT; ++v) w[v] = w[v] * ir;
}

// Half van Leer slope of one passive-scalar concentration (one reciprocal)
// from its left and right differences.
template <class T>
__device__ __forceinline__ T vanleer_half_rcp_d(T dl, T dr) {
  const T prod = dl * dr;
  return same_sign_nonzero(dl, dr) ? prod * rcp(dl + dr) : T(0);
}
template <class T>
__device__ __forceinline__ T vanleer_half_rcp(T wm, T w0, T wp) {
  return vanleer_half_rcp_d(w0 - wm, wp - w0);
}

// Half of the van Leer (harmonic) limited slope of a cell from its two
// neighbours: dL dR / (dL + dR) where dL dR > 0, else 0.  The face states are
// w -+ this value (the factors 2 and 1/2 of the slope cancel exactly).
template <class T>
__device__ __forceinline__ T vanleer_half(T wm, T w0, T wp) {
  const T dl = w0 - wm, dr = wp - w0, prod = dl * dr;
  return prod > T(0) ? prod / (dl + dr) : T(0);
}

// The five half-slopes of one cell along one direction with one division:
// 1/(dL+dR) of every variable comes from the reciprocal of their product
// (Montgomery's simultaneous-inversion trick: prefix products, one
// reciprocal, then one multiply back per factor).  Variables with dL dR <= 0
// take the factor 1 and a zero slope.  If any factor is outside
// [2^-150, 2^150] the product could leave the normal range, and the slopes
// are divided one by one instead.  The reciprocals carry a few ulp of
// rounding more than separate divisions.
// (vanleer_half5_d takes the differences dL = w0 - wm, dR = wp - w0.)
template <class T>
__device__ __forceinline__ void vanleer_half5_d(const T dl[NV], const T dr[NV], T h[NV]) {
  if constexpr (sizeof(T) == 4) {
    // FP32: a reciprocal is one special-function op and two FMAs, cheaper
    // than the range checks of the batched form; one per variable.
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const T prod = dl[v] * dr[v];
      h[v] = prod > T(0) ? prod * rcp(dl[v] + dr[v]) : T(0);
    }
    return;
  }
  T s[NV];
  bool on[NV];
  bool ok = true, any = false;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    on[v] = same_sign_nonzero(dl[v], dr[v]);
    any = any || on[v];
    s[v] = on[v] ? dl[v] + dr[v] : T(1);
    ok = ok && mid_range(s[v]);
  }
  if (!any) {  // flat or extremal in every variable: no division at all
#pragma unroll
    for (int v = 0; v < NV; ++v) h[v] = T(0);
  } else if (ok) {
    T p[NV];
    p[0] = s[0];
#pragma unroll
    for (int v = 1; v < NV; ++v) p[v] = p[v - 1] * s[v];
    T inv = rcp(p[NV - 1]);
    T is[NV];
#pragma unroll
    for (int v = NV - 1; v > 0; --v) {
      is[v] = inv * p[v - 1];
      inv = inv * s[v];
    }
    is[0] = inv;
#pragma unroll
    for (int v = 0; v < NV; ++v) h[v] = on[v] ? (dl[v] * dr[v]) * is[v] : T(0);
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) h[v] = on[v] ? (dl[v] * dr[v]) / s[v] : T(0);
  }
}
template <class T>
__device__ __forceinline__ void vanleer_half5(const T wm[NV], const T w0[NV], const T wp[NV],
                                              T h[NV]) {
  T dl[NV], dr[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    dl[v] = w0[v] - wm[v];
    dr[v] = wp[v] - w0[v];
  }
  vanleer_half5_d(dl, dr, h);
}

// HLLE flux with Einfeldt's wave-speed bounds (Roe averages) through a face
// whose normal is x_{DIR+1}; wl/wr are primitive states.
//   F = (b+ F_L - b- F_R + b+ b- (U_R - U_L)) / (b+ - b-)
// is evaluated as F = cL F_L + cR F_R + cD (U_R - U_L) with cL = b+/(b+ - b-),
// cR = -b-/(b+ - b-), cD = b+ b-/(b+ - b-).  With alL = cL v_nL - cD and
// alR = cR v_nR + cD, every conserved density q carried with the flow has
// the flux alL q_L + alR q_R: the mass flux is aL + aR (aL = alL rho_L,
// aR = alR rho_R), the momentum flux aL v_L + aR v_R plus the pressure term
// on the normal component, and since E = rho h - p the energy flux is
// alL (rho h)_L + alR (rho h)_R - cD (p_R - p_L).  Roe averages use
// sqrt(rho) v and h sqrt(rho) = (rho h)/sqrt(rho).
template <class T, int DIR, int NVT = NV>
__device__ __forceinline__ void hlle(const T wl[NVT], const T wr[NVT], const Phys<T>& P, T f[NVT]) {
  // Every multiply-add is an explicit fma, so that the rounding is the same
  // in every kernel this is inlined into (the single-mesh and the batched
  // kernels agree bit for bit).  Sums over the velocity components run in
  // the cyclic order (normal, next, next but one), so that the flux of a
  // state whose components were rotated to put the normal first is the same
  // to the last bit.
  constexpr int IN = 1 + DIR;
  constexpr int IB = 1 + (DIR + 1) % 3, IC = 1 + (DIR + 2) % 3;
  const T rl = wl[0], pl = wl[4], rr = wr[0], pr = wr[4];
  const T vnl = wl[IN], vnr = wr[IN];
  const T kl = fma(wl[IN], wl[IN], fma(wl[IB], wl[IB], wl[IC] * wl[IC]));
  const T kr = fma(wr[IN], wr[IN], fma(wr[IB], wr[IB], wr[IC] * wr[IC]));
  // rho h = E + p = p / (gamma - 1) + rho |v|^2 / 2 + p
  const T hl = fma(pl, P.igm1, fma(T(0.5) * rl, kl, pl));
  const T hr = fma(pr, P.igm1, fma(T(0.5) * rr, kr, pr));
  const T ql = rsq(rl), qr = rsq(rr);            // 1/sqrt(rho)
  const T sl = rl * ql, sr = rr * qr;            // sqrt(rho)
  const T gl = sq(P.gamma * pl), gr = sq(P.gamma * pr);  // c = g / sqrt(rho)
  const T isum = rcp(add_rn(sl, sr));
  const T wsl = sl * isum, wsr = sr * isum;      // Roe weights
  const T un = fma(wsl, wl[IN], wsr * wr[IN]);  // Roe velocity, normal first
  const T ub = fma(wsl, wl[IB], wsr * wr[IB]);
  const T uc = fma(wsl, wl[IC], wsr * wr[IC]);
  const T hroe = fma(hl, ql, hr * qr) * isum;
  const T a2 = P.gm1 * fma(T(-0.5), fma(un, un, fma(ub, ub, uc * uc)), hroe);
  const T croe = positive(a2) ? sq(a2) : T(0);
  const T bp = max0(fma(gr, qr, vnr), add_rn(un, croe));
  const T bm = min0(fma(-gl, ql, vnl), sub_rn(un, croe));
  const T idb = rcp(bp - bm);
  const T cL = bp * idb, cR = -bm * idb, cD = (bp * bm) * idb;
  const T alL = fma(cL, vnl, -cD), alR = fma(cR, vnr, cD);
  const T aL = alL * rl, aR = alR * rr;
  f[0] = aL + aR;
#pragma unroll
  for (int a = 1; a <= 3; ++a) f[a] = fma(aL, wl[a], aR * wr[a]);
  f[IN] += fma(cL, pl, cR * pr);
  f[4] = fma(alL, hl, fma(alR, hr, -cD * (pr - pl)));
  // passive scalars: mass flux split like a transverse velocity component
#pragma unroll
  for (int v = NV; v < NVT; ++v) f[v] = fma(aL, wl[v], aR * wr[v]);
}

// Max of two signal rates (non-negative numbers or NaN) on their bit
// patterns, unsigned: for non-negative numbers that is the numeric max, and
// a NaN of either sign lands above every number, so a NaN rate is never
// replaced by a later finite one (integer instructions, not FP64 compares).
__device__ __forceinline__ double rate_max(double a, double b) {
  const unsigned long long x = __double_as_longlong(a), y = __double_as_longlong(b);
  return __longlong_as_double((long long)(x > y ? x : y));
}
__device__ __forceinline__ float rate_max(float a, float b) {
  return __uint_as_float(max(__float_as_uint(a), __float_as_uint(b)));
}

// Largest signal speed over cell width of one primitive state:
// max_d (|v_d| + c) / dx_d.  dt = cfl / (max over cells).
template <class T>
__device__ __forceinline__ T wave_rate(const T w[NV], const Phys<T>& P, T idx1, T idx2, T idx3) {
  const T g = P.gamma * w[4];
  const T c = g * rsq(g * w[0]);   // sqrt(gamma p / rho)
  if constexpr (sizeof(T) == 8) {
    // Cubic cells (equal 1/dx_d, compared as bit patterns): rounding is
    // monotone, so max_d (|v_d| + c) / dx = (max_d |v_d| + c) / dx to the
    // last bit, and |v_d| (sign bit cleared) order like 64-bit integers (a
    // NaN above every number, so it still propagates): two FP64 adds and
    // multiplies fewer per cell.
    const long long e1 = __double_as_longlong(idx1);
    if (e1 == __double_as_longlong(idx2) && e1 == __double_as_longlong(idx3)) {
      constexpr long long MAG = 0x7fffffffffffffffll;
      const long long m = max(__double_as_longlong(w[1]) & MAG,
                              max(__double_as_longlong(w[2]) & MAG, __double_as_longlong(w[3]) & MAG));
      return add_rn(__longlong_as_double(m), c) * idx1;
    }
  }
  const T a = add_rn(fabs(w[1]), c) * idx1;
  const T b = add_rn(fabs(w[2]), c) * idx2;
  const T d = add_rn(fabs(w[3]), c) * idx3;
  return rate_max(a, rate_max(b, d));  // a NaN in any direction propagates
}

// Block-wide NaN-propagating max of a non-negative double, then one atomic
// max on its bit pattern (for non-negative doubles and NaN, the unsigned bit
// order is the numeric order, NaN above +inf).
__device__ __forceinline__ void block_max_to(unsigned long long* dst, double v, double* red) {
  unsigned long long bits = __double_as_longlong(v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long ob = __shfl_xor_sync(0xffffffffu, bits, o);
    bits = ob > bits ? ob : bits;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarp = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = __longlong_as_double(bits);
  __syncthreads();
  if (warp == 0) {
    unsigned long long b2 = lane < nwarp ? (unsigned long long)__double_as_longlong(red[lane]) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long ob = __shfl_xor_sync(0xffffffffu, b2, o);
      b2 = ob > b2 ? ob : b2;
    }
    if (lane == 0 && b2 != 0ull) atomicMax(dst, b2);
  }
}

// --------------------------------------------------------------------------
// Ghost-shell enumeration: the ghost cells of a padded block, flattened as
// (A) the 4 x3-ghost planes, (B) the 4 x2-ghost rows of each interior plane,
// (C) the 4 x1-ghost cells of each interior row.  Rows stay contiguous in x1.
// (Host and device: the host lists the cells a kernel will visit.)
// --------------------------------------------------------------------------
struct Shell {
  int n1, n2, n3, S1, S2, nA, nB, nC;
  __host__ __device__ __forceinline__ Shell(const int nx[3]) {
    n1 = nx[0]; n2 = nx[1]; n3 = nx[2];
    S1 = n1 + 2 * NG; S2 = n2 + 2 * NG;
    nA = 4 * S2 * S1;
    nB = n3 * 4 * S1;
    nC = n3 * n2 * 4;
  }
  __host__ __device__ __forceinline__ int count() const { return nA + nB + nC; }
  __host__ __device__ __forceinline__ void cell(int c, int& i, int& j, int& k) const {
    if (c < nA) {
      const int kk = c / (S2 * S1), r = c - kk * S2 * S1;
      j = r / S1;
      i = r - j * S1;
      k = kk < 2 ? kk : n3 + kk;
    } else if (c < nA + nB) {
      c -= nA;
      const int kq = c / (4 * S1), r = c - kq * 4 * S1;
      const int jj = r / S1;
      i = r - jj * S1;
      k = kq + NG;
      j = jj < 2 ? jj : n2 + jj;
    } else {
      c -= nA + nB;
      const int kq = c / (4 * n2), r = c - kq * 4 * n2;
      const int jq = r >> 2, ii = r & 3;
      k = kq + NG;
      j = jq + NG;
      i = ii < 2 ? ii : n1 + ii;
    }
  }
};

}  // namespace ph
