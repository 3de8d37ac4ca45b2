// ph_stage_pair.cuh -- the FP32 fused stage kernel with two x1-adjacent cells
// per thread.
//
// The FP32 stage is bound by instruction issue, not by HBM.  Blackwell issues
// FP32 add / multiply / fma on two lanes at once (PTX add/mul/fma .f32x2), and
// shared memory serves 8-byte accesses as cheaply as 4-byte ones.  Here every
// thread owns a pair of cells (i, i+1) of a 32 x 16 tile (256 threads) or of
// a 16 x 16 tile (128 threads, for blocks 16 cells wide), and
// slopes, face states, HLLE fluxes and the update are computed on both cells
// with one paired instruction where the method is the same on both lanes
// (compares, selects and the special-function approximations stay per lane).
// The method and the order of the tile march are those of ph_stage.cuh:
// TMA-staged planes of primitives in a 4-slot ring, x3 slopes and fluxes in
// registers, x1 / x2 slopes and fluxes in shared memory, SSPRK2 update and
// the signal-speed max for dt in the epilogue.  Uniform meshes only (no
// flux-correction capture).
#pragma once
#include "ph_stage.cuh"

namespace ph {

// Two FP32 lanes in one 64-bit register.
struct __align__(8) F2 {
  unsigned long long r;
};

__device__ __forceinline__ F2 f2(float a, float b) {
  F2 o;
  asm("mov.b64 %0, {%1, %2};" : "=l"(o.r) : "f"(a), "f"(b));
  return o;
}
__device__ __forceinline__ F2 f2(float a) { return f2(a, a); }
__device__ __forceinline__ void split(F2 x, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x.r));
}
__device__ __forceinline__ float lane0(F2 x) {
  float a, b;
  split(x, a, b);
  return a;
}
__device__ __forceinline__ float lane1(F2 x) {
  float a, b;
  split(x, a, b);
  return b;
}
__device__ __forceinline__ F2 operator+(F2 a, F2 b) {
  F2 o;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(o.r) : "l"(a.r), "l"(b.r));
  return o;
}
__device__ __forceinline__ F2 operator-(F2 a, F2 b) {
  F2 o;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(o.r) : "l"(a.r), "l"(b.r));
  return o;
}
__device__ __forceinline__ F2 operator*(F2 a, F2 b) {
  F2 o;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(o.r) : "l"(a.r), "l"(b.r));
  return o;
}
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) {
  F2 o;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(o.r) : "l"(a.r), "l"(b.r), "l"(c.r));
  return o;
}
__device__ __forceinline__ F2 operator-(F2 a) {  // flip both sign bits
  F2 o;
  o.r = a.r ^ 0x8000000080000000ull;
  return o;
}
// Per-lane helpers: the scalar FP32 routines of ph_device.cuh on each lane
// (the special-function unit has no paired form).
__device__ __forceinline__ F2 rcp2(F2 x) {
  float a, b;
  split(x, a, b);
  return f2(rcp(a), rcp(b));
}
__device__ __forceinline__ F2 rsq2(F2 x) {
  float a, b;
  split(x, a, b);
  return f2(rsq(a), rsq(b));
}
__device__ __forceinline__ F2 sq2(F2 x) {
  float a, b;
  split(x, a, b);
  return f2(sq(a), sq(b));
}
__device__ __forceinline__ F2 max0_2(F2 x, F2 y) {
  float a, b, c, d;
  split(x, a, b);
  split(y, c, d);
  return f2(max0(a, c), max0(b, d));
}
__device__ __forceinline__ F2 min0_2(F2 x, F2 y) {
  float a, b, c, d;
  split(x, a, b);
  split(y, c, d);
  return f2(min0(a, c), min0(b, d));
}
__device__ __forceinline__ F2 ld2(const float* p) { return *reinterpret_cast<const F2*>(p); }
// A pair from global memory the kernel never writes, through the read-only
// path, issued where it stands (the compiler may not sink it towards its use).
__device__ __forceinline__ F2 ldg2_now(const float* p) {
  F2 o;
  asm volatile("ld.global.nc.b64 %0, [%1];" : "=l"(o.r) : "l"(p));
  return o;
}
__device__ __forceinline__ void st2(float* p, F2 v) { *reinterpret_cast<F2*>(p) = v; }

// cons -> prim in place on both lanes, floors per lane (each counted).
__device__ __forceinline__ void cons_to_prim2(F2 w[NV], const Phys<float>& P, unsigned& floors) {
  float r0, r1;
  split(w[0], r0, r1);
  if (below_floor(r0, P.dfloor)) { r0 = P.dfloor; ++floors; }
  if (below_floor(r1, P.dfloor)) { r1 = P.dfloor; ++floors; }
  const F2 rho = f2(r0, r1);
  const F2 ir = rcp2(rho);
  const F2 v1 = w[1] * ir, v2 = w[2] * ir, v3 = w[3] * ir;
  const F2 ke = fma2(w[3], v3, fma2(w[2], v2, w[1] * v1));  // the order of cons_to_prim()
  F2 p = f2(P.gm1) * fma2(f2(-0.5f), ke, w[4]);
  float p0, p1;
  split(p, p0, p1);
  if (below_floor(p0, P.pfloor)) { p0 = P.pfloor; ++floors; }
  if (below_floor(p1, P.pfloor)) { p1 = P.pfloor; ++floors; }
  w[0] = rho;
  w[1] = v1;
  w[2] = v2;
  w[3] = v3;
  w[4] = f2(p0, p1);
}

// Signal rate max_d (|v_d| + c)/dx_d of a primitive state on both lanes
// (the arithmetic of wave_rate() in ph_device.cuh); the max over directions
// per lane on the bit patterns (rate_max: a NaN propagates).
__device__ __forceinline__ F2 abs2(F2 x) {
  F2 o;
  o.r = x.r & 0x7fffffff7fffffffull;
  return o;
}
__device__ __forceinline__ void wave_rate2(const F2 w[NV], const Phys<float>& P, float idx1, float idx2,
                                           float idx3, float& ra, float& rb) {
  const F2 g = f2(P.gamma) * w[4];
  const F2 c = g * rsq2(g * w[0]);
  const F2 a = (abs2(w[1]) + c) * f2(idx1);
  const F2 b = (abs2(w[2]) + c) * f2(idx2);
  const F2 d = (abs2(w[3]) + c) * f2(idx3);
  float a0, a1, b0, b1, d0, d1;
  split(a, a0, a1);
  split(b, b0, b1);
  split(d, d0, d1);
  ra = rate_max(a0, rate_max(b0, d0));
  rb = rate_max(a1, rate_max(b1, d1));
}

// Half van Leer slopes of the five variables on both lanes, from the
// differences dL = w0 - wm and dR = wp - w0 or from the three values.
__device__ __forceinline__ void vanleer_half5_2d(const F2 dl[NV], const F2 dr[NV], F2 h[NV]) {
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const F2 prod = dl[v] * dr[v];
    const F2 t = prod * rcp2(dl[v] + dr[v]);
    float p0, p1, t0, t1;
    split(prod, p0, p1);
    split(t, t0, t1);
    h[v] = f2(p0 > 0.f ? t0 : 0.f, p1 > 0.f ? t1 : 0.f);
  }
}
__device__ __forceinline__ void vanleer_half5_2(const F2 wm[NV], const F2 w0[NV], const F2 wp[NV],
                                                F2 h[NV]) {
  F2 dl[NV], dr[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    dl[v] = w0[v] - wm[v];
    dr[v] = wp[v] - w0[v];
  }
  vanleer_half5_2d(dl, dr, h);
}

// HLLE flux (Einfeldt bounds, Roe averages) on both lanes; the arithmetic of
// hlle() in ph_device.cuh, two lanes per instruction.
template <int DIR>
__device__ __forceinline__ void hlle2(const F2 wl[NV], const F2 wr[NV], const Phys<float>& P, F2 f[NV]) {
  constexpr int IN = 1 + DIR;
  const F2 rl = wl[0], pl = wl[4], rr = wr[0], pr = wr[4];
  const F2 vnl = wl[IN], vnr = wr[IN];
  const F2 half = f2(0.5f);
  const F2 kl = fma2(wl[1], wl[1], fma2(wl[2], wl[2], wl[3] * wl[3]));
  const F2 kr = fma2(wr[1], wr[1], fma2(wr[2], wr[2], wr[3] * wr[3]));
  const F2 hl = fma2(pl, f2(P.igm1), fma2(half * rl, kl, pl));  // rho h
  const F2 hr = fma2(pr, f2(P.igm1), fma2(half * rr, kr, pr));
  const F2 ql = rsq2(rl), qr = rsq2(rr);
  const F2 sl = rl * ql, sr = rr * qr;
  const F2 gam = f2(P.gamma);
  const F2 gl = sq2(gam * pl), gr = sq2(gam * pr);
  const F2 isum = rcp2(sl + sr);
  const F2 wsl = sl * isum, wsr = sr * isum;
  const F2 u1 = fma2(wsl, wl[1], wsr * wr[1]);
  const F2 u2 = fma2(wsl, wl[2], wsr * wr[2]);
  const F2 u3 = fma2(wsl, wl[3], wsr * wr[3]);
  const F2 hroe = fma2(hl, ql, hr * qr) * isum;
  const F2 a2 = f2(P.gm1) * fma2(f2(-0.5f), fma2(u1, u1, fma2(u2, u2, u3 * u3)), hroe);
  float a20, a21;
  split(a2, a20, a21);
  const F2 croe = f2(sq(fmaxf(a20, 0.f)), sq(fmaxf(a21, 0.f)));
  const F2 un = (IN == 1) ? u1 : ((IN == 2) ? u2 : u3);
  const F2 bp = max0_2(fma2(gr, qr, vnr), un + croe);
  const F2 bm = min0_2(fma2(-gl, ql, vnl), un - croe);
  const F2 idb = rcp2(bp - bm);
  const F2 cL = bp * idb, cR = (-bm) * idb, cD = (bp * bm) * idb;
  const F2 alL = fma2(cL, vnl, -cD), alR = fma2(cR, vnr, cD);
  const F2 aL = alL * rl, aR = alR * rr;
  f[0] = aL + aR;
#pragma unroll
  for (int a = 1; a <= 3; ++a) f[a] = fma2(aL, wl[a], aR * wr[a]);
  f[IN] = f[IN] + fma2(cL, pl, cR * pr);
  f[4] = fma2(alL, hl, fma2(alR, hr, -(cD * (pr - pl))));
}

// Shared-memory layout of the paired kernel for tiles TX_ x 16 (TX_ = 32 or
// 16: one thread per cell pair, 256 or 128 threads; floats, every section
// starting on an 8-byte boundary so that pairs load and store whole).
template <int TX_>
struct PairSmemT {
  static_assert(TX_ == 32 || TX_ == 16, "paired tiles are 32 or 16 cells wide");
  static constexpr int TX = TX_, TY = 16, NT = TX / 2 * TY;
  static constexpr int PR = TX / 2;                  // pairs per row
  static constexpr int MINB = TX == 32 ? 2 : 4;      // CTAs per SM (128 registers a thread)
  static constexpr int WX = TX + 4, WY = TY + 4;
  static constexpr int PLANE = NV * WX * WY;
  static constexpr int SLOT = (PLANE * 4 + 127) / 128 * 128 / 4;
  static constexpr unsigned PLANE_BYTES = PLANE * 4;
  static constexpr int FPX = TX + 2;                 // x1 face pitch (faces 0..TX, one spare)
  static constexpr int DXN = NV * TY * WX;           // x1 slopes, indexed by plane position
  static constexpr int DYN = NV * (TY + 2) * TX;     // x2 slopes, rows -1..TY
  static constexpr int FXN = NV * TY * FPX;          // x1 face fluxes
  static constexpr int FYN = NV * (TY + 1) * TX;     // x2 face fluxes
  static constexpr size_t body = 4 * (size_t)(4 * SLOT + DXN + DYN + FXN + FYN);
  static constexpr size_t red_off = (body + 15) / 16 * 16;
  static constexpr size_t bar_off = red_off + 32 * sizeof(double);
  static constexpr size_t bytes = bar_off + 4 * sizeof(uint64_t) + 128;
};
using PairSmem = PairSmemT<32>;
using PairSmem16 = PairSmemT<16>;

// One TX x 16 tile of one block for one stage (TMA staging); returns the
// tile's max signal rate when J.want_rate.  The cells of a tile and the
// arithmetic of every face and cell do not depend on TX: the 32- and
// 16-wide tiles give the same bits.
// STAGE (1 or 2) is a template argument: the two stages keep different
// values live across the plane (stage 2 also U0), and each gets its own
// register allocation.  parity_io (optional): the mbarrier phase bits,
// carried across calls by a CTA that runs several tiles on the same barriers.
// LEAN: the own pair's values are read from shared memory at every use and
// the x3 face comes first (fewer registers live across the plane step, for
// a kernel that holds more state besides); otherwise they are loaded once
// and kept in registers.  Both give the same bits.
template <int TXP, int STAGE, bool LEAN = false>
__device__ __forceinline__ double stage_tile_pair(const TileJob<float>& J, const Phys<float>& P,
                                                  unsigned char* smem_raw, unsigned& floors,
                                                  const CUtensorMap* tmap, int vz0, uint64_t* bars,
                                                  int* failed, unsigned* parity_io = nullptr) {
  using SM = PairSmemT<TXP>;
  constexpr int TX = SM::TX, TY = SM::TY, NT = SM::NT, WX = SM::WX, WY = SM::WY, FPX = SM::FPX;
  constexpr int PR = SM::PR;
  float* ring = reinterpret_cast<float*>(smem_raw);
  float* sdx = ring + 4 * SM::SLOT;
  float* sdy = sdx + SM::DXN;
  float* sfx = sdy + SM::DYN;
  float* sfy = sfx + SM::FXN;
  const int tid = threadIdx.x;
  // own cells (tx, tx+1) of row ty.  16-wide tiles: a half-warp's 16 threads
  // take rows r and r + 4 (not r and r + 1), 80 floats apart in the planes
  // and the x1 slopes (rows of 20): the two rows fall on disjoint banks.
  const int q = tid / PR;
  const int tx = 2 * (tid % PR), ty = TXP == 16 ? (((q & 1) << 2) | ((q >> 1) & 3) | (q & 8)) : q;
  // Work lists: every thread's main item in every list is its own pair;
  // the halo items of a list go to one warp (x1 slopes: warp 0, x2 slopes:
  // warp 1, x1 faces: warp 2, x2 faces: warp 3, conversion: the last
  // CEXTRA threads, 104 or 72), so index arithmetic is shifts of the thread
  // index.
  constexpr int CEXTRA = 4 * (WX / 2) + 2 * TY;
  static_assert(CEXTRA <= NT, "conversion halo fits one round");
  const int warp = tid >> 5, lane = tid & 31;
  const int S1 = J.S[0], S2 = J.S[1];
  const int i0 = J.i0, j0 = J.j0, k0 = J.k0, k1 = J.k1;
  const size_t vstride = (size_t)J.S[0] * J.S[1] * J.S[2];

  unsigned parity = parity_io ? *parity_io : 0u;
  auto issue = [&](int p) {
    if (tid == 0) {
      const int sl = (p + 4) & 3;
      mbar_expect_tx(bars + sl, SM::PLANE_BYTES);
      tma_load_4d(ring + sl * SM::SLOT, tmap, bars + sl, i0, j0, p + NG, vz0);
    }
  };
  auto convert = [&](int p) -> bool {
    const int sl = (p + 4) & 3;
    const bool ok = mbar_wait(bars + sl, (parity >> sl) & 1u, 1u << 22);
    parity ^= 1u << sl;
    float* dst = ring + sl * SM::SLOT;
    auto conv = [&](int r, int q) {
      F2 w[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) w[v] = ld2(dst + (v * WY + r) * WX + q);
      cons_to_prim2(w, P, floors);
#pragma unroll
      for (int v = 0; v < NV; ++v) st2(dst + (v * WY + r) * WX + q, w[v]);
    };
    conv(ty + 2, tx + 2);  // own pair
    if (tid >= NT - CEXTRA) {  // plane rows 0, 1, TY+2, TY+3 and the x1 halo columns
      const int e = tid - (NT - CEXTRA);
      if (e < 4 * (WX / 2)) {
        const int rr = e / (WX / 2);
        conv(rr < 2 ? rr : rr + TY, 2 * (e - rr * (WX / 2)));
      } else {
        const int t = e - 4 * (WX / 2);
        conv(2 + (t >> 1), (t & 1) ? WX - 2 : 0);
      }
    }
    return ok;
  };
  auto check_failed = [&](bool ok) -> bool {
    if (!ok) atomicExch(failed, 1);
    __syncthreads();
    return *(volatile int*)failed != 0;
  };
  auto col = [&](int p, F2 w[NV]) {
    const float* s = ring + ((p + 4) & 3) * SM::SLOT;
#pragma unroll
    for (int v = 0; v < NV; ++v) w[v] = ld2(s + (v * WY + ty + 2) * WX + tx + 2);
  };

  // priming: planes k0-2 .. k0+1, the x3 slope at k0 and the flux below it
  for (int p = k0 - 2; p <= k0 + 1; ++p) issue(p);
  {
    bool ok = true;
    for (int p = k0 - 2; p <= k0 + 1; ++p) ok = convert(p) && ok;
    fence_proxy_async_smem();
    if (check_failed(ok)) return 0.0;
  }
  F2 dz[NV], dzr[NV], fzm[NV];  // dzr: the difference to the plane above (next left difference)
  {
    F2 wa[NV], wb[NV], wc[NV], wd[NV], wl[NV], wr[NV], d0[NV];
    col(k0 - 2, wa);
    col(k0 - 1, wb);
    col(k0, wc);
    col(k0 + 1, wd);
    vanleer_half5_2(wa, wb, wc, d0);
    vanleer_half5_2(wb, wc, wd, dz);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      wl[v] = wb[v] + d0[v];
      wr[v] = wc[v] - dz[v];
      dzr[v] = wd[v] - wc[v];
    }
    hlle2<2>(wl, wr, P, fzm);
  }
  __syncthreads();
  issue(k0 + 2);
  {
    const bool ok = convert(k0 + 2);
    fence_proxy_async_smem();
    if (check_failed(ok)) return 0.0;
  }
  if (k0 + 3 <= k1 + 1) issue(k0 + 3);

  const int i = i0 + tx, j = j0 + ty;
  const F2 tdt = f2(J.dt);
  float rate = 0.f;  // running max in FP32 (widened once at the end: the same value)
  const F2 idx1 = f2(J.idx1), idx2 = f2(J.idx2), idx3 = f2(J.idx3);

  for (int k = k0; k < k1; ++k) {
    // stage 2 reads U0 at plane k+1 in the next step's (G): bring its rows
    // into L2 now (the last 80 threads, one row of TX + 4 cells each)
    if (STAGE == 2 && k + 1 < k1 && tid >= NT - NV * TY) {
      const int r = tid - (NT - NV * TY), v = r / TY, row = r - v * TY;
      prefetch_l2(J.U0b + v * vstride + ((size_t)(k + 1 + NG) * S2 + (j0 + row + NG)) * S1 + i0,
                  (TX + 4) * 4);
    }
    // the own pair's current state (stage 2 also U0), loaded now so that the
    // loads complete while the plane's slopes and fluxes are computed.  Stage
    // 1 reads U0 and writes U1 only, so its loads take the read-only path and
    // stay here; stage 2 writes the U0 it reads, and leaving the compiler
    // free to place its loads measured faster (0.645 against 0.655 ms on the
    // 256^3 wave, where stage 1 gains 0.562 -> 0.534 ms).
    const size_t cell = (size_t)(k + NG) * S2 * S1 + (size_t)(j + NG) * S1 + (i + NG);
    F2 ucur[NV], u0[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) ucur[v] = STAGE == 1 ? ldg2_now(J.Ub + cell + v * vstride) : ld2(J.Ub + cell + v * vstride);
    if (STAGE == 2) {
#pragma unroll
      for (int v = 0; v < NV; ++v) u0[v] = ld2(J.U0b + cell + v * vstride);
    }
    // the own pair's primitives at plane k, loaded once: both slopes, both
    // faces and the x3 face take them from registers (own = nullptr: LEAN)
    F2 fzlo[NV], wk[NV];
    if constexpr (!LEAN) col(k, wk);
    const F2* own = LEAN ? nullptr : wk;
    // (C1) own x3 slope and flux: first in LEAN mode, else after the x1 / x2
    // faces (the flux below, fzlo, then is not live across them)
    auto x3_face = [&]() {
      F2 wb[NV], wc[NV], wl[NV], wr[NV], d1[NV], dr[NV], f[NV];
      col(k + 1, wb);
      col(k + 2, wc);
#pragma unroll
      for (int v = 0; v < NV; ++v) dr[v] = wc[v] - wb[v];
      vanleer_half5_2d(dzr, dr, d1);
      if constexpr (LEAN) col(k, wl);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        wl[v] = (LEAN ? wl[v] : wk[v]) + dz[v];
        wr[v] = wb[v] - d1[v];
        dz[v] = d1[v];
        dzr[v] = dr[v];
      }
      hlle2<2>(wl, wr, P, f);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        fzlo[v] = fzm[v];
        fzm[v] = f[v];
      }
    };
    if constexpr (LEAN) x3_face();
    const float* W = ring + ((k + 4) & 3) * SM::SLOT;
    // (C2) x1 slopes at plane positions (q, q+1): own pair q = tx + 2 (its
    // values from wk; its left neighbours kept in lo_own for the x1 faces);
    // the halo pairs q = 0 and WX-2 of each row (their outermost lanes read
    // clamped neighbours and are never used)
    float lo_own[NV];
    auto x1_slope = [&](int jj, int q, bool edge, const F2* own) {
      F2 a[NV], b[NV], r[NV], h[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const float* row = W + (v * WY + jj + 2) * WX;
        b[v] = own ? own[v] : ld2(row + q);
        const float lo = edge ? row[q > 0 ? q - 1 : 0] : row[q - 1];
        const float hi = edge ? row[q + 2 < WX ? q + 2 : WX - 1] : row[q + 2];
        if (own) lo_own[v] = lo;
        a[v] = f2(lo, lane0(b[v]));
        r[v] = f2(lane1(b[v]), hi);
      }
      vanleer_half5_2(a, b, r, h);
#pragma unroll
      for (int v = 0; v < NV; ++v) st2(sdx + (v * TY + jj) * WX + q, h[v]);
    };
    // (C3) x2 slopes of rows jj - 1 (jj = 0 .. TY + 1), column pair q; the
    // own pair's (own = wk) also kept in hy_own for its x2 face
    F2 hy_own[NV];
    auto x2_slope = [&](int jj, int q, const F2* own) {
      F2 a[NV], b[NV], r[NV], h[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const float* p = W + (v * WY + jj) * WX + q + 2;
        a[v] = ld2(p);
        b[v] = own ? own[v] : ld2(p + WX);
        r[v] = ld2(p + 2 * WX);
      }
      vanleer_half5_2(a, b, r, h);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        if (own) hy_own[v] = h[v];
        st2(sdy + (v * (TY + 2) + jj) * TX + q, h[v]);
      }
    };
    x1_slope(ty, tx + 2, false, own);
    x2_slope(ty + 1, tx, own);
    if (warp == 0) x1_slope(lane >> 1, (lane & 1) ? WX - 2 : 0, true, nullptr);
    if (warp == 1 && lane < 2 * PR) x2_slope(lane >= PR ? TY + 1 : 0, 2 * (lane % PR), nullptr);
    __syncthreads();
    // (E1) x1 face pairs (f, f+1), f even; face f joins cells f-1 and f
    auto x1_face = [&](int jj, int f, const F2* own) {
      F2 wl[NV], wr[NV], fl[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const float* row = W + (v * WY + jj + 2) * WX;
        const float* srow = sdx + (v * TY + jj) * WX;
        const F2 R = own ? own[v] : ld2(row + f + 2), SR = ld2(srow + f + 2);
        const F2 L = f2(own ? lo_own[v] : row[f + 1], lane0(R)), SL = f2(srow[f + 1], lane0(SR));
        wl[v] = L + SL;
        wr[v] = R - SR;
      }
      hlle2<0>(wl, wr, P, fl);
#pragma unroll
      for (int v = 0; v < NV; ++v) st2(sfx + (v * TY + jj) * FPX + f, fl[v]);
    };
    // (E2) x2 faces between rows g-1 and g, column pair q
    auto x2_face = [&](int g, int q, const F2* own) {
      F2 wl[NV], wr[NV], fl[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const float* p = W + (v * WY + g + 1) * WX + q + 2;
        const float* s = sdy + (v * (TY + 2) + g) * TX + q;
        wl[v] = ld2(p) + ld2(s);
        wr[v] = (own ? own[v] : ld2(p + WX)) - (own ? hy_own[v] : ld2(s + TX));
      }
      hlle2<1>(wl, wr, P, fl);
#pragma unroll
      for (int v = 0; v < NV; ++v) st2(sfy + (v * (TY + 1) + g) * TX + q, fl[v]);
    };
    x1_face(ty, tx, own);
    x2_face(ty, tx, own);
    if (warp == 2 && lane < TY) x1_face(lane, TX, nullptr);
    if (warp == 3 && lane < TX / 2) x2_face(TY, 2 * lane, nullptr);
    if constexpr (!LEAN) x3_face();
    // (F) plane k+3 into the slot of plane k-1; then plane k+4 into the slot of plane k
    {
      const bool ok = k + 3 <= k1 + 1 ? convert(k + 3) : true;
      fence_proxy_async_smem();
      if (check_failed(ok)) return 0.0;
      if (k + 4 <= k1 + 1) issue(k + 4);
    }
    // (G) flux divergence + SSPRK2 on the own pair
    {
      F2 unew[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const float* fr = sfx + (v * TY + ty) * FPX + tx;
        const F2 fa = ld2(fr);
        const F2 fb = f2(lane1(fa), fr[2]);
        const F2 dfx = fb - fa;
        const F2 dfy = ld2(sfy + (v * (TY + 1) + ty + 1) * TX + tx) - ld2(sfy + (v * (TY + 1) + ty) * TX + tx);
        const F2 L = -fma2(dfx, idx1, fma2(dfy, idx2, (fzm[v] - fzlo[v]) * idx3));
        if (STAGE == 1) {
          unew[v] = fma2(tdt, L, ucur[v]);
        } else {
          unew[v] = fma2(f2(0.5f), u0[v], f2(0.5f) * fma2(tdt, L, ucur[v]));
        }
        st2(J.Uoutb + cell + v * vstride, unew[v]);
      }
      if (J.nbr27) {
        float u[2 * NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) split(unew[v], u[2 * v], u[2 * v + 1]);
        push_ghosts<float, 2, NV>(J, i, j, k, u, vstride);
      }
      if (J.want_rate) {
        F2 w[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) w[v] = unew[v];
        cons_to_prim2(w, P, floors);
        float ra, rb;
        wave_rate2(w, P, J.idx1, J.idx2, J.idx3, ra, rb);
        rate = rate_max(rate, rate_max(ra, rb));
      }
    }
  }
  if (parity_io) *parity_io = parity;
  return (double)rate;
}

template <int TXP, int STAGE>
__global__ void __launch_bounds__(PairSmemT<TXP>::NT, PairSmemT<TXP>::MINB)
stage_kernel_pair(const __grid_constant__ StageArgs<float> a, const __grid_constant__ CUtensorMap tmap) {
  using SM = PairSmemT<TXP>;
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  unsigned char* smem_raw = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_dyn) + 127) & ~uintptr_t(127));
  double* red = reinterpret_cast<double*>(smem_raw + SM::red_off);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + SM::bar_off);
  __shared__ int failed;
  TileJob<float> J;
  if (!make_job<float, SM::TX, SM::TY>(a, J)) return;
  if (threadIdx.x == 0) {
    failed = 0;
    for (int s = 0; s < 4; ++s) mbar_init(bars + s, 1);
    mbar_fence_init();
  }
  __syncthreads();
  unsigned floors = 0;
  const double rate = stage_tile_pair<TXP, STAGE>(J, a.P, smem_raw, floors, &tmap, J.leaf * NV, bars, &failed);
  if (failed) {
    if (threadIdx.x == 0) atomicExch(&a.sc->error, 1);
    return;
  }
  if (a.want_rate) block_max_to(&a.sc->wmax_bits, rate, red);
  if (floors) atomicAdd(&a.sc->floor_hits, (unsigned long long)floors);
}

}  // namespace ph
