// adj_ff.cuh -- plane-sweep tile of the adjoint for binary64 storage with
// double-float arithmetic (ADVECT_F64_FF), columns of 2^m level pairs.
//
// The gather form of adj_core.cuh (the same per-field sums), evaluated the
// way the double-float forward of sweep_ff.cuh is:
//
//  * Each landed six-field slab is split once per CTA, in place, into
//    16-byte level pairs (hi_k, hi_k+1, lo_k, lo_k+1); the cotangent masks
//    (dsu, dsv zero at level 0; dsw zero at levels 0 and nz-1) are applied
//    by the split, so the arithmetic reads masked values.  Every warp splits
//    its share of plane ql+2 after computing plane ql and arrives on the
//    slot's conversion mbarrier; a warp starts plane ql+1 once all warps have
//    split it, one plane of compute after they did.  The split is spread
//    over all warps (no scheduler is left with a converter warp's extra
//    load), and warps still drift up to a plane apart.  Ring: planes ql-1,
//    ql, ql+1 read, ql+2 being split, so four slots at least.
//  * A thread owns the levels (k0, k0+1) of one column; both levels run in
//    the two-wide binary32 instructions.
//  * No vector is carried across planes: every vector is read from shared
//    memory by the term that uses it (volatile loads), and the seven
//    shifted vertical coefficient tables, tcx and tcy sit in a shared table.
//    Only five terms a plane shares with the next are carried: a sum or
//    product of plane i's values that reappears at plane i+1 as its x-1
//    counterpart (lu(y+)u - lu u(y+) in dv; u + u(y+) in dv; u + u(z+),
//    lu(z+)u and lu u(z+) in dw).
//  * Face sums and products that reach level k from level k-1 are formed at
//    the thread's own levels and shifted down one level by shuffle (the
//    lower faces of the vertical terms; the w-cotangent brackets of du and
//    dv, which pair a product at level k with the same product at k-1).
//
// Levels beyond the column: every shifted value that reaches a level
// outside the column is multiplied there by a zero coefficient (tzc1(nz),
// tzc2(-1), tzd1(nz), tzd2(-1), the masked tzc2(nz-1)) or a masked
// cotangent, except the shifted w-cotangent products, which are zeroed.
// The neighbouring lane's value there is another level's finite datum.
//
// SPLIT: a column's pairs span whole warps (nz / 2 a multiple of 32); the
// neighbours of a warp's first and last lanes then come from shared memory
// (loaded vectors) or are recomputed from it in scalar double-float
// (computed values shifted down).
#pragma once

#include "sweep_ff.cuh"

namespace advect {
namespace sweep {
namespace affx {

using namespace ffx;

// Vertical coefficient tables of the adjoint, level pairs (k, k+1): each
// row is one table with its level shift.
enum { C1U = 0, C2D, C20, D10, D1U, D20, D2D, kTables };

// Shared-memory bytes after the ring: the tables (kTables rows of nz / 2
// pairs, then tcx and tcy broadcast) and the conversion mbarriers.
__host__ __device__ inline size_t adj_ff_extra_bytes(int nb, int nz) {
  return (size_t)(kTables * (nz / 2) + 2) * 16 + (size_t)nb * sizeof(uint64_t);
}

__device__ __forceinline__ float lds32(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}

// Scalar double-float values of one level from a converted pair at shared
// address a: level 2p (.x) or 2p+1 (.y).
__device__ __forceinline__ ff lx(uint32_t a) { return ff(lds32(a), lds32(a + 8)); }
__device__ __forceinline__ ff ly(uint32_t a) { return ff(lds32(a + 4), lds32(a + 12)); }

__device__ __forceinline__ FF2 dbl(const FF2& v) { return FF2{add2(v.hi, v.hi), add2(v.lo, v.lo)}; }

__device__ __forceinline__ F1 f1(const ff& v) { return F1{v.hi, v.lo}; }

}  // namespace affx

// Sweep one adjoint tile with blockDim.x = t.ty * t.kb threads (a multiple of
// 32), t.kb = nz / 2 a power of two; R.nb >= 4.
// NZC, TYC: the column height and rows per tile fixed at compile time (then
// t.nz == NZC, t.ty == TYC and every slab offset is an immediate), or 0 to
// take them from the tile.
template <bool SPLIT, int NZC = 0, int TYC = 0>
__device__ inline bool adjoint_tile_ff(const Tile<f64ff>& t, const Ring& R, int* flag) {
  using namespace affx;
  const int NB = R.nb;
  const int tid = threadIdx.x, lane = tid & 31;
  const int nz = NZC ? NZC : t.nz, ty = TYC ? TYC : t.ty, ny = t.ny;
  const int KB = nz / P;
  const int nthreads = ty * KB;
  const int nwarps = nthreads >> 5;
  const int nplanes = t.i_hi - t.i_lo + 2;
  const int rows = ty + 2;
  // slot stride: the slab of six binary64 fields
  const uint32_t cap = (NZC && TYC) ? 6u * (TYC + 2) * NZC * 8u : (uint32_t)R.slot_cap;
  const uint32_t ring = (uint32_t)__cvta_generic_to_shared(R.slots);
  float4* ctab = reinterpret_cast<float4*>(R.slots + ring_bytes(R.nb, R.slot_cap));
  uint64_t* conv = reinterpret_cast<uint64_t*>(ctab + kTables * KB + 2);
  if (tid == 0)  // made visible by start_tile's fence and barrier
    for (int s = 0; s < NB; ++s) mbar_init(&conv[s], nwarps);
  // the split constants (visible after start_tile's barrier); zero beyond
  // the column
  for (int e = tid; e < kTables * KB + 2; e += nthreads) {
    FF2 c;
    if (e < kTables * KB) {
      const int m = e / KB, kp = e - m * KB;
      int tab = TZC1, sh = 0;  // table row m holds table `tab` at level k + sh
      switch (m) {
        case C1U: tab = TZC1; sh = 1; break;
        case C2D: tab = TZC2; sh = -1; break;
        case C20: tab = TZC2; break;
        case D10: tab = TZD1; break;
        case D1U: tab = TZD1; sh = 1; break;
        case D20: tab = TZD2; break;
        default: tab = TZD2; sh = -1; break;  // D2D
      }
      const int k = 2 * kp + sh;
      const double a = (k >= 0 && k < nz) ? __ldg(t.c.d + tab * nz + k) : 0.0;
      const double b = (k + 1 >= 0 && k + 1 < nz) ? __ldg(t.c.d + tab * nz + k + 1) : 0.0;
      const ff fa(a), fb(b);
      c = FF2{make_float2(fa.hi, fb.hi), make_float2(fa.lo, fb.lo)};
    } else {
      c = bcast(ff(e == kTables * KB ? t.c.tcx : t.c.tcy));
    }
    ctab[e] = make_float4(c.hi.x, c.hi.y, c.lo.x, c.lo.y);
  }
  start_tile<6>(t, R, nplanes);
  int timed_out = 0;

  const int kb = tid % KB, rr = tid / KB;
  // Split this thread's share of plane ql's slab in place and arrive on the
  // slot's conversion barrier: pair kb of the slab rows rr, rr + ty, ...
  // (six fields of `rows` rows each).
  const uint32_t o_conv = (uint32_t)(rr * KB + kb) * 16u, step = (uint32_t)(ty * KB) * 16u;
  auto convert = [&](SlotPos q) {
    if (!mbar_wait_bounded(&R.full[q.slot], (uint32_t)(q.use & 1), t.wait_budget)) {
      atomicExch(flag, 1);
      timed_out = 1;
    }
    if (!timed_out) {
      uint32_t a = ring + (uint32_t)q.slot * cap + o_conv;
      for (int sr = rr; sr < 6 * rows; sr += ty, a += step) {
        if (sr == 0 || sr == 2 * rows) continue;  // u and w are never read at y-1
        const double2 d = lds_f64x2(a);
        ff x(d.x), y(d.y);
        // cotangents: dsu, dsv live on k >= 1, dsw on 1 <= k <= nz-2
        if (sr >= 3 * rows && kb == 0) x = ff(0.f, 0.f);
        if (sr >= 5 * rows && kb == KB - 1) y = ff(0.f, 0.f);
        sts128(a, make_float4(x.hi, y.hi, x.lo, y.lo));
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&conv[q.slot]);
  };
  auto wait_conv = [&](SlotPos q) {
    if (!mbar_wait_bounded(&conv[q.slot], (uint32_t)(q.use & 1), t.wait_budget)) {
      atomicExch(flag, 1);
      timed_out = 1;
    }
  };

  const int k0 = kb * P;
  const int j = t.j0 + rr;
  const bool row_ok = j < ny;
  const bool bottom = kb == 0;
  const int r = rr + 1;
  // byte offsets in a slab: this thread's u vector, one row, one field
  const uint32_t o_u0 = (uint32_t)(r * nz + k0) * 8u, R8 = (uint32_t)nz * 8u;
  const uint32_t F8 = (uint32_t)rows * R8;
  const uint32_t a_c = (uint32_t)__cvta_generic_to_shared(ctab + kb);
  const uint32_t a_tc = (uint32_t)__cvta_generic_to_shared(ctab + kTables * KB);
  auto coef = [&](int m) { return ldc(a_c + (uint32_t)(m * KB) * 16u); };
  const size_t plane_elems = (size_t)ny * nz;
  const size_t o_row = (size_t)j * nz + k0;
  // split-row fix-ups: this lane's neighbour level lives in another warp
  const bool fix_lo = SPLIT && lane == 0 && kb > 0;
  const bool fix_hi = SPLIT && lane == 31 && kb < KB - 1;

  // a loaded vector shifted down (levels k0-1, k0) or up (k0+1, k0+2); a is
  // its shared address
  auto dn = [&](uint32_t a, const FF2& v) {
    F1 b = below(v);
    if (fix_lo) b = f1(ly(a - 16u));
    return zm(v, b);
  };
  auto up = [&](uint32_t a, const FF2& v) {
    F1 b = above<false>(v, false);
    if (fix_hi) b = f1(lx(a + 16u));
    return zp(v, b);
  };
  // a computed value shifted down, its level k0-1 given by `fix` on the
  // split-row lanes; zeroed at the column's first level when ZERO
  auto dnc = [&](const FF2& v, const ff& fix, bool zero) {
    F1 b = below(v);
    if (fix_lo) b = f1(fix);
    if (zero && bottom) b = F1{0.f, 0.f};
    return zm(v, b);
  };

  SlotPos pm{0, 0}, pc{0, 0}, pn{0, 0}, pq{0, 0};
  pc.next(NB);
  pn = pc;
  pn.next(NB);
  pq = pn;
  pq.next(NB);
  // the first three planes are split before the sweep starts
  convert(pm);
  convert(pc);
  convert(pn);
  wait_conv(pm);
  wait_conv(pc);
  // terms that plane i shares with plane i+1, carried: as plane i+1's x-1
  // terms they are QC = lu(y+)u - lu u(y+), FY = u + u(y+), FZ = u + u(z+),
  // P1C = lu(z+)u, R1C = lu u(z+) (all of the x-1 column)
  FF2 QC, FY, FZ, P1C, R1C;
  {
    const uint32_t Pm = ring + (uint32_t)pm.slot * cap + o_u0;
    const FF2 UM = ldc(Pm), UMYP = ldc(Pm + R8), LM = ldc(Pm + 3 * F8), LMYP = ldc(Pm + 3 * F8 + R8);
    const FF2 UMu = up(Pm, UM);
    QC = sub(mul(LMYP, UM), mul(LM, UMYP));
    FY = add(UM, UMYP);
    FZ = add(UM, UMu);
    P1C = mul(up(Pm + 3 * F8, LM), UM);
    R1C = mul(LM, UMu);
  }
  for (int i = t.i_lo; i < t.i_hi; ++i) {
    const int ql = i - t.i_lo + 1;
    wait_conv(pn);
    if (__any_sync(0xffffffffu, timed_out)) break;
    // this thread's u vector in the slabs of planes i-1, i, i+1
    const uint32_t Pm = ring + (uint32_t)pm.slot * cap + o_u0;
    const uint32_t Pc = ring + (uint32_t)pc.slot * cap + o_u0;
    const uint32_t Pn = ring + (uint32_t)pn.slot * cap + o_u0;
    const size_t o = (size_t)i * plane_elems + o_row;
    const FF2 tcx = ldc(a_tc), tcy = ldc(a_tc + 16u);
    // du
    {
      const FF2 U0 = ldc(Pc), UP = ldc(Pn), UM = ldc(Pm);
      const FF2 L0 = ldc(Pc + 3 * F8), LP = ldc(Pn + 3 * F8), LM = ldc(Pm + 3 * F8);
      const FF2 U2 = dbl(U0);
      // x faces of su: lu(x+)(u(x+)+2u) + lu(u(x-)-u(x+)) - lu(x-)(u(x-)+2u)
      FF2 ax = sub(add(mul(LP, add(UP, U2)), mul(L0, sub(UM, UP))), mul(LM, add(UM, U2)));
      {
        // sv's x faces: lv(x+)v + lv(x+,y-)v(y-) - lv v(x+) - lv(y-)v(y-,x+)
        const FF2 MP = ldc(Pn + 4 * F8), MPYM = ldc(Pn + 4 * F8 - R8), M0 = ldc(Pc + 4 * F8),
                  MYM = ldc(Pc + 4 * F8 - R8);
        const FF2 V0 = ldc(Pc + F8), VYM = ldc(Pc + F8 - R8), VP = ldc(Pn + F8), VPYM = ldc(Pn + F8 - R8);
        ax = add(ax, sub(add(mul(MP, V0), mul(MPYM, VYM)), add(mul(M0, VP), mul(MYM, VPYM))));
      }
      {
        // sw's x faces: X + X(z-), X = lw(x+)w - lw w(x+)
        const FF2 NP = ldc(Pn + 5 * F8), N0 = ldc(Pc + 5 * F8);
        const FF2 W0 = ldc(Pc + 2 * F8), WP = ldc(Pn + 2 * F8);
        const FF2 X = sub(mul(NP, W0), mul(N0, WP));
        ff fx;
        if (fix_lo) {
          const uint32_t b = Pc - 16u, bn = Pn - 16u;
          fx = ly(bn + 5 * F8) * ly(b + 2 * F8) - ly(b + 5 * F8) * ly(bn + 2 * F8);
        }
        ax = add(ax, add(X, dnc(X, fx, true)));
      }
      FF2 gu = mul(tcx, ax);
      {
        // su's y faces: lu(y+)(v+v(x+)) - lu(y-)(v(y-)+v(y-,x+))
        const FF2 LYP = ldc(Pc + 3 * F8 + R8), LYM = ldc(Pc + 3 * F8 - R8);
        const FF2 V0 = ldc(Pc + F8), VP = ldc(Pn + F8), VYM = ldc(Pc + F8 - R8), VPYM = ldc(Pn + F8 - R8);
        gu = add(gu, mul(tcy, sub(mul(LYP, add(V0, VP)), mul(LYM, add(VYM, VPYM)))));
      }
      {
        // su's z faces: tzc1(k+1) lu(z+)F - tzc2(k-1) lu(z-)F(z-), F = w + w(x+)
        const FF2 W0 = ldc(Pc + 2 * F8), WP = ldc(Pn + 2 * F8);
        const FF2 F = add(W0, WP);
        ff ff_;
        if (fix_lo) ff_ = ly(Pc - 16u + 2 * F8) + ly(Pn - 16u + 2 * F8);
        const FF2 L0 = ldc(Pc + 3 * F8);
        gu = add(gu, sub(mul(mul(coef(C1U), up(Pc + 3 * F8, L0)), F),
                         mul(mul(coef(C2D), dn(Pc + 3 * F8, L0)), dnc(F, ff_, false))));
      }
      if (row_ok) {
        __stcs(reinterpret_cast<double2*>(t.o[0]) + o / 2,
               make_double2(assemble(gu.hi.x, gu.lo.x), assemble(gu.hi.y, gu.lo.y)));
      }
    }
    // dv
    {
      const FF2 U0 = ldc(Pc), UYP = ldc(Pc + R8);
      // su's y faces: lu(y+)u + lu(x-,y+)u(x-) - lu u(y+) - lu(x-)u(x-,y+) = Q + Q(x-)
      FF2 ay;
      {
        const FF2 LYP = ldc(Pc + 3 * F8 + R8), L0 = ldc(Pc + 3 * F8);
        const FF2 q = sub(mul(LYP, U0), mul(L0, UYP));
        ay = add(q, QC);
        QC = q;
      }
      {
        // sv's y faces: lv(y+)(v(y+)+2v) + lv(v(y-)-v(y+)) - lv(y-)(v(y-)+2v)
        const FF2 V0 = ldc(Pc + F8), VYP = ldc(Pc + F8 + R8), VYM = ldc(Pc + F8 - R8);
        const FF2 MYP = ldc(Pc + 4 * F8 + R8), M0 = ldc(Pc + 4 * F8), MYM = ldc(Pc + 4 * F8 - R8);
        const FF2 V2 = dbl(V0);
        ay = add(ay, sub(add(mul(MYP, add(VYP, V2)), mul(M0, sub(VYM, VYP))), mul(MYM, add(VYM, V2))));
      }
      {
        // sw's y faces: Z + Z(z-), Z = lw(y+)w - lw w(y+)
        const FF2 NYP = ldc(Pc + 5 * F8 + R8), N0 = ldc(Pc + 5 * F8);
        const FF2 W0 = ldc(Pc + 2 * F8), WYP = ldc(Pc + 2 * F8 + R8);
        const FF2 Z = sub(mul(NYP, W0), mul(N0, WYP));
        ff fz;
        if (fix_lo) {
          const uint32_t b = Pc - 16u;
          fz = ly(b + 5 * F8 + R8) * ly(b + 2 * F8) - ly(b + 5 * F8) * ly(b + 2 * F8 + R8);
        }
        ay = add(ay, add(Z, dnc(Z, fz, true)));
      }
      FF2 gv = mul(tcy, ay);
      {
        // sv's x faces: lv(x+)(u+u(y+)) - lv(x-)(u(x-)+u(x-,y+))
        const FF2 MP = ldc(Pn + 4 * F8), MM = ldc(Pm + 4 * F8);
        const FF2 fy = add(U0, UYP);
        gv = add(gv, mul(tcx, sub(mul(MP, fy), mul(MM, FY))));
        FY = fy;
      }
      {
        // sv's z faces: tzc1(k+1) lv(z+)G - tzc2(k-1) lv(z-)G(z-), G = w + w(y+)
        const FF2 W0 = ldc(Pc + 2 * F8), WYP = ldc(Pc + 2 * F8 + R8);
        const FF2 G = add(W0, WYP);
        ff fg;
        if (fix_lo) fg = ly(Pc - 16u + 2 * F8) + ly(Pc - 16u + 2 * F8 + R8);
        const FF2 M0 = ldc(Pc + 4 * F8);
        gv = add(gv, sub(mul(mul(coef(C1U), up(Pc + 4 * F8, M0)), G),
                         mul(mul(coef(C2D), dn(Pc + 4 * F8, M0)), dnc(G, fg, false))));
      }
      if (row_ok) {
        __stcs(reinterpret_cast<double2*>(t.o[1]) + o / 2,
               make_double2(assemble(gv.hi.x, gv.lo.x), assemble(gv.hi.y, gv.lo.y)));
      }
    }
    // dw
    {
      const FF2 U0 = ldc(Pc), V0 = ldc(Pc + F8), VYM = ldc(Pc + F8 - R8);
      const FF2 U0u = up(Pc, U0), V0u = up(Pc + F8, V0), VYMu = up(Pc + F8 - R8, VYM);
      FF2 gw;
      {
        // su, sv z faces through w: tzc1(k+1)[lu(z+)u + lu(x-,z+)u(x-) + lv(z+)v + lv(y-,z+)v(y-)]
        //                         - tzc2(k)[lu u(z+) + lu(x-)u(x-,z+) + lv v(z+) + lv(y-)v(y-,z+)]
        const FF2 L0 = ldc(Pc + 3 * F8), M0 = ldc(Pc + 4 * F8), MYM = ldc(Pc + 4 * F8 - R8);
        const FF2 p1 = mul(up(Pc + 3 * F8, L0), U0), r1 = mul(L0, U0u);
        const FF2 z1 = add(add(p1, P1C), add(mul(up(Pc + 4 * F8, M0), V0), mul(up(Pc + 4 * F8 - R8, MYM), VYM)));
        const FF2 z2 = add(add(r1, R1C), add(mul(M0, V0u), mul(MYM, VYMu)));
        P1C = p1;
        R1C = r1;
        gw = sub(mul(coef(C1U), z1), mul(coef(C20), z2));
      }
      {
        // sw's x and y faces: tcx[lw(x+)(u+u(z+)) - lw(x-)(u(x-)+u(x-,z+))]
        //                   + tcy[lw(y+)(v+v(z+)) - lw(y-)(v(y-)+v(y-,z+))]
        const FF2 NP = ldc(Pn + 5 * F8), NM = ldc(Pm + 5 * F8), NYP = ldc(Pc + 5 * F8 + R8),
                  NYM = ldc(Pc + 5 * F8 - R8);
        const FF2 fz = add(U0, U0u);
        const FF2 zx = sub(mul(NP, fz), mul(NM, FZ));
        FZ = fz;
        const FF2 zy = sub(mul(NYP, add(V0, V0u)), mul(NYM, add(VYM, VYMu)));
        gw = add(gw, add(mul(tcx, zx), mul(tcy, zy)));
      }
      {
        // sw's z faces: tzd1(k+1) lw(z+)(w(z+)+2w) + lw (tzd1(k) w(z-) - tzd2(k) w(z+))
        //             - tzd2(k-1) lw(z-)(w(z-)+2w)
        const FF2 W0 = ldc(Pc + 2 * F8), N0 = ldc(Pc + 5 * F8);
        const FF2 W2 = dbl(W0), Wu = up(Pc + 2 * F8, W0), Wd = dn(Pc + 2 * F8, W0);
        const FF2 z5 = sub(add(mul(mul(coef(D1U), up(Pc + 5 * F8, N0)), add(Wu, W2)),
                               mul(N0, sub(mul(coef(D10), Wd), mul(coef(D20), Wu)))),
                           mul(mul(coef(D2D), dn(Pc + 5 * F8, N0)), add(Wd, W2)));
        gw = add(gw, z5);
      }
      if (row_ok) {
        __stcs(reinterpret_cast<double2*>(t.o[2]) + o / 2,
               make_double2(assemble(gw.hi.x, gw.lo.x), assemble(gw.hi.y, gw.lo.y)));
      }
    }
    // plane i-1 is no longer read by this warp; split plane i+2 (ql+2)
    release_plane<6>(t, R, ql - 1, pm, nplanes, nwarps, lane);
    if (ql + 2 < nplanes) convert(pq);
    pm = pc;
    pc = pn;
    pn = pq;
    pq.next(NB);
  }
  // end of the tile (all threads): on a timeout wait (bounded) for the last
  // copy issued into each slot; otherwise invalidate the slots' barriers so
  // that the ring can be re-initialised
  const int any_fail = __syncthreads_or(timed_out);
  if (tid == 0) {
    for (int s = 0; s < NB; ++s) {
      const int n = R.issued[s];
      if (any_fail) {
        if (n > 0) mbar_wait_bounded(&R.full[s], (uint32_t)((n - 1) & 1), 1 << 20);
      } else {
        mbar_inval(&R.full[s]);
        mbar_inval(&conv[s]);
      }
    }
  }
  __syncthreads();
  return !any_fail;
}

}  // namespace sweep
}  // namespace advect
