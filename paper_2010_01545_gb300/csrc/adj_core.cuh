// adj_core.cuh -- plane-sweep tile of the adjoint (gather form).
//
// The adjoint of the forward map (u, v, w) -> (su, sv, sw) applied to the
// cotangents (lu, lv, lw) = (dsu, dsv, dsw) is accumulated at each input
// point p as the sum, over every forward term c * A * (B + C) that reads p,
// of the product-rule contribution (c*l*(B+C) if p is A; c*l*A if p is B or
// C).  Written out per field that gives, with l masked to the levels the
// forward computes (lu, lv on k >= 1; lw on 1 <= k <= nz-2) and tzc2 already
// zero at the top level:
//
//  du = tcx [lu(x+)(u(x+)+2u) + lu(u(x-)-u(x+)) - lu(x-)(u(x-)+2u)]
//     + tcy [lu(y+)(v+v(x+)) - lu(y-)(v(y-)+v(y-,x+))]
//     + tzc1(k+1) lu(z+)(w+w(x+)) - tzc2(k-1) lu(z-)(w(z-)+w(z-,x+))
//     + tcx [lv(x+)v + lv(x+,y-)v(y-) - lv v(x+) - lv(y-)v(y-,x+)]
//     + tcx [lw(x+)w + lw(x+,z-)w(z-) - lw w(x+) - lw(z-)w(z-,x+)]
//  dv = tcy [lu(y+)u + lu(x-,y+)u(x-) - lu u(y+) - lu(x-)u(x-,y+)]
//     + tcx [lv(x+)(u+u(y+)) - lv(x-)(u(x-)+u(x-,y+))]
//     + tcy [lv(y+)(v(y+)+2v) + lv(v(y-)-v(y+)) - lv(y-)(v(y-)+2v)]
//     + tzc1(k+1) lv(z+)(w+w(y+)) - tzc2(k-1) lv(z-)(w(z-)+w(z-,y+))
//     + tcy [lw(y+)w + lw(y+,z-)w(z-) - lw w(y+) - lw(z-)w(z-,y+)]
//  dw = tzc1(k+1) [lu(z+)u + lu(x-,z+)u(x-) + lv(z+)v + lv(y-,z+)v(y-)]
//     - tzc2(k)   [lu u(z+) + lu(x-)u(x-,z+) + lv v(z+) + lv(y-)v(y-,z+)]
//     + tcx [lw(x+)(u+u(z+)) - lw(x-)(u(x-)+u(x-,z+))]
//     + tcy [lw(y+)(v+v(z+)) - lw(y-)(v(y-)+v(y-,z+))]
//     + tzd1(k+1) lw(z+)(w(z+)+2w) + lw (tzd1(k) w(z-) - tzd2(k) w(z+))
//     - tzd2(k-1) lw(z-)(w(z-)+2w)
//
// All six inputs are needed at x and y offsets -1, 0, +1, so the tile
// streams six-field slabs through the same ring as the forward sweep.  A
// thread owns P levels of one column and rolls the own-row values of planes
// i-1, i (and the diagonal off-row values) in registers; each plane costs 16
// vector loads and 14 shuffles per thread.
#pragma once

#include "sweep_core.cuh"

namespace advect {
namespace sweep {

template <typename T>
struct AdjIO;

template <>
struct AdjIO<double> {
  static constexpr int P = 1;
  using C = double;
  __device__ static __forceinline__ void ld(const double* s, C (&o)[P]) { o[0] = *s; }
  __device__ static __forceinline__ void st(double* g, const C (&v)[P]) { __stcs(g, v[0]); }
};

template <>
struct AdjIO<float> {
  static constexpr int P = 2;
  using C = float;
  __device__ static __forceinline__ void ld(const float* s, C (&o)[P]) {
    const float2 x = *reinterpret_cast<const float2*>(s);
    o[0] = x.x;
    o[1] = x.y;
  }
  __device__ static __forceinline__ void st(float* g, const C (&v)[P]) {
    __stcs(reinterpret_cast<float2*>(g), make_float2(v[0], v[1]));
  }
};

template <>
struct AdjIO<f64ff> {
  static constexpr int P = 1;
  using C = ff;
  __device__ static __forceinline__ void ld(const f64ff* s, C (&o)[P]) { o[0] = ff(s->v); }
  __device__ static __forceinline__ void st(f64ff* g, const C (&v)[P]) {
    __stcs(reinterpret_cast<double*>(g), (double)v[0]);
  }
};

template <typename T, bool SPLIT = true>
__device__ bool adjoint_tile(const Tile<T>& t, const Ring& R, int* flag) {
  using IO = AdjIO<T>;
  using C = typename IO::C;
  using S = Store<T>;
  constexpr int P = IO::P;
  const int tid = threadIdx.x, lane = tid & 31;
  const int KB = t.kb, nz = t.nz, ny = t.ny;
  const int active_threads = t.ty * KB;  // a multiple of 32
  const int nwarps = active_threads >> 5;
  const int nplanes = t.i_hi - t.i_lo + 2;
  const int rows = t.ty + 2;
  start_tile<6>(t, R, nplanes);
  bool ok = true;
  if (tid < active_threads) {
    const int kb = tid % KB, rr = tid / KB;
    const int k0 = kb * P;
    const int j = t.j0 + rr;
    const bool row_ok = j < ny;
    const int r = rr + 1;
    // row offsets of field f, row r + d within a slot
    auto off = [&](int f, int d) { return (f * rows + r + d) * nz + k0; };
    const int o_u0 = off(0, 0), o_uyp = off(0, 1);
    const int o_v0 = off(1, 0), o_vym = off(1, -1), o_vyp = off(1, 1);
    const int o_w0 = off(2, 0), o_wyp = off(2, 1);
    const int o_l0 = off(3, 0), o_lym = off(3, -1), o_lyp = off(3, 1);
    const int o_m0 = off(4, 0), o_mym = off(4, -1), o_myp = off(4, 1);
    const int o_n0 = off(5, 0), o_nym = off(5, -1), o_nyp = off(5, 1);
    auto slot_ptr = [&](SlotPos q) -> const T* {
      return reinterpret_cast<const T*>(R.slots + (size_t)q.slot * R.slot_cap);
    };
    int timed_out = 0;
    auto wait = [&](SlotPos q) {
      if (!wait_plane(R, q, flag, t.wait_budget)) timed_out = 1;
    };
    auto release = [&](int ql, SlotPos q) { release_plane<6>(t, R, ql, q, nplanes, nwarps, lane); };
    const SlotPos q0{0, 0};
    SlotPos q1{0, 0};
    q1.next(R.nb);
    // cotangent masks: lu, lv live on k >= 1; lw on 1 <= k <= nz-2.  Only the
    // first level of the column (q = 0 of k-block 0) and, for lw, the top
    // level can be masked, so each vector needs at most two selects.
    auto muv = [&](int k) { return k >= 1; };
    auto mw = [&](int k) { return k >= 1 && k <= nz - 2; };
    const bool bottom = k0 == 0;                    // element 0 is level 0
    const bool lid = k0 + P - 1 == nz - 1;          // element P-1 is the top level
    auto mask_uv = [&](C (&a)[P]) { a[0] = bottom ? C(0) : a[0]; };
    auto mask_w = [&](C (&a)[P]) {
      a[0] = bottom ? C(0) : a[0];
      a[P - 1] = lid ? C(0) : a[P - 1];
    };
    auto coef = [&](int table, int k) -> C { return (k < 0 || k >= nz) ? C(0) : S::coef(t.c, table, nz, k); };
    C c1u[P], c2d[P], c20[P], d10[P], d1u[P], d20[P], d2d[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const int k = k0 + q;
      c1u[q] = coef(TZC1, k + 1);
      c2d[q] = coef(TZC2, k - 1);
      c20[q] = coef(TZC2, k);
      d10[q] = coef(TZD1, k);
      d1u[q] = coef(TZD1, k + 1);
      d20[q] = coef(TZD2, k);
      d2d[q] = coef(TZD2, k - 1);
    }
    const C tcx = S::tcx(t.c), tcy = S::tcy(t.c);
    const bool hm_uv = muv(k0 - 1), hm_w = mw(k0 - 1), hp_w = mw(k0 + P);
    const float one = 1.f;

    // rolled state (plane i): see the names in the file comment
    C UM[P], U0[P], UMYP[P], V0[P], VYM[P], W0[P];
    C LUM[P], LU0[P], LUMYP[P], LVM[P], LV0[P], LVYM[P], LWM[P], LW0[P];
    C u0P, umP, v0P, vymP, w0M, w0P, lu0M, lu0P, lumP, lv0M, lv0P, lvymP, lw0M, lw0P;

    wait(q0);
    wait(q1);
    {
      const T* A = slot_ptr(q0);
      const T* B = slot_ptr(q1);
      IO::ld(A + o_u0, UM);
      IO::ld(B + o_u0, U0);
      IO::ld(A + o_uyp, UMYP);
      IO::ld(B + o_v0, V0);
      IO::ld(B + o_vym, VYM);
      IO::ld(B + o_w0, W0);
      IO::ld(A + o_l0, LUM);
      IO::ld(B + o_l0, LU0);
      IO::ld(A + o_lyp, LUMYP);
      IO::ld(A + o_m0, LVM);
      IO::ld(B + o_m0, LV0);
      IO::ld(B + o_mym, LVYM);
      IO::ld(A + o_n0, LWM);
      IO::ld(B + o_n0, LW0);
      u0P = halo_above<SPLIT, T, C, P>(U0, B + o_u0 - k0, k0, kb, KB, lane, one);
      umP = halo_above<SPLIT, T, C, P>(UM, A + o_u0 - k0, k0, kb, KB, lane, one);
      v0P = halo_above<SPLIT, T, C, P>(V0, B + o_v0 - k0, k0, kb, KB, lane, one);
      vymP = halo_above<SPLIT, T, C, P>(VYM, B + o_vym - k0, k0, kb, KB, lane, one);
      w0M = halo_below<SPLIT, T, C, P>(W0, B + o_w0 - k0, k0, kb, lane, one);
      w0P = halo_above<SPLIT, T, C, P>(W0, B + o_w0 - k0, k0, kb, KB, lane, one);
      lu0M = halo_below<SPLIT, T, C, P>(LU0, B + o_l0 - k0, k0, kb, lane, one);
      lu0P = halo_above<SPLIT, T, C, P>(LU0, B + o_l0 - k0, k0, kb, KB, lane, one);
      lumP = halo_above<SPLIT, T, C, P>(LUM, A + o_l0 - k0, k0, kb, KB, lane, one);
      lv0M = halo_below<SPLIT, T, C, P>(LV0, B + o_m0 - k0, k0, kb, lane, one);
      lv0P = halo_above<SPLIT, T, C, P>(LV0, B + o_m0 - k0, k0, kb, KB, lane, one);
      lvymP = halo_above<SPLIT, T, C, P>(LVYM, B + o_mym - k0, k0, kb, KB, lane, one);
      lw0M = halo_below<SPLIT, T, C, P>(LW0, B + o_n0 - k0, k0, kb, lane, one);
      lw0P = halo_above<SPLIT, T, C, P>(LW0, B + o_n0 - k0, k0, kb, KB, lane, one);
    }
    release(0, q0);
    SlotPos pc = q1, pn = q1;
    pn.next(R.nb);
    mask_uv(LUM);
    mask_uv(LU0);
    mask_uv(LUMYP);
    mask_uv(LVM);
    mask_uv(LV0);
    mask_uv(LVYM);
    mask_w(LWM);
    mask_w(LW0);
    if (!hm_uv) { lu0M = C(0); lv0M = C(0); }
    if (!hm_w) lw0M = C(0);
    if (!hp_w) lw0P = C(0);

    for (int i = t.i_lo; i < t.i_hi; ++i) {
      const int qc = i - t.i_lo + 1;
      wait(pn);
      if (__any_sync(0xffffffffu, timed_out)) break;
      const T* Pc = slot_ptr(pc);
      const T* Pn = slot_ptr(pn);
      C UP[P], UYP[P], VP[P], VYP[P], VPYM[P], WP[P], WYP[P];
      C LUP[P], LUYM[P], LUYP[P], LVP[P], LVYP[P], LVPYM[P], LWP[P], LWYM[P], LWYP[P];
      IO::ld(Pn + o_u0, UP);
      IO::ld(Pc + o_uyp, UYP);
      IO::ld(Pn + o_v0, VP);
      IO::ld(Pc + o_vyp, VYP);
      IO::ld(Pn + o_vym, VPYM);
      IO::ld(Pn + o_w0, WP);
      IO::ld(Pc + o_wyp, WYP);
      IO::ld(Pn + o_l0, LUP);
      IO::ld(Pc + o_lym, LUYM);
      IO::ld(Pc + o_lyp, LUYP);
      IO::ld(Pn + o_m0, LVP);
      IO::ld(Pc + o_myp, LVYP);
      IO::ld(Pn + o_mym, LVPYM);
      IO::ld(Pn + o_n0, LWP);
      IO::ld(Pc + o_nym, LWYM);
      IO::ld(Pc + o_nyp, LWYP);
      const C upP = halo_above<SPLIT, T, C, P>(UP, Pn + o_u0 - k0, k0, kb, KB, lane, one);
      const C vpP = halo_above<SPLIT, T, C, P>(VP, Pn + o_v0 - k0, k0, kb, KB, lane, one);
      const C wpM = halo_below<SPLIT, T, C, P>(WP, Pn + o_w0 - k0, k0, kb, lane, one);
      const C wpP = halo_above<SPLIT, T, C, P>(WP, Pn + o_w0 - k0, k0, kb, KB, lane, one);
      const C vpymP = halo_above<SPLIT, T, C, P>(VPYM, Pn + o_vym - k0, k0, kb, KB, lane, one);
      const C wypM = halo_below<SPLIT, T, C, P>(WYP, Pc + o_wyp - k0, k0, kb, lane, one);
      C lupM = halo_below<SPLIT, T, C, P>(LUP, Pn + o_l0 - k0, k0, kb, lane, one);
      C lupP = halo_above<SPLIT, T, C, P>(LUP, Pn + o_l0 - k0, k0, kb, KB, lane, one);
      C lvpM = halo_below<SPLIT, T, C, P>(LVP, Pn + o_m0 - k0, k0, kb, lane, one);
      C lvpP = halo_above<SPLIT, T, C, P>(LVP, Pn + o_m0 - k0, k0, kb, KB, lane, one);
      C lwpM = halo_below<SPLIT, T, C, P>(LWP, Pn + o_n0 - k0, k0, kb, lane, one);
      C lwpP = halo_above<SPLIT, T, C, P>(LWP, Pn + o_n0 - k0, k0, kb, KB, lane, one);
      const C lvpymP = halo_above<SPLIT, T, C, P>(LVPYM, Pn + o_mym - k0, k0, kb, KB, lane, one);
      C lwypM = halo_below<SPLIT, T, C, P>(LWYP, Pc + o_nyp - k0, k0, kb, lane, one);
      release(qc, pc);
      pc = pn;
      pn.next(R.nb);
      mask_uv(LUP);
      mask_uv(LUYM);
      mask_uv(LUYP);
      mask_uv(LVP);
      mask_uv(LVYP);
      mask_uv(LVPYM);
      mask_w(LWP);
      mask_w(LWYM);
      mask_w(LWYP);
      if (!hm_uv) { lupM = C(0); lvpM = C(0); }
      if (!hm_w) { lwpM = C(0); lwypM = C(0); }
      if (!hp_w) lwpP = C(0);

      C gu[P], gv[P], gw[P];
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const C u0 = U0[q], uxm = UM[q], uxp = UP[q], uyp = UYP[q], uxm_yp = UMYP[q];
        const C uzp = q < P - 1 ? U0[q + 1] : u0P;
        const C uxm_zp = q < P - 1 ? UM[q + 1] : umP;
        const C v0 = V0[q], vxp = VP[q], vym = VYM[q], vyp = VYP[q], vym_xp = VPYM[q];
        const C vzp = q < P - 1 ? V0[q + 1] : v0P;
        const C vym_zp = q < P - 1 ? VYM[q + 1] : vymP;
        const C w0 = W0[q], wxp = WP[q], wyp = WYP[q];
        const C wzm = q > 0 ? W0[q - 1] : w0M;
        const C wzp = q < P - 1 ? W0[q + 1] : w0P;
        const C wzm_xp = q > 0 ? WP[q - 1] : wpM;
        const C wzm_yp = q > 0 ? WYP[q - 1] : wypM;
        const C lu0 = LU0[q], luxp = LUP[q], luxm = LUM[q], luyp = LUYP[q], luym = LUYM[q];
        const C luzp = q < P - 1 ? LU0[q + 1] : lu0P;
        const C luzm = q > 0 ? LU0[q - 1] : lu0M;
        const C luxm_yp = LUMYP[q];
        const C luxm_zp = q < P - 1 ? LUM[q + 1] : lumP;
        const C lv0 = LV0[q], lvxp = LVP[q], lvxm = LVM[q], lvyp = LVYP[q], lvym = LVYM[q];
        const C lvzp = q < P - 1 ? LV0[q + 1] : lv0P;
        const C lvzm = q > 0 ? LV0[q - 1] : lv0M;
        const C lvxp_ym = LVPYM[q];
        const C lvym_zp = q < P - 1 ? LVYM[q + 1] : lvymP;
        const C lw0 = LW0[q], lwxp = LWP[q], lwxm = LWM[q], lwyp = LWYP[q], lwym = LWYM[q];
        const C lwzp = q < P - 1 ? LW0[q + 1] : lw0P;
        const C lwzm = q > 0 ? LW0[q - 1] : lw0M;
        const C lwxp_zm = q > 0 ? LWP[q - 1] : lwpM;
        const C lwyp_zm = q > 0 ? LWYP[q - 1] : lwypM;

        const C u2 = u0 + u0, v2 = v0 + v0, w2 = w0 + w0;  // exact doublings
        C a = tcx * (luxp * (uxp + u2) + lu0 * (uxm - uxp) - luxm * (uxm + u2));
        a += tcy * (luyp * (v0 + vxp) - luym * (vym + vym_xp));
        a += c1u[q] * luzp * (w0 + wxp) - c2d[q] * luzm * (wzm + wzm_xp);
        a += tcx * (lvxp * v0 + lvxp_ym * vym - lv0 * vxp - lvym * vym_xp);
        a += tcx * (lwxp * w0 + lwxp_zm * wzm - lw0 * wxp - lwzm * wzm_xp);
        C b = tcy * (luyp * u0 + luxm_yp * uxm - lu0 * uyp - luxm * uxm_yp);
        b += tcx * (lvxp * (u0 + uyp) - lvxm * (uxm + uxm_yp));
        b += tcy * (lvyp * (vyp + v2) + lv0 * (vym - vyp) - lvym * (vym + v2));
        b += c1u[q] * lvzp * (w0 + wyp) - c2d[q] * lvzm * (wzm + wzm_yp);
        b += tcy * (lwyp * w0 + lwyp_zm * wzm - lw0 * wyp - lwzm * wzm_yp);
        C c = c1u[q] * (luzp * u0 + luxm_zp * uxm + lvzp * v0 + lvym_zp * vym);
        c -= c20[q] * (lu0 * uzp + luxm * uxm_zp + lv0 * vzp + lvym * vym_zp);
        c += tcx * (lwxp * (u0 + uzp) - lwxm * (uxm + uxm_zp));
        c += tcy * (lwyp * (v0 + vzp) - lwym * (vym + vym_zp));
        c += d1u[q] * lwzp * (wzp + w2) + lw0 * (d10[q] * wzm - d20[q] * wzp) - d2d[q] * lwzm * (wzm + w2);
        gu[q] = a;
        gv[q] = b;
        gw[q] = c;
      }
      if (row_ok) {
        const size_t o = ((size_t)i * ny + j) * nz + k0;
        IO::st(t.o[0] + o, gu);
        IO::st(t.o[1] + o, gv);
        IO::st(t.o[2] + o, gw);
      }
      // roll to plane i+1
#pragma unroll
      for (int q = 0; q < P; ++q) {
        UM[q] = U0[q];
        U0[q] = UP[q];
        UMYP[q] = UYP[q];
        V0[q] = VP[q];
        VYM[q] = VPYM[q];
        W0[q] = WP[q];
        LUM[q] = LU0[q];
        LU0[q] = LUP[q];
        LUMYP[q] = LUYP[q];
        LVM[q] = LV0[q];
        LV0[q] = LVP[q];
        LVYM[q] = LVPYM[q];
        LWM[q] = LW0[q];
        LW0[q] = LWP[q];
      }
      umP = u0P;
      u0P = upP;
      v0P = vpP;
      vymP = vpymP;
      w0M = wpM;
      w0P = wpP;
      lumP = lu0P;
      lu0M = lupM;
      lu0P = lupP;
      lv0M = lvpM;
      lv0P = lvpP;
      lvymP = lvpymP;
      lw0M = lwpM;
      lw0P = lwpP;
    }
    ok = !timed_out;
  }
  return finish_tile(R, ok);
}

}  // namespace sweep
}  // namespace advect
