// adj_f32.cuh -- plane-sweep tile of the binary32 adjoint, 4 levels per
// thread.
//
// Same gather form, ring and bounded waits as adjoint_tile (adj_core.cuh,
// whose file comment has the formulas).  What differs is how a thread holds
// its data.  A thread owns 4 consecutive levels of one column (16-byte
// vectors), so a 128-level column is one warp and the vertical halos never
// cross a warp.  Plane i's vectors are read from shared memory in the
// iteration that computes plane i (the slot of plane i and that of plane
// i+1 are both resident then), instead of being carried in registers from
// the previous iteration; only the six x-1 vectors (u, u(y+1), lu, lu(y+1),
// lv, lw of plane i-1) and two of their halos are carried.  That trades
// register moves and registers for shared-memory loads: 24 vector loads
// and 16 shuffles per plane of 4 points per thread.
#pragma once

#include "adj_core.cuh"

namespace advect {
namespace sweep {

namespace a4 {

constexpr int P = 4;

__device__ __forceinline__ void ld4(const float* s, float (&o)[P]) {
  const float4 x = *reinterpret_cast<const float4*>(s);
  o[0] = x.x;
  o[1] = x.y;
  o[2] = x.z;
  o[3] = x.w;
}

__device__ __forceinline__ void st4(float* g, const float (&v)[P]) {
  __stcs(reinterpret_cast<float4*>(g), make_float4(v[0], v[1], v[2], v[3]));
}

// Per-level coefficient table in shared memory after the ring: the four
// tables tzc1, tzc2, tzd1, tzd2 (binary32), each a row of nz + 8 values with
// level k at 4 + k and zeros at levels -4..-1 and nz..nz+3, so that the
// levels k-1 and k+1 a thread's formulas read at its first and last level
// are plain loads (zero beyond the column).  A thread reads its 4 levels of
// a row with one 16-byte load (consecutive k-blocks, consecutive addresses)
// plus one 4-byte load for the level below or above.
constexpr int kTables = 4;
__host__ __device__ inline int table_row(int nz) { return nz + 8; }
__host__ __device__ inline size_t table_bytes(int nz) { return (size_t)kTables * table_row(nz) * sizeof(float); }

__device__ __forceinline__ float4 lds4(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
  return v;
}

__device__ __forceinline__ float lds1(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}

}  // namespace a4

// Sweep one binary32 adjoint tile (same contract as adjoint_tile; t.kb =
// nz / 4).
template <bool SPLIT>
__device__ bool adjoint_tile_f32v4(const Tile<float>& t, const Ring& R, int* flag) {
  using namespace a4;
  using C = float;
  using S = Store<float>;
  const int tid = threadIdx.x, lane = tid & 31;
  const int KB = t.kb, nz = t.nz, ny = t.ny;
  const int active_threads = t.ty * KB;  // a multiple of 32
  const int nwarps = active_threads >> 5;
  const int nplanes = t.i_hi - t.i_lo + 2;
  const int rows = t.ty + 2;
  // coefficient table after the ring (ordered before use by start_tile's
  // barrier)
  float* tab = reinterpret_cast<float*>(R.slots + ring_bytes(R.nb, R.slot_cap));
  const int trow = table_row(nz);
  for (int e = tid; e < kTables * trow; e += blockDim.x) {
    const int table = e / trow, k = e % trow - 4;
    tab[e] = (k < 0 || k >= nz) ? 0.f : S::coef(t.c, table, nz, k);  // tables ordered TZC1..TZD2
  }
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
    auto slot_ptr = [&](SlotPos q) -> const float* {
      return reinterpret_cast<const float*>(R.slots + (size_t)q.slot * R.slot_cap);
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
    // first level of the column (element 0 of k-block 0) and, for lw, the
    // top level (element 3 of the last k-block) are masked; the halo levels
    // k0-1 and k0+4 are never 0 or nz-1 (nz and k0 are multiples of 4).
    const bool bottom = kb == 0, lid = kb == KB - 1;
    auto mask_uv = [&](C (&a)[P]) { a[0] = bottom ? 0.f : a[0]; };
    auto mask_w = [&](C (&a)[P]) {
      a[0] = bottom ? 0.f : a[0];
      a[P - 1] = lid ? 0.f : a[P - 1];
    };
    const uint32_t tab_k = smem_addr(tab + 4 + k0), tab_row = (uint32_t)(trow * sizeof(float));
    const C tcx = S::tcx(t.c), tcy = S::tcy(t.c);
    const float one = 1.f;
    auto above = [&](const C (&a)[P], const float* row) {
      return halo_above<SPLIT, float, C, P>(a, row, k0, kb, KB, lane, one);
    };
    auto below = [&](const C (&a)[P], const float* row) {
      return halo_below<SPLIT, float, C, P>(a, row, k0, kb, lane, one);
    };

    // x-1 vectors carried from plane to plane (see the file comment)
    C UM[P], UMYP[P], LUM[P], LUMYP[P], LVM[P], LWM[P];
    C umP, lumP;
    wait(q0);
    {
      const float* A = slot_ptr(q0);
      ld4(A + o_u0, UM);
      ld4(A + o_uyp, UMYP);
      ld4(A + o_l0, LUM);
      ld4(A + o_lyp, LUMYP);
      ld4(A + o_m0, LVM);
      ld4(A + o_n0, LWM);
      umP = above(UM, A + o_u0 - k0);
      lumP = above(LUM, A + o_l0 - k0);
    }
    release(0, q0);
    mask_uv(LUM);
    mask_uv(LUMYP);
    mask_uv(LVM);
    mask_w(LWM);
    SlotPos pc = q1, pn = q1;
    pn.next(R.nb);
    wait(pc);

    for (int i = t.i_lo; i < t.i_hi; ++i) {
      const int qc = i - t.i_lo + 1;
      wait(pn);
      if (__any_sync(0xffffffffu, timed_out)) break;
      const float* Pc = slot_ptr(pc);
      const float* Pn = slot_ptr(pn);
      // plane i
      C U0[P], UYP[P], V0[P], VYM[P], VYP[P], W0[P], WYP[P];
      C LU0[P], LUYM[P], LUYP[P], LV0[P], LVYM[P], LVYP[P], LW0[P], LWYM[P], LWYP[P];
      ld4(Pc + o_u0, U0);
      ld4(Pc + o_uyp, UYP);
      ld4(Pc + o_v0, V0);
      ld4(Pc + o_vym, VYM);
      ld4(Pc + o_vyp, VYP);
      ld4(Pc + o_w0, W0);
      ld4(Pc + o_wyp, WYP);
      ld4(Pc + o_l0, LU0);
      ld4(Pc + o_lym, LUYM);
      ld4(Pc + o_lyp, LUYP);
      ld4(Pc + o_m0, LV0);
      ld4(Pc + o_mym, LVYM);
      ld4(Pc + o_myp, LVYP);
      ld4(Pc + o_n0, LW0);
      ld4(Pc + o_nym, LWYM);
      ld4(Pc + o_nyp, LWYP);
      // plane i+1
      C UP[P], VP[P], VPYM[P], WP[P], LUP[P], LVP[P], LVPYM[P], LWP[P];
      ld4(Pn + o_u0, UP);
      ld4(Pn + o_v0, VP);
      ld4(Pn + o_vym, VPYM);
      ld4(Pn + o_w0, WP);
      ld4(Pn + o_l0, LUP);
      ld4(Pn + o_m0, LVP);
      ld4(Pn + o_mym, LVPYM);
      ld4(Pn + o_n0, LWP);
      mask_uv(LU0);
      mask_uv(LUYM);
      mask_uv(LUYP);
      mask_uv(LV0);
      mask_uv(LVYM);
      mask_uv(LVYP);
      mask_w(LW0);
      mask_w(LWYM);
      mask_w(LWYP);
      mask_uv(LUP);
      mask_uv(LVP);
      mask_uv(LVPYM);
      mask_w(LWP);
      const C u0P = above(U0, Pc + o_u0 - k0);
      const C v0P = above(V0, Pc + o_v0 - k0);
      const C vymP = above(VYM, Pc + o_vym - k0);
      const C w0M = below(W0, Pc + o_w0 - k0);
      const C w0P = above(W0, Pc + o_w0 - k0);
      const C wypM = below(WYP, Pc + o_wyp - k0);
      const C lu0M = below(LU0, Pc + o_l0 - k0);
      const C lu0P = above(LU0, Pc + o_l0 - k0);
      const C lv0M = below(LV0, Pc + o_m0 - k0);
      const C lv0P = above(LV0, Pc + o_m0 - k0);
      const C lvymP = above(LVYM, Pc + o_mym - k0);
      const C lw0M = below(LW0, Pc + o_n0 - k0);
      const C lw0P = above(LW0, Pc + o_n0 - k0);
      const C lwypM = below(LWYP, Pc + o_nyp - k0);
      const C wpM = below(WP, Pn + o_w0 - k0);
      const C lwpM = below(LWP, Pn + o_n0 - k0);
      // plane i is no longer read from shared memory by this warp
      release(qc, pc);
      pc = pn;
      pn.next(R.nb);

      // per-level coefficients: tzc1(k+1), tzc2(k-1), tzc2(k), tzd1(k),
      // tzd1(k+1), tzd2(k), tzd2(k-1) at the thread's levels k
      const float4 z1 = lds4(tab_k), z2 = lds4(tab_k + tab_row);
      const float4 e1 = lds4(tab_k + 2 * tab_row), e2 = lds4(tab_k + 3 * tab_row);
      const float z1u = lds1(tab_k + 16), z2d = lds1(tab_k + tab_row - 4);
      const float e1u = lds1(tab_k + 2 * tab_row + 16), e2d = lds1(tab_k + 3 * tab_row - 4);
      const C c1u[P] = {z1.y, z1.z, z1.w, z1u}, c2d[P] = {z2d, z2.x, z2.y, z2.z};
      const C c20[P] = {z2.x, z2.y, z2.z, z2.w}, d10[P] = {e1.x, e1.y, e1.z, e1.w};
      const C d1u[P] = {e1.y, e1.z, e1.w, e1u}, d20[P] = {e2.x, e2.y, e2.z, e2.w};
      const C d2d[P] = {e2d, e2.x, e2.y, e2.z};
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
        st4(t.o[0] + o, gu);
        st4(t.o[1] + o, gv);
        st4(t.o[2] + o, gw);
      }
      // plane i's u, u(y+1), lu, lu(y+1), lv, lw are plane i+1's x-1 vectors
#pragma unroll
      for (int q = 0; q < P; ++q) {
        UM[q] = U0[q];
        UMYP[q] = UYP[q];
        LUM[q] = LU0[q];
        LUMYP[q] = LUYP[q];
        LVM[q] = LV0[q];
        LWM[q] = LW0[q];
      }
      umP = u0P;
      lumP = lu0P;
    }
    ok = !timed_out;
  }
  return finish_tile(R, ok);
}

}  // namespace sweep
}  // namespace advect
