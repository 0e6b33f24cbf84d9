// sweep_h16.cuh -- plane-sweep tile of the forward for binary16 storage with
// per-field power-of-two scales (F16S), arithmetic in binary32.
//
// Same ring, slabs and bounded waits as the generic sweep (sweep_core.cuh);
// what differs is the arithmetic.  Every term of Listing 1 and of its v/w
// analogues has the form  A * (B + C)  with A, B, C stored values, so it is
// evaluated as the two products  A*B + A*C  of raw binary16 values, each with
// one mixed-precision fused multiply-add (binary16 operands, binary32
// addend and result: the product of two binary16 numbers is exact in
// binary32).  The stored halves are never converted: they stay packed two
// to a register, and the multiply-add takes its operands from either half.
// Each horizontal direction's four products are one chain (the outflow
// pair first, its sum entering the inflow pair's chain negated), and the x,
// y and two vertical sums are combined with their coefficients by two-wide
// binary32 multiply-adds on the levels (q, q+1) of a register pair.
//
// A thread owns 8 consecutive levels of one column (one 16-byte vector per
// field and row).  The input scales are powers of two and are folded into
// the horizontal coefficients and the output scale exactly as in the generic
// sweep: with raw values every product of the field f's sum is scaled by
// s_f s_w, the x and y sums carry s_u / s_w and s_v / s_w, and the output
// factor s_f s_w / s_out,f restores the true value over the output scale.
#pragma once

#include "sweep_core.cuh"

namespace advect {
namespace sweep {

namespace h16 {

constexpr int P = 8;  // levels per thread

// a.half(HA) * b.half(HB) + c: binary16 operands taken from either half of a
// 32-bit register, exact product, binary32 addend and result.
template <int HA, int HB>
__device__ __forceinline__ float mfma(uint32_t a, uint32_t b, float c) {
  float d;
  if constexpr (HA == 0 && HB == 0)
    asm("{.reg .f16 a0, a1, b0, b1;\n\tmov.b32 {a0, a1}, %1;\n\tmov.b32 {b0, b1}, %2;\n\t"
        "fma.rn.f32.f16 %0, a0, b0, %3;\n\t}"
        : "=f"(d) : "r"(a), "r"(b), "f"(c));
  else if constexpr (HA == 0 && HB == 1)
    asm("{.reg .f16 a0, a1, b0, b1;\n\tmov.b32 {a0, a1}, %1;\n\tmov.b32 {b0, b1}, %2;\n\t"
        "fma.rn.f32.f16 %0, a0, b1, %3;\n\t}"
        : "=f"(d) : "r"(a), "r"(b), "f"(c));
  else if constexpr (HA == 1 && HB == 0)
    asm("{.reg .f16 a0, a1, b0, b1;\n\tmov.b32 {a0, a1}, %1;\n\tmov.b32 {b0, b1}, %2;\n\t"
        "fma.rn.f32.f16 %0, a1, b0, %3;\n\t}"
        : "=f"(d) : "r"(a), "r"(b), "f"(c));
  else
    asm("{.reg .f16 a0, a1, b0, b1;\n\tmov.b32 {a0, a1}, %1;\n\tmov.b32 {b0, b1}, %2;\n\t"
        "fma.rn.f32.f16 %0, a1, b1, %3;\n\t}"
        : "=f"(d) : "r"(a), "r"(b), "f"(c));
  return d;
}

// An 8-level vector with its vertical neighbours: e[0] holds level -1 in its
// high half (from the lane below), e[1..4] levels 0..7 (level L in e[1 + L/2],
// half L%2), e[5] level 8 in its low half (from the lane above).
struct Ext {
  uint32_t e[6];
};

template <int L>
struct At {
  static constexpr int reg = L < 0 ? 0 : (L > 7 ? 5 : 1 + L / 2);
  static constexpr int half = L < 0 ? 1 : (L > 7 ? 0 : (L & 1));
};

// a(LA) * b(LB) + c
template <int LA, int LB>
__device__ __forceinline__ float mf(const Ext& a, const Ext& b, float c) {
  return mfma<At<LA>::half, At<LB>::half>(a.e[At<LA>::reg], b.e[At<LB>::reg], c);
}

__device__ __forceinline__ void ld8(const __half* s, Ext& v) {
  const uint4 x = *reinterpret_cast<const uint4*>(s);
  v.e[1] = x.x;
  v.e[2] = x.y;
  v.e[3] = x.z;
  v.e[4] = x.w;
}

__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ uint32_t pack_h2(float2 v) {
  const __half2 h = __floats2half2_rn(v.x, v.y);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// Per-thread constants of the sweep (pairs for levels (q, q+1)).  The
// per-level coefficients are read from a shared-memory table each plane
// (registers are the scarce resource at four CTAs per SM).  For the level
// pair (k, k+1), k = 8 kb + 2 qp, the table holds (tzc1, tzc1, -tzc2, -tzc2)
// of levels (k, k+1, k, k+1) at entry qp * KB + kb of its first half and
// (tzd1, tzd1, -tzd2, -tzd2) at the same entry of its second half, so the
// k-blocks of a row read consecutive 16-byte entries (no bank conflicts).
struct Consts {
  float2 tcx, tcy;  // folded horizontal coefficients
  float2 o[3];                  // output factors of su, sv, sw
  uint32_t tab;                 // shared-memory address of the thread's entry for qp = 0
  uint32_t qstride, half;       // bytes between qp entries, and to the tzd half
};

// Shared-memory bytes of the coefficient table of an nz-level column.
__host__ __device__ inline size_t table_bytes(int nz) { return (size_t)(nz / 2) * 2 * sizeof(float4); }

__device__ __forceinline__ float4 lds128(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
  return v;
}

// The vectors a plane's arithmetic reads (see the file comment of
// sweep_core.cuh for the names: X = plane offset, Y = row offset).
struct Plane {
  Ext UXM, U0, UXP, UYM, UYP, UXMYP;
  Ext VXM, V0, VXP, VYM, VYP, VXPYM;
  Ext WXM, W0, WXP, WYM, WYP;
};

// Levels Q and Q+1 of the three fields; packed binary16 results.
template <int Q>
__device__ __forceinline__ void level_pair(const Plane& p, const Consts& k, uint32_t& ou, uint32_t& ov,
                                           uint32_t& ow) {
  const uint32_t a = k.tab + (Q / 2) * k.qstride;
  const float4 zc = lds128(a), zd = lds128(a + k.half);
  const float2 c1 = make_float2(zc.x, zc.y), nc2 = make_float2(zc.z, zc.w);
  const float2 d1 = make_float2(zd.x, zd.y), nd2 = make_float2(zd.z, zd.w);
  float2 X, Y, L, H;
  // su (Listing 1): x faces in minus out, y faces in minus out (each a chain
  // of four products ending in the inflow pair, the outflow pair's sum
  // entering negated), lower and upper vertical faces
  X.x = mf<Q, Q>(p.UXM, p.UXM, mf<Q, Q>(p.UXM, p.U0, -mf<Q, Q>(p.UXP, p.U0, mf<Q, Q>(p.UXP, p.UXP, 0.f))));
  X.y = mf<Q + 1, Q + 1>(p.UXM, p.UXM,
                         mf<Q + 1, Q + 1>(p.UXM, p.U0, -mf<Q + 1, Q + 1>(p.UXP, p.U0, mf<Q + 1, Q + 1>(p.UXP, p.UXP, 0.f))));
  Y.x = mf<Q, Q>(p.UYM, p.VYM, mf<Q, Q>(p.UYM, p.VXPYM, -mf<Q, Q>(p.UYP, p.V0, mf<Q, Q>(p.UYP, p.VXP, 0.f))));
  Y.y = mf<Q + 1, Q + 1>(p.UYM, p.VYM,
                         mf<Q + 1, Q + 1>(p.UYM, p.VXPYM, -mf<Q + 1, Q + 1>(p.UYP, p.V0, mf<Q + 1, Q + 1>(p.UYP, p.VXP, 0.f))));
  L.x = mf<Q - 1, Q - 1>(p.U0, p.W0, mf<Q - 1, Q - 1>(p.U0, p.WXP, 0.f));
  L.y = mf<Q, Q>(p.U0, p.W0, mf<Q, Q>(p.U0, p.WXP, 0.f));
  H.x = mf<Q + 1, Q>(p.U0, p.W0, mf<Q + 1, Q>(p.U0, p.WXP, 0.f));
  H.y = mf<Q + 2, Q + 1>(p.U0, p.W0, mf<Q + 2, Q + 1>(p.U0, p.WXP, 0.f));
  float2 h = f2mul(k.tcx, X);
  h = f2fma(k.tcy, Y, h);
  h = f2fma(c1, L, h);
  h = f2fma(nc2, H, h);
  ou = pack_h2(f2mul(k.o[0], h));
  // sv
  X.x = mf<Q, Q>(p.VXM, p.UXM, mf<Q, Q>(p.VXM, p.UXMYP, -mf<Q, Q>(p.VXP, p.U0, mf<Q, Q>(p.VXP, p.UYP, 0.f))));
  X.y = mf<Q + 1, Q + 1>(p.VXM, p.UXM,
                         mf<Q + 1, Q + 1>(p.VXM, p.UXMYP, -mf<Q + 1, Q + 1>(p.VXP, p.U0, mf<Q + 1, Q + 1>(p.VXP, p.UYP, 0.f))));
  Y.x = mf<Q, Q>(p.VYM, p.V0, mf<Q, Q>(p.VYM, p.VYM, -mf<Q, Q>(p.VYP, p.V0, mf<Q, Q>(p.VYP, p.VYP, 0.f))));
  Y.y = mf<Q + 1, Q + 1>(p.VYM, p.V0,
                         mf<Q + 1, Q + 1>(p.VYM, p.VYM, -mf<Q + 1, Q + 1>(p.VYP, p.V0, mf<Q + 1, Q + 1>(p.VYP, p.VYP, 0.f))));
  L.x = mf<Q - 1, Q - 1>(p.V0, p.W0, mf<Q - 1, Q - 1>(p.V0, p.WYP, 0.f));
  L.y = mf<Q, Q>(p.V0, p.W0, mf<Q, Q>(p.V0, p.WYP, 0.f));
  H.x = mf<Q + 1, Q>(p.V0, p.W0, mf<Q + 1, Q>(p.V0, p.WYP, 0.f));
  H.y = mf<Q + 2, Q + 1>(p.V0, p.W0, mf<Q + 2, Q + 1>(p.V0, p.WYP, 0.f));
  h = f2mul(k.tcx, X);
  h = f2fma(k.tcy, Y, h);
  h = f2fma(c1, L, h);
  h = f2fma(nc2, H, h);
  ov = pack_h2(f2mul(k.o[1], h));
  // sw
  X.x = mf<Q, Q>(p.WXM, p.UXM, mf<Q, Q + 1>(p.WXM, p.UXM, -mf<Q, Q>(p.WXP, p.U0, mf<Q, Q + 1>(p.WXP, p.U0, 0.f))));
  X.y = mf<Q + 1, Q + 1>(p.WXM, p.UXM,
                         mf<Q + 1, Q + 2>(p.WXM, p.UXM, -mf<Q + 1, Q + 1>(p.WXP, p.U0, mf<Q + 1, Q + 2>(p.WXP, p.U0, 0.f))));
  Y.x = mf<Q, Q>(p.WYM, p.VYM, mf<Q, Q + 1>(p.WYM, p.VYM, -mf<Q, Q>(p.WYP, p.V0, mf<Q, Q + 1>(p.WYP, p.V0, 0.f))));
  Y.y = mf<Q + 1, Q + 1>(p.WYM, p.VYM,
                         mf<Q + 1, Q + 2>(p.WYM, p.VYM, -mf<Q + 1, Q + 1>(p.WYP, p.V0, mf<Q + 1, Q + 2>(p.WYP, p.V0, 0.f))));
  L.x = mf<Q - 1, Q>(p.W0, p.W0, mf<Q - 1, Q - 1>(p.W0, p.W0, 0.f));
  L.y = mf<Q, Q + 1>(p.W0, p.W0, mf<Q, Q>(p.W0, p.W0, 0.f));
  H.x = mf<Q + 1, Q>(p.W0, p.W0, mf<Q + 1, Q + 1>(p.W0, p.W0, 0.f));
  H.y = mf<Q + 2, Q + 1>(p.W0, p.W0, mf<Q + 2, Q + 2>(p.W0, p.W0, 0.f));
  h = f2mul(k.tcx, X);
  h = f2fma(k.tcy, Y, h);
  h = f2fma(d1, L, h);
  h = f2fma(nd2, H, h);
  ow = pack_h2(f2mul(k.o[2], h));
}

// Vertical halos by warp shuffle: the register holding level -1 (high half)
// or level 8 (low half) of the neighbouring lane's vector; from shared
// memory where the row crosses a warp boundary (SPLIT).  Beyond the column
// the value is some other column's level; it is zeroed only where it can
// reach an output that is kept.  Level -1 is read only by the arithmetic of
// level 0, whose su, sv and sw are all cleared bit for bit afterwards, so the
// halo below is never zeroed; level nz is read only at level nz-1, where sw
// is cleared but su and sv multiply it by tzc2(nz-1) = 0, so the halos above
// of u and v are zeroed (a non-finite neighbour times zero would not be
// zero) and those of the other vectors are not (ZERO).
template <bool SPLIT>
__device__ __forceinline__ uint32_t halo_lo(const Ext& v, const __half* row, int k0, int kb, int lane) {
  uint32_t r = __shfl_up_sync(0xffffffffu, v.e[4], 1);
  if (SPLIT && lane == 0 && kb > 0) r = *reinterpret_cast<const uint32_t*>(row + k0 - 2);
  return r;
}

template <bool SPLIT, bool ZERO>
__device__ __forceinline__ uint32_t halo_hi(const Ext& v, const __half* row, int k0, int kb, int KB, int lane) {
  uint32_t r = __shfl_down_sync(0xffffffffu, v.e[1], 1);
  if (SPLIT && lane == 31 && kb < KB - 1) r = *reinterpret_cast<const uint32_t*>(row + k0 + P);
  return (ZERO && kb == KB - 1) ? 0u : r;
}

__device__ __forceinline__ void copy_levels(Ext& d, const Ext& s) {
  d.e[1] = s.e[1];
  d.e[2] = s.e[2];
  d.e[3] = s.e[3];
  d.e[4] = s.e[4];
}

}  // namespace h16

// Sweep one F16S tile (same contract as forward_tile; t.kb = nz / 8).
template <bool SPLIT>
__device__ bool forward_tile_h16(const Tile<__half>& t, const Ring& R, int* flag) {
  using namespace h16;
  const int NB = R.nb;
  const int tid = threadIdx.x, lane = tid & 31;
  const int KB = t.kb, nz = t.nz, ny = t.ny;
  const int active_threads = t.ty * KB;  // a multiple of 32
  const int nwarps = active_threads >> 5;
  const int nplanes = t.i_hi - t.i_lo + 2;
  const int rows = t.ty + 2;

  // coefficient table after the ring (ordered before use by start_tile's
  // barrier)
  float4* tab = reinterpret_cast<float4*>(R.slots + ring_bytes(R.nb, R.slot_cap));
  for (int pq = tid; pq < nz / 2; pq += blockDim.x) {
    const float* f = t.c.f;
    const int k = 2 * pq, e = (pq % 4) * KB + pq / 4;
    tab[e] = make_float4(f[TZC1 * nz + k], f[TZC1 * nz + k + 1], -f[TZC2 * nz + k], -f[TZC2 * nz + k + 1]);
    tab[nz / 2 + e] =
        make_float4(f[TZD1 * nz + k], f[TZD1 * nz + k + 1], -f[TZD2 * nz + k], -f[TZD2 * nz + k + 1]);
  }
  start_tile<3>(t, R, nplanes);
  bool ok = true;
  if (tid < active_threads) {
    const int kb = tid % KB, rr = tid / KB;
    const int k0 = kb * P;
    const int j = t.j0 + rr;
    const bool row_ok = j < ny;
    Consts K;
    K.tab = smem_addr(tab + kb);
    K.qstride = (uint32_t)(KB * sizeof(float4));
    K.half = (uint32_t)(nz / 2 * sizeof(float4));
    {
      const float s_u = t.sc.in[0], s_v = t.sc.in[1], s_w = t.sc.in[2];
      const float iw = 1.f / s_w;
      const float tx = t.c.tcx_f * s_u * iw, ty = t.c.tcy_f * s_v * iw;
      K.tcx = make_float2(tx, tx);
      K.tcy = make_float2(ty, ty);
      const float ou = t.sc.inv_out[0] * s_u * s_w, ov = t.sc.inv_out[1] * s_v * s_w,
                  ow = t.sc.inv_out[2] * s_w * s_w;
      K.o[0] = make_float2(ou, ou);
      K.o[1] = make_float2(ov, ov);
      K.o[2] = make_float2(ow, ow);
    }
    // su, sv (level 0) and sw (levels 0 and nz-1) are zero: masks on the
    // packed results of the first and last level pair
    const uint32_t keep_first = kb == 0 ? 0xffff0000u : 0xffffffffu;
    const uint32_t keep_last = kb == KB - 1 ? 0x0000ffffu : 0xffffffffu;

    const int r = rr + 1;
    const int o_u0 = r * nz + k0, o_um = (r - 1) * nz + k0, o_up = (r + 1) * nz + k0;
    const int o_v0 = (rows + r) * nz + k0, o_vm = (rows + r - 1) * nz + k0, o_vp = (rows + r + 1) * nz + k0;
    const int o_w0 = (2 * rows + r) * nz + k0, o_wm = (2 * rows + r - 1) * nz + k0,
              o_wp = (2 * rows + r + 1) * nz + k0;
    auto slot_ptr = [&](SlotPos q) -> const __half* {
      return reinterpret_cast<const __half*>(R.slots + (size_t)q.slot * R.slot_cap);
    };
    int timed_out = 0;
    auto wait = [&](SlotPos q) {
      if (!wait_plane(R, q, flag, t.wait_budget)) timed_out = 1;
    };
    auto release = [&](int ql, SlotPos q) { release_plane<3>(t, R, ql, q, nplanes, nwarps, lane); };
    const SlotPos q0{0, 0};
    SlotPos q1{0, 0};
    q1.next(NB);

    Plane p;
    wait(q0);
    wait(q1);
    {
      const __half* P0 = slot_ptr(q0);
      const __half* P1 = slot_ptr(q1);
      ld8(P0 + o_u0, p.UXM);
      ld8(P1 + o_u0, p.U0);
      ld8(P0 + o_up, p.UXMYP);
      ld8(P0 + o_v0, p.VXM);
      ld8(P1 + o_v0, p.V0);
      ld8(P1 + o_vm, p.VYM);
      ld8(P0 + o_w0, p.WXM);
      ld8(P1 + o_w0, p.W0);
      // halos carried into the first plane (the others come with each plane)
      p.U0.e[0] = halo_lo<SPLIT>(p.U0, P1 + o_u0 - k0, k0, kb, lane);
      p.U0.e[5] = halo_hi<SPLIT, true>(p.U0, P1 + o_u0 - k0, k0, kb, KB, lane);
      p.UXM.e[5] = halo_hi<SPLIT, false>(p.UXM, P0 + o_u0 - k0, k0, kb, KB, lane);
      p.V0.e[0] = halo_lo<SPLIT>(p.V0, P1 + o_v0 - k0, k0, kb, lane);
      p.V0.e[5] = halo_hi<SPLIT, true>(p.V0, P1 + o_v0 - k0, k0, kb, KB, lane);
      p.VYM.e[5] = halo_hi<SPLIT, false>(p.VYM, P1 + o_vm - k0, k0, kb, KB, lane);
      p.W0.e[0] = halo_lo<SPLIT>(p.W0, P1 + o_w0 - k0, k0, kb, lane);
      p.W0.e[5] = halo_hi<SPLIT, false>(p.W0, P1 + o_w0 - k0, k0, kb, KB, lane);
    }
    release(0, q0);
    SlotPos pc = q1, pn = q1;
    pn.next(NB);
    const size_t plane_elems = (size_t)ny * nz;
    const size_t o_row = (size_t)j * nz + k0;

    for (int i = t.i_lo; i < t.i_hi; ++i) {
      const int qc = i - t.i_lo + 1;
      wait(pn);
      if (__any_sync(0xffffffffu, timed_out)) break;
      const __half* Pc = slot_ptr(pc);
      const __half* Pn = slot_ptr(pn);
      ld8(Pn + o_u0, p.UXP);
      ld8(Pc + o_um, p.UYM);
      ld8(Pc + o_up, p.UYP);
      ld8(Pn + o_v0, p.VXP);
      ld8(Pc + o_vp, p.VYP);
      ld8(Pn + o_vm, p.VXPYM);
      ld8(Pn + o_w0, p.WXP);
      ld8(Pc + o_wm, p.WYM);
      ld8(Pc + o_wp, p.WYP);
      // halos plane i reads of the new vectors, and those carried to plane i+1
      p.WXP.e[0] = halo_lo<SPLIT>(p.WXP, Pn + o_w0 - k0, k0, kb, lane);
      p.WYP.e[0] = halo_lo<SPLIT>(p.WYP, Pc + o_wp - k0, k0, kb, lane);
      p.UXP.e[0] = halo_lo<SPLIT>(p.UXP, Pn + o_u0 - k0, k0, kb, lane);
      p.UXP.e[5] = halo_hi<SPLIT, true>(p.UXP, Pn + o_u0 - k0, k0, kb, KB, lane);
      p.VXP.e[0] = halo_lo<SPLIT>(p.VXP, Pn + o_v0 - k0, k0, kb, lane);
      p.VXP.e[5] = halo_hi<SPLIT, true>(p.VXP, Pn + o_v0 - k0, k0, kb, KB, lane);
      p.VXPYM.e[5] = halo_hi<SPLIT, false>(p.VXPYM, Pn + o_vm - k0, k0, kb, KB, lane);
      p.WXP.e[5] = halo_hi<SPLIT, false>(p.WXP, Pn + o_w0 - k0, k0, kb, KB, lane);
      release(qc, pc);
      pc = pn;
      pn.next(NB);

      uint32_t su[4], sv[4], sw[4];
      level_pair<0>(p, K, su[0], sv[0], sw[0]);
      level_pair<2>(p, K, su[1], sv[1], sw[1]);
      level_pair<4>(p, K, su[2], sv[2], sw[2]);
      level_pair<6>(p, K, su[3], sv[3], sw[3]);
      su[0] &= keep_first;
      sv[0] &= keep_first;
      sw[0] &= keep_first;
      sw[3] &= keep_last;
      if (row_ok) {
        const size_t o = (size_t)i * plane_elems + o_row;
        __stcs(reinterpret_cast<uint4*>(t.o[0] + o), make_uint4(su[0], su[1], su[2], su[3]));
        __stcs(reinterpret_cast<uint4*>(t.o[1] + o), make_uint4(sv[0], sv[1], sv[2], sv[3]));
        __stcs(reinterpret_cast<uint4*>(t.o[2] + o), make_uint4(sw[0], sw[1], sw[2], sw[3]));
      }
      // roll to plane i+1 (with the halos each vector carries)
      p.UXM.e[5] = p.U0.e[5];
      copy_levels(p.UXM, p.U0);
      p.U0 = p.UXP;
      copy_levels(p.UXMYP, p.UYP);
      copy_levels(p.VXM, p.V0);
      p.V0 = p.VXP;
      p.VYM.e[5] = p.VXPYM.e[5];
      copy_levels(p.VYM, p.VXPYM);
      copy_levels(p.WXM, p.W0);
      p.W0.e[0] = p.WXP.e[0];
      p.W0.e[5] = p.WXP.e[5];
      copy_levels(p.W0, p.WXP);
    }
    ok = !timed_out;
  }
  return finish_tile(R, ok);
}

}  // namespace sweep
}  // namespace advect
