// sweep_ff.cuh -- plane-sweep tile of the forward for binary64 storage with
// double-float arithmetic (ADVECT_F64_FF), columns whose rows fit in a warp.
//
// Same ring of bulk-copied slabs and bounded waits as the generic sweep
// (sweep_core.cuh).  What differs:
//
//  * A converter warp (the CTA's last) splits every landed slab once, in
//    place: each pair of binary64 values (levels k, k+1, k even) becomes the
//    16 bytes (hi_k, hi_k+1, lo_k, lo_k+1) of binary32 numbers (ff.cuh's
//    split), and the warp then arrives on the slot's conversion mbarrier.
//    The compute warps wait on that barrier instead of the copy's, so a
//    binary64 value is split once per CTA rather than by each of the (up to
//    three) threads that read it, and the compute warps keep drifting within
//    the ring independently of each other (the converter runs ahead).
//  * A compute thread owns the levels (k0, k0+1) of one column, and the
//    double-float arithmetic of both levels runs in two-wide binary32
//    instructions (__fadd2_rn, __fmul2_rn, __ffma2_rn: one instruction for
//    both levels), on register pairs laid out as the converted slab is.
//  * Registers, not shared-memory bandwidth, limit the sweep: no vector is
//    carried across planes (plane i-1's slot stays resident until plane i is
//    done), every vector is re-read from shared memory by the source term
//    that uses it (volatile loads, which the compiler cannot merge), and the
//    split constants (vertical coefficients, tcx, tcy) sit in a shared table.
//    Only the three x-face sums a plane shares with the next (u(i) + u(i+1),
//    u + u(y+1), u + u(z+1) of plane i are plane i+1's x-1 faces) are carried.
//    That fits the code in 128 registers without spills, so two CTAs of
//    seven compute warps and the converter run per SM.
//  * The three source terms are evaluated side by side, stage by stage (x
//    faces of su, sv, sw, then their y faces, then the vertical faces): the
//    double-float chains of one term depend on each other, the three terms
//    do not, so each warp has three independent chains in flight.
//
// Double-float sums are TwoSum of the high parts with the low parts added,
// products the exact product of the high parts (FMA) plus the two cross
// terms, as in ff.cuh (no renormalisation until the result is assembled into
// a binary64 value).  Levels below and above the column: the halo below is
// read only by level 0, whose three outputs are written as zero, and the
// halo above only by level nz-1, where sw is written as zero and su, sv
// multiply it by tzc2(nz-1) = 0, so only the u and v halos above are zeroed.
#pragma once

#include "sweep_core.cuh"

namespace advect {
namespace sweep {
namespace ffx {

constexpr int P = 2;

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b, rounded once
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// Two levels of double-float values: level k in (hi.x, lo.x), k+1 in (hi.y, lo.y).
struct FF2 {
  float2 hi, lo;
};

// one level: hi + lo
struct F1 {
  float hi, lo;
};

__device__ __forceinline__ FF2 add(const FF2& a, const FF2& b) {
  const float2 s = add2(a.hi, b.hi);
  const float2 bb = sub2(s, a.hi);
  const float2 e = add2(sub2(a.hi, sub2(s, bb)), sub2(b.hi, bb));
  return FF2{s, add2(e, add2(a.lo, b.lo))};
}

// a - b: TwoSum of a.hi and -b.hi (b.hi + bb is exactly -(-b.hi - bb))
__device__ __forceinline__ FF2 sub(const FF2& a, const FF2& b) {
  const float2 s = sub2(a.hi, b.hi);
  const float2 bb = sub2(s, a.hi);
  const float2 e = sub2(sub2(a.hi, sub2(s, bb)), add2(b.hi, bb));
  return FF2{s, add2(e, sub2(a.lo, b.lo))};
}

__device__ __forceinline__ FF2 mul(const FF2& a, const FF2& b) {
  const float2 p = mul2(a.hi, b.hi);
  float2 e = fma2(a.hi, b.hi, make_float2(-p.x, -p.y));  // exact error of p (negation folded into the FMA)
  e = fma2(a.hi, b.lo, e);
  e = fma2(a.lo, b.hi, e);
  return FF2{p, e};
}

// The pair shifted down one level: (level k0-1 from below, level k0).
__device__ __forceinline__ FF2 zm(const FF2& v, const F1& below) {
  return FF2{make_float2(below.hi, v.hi.x), make_float2(below.lo, v.lo.x)};
}
// The pair shifted up one level: (level k0+1, level k0+2 from above).
__device__ __forceinline__ FF2 zp(const FF2& v, const F1& above) {
  return FF2{make_float2(v.hi.y, above.hi), make_float2(v.lo.y, above.lo)};
}

// Vertical halos from the neighbouring lanes (rows do not straddle warps).
__device__ __forceinline__ F1 below(const FF2& v) {
  return F1{__shfl_up_sync(0xffffffffu, v.hi.y, 1), __shfl_up_sync(0xffffffffu, v.lo.y, 1)};
}
template <bool ZERO>
__device__ __forceinline__ F1 above(const FF2& v, bool top) {
  F1 r{__shfl_down_sync(0xffffffffu, v.hi.x, 1), __shfl_down_sync(0xffffffffu, v.lo.x, 1)};
  if (ZERO && top) r = F1{0.f, 0.f};
  return r;
}

__device__ __forceinline__ float4 lds128(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
  return v;
}
// A raw slab pair of binary64 values and a converted 16-byte vector, by
// shared address (the converter warps' in-place split).
__device__ __forceinline__ double2 lds_f64x2(uint32_t a) {
  double2 v;
  asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void sts128(uint32_t a, float4 v) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
               : "memory");
}

// A converted slab vector or table entry (16 bytes: hi_k, hi_k+1, lo_k,
// lo_k+1) at shared address a.  The load is volatile: the compiler re-reads
// a vector where it is used instead of holding it across the three source
// terms (registers, not shared-memory bandwidth, limit the sweep).
__device__ __forceinline__ FF2 ldc(uint32_t a) {
  const float4 v = lds128(a);
  return FF2{make_float2(v.x, v.y), make_float2(v.z, v.w)};
}

// A level pair of a per-level binary64 table, split.
__device__ __forceinline__ FF2 coef2(const double* tab, int k) {
  const ff a(__ldg(tab + k)), b(__ldg(tab + k + 1));
  return FF2{make_float2(a.hi, b.hi), make_float2(a.lo, b.lo)};
}

__device__ __forceinline__ FF2 bcast(const ff& x) { return FF2{make_float2(x.hi, x.hi), make_float2(x.lo, x.lo)}; }

// A binary32 value as binary64 by integer bit operations (exact for normal
// values: the exponent rebiased from 127 to 1023, the significand shifted
// into place); a signed zero stays exact, binary32 subnormals (below 2^-126)
// come out below 2^-1000; infinities and NaN lie outside the double-float
// mode's range (as for the split).
__device__ __forceinline__ double widen(float x) {
  const uint32_t b = __float_as_uint(x);
  const uint32_t mag = b & 0x7fffffffu;
  const uint32_t bias = mag >= 0x00800000u ? 0x38000000u : 0u;
  return __hiloint2double((int)(((mag >> 3) + bias) | (b & 0x80000000u)), (int)(b << 29));
}

// (hi, lo) of one level -> binary64, rounded once: both parts widened by
// integer operations, then one binary64 add (the conversion instructions of
// the binary64 pipe cost as much there as the add: measured 52.0 against
// 51.5 Gpts/s with the high part converted on that pipe, 47.8 with both).
__device__ __forceinline__ double assemble(float hi, float lo) { return widen(hi) + widen(lo); }

}  // namespace ffx

// Converter warps per CTA (after the compute warps).
constexpr int kConverters = 1;

// Threads a CTA of the converter-warp sweep may have at a given number of
// CTAs per SM (the register file is split between the SM's four schedulers:
// 5 warps x 3 CTAs and 8 warps x 2 CTAs both leave 128 registers a thread).
__host__ __device__ constexpr int ff_max_threads(int occ) { return occ >= 3 ? 160 : 256; }

// Shared-memory bytes after the ring: the split constants (the four vertical
// coefficient tables as level pairs, rows [c1 | c2 | d1 | d2] of nz / 2
// entries, then tcx and tcy broadcast to both levels; 16 bytes an entry) and
// the conversion mbarriers.
__host__ __device__ inline size_t ff_const_bytes(int nz) { return (size_t)(2 * nz + 2) * 16; }
__host__ __device__ inline size_t ff_extra_bytes(int nb, int nz) {
  return ff_const_bytes(nz) + (size_t)nb * sizeof(uint64_t);
}

// Sweep one double-float tile with blockDim.x = t.ty * t.kb + 32 kConverters
// threads: the compute warps first, the converter warps last.  t.kb = nz / 2
// divides 32.
__device__ inline bool forward_tile_ff(const Tile<f64ff>& t, const Ring& R, int* flag) {
  using namespace ffx;
  const int NB = R.nb;
  const int tid = threadIdx.x, lane = tid & 31;
  const int nz = t.nz, ty = t.ty, ny = t.ny;
  const int KB = nz / P;
  const int compute_threads = ty * KB;  // a multiple of 32
  const int nwarps = compute_threads >> 5;
  const int nplanes = t.i_hi - t.i_lo + 2;
  const int rows = ty + 2;
  const uint32_t cap = (uint32_t)R.slot_cap;  // slot stride
  const uint32_t ring = (uint32_t)__cvta_generic_to_shared(R.slots);
  float4* ctab = reinterpret_cast<float4*>(R.slots + ring_bytes(R.nb, R.slot_cap));
  uint64_t* conv = reinterpret_cast<uint64_t*>(ctab + 2 * nz + 2);
  if (tid == 0)  // made visible by start_tile's fence and barrier
    for (int s = 0; s < NB; ++s) mbar_init(&conv[s], kConverters);
  // the split constants (visible after start_tile's barrier)
  for (int e = tid; e < 2 * nz + 2; e += blockDim.x) {
    FF2 c;
    if (e < 4 * KB) {
      const int m = e / KB, kp = e - m * KB;
      const int tab = m == 0 ? TZC1 : m == 1 ? TZC2 : m == 2 ? TZD1 : TZD2;
      c = coef2(t.c.d + tab * nz, 2 * kp);
    } else {
      c = bcast(ff(e == 4 * KB ? t.c.tcx : t.c.tcy));
    }
    ctab[e] = make_float4(c.hi.x, c.hi.y, c.lo.x, c.lo.y);
  }
  start_tile<3>(t, R, nplanes);
  int timed_out = 0;
  if (tid >= compute_threads) {
    // converter warps: split each slab in place, in plane order; each of the
    // kConverters warps takes every kConverters-th pair and arrives on the
    // slot's conversion barrier (expected arrivals: kConverters)
    const int pairs = 3 * rows * nz / 2;
    const int cw = (tid - compute_threads) >> 5;  // converter warp index
    const int stride = 32 * kConverters;
    SlotPos q{0, 0};
    for (int ql = 0; ql < nplanes; ++ql) {
      if (!mbar_wait_bounded(&R.full[q.slot], (uint32_t)(q.use & 1), t.wait_budget)) {
        atomicExch(flag, 1);
        timed_out = 1;
      }
      if (__any_sync(0xffffffffu, timed_out)) break;
      const uint32_t sb = ring + (uint32_t)q.slot * cap;
      int e = cw * 32 + lane;
      // four pairs at a time: loads first, then the splits, then the stores
      for (; e + 3 * stride < pairs; e += 4 * stride) {
        double2 d[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) d[u] = lds_f64x2(sb + (uint32_t)(e + u * stride) * 16u);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const ff a(d[u].x), b(d[u].y);
          sts128(sb + (uint32_t)(e + u * stride) * 16u, make_float4(a.hi, b.hi, a.lo, b.lo));
        }
      }
      for (; e < pairs; e += stride) {
        const double2 d = lds_f64x2(sb + (uint32_t)e * 16u);
        const ff a(d.x), b(d.y);
        sts128(sb + (uint32_t)e * 16u, make_float4(a.hi, b.hi, a.lo, b.lo));
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&conv[q.slot]);
      q.next(NB);
    }
  } else {
    const int kb = tid % KB, rr = tid / KB;
    const int k0 = kb * P;
    const int j = t.j0 + rr;
    const bool row_ok = j < ny;
    const bool top = kb == KB - 1;
    const bool bottom = kb == 0;
    const int r = rr + 1;
    // byte offsets in a slab: this thread's u vector, one row, one field
    const uint32_t o_u0 = (uint32_t)(r * nz + k0) * 8u, o_row8 = (uint32_t)nz * 8u;
    const uint32_t o_fld = (uint32_t)rows * o_row8;
    auto wait = [&](SlotPos q) {
      if (!mbar_wait_bounded(&conv[q.slot], (uint32_t)(q.use & 1), t.wait_budget)) {
        atomicExch(flag, 1);
        timed_out = 1;
      }
    };
    auto release = [&](int ql, SlotPos q) { release_plane<3>(t, R, ql, q, nplanes, nwarps, lane); };
    // shared addresses of this thread's constants
    const uint32_t a_c1 = (uint32_t)__cvta_generic_to_shared(ctab + kb);
    const uint32_t a_tc = (uint32_t)__cvta_generic_to_shared(ctab + 4 * KB);
    const size_t plane_elems = (size_t)ny * nz;
    const size_t o_row = (size_t)j * nz + k0;

    // slots of planes i-1, i, i+1; every vector is read from shared memory
    // where it is used
    SlotPos pm{0, 0}, pc{0, 0}, pn{0, 0};
    pc.next(NB);
    pn = pc;
    pn.next(NB);
    wait(pm);
    wait(pc);
    // x faces of plane i-1 (i - 1/2), carried from the previous plane:
    // u(i-1) + u(i), u(i-1) + u(i-1, y+1), u(i-1) + u(i-1, z+1)
    FF2 FU, FV, FW;
    {
      const uint32_t Pm = ring + (uint32_t)pm.slot * cap + o_u0;
      const uint32_t Pc = ring + (uint32_t)pc.slot * cap + o_u0;
      const FF2 UM = ldc(Pm);
      FU = add(UM, ldc(Pc));
      FV = add(UM, ldc(Pm + o_row8));
      FW = add(UM, zp(UM, above<true>(UM, top)));
    }
    for (int i = t.i_lo; i < t.i_hi; ++i) {
      wait(pn);
      if (__any_sync(0xffffffffu, timed_out)) break;
      // this thread's u vector in the slabs of planes i-1, i, i+1
      const uint32_t Pm = ring + (uint32_t)pm.slot * cap + o_u0;
      const uint32_t Pc = ring + (uint32_t)pc.slot * cap + o_u0;
      const uint32_t Pn = ring + (uint32_t)pn.slot * cap + o_u0;
      const uint32_t o_um = 0u - o_row8, o_up = o_row8, o_v0 = o_fld, o_vm = o_fld - o_row8, o_vp = o_fld + o_row8;
      const uint32_t o_w0 = 2u * o_fld, o_wm = 2u * o_fld - o_row8, o_wp = 2u * o_fld + o_row8;
      const size_t o = (size_t)i * plane_elems + o_row;
      // su, sv, sw (Listing 1 and its v, w counterparts) stage by stage
      FF2 hu, hv, hw;
      {
        // x faces
        const FF2 U0 = ldc(Pc);
        const FF2 fu = add(U0, ldc(Pn));
        const FF2 fv = add(U0, ldc(Pc + o_up));
        const FF2 fw = add(U0, zp(U0, above<true>(U0, top)));
        const FF2 xu = sub(mul(ldc(Pm), FU), mul(ldc(Pn), fu));
        const FF2 xv = sub(mul(ldc(Pm + o_v0), FV), mul(ldc(Pn + o_v0), fv));
        const FF2 xw = sub(mul(ldc(Pm + o_w0), FW), mul(ldc(Pn + o_w0), fw));
        FU = fu;
        FV = fv;
        FW = fw;
        const FF2 tcx = ldc(a_tc);
        hu = mul(tcx, xu);
        hv = mul(tcx, xv);
        hw = mul(tcx, xw);
      }
      {
        // y faces
        const FF2 V0 = ldc(Pc + o_v0), VYM = ldc(Pc + o_vm);
        const FF2 yu = sub(mul(ldc(Pc + o_um), add(VYM, ldc(Pn + o_vm))), mul(ldc(Pc + o_up), add(V0, ldc(Pn + o_v0))));
        const FF2 VYP = ldc(Pc + o_vp);
        const FF2 yv = sub(mul(VYM, add(V0, VYM)), mul(VYP, add(V0, VYP)));
        const FF2 yw = sub(mul(ldc(Pc + o_wm), add(VYM, zp(VYM, above<false>(VYM, top)))),
                           mul(ldc(Pc + o_wp), add(V0, zp(V0, above<true>(V0, top)))));
        const FF2 tcy = ldc(a_tc + 16);
        hu = add(hu, mul(tcy, yu));
        hv = add(hv, mul(tcy, yv));
        hw = add(hw, mul(tcy, yw));
      }
      {
        // vertical faces: the lower face of level k is the upper face of
        // level k-1 (the lane below holds it for the first level)
        const FF2 W0 = ldc(Pc + o_w0);
        const FF2 U0 = ldc(Pc), V0 = ldc(Pc + o_v0);
        const FF2 wu_hi = add(W0, ldc(Pn + o_w0));
        const FF2 wv_hi = add(W0, ldc(Pc + o_wp));
        const FF2 wzp = zp(W0, above<false>(W0, top));
        const FF2 ww_hi = add(W0, wzp);
        const FF2 wu_lo = zm(wu_hi, below(wu_hi)), wv_lo = zm(wv_hi, below(wv_hi)), ww_lo = zm(ww_hi, below(ww_hi));
        const FF2 c1 = ldc(a_c1), c2 = ldc(a_c1 + 16 * KB);
        hu = add(hu, mul(mul(c1, zm(U0, below(U0))), wu_lo));
        hv = add(hv, mul(mul(c1, zm(V0, below(V0))), wv_lo));
        hw = add(hw, mul(mul(ldc(a_c1 + 32 * KB), zm(W0, below(W0))), ww_lo));
        hu = sub(hu, mul(mul(c2, zp(U0, above<true>(U0, top))), wu_hi));
        hv = sub(hv, mul(mul(c2, zp(V0, above<true>(V0, top))), wv_hi));
        hw = sub(hw, mul(mul(ldc(a_c1 + 48 * KB), wzp), ww_hi));
      }
      if (row_ok) {
        // su, sv at level 0 and sw at levels 0 and nz-1 are zero
        const double u0 = bottom ? 0.0 : assemble(hu.hi.x, hu.lo.x), u1 = assemble(hu.hi.y, hu.lo.y);
        const double v0 = bottom ? 0.0 : assemble(hv.hi.x, hv.lo.x), v1 = assemble(hv.hi.y, hv.lo.y);
        const double w0 = bottom ? 0.0 : assemble(hw.hi.x, hw.lo.x);
        const double w1 = top ? 0.0 : assemble(hw.hi.y, hw.lo.y);
        __stcs(reinterpret_cast<double2*>(t.o[0]) + o / 2, make_double2(u0, u1));
        __stcs(reinterpret_cast<double2*>(t.o[1]) + o / 2, make_double2(v0, v1));
        __stcs(reinterpret_cast<double2*>(t.o[2]) + o / 2, make_double2(w0, w1));
      }
      // plane i-1 is no longer read by this warp
      release(i - t.i_lo, pm);
      pm = pc;
      pc = pn;
      pn.next(NB);
    }
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
