// sweep_core.cuh -- the plane-sweep machinery shared by the single-grid and
// ensemble forward kernels.
//
// A tile is TY rows (j0 .. j0+TY-1) of one grid over the x-planes
// [i_lo, i_hi).  For each plane the CTA needs the (TY+2)-row slab
// j0-1 .. j0+TY of u, v and w, which in the [nx][ny][nz] layout is one
// contiguous run per field (three runs where the periodic wrap in y splits
// it).  The slabs stream through a ring of NB shared-memory slots filled by
// cp.async.bulk (the TMA engine) with one mbarrier per slot counting the
// bytes.  There is no CTA-wide barrier per plane: each warp, when done with a
// slot, bumps that slot's arrival counter, and the last warp to arrive issues
// the copy of the plane NB ahead into it.  So warps drift within the ring and
// overlap each other's latencies.
//
// Thread (row rr, k-block kb) owns P consecutive levels of one column for the
// whole tile.  The own-row values of planes i-1 and i, the off-row values
// reused one plane later, and (for 8-byte arithmetic; binary32 recomputes
// them) the face sums shared between consecutive planes stay in registers;
// vertical neighbours come from the adjacent lanes by shuffle.  Each plane
// then costs nine vector loads from shared memory per thread.  Per point the
// arithmetic and its order follow Listing 1 (Sec. 2.1) for su and the same
// pattern for sv and sw; the lid branch comes from tzc2[nz-1] == 0 and zero
// values above the top level.
#pragma once

#include <type_traits>

#include "bulk.cuh"
#include "kernels.h"

namespace advect {
namespace sweep {

template <typename T>
struct VecIO;

template <>
struct VecIO<double> {
  static constexpr int P = 2;
  using C = double;
  __device__ static __forceinline__ void ld(const double* s, float, C (&o)[P]) {
    const double2 x = *reinterpret_cast<const double2*>(s);
    o[0] = x.x;
    o[1] = x.y;
  }
  __device__ static __forceinline__ C ld1(const double* s, float) { return *s; }
  __device__ static __forceinline__ void gld(const double* g, float, C (&o)[P]) {
    const double2 x = __ldcs(reinterpret_cast<const double2*>(g));
    o[0] = x.x;
    o[1] = x.y;
  }
  __device__ static __forceinline__ void st(double* g, const C (&v)[P], float) {
    __stcs(reinterpret_cast<double2*>(g), make_double2(v[0], v[1]));
  }
};

template <>
struct VecIO<float> {
  static constexpr int P = 4;
  using C = float;
  __device__ static __forceinline__ void ld(const float* s, float, C (&o)[P]) {
    const float4 x = *reinterpret_cast<const float4*>(s);
    o[0] = x.x;
    o[1] = x.y;
    o[2] = x.z;
    o[3] = x.w;
  }
  __device__ static __forceinline__ C ld1(const float* s, float) { return *s; }
  __device__ static __forceinline__ void gld(const float* g, float, C (&o)[P]) {
    const float4 x = __ldcs(reinterpret_cast<const float4*>(g));
    o[0] = x.x;
    o[1] = x.y;
    o[2] = x.z;
    o[3] = x.w;
  }
  __device__ static __forceinline__ void st(float* g, const C (&v)[P], float) {
    __stcs(reinterpret_cast<float4*>(g), make_float4(v[0], v[1], v[2], v[3]));
  }
};

template <>
struct VecIO<__half> {
  static constexpr int P = 4;
  using C = float;
  __device__ static __forceinline__ void ld(const __half* s, float sc, C (&o)[P]) {
    const uint2 x = *reinterpret_cast<const uint2*>(s);
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&x.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&x.y));
    o[0] = a.x * sc;
    o[1] = a.y * sc;
    o[2] = b.x * sc;
    o[3] = b.y * sc;
  }
  __device__ static __forceinline__ C ld1(const __half* s, float sc) { return __half2float(*s) * sc; }
  __device__ static __forceinline__ void gld(const __half* g, float sc, C (&o)[P]) {
    const uint2 x = __ldcs(reinterpret_cast<const uint2*>(g));
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&x.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&x.y));
    o[0] = a.x * sc;
    o[1] = a.y * sc;
    o[2] = b.x * sc;
    o[3] = b.y * sc;
  }
  __device__ static __forceinline__ void st(__half* g, const C (&v)[P], float inv) {
    const __half2 a = __floats2half2_rn(v[0] * inv, v[1] * inv);
    const __half2 b = __floats2half2_rn(v[2] * inv, v[3] * inv);
    uint2 x;
    x.x = *reinterpret_cast<const uint32_t*>(&a);
    x.y = *reinterpret_cast<const uint32_t*>(&b);
    __stcs(reinterpret_cast<uint2*>(g), x);
  }
};

template <>
struct VecIO<f64ff> {
  static constexpr int P = 2;
  using C = ff;
  __device__ static __forceinline__ void ld(const f64ff* s, float, C (&o)[P]) {
    const double2 x = *reinterpret_cast<const double2*>(s);
    o[0] = ff(x.x);
    o[1] = ff(x.y);
  }
  __device__ static __forceinline__ C ld1(const f64ff* s, float) { return ff(s->v); }
  __device__ static __forceinline__ void gld(const f64ff* g, float, C (&o)[P]) {
    const double2 x = __ldcs(reinterpret_cast<const double2*>(g));
    o[0] = ff(x.x);
    o[1] = ff(x.y);
  }
  __device__ static __forceinline__ void st(f64ff* g, const C (&v)[P], float) {
    __stcs(reinterpret_cast<double2*>(g), make_double2(to_double_fp64(v[0]), to_double_fp64(v[1])));
  }
};

// The integration step dt in each arithmetic type.
__device__ __forceinline__ double step_of(double, double dt, float, float) { return dt; }
__device__ __forceinline__ float step_of(float, double, float hi, float) { return hi; }
__device__ __forceinline__ ff step_of(const ff&, double, float hi, float lo) { return ff(hi, lo); }

// Warp shuffles for every arithmetic type.
__device__ __forceinline__ float shfl_up_c(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_up_c(double v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ ff shfl_up_c(const ff& v) { return shfl_up(v, 1); }
__device__ __forceinline__ float shfl_down_c(float v) { return __shfl_down_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_down_c(double v) { return __shfl_down_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ ff shfl_down_c(const ff& v) { return shfl_down(v, 1); }

// Shared-memory ring: NB slots of slot_cap bytes, then NB mbarriers, then NB
// arrival counters and NB issue counters.
struct Ring {
  unsigned char* slots;
  uint64_t* full;
  int* arrived;  // warps done with the slot, cumulative over the tile
  int* issued;   // copies issued into the slot during the tile
  int nb;
  size_t slot_cap;
};

__host__ __device__ inline size_t ring_bytes(int nb, size_t slot_cap) {
  return (size_t)nb * slot_cap + (size_t)nb * sizeof(uint64_t) + 2 * (size_t)nb * sizeof(int);
}

__device__ inline Ring make_ring(unsigned char* smem, int nb, size_t slot_cap) {
  Ring r;
  r.slots = smem;
  r.full = reinterpret_cast<uint64_t*>(smem + (size_t)nb * slot_cap);
  r.arrived = reinterpret_cast<int*>(smem + (size_t)nb * slot_cap + (size_t)nb * sizeof(uint64_t));
  r.issued = r.arrived + nb;
  r.nb = nb;
  r.slot_cap = slot_cap;
  return r;
}

// One tile of one grid.
template <typename T>
struct Tile {
  const T* f[6];  // inputs: u, v, w (forward); u, v, w, dsu, dsv, dsw (adjoint)
  T* o[3];        // outputs: su, sv, sw or du, dv, dw
  int nf;         // number of input fields streamed per plane
  int nx, ny, nz;
  int j0, ty, kb;  // first row, rows per tile, k-blocks per row (nz / P)
  int i_lo, i_hi;  // x-planes computed
  Coeffs c;
  Scales sc;
  int f64_levels;
  long long wait_budget = kWaitBudgetCycles;  // clock64 cycles per bounded wait
  int skip_plane = -1;  // test-only fault injection: this plane's copy is never issued
  // Integration epilogue (forward_tile<..., INTEG = true> only): outputs
  // base + dt * source term, base = b[f], or the winds where b[f] is NULL.
  int integ = 0;
  const T* b[3] = {nullptr, nullptr, nullptr};
  double dt = 0.0;
  float dt_hi = 0.f, dt_lo = 0.f;
};

// Integration epilogue of one field: s = base + dt * s, the base read with a
// streaming global load (each element by the one thread that overwrites the
// output there, so the output may be the base itself) or taken from x, the
// thread's own wind values.
template <typename T, typename C, int P>
__device__ __forceinline__ void add_step(const T* base, size_t o, float scale, const C (&x)[P], C dt, C (&s)[P]) {
  C b[P];
  if (base) {
    VecIO<T>::gld(base + o, scale, b);
  } else {
#pragma unroll
    for (int q = 0; q < P; ++q) b[q] = x[q];
  }
#pragma unroll
  for (int q = 0; q < P; ++q) s[q] = b[q] + dt * s[q];
}

// Pull one base vector of the integration step into L2 ahead of its load
// (addresses inside the base field only; no registers held).
template <typename T, int P>
__device__ __forceinline__ void prefetch_base(const T* base, size_t o) {
  if (base) asm volatile("prefetch.global.L2 [%0];" ::"l"(base + o));
}

// Bulk-copy plane ql of the tile (x index i_lo-1+ql, periodic) into its slot;
// NF fields (t.nf == NF).
template <int NF, typename T>
__device__ __forceinline__ void issue_plane(const Tile<T>& t, const Ring& R, int ql, int slot) {
  int ig = t.i_lo - 1 + ql;
  ig = ig < 0 ? ig + t.nx : (ig >= t.nx ? ig - t.nx : ig);
  const int ty_eff = min(t.ty, t.ny - t.j0);
  const int rows = t.ty + 2;
  const uint32_t row_bytes = (uint32_t)(t.nz * sizeof(T));
  if (ql == t.skip_plane) return;  // injected fault: waits on this plane must run out
  uint64_t* bar = &R.full[slot];
  R.issued[slot] += 1;  // one issuer per slot at a time
  mbar_arrive_expect_tx(bar, (uint32_t)NF * (uint32_t)(ty_eff + 2) * row_bytes);
  T* dst0 = reinterpret_cast<T*>(R.slots + (size_t)slot * R.slot_cap);
  const int j0 = t.j0;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const T* plane = t.f[f] + (size_t)ig * t.ny * t.nz;
    T* dst = dst0 + (size_t)f * rows * t.nz;
    if (j0 >= 1 && j0 + ty_eff <= t.ny - 1) {
      bulk_copy_g2s(dst, plane + (size_t)(j0 - 1) * t.nz, (uint32_t)(ty_eff + 2) * row_bytes, bar);
    } else {
      const int jt = j0 == 0 ? t.ny - 1 : j0 - 1;
      const int jb = j0 + ty_eff == t.ny ? 0 : j0 + ty_eff;
      bulk_copy_g2s(dst, plane + (size_t)jt * t.nz, row_bytes, bar);
      bulk_copy_g2s(dst + t.nz, plane + (size_t)j0 * t.nz, (uint32_t)ty_eff * row_bytes, bar);
      bulk_copy_g2s(dst + (size_t)(ty_eff + 1) * t.nz, plane + (size_t)jb * t.nz, row_bytes, bar);
    }
  }
}

// Fresh barriers and counters for a tile, then the first NB copies.  The
// caller guarantees the ring is idle.
template <int NF, typename T>
__device__ __forceinline__ void start_tile(const Tile<T>& t, const Ring& R, int nplanes) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int s = 0; s < R.nb; ++s) {
      mbar_init(&R.full[s], 1);
      R.arrived[s] = 0;
      R.issued[s] = 0;
    }
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    for (int q = 0; q < R.nb && q < nplanes; ++q) issue_plane<NF>(t, R, q, q);
  }
}

// End of a tile: all warps are done; after a timeout, wait (bounded) for the
// last copy issued into each slot; then invalidate the barriers so the ring
// can be re-initialised.  Returns true if no thread reported a timeout.
__device__ __forceinline__ bool finish_tile(const Ring& R, bool ok) {
  const int any_fail = __syncthreads_or(!ok);
  if (threadIdx.x == 0) {
    for (int s = 0; s < R.nb; ++s) {
      const int n = R.issued[s];  // the copy of phase n-1 is the only one that can be pending
      if (any_fail) {
        if (n > 0) mbar_wait_bounded(&R.full[s], (uint32_t)((n - 1) & 1), 1 << 20);
      } else {
        mbar_inval(&R.full[s]);  // the ring is re-initialised for the next tile
      }
    }
  }
  __syncthreads();
  return !any_fail;
}

// Wait for plane ql of the tile; false (and the error flag raised) if the
// bounded wait ran out.
// Plane ql of a tile sits in slot ql % NB and is that slot's (ql / NB)-th
// use; sweeps advance these incrementally (no division in the loop).
struct SlotPos {
  int slot, use;
  __device__ __forceinline__ void next(int nb) {
    if (++slot == nb) {
      slot = 0;
      ++use;
    }
  }
};

__device__ __forceinline__ bool wait_plane(const Ring& R, SlotPos p, int* flag, long long budget) {
  if (mbar_wait_bounded(&R.full[p.slot], (uint32_t)(p.use & 1), budget)) return true;
  atomicExch(flag, 1);
  return false;
}

// This warp is done reading plane ql (at position p); the last of the
// tile's nwarps warps to arrive issues the copy of plane ql + NB into it.
template <int NF, typename T>
__device__ __forceinline__ void release_plane(const Tile<T>& t, const Ring& R, int ql, SlotPos p, int nplanes,
                                              int nwarps, int lane) {
  __syncwarp();
  if (lane == 0) {
    __threadfence_block();
    const int prev = atomicAdd(&R.arrived[p.slot], 1);
    if (prev + 1 == (p.use + 1) * nwarps && ql + R.nb < nplanes) {
      __threadfence_block();
      fence_proxy_async_smem();
      issue_plane<NF>(t, R, ql + R.nb, p.slot);
    }
  }
}

// Vertical halo of a P-vector: the values just below (k0-1) and just above
// (k0+P) the thread's levels, taken from the neighbouring lanes of the same
// row; zero beyond the column; a shared-memory read where the row crosses a
// warp boundary (only when a row spans more than one warp).
// SPLIT (compile time): rows may straddle warps (32 is not a multiple of the
// k-blocks per row); only then is the shared-memory fallback compiled.
template <bool SPLIT, typename T, typename C, int P>
__device__ __forceinline__ C halo_below(const C (&a)[P], const T* row, int k0, int kb, int lane, float sc) {
  C below = shfl_up_c(a[P - 1]);
  if (SPLIT && lane == 0 && kb > 0) below = VecIO<T>::ld1(row + k0 - 1, sc);
  return kb == 0 ? C(0) : below;
}

template <bool SPLIT, typename T, typename C, int P>
__device__ __forceinline__ C halo_above(const C (&a)[P], const T* row, int k0, int kb, int KB, int lane,
                                        float sc) {
  C above = shfl_down_c(a[0]);
  if (SPLIT && lane == 31 && kb < KB - 1) above = VecIO<T>::ld1(row + k0 + P, sc);
  return kb == KB - 1 ? C(0) : above;
}

// Sweep one tile with the whole CTA.  The caller guarantees that the ring is
// idle (no copy in flight, no thread reading it) on entry; on exit every copy
// this call issued has completed or, after a timeout, been waited for with a
// bounded budget.  Returns false if any wait of this thread's warp timed out.
// F64Z: compile the binary64 near-surface branch (F32/F16S with
// f64_levels > 0); the default instantiation has no binary64 code at all.
// INTEG: compile the integration epilogue (t.integ must then be set); the
// plain forward has none of its code.
template <typename T, bool F64Z = false, bool SPLIT = true, bool INTEG = false>
__device__ bool forward_tile(const Tile<T>& t, const Ring& R, int* flag) {
  using IO = VecIO<T>;
  using C = typename IO::C;
  using S = Store<T>;
  constexpr int P = IO::P;
  const int NB = R.nb;
  const int tid = threadIdx.x, lane = tid & 31;
  const int KB = t.kb, nz = t.nz, ny = t.ny;
  const int active_threads = t.ty * KB;  // a multiple of 32
  const int nwarps = active_threads >> 5;
  const int nplanes = t.i_hi - t.i_lo + 2;  // planes i_lo-1 .. i_hi
  const int rows = t.ty + 2;

  start_tile<3>(t, R, nplanes);
  bool ok = true;
  if (tid < active_threads) {
    const int kb = tid % KB, rr = tid / KB;
    const int k0 = kb * P;
    const int j = t.j0 + rr;
    const bool row_ok = j < ny;
    // F16S: the input scales are powers of two, so they fold exactly into
    // the constants.  With raw (unscaled) values every product is u*u, u*v,
    // u*w, v*v, v*w or w*w scaled by the product of two field scales; taking
    // tcx' = tcx s_u / s_w and tcy' = tcy s_v / s_w makes each field's sum
    // the true one times 1 / (s_f s_w), which the output scale then absorbs.
    // Same rounding as scaling every loaded value, one multiply fewer per
    // value.  (Not with the binary64 near-surface terms or the integration
    // epilogue, which need true values.)
    constexpr bool kFold = std::is_same<T, __half>::value && !F64Z && !INTEG;
    float s_u = t.sc.in[0], s_v = t.sc.in[1], s_w = t.sc.in[2];
    float o_u = t.sc.inv_out[0], o_v = t.sc.inv_out[1], o_w = t.sc.inv_out[2];
    C tcx = S::tcx(t.c), tcy = S::tcy(t.c);
    if constexpr (kFold) {
      const float iw = 1.f / s_w;
      tcx = tcx * s_u * iw;
      tcy = tcy * s_v * iw;
      o_u = o_u * s_u * s_w;
      o_v = o_v * s_v * s_w;
      o_w = o_w * s_w * s_w;
      s_u = 1.f;
      s_v = 1.f;
      s_w = 1.f;
    }
    const int r = rr + 1;
    const int o_u0 = r * nz, o_um = (r - 1) * nz, o_up = (r + 1) * nz;
    const int o_v0 = (rows + r) * nz, o_vm = (rows + r - 1) * nz, o_vp = (rows + r + 1) * nz;
    const int o_w0 = (2 * rows + r) * nz, o_wm = (2 * rows + r - 1) * nz, o_wp = (2 * rows + r + 1) * nz;
    auto slot_ptr = [&](SlotPos q) -> const T* {
      return reinterpret_cast<const T*>(R.slots + (size_t)q.slot * R.slot_cap);
    };
    int timed_out = 0;
    auto wait = [&](SlotPos q) {
      if (!wait_plane(R, q, flag, t.wait_budget)) timed_out = 1;
    };
    auto release = [&](int ql, SlotPos q) { release_plane<3>(t, R, ql, q, nplanes, nwarps, lane); };
    const SlotPos q0{0, 0};
    SlotPos q1{0, 0};
    q1.next(NB);

    C c1[P], c2[P], d1[P], d2[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const int k = min(k0 + q, nz - 1);
      c1[q] = S::coef(t.c, TZC1, nz, k);
      c2[q] = S::coef(t.c, TZC2, nz, k);
      d1[q] = S::coef(t.c, TZD1, nz, k);
      d2[q] = S::coef(t.c, TZD2, nz, k);
    }

    // Face sums shared with the previous plane: rolled in registers where the
    // arithmetic is the bottleneck (binary64, double-float); recomputed (three
    // adds per point) for binary32 arithmetic, where the 3P registers they
    // would hold cost more than the adds.
    constexpr bool kRoll = sizeof(C) != 4;
    // 8-byte arithmetic (binary64, double-float): re-derive the vertical
    // halos of the current plane each plane instead of carrying them
    constexpr bool kRehalo = sizeof(C) == 8;
    constexpr int PS = kRoll ? P : 1;
    C UXM[P], U0[P], UXMYP[P], VXM[P], V0[P], VYM[P], WXM[P], W0[P];
    C SXm[PS], SVm[PS], SWm[PS];
    C u0m, u0p, uxmp, v0m, v0p, vymp, w0m, w0p;
    wait(q0);
    wait(q1);
    {
      const T* P0 = slot_ptr(q0);
      const T* P1 = slot_ptr(q1);
      IO::ld(P0 + o_u0 + k0, s_u, UXM);
      IO::ld(P1 + o_u0 + k0, s_u, U0);
      IO::ld(P0 + o_up + k0, s_u, UXMYP);
      IO::ld(P0 + o_v0 + k0, s_v, VXM);
      IO::ld(P1 + o_v0 + k0, s_v, V0);
      IO::ld(P1 + o_vm + k0, s_v, VYM);
      IO::ld(P0 + o_w0 + k0, s_w, WXM);
      IO::ld(P1 + o_w0 + k0, s_w, W0);
      u0m = halo_below<SPLIT, T, C, P>(U0, P1 + o_u0, k0, kb, lane, s_u);
      u0p = halo_above<SPLIT, T, C, P>(U0, P1 + o_u0, k0, kb, KB, lane, s_u);
      uxmp = halo_above<SPLIT, T, C, P>(UXM, P0 + o_u0, k0, kb, KB, lane, s_u);
      v0m = halo_below<SPLIT, T, C, P>(V0, P1 + o_v0, k0, kb, lane, s_v);
      v0p = halo_above<SPLIT, T, C, P>(V0, P1 + o_v0, k0, kb, KB, lane, s_v);
      vymp = halo_above<SPLIT, T, C, P>(VYM, P1 + o_vm, k0, kb, KB, lane, s_v);
      w0m = halo_below<SPLIT, T, C, P>(W0, P1 + o_w0, k0, kb, lane, s_w);
      w0p = halo_above<SPLIT, T, C, P>(W0, P1 + o_w0, k0, kb, KB, lane, s_w);
    }
    release(0, q0);
    SlotPos pc = q1, pn = q1;  // planes i and i+1
    pn.next(NB);
    if constexpr (kRoll) {
#pragma unroll
      for (int q = 0; q < P; ++q) {
        SXm[q] = UXM[q] + U0[q];
        SVm[q] = UXM[q] + UXMYP[q];
        SWm[q] = UXM[q] + (q < P - 1 ? UXM[q + 1] : uxmp);
      }
    }
    const bool f64z = sizeof(C) == 4 && t.f64_levels > 0 && k0 <= t.f64_levels;
    // integration: the base vectors of the next plane are pulled into L2 one
    // plane ahead of their streaming loads in the epilogue
    const size_t plane_elems = (size_t)ny * nz;
    const size_t o_row = (size_t)j * nz + k0;
    if constexpr (INTEG) {
      if (row_ok && t.i_lo < t.i_hi) {
        const size_t o = (size_t)t.i_lo * plane_elems + o_row;
        prefetch_base<T, P>(t.b[0], o);
        prefetch_base<T, P>(t.b[1], o);
        prefetch_base<T, P>(t.b[2], o);
      }
    }

    for (int i = t.i_lo; i < t.i_hi; ++i) {
      const int qc = i - t.i_lo + 1;  // plane i (plane i+1 is qc + 1)
      wait(pn);
      if (__any_sync(0xffffffffu, timed_out)) break;
      const T* Pc = slot_ptr(pc);
      const T* Pn = slot_ptr(pn);
      if constexpr (kRehalo) {
        // the vertical halos of plane i, from its registers (not carried
        // over from the previous plane: saves their registers)
        u0m = halo_below<SPLIT, T, C, P>(U0, Pc + o_u0, k0, kb, lane, s_u);
        u0p = halo_above<SPLIT, T, C, P>(U0, Pc + o_u0, k0, kb, KB, lane, s_u);
        v0m = halo_below<SPLIT, T, C, P>(V0, Pc + o_v0, k0, kb, lane, s_v);
        v0p = halo_above<SPLIT, T, C, P>(V0, Pc + o_v0, k0, kb, KB, lane, s_v);
        vymp = halo_above<SPLIT, T, C, P>(VYM, Pc + o_vm, k0, kb, KB, lane, s_v);
        w0m = halo_below<SPLIT, T, C, P>(W0, Pc + o_w0, k0, kb, lane, s_w);
        w0p = halo_above<SPLIT, T, C, P>(W0, Pc + o_w0, k0, kb, KB, lane, s_w);
      }
      if constexpr (INTEG) {
        if (row_ok && i + 1 < t.i_hi) {
          const size_t o = (size_t)(i + 1) * plane_elems + o_row;
          prefetch_base<T, P>(t.b[0], o);
          prefetch_base<T, P>(t.b[1], o);
          prefetch_base<T, P>(t.b[2], o);
        }
      }
      C UXP[P], UYM[P], UYP[P], VXP[P], VYP[P], VXPYM[P], WXP[P], WYM[P], WYP[P];
      IO::ld(Pn + o_u0 + k0, s_u, UXP);
      IO::ld(Pc + o_um + k0, s_u, UYM);
      IO::ld(Pc + o_up + k0, s_u, UYP);
      IO::ld(Pn + o_v0 + k0, s_v, VXP);
      IO::ld(Pc + o_vp + k0, s_v, VYP);
      IO::ld(Pn + o_vm + k0, s_v, VXPYM);
      IO::ld(Pn + o_w0 + k0, s_w, WXP);
      IO::ld(Pc + o_wm + k0, s_w, WYM);
      IO::ld(Pc + o_wp + k0, s_w, WYP);
      // halos that plane i reads of the loaded vectors, then (unless they are
      // re-derived next plane) the ones carried over to plane i+1
      const C wxpm = halo_below<SPLIT, T, C, P>(WXP, Pn + o_w0, k0, kb, lane, s_w);
      const C wypm = halo_below<SPLIT, T, C, P>(WYP, Pc + o_wp, k0, kb, lane, s_w);
      struct {
        C um, up, vm, vp, wp, vymp;
      } nx;
      if constexpr (!kRehalo) {
        nx.um = halo_below<SPLIT, T, C, P>(UXP, Pn + o_u0, k0, kb, lane, s_u);
        nx.up = halo_above<SPLIT, T, C, P>(UXP, Pn + o_u0, k0, kb, KB, lane, s_u);
        nx.vm = halo_below<SPLIT, T, C, P>(VXP, Pn + o_v0, k0, kb, lane, s_v);
        nx.vp = halo_above<SPLIT, T, C, P>(VXP, Pn + o_v0, k0, kb, KB, lane, s_v);
        nx.wp = halo_above<SPLIT, T, C, P>(WXP, Pn + o_w0, k0, kb, KB, lane, s_w);
        nx.vymp = halo_above<SPLIT, T, C, P>(VXPYM, Pn + o_vm, k0, kb, KB, lane, s_v);
      }
      // plane i is no longer read from shared memory by this warp
      release(qc, pc);
      pc = pn;
      pn.next(NB);

      C ou[P], ov[P], ow[P];
      C wu_lo = w0m + wxpm;   // w(i,k-1) + w(i+1,k-1): lower face of the u cell
      C wv_lo = w0m + wypm;   // w(i,j,k-1) + w(i,j+1,k-1): lower face of the v cell
      C ww_lo = W0[0] + w0m;  // w(k) + w(k-1): lower face of the w cell
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const C uzm = q > 0 ? U0[q - 1] : u0m;
        const C uzp = q < P - 1 ? U0[q + 1] : u0p;
        const C vzm = q > 0 ? V0[q - 1] : v0m;
        const C vzp = q < P - 1 ? V0[q + 1] : v0p;
        const C wzm = q > 0 ? W0[q - 1] : w0m;
        const C wzp = q < P - 1 ? W0[q + 1] : w0p;
        const C vym_zp = q < P - 1 ? VYM[q + 1] : vymp;
        C sxm, svm, swm;  // face sums at x = i (shared with plane i-1)
        if constexpr (kRoll) {
          sxm = SXm[q];
          svm = SVm[q];
          swm = SWm[q];
        } else {
          sxm = UXM[q] + U0[q];
          svm = UXM[q] + UXMYP[q];
          swm = UXM[q] + (q < P - 1 ? UXM[q + 1] : uxmp);
        }
        // su (Listing 1)
        const C sx = U0[q] + UXP[q];
        const C xu = UXM[q] * sxm - UXP[q] * sx;
        const C yu = UYM[q] * (VYM[q] + VXPYM[q]) - UYP[q] * (V0[q] + VXP[q]);
        const C wu_hi = W0[q] + WXP[q];
        // sv
        const C sv_x = U0[q] + UYP[q];
        const C xv = VXM[q] * svm - VXP[q] * sv_x;
        const C yv = VYM[q] * (V0[q] + VYM[q]) - VYP[q] * (V0[q] + VYP[q]);
        const C wv_hi = W0[q] + WYP[q];
        // sw
        const C sw_x = U0[q] + uzp;
        const C xw = WXM[q] * swm - WXP[q] * sw_x;
        const C yw = WYM[q] * (VYM[q] + vym_zp) - WYP[q] * (V0[q] + vzp);
        const C ww_hi = W0[q] + wzp;
        C hu = tcx * xu + tcy * yu;
        C hv = tcx * xv + tcy * yv;
        C hw = tcx * xw + tcy * yw;
        const int k = k0 + q;
        if (F64Z && f64z && k >= 1 && k <= t.f64_levels) {
          const double* dt = t.c.d;
          const double e1 = dt[k], e2 = dt[nz + k], e3 = dt[2 * nz + k], e4 = dt[3 * nz + k];
          hu = (C)((double)hu + e1 * (double)uzm * (double)wu_lo - e2 * (double)uzp * (double)wu_hi);
          hv = (C)((double)hv + e1 * (double)vzm * (double)wv_lo - e2 * (double)vzp * (double)wv_hi);
          hw = (C)((double)hw + e3 * (double)wzm * (double)ww_lo - e4 * (double)wzp * (double)ww_hi);
        } else {
          hu = hu + c1[q] * uzm * wu_lo - c2[q] * uzp * wu_hi;
          hv = hv + c1[q] * vzm * wv_lo - c2[q] * vzp * wv_hi;
          hw = hw + d1[q] * wzm * ww_lo - d2[q] * wzp * ww_hi;
        }
        ou[q] = k >= 1 ? hu : C(0);
        ov[q] = k >= 1 ? hv : C(0);
        ow[q] = (k >= 1 && k < nz - 1) ? hw : C(0);
        if constexpr (kRoll) {
          SXm[q] = sx;
          SVm[q] = sv_x;
          SWm[q] = sw_x;
        }
        wu_lo = wu_hi;
        wv_lo = wv_hi;
        ww_lo = ww_hi;
      }
      if (row_ok) {
        const size_t o = ((size_t)i * ny + j) * nz + k0;
        if constexpr (INTEG) {
          const C dt = step_of(C(0), t.dt, t.dt_hi, t.dt_lo);
          add_step<T, C, P>(t.b[0], o, t.sc.base[0], U0, dt, ou);
          add_step<T, C, P>(t.b[1], o, t.sc.base[1], V0, dt, ov);
          add_step<T, C, P>(t.b[2], o, t.sc.base[2], W0, dt, ow);
        }
        IO::st(t.o[0] + o, ou, o_u);
        IO::st(t.o[1] + o, ov, o_v);
        IO::st(t.o[2] + o, ow, o_w);
      }
      uxmp = u0p;
#pragma unroll
      for (int q = 0; q < P; ++q) {
        UXM[q] = U0[q];
        U0[q] = UXP[q];
        UXMYP[q] = UYP[q];
        VXM[q] = V0[q];
        V0[q] = VXP[q];
        VYM[q] = VXPYM[q];
        WXM[q] = W0[q];
        W0[q] = WXP[q];
      }
      if constexpr (!kRehalo) {
        u0m = nx.um;
        u0p = nx.up;
        v0m = nx.vm;
        v0p = nx.vp;
        vymp = nx.vymp;
        w0m = wxpm;
        w0p = nx.wp;
      }
    }
    ok = !timed_out;
  }
  return finish_tile(R, ok);
}

}  // namespace sweep
}  // namespace advect
