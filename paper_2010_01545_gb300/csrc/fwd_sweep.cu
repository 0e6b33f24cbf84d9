// fwd_sweep.cu -- plane-sweep forward kernel (the HBM-streaming fast path).
//
// Design (GB300 recast of the paper's loop reordering, Sec. 3, Listing 4:
// march along x so each column is fetched from DRAM once):
//  * A CTA owns TY rows of y (j0 .. j0+TY-1) and a range of x-planes.  For
//    each plane it needs the (TY+2)-row slab j0-1 .. j0+TY of u, v, w; in the
//    [nx][ny][nz] layout that slab is contiguous in memory (one bulk copy per
//    field, or three where the periodic wrap in y splits it).
//  * One thread issues the bulk copies (cp.async.bulk, the TMA engine) into a
//    ring of NB shared-memory plane slots; an mbarrier per slot tracks the
//    bytes.  After a plane is consumed the slot is refilled NB planes ahead.
//  * Thread (row r, k-block kb) owns P consecutive levels of one column for
//    the whole sweep.  Values of the previous and current plane, and the face
//    sums shared between consecutive planes, roll in registers, so each
//    plane costs 9 vector loads from shared memory per thread.  Vertical
//    neighbours (k-1, k+P) come from the adjacent lanes by warp shuffle.
//  * Outputs go straight to global memory with streaming 16/8-byte stores.
// Arithmetic and evaluation order per point follow Listing 1 (Sec. 2.1) and
// its v/w analogues; the lid branch comes from tzc2[nz-1] == 0 and zero
// values above the top level.
#include "bulk.cuh"
#include "kernels.h"

namespace advect {
namespace {

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
  __device__ static __forceinline__ void st(__half* g, const C (&v)[P], float inv) {
    const __half2 a = __floats2half2_rn(v[0] * inv, v[1] * inv);
    const __half2 b = __floats2half2_rn(v[2] * inv, v[3] * inv);
    uint2 x;
    x.x = *reinterpret_cast<const uint32_t*>(&a);
    x.y = *reinterpret_cast<const uint32_t*>(&b);
    __stcs(reinterpret_cast<uint2*>(g), x);
  }
};

struct SweepParams {
  FwdArgs a;
  int ty, kb, lx, nb;
  int* flag;
};

// Vertical halo of a P-vector: the value just below (k0-1) and just above
// (k0+P) the thread's levels, from the neighbouring lanes of the same row;
// zero beyond the column, a shared-memory read where the row crosses a warp.
template <typename T, typename C, int P>
__device__ __forceinline__ void halo(const C (&a)[P], const T* row, int k0, int kb, int KB, int lane,
                                     float sc, C& below, C& above) {
  below = __shfl_up_sync(0xffffffffu, a[P - 1], 1);
  above = __shfl_down_sync(0xffffffffu, a[0], 1);
  if (kb == 0) below = C(0);
  else if (lane == 0) below = VecIO<T>::ld1(row + k0 - 1, sc);
  if (kb == KB - 1) above = C(0);
  else if (lane == 31) above = VecIO<T>::ld1(row + k0 + P, sc);
}

template <typename T, typename C, int P>
__device__ __forceinline__ C halo_above(const C (&a)[P], const T* row, int k0, int kb, int KB, int lane,
                                        float sc) {
  C above = __shfl_down_sync(0xffffffffu, a[0], 1);
  if (kb == KB - 1) above = C(0);
  else if (lane == 31) above = VecIO<T>::ld1(row + k0 + P, sc);
  return above;
}

template <typename T, typename C, int P>
__device__ __forceinline__ C halo_below(const C (&a)[P], const T* row, int k0, int kb, int lane, float sc) {
  C below = __shfl_up_sync(0xffffffffu, a[P - 1], 1);
  if (kb == 0) below = C(0);
  else if (lane == 0) below = VecIO<T>::ld1(row + k0 - 1, sc);
  return below;
}

template <typename T>
__global__ void __launch_bounds__(256, 1) fwd_sweep_kernel(SweepParams p) {
  using IO = VecIO<T>;
  using C = typename IO::C;
  constexpr int P = IO::P;
  extern __shared__ __align__(128) unsigned char smem_raw[];

  const int nx = p.a.s.nx, ny = p.a.s.ny, nz = p.a.s.nz;
  const int TY = p.ty, KB = p.kb, NB = p.nb;
  const int rows = TY + 2;
  const size_t slot_elems = (size_t)3 * rows * nz;
  T* slots = reinterpret_cast<T*>(smem_raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + (size_t)NB * slot_elems * sizeof(T));

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int kb = tid % KB, rr = tid / KB;
  const int k0 = kb * P;
  const int j0 = blockIdx.x * TY;
  const int ty_eff = min(TY, ny - j0);
  const int j = j0 + rr;
  const bool row_ok = rr < ty_eff;
  const int i_lo = p.a.i0 + blockIdx.y * p.lx;
  const int i_hi = min(i_lo + p.lx, p.a.i1);
  const int nplanes = i_hi - i_lo + 2;  // planes i_lo-1 .. i_hi
  const float s_u = p.a.sc.in[0], s_v = p.a.sc.in[1], s_w = p.a.sc.in[2];

  const T* fld[3] = {(const T*)p.a.u, (const T*)p.a.v, (const T*)p.a.w};

  // Producer: bulk-copy plane q (x index i_lo-1+q, periodic) into its slot.
  auto issue = [&](int q) {
    const int slot = q % NB;
    int ig = i_lo - 1 + q;
    ig = ig < 0 ? ig + nx : (ig >= nx ? ig - nx : ig);
    const uint32_t row_bytes = (uint32_t)(nz * sizeof(T));
    mbar_arrive_expect_tx(&bars[slot], 3u * (uint32_t)(ty_eff + 2) * row_bytes);
    T* dst0 = slots + (size_t)slot * slot_elems;
    for (int f = 0; f < 3; ++f) {
      const T* plane = fld[f] + (size_t)ig * ny * nz;
      T* dst = dst0 + (size_t)f * rows * nz;
      if (j0 >= 1 && j0 + ty_eff <= ny - 1) {
        bulk_copy_g2s(dst, plane + (size_t)(j0 - 1) * nz, (uint32_t)(ty_eff + 2) * row_bytes, &bars[slot]);
      } else {
        const int jt = j0 == 0 ? ny - 1 : j0 - 1;
        const int jb = j0 + ty_eff == ny ? 0 : j0 + ty_eff;
        bulk_copy_g2s(dst, plane + (size_t)jt * nz, row_bytes, &bars[slot]);
        bulk_copy_g2s(dst + nz, plane + (size_t)j0 * nz, (uint32_t)ty_eff * row_bytes, &bars[slot]);
        bulk_copy_g2s(dst + (size_t)(ty_eff + 1) * nz, plane + (size_t)jb * nz, row_bytes, &bars[slot]);
      }
    }
  };

  if (tid == 0) {
    for (int s = 0; s < NB; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  int issued = 0;  // meaningful in thread 0 only
  if (tid == 0) {
    for (; issued < NB && issued < nplanes; ++issued) issue(issued);
  }

  // Row pointers of plane q, field f, local row lr (0 = j0-1).
  auto rowp = [&](int q, int f, int lr) -> const T* {
    return slots + (size_t)(q % NB) * slot_elems + ((size_t)f * rows + lr) * nz;
  };
  int timed_out = 0;  // this thread gave up a wait; combined with __syncthreads_or
  auto wait_plane = [&](int q) {
    if (!mbar_wait_bounded(&bars[q % NB], (uint32_t)((q / NB) & 1))) {
      timed_out = 1;
      atomicExch(p.flag, 1);
    }
  };

  // Per-level coefficients of this thread's levels (constant over the sweep).
  using S = Store<T>;
  C c1[P], c2[P], d1[P], d2[P];
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const int k = min(k0 + q, nz - 1);
    c1[q] = S::coef(p.a.c, TZC1, nz, k);
    c2[q] = S::coef(p.a.c, TZC2, nz, k);
    d1[q] = S::coef(p.a.c, TZD1, nz, k);
    d2[q] = S::coef(p.a.c, TZD2, nz, k);
  }
  const C tcx = S::tcx(p.a.c), tcy = S::tcy(p.a.c);
  const int r = rr + 1;  // local row of this thread's column

  // Rolling state (plane i): see the file comment for the naming.
  C UXM[P], U0[P], UXMYP[P], VXM[P], V0[P], VYM[P], WXM[P], W0[P];
  C SXm[P], SVm[P], SWm[P];  // face sums shared with the previous plane
  C u0m, u0p, uxmp, v0m, v0p, vymp, w0m, w0p;

  wait_plane(0);
  wait_plane(1);
  IO::ld(rowp(0, 0, r) + k0, s_u, UXM);
  IO::ld(rowp(1, 0, r) + k0, s_u, U0);
  IO::ld(rowp(0, 0, r + 1) + k0, s_u, UXMYP);
  IO::ld(rowp(0, 1, r) + k0, s_v, VXM);
  IO::ld(rowp(1, 1, r) + k0, s_v, V0);
  IO::ld(rowp(1, 1, r - 1) + k0, s_v, VYM);
  IO::ld(rowp(0, 2, r) + k0, s_w, WXM);
  IO::ld(rowp(1, 2, r) + k0, s_w, W0);
  halo<T, C, P>(U0, rowp(1, 0, r), k0, kb, KB, lane, s_u, u0m, u0p);
  uxmp = halo_above<T, C, P>(UXM, rowp(0, 0, r), k0, kb, KB, lane, s_u);
  halo<T, C, P>(V0, rowp(1, 1, r), k0, kb, KB, lane, s_v, v0m, v0p);
  vymp = halo_above<T, C, P>(VYM, rowp(1, 1, r - 1), k0, kb, KB, lane, s_v);
  halo<T, C, P>(W0, rowp(1, 2, r), k0, kb, KB, lane, s_w, w0m, w0p);
#pragma unroll
  for (int q = 0; q < P; ++q) {
    SXm[q] = UXM[q] + U0[q];
    SVm[q] = UXM[q] + UXMYP[q];
    SWm[q] = UXM[q] + (q < P - 1 ? UXM[q + 1] : uxmp);
  }

  int consumed = 1;  // highest plane index waited for
  bool aborted = false;
  __syncthreads();   // plane i_lo-1 (slot 0) has been read into registers
  if (tid == 0 && issued < nplanes) {
    fence_proxy_async_smem();
    issue(issued);
    ++issued;
  }

  T* out[3] = {(T*)p.a.su, (T*)p.a.sv, (T*)p.a.sw};
  const bool f64z = sizeof(C) == 4 && p.a.f64_levels > 0 && k0 <= p.a.f64_levels;

  // Row offsets (elements) within a slot, fixed for the sweep.
  const int o_u0 = r * nz, o_um = (r - 1) * nz, o_up = (r + 1) * nz;
  const int o_v0 = (rows + r) * nz, o_vm = (rows + r - 1) * nz, o_vp = (rows + r + 1) * nz;
  const int o_w0 = (2 * rows + r) * nz, o_wm = (2 * rows + r - 1) * nz, o_wp = (2 * rows + r + 1) * nz;
  int slot_c = 1 % NB, slot_n = 2 % NB;  // slots of planes i and i+1

  for (int i = i_lo; i < i_hi; ++i) {
    const int qn = i - i_lo + 2;  // plane i+1
    wait_plane(qn);
    consumed = qn;
    const T* Pc = slots + (size_t)slot_c * slot_elems;
    const T* Pn = slots + (size_t)slot_n * slot_elems;
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
    C uxpm, uxpp, vxpm, vxpp, wxpm, wxpp;
    halo<T, C, P>(UXP, Pn + o_u0, k0, kb, KB, lane, s_u, uxpm, uxpp);
    halo<T, C, P>(VXP, Pn + o_v0, k0, kb, KB, lane, s_v, vxpm, vxpp);
    halo<T, C, P>(WXP, Pn + o_w0, k0, kb, KB, lane, s_w, wxpm, wxpp);
    const C vxpymp = halo_above<T, C, P>(VXPYM, Pn + o_vm, k0, kb, KB, lane, s_v);
    const C wypm = halo_below<T, C, P>(WYP, Pc + o_wp, k0, kb, lane, s_w);
    slot_c = slot_n;
    slot_n = slot_n + 1 == NB ? 0 : slot_n + 1;

    C ou[P], ov[P], ow[P];
    C wu_lo = w0m + wxpm;   // w(i,k-1) + w(i+1,k-1): su's lower face
    C wv_lo = w0m + wypm;   // w(i,j,k-1) + w(i,j+1,k-1): sv's lower face
    C ww_lo = W0[0] + w0m;  // w(k) + w(k-1): sw's lower face
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const C uzm = q > 0 ? U0[q - 1] : u0m;
      const C uzp = q < P - 1 ? U0[q + 1] : u0p;
      const C vzm = q > 0 ? V0[q - 1] : v0m;
      const C vzp = q < P - 1 ? V0[q + 1] : v0p;
      const C wzm = q > 0 ? W0[q - 1] : w0m;
      const C wzp = q < P - 1 ? W0[q + 1] : w0p;
      const C vym_zp = q < P - 1 ? VYM[q + 1] : vymp;
      // su (Listing 1)
      const C sx = U0[q] + UXP[q];
      const C xu = UXM[q] * SXm[q] - UXP[q] * sx;
      const C yu = UYM[q] * (VYM[q] + VXPYM[q]) - UYP[q] * (V0[q] + VXP[q]);
      const C wu_hi = W0[q] + WXP[q];
      // sv
      const C sv_x = U0[q] + UYP[q];
      const C xv = VXM[q] * SVm[q] - VXP[q] * sv_x;
      const C yv = VYM[q] * (V0[q] + VYM[q]) - VYP[q] * (V0[q] + VYP[q]);
      const C wv_hi = W0[q] + WYP[q];
      // sw
      const C sw_x = U0[q] + uzp;
      const C xw = WXM[q] * SWm[q] - WXP[q] * sw_x;
      const C yw = WYM[q] * (VYM[q] + vym_zp) - WYP[q] * (V0[q] + vzp);
      const C ww_hi = W0[q] + wzp;
      C hu = tcx * xu + tcy * yu;
      C hv = tcx * xv + tcy * yv;
      C hw = tcx * xw + tcy * yw;
      if (f64z && k0 + q >= 1 && k0 + q <= p.a.f64_levels) {
        const double* dt = p.a.c.d;
        const int k = k0 + q;
        const double e1 = dt[k], e2 = dt[nz + k], e3 = dt[2 * nz + k], e4 = dt[3 * nz + k];
        hu = (C)((double)hu + e1 * (double)uzm * (double)wu_lo - e2 * (double)uzp * (double)wu_hi);
        hv = (C)((double)hv + e1 * (double)vzm * (double)wv_lo - e2 * (double)vzp * (double)wv_hi);
        hw = (C)((double)hw + e3 * (double)wzm * (double)ww_lo - e4 * (double)wzp * (double)ww_hi);
      } else {
        hu = hu + c1[q] * uzm * wu_lo - c2[q] * uzp * wu_hi;
        hv = hv + c1[q] * vzm * wv_lo - c2[q] * vzp * wv_hi;
        hw = hw + d1[q] * wzm * ww_lo - d2[q] * wzp * ww_hi;
      }
      const int k = k0 + q;
      ou[q] = k >= 1 ? hu : C(0);
      ov[q] = k >= 1 ? hv : C(0);
      ow[q] = (k >= 1 && k < nz - 1) ? hw : C(0);
      // roll the face sums to the next plane
      SXm[q] = sx;
      SVm[q] = sv_x;
      SWm[q] = sw_x;
      wu_lo = wu_hi;
      wv_lo = wv_hi;
      ww_lo = ww_hi;
    }
    if (row_ok) {
      const size_t o = ((size_t)i * ny + j) * nz + k0;
      IO::st(out[0] + o, ou, p.a.sc.inv_out[0]);
      IO::st(out[1] + o, ov, p.a.sc.inv_out[1]);
      IO::st(out[2] + o, ow, p.a.sc.inv_out[2]);
    }
    // roll plane values
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
    u0m = uxpm;
    u0p = uxpp;
    v0m = vxpm;
    v0p = vxpp;
    vymp = vxpymp;
    w0m = wxpm;
    w0p = wxpp;

    // every thread is done with plane i's slot (plane i-1 lives in registers);
    // the barrier also makes the give-up decision uniform across the CTA
    if (__syncthreads_or(timed_out)) {
      aborted = true;
      break;
    }
    if (tid == 0 && issued < nplanes) {  // issued == qc + NB: refill the slot of plane i
      fence_proxy_async_smem();
      issue(issued);
      ++issued;
    }
  }
  if (aborted && tid == 0) {
    // drain copies still in flight before the CTA's shared memory is released
    for (int q = consumed + 1; q < issued; ++q)
      mbar_wait_bounded(&bars[q % NB], (uint32_t)((q / NB) & 1), 1 << 20);
  }
}

template <typename T>
cudaError_t launch_t(const FwdArgs& a, const SweepCfg& cfg, int* flag, cudaStream_t st) {
  constexpr int P = VecIO<T>::P;
  SweepParams p;
  p.a = a;
  p.ty = cfg.ty;
  p.kb = a.s.nz / P;
  p.lx = cfg.lx;
  p.nb = cfg.nb;
  p.flag = flag;
  const size_t smem = sweep_smem_bytes(a.s.nz, (int)sizeof(T), cfg);
  static int attr_bytes = -1;  // largest dynamic shared memory size already allowed
  if ((int)smem > attr_bytes) {
    cudaError_t e = cudaFuncSetAttribute(fwd_sweep_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    attr_bytes = (int)smem;
  }
  const dim3 grid((a.s.ny + cfg.ty - 1) / cfg.ty, (a.i1 - a.i0 + cfg.lx - 1) / cfg.lx);
  fwd_sweep_kernel<T><<<grid, cfg.ty * p.kb, smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace

size_t sweep_smem_bytes(int nz, int elem, const SweepCfg& cfg) {
  return (size_t)cfg.nb * 3 * (cfg.ty + 2) * nz * elem + (size_t)cfg.nb * sizeof(uint64_t);
}

int sweep_vec(int elem) { return elem == 8 ? 2 : 4; }

cudaError_t launch_fwd_sweep(int dtype, const FwdArgs& a, const SweepCfg& cfg, int* flag, cudaStream_t st) {
  if (a.i1 <= a.i0) return cudaSuccess;
  switch (dtype) {
    case kF64: return launch_t<double>(a, cfg, flag, st);
    case kF32: return launch_t<float>(a, cfg, flag, st);
    case kF16S: return launch_t<__half>(a, cfg, flag, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace advect
