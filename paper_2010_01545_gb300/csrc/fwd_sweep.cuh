// fwd_sweep.cuh -- the single-grid plane-sweep forward kernel and its
// launchers, as templates.  Instantiated by fwd_sweep.cu (the source terms)
// and fwd_integ.cu (the source terms integrated into the flow fields), each
// in its own translation unit so the two builds run in parallel and neither
// kernel carries the other's code.
//
// The grid of CTAs is (ceil(ny / TY), ceil((i1 - i0) / LX)); blockIdx.x runs
// over y so that CTAs resident at the same time hold neighbouring rows and
// share their halo rows through L2.  The sweep itself is sweep::forward_tile
// (sweep_core.cuh).
#pragma once

#include <type_traits>

#include "sweep_core.cuh"
#include "sweep_ff.cuh"
#include "sweep_h16.cuh"

namespace advect {
namespace {  // internal linkage: each translation unit keeps its own kernels

struct SweepParams {
  FwdArgs a;
  int ty, kb, lx, nb;
  size_t slot_cap;
  int* flag;
};

template <typename T, int OCC, bool F64Z, bool SPLIT, bool INTEG>
__global__ void __launch_bounds__(OCC == 1 ? 256 : 128, OCC) fwd_sweep_kernel(SweepParams p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const sweep::Ring R = sweep::make_ring(smem_raw, p.nb, p.slot_cap);
  sweep::Tile<T> t;
  t.f[0] = (const T*)p.a.u;
  t.f[1] = (const T*)p.a.v;
  t.f[2] = (const T*)p.a.w;
  t.nf = 3;
  t.o[0] = (T*)p.a.su;
  t.o[1] = (T*)p.a.sv;
  t.o[2] = (T*)p.a.sw;
  t.nx = p.a.s.nx;
  t.ny = p.a.s.ny;
  t.nz = p.a.s.nz;
  t.j0 = blockIdx.x * p.ty;
  t.ty = p.ty;
  t.kb = p.kb;
  t.i_lo = p.a.i0 + blockIdx.y * p.lx;
  t.i_hi = min(t.i_lo + p.lx, p.a.i1);
  t.c = p.a.c;
  t.sc = p.a.sc;
  t.f64_levels = p.a.f64_levels;
  t.wait_budget = p.a.wait_budget;
  t.skip_plane = p.a.skip_plane;
  t.integ = p.a.integ;
  t.b[0] = (const T*)p.a.bu;
  t.b[1] = (const T*)p.a.bv;
  t.b[2] = (const T*)p.a.bw;
  t.dt = p.a.dt;
  t.dt_hi = p.a.dt_hi;
  t.dt_lo = p.a.dt_lo;
  sweep::forward_tile<T, F64Z, SPLIT, INTEG>(t, R, p.flag);
}

// F16S source terms without binary64 levels: the 8-level sweep of
// sweep_h16.cuh (p.kb = nz / 8).
template <int OCC, bool SPLIT>
__global__ void __launch_bounds__(OCC == 1 ? 256 : 128, OCC) fwd_h16_kernel(SweepParams p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const sweep::Ring R = sweep::make_ring(smem_raw, p.nb, p.slot_cap);
  sweep::Tile<__half> t;
  t.f[0] = (const __half*)p.a.u;
  t.f[1] = (const __half*)p.a.v;
  t.f[2] = (const __half*)p.a.w;
  t.nf = 3;
  t.o[0] = (__half*)p.a.su;
  t.o[1] = (__half*)p.a.sv;
  t.o[2] = (__half*)p.a.sw;
  t.nx = p.a.s.nx;
  t.ny = p.a.s.ny;
  t.nz = p.a.s.nz;
  t.j0 = blockIdx.x * p.ty;
  t.ty = p.ty;
  t.kb = p.kb;
  t.i_lo = p.a.i0 + blockIdx.y * p.lx;
  t.i_hi = min(t.i_lo + p.lx, p.a.i1);
  t.c = p.a.c;
  t.sc = p.a.sc;
  t.f64_levels = 0;
  t.wait_budget = p.a.wait_budget;
  t.skip_plane = p.a.skip_plane;
  sweep::forward_tile_h16<SPLIT>(t, R, p.flag);
}

template <int OCC, bool SPLIT>
cudaError_t launch_h16_v(const SweepParams& p, dim3 grid, int threads, size_t smem, cudaStream_t st) {
  if (threads > (OCC == 1 ? 256 : 128)) return cudaErrorInvalidConfiguration;
  static int attr_bytes = -1;
  if ((int)smem > attr_bytes) {
    cudaError_t e = cudaFuncSetAttribute(fwd_h16_kernel<OCC, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    attr_bytes = (int)smem;
  }
  fwd_h16_kernel<OCC, SPLIT><<<grid, threads, smem, st>>>(p);
  return cudaGetLastError();
}

template <int OCC>
cudaError_t launch_h16_occ(const SweepParams& p, dim3 grid, int threads, size_t smem, cudaStream_t st) {
  if (32 % p.kb != 0) return launch_h16_v<OCC, true>(p, grid, threads, smem, st);
  return launch_h16_v<OCC, false>(p, grid, threads, smem, st);
}

// Double-float source terms where a column's k-blocks divide a warp: the
// converter-warp sweep of sweep_ff.cuh (p.kb = nz / 2; kConverters more
// warps than the tile's compute threads; ff_max_threads(OCC) threads at most).
template <int OCC>
__global__ void __launch_bounds__(sweep::ff_max_threads(OCC), OCC) fwd_ff_kernel(SweepParams p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const sweep::Ring R = sweep::make_ring(smem_raw, p.nb, p.slot_cap);
  sweep::Tile<f64ff> t;
  t.f[0] = (const f64ff*)p.a.u;
  t.f[1] = (const f64ff*)p.a.v;
  t.f[2] = (const f64ff*)p.a.w;
  t.nf = 3;
  t.o[0] = (f64ff*)p.a.su;
  t.o[1] = (f64ff*)p.a.sv;
  t.o[2] = (f64ff*)p.a.sw;
  t.nx = p.a.s.nx;
  t.ny = p.a.s.ny;
  t.nz = p.a.s.nz;
  t.j0 = blockIdx.x * p.ty;
  t.ty = p.ty;
  t.kb = p.kb;
  t.i_lo = p.a.i0 + blockIdx.y * p.lx;
  t.i_hi = min(t.i_lo + p.lx, p.a.i1);
  t.c = p.a.c;
  t.sc = p.a.sc;
  t.f64_levels = 0;
  t.wait_budget = p.a.wait_budget;
  t.skip_plane = p.a.skip_plane;
  sweep::forward_tile_ff(t, R, p.flag);
}

template <int OCC>
cudaError_t launch_ff_v(const SweepParams& p, dim3 grid, int threads, size_t smem, cudaStream_t st) {
  if (threads > sweep::ff_max_threads(OCC)) return cudaErrorInvalidConfiguration;
  static int attr_bytes = -1;
  if ((int)smem > attr_bytes) {
    cudaError_t e =
        cudaFuncSetAttribute(fwd_ff_kernel<OCC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_bytes = (int)smem;
  }
  fwd_ff_kernel<OCC><<<grid, threads, smem, st>>>(p);
  return cudaGetLastError();
}

template <typename T, int OCC, bool F64Z, bool SPLIT, bool INTEG>
cudaError_t launch_v(const SweepParams& p, dim3 grid, int threads, size_t smem, cudaStream_t st) {
  if (threads > (OCC == 1 ? 256 : 128)) return cudaErrorInvalidConfiguration;
  static int attr_bytes = -1;  // largest dynamic shared memory size already allowed
  if ((int)smem > attr_bytes) {
    cudaError_t e = cudaFuncSetAttribute(fwd_sweep_kernel<T, OCC, F64Z, SPLIT, INTEG>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_bytes = (int)smem;
  }
  fwd_sweep_kernel<T, OCC, F64Z, SPLIT, INTEG><<<grid, threads, smem, st>>>(p);
  return cudaGetLastError();
}

template <typename T, bool INTEG, int OCC, bool F64Z = false>
cudaError_t launch_occ(const SweepParams& p, dim3 grid, int threads, size_t smem, cudaStream_t st) {
  if (32 % p.kb != 0) return launch_v<T, OCC, F64Z, true, INTEG>(p, grid, threads, smem, st);
  return launch_v<T, OCC, F64Z, false, INTEG>(p, grid, threads, smem, st);
}

// Binary64 near-surface levels (F32/F16S only): one uncapped variant.
template <typename T, bool INTEG>
cudaError_t launch_f64z(const SweepParams& p, dim3 grid, int threads, size_t smem, cudaStream_t st) {
  if constexpr (sizeof(typename Store<T>::C) == 4) return launch_occ<T, INTEG, 1, true>(p, grid, threads, smem, st);
  return launch_occ<T, INTEG, 1, false>(p, grid, threads, smem, st);
}

template <typename T, bool INTEG>
cudaError_t launch_t(const FwdArgs& a, const SweepCfg& cfg_in, int* flag, cudaStream_t st) {
  constexpr int P = sweep::VecIO<T>::P;
  SweepCfg cfg = cfg_in;
  if constexpr (std::is_same<T, __half>::value) {
    if (!INTEG && a.f64_levels == 0) {
      // the 8-level F16S sweep, tile as given
      SweepParams p;
      p.a = a;
      p.ty = cfg.ty;
      p.kb = a.s.nz / sweep::h16::P;
      p.lx = cfg.lx;
      p.nb = cfg.nb;
      p.slot_cap = (size_t)3 * (cfg.ty + 2) * a.s.nz * sizeof(__half);
      p.flag = flag;
      const size_t smem = sweep_smem_bytes(a.s.nz, (int)sizeof(__half), cfg);
      const dim3 grid((a.s.ny + cfg.ty - 1) / cfg.ty, (a.i1 - a.i0 + cfg.lx - 1) / cfg.lx);
      const int threads = cfg.ty * p.kb;
      switch (cfg.occ) {
        case 3: return launch_h16_occ<3>(p, grid, threads, smem, st);
        case 4: return launch_h16_occ<4>(p, grid, threads, smem, st);
        default: return launch_h16_occ<1>(p, grid, threads, smem, st);
      }
    }
    // the integration epilogue and the binary64 near-surface levels run the
    // generic sweep with 4-level binary16 vectors: its own default tile
    cfg = fit_planes(default_sweep_vec(a.s.nz, (int)sizeof(__half), P), a.i1 - a.i0);
    if (cfg.ty == 0) return launch_fwd_point(kF16S, a, st);
  }
  if constexpr (std::is_same<T, f64ff>::value && !INTEG) {
    if (ff_sweep_fits(a.s.nz) && cfg.ty * (a.s.nz / P) + 32 * sweep::kConverters <= sweep::ff_max_threads(cfg.occ)) {
      SweepParams p;
      p.a = a;
      p.ty = cfg.ty;
      p.kb = a.s.nz / P;
      p.lx = cfg.lx;
      p.nb = cfg.nb;
      p.slot_cap = (size_t)3 * (cfg.ty + 2) * a.s.nz * sizeof(f64ff);
      p.flag = flag;
      const size_t smem = sweep_smem_bytes(a.s.nz, (int)sizeof(f64ff), cfg) + sweep::ff_extra_bytes(cfg.nb, a.s.nz);
      const dim3 grid((a.s.ny + cfg.ty - 1) / cfg.ty, (a.i1 - a.i0 + cfg.lx - 1) / cfg.lx);
      const int threads = cfg.ty * p.kb + 32 * sweep::kConverters;
      switch (cfg.occ) {
        case 4: return launch_ff_v<4>(p, grid, threads, smem, st);
        case 3: return launch_ff_v<3>(p, grid, threads, smem, st);
        case 2: return launch_ff_v<2>(p, grid, threads, smem, st);
        default: return launch_ff_v<1>(p, grid, threads, smem, st);
      }
    }
  }
  SweepParams p;
  p.a = a;
  p.ty = cfg.ty;
  p.kb = a.s.nz / P;
  p.lx = cfg.lx;
  p.nb = cfg.nb;
  p.slot_cap = (size_t)3 * (cfg.ty + 2) * a.s.nz * sizeof(T);
  p.flag = flag;
  const size_t smem = sweep_smem_bytes(a.s.nz, (int)sizeof(T), cfg);
  const dim3 grid((a.s.ny + cfg.ty - 1) / cfg.ty, (a.i1 - a.i0 + cfg.lx - 1) / cfg.lx);
  const int threads = cfg.ty * p.kb;
  if (a.f64_levels > 0) return launch_f64z<T, INTEG>(p, grid, threads, smem, st);
  switch (cfg.occ) {
    case 3: return launch_occ<T, INTEG, 3>(p, grid, threads, smem, st);
    case 4: return launch_occ<T, INTEG, 4>(p, grid, threads, smem, st);
    default: return launch_occ<T, INTEG, 1>(p, grid, threads, smem, st);
  }
}

}  // namespace
}  // namespace advect
