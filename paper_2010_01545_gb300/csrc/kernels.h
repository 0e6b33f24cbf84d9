// kernels.h -- host-side launchers of the advection kernels (internal API).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace advect {

// Element type codes (same values as advect_dtype).
enum Dtype { kF64 = 0, kF32 = 1, kF16S = 2, kF64FF = 3 };

struct FwdArgs {
  const void *u, *v, *w;
  void *su, *sv, *sw;
  Shape s;
  Coeffs c;
  Scales sc;
  int f64_levels;  // F32/F16S: levels 1..f64_levels use binary64 vertical terms
  int i0, i1;      // x-planes [i0, i1) are computed (the others are untouched)
  long long wait_budget = 2LL * 1000 * 1000 * 1000;  // clock64 cycles per bounded wait
  int skip_plane = -1;  // test-only: plane index of each tile whose copy is never issued
  // Integration epilogue: when integ != 0 the outputs are base + dt * (su, sv,
  // sw) instead of the source terms; base = (bu, bv, bw), or the winds
  // themselves where bu is NULL.  dt_hi + dt_lo is dt split into binary32.
  int integ = 0;
  const void *bu = nullptr, *bv = nullptr, *bw = nullptr;
  double dt = 0.0;
  float dt_hi = 0.f, dt_lo = 0.f;
};

struct AdjArgs {
  const void *u, *v, *w, *dsu, *dsv, *dsw;
  void *du, *dv, *dw;
  Shape s;
  Coeffs c;
  long long wait_budget = 2LL * 1000 * 1000 * 1000;
  int skip_plane = -1;
};

// Plane-sweep tile configuration (see fwd_sweep.cu).
struct SweepCfg {
  int ty;   // rows (y) per CTA
  int lx;   // x-planes per CTA
  int nb;   // shared-memory plane slots (>= 4)
  int occ;  // CTAs per SM the register allocation is capped for (1, 3 or 4)
};

// One thread per grid point, plain loads: any shape and alignment.
cudaError_t launch_fwd_point(int dtype, const FwdArgs& a, cudaStream_t st);
cudaError_t launch_adj_point(int dtype, const AdjArgs& a, cudaStream_t st);

// Plane sweep: needs nz % sweep_vec(elem) == 0, nz * elem % 16 == 0, 16-byte
// aligned fields, ty * nz / sweep_vec(elem) a multiple of 32 and <= 256.
int sweep_vec(int elem);
size_t sweep_smem_bytes(int nz, int elem, const SweepCfg& cfg);
// The double-float forward uses its converter-warp sweep (sweep_ff.cuh) when
// a column's 2-level k-blocks divide a warp (nz = 2, 4, ..., 64).
inline bool ff_sweep_fits(int nz) { return nz % 2 == 0 && nz / 2 <= 32 && 32 % (nz / 2) == 0; }
// Default tile for vectors of vec levels per thread (ty == 0: not sweepable).
SweepCfg default_sweep_vec(int nz, int elem, int vec);
// A sweep launch is (ceil(ny / ty), ceil(planes / lx)) CTAs and gridDim.y is
// at most 65535, so an x extent longer than 65535 tiles takes longer tiles.
inline SweepCfg fit_planes(SweepCfg c, int planes) {
  const int need = (int)(((long long)planes + 65534) / 65535);
  if (c.lx < need) c.lx = need;
  return c;
}
cudaError_t launch_fwd_sweep(int dtype, const FwdArgs& a, const SweepCfg& cfg, int* flag, cudaStream_t st);
// The same sweep with the integration epilogue (a.integ != 0; fwd_integ.cu).
cudaError_t launch_fwd_sweep_integ(int dtype, const FwdArgs& a, const SweepCfg& cfg, int* flag,
                                   cudaStream_t st);

// Adjoint plane sweep (F64, F32): nz % adj_sweep_vec(elem) == 0, nz * elem % 16
// == 0, 16-byte aligned fields, ty * nz / adj_sweep_vec(elem) a multiple of 32.
int adj_sweep_vec(int elem);
// The double-float adjoint's own sweep (adj_ff.cuh, two levels per thread):
// whether a tile fits it, and its default tile (ty = 0: the shape does not).
bool adj_ff_fits(int nz, const SweepCfg& c);
SweepCfg default_adj_ff(int nz);
size_t adj_sweep_smem_bytes(int nz, int elem, const SweepCfg& cfg);
cudaError_t launch_adj_sweep(int dtype, const AdjArgs& a, const SweepCfg& cfg, int* flag, cudaStream_t st);

}  // namespace advect
