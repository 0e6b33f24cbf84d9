// adj_sweep.cu -- single-grid plane-sweep adjoint: one tile per CTA.
#include <type_traits>

#include "adj_f32.cuh"

namespace advect {
namespace {

struct AdjParams {
  AdjArgs a;
  int ty, kb, lx, nb;
  size_t slot_cap;
  int* flag;
};

template <typename T, int OCC, bool SPLIT>
__global__ void __launch_bounds__(OCC == 1 ? 256 : 128, OCC) adj_sweep_kernel(AdjParams p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const sweep::Ring R = sweep::make_ring(smem_raw, p.nb, p.slot_cap);
  sweep::Tile<T> t;
  t.f[0] = (const T*)p.a.u;
  t.f[1] = (const T*)p.a.v;
  t.f[2] = (const T*)p.a.w;
  t.f[3] = (const T*)p.a.dsu;
  t.f[4] = (const T*)p.a.dsv;
  t.f[5] = (const T*)p.a.dsw;
  t.nf = 6;
  t.o[0] = (T*)p.a.du;
  t.o[1] = (T*)p.a.dv;
  t.o[2] = (T*)p.a.dw;
  t.nx = p.a.s.nx;
  t.ny = p.a.s.ny;
  t.nz = p.a.s.nz;
  t.j0 = blockIdx.x * p.ty;
  t.ty = p.ty;
  t.kb = p.kb;
  t.i_lo = blockIdx.y * p.lx;
  t.i_hi = min(t.i_lo + p.lx, p.a.s.nx);
  t.c = p.a.c;
  for (int q = 0; q < 3; ++q) {
    t.sc.in[q] = 1.f;
    t.sc.inv_out[q] = 1.f;
    t.sc.base[q] = 1.f;
  }
  t.f64_levels = 0;
  t.wait_budget = p.a.wait_budget;
  t.skip_plane = p.a.skip_plane;
  if constexpr (std::is_same<T, float>::value)
    sweep::adjoint_tile_f32v4<SPLIT>(t, R, p.flag);  // 4 levels per thread
  else
    sweep::adjoint_tile<T, SPLIT>(t, R, p.flag);
}

template <typename T, int OCC, bool SPLIT>
cudaError_t launch_v(const AdjParams& p, dim3 grid, int threads, size_t smem, cudaStream_t st) {
  if (threads > (OCC == 1 ? 256 : 128)) return cudaErrorInvalidConfiguration;
  static int attr_bytes = -1;
  if ((int)smem > attr_bytes) {
    cudaError_t e = cudaFuncSetAttribute(adj_sweep_kernel<T, OCC, SPLIT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_bytes = (int)smem;
  }
  adj_sweep_kernel<T, OCC, SPLIT><<<grid, threads, smem, st>>>(p);
  return cudaGetLastError();
}

template <typename T, int OCC>
cudaError_t launch_occ(const AdjParams& p, dim3 grid, int threads, size_t smem, cudaStream_t st) {
  if (32 % p.kb != 0) return launch_v<T, OCC, true>(p, grid, threads, smem, st);
  return launch_v<T, OCC, false>(p, grid, threads, smem, st);
}

template <typename T>
cudaError_t launch_t(const AdjArgs& a, const SweepCfg& cfg, int* flag, cudaStream_t st) {
  AdjParams p;
  p.a = a;
  p.ty = cfg.ty;
  p.kb = a.s.nz / adj_sweep_vec((int)sizeof(T));
  p.lx = cfg.lx;
  p.nb = cfg.nb;
  p.slot_cap = (size_t)6 * (cfg.ty + 2) * a.s.nz * sizeof(T);
  p.flag = flag;
  const size_t smem = adj_sweep_smem_bytes(a.s.nz, (int)sizeof(T), cfg);
  const dim3 grid((a.s.ny + cfg.ty - 1) / cfg.ty, (a.s.nx + cfg.lx - 1) / cfg.lx);
  const int threads = cfg.ty * p.kb;
  switch (cfg.occ) {
    case 3: return launch_occ<T, 3>(p, grid, threads, smem, st);
    case 4: return launch_occ<T, 4>(p, grid, threads, smem, st);
    default: return launch_occ<T, 1>(p, grid, threads, smem, st);
  }
}

}  // namespace

size_t adj_sweep_smem_bytes(int nz, int elem, const SweepCfg& cfg) {
  // the binary32 sweep keeps its coefficient table after the ring
  return sweep::ring_bytes(cfg.nb, (size_t)6 * (cfg.ty + 2) * nz * elem) +
         (elem == 4 ? sweep::a4::table_bytes(nz) : 0);
}

// levels per thread of the adjoint sweep: 8-byte types 1, binary32 4
int adj_sweep_vec(int elem) { return elem == 8 ? 1 : 4; }

cudaError_t launch_adj_sweep(int dtype, const AdjArgs& a, const SweepCfg& cfg, int* flag, cudaStream_t st) {
  switch (dtype) {
    case kF64: return launch_t<double>(a, cfg, flag, st);
    case kF32: return launch_t<float>(a, cfg, flag, st);
    case kF64FF: return launch_t<f64ff>(a, cfg, flag, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace advect
