// adj_sweep.cu -- single-grid plane-sweep adjoint: one tile per CTA.
#include <type_traits>

#include "adj_f32.cuh"
#include "adj_ff.cuh"

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

// Double-float adjoint of adj_ff.cuh: one CTA per SM of up to 384 threads.
constexpr int kAdjFFThreads = 384;

template <bool SPLIT, int NZC, int TYC>
__global__ void __launch_bounds__(kAdjFFThreads, 1) adj_ff_kernel(AdjParams p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const sweep::Ring R = sweep::make_ring(smem_raw, p.nb, p.slot_cap);
  sweep::Tile<f64ff> t;
  t.f[0] = (const f64ff*)p.a.u;
  t.f[1] = (const f64ff*)p.a.v;
  t.f[2] = (const f64ff*)p.a.w;
  t.f[3] = (const f64ff*)p.a.dsu;
  t.f[4] = (const f64ff*)p.a.dsv;
  t.f[5] = (const f64ff*)p.a.dsw;
  t.nf = 6;
  t.o[0] = (f64ff*)p.a.du;
  t.o[1] = (f64ff*)p.a.dv;
  t.o[2] = (f64ff*)p.a.dw;
  t.nx = p.a.s.nx;
  t.ny = p.a.s.ny;
  t.nz = p.a.s.nz;
  t.j0 = blockIdx.x * p.ty;
  t.ty = p.ty;
  t.kb = p.kb;
  t.i_lo = blockIdx.y * p.lx;
  t.i_hi = min(t.i_lo + p.lx, p.a.s.nx);
  t.c = p.a.c;
  t.f64_levels = 0;
  t.wait_budget = p.a.wait_budget;
  t.skip_plane = p.a.skip_plane;
  sweep::adjoint_tile_ff<SPLIT, NZC, TYC>(t, R, p.flag);
}

size_t adj_ff_smem_bytes(int nz, const SweepCfg& c) {
  return sweep::ring_bytes(c.nb, (size_t)6 * (c.ty + 2) * nz * sizeof(f64ff)) +
         sweep::affx::adj_ff_extra_bytes(c.nb, nz);
}

template <bool SPLIT, int NZC = 0, int TYC = 0>
cudaError_t launch_ff(const AdjParams& p, dim3 grid, int threads, size_t smem, cudaStream_t st) {
  static int attr_bytes = -1;
  if ((int)smem > attr_bytes) {
    cudaError_t e = cudaFuncSetAttribute(adj_ff_kernel<SPLIT, NZC, TYC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_bytes = (int)smem;
  }
  adj_ff_kernel<SPLIT, NZC, TYC><<<grid, threads, smem, st>>>(p);
  return cudaGetLastError();
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
  if constexpr (std::is_same<T, f64ff>::value) {
    if (adj_ff_fits(a.s.nz, cfg)) {
      AdjParams p;
      p.a = a;
      p.ty = cfg.ty;
      p.kb = a.s.nz / 2;
      p.lx = cfg.lx;
      p.nb = cfg.nb;
      p.slot_cap = (size_t)6 * (cfg.ty + 2) * a.s.nz * sizeof(f64ff);
      p.flag = flag;
      const dim3 grid((a.s.ny + cfg.ty - 1) / cfg.ty, (a.s.nx + cfg.lx - 1) / cfg.lx);
      const int threads = cfg.ty * p.kb;
      const size_t smem = adj_ff_smem_bytes(a.s.nz, cfg);
      // the default tile of 128-level columns with its offsets compiled in
      if (a.s.nz == 128 && cfg.ty == 6) return launch_ff<true, 128, 6>(p, grid, threads, smem, st);
      if (p.kb > 32) return launch_ff<true>(p, grid, threads, smem, st);
      return launch_ff<false>(p, grid, threads, smem, st);
    }
  }
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

// The double-float adjoint of adj_ff.cuh takes a tile when nz / 2 is a power
// of two, its ty * nz / 2 threads are a multiple of 32 and at most 384, the
// ring has four slots or more and fits the CTA's shared memory.
bool adj_ff_fits(int nz, const SweepCfg& c) {
  if (nz < 2 || nz % 2) return false;
  const int kb = nz / 2;
  if (kb & (kb - 1)) return false;
  const long long threads = (long long)c.ty * kb;
  if (c.ty < 1 || c.lx < 1 || c.nb < 4 || threads % 32 || threads > kAdjFFThreads) return false;
  if ((uint64_t)6 * (c.ty + 2) * nz * sizeof(f64ff) >= (1u << 20)) return false;
  return adj_ff_smem_bytes(nz, c) <= 227 * 1024;
}

// Its default tile: 384 threads (12 warps, one CTA per SM) where four slots
// fit, fewer rows where not; the deepest ring up to six slots that fits.
SweepCfg default_adj_ff(int nz) {
  SweepCfg c{0, 64, 4, 1};
  if (nz < 2 || nz % 2 || ((nz / 2) & (nz / 2 - 1))) return c;
  const int kb = nz / 2;
  for (int ty = (kAdjFFThreads / kb > 0 ? kAdjFFThreads / kb : 1); ty >= 1; --ty) {
    SweepCfg t{ty, 64, 4, 1};
    if (adj_ff_fits(nz, t)) {
      c = t;
      break;
    }
  }
  if (c.ty == 0) return c;
  while (c.nb < 6) {
    SweepCfg d = c;
    ++d.nb;
    if (!adj_ff_fits(nz, d) || adj_ff_smem_bytes(nz, d) > 220 * 1024) break;
    c = d;
  }
  return c;
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
