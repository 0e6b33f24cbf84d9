// ens.cu -- ensembles: many independent grids of uneven shape in one
// persistent launch.
//
// The members are cut into tiles (TY rows x LX planes, TY chosen per member
// so that a tile has 128 threads' worth of columns).  The launch has about
// as many CTAs as fit on the GPU at once; each CTA takes the next tile index
// from a device counter (atomicAdd), decodes it against the member table and
// sweeps the tile with the same code as the single-grid kernels
// (sweep::forward_tile; for the adjoint sweep::adjoint_tile, or
// sweep::adjoint_tile_f32v4 with binary32, whose coefficient table after the
// ring is refilled per tile and sized for the largest column).  Tiles are
// ordered largest member first, so the dynamic queue ends with small tiles.
//
// The member table lives in device memory and is re-uploaded (on the
// caller's stream) only when the buffer pointers change.  Counter reset and
// kernel are captured once in a CUDA graph per direction and replayed.
// Independent members need no communication: this is the paper's split of
// the domain over independent kernel instances (Sec. 5), as data
// parallelism over grids.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include <type_traits>

#include "../../include/advect.h"
#include "adj_f32.cuh"
#include "ctx.h"
#include "ens.h"

namespace advect {

namespace {

template <typename T>
struct MemberDesc {
  const T* in[6];
  T* out[3];
  int nx, ny, nz, ty, kb;
  int n_jb, n_xr, tile_begin;
  Coeffs c;
};

struct EnsParams {
  const void* desc;
  int n_members, n_tiles, lx, nb;
  size_t slot_cap;
  int* counter;
  int* flag;
};

constexpr int kEnsThreads = 128;

template <typename T, int OCC, int ADJ, bool SPLIT>
__global__ void __launch_bounds__(kEnsThreads, OCC) ens_kernel(EnsParams p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int s_tile;
  const sweep::Ring R = sweep::make_ring(smem_raw, p.nb, p.slot_cap);
  const MemberDesc<T>* D = reinterpret_cast<const MemberDesc<T>*>(p.desc);
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(p.counter, 1);
    __syncthreads();
    const int tile = s_tile;
    __syncthreads();
    if (tile >= p.n_tiles) break;
    int lo = 0, hi = p.n_members - 1;  // last member with tile_begin <= tile
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (D[mid].tile_begin <= tile) lo = mid;
      else hi = mid - 1;
    }
    const MemberDesc<T>& d = D[lo];
    const int local = tile - d.tile_begin;
    const int jb = local % d.n_jb, xr = local / d.n_jb;
    sweep::Tile<T> t;
#pragma unroll
    for (int f = 0; f < 6; ++f) t.f[f] = d.in[f];
    t.o[0] = d.out[0];
    t.o[1] = d.out[1];
    t.o[2] = d.out[2];
    t.nf = ADJ ? 6 : 3;
    t.nx = d.nx;
    t.ny = d.ny;
    t.nz = d.nz;
    t.j0 = jb * d.ty;
    t.ty = d.ty;
    t.kb = d.kb;
    t.i_lo = xr * p.lx;
    t.i_hi = min(t.i_lo + p.lx, d.nx);
    t.c = d.c;
    for (int q = 0; q < 3; ++q) {
      t.sc.in[q] = 1.f;
      t.sc.inv_out[q] = 1.f;
      t.sc.base[q] = 1.f;
    }
    t.f64_levels = 0;
    bool ok;
    if constexpr (ADJ && std::is_same<T, float>::value)
      ok = sweep::adjoint_tile_f32v4<SPLIT>(t, R, p.flag);
    else if constexpr (ADJ)
      ok = sweep::adjoint_tile<T, SPLIT>(t, R, p.flag);
    else
      ok = sweep::forward_tile<T, false, SPLIT>(t, R, p.flag);
    if (!ok) break;  // uniform across the CTA
  }
}

template <typename T>
int vec_of(bool adj) {
  if (adj && std::is_same<T, float>::value) return sweep::a4::P;
  return adj ? sweep::AdjIO<T>::P : sweep::VecIO<T>::P;
}

// Rows per tile for a member: the most rows whose k-blocks fit 128 threads in
// whole warps (0 if none).
int member_ty(int kb) {
  if (kb > kEnsThreads) return 0;
  int ty = kEnsThreads / kb;
  while (ty > 0 && (ty * kb) % 32) --ty;
  return ty;
}

template <typename T, int OCC, int ADJ>
void* kernel_ptr(bool split) {
  return split ? (void*)ens_kernel<T, OCC, ADJ, true> : (void*)ens_kernel<T, OCC, ADJ, false>;
}

template <typename T, int ADJ>
void* kernel_for(int occ, bool split) {
  switch (occ) {
    case 4: return kernel_ptr<T, 4, ADJ>(split);
    case 3: return kernel_ptr<T, 3, ADJ>(split);
    default: return kernel_ptr<T, 2, ADJ>(split);
  }
}

}  // namespace

// ---------------------------------------------------------------- state
struct EnsDir {  // one direction (forward or adjoint)
  std::vector<unsigned char> host_desc;
  void* d_desc = nullptr;
  size_t desc_bytes = 0;
  std::vector<const void*> last_ptrs;
  int n_tiles = 0;
  size_t slot_cap = 0;
  bool split = false;  // some member's rows straddle warps
  size_t table = 0;    // shared-memory coefficient table after the ring
  EnsCfg cfg{64, 6, 4};
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  EnsCfg graph_cfg{0, 0, 0};
};

struct EnsState {
  std::vector<int> order;  // member indices, largest first
  int* d_counter = nullptr;
  EnsDir dir[2];
};

size_t ens_elem(advect_dtype d) { return d == ADVECT_F64 ? 8 : 4; }

// Fill the member table for one direction from the members and pointers.
template <typename T>
static void build_table(const advect_ctx& ctx, EnsState& st, int adj, const void* const* const* in,
                        void* const* const* out) {
  EnsDir& D = st.dir[adj];
  const int n = (int)ctx.members.size();
  std::vector<MemberDesc<T>> v(n);
  int tile = 0;
  size_t cap = 0;
  int max_nz = 0;
  bool split = false;
  const int P = vec_of<T>(adj != 0);
  for (int r = 0; r < n; ++r) {
    const int m = st.order[r];
    const Member& mm = ctx.members[m];
    MemberDesc<T>& d = v[r];
    std::memset(&d, 0, sizeof d);
    for (int f = 0; f < (adj ? 6 : 3); ++f) d.in[f] = in ? (const T*)in[f][m] : nullptr;
    for (int f = 0; f < 3; ++f) d.out[f] = out ? (T*)out[f][m] : nullptr;
    d.nx = mm.nx;
    d.ny = mm.ny;
    d.nz = mm.nz;
    d.kb = mm.nz / P;
    d.ty = member_ty(d.kb);
    d.n_jb = (mm.ny + d.ty - 1) / d.ty;
    d.n_xr = (mm.nx + D.cfg.lx - 1) / D.cfg.lx;
    d.tile_begin = tile;
    tile += d.n_jb * d.n_xr;
    d.c.d = mm.d_tabs;
    d.c.f = mm.f_tabs;
    d.c.tcx = mm.tcx;
    d.c.tcy = mm.tcy;
    d.c.tcx_f = (float)mm.tcx;
    d.c.tcy_f = (float)mm.tcy;
    cap = std::max(cap, (size_t)(adj ? 6 : 3) * (d.ty + 2) * mm.nz * sizeof(T));
    split = split || (32 % d.kb) != 0;
    max_nz = std::max(max_nz, mm.nz);
  }
  D.split = split;
  D.table = (adj && std::is_same<T, float>::value) ? sweep::a4::table_bytes(max_nz) : 0;
  D.n_tiles = tile;
  D.slot_cap = (cap + 127) / 128 * 128;
  D.host_desc.resize(v.size() * sizeof(MemberDesc<T>));
  std::memcpy(D.host_desc.data(), v.data(), D.host_desc.size());
}

size_t ens_smem_bytes(const EnsState& st, int adj, const EnsCfg& cfg) {
  return sweep::ring_bytes(cfg.nb, st.dir[adj].slot_cap) + st.dir[adj].table;
}

// Check that every member can run the ensemble sweep for this element type.
advect_status ens_check_members(const advect_ctx& ctx, std::string& why) {
  const int elem = (int)ens_elem(ctx.dtype);
  for (size_t m = 0; m < ctx.members.size(); ++m) {
    const int nz = ctx.members[m].nz;
    for (int adj = 0; adj < 2; ++adj) {
      const int P = elem == 8 ? vec_of<double>(adj != 0) : vec_of<float>(adj != 0);
      if (nz % P || (nz * elem) % 16 || member_ty(nz / P) == 0) {
        why = "member " + std::to_string(m) + ": nz = " + std::to_string(nz) +
              " not supported by the ensemble kernels (need nz * element size a multiple of 16 and"
              " nz / vector width <= 128)";
        return ADVECT_EUNSUPPORTED;
      }
    }
  }
  return ADVECT_OK;
}

EnsState* ens_new(advect_ctx& ctx) {
  EnsState* st = new (std::nothrow) EnsState();
  if (!st) return nullptr;
  const int n = (int)ctx.members.size();
  st->order.resize(n);
  std::iota(st->order.begin(), st->order.end(), 0);
  std::stable_sort(st->order.begin(), st->order.end(), [&](int a, int b) {
    const Member& x = ctx.members[a];
    const Member& y = ctx.members[b];
    return (size_t)x.nx * x.ny * x.nz > (size_t)y.nx * y.ny * y.nz;
  });
  if (cudaMalloc(&st->d_counter, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    delete st;
    return nullptr;
  }
  return st;
}

void ens_free(EnsState* st) {
  if (!st) return;
  for (auto& d : st->dir) {
    if (d.exec) cudaGraphExecDestroy(d.exec);
    if (d.graph) cudaGraphDestroy(d.graph);
    if (d.d_desc) cudaFree(d.d_desc);
  }
  if (st->d_counter) cudaFree(st->d_counter);
  delete st;
}

static cudaError_t set_smem_attr(void* fn, size_t smem) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// Number of CTAs for the persistent launch.
static int ens_grid(void* fn, size_t smem, int n_tiles) {
  int dev = 0, sms = 152, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kEnsThreads, smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return std::max(1, std::min(n_tiles, sms * per_sm));
}

// (Re)build the table for cfg, upload it on `stream` and launch the
// persistent kernel there, through the captured graph when `use_graph`.
template <typename T>
static cudaError_t ens_run_t(advect_ctx& ctx, EnsState& st, int adj, const EnsCfg& cfg,
                             const void* const* const* in, void* const* const* out, bool ptrs_changed,
                             cudaStream_t stream, bool use_graph) {
  EnsDir& D = st.dir[adj];
  const bool cfg_changed = cfg.lx != D.cfg.lx || D.host_desc.empty();
  D.cfg = cfg;
  if (cfg_changed || ptrs_changed) {
    build_table<T>(ctx, st, adj, in, out);
    if (D.desc_bytes < D.host_desc.size()) {
      if (D.d_desc) cudaFree(D.d_desc);
      D.d_desc = nullptr;
      cudaError_t e = cudaMalloc(&D.d_desc, D.host_desc.size());
      if (e != cudaSuccess) return e;
      D.desc_bytes = D.host_desc.size();
    }
    cudaError_t e = cudaMemcpyAsync(D.d_desc, D.host_desc.data(), D.host_desc.size(), cudaMemcpyHostToDevice,
                                    stream);
    if (e != cudaSuccess) return e;
  }
  void* fn = adj ? kernel_for<T, 1>(cfg.occ, D.split) : kernel_for<T, 0>(cfg.occ, D.split);
  const size_t smem = ens_smem_bytes(st, adj, cfg);
  cudaError_t e = set_smem_attr(fn, smem);
  if (e != cudaSuccess) return e;
  EnsParams p;
  p.desc = D.d_desc;
  p.n_members = (int)ctx.members.size();
  p.n_tiles = D.n_tiles;
  p.lx = cfg.lx;
  p.nb = cfg.nb;
  p.slot_cap = D.slot_cap;
  p.counter = st.d_counter;
  p.flag = ctx.d_flag;
  const int grid = ens_grid(fn, smem, D.n_tiles);
  void* args[] = {&p};
  if (!use_graph) {
    e = cudaMemsetAsync(st.d_counter, 0, sizeof(int), stream);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernel(fn, dim3(grid), dim3(kEnsThreads), args, smem, stream);
  }
  const bool same = D.exec && D.graph_cfg.lx == cfg.lx && D.graph_cfg.nb == cfg.nb && D.graph_cfg.occ == cfg.occ &&
                    !cfg_changed;
  if (!same) {
    if (D.exec) cudaGraphExecDestroy(D.exec);
    if (D.graph) cudaGraphDestroy(D.graph);
    D.exec = nullptr;
    D.graph = nullptr;
    cudaStream_t cap;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaMemsetAsync(st.d_counter, 0, sizeof(int), cap);
      cudaLaunchKernel(fn, dim3(grid), dim3(kEnsThreads), args, smem, cap);
      e = cudaStreamEndCapture(cap, &D.graph);
    }
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(&D.exec, D.graph, 0);
    if (e != cudaSuccess) return e;
    D.graph_cfg = cfg;
  }
  return cudaGraphLaunch(D.exec, stream);
}

cudaError_t ens_run(advect_ctx& ctx, EnsState& st, int adj, const EnsCfg& cfg, const void* const* const* in,
                    void* const* const* out, bool ptrs_changed, cudaStream_t stream, bool use_graph) {
  if (ctx.dtype == ADVECT_F64)
    return ens_run_t<double>(ctx, st, adj, cfg, in, out, ptrs_changed, stream, use_graph);
  return ens_run_t<float>(ctx, st, adj, cfg, in, out, ptrs_changed, stream, use_graph);
}

EnsCfg& ens_cfg(EnsState& st, int adj) { return st.dir[adj].cfg; }

bool ens_ptrs_changed(EnsState& st, int adj, const void* const* const* in, int n_in, void* const* const* out,
                      int n_members) {
  std::vector<const void*> cur;
  cur.reserve((size_t)(n_in + 3) * n_members);
  for (int f = 0; f < n_in; ++f)
    for (int m = 0; m < n_members; ++m) cur.push_back(in[f][m]);
  for (int f = 0; f < 3; ++f)
    for (int m = 0; m < n_members; ++m) cur.push_back(out[f][m]);
  if (cur == st.dir[adj].last_ptrs) return false;
  st.dir[adj].last_ptrs.swap(cur);
  return true;
}

}  // namespace advect
