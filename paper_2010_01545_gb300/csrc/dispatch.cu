// dispatch.cu -- kernel selection, context resources.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstdlib>

#include "ctx.h"
#include "ens.h"
#include "sweep_core.cuh"
#include "sweep_ff.cuh"
#include "tune.h"

#include <functional>
#include <string>
#include <vector>

namespace advect {

namespace {

int elem_of(int dtype) { return (dtype == kF64 || dtype == kF64FF) ? 8 : (dtype == kF32 ? 4 : 2); }

bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

}  // namespace

// Default plane-sweep tile for a column height and element size; ty = 0 when
// the sweep kernel cannot take this shape.
SweepCfg default_sweep(int nz, int elem) { return default_sweep_vec(nz, elem, sweep_vec(elem)); }

// The same for vectors of P levels per thread.
SweepCfg default_sweep_vec(int nz, int elem, int P) {
  SweepCfg c{0, 64, 4, 1};
  if (nz % P || (nz * elem) % 16) return c;
  const int kb = nz / P;
  if (kb > 256) return c;
  // ~128 threads per CTA: at ~150-170 registers per thread three CTAs fit
  // per SM, which hides latency better than one 256-thread CTA (measured
  // on the 2048 x 2048 x 64 grid).
  int ty = kb >= 128 ? 1 : 128 / kb;
  while (ty > 1 && (ty * kb) % 32) --ty;
  if ((ty * kb) % 32) {
    ty = 256 / kb;
    while (ty > 1 && (ty * kb) % 32) --ty;
    if ((ty * kb) % 32) return c;
  }
  c.ty = ty;
  // FP32/F16S: registers capped for four 128-thread CTAs per SM (no spills),
  // which beat three or one larger CTA on the 2048 x 2048 x 64 grid; the ring
  // then gets a quarter of the SM's shared memory.  FP64 is bound by the FP64
  // pipe and keeps the uncapped allocation.
  c.occ = (elem <= 4 && ty * kb <= 128) ? 4 : 1;
  const size_t cap = c.occ == 4 ? 54 * 1024 : 72 * 1024;
  c.nb = elem == 2 ? 12 : (elem == 4 ? 6 : 7);
  while (c.nb > 4 && sweep_smem_bytes(nz, elem, c) > cap) --c.nb;
  while (c.ty > 1 && sweep_smem_bytes(nz, elem, c) > 220 * 1024) {
    int t = c.ty - 1;
    while (t > 1 && (t * kb) % 32) --t;
    if ((t * kb) % 32) break;
    c.ty = t;
  }
  if (sweep_smem_bytes(nz, elem, c) > 220 * 1024 || (uint64_t)3 * (c.ty + 2) * nz * elem >= (1u << 20))
    c.ty = 0;
  return c;
}

// A tile override "ty,lx,nb[,occ]" from the environment (ignored unless valid):
// ADVECT_SWEEP for the forward, ADVECT_ADJ_SWEEP for the adjoint.
static void sweep_override(const char* var, SweepCfg& c, int nz, int elem, int vec, int nf) {
  const char* s = getenv(var);
  if (!s || c.ty == 0) return;
  SweepCfg o{0, 0, 0, 1};
  const int n = sscanf(s, "%d,%d,%d,%d", &o.ty, &o.lx, &o.nb, &o.occ);
  if (n < 3) return;
  if (n == 3) o.occ = 1;
  const int kb = nz / vec;
  if (o.ty < 1 || o.lx < 1 || o.nb < 4 || o.ty * kb > 256 || (o.ty * kb) % 32) return;
  if (o.occ < 1 || o.occ > 4) return;
  if (o.occ > 2 && o.ty * kb > 128) return;
  if (o.occ == 2 && o.ty * kb > 224) return;
  const size_t smem = sweep::ring_bytes(o.nb, (size_t)nf * (o.ty + 2) * nz * elem);
  if (smem > 220 * 1024 || (uint64_t)nf * (o.ty + 2) * nz * elem >= (1u << 20)) return;
  c = o;
}

// ADVECT_ADJ_SWEEP "ty,lx,nb[,occ]" for the double-float adjoint's own sweep
// (two levels per thread); false (nothing changed) unless set and valid there.
static bool adj_ff_override(SweepCfg& c, int nz) {
  const char* s = getenv("ADVECT_ADJ_SWEEP");
  if (!s) return false;
  SweepCfg o{0, 0, 0, 1};
  const int n = sscanf(s, "%d,%d,%d,%d", &o.ty, &o.lx, &o.nb, &o.occ);
  if (n < 3 || !adj_ff_fits(nz, o)) return false;
  o.occ = 1;
  c = o;
  return true;
}

// Default adjoint tile (six streamed fields): 128 threads with registers
// capped for four CTAs per SM (binary32) or three (8-byte types: binary64
// and double-float; measured at 1024 x 1024 x 128 against one uncapped
// 256-thread CTA: double-float 15.9 against 14.9 Gpts/s, binary64 6.08
// against 6.00); one uncapped 256-thread CTA for 8-byte columns of more than
// 128 levels; ty = 0 when the shape does not fit the sweep.
SweepCfg default_adj_sweep(int nz, int elem) {
  SweepCfg c{0, 64, 4, 1};
  if (elem != 8 && elem != 4) return c;
  const int P = adj_sweep_vec(elem);
  if (nz % P || (nz * elem) % 16) return c;
  const int kb = nz / P;
  const int target = (elem == 8 && kb > 128) ? 256 : 128;
  if (kb > target) return c;
  int ty = target / kb;
  while (ty > 1 && (ty * kb) % 32) --ty;
  if ((ty * kb) % 32) return c;
  c.ty = ty;
  // binary32 (4 levels per thread, adj_f32.cuh): code for <= 168 registers
  // (167, no spills) and three CTAs per SM, whose rings and coefficient
  // tables must then fit a third of the SM's shared memory (measured at
  // 1024 x 1024 x 128: 136.4 Gpts/s; uncapped at two CTAs per SM 115.5;
  // capped at 128 registers for four CTAs, spilling, 54)
  c.occ = target == 256 ? 1 : 3;
  const size_t cap = elem == 4 ? 75 * 1024 : (c.occ == 3 ? 72 * 1024 : 100 * 1024);
  c.nb = 8;
  while (c.nb > 4 && adj_sweep_smem_bytes(nz, elem, c) > cap) --c.nb;
  if (adj_sweep_smem_bytes(nz, elem, c) > 220 * 1024 || (uint64_t)6 * (c.ty + 2) * nz * elem >= (1u << 20))
    c.ty = 0;
  return c;
}

namespace {

const char* dname(int d) { return d == kF64 ? "f64" : (d == kF32 ? "f32" : (d == kF64FF ? "f64ff" : "f16s")); }

std::string single_key(const advect_ctx& ctx, int adj) {
  const Member& m = ctx.members[0];
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  char buf[128];
  snprintf(buf, sizeof buf, "%s|%s|%dx%dx%d|sm%d", adj ? "adj" : "fwd", dname((int)ctx.dtype), m.nx, m.ny, m.nz,
           sms);
  return buf;
}

std::string fmt_cfg(int kind, const SweepCfg& c) {
  if (kind == 0) return "point";
  char buf[64];
  snprintf(buf, sizeof buf, "%d,%d,%d,%d", c.ty, c.lx, c.nb, c.occ);
  return buf;
}

// Parse a cached choice; validates against the shape like the env override.
bool parse_cfg(const std::string& v, int nz, int elem, int vec, int nf, int& kind, SweepCfg& c) {
  if (v == "point") {
    kind = 0;
    return true;
  }
  SweepCfg o{0, 0, 0, 1};
  if (sscanf(v.c_str(), "%d,%d,%d,%d", &o.ty, &o.lx, &o.nb, &o.occ) != 4) return false;
  if (nz % vec || (nz * elem) % 16) return false;
  const int kb = nz / vec;
  if (o.ty < 1 || o.lx < 1 || o.nb < 4 || o.ty * kb > 256 || (o.ty * kb) % 32) return false;
  if (o.occ < 1 || o.occ > 4) return false;
  if (o.occ > 2 && o.ty * kb > 128) return false;
  if (o.occ == 2 && o.ty * kb > 224) return false;
  if (sweep::ring_bytes(o.nb, (size_t)nf * (o.ty + 2) * nz * elem) > 220 * 1024) return false;
  kind = 1;
  c = o;
  return true;
}

// Candidate tiles for a column height: 128-thread tiles with register caps
// for 4 or 3 CTAs per SM, 224-thread tiles for 2 (the double-float sweep's
// converter warp makes them 256) and up-to-256-thread tiles without cap, over x-range
// lengths and ring depths that fit the shared memory of those CTAs.
std::vector<SweepCfg> candidates(int nz, int elem, int vec, int nf) {
  std::vector<SweepCfg> out;
  if (nz % vec || (nz * elem) % 16) return out;
  const int kb = nz / vec;
  for (int occ : {4, 3, 2, 1}) {
    const int threads = occ == 1 ? 256 : occ == 2 ? 224 : 128;
    if (kb > threads) continue;
    int ty = threads / kb;
    while (ty > 1 && (ty * kb) % 32) --ty;
    if ((ty * kb) % 32) continue;
    for (int lx : {32, 64, 128})
      for (int nb : {4, 6, 8, 12}) {
        SweepCfg c{ty, lx, nb, occ};
        const size_t smem = sweep::ring_bytes(nb, (size_t)nf * (ty + 2) * nz * elem);
        // a ring too large for `occ` CTAs per SM still runs (at fewer CTAs)
        // and the register cap alone can pay, so only the per-CTA limit prunes
        if (smem > 220 * 1024) continue;
        if ((uint64_t)nf * (ty + 2) * nz * elem >= (1u << 20)) continue;
        out.push_back(c);
      }
  }
  return out;
}

float time_ms(cudaStream_t st, const std::function<cudaError_t()>& fn, cudaError_t& err) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  err = fn();
  cudaEventRecord(a, st);
  const int reps = 2;
  for (int r = 0; r < reps && err == cudaSuccess; ++r) err = fn();
  cudaEventRecord(b, st);
  cudaEventSynchronize(b);
  float ms = 0;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms / reps;
}

}  // namespace

// Time the point kernel and every candidate tile on the call's buffers, keep
// the fastest (in the context and the tuning cache).  The caller then runs
// the call with the chosen kernel.
cudaError_t tune_single(advect_ctx& ctx, int adj, const FwdArgs* fa, const AdjArgs* aa, cudaStream_t st) {
  const Member& m = ctx.members[0];
  const int elem = elem_of((int)ctx.dtype);
  const int vec = adj ? adj_sweep_vec(elem) : sweep_vec(elem);
  const int nf = adj ? 6 : 3;
  int& kind = adj ? ctx.adj_kind : ctx.fwd_kind;
  SweepCfg& cfg = adj ? ctx.adj_sweep : ctx.sweep;
  int best_kind = 0;
  SweepCfg best = cfg;
  cudaError_t e = cudaSuccess;
  float best_ms = time_ms(st, [&]() {
    return adj ? launch_adj_point((int)ctx.dtype, *aa, st) : launch_fwd_point((int)ctx.dtype, *fa, st);
  }, e);
  if (e != cudaSuccess) return e;
  if (!(adj && ctx.dtype == ADVECT_F16S)) {
    // the context's current tile competes too (the double-float adjoint's
    // default is not among the generic candidates)
    std::vector<SweepCfg> cands = candidates(m.nz, elem, vec, nf);
    if (kind == 1) cands.insert(cands.begin(), cfg);
    for (const SweepCfg& c : cands) {
      const float ms = time_ms(st, [&]() {
        return adj ? launch_adj_sweep((int)ctx.dtype, *aa, fit_planes(c, aa->s.nx), ctx.d_flag, st)
                   : launch_fwd_sweep((int)ctx.dtype, *fa, fit_planes(c, fa->i1 - fa->i0), ctx.d_flag, st);
      }, e);
      if (e != cudaSuccess) return e;
      if (ms < best_ms) {
        best_ms = ms;
        best = c;
        best_kind = 1;
      }
    }
  }
  kind = best_kind;
  if (best_kind) cfg = best;
  const std::string name = adj ? (kind ? "adj_sweep" : "adj_point") : (kind ? "fwd_sweep" : "fwd_point");
  (adj ? ctx.adj_name : ctx.fwd_name) = name;
  tune_cache_put(single_key(ctx, adj), fmt_cfg(kind, cfg));
  return cudaSuccess;
}

SweepCfg default_fwd_sweep(int nz, int dtype) {
  const int elem = elem_of(dtype);
  SweepCfg c = default_sweep(nz, elem);
  if (dtype == kF64FF && c.ty > 0 && ff_sweep_fits(nz)) {
    // converter-warp sweep: seven compute warps and the converter warp, two
    // CTAs per SM (128 registers a thread), a ring of up to 8 slots
    c.ty = 224 / (nz / sweep_vec(elem));
    c.occ = 2;
    c.nb = 8;
    while (c.nb > 4 && sweep_smem_bytes(nz, elem, c) + sweep::ff_extra_bytes(c.nb, nz) > 110 * 1024) --c.nb;
  } else if (dtype == kF64FF && c.ty > 0 && c.ty * (nz / sweep_vec(elem)) <= 128) {
    // double-float arithmetic is bound by the binary32 issue rate: four CTAs
    // per SM with the code compiled for <= 128 registers (a few spilled
    // values) and a ring that lets four fit (measured at 2048 x 2048 x 64:
    // 48.4 Gpts/s with 5 slots, 47.9 with 6, 44.3 with the <= 168-register
    // build at three CTAs)
    c.occ = 4;
    while (c.nb > 4 && sweep_smem_bytes(nz, elem, c) > 47 * 1024) --c.nb;
  }
  // F16S: 40-plane tiles (measured at 2048 x 2048 x 64, same box: 389-392
  // against 386-388 Gpts/s with 64-plane tiles; 32, 48, 80 and 96 in between
  // or slower)
  if (dtype == kF16S && c.ty > 0) c.lx = 40;
  return c;
}

void select_kernels(advect_ctx& ctx) {
  const Member& m = ctx.members[0];
  const int elem = elem_of((int)ctx.dtype);
  ctx.sweep = default_fwd_sweep(m.nz, (int)ctx.dtype);
  sweep_override("ADVECT_SWEEP", ctx.sweep, m.nz, elem, sweep_vec(elem), 3);
  ctx.fwd_kind = ctx.sweep.ty > 0 ? 1 : 0;
  ctx.fwd_name = ctx.fwd_kind ? "fwd_sweep" : "fwd_point";
  ctx.adj_sweep = default_adj_sweep(m.nz, elem);
  const SweepCfg aff = ctx.dtype == ADVECT_F64_FF ? default_adj_ff(m.nz) : SweepCfg{0, 0, 0, 1};
  if (aff.ty > 0) {
    // double-float adjoint with its own sweep (adj_ff.cuh)
    ctx.adj_sweep = aff;
  } else if (ctx.dtype == ADVECT_F64_FF && ctx.adj_sweep.ty > 0) {
    // double-float adjoint: 128-plane tiles where the grid still gives at
    // least eight CTAs per resident slot on the device's SMs (measured on
    // 152 SMs: 16.2 against 15.8 Gpts/s at 1024 x 1024 x 128; at 512 x 512 x
    // 128, four per slot, 2.23 against 2.19 ms, so smaller grids keep
    // 64-plane tiles)
    const long long ctas = (long long)((m.nx + 127) / 128) * ((m.ny + ctx.adj_sweep.ty - 1) / ctx.adj_sweep.ty);
    if (ctas >= 8LL * ctx.sms * ctx.adj_sweep.occ) ctx.adj_sweep.lx = 128;
  }
  if (!(aff.ty > 0 && adj_ff_override(ctx.adj_sweep, m.nz)))
    sweep_override("ADVECT_ADJ_SWEEP", ctx.adj_sweep, m.nz, elem, adj_sweep_vec(elem), 6);
  ctx.adj_kind = ctx.adj_sweep.ty > 0 ? 1 : 0;
  // a tuned choice from the cache wins over the defaults; an environment
  // override wins over both
  for (int adj = 0; adj < 2; ++adj) {
    std::string v;
    const char* env = getenv(adj ? "ADVECT_ADJ_SWEEP" : "ADVECT_SWEEP");
    if (env || !tune_cache_get(single_key(ctx, adj), v)) continue;
    int kind = 0;
    SweepCfg c{0, 0, 0, 1};
    if (adj && ctx.dtype == ADVECT_F16S) continue;
    if (parse_cfg(v, m.nz, elem, adj ? adj_sweep_vec(elem) : sweep_vec(elem), adj ? 6 : 3, kind, c)) {
      (adj ? ctx.adj_kind : ctx.fwd_kind) = kind;
      if (kind) (adj ? ctx.adj_sweep : ctx.sweep) = c;
    }
  }
  ctx.fwd_name = ctx.fwd_kind ? "fwd_sweep" : "fwd_point";
  ctx.adj_name = ctx.adj_kind ? "adj_sweep" : "adj_point";
  ctx.tune_fwd = ctx.tune_adj = tune_env_enabled();
  if (const char* h = getenv("ADVECT_HOST_CHUNKS")) {
    const int n = atoi(h);
    if (n >= 1 && n <= HostPath::kMaxChunks) ctx.hp.nchunk = n;
  }
  if (const char* q = getenv("ADVECT_TEST_SKIP_PLANE")) ctx.test_skip_plane = atoi(q);
  if (const char* b = getenv("ADVECT_TEST_WAIT_CYCLES")) {
    const long long v = atoll(b);
    if (v > 0) ctx.wait_budget = v;
  }
}

cudaError_t launch_fwd(const advect_ctx& ctx, const FwdArgs& a, cudaStream_t st) {
  if (ctx.fwd_kind == 1 && aligned16(a.u) && aligned16(a.v) && aligned16(a.w) && aligned16(a.su) &&
      aligned16(a.sv) && aligned16(a.sw) && aligned16(a.bu) && aligned16(a.bv) && aligned16(a.bw))
    return launch_fwd_sweep((int)ctx.dtype, a, fit_planes(ctx.sweep, a.i1 - a.i0), ctx.d_flag, st);
  return launch_fwd_point((int)ctx.dtype, a, st);
}

cudaError_t launch_adj(const advect_ctx& ctx, const AdjArgs& a, cudaStream_t st) {
  if (ctx.adj_kind == 1 && aligned16(a.u) && aligned16(a.v) && aligned16(a.w) && aligned16(a.dsu) &&
      aligned16(a.dsv) && aligned16(a.dsw) && aligned16(a.du) && aligned16(a.dv) && aligned16(a.dw))
    return launch_adj_sweep((int)ctx.dtype, a, fit_planes(ctx.adj_sweep, a.s.nx), ctx.d_flag, st);
  return launch_adj_point((int)ctx.dtype, a, st);
}

}  // namespace advect

advect_status advect_ctx::ensure_host_path(size_t bytes) {
  using namespace advect;
  if (hp.bytes == bytes && hp.d_in[0]) return ADVECT_OK;
  for (int f = 0; f < 3; ++f) {
    if (hp.d_in[f]) cudaFree(hp.d_in[f]);
    if (hp.d_out[f]) cudaFree(hp.d_out[f]);
    hp.d_in[f] = hp.d_out[f] = nullptr;
  }
  hp.bytes = 0;
  for (int f = 0; f < 3; ++f) {
    if (cudaMalloc(&hp.d_in[f], bytes) != cudaSuccess || cudaMalloc(&hp.d_out[f], bytes) != cudaSuccess) {
      cudaGetLastError();
      return ADVECT_ENOMEM;
    }
  }
  if (!hp.s_in) {
    if (cudaStreamCreateWithFlags(&hp.s_in, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&hp.s_k, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&hp.s_out, cudaStreamNonBlocking) != cudaSuccess)
      return ADVECT_ECUDA;
    for (int c = 0; c < HostPath::kMaxChunks; ++c)
      if (cudaEventCreateWithFlags(&hp.ev_in[c], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&hp.ev_k[c], cudaEventDisableTiming) != cudaSuccess)
        return ADVECT_ECUDA;
  }
  hp.bytes = bytes;
  return ADVECT_OK;
}

void advect_ctx::release() {
  using namespace advect;
  cudaDeviceSynchronize();
  if (ens) ens_free(static_cast<EnsState*>(ens));
  ens = nullptr;
  for (auto& m : members)
    if (m.d_tabs) cudaFree(m.d_tabs);
  members.clear();
  if (d_flag) cudaFree(d_flag);
  d_flag = nullptr;
  for (int f = 0; f < 3; ++f) {
    if (hp.d_in[f]) cudaFree(hp.d_in[f]);
    if (hp.d_out[f]) cudaFree(hp.d_out[f]);
  }
  for (int c = 0; c < HostPath::kMaxChunks; ++c) {
    if (hp.ev_in[c]) cudaEventDestroy(hp.ev_in[c]);
    if (hp.ev_k[c]) cudaEventDestroy(hp.ev_k[c]);
  }
  if (hp.s_in) cudaStreamDestroy(hp.s_in);
  if (hp.s_k) cudaStreamDestroy(hp.s_k);
  if (hp.s_out) cudaStreamDestroy(hp.s_out);
}
