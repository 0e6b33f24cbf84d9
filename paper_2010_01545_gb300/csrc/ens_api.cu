// ens_api.cu -- C ABI of ensembles and of the autotuner.
//
// Autotuning: when enabled for a context (advect_autotune, or ADVECT_TUNE=1
// in the environment at create time), the next forward and the next adjoint
// call time every candidate tile configuration on that call's own buffers
// with CUDA events, keep the fastest, store it in the tuning cache
// (tune.h) and finish with the winner, so the call's outputs are those of
// the chosen kernel.  Contexts created later with the same key start from the
// cached choice.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <functional>
#include <string>
#include <vector>

#include "../../include/advect.h"
#include "abi_util.h"
#include "ctx.h"
#include "ens.h"
#include "tune.h"

using namespace advect;
using namespace advect::abi;

namespace {

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

const char* dtype_name(advect_dtype d) { return d == ADVECT_F64 ? "f64" : (d == ADVECT_F32 ? "f32" : "other"); }

std::string ens_key(const advect_ctx& ctx, int adj) {
  // FNV-1a over the member shapes
  unsigned long long h = 1469598103934665603ull;
  for (const auto& m : ctx.members)
    for (int v : {m.nx, m.ny, m.nz}) {
      h ^= (unsigned long long)(unsigned)v;
      h *= 1099511628211ull;
    }
  char buf[128];
  snprintf(buf, sizeof buf, "ens_%s|%s|n%zu|%016llx|sm%d", adj ? "adj" : "fwd", dtype_name(ctx.dtype),
           ctx.members.size(), h, sm_count());
  return buf;
}

bool parse_ens_cfg(const std::string& s, EnsCfg& c) {
  EnsCfg o{0, 0, 0};
  if (sscanf(s.c_str(), "%d,%d,%d", &o.lx, &o.nb, &o.occ) != 3) return false;
  if (o.lx < 1 || o.nb < 4 || o.nb > 16 || (o.occ != 2 && o.occ != 3 && o.occ != 4)) return false;
  c = o;
  return true;
}

std::string fmt_ens_cfg(const EnsCfg& c) {
  char buf[64];
  snprintf(buf, sizeof buf, "%d,%d,%d", c.lx, c.nb, c.occ);
  return buf;
}

float time_launches(cudaStream_t st, int reps, const std::function<cudaError_t()>& fn, cudaError_t& err) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  err = fn();  // warm-up
  cudaEventRecord(a, st);
  for (int r = 0; r < reps && err == cudaSuccess; ++r) err = fn();
  cudaEventRecord(b, st);
  cudaEventSynchronize(b);
  float ms = 0;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms / reps;
}

// Validate the member buffers of an ensemble call.
advect_status check_members(advect_ctx* ctx, const void* const* const* in, int n_in, void* const* const* out,
                            const char* const* names) {
  const int n = (int)ctx->members.size();
  const size_t eb = elem_bytes(ctx->dtype);
  for (int f = 0; f < n_in; ++f)
    if (!in[f]) return fail(ADVECT_EINVAL, "pointer array %s is NULL", names[f]);
  for (int f = 0; f < 3; ++f)
    if (!out[f]) return fail(ADVECT_EINVAL, "pointer array %s is NULL", names[n_in + f]);
  std::vector<std::pair<const void*, size_t>> ins, outs;
  for (int m = 0; m < n; ++m) {
    const Member& mm = ctx->members[m];
    const size_t bytes = (size_t)mm.nx * mm.ny * mm.nz * eb;
    for (int f = 0; f < n_in + 3; ++f) {
      const void* p = f < n_in ? in[f][m] : out[f - n_in][m];
      advect_status s = check_device_ptr(p, names[f], eb, ctx->device);
      if (s) return fail(s, "member %d: %s", m, g_last_error.c_str());
      if ((uintptr_t)p & 15) return fail(ADVECT_EINVAL, "member %d: %s is not 16-byte aligned", m, names[f]);
      (f < n_in ? ins : outs).push_back({p, bytes});
    }
  }
  for (size_t o = 0; o < outs.size(); ++o) {
    for (const auto& i : ins) {
      const uintptr_t a = (uintptr_t)outs[o].first, b = (uintptr_t)i.first;
      if (a < b + i.second && b < a + outs[o].second) return fail(ADVECT_EINVAL, "an output overlaps an input");
    }
    for (size_t q = o + 1; q < outs.size(); ++q) {
      const uintptr_t a = (uintptr_t)outs[o].first, b = (uintptr_t)outs[q].first;
      if (a < b + outs[q].second && b < a + outs[o].second) return fail(ADVECT_EINVAL, "two outputs overlap");
    }
  }
  return ADVECT_OK;
}

advect_status ens_call(advect_ctx* ctx, int adj, const void* const* const* in, void* const* const* out,
                       cudaStream_t stream) {
  EnsState& st = *static_cast<EnsState*>(ctx->ens);
  const int n = (int)ctx->members.size();
  const int n_in = adj ? 6 : 3;
  const bool changed = ens_ptrs_changed(st, adj, in, n_in, out, n);
  if (changed) {
    static const char* fwd_names[6] = {"u", "v", "w", "su", "sv", "sw"};
    static const char* adj_names[9] = {"u", "v", "w", "dsu", "dsv", "dsw", "du", "dv", "dw"};
    advect_status s = check_members(ctx, in, n_in, out, adj ? adj_names : fwd_names);
    if (s) {
      ens_ptrs_changed(st, adj, nullptr, 0, nullptr, 0);  // forget the rejected set
      return s;
    }
  }
  bool& tune = adj ? ctx->tune_adj : ctx->tune_fwd;
  if (tune) {
    tune = false;
    const int elem = (int)elem_bytes(ctx->dtype);
    EnsCfg best = ens_cfg(st, adj);
    float best_ms = 1e30f;
    for (int occ : {4, 3, 2})
      for (int lx : {16, 32, 64, 128})
        for (int nb : {4, 6, 8, 12}) {
          EnsCfg c{lx, nb, occ};
          if (ens_smem_bytes(st, adj, c) * occ > 225 * 1024 && occ > 2) continue;
          if (ens_smem_bytes(st, adj, c) > 220 * 1024) continue;
          cudaError_t e = cudaSuccess;
          const float ms = time_launches(stream, 2, [&]() {
            return ens_run(*ctx, st, adj, c, in, out, true, stream, false);
          }, e);
          if (e != cudaSuccess) return cuda_fail(e, "ensemble tuning launch");
          if (ms < best_ms) {
            best_ms = ms;
            best = c;
          }
        }
    (void)elem;
    ens_cfg(st, adj) = best;
    tune_cache_put(ens_key(*ctx, adj), fmt_ens_cfg(best));
    cudaError_t e = ens_run(*ctx, st, adj, best, in, out, true, stream, true);
    if (e != cudaSuccess) return cuda_fail(e, "ensemble launch");
    return ADVECT_OK;
  }
  cudaError_t e = ens_run(*ctx, st, adj, ens_cfg(st, adj), in, out, changed, stream, true);
  if (e != cudaSuccess) return cuda_fail(e, "ensemble launch");
  return ADVECT_OK;
}

}  // namespace

extern "C" {

advect_status advect_ensemble_create(int n, const int* nx, const int* ny, const int* nz, const advect_coeffs* c,
                                     advect_dtype dtype, advect_ctx** out) {
  if (!out) return fail(ADVECT_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1 || !nx || !ny || !nz || !c) return fail(ADVECT_EINVAL, "need n >= 1 and non-NULL shape/coefficient arrays");
  if (!valid_dtype(dtype)) return fail(ADVECT_EINVAL, "unknown dtype %d", (int)dtype);
  if (dtype == ADVECT_F16S || dtype == ADVECT_F64_FF) return fail(ADVECT_EUNSUPPORTED, "ensembles support F64 and F32");
  for (int m = 0; m < n; ++m) {
    advect_status s = check_shape(nx[m], ny[m], nz[m]);
    if (s) return fail(s, "member %d: %s", m, g_last_error.c_str());
    s = check_coeffs(&c[m], nz[m]);
    if (s) return fail(s, "member %d: %s", m, g_last_error.c_str());
  }
  advect_ctx* ctx = new (std::nothrow) advect_ctx();
  if (!ctx) return fail(ADVECT_ENOMEM, "host allocation failed");
  ctx->ensemble = true;
  ctx->dtype = dtype;
  ctx->members.resize(n);
  std::string why;
  for (int m = 0; m < n; ++m) {
    ctx->members[m].nx = nx[m];
    ctx->members[m].ny = ny[m];
    ctx->members[m].nz = nz[m];
  }
  advect_status s = ens_check_members(*ctx, why);  // host-only checks come first
  if (s) {
    delete ctx;
    return fail(s, "%s", why.c_str());
  }
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e != cudaSuccess) {
    delete ctx;
    return cuda_fail(e, "cudaGetDevice");
  }
  for (int m = 0; m < n; ++m) {
    s = upload_member(ctx->members[m], &c[m]);
    if (s) {
      advect_destroy(ctx);
      return s;
    }
  }
  e = cudaMalloc(&ctx->d_flag, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(ctx->d_flag, 0, sizeof(int));
  if (e != cudaSuccess) {
    advect_destroy(ctx);
    return fail(ADVECT_ENOMEM, "device error flag: %s", cudaGetErrorString(e));
  }
  EnsState* st = ens_new(*ctx);
  if (!st) {
    advect_destroy(ctx);
    return fail(ADVECT_ENOMEM, "ensemble state");
  }
  ctx->ens = st;
  for (int adj = 0; adj < 2; ++adj) {
    EnsCfg& cfg = ens_cfg(*st, adj);
    // the binary32 adjoint (4 levels per thread) is built for three CTAs
    // per SM (167 registers) and its ring must then fit a third of the SM
    cfg = (adj && dtype == ADVECT_F32) ? EnsCfg{64, 4, 3} : EnsCfg{64, 6, 4};
    std::string v;
    if (tune_cache_get(ens_key(*ctx, adj), v)) parse_ens_cfg(v, cfg);
  }
  ctx->fwd_name = "ens_fwd";
  ctx->adj_name = "ens_adj";
  ctx->tune_fwd = ctx->tune_adj = tune_env_enabled();
  *out = ctx;
  return ADVECT_OK;
}

advect_status advect_ensemble_forward(advect_ctx* ctx, const void* const* u, const void* const* v,
                                      const void* const* w, void* const* su, void* const* sv, void* const* sw,
                                      advect_stream stream) {
  if (!ctx) return fail(ADVECT_EINVAL, "context is NULL");
  if (!ctx->ensemble) return fail(ADVECT_EINVAL, "not an ensemble context: use advect_forward");
  const void* const* in[3] = {u, v, w};
  void* const* out[3] = {su, sv, sw};
  return ens_call(ctx, 0, in, out, (cudaStream_t)stream);
}

advect_status advect_ensemble_adjoint(advect_ctx* ctx, const void* const* u, const void* const* v,
                                      const void* const* w, const void* const* dsu, const void* const* dsv,
                                      const void* const* dsw, void* const* du, void* const* dv, void* const* dw,
                                      advect_stream stream) {
  if (!ctx) return fail(ADVECT_EINVAL, "context is NULL");
  if (!ctx->ensemble) return fail(ADVECT_EINVAL, "not an ensemble context: use advect_adjoint");
  const void* const* in[6] = {u, v, w, dsu, dsv, dsw};
  void* const* out[3] = {du, dv, dw};
  return ens_call(ctx, 1, in, out, (cudaStream_t)stream);
}

advect_status advect_autotune(advect_ctx* ctx, int enable) {
  if (!ctx) return fail(ADVECT_EINVAL, "context is NULL");
  ctx->tune_fwd = ctx->tune_adj = enable != 0;
  return ADVECT_OK;
}

const char* advect_tuned_config(const advect_ctx* ctx, int adjoint) {
  if (!ctx) return "";
  advect_ctx* c = const_cast<advect_ctx*>(ctx);
  char buf[96];
  if (ctx->ensemble) {
    const EnsCfg& e = ens_cfg(*static_cast<EnsState*>(c->ens), adjoint ? 1 : 0);
    snprintf(buf, sizeof buf, "lx=%d,nb=%d,occ=%d", e.lx, e.nb, e.occ);
  } else {
    const SweepCfg& s = adjoint ? ctx->adj_sweep : ctx->sweep;
    const int kind = adjoint ? ctx->adj_kind : ctx->fwd_kind;
    if (kind == 0) snprintf(buf, sizeof buf, "point");
    else snprintf(buf, sizeof buf, "ty=%d,lx=%d,nb=%d,occ=%d", s.ty, s.lx, s.nb, s.occ);
  }
  c->cfg_text[adjoint ? 1 : 0] = buf;
  return c->cfg_text[adjoint ? 1 : 0].c_str();
}

}  // extern "C"
