// api.cu -- the C ABI declared in include/advect.h.
//
// Host-side runtime: argument validation, per-context device state
// (coefficient tables, error flag, staging buffers), kernel selection and
// the chunked host-buffer pipeline.  No C++ exception crosses the ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/advect.h"
#include "abi_util.h"
#include "ctx.h"
#include "kernels.h"

using namespace advect;
using namespace advect::abi;

namespace advect {
namespace abi {

thread_local std::string g_last_error;

advect_status fail(advect_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

advect_status cuda_fail(cudaError_t e, const char* what) {
  return fail(ADVECT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CUDA_TRY(call, what)                         \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

size_t elem_bytes(advect_dtype d) { return (d == ADVECT_F64 || d == ADVECT_F64_FF) ? 8 : (d == ADVECT_F32 ? 4 : 2); }

bool valid_dtype(int d) { return d == ADVECT_F64 || d == ADVECT_F32 || d == ADVECT_F16S || d == ADVECT_F64_FF; }

// Host copy of one member's tables with the entries no formula reads set to
// zero, and tzc2[nz-1] = 0 (Listing 1 drops the upper flux at the top).
void masked_tables(const advect_coeffs* c, int nz, double* t) {
  for (size_t q = 0; q < 4 * (size_t)nz; ++q) t[q] = 0.0;
  for (int k = 1; k < nz; ++k) {
    t[k] = c->tzc1[k];
    if (k < nz - 1) t[nz + k] = c->tzc2[k];
  }
  for (int k = 1; k < nz - 1; ++k) {
    t[2 * nz + k] = c->tzd1[k];
    t[3 * nz + k] = c->tzd2[k];
  }
}

void masked_tables(const advect_coeffs* c, int nz, std::vector<double>& t) {
  t.resize(4 * (size_t)nz);
  masked_tables(c, nz, t.data());
}

bool is_finite(double x) { return std::isfinite(x); }

// F16S scales: positive, finite powers of two (the sweep folds the input
// scales into the constants, which is exact only for powers of two).
advect_status check_f16s_scales(const float* s, int n) {
  for (int q = 0; q < n; ++q) {
    int e = 0;
    if (!(s[q] > 0.f) || !std::isfinite(s[q]) || std::frexp(s[q], &e) != 0.5f)
      return fail(ADVECT_EINVAL, "scale %d (%g) must be a positive, finite power of two", q, (double)s[q]);
  }
  return ADVECT_OK;
}

advect_status check_coeffs(const advect_coeffs* c, int nz) {
  if (!c) return fail(ADVECT_EINVAL, "coefficients pointer is NULL");
  if (!c->tzc1 || !c->tzc2 || !c->tzd1 || !c->tzd2)
    return fail(ADVECT_EINVAL, "a coefficient table pointer is NULL");
  if (!is_finite(c->tcx) || !is_finite(c->tcy)) return fail(ADVECT_EINVAL, "tcx/tcy not finite");
  for (int k = 0; k < nz; ++k)
    if (!is_finite(c->tzc1[k]) || !is_finite(c->tzc2[k]) || !is_finite(c->tzd1[k]) || !is_finite(c->tzd2[k]))
      return fail(ADVECT_EINVAL, "coefficient table entry %d not finite", k);
  return ADVECT_OK;
}

advect_status check_shape(int nx, int ny, int nz) {
  if (nx < 1 || ny < 1 || nz < 3)
    return fail(ADVECT_EINVAL, "invalid shape %d x %d x %d (need nx, ny >= 1, nz >= 3)", nx, ny, nz);
  if ((double)nx * ny * nz > 4.0e12) return fail(ADVECT_EINVAL, "grid too large");
  return ADVECT_OK;
}

// Upload one member's tables (binary64 + binary32 copies).
advect_status upload_member(Member& m, const advect_coeffs* c) {
  std::vector<double> t;
  masked_tables(c, m.nz, t);
  m.h_tabs = t;
  std::vector<float> tf(t.size());
  for (size_t q = 0; q < t.size(); ++q) tf[q] = (float)t[q];
  m.tcx = c->tcx;
  m.tcy = c->tcy;
  const size_t bd = t.size() * sizeof(double), bf = tf.size() * sizeof(float);
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bd + bf);
  if (e != cudaSuccess) return fail(ADVECT_ENOMEM, "cudaMalloc of coefficient tables: %s", cudaGetErrorString(e));
  m.d_tabs = (double*)p;
  m.f_tabs = (float*)((char*)p + bd);
  CUDA_TRY(cudaMemcpy(m.d_tabs, t.data(), bd, cudaMemcpyHostToDevice), "copy of coefficient tables");
  CUDA_TRY(cudaMemcpy(m.f_tabs, tf.data(), bf, cudaMemcpyHostToDevice), "copy of coefficient tables");
  return ADVECT_OK;
}

bool overlaps(const void* a, const void* b, size_t n) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + n && y < x + n;
}

advect_status check_device_ptr(const void* p, const char* name, size_t elem, int device) {
  if (!p) return fail(ADVECT_EINVAL, "%s is NULL", name);
  if ((uintptr_t)p % elem) return fail(ADVECT_EINVAL, "%s is not aligned to its element size", name);
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ADVECT_EINVAL, "%s is not a CUDA pointer", name);
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
    return fail(ADVECT_EINVAL, "%s is not device memory", name);
  if (at.type == cudaMemoryTypeDevice && at.device != device)
    return fail(ADVECT_EINVAL, "%s belongs to device %d, context is on device %d", name, at.device, device);
  return ADVECT_OK;
}

// Validate the six (or nine) buffers of a call: device memory of the
// context's device, element-aligned, outputs disjoint from inputs and from
// each other.
advect_status check_buffers(const void* const* in, int n_in, void* const* out, int n_out,
                            const char* const* names, size_t bytes, size_t elem, int device) {
  for (int q = 0; q < n_in; ++q) {
    advect_status s = check_device_ptr(in[q], names[q], elem, device);
    if (s) return s;
  }
  for (int q = 0; q < n_out; ++q) {
    advect_status s = check_device_ptr(out[q], names[n_in + q], elem, device);
    if (s) return s;
  }
  for (int o = 0; o < n_out; ++o) {
    for (int q = 0; q < n_in; ++q)
      if (overlaps(out[o], in[q], bytes))
        return fail(ADVECT_EINVAL, "output %s overlaps input %s", names[n_in + o], names[q]);
    for (int p = o + 1; p < n_out; ++p)
      if (overlaps(out[o], out[p], bytes))
        return fail(ADVECT_EINVAL, "outputs %s and %s overlap", names[n_in + o], names[n_in + p]);
  }
  return ADVECT_OK;
}

advect_status check_flag(advect_ctx* ctx) {
  int h = 0;
  CUDA_TRY(cudaMemcpy(&h, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost), "read of the device error flag");
  if (h) {
    CUDA_TRY(cudaMemset(ctx->d_flag, 0, sizeof(int)), "reset of the device error flag");
    return fail(ADVECT_ETIMEOUT, "a kernel gave up a bounded wait (code %d)", h);
  }
  return ADVECT_OK;
}

Coeffs coeffs_of(const Member& m) {
  Coeffs c;
  c.d = m.d_tabs;
  c.f = m.f_tabs;
  c.tcx = m.tcx;
  c.tcy = m.tcy;
  c.tcx_f = (float)m.tcx;
  c.tcy_f = (float)m.tcy;
  return c;
}

}  // namespace abi
}  // namespace advect

namespace {

advect_status read_scales(advect_ctx* ctx, const float* scales, Scales& sc, bool with_base = false) {
  for (int q = 0; q < 3; ++q) {
    sc.in[q] = 1.f;
    sc.inv_out[q] = 1.f;
    sc.base[q] = 1.f;
  }
  if (ctx->dtype != ADVECT_F16S) return ADVECT_OK;
  if (!scales)
    return fail(ADVECT_EINVAL, with_base ? "F16S needs 9 scales (u, v, w, 3 outputs, 3 bases)"
                                         : "F16S needs 6 scales (u, v, w, su, sv, sw)");
  advect_status s = check_f16s_scales(scales, with_base ? 9 : 6);
  if (s) return s;
  for (int q = 0; q < 3; ++q) {
    sc.in[q] = scales[q];
    sc.inv_out[q] = 1.f / scales[3 + q];
  }
  if (with_base)
    for (int q = 0; q < 3; ++q) sc.base[q] = scales[6 + q];
  return ADVECT_OK;
}

}  // namespace

// Launch the forward on planes [i0, i1) of a single-grid context.
advect_status advect_ctx::launch_forward(const void* u, const void* v, const void* w, void* su,
                                          void* sv, void* sw, const Scales& sc, int i0, int i1,
                                          cudaStream_t st, const Step* step) {
  const Member& m = members[0];
  FwdArgs a;
  a.u = u; a.v = v; a.w = w;
  a.su = su; a.sv = sv; a.sw = sw;
  a.s = Shape{m.nx, m.ny, m.nz};
  a.c = coeffs_of(m);
  a.sc = sc;
  a.f64_levels = f64_levels;
  a.i0 = i0;
  a.i1 = i1;
  a.wait_budget = wait_budget;
  a.skip_plane = test_skip_plane;
  if (step) {
    a.integ = 1;
    a.bu = step->b[0];
    a.bv = step->b[1];
    a.bw = step->b[2];
    a.dt = step->dt;
    a.dt_hi = (float)step->dt;
    a.dt_lo = (float)(step->dt - (double)a.dt_hi);
  } else if (tune_fwd) {
    tune_fwd = false;
    cudaError_t e = tune_single(*this, 0, &a, nullptr, st);
    if (e != cudaSuccess) return cuda_fail(e, "forward tuning");
  }
  cudaError_t e = launch_fwd(*this, a, st);
  if (e != cudaSuccess) return cuda_fail(e, "forward kernel launch");
  return ADVECT_OK;
}

extern "C" {

advect_status advect_coeffs_from_grid(const advect_grid* g, double* tcx, double* tcy, double* tzc1,
                                      double* tzc2, double* tzd1, double* tzd2) {
  if (!g || !tcx || !tcy || !tzc1 || !tzc2 || !tzd1 || !tzd2)
    return fail(ADVECT_EINVAL, "NULL argument");
  const int nz = g->nz;
  if (nz < 3) return fail(ADVECT_EINVAL, "nz must be >= 3");
  if (!g->z || !g->zn || !g->rho || !g->rhon) return fail(ADVECT_EINVAL, "NULL level array");
  if (!(g->dx > 0) || !(g->dy > 0) || !is_finite(g->dx) || !is_finite(g->dy))
    return fail(ADVECT_EINVAL, "dx and dy must be positive and finite");
  for (int k = 0; k < nz; ++k) {
    if (!(g->rho[k] > 0) || !(g->rhon[k] > 0) || !is_finite(g->rho[k]) || !is_finite(g->rhon[k]))
      return fail(ADVECT_EINVAL, "density at level %d must be positive and finite", k);
    if (k >= 1 && !(g->z[k] > g->z[k - 1])) return fail(ADVECT_EINVAL, "z must increase (level %d)", k);
    if (k >= 2 && !(g->zn[k] > g->zn[k - 1])) return fail(ADVECT_EINVAL, "zn must increase (level %d)", k);
  }
  *tcx = 1.0 / (4.0 * g->dx);
  *tcy = 1.0 / (4.0 * g->dy);
  for (int k = 0; k < nz; ++k) tzc1[k] = tzc2[k] = tzd1[k] = tzd2[k] = 0.0;
  for (int k = 1; k < nz; ++k) {
    const double dz = g->z[k] - g->z[k - 1];
    const double den = 4.0 * dz * g->rhon[k];
    tzc1[k] = g->rho[k - 1] / den;
    tzc2[k] = g->rho[k] / den;
  }
  for (int k = 1; k < nz - 1; ++k) {
    const double dzn = g->zn[k + 1] - g->zn[k];
    const double den = 4.0 * dzn * g->rho[k];
    tzd1[k] = g->rhon[k] / den;
    tzd2[k] = g->rhon[k + 1] / den;
  }
  return ADVECT_OK;
}

advect_status advect_create(int nx, int ny, int nz, const advect_coeffs* c, advect_dtype dtype,
                            advect_ctx** out) {
  if (!out) return fail(ADVECT_EINVAL, "out is NULL");
  *out = nullptr;
  if (!valid_dtype(dtype)) return fail(ADVECT_EINVAL, "unknown dtype %d", (int)dtype);
  advect_status s = check_shape(nx, ny, nz);
  if (s) return s;
  s = check_coeffs(c, nz);
  if (s) return s;
  advect_ctx* ctx = new (std::nothrow) advect_ctx();
  if (!ctx) return fail(ADVECT_ENOMEM, "host allocation failed");
  ctx->dtype = dtype;
  CUDA_TRY(cudaGetDevice(&ctx->device), "cudaGetDevice");
  CUDA_TRY(cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device),
           "cudaDeviceGetAttribute");
  ctx->members.resize(1);
  ctx->members[0].nx = nx;
  ctx->members[0].ny = ny;
  ctx->members[0].nz = nz;
  s = upload_member(ctx->members[0], c);
  if (s) {
    advect_destroy(ctx);
    return s;
  }
  cudaError_t e = cudaMalloc(&ctx->d_flag, sizeof(int));
  if (e != cudaSuccess) {
    advect_destroy(ctx);
    return fail(ADVECT_ENOMEM, "cudaMalloc of the error flag: %s", cudaGetErrorString(e));
  }
  e = cudaMemset(ctx->d_flag, 0, sizeof(int));
  if (e != cudaSuccess) {
    advect_destroy(ctx);
    return cuda_fail(e, "cudaMemset");
  }
  select_kernels(*ctx);
  *out = ctx;
  return ADVECT_OK;
}

advect_status advect_forward(advect_ctx* ctx, const void* u, const void* v, const void* w, void* su,
                             void* sv, void* sw, const float* scales, advect_stream stream) {
  if (!ctx) return fail(ADVECT_EINVAL, "context is NULL");
  if (ctx->ensemble) return fail(ADVECT_EINVAL, "ensemble context: use advect_ensemble_forward");
  const Member& m = ctx->members[0];
  const size_t bytes = (size_t)m.nx * m.ny * m.nz * elem_bytes(ctx->dtype);
  const void* in[3] = {u, v, w};
  void* outp[3] = {su, sv, sw};
  static const char* names[6] = {"u", "v", "w", "su", "sv", "sw"};
  advect_status s = check_buffers(in, 3, outp, 3, names, bytes, elem_bytes(ctx->dtype), ctx->device);
  if (s) return s;
  Scales sc;
  s = read_scales(ctx, scales, sc);
  if (s) return s;
  return ctx->launch_forward(u, v, w, su, sv, sw, sc, 0, m.nx, (cudaStream_t)stream);
}

advect_status advect_forward_integrate(advect_ctx* ctx, const void* u, const void* v, const void* w,
                                       const void* u_base, const void* v_base, const void* w_base, double dt,
                                       void* u_out, void* v_out, void* w_out, const float* scales,
                                       advect_stream stream) {
  if (!ctx) return fail(ADVECT_EINVAL, "context is NULL");
  if (ctx->ensemble) return fail(ADVECT_EINVAL, "ensemble context: the integration step is single-grid only");
  if (!is_finite(dt)) return fail(ADVECT_EINVAL, "dt must be finite");
  const int nb = (u_base != nullptr) + (v_base != nullptr) + (w_base != nullptr);
  if (nb != 0 && nb != 3) return fail(ADVECT_EINVAL, "give all three base fields or none");
  const Member& m = ctx->members[0];
  const size_t elem = elem_bytes(ctx->dtype);
  const size_t bytes = (size_t)m.nx * m.ny * m.nz * elem;
  const void* in[3] = {u, v, w};
  void* outp[3] = {u_out, v_out, w_out};
  static const char* names[6] = {"u", "v", "w", "u_out", "v_out", "w_out"};
  advect_status s = check_buffers(in, 3, outp, 3, names, bytes, elem, ctx->device);
  if (s) return s;
  const void* base[3] = {u_base, v_base, w_base};
  static const char* bnames[3] = {"u_base", "v_base", "w_base"};
  if (nb == 3) {
    for (int f = 0; f < 3; ++f) {
      s = check_device_ptr(base[f], bnames[f], elem, ctx->device);
      if (s) return s;
      // each base element is read by the thread that then writes that output
      // element, so a base may be its own output (in place), but must not
      // overlap any other output
      for (int o = 0; o < 3; ++o)
        if (!(o == f && base[f] == outp[o]) && overlaps(base[f], outp[o], bytes))
          return fail(ADVECT_EINVAL, "base %s overlaps output %s", bnames[f], names[3 + o]);
    }
  }
  Scales sc;
  s = read_scales(ctx, scales, sc, nb == 3);
  if (s) return s;
  const advect_ctx::Step step{{base[0], base[1], base[2]}, dt};
  return ctx->launch_forward(u, v, w, u_out, v_out, w_out, sc, 0, m.nx, (cudaStream_t)stream, &step);
}

advect_status advect_adjoint(advect_ctx* ctx, const void* u, const void* v, const void* w,
                             const void* dsu, const void* dsv, const void* dsw, void* du, void* dv,
                             void* dw, advect_stream stream) {
  if (!ctx) return fail(ADVECT_EINVAL, "context is NULL");
  if (ctx->ensemble) return fail(ADVECT_EINVAL, "ensemble context: use advect_ensemble_adjoint");
  if (ctx->dtype == ADVECT_F16S) return fail(ADVECT_EUNSUPPORTED, "the adjoint supports F64 and F32 only");
  const Member& m = ctx->members[0];
  const size_t bytes = (size_t)m.nx * m.ny * m.nz * elem_bytes(ctx->dtype);
  const void* in[6] = {u, v, w, dsu, dsv, dsw};
  void* outp[3] = {du, dv, dw};
  static const char* names[9] = {"u", "v", "w", "dsu", "dsv", "dsw", "du", "dv", "dw"};
  advect_status s = check_buffers(in, 6, outp, 3, names, bytes, elem_bytes(ctx->dtype), ctx->device);
  if (s) return s;
  AdjArgs a;
  a.u = u; a.v = v; a.w = w;
  a.dsu = dsu; a.dsv = dsv; a.dsw = dsw;
  a.du = du; a.dv = dv; a.dw = dw;
  a.s = Shape{m.nx, m.ny, m.nz};
  a.c = coeffs_of(m);
  a.wait_budget = ctx->wait_budget;
  a.skip_plane = ctx->test_skip_plane;
  if (ctx->tune_adj) {
    ctx->tune_adj = false;
    cudaError_t e = tune_single(*ctx, 1, nullptr, &a, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint tuning");
  }
  cudaError_t e = launch_adj(*ctx, a, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "adjoint kernel launch");
  return ADVECT_OK;
}

advect_status advect_forward_host(advect_ctx* ctx, const void* u, const void* v, const void* w,
                                  void* su, void* sv, void* sw, const float* scales) {
  if (!ctx) return fail(ADVECT_EINVAL, "context is NULL");
  if (ctx->ensemble) return fail(ADVECT_EINVAL, "ensemble context has no host path");
  if (!u || !v || !w || !su || !sv || !sw) return fail(ADVECT_EINVAL, "NULL buffer");
  const Member& m = ctx->members[0];
  const size_t eb = elem_bytes(ctx->dtype);
  const size_t plane = (size_t)m.ny * m.nz * eb;
  const size_t bytes = plane * m.nx;
  const void* in[3] = {u, v, w};
  void* outp[3] = {su, sv, sw};
  for (int o = 0; o < 3; ++o) {
    for (int q = 0; q < 3; ++q)
      if (overlaps(outp[o], in[q], bytes)) return fail(ADVECT_EINVAL, "an output overlaps an input");
    for (int p = o + 1; p < 3; ++p)
      if (overlaps(outp[o], outp[p], bytes)) return fail(ADVECT_EINVAL, "outputs overlap");
  }
  Scales sc;
  advect_status s = read_scales(ctx, scales, sc);
  if (s) return s;
  s = ctx->ensure_host_path(bytes);
  if (s) return s;
  HostPath& hp = ctx->hp;
  // Chunks of x-planes.  Chunk c's kernel needs plane i0-1 (previous chunk,
  // or the last plane for c = 0) and plane i1 (next chunk, or plane 0), so
  // each chunk's copy also carries its first plane of the next chunk, and
  // the last plane is copied first.
  const int nchunk = std::max(1, std::min(m.nx, hp.nchunk));
  std::vector<int> b(nchunk + 1);
  for (int c = 0; c <= nchunk; ++c) b[c] = (int)((long long)m.nx * c / nchunk);
  cudaStream_t sin = hp.s_in, sk = hp.s_k, sout = hp.s_out;
  for (int f = 0; f < 3; ++f)
    CUDA_TRY(cudaMemcpyAsync((char*)hp.d_in[f] + plane * (m.nx - 1), (const char*)in[f] + plane * (m.nx - 1),
                             plane, cudaMemcpyHostToDevice, sin), "host-to-device copy");
  for (int c = 0; c < nchunk; ++c) {
    const int i0 = b[c], i1 = b[c + 1];
    const int hi = std::min(i1 + 1, m.nx);
    for (int f = 0; f < 3; ++f)
      CUDA_TRY(cudaMemcpyAsync((char*)hp.d_in[f] + plane * i0, (const char*)in[f] + plane * i0,
                               plane * (hi - i0), cudaMemcpyHostToDevice, sin), "host-to-device copy");
    CUDA_TRY(cudaEventRecord(hp.ev_in[c], sin), "cudaEventRecord");
  }
  for (int c = 0; c < nchunk; ++c) {
    const int i0 = b[c], i1 = b[c + 1];
    CUDA_TRY(cudaStreamWaitEvent(sk, hp.ev_in[c], 0), "cudaStreamWaitEvent");
    if (c == nchunk - 1) CUDA_TRY(cudaStreamWaitEvent(sk, hp.ev_in[0], 0), "cudaStreamWaitEvent");
    s = ctx->launch_forward(hp.d_in[0], hp.d_in[1], hp.d_in[2], hp.d_out[0], hp.d_out[1], hp.d_out[2], sc, i0,
                            i1, sk);
    if (s) return s;
    CUDA_TRY(cudaEventRecord(hp.ev_k[c], sk), "cudaEventRecord");
    CUDA_TRY(cudaStreamWaitEvent(sout, hp.ev_k[c], 0), "cudaStreamWaitEvent");
    for (int f = 0; f < 3; ++f)
      CUDA_TRY(cudaMemcpyAsync((char*)outp[f] + plane * i0, (const char*)hp.d_out[f] + plane * i0,
                               plane * (i1 - i0), cudaMemcpyDeviceToHost, sout), "device-to-host copy");
  }
  CUDA_TRY(cudaStreamSynchronize(sout), "cudaStreamSynchronize");
  return check_flag(ctx);
}

advect_status advect_f16s_output_scales(const advect_ctx* ctx, const float* in, float* out) {
  if (!ctx || !in || !out) return fail(ADVECT_EINVAL, "NULL argument");
  for (int q = 0; q < 3; ++q)
    if (!(in[q] > 0.f) || !std::isfinite(in[q])) return fail(ADVECT_EINVAL, "input scale %d invalid", q);
  const Member& m = ctx->members[0];
  const int nz = m.nz;
  double zc = 0, zd = 0;
  for (int k = 0; k < nz; ++k) {
    zc = std::max(zc, std::fabs(m.h_tabs[k]) + std::fabs(m.h_tabs[nz + k]));
    zd = std::max(zd, std::fabs(m.h_tabs[2 * nz + k]) + std::fabs(m.h_tabs[3 * nz + k]));
  }
  const double Mu = in[0], Mv = in[1], Mw = in[2];
  const double tx = std::fabs(m.tcx), ty = std::fabs(m.tcy);
  const double B[3] = {4 * tx * Mu * Mu + 4 * ty * Mu * Mv + 2 * zc * Mu * Mw,
                       4 * tx * Mv * Mu + 4 * ty * Mv * Mv + 2 * zc * Mv * Mw,
                       4 * tx * Mw * Mu + 4 * ty * Mw * Mv + 2 * zd * Mw * Mw};
  for (int q = 0; q < 3; ++q) {
    double b = B[q] > 0 ? B[q] : 1.0;
    int e = (int)std::ceil(std::log2(b));
    out[q] = std::ldexp(1.0f, e);
  }
  return ADVECT_OK;
}

advect_status advect_set_f64_levels(advect_ctx* ctx, int n) {
  if (!ctx) return fail(ADVECT_EINVAL, "context is NULL");
  if (n < 0) return fail(ADVECT_EINVAL, "level count must be >= 0");
  ctx->f64_levels = n;
  return ADVECT_OK;
}

advect_status advect_sync(advect_ctx* ctx, advect_stream stream) {
  if (!ctx) return fail(ADVECT_EINVAL, "context is NULL");
  CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream), "cudaStreamSynchronize");
  return check_flag(ctx);
}

const char* advect_kernel_name(const advect_ctx* ctx, int adjoint) {
  if (!ctx) return "";
  return adjoint ? ctx->adj_name.c_str() : ctx->fwd_name.c_str();
}

void advect_destroy(advect_ctx* ctx) {
  if (!ctx) return;
  ctx->release();
  delete ctx;
}

const char* advect_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
