// noalloc.cu -- forward pass for callers that cannot allocate device memory.
//
// Why: some callers are not allowed to call cudaMalloc -- code that runs
// inside a framework that owns every device allocation through its own pool,
// code on a latency-critical path where an allocation may block or
// synchronise the device, or code that must not grow the device footprint
// after start-up.  The context API allocates at create time (coefficient
// tables, error flag); this entry point needs no context and allocates
// nothing.
//
// How: the only device memory it needs besides the caller's fields -- the
// per-level coefficient tables (binary64 and binary32 copies) and the
// kernels' error flag -- lives in one file-scope __device__ array of fixed
// size, g_noalloc_scratch, which every GPU that loads this library holds for
// as long as the library stays loaded.  A one-block set-up kernel, which
// receives the tables by value as a kernel parameter, writes them there and
// clears the flag before each forward launch on the caller's stream; then
// the ordinary forward kernel (plane sweep or point kernel, with the tile a
// new context of the same type starts from) runs with pointers into the
// array.
//
// In host code the array's name is only a stand-in for the symbol, not a
// device address: its address on a device is looked up with
// cudaGetSymbolAddress on the first call made with that device current, and
// cached together with the device's current context, so that after a
// cudaDeviceReset (or under another context) the next call looks it up again
// instead of using a stale address.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/advect.h"
#include "abi_util.h"
#include "ctx.h"
#include "kernels.h"

using namespace advect;
using namespace advect::abi;

namespace {

constexpr int kMaxNz = ADVECT_NOALLOC_MAX_NZ;
constexpr size_t kTabOffset = 256;                                   // after the flag
constexpr size_t kF32Offset = kTabOffset + 4 * (size_t)kMaxNz * sizeof(double);
constexpr size_t kScratchBytes = kF32Offset + 4 * (size_t)kMaxNz * sizeof(float);
constexpr int kMaxDevices = 64;

// The shared scratch: [0, 256) error flag, then 4*kMaxNz binary64 table
// entries, then 4*kMaxNz binary32 entries (tables packed by the call's nz).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct SetupParams {
  double t[4 * kMaxNz];  // tzc1 | tzc2 | tzd1 | tzd2, each nz entries, masked
  int nz;
};

__global__ void noalloc_setup_kernel(SetupParams p) {
  double* d = reinterpret_cast<double*>(g_noalloc_scratch + kTabOffset);
  float* f = reinterpret_cast<float*>(g_noalloc_scratch + kF32Offset);
  for (int q = threadIdx.x; q < 4 * p.nz; q += blockDim.x) {
    d[q] = p.t[q];
    f[q] = (float)p.t[q];
  }
  if (threadIdx.x == 0) *reinterpret_cast<int*>(g_noalloc_scratch) = 0;  // the flag starts at zero
}

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};
void* g_scratch_ctx[kMaxDevices] = {};  // the driver context the address belongs to

// The driver's current context (cuCtxGetCurrent through the runtime's entry
// point lookup, so the library links no driver library); NULL if unknown.
void* current_driver_context() {
  using Fn = int (*)(void**);
  static Fn fn = []() -> Fn {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<Fn>(f);
  }();
  void* c = nullptr;
  if (fn && fn(&c) != 0) c = nullptr;
  return c;
}

// Device address of the scratch on the current device: looked up on the
// first call with this device current and again whenever the device's
// current context has changed since (e.g. after cudaDeviceReset).
advect_status scratch_address(int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices) return fail(ADVECT_EUNSUPPORTED, "device ordinal %d too large", device);
  std::lock_guard<std::mutex> lk(g_mu);
  void* cur = current_driver_context();
  if (!g_scratch_addr[device] || cur != g_scratch_ctx[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress of the no-allocation scratch");
    g_scratch_addr[device] = p;
    g_scratch_ctx[device] = current_driver_context();  // the lookup may have created the context
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[device]);
  return ADVECT_OK;
}

}  // namespace

extern "C" advect_status advect_forward_noalloc(int nx, int ny, int nz, const advect_coeffs* c,
                                                advect_dtype dtype, const void* u, const void* v,
                                                const void* w, void* su, void* sv, void* sw,
                                                const float* scales, advect_stream stream) {
  if (!valid_dtype(dtype)) return fail(ADVECT_EINVAL, "unknown dtype %d", (int)dtype);
  advect_status s = check_shape(nx, ny, nz);
  if (s) return s;
  if (nz > kMaxNz)
    return fail(ADVECT_EINVAL, "nz = %d exceeds the no-allocation limit of %d levels", nz, kMaxNz);
  s = check_coeffs(c, nz);
  if (s) return s;
  Scales sc;
  for (int q = 0; q < 3; ++q) {
    sc.in[q] = 1.f;
    sc.inv_out[q] = 1.f;
    sc.base[q] = 1.f;
  }
  if (dtype == ADVECT_F16S) {
    if (!scales) return fail(ADVECT_EINVAL, "F16S needs 6 scales (u, v, w, su, sv, sw)");
    s = check_f16s_scales(scales, 6);
    if (s) return s;
    for (int q = 0; q < 3; ++q) {
      sc.in[q] = scales[q];
      sc.inv_out[q] = 1.f / scales[3 + q];
    }
  }
  int device = 0;
  ADVECT_CUDA_TRY(cudaGetDevice(&device), "cudaGetDevice");
  const size_t eb = elem_bytes(dtype);
  const size_t bytes = (size_t)nx * ny * nz * eb;
  const void* in[3] = {u, v, w};
  void* out[3] = {su, sv, sw};
  static const char* names[6] = {"u", "v", "w", "su", "sv", "sw"};
  for (int q = 0; q < 6; ++q) {
    s = check_device_ptr(q < 3 ? in[q] : out[q - 3], names[q], eb, device);
    if (s) return s;
  }
  for (int o = 0; o < 3; ++o) {
    for (int q = 0; q < 3; ++q)
      if (overlaps(out[o], in[q], bytes)) return fail(ADVECT_EINVAL, "output %s overlaps input %s", names[3 + o], names[q]);
    for (int p = o + 1; p < 3; ++p)
      if (overlaps(out[o], out[p], bytes)) return fail(ADVECT_EINVAL, "outputs %s and %s overlap", names[3 + o], names[3 + p]);
  }
  unsigned char* scratch = nullptr;
  s = scratch_address(device, &scratch);
  if (s) return s;

  // Tables as the context path stores them: unused entries zero and
  // tzc2[nz-1] = 0 (Listing 1 drops the upper flux at the lid).
  SetupParams sp;
  sp.nz = nz;
  masked_tables(c, nz, sp.t);
  cudaStream_t st = (cudaStream_t)stream;
  noalloc_setup_kernel<<<1, 256, 0, st>>>(sp);
  ADVECT_CUDA_TRY(cudaGetLastError(), "no-allocation set-up kernel");

  FwdArgs a;
  a.u = u;
  a.v = v;
  a.w = w;
  a.su = su;
  a.sv = sv;
  a.sw = sw;
  a.s = Shape{nx, ny, nz};
  a.c.d = reinterpret_cast<const double*>(scratch + kTabOffset);
  a.c.f = reinterpret_cast<const float*>(scratch + kF32Offset);
  a.c.tcx = c->tcx;
  a.c.tcy = c->tcy;
  a.c.tcx_f = (float)c->tcx;
  a.c.tcy_f = (float)c->tcy;
  a.sc = sc;
  a.f64_levels = 0;
  a.i0 = 0;
  a.i1 = nx;
  int* flag = reinterpret_cast<int*>(scratch);
  const SweepCfg cfg = fit_planes(default_fwd_sweep(nz, (int)dtype), nx);
  auto al16 = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
  cudaError_t e;
  if (cfg.ty > 0 && al16(u) && al16(v) && al16(w) && al16(su) && al16(sv) && al16(sw))
    e = launch_fwd_sweep((int)dtype, a, cfg, flag, st);
  else
    e = launch_fwd_point((int)dtype, a, st);
  if (e != cudaSuccess) return cuda_fail(e, "forward kernel launch");
  return ADVECT_OK;
}
