// abi_util.h -- helpers shared by the C-ABI translation units (internal).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "../../include/advect.h"
#include "ctx.h"

namespace advect {
namespace abi {

extern thread_local std::string g_last_error;

// Record a message for advect_last_error() and return s.
advect_status fail(advect_status s, const char* fmt, ...);
advect_status cuda_fail(cudaError_t e, const char* what);
size_t elem_bytes(advect_dtype d);
bool valid_dtype(int d);
advect_status check_coeffs(const advect_coeffs* c, int nz);
advect_status check_shape(int nx, int ny, int nz);
advect_status upload_member(Member& m, const advect_coeffs* c);
bool overlaps(const void* a, const void* b, size_t n);
advect_status check_device_ptr(const void* p, const char* name, size_t elem, int device);
advect_status check_flag(advect_ctx* ctx);
Coeffs coeffs_of(const Member& m);

}  // namespace abi
}  // namespace advect

#define ADVECT_CUDA_TRY(call, what)                                  \
  do {                                                               \
    cudaError_t e_ = (call);                                         \
    if (e_ != cudaSuccess) return ::advect::abi::cuda_fail(e_, what); \
  } while (0)
