// abi_util.h -- helpers shared by the C-ABI translation units (internal).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

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
// Host copy of one grid's tables (tzc1 | tzc2 | tzd1 | tzd2, nz entries each)
// with the entries no formula reads set to zero and tzc2[nz-1] = 0.
void masked_tables(const advect_coeffs* c, int nz, double* t);  // t: 4 * nz entries
void masked_tables(const advect_coeffs* c, int nz, std::vector<double>& t);
// F16S scales: n positive, finite powers of two, else EINVAL.
advect_status check_f16s_scales(const float* s, int n);
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
