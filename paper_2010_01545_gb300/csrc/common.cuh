// common.cuh -- device-side building blocks shared by the advection kernels.
//
// Storage types: double (F64), float (F32) and __half with a per-field
// power-of-two scale (F16S).  Arithmetic type: double for F64, float for the
// others.  Layout of every field: [nx][ny][nz], z contiguous (Sec. 2.1,
// Listing 1's u(k,j,i)); lateral directions periodic.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ff.cuh"

namespace advect {

// Per-level coefficient tables on the device, 4 tables of nz entries each in
// the order tzc1, tzc2, tzd1, tzd2.  Entries no formula reads are zero, and
// tzc2[nz-1] is zero: that implements Listing 1's top-level else branch
// (the upper vertical flux of su and sv is dropped at the lid).
struct Coeffs {
  const double* d;   // binary64 tables
  const float* f;    // binary32 copies
  double tcx, tcy;
  float tcx_f, tcy_f;
};

enum { TZC1 = 0, TZC2 = 1, TZD1 = 2, TZD2 = 3 };

struct Shape {
  int nx, ny, nz;
};

// Scales for F16S (stored = true / scale); unused for other types.
struct Scales {
  float in[3];       // u, v, w
  float inv_out[3];  // 1 / scale of su, sv, sw (or of the integrated fields)
  float base[3];     // base fields of an integration step
};

template <typename T>
struct Store;

template <>
struct Store<double> {
  using C = double;
  static constexpr int kBytes = 8;
  __device__ static __forceinline__ C load(const double* p, size_t i, float) { return __ldg(p + i); }
  __device__ static __forceinline__ void store(double* p, size_t i, C v, float) { p[i] = v; }
  __device__ static __forceinline__ C coef(const Coeffs& c, int table, int nz, int k) {
    return __ldg(c.d + (size_t)table * nz + k);
  }
  __device__ static __forceinline__ C tcx(const Coeffs& c) { return c.tcx; }
  __device__ static __forceinline__ C tcy(const Coeffs& c) { return c.tcy; }
};

template <>
struct Store<float> {
  using C = float;
  static constexpr int kBytes = 4;
  __device__ static __forceinline__ C load(const float* p, size_t i, float) { return __ldg(p + i); }
  __device__ static __forceinline__ void store(float* p, size_t i, C v, float) { p[i] = v; }
  __device__ static __forceinline__ C coef(const Coeffs& c, int table, int nz, int k) {
    return __ldg(c.f + (size_t)table * nz + k);
  }
  __device__ static __forceinline__ C tcx(const Coeffs& c) { return c.tcx_f; }
  __device__ static __forceinline__ C tcy(const Coeffs& c) { return c.tcy_f; }
};

template <>
struct Store<__half> {
  using C = float;
  static constexpr int kBytes = 2;
  __device__ static __forceinline__ C load(const __half* p, size_t i, float s) {
    return __half2float(p[i]) * s;
  }
  __device__ static __forceinline__ void store(__half* p, size_t i, C v, float inv_s) {
    p[i] = __float2half_rn(v * inv_s);
  }
  __device__ static __forceinline__ C coef(const Coeffs& c, int table, int nz, int k) {
    return __ldg(c.f + (size_t)table * nz + k);
  }
  __device__ static __forceinline__ C tcx(const Coeffs& c) { return c.tcx_f; }
  __device__ static __forceinline__ C tcy(const Coeffs& c) { return c.tcy_f; }
};

// binary64 storage, double-float arithmetic (ff.cuh)
template <>
struct Store<f64ff> {
  using C = ff;
  static constexpr int kBytes = 8;
  __device__ static __forceinline__ C load(const f64ff* p, size_t i, float) {
    return ff(__ldg(reinterpret_cast<const double*>(p) + i));
  }
  __device__ static __forceinline__ void store(f64ff* p, size_t i, C v, float) {
    reinterpret_cast<double*>(p)[i] = (double)v;
  }
  __device__ static __forceinline__ C coef(const Coeffs& c, int table, int nz, int k) {
    return ff(__ldg(c.d + (size_t)table * nz + k));
  }
  __device__ static __forceinline__ C tcx(const Coeffs& c) { return ff(c.tcx); }
  __device__ static __forceinline__ C tcy(const Coeffs& c) { return ff(c.tcy); }
};

__device__ __forceinline__ int wrap_dec(int a, int n) { return a == 0 ? n - 1 : a - 1; }
__device__ __forceinline__ int wrap_inc(int a, int n) { return a == n - 1 ? 0 : a + 1; }

}  // namespace advect
