// point.cu -- one-thread-per-grid-point kernels (forward and adjoint).
//
// These take any shape and any element-aligned pointers; they read every
// neighbour straight from global memory (L1/L2 serve the reuse).  The tiled
// plane-sweep kernels are used where their alignment conditions hold.
#include "kernels.h"

namespace advect {
namespace {

constexpr int kThreads = 256;

template <typename T>
struct Grid3 {
  const T* p;
  int nx, ny, nz;
  float scale;
  // Value at (i, j, k) with periodic i, j; zero outside 0 <= k < nz.
  __device__ __forceinline__ typename Store<T>::C at(int i, int j, int k) const {
    if (k < 0 || k >= nz) return 0;
    i = i < 0 ? i + nx : (i >= nx ? i - nx : i);
    j = j < 0 ? j + ny : (j >= ny ? j - ny : j);
    return Store<T>::load(p, ((size_t)i * ny + j) * nz + k, scale);
  }
};

// The integration step dt in each arithmetic type.
__device__ __forceinline__ void step_into(double& o, const FwdArgs& a) { o = a.dt; }
__device__ __forceinline__ void step_into(float& o, const FwdArgs& a) { o = a.dt_hi; }
__device__ __forceinline__ void step_into(ff& o, const FwdArgs& a) { o = ff(a.dt_hi, a.dt_lo); }

// ---------------------------------------------------------------- forward
// su, sv, sw at one point: Listing 1 (Sec. 2.1) for su and the same pattern
// for sv (x<->y) and sw (w cell).  The top-level branch of Listing 1 comes
// from tzc2[nz-1] == 0 and zero loads above the lid.
template <typename T>
__global__ void __launch_bounds__(kThreads)
fwd_point_kernel(FwdArgs a) {
  using S = Store<T>;
  using C = typename S::C;
  const int nx = a.s.nx, ny = a.s.ny, nz = a.s.nz;
  const Grid3<T> U{(const T*)a.u, nx, ny, nz, a.sc.in[0]};
  const Grid3<T> V{(const T*)a.v, nx, ny, nz, a.sc.in[1]};
  const Grid3<T> W{(const T*)a.w, nx, ny, nz, a.sc.in[2]};
  T* su = (T*)a.su;
  T* sv = (T*)a.sv;
  T* sw = (T*)a.sw;
  const size_t n = (size_t)(a.i1 - a.i0) * ny * nz;
  const size_t base = (size_t)a.i0 * ny * nz;
  const C tcx = S::tcx(a.c), tcy = S::tcy(a.c);
  for (size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (size_t)gridDim.x * blockDim.x) {
    const size_t t = base + r;
    const int k = (int)(t % nz);
    const size_t col = t / nz;
    const int j = (int)(col % ny);
    const int i = (int)(col / ny);
    C ou = 0, ov = 0, ow = 0;
    if (k >= 1) {
      const C u0 = U.at(i, j, k), uxm = U.at(i - 1, j, k), uxp = U.at(i + 1, j, k);
      const C uym = U.at(i, j - 1, k), uyp = U.at(i, j + 1, k);
      const C uzm = U.at(i, j, k - 1), uzp = U.at(i, j, k + 1);
      const C uxm_yp = U.at(i - 1, j + 1, k), uxm_zp = U.at(i - 1, j, k + 1);
      const C v0 = V.at(i, j, k), vxm = V.at(i - 1, j, k), vxp = V.at(i + 1, j, k);
      const C vym = V.at(i, j - 1, k), vyp = V.at(i, j + 1, k);
      const C vzm = V.at(i, j, k - 1), vzp = V.at(i, j, k + 1);
      const C vym_xp = V.at(i + 1, j - 1, k), vym_zp = V.at(i, j - 1, k + 1);
      const C w0 = W.at(i, j, k), wxm = W.at(i - 1, j, k), wxp = W.at(i + 1, j, k);
      const C wym = W.at(i, j - 1, k), wyp = W.at(i, j + 1, k);
      const C wzm = W.at(i, j, k - 1), wzp = W.at(i, j, k + 1);
      const C wzm_xp = W.at(i + 1, j, k - 1), wzm_yp = W.at(i, j + 1, k - 1);

      ou = tcx * (uxm * (u0 + uxm) - uxp * (u0 + uxp)) +
           tcy * (uym * (vym + vym_xp) - uyp * (v0 + vxp));
      ov = tcx * (vxm * (uxm + uxm_yp) - vxp * (u0 + uyp)) +
           tcy * (vym * (v0 + vym) - vyp * (v0 + vyp));
      ow = tcx * (wxm * (uxm + uxm_zp) - wxp * (u0 + uzp)) +
           tcy * (wym * (vym + vym_zp) - wyp * (v0 + vzp));
      if (sizeof(C) == 4 && a.f64_levels > 0 && k <= a.f64_levels) {
        // near-surface levels: vertical terms in binary64 with binary64 tables
        const double* d = a.c.d;
        const double c1 = d[k], c2 = d[nz + k], d1 = d[2 * nz + k], d2 = d[3 * nz + k];
        const double zu = c1 * (double)uzm * ((double)wzm + (double)wzm_xp) -
                          c2 * (double)uzp * ((double)w0 + (double)wxp);
        const double zv = c1 * (double)vzm * ((double)wzm + (double)wzm_yp) -
                          c2 * (double)vzp * ((double)w0 + (double)wyp);
        const double zw = d1 * (double)wzm * ((double)w0 + (double)wzm) -
                          d2 * (double)wzp * ((double)w0 + (double)wzp);
        ou = (C)((double)ou + zu);
        ov = (C)((double)ov + zv);
        ow = (C)((double)ow + zw);
      } else {
        const C c1 = S::coef(a.c, TZC1, nz, k), c2 = S::coef(a.c, TZC2, nz, k);
        const C d1 = S::coef(a.c, TZD1, nz, k), d2 = S::coef(a.c, TZD2, nz, k);
        ou = ou + c1 * uzm * (wzm + wzm_xp) - c2 * uzp * (w0 + wxp);
        ov = ov + c1 * vzm * (wzm + wzm_yp) - c2 * vzp * (w0 + wyp);
        ow = ow + d1 * wzm * (w0 + wzm) - d2 * wzp * (w0 + wzp);
      }
      if (k == nz - 1) ow = 0;
    }
    if (a.integ) {  // integration epilogue: base + dt * source term
      C dt;
      step_into(dt, a);
      const C bu = a.bu ? S::load((const T*)a.bu, t, a.sc.base[0]) : U.at(i, j, k);
      const C bv = a.bv ? S::load((const T*)a.bv, t, a.sc.base[1]) : V.at(i, j, k);
      const C bw = a.bw ? S::load((const T*)a.bw, t, a.sc.base[2]) : W.at(i, j, k);
      ou = bu + dt * ou;
      ov = bv + dt * ov;
      ow = bw + dt * ow;
    }
    S::store(su, t, ou, a.sc.inv_out[0]);
    S::store(sv, t, ov, a.sc.inv_out[1]);
    S::store(sw, t, ow, a.sc.inv_out[2]);
  }
}

// ---------------------------------------------------------------- adjoint
// Gather form of J^T: each point sums every forward term that reads it
// (product rule on coefficient * A * (B + C)), with cotangents masked to the
// levels the forward computes (su, sv: 1..nz-1; sw: 1..nz-2).
template <typename T>
__global__ void __launch_bounds__(kThreads)
adj_point_kernel(AdjArgs a) {
  using S = Store<T>;
  using C = typename S::C;
  const int nx = a.s.nx, ny = a.s.ny, nz = a.s.nz;
  const Grid3<T> U{(const T*)a.u, nx, ny, nz, 1.f}, V{(const T*)a.v, nx, ny, nz, 1.f},
      W{(const T*)a.w, nx, ny, nz, 1.f};
  const Grid3<T> GU{(const T*)a.dsu, nx, ny, nz, 1.f}, GV{(const T*)a.dsv, nx, ny, nz, 1.f},
      GW{(const T*)a.dsw, nx, ny, nz, 1.f};
  T* du = (T*)a.du;
  T* dv = (T*)a.dv;
  T* dw = (T*)a.dw;
  const size_t n = (size_t)nx * ny * nz;
  const C tcx = S::tcx(a.c), tcy = S::tcy(a.c);
  auto coef = [&](int table, int k) -> C {
    return (k < 0 || k >= nz) ? C(0) : S::coef(a.c, table, nz, k);
  };
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(t % nz);
    const size_t col = t / nz;
    const int j = (int)(col % ny);
    const int i = (int)(col / ny);
    auto Lu = [&](int di, int dj, int dk) -> C {
      const int kk = k + dk;
      return (kk >= 1 && kk <= nz - 1) ? GU.at(i + di, j + dj, kk) : C(0);
    };
    auto Lv = [&](int di, int dj, int dk) -> C {
      const int kk = k + dk;
      return (kk >= 1 && kk <= nz - 1) ? GV.at(i + di, j + dj, kk) : C(0);
    };
    auto Lw = [&](int di, int dj, int dk) -> C {
      const int kk = k + dk;
      return (kk >= 1 && kk <= nz - 2) ? GW.at(i + di, j + dj, kk) : C(0);
    };
    const C u0 = U.at(i, j, k), uxm = U.at(i - 1, j, k), uxp = U.at(i + 1, j, k);
    const C uyp = U.at(i, j + 1, k), uzp = U.at(i, j, k + 1);
    const C uxm_yp = U.at(i - 1, j + 1, k), uxm_zp = U.at(i - 1, j, k + 1);
    const C v0 = V.at(i, j, k), vxp = V.at(i + 1, j, k), vym = V.at(i, j - 1, k);
    const C vyp = V.at(i, j + 1, k), vzp = V.at(i, j, k + 1);
    const C vym_xp = V.at(i + 1, j - 1, k), vym_zp = V.at(i, j - 1, k + 1);
    const C w0 = W.at(i, j, k), wxp = W.at(i + 1, j, k), wyp = W.at(i, j + 1, k);
    const C wzm = W.at(i, j, k - 1), wzp = W.at(i, j, k + 1);
    const C wzm_xp = W.at(i + 1, j, k - 1), wzm_yp = W.at(i, j + 1, k - 1);

    const C lu0 = Lu(0, 0, 0), luxp = Lu(1, 0, 0), luxm = Lu(-1, 0, 0);
    const C luyp = Lu(0, 1, 0), luym = Lu(0, -1, 0), luzp = Lu(0, 0, 1), luzm = Lu(0, 0, -1);
    const C luxm_yp = Lu(-1, 1, 0), luxm_zp = Lu(-1, 0, 1);
    const C lv0 = Lv(0, 0, 0), lvxp = Lv(1, 0, 0), lvxm = Lv(-1, 0, 0);
    const C lvyp = Lv(0, 1, 0), lvym = Lv(0, -1, 0), lvzp = Lv(0, 0, 1), lvzm = Lv(0, 0, -1);
    const C lvxp_ym = Lv(1, -1, 0), lvym_zp = Lv(0, -1, 1);
    const C lw0 = Lw(0, 0, 0), lwxp = Lw(1, 0, 0), lwxm = Lw(-1, 0, 0);
    const C lwyp = Lw(0, 1, 0), lwym = Lw(0, -1, 0), lwzp = Lw(0, 0, 1), lwzm = Lw(0, 0, -1);
    const C lwxp_zm = Lw(1, 0, -1), lwyp_zm = Lw(0, 1, -1);
    const C tzc1_up = coef(TZC1, k + 1), tzc2_dn = coef(TZC2, k - 1), tzc2_0 = coef(TZC2, k);
    const C tzd1_0 = coef(TZD1, k), tzd1_up = coef(TZD1, k + 1);
    const C tzd2_0 = coef(TZD2, k), tzd2_dn = coef(TZD2, k - 1);

    // du
    C gu = tcx * (luxp * (uxp + u0 + u0) + lu0 * (uxm - uxp) - luxm * (uxm + u0 + u0));
    gu += tcy * (luyp * (v0 + vxp) - luym * (vym + vym_xp));
    gu += tzc1_up * luzp * (w0 + wxp) - tzc2_dn * luzm * (wzm + wzm_xp);
    gu += tcx * (lvxp * v0 + lvxp_ym * vym - lv0 * vxp - lvym * vym_xp);
    gu += tcx * (lwxp * w0 + lwxp_zm * wzm - lw0 * wxp - lwzm * wzm_xp);
    // dv
    C gv = tcy * (luyp * u0 + luxm_yp * uxm - lu0 * uyp - luxm * uxm_yp);
    gv += tcx * (lvxp * (u0 + uyp) - lvxm * (uxm + uxm_yp));
    gv += tcy * (lvyp * (vyp + v0 + v0) + lv0 * (vym - vyp) - lvym * (vym + v0 + v0));
    gv += tzc1_up * lvzp * (w0 + wyp) - tzc2_dn * lvzm * (wzm + wzm_yp);
    gv += tcy * (lwyp * w0 + lwyp_zm * wzm - lw0 * wyp - lwzm * wzm_yp);
    // dw
    C gw = tzc1_up * (luzp * u0 + luxm_zp * uxm + lvzp * v0 + lvym_zp * vym);
    gw -= tzc2_0 * (lu0 * uzp + luxm * uxm_zp + lv0 * vzp + lvym * vym_zp);
    gw += tcx * (lwxp * (u0 + uzp) - lwxm * (uxm + uxm_zp));
    gw += tcy * (lwyp * (v0 + vzp) - lwym * (vym + vym_zp));
    gw += tzd1_up * lwzp * (wzp + w0 + w0) + lw0 * (tzd1_0 * wzm - tzd2_0 * wzp) -
          tzd2_dn * lwzm * (wzm + w0 + w0);
    S::store(du, t, gu, 1.f);
    S::store(dv, t, gv, 1.f);
    S::store(dw, t, gw, 1.f);
  }
}

int grid_for(size_t n) {
  size_t b = (n + kThreads - 1) / kThreads;
  const size_t cap = 152 * 16;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

}  // namespace

cudaError_t launch_fwd_point(int dtype, const FwdArgs& a, cudaStream_t st) {
  const size_t n = (size_t)(a.i1 - a.i0) * a.s.ny * a.s.nz;
  if (n == 0) return cudaSuccess;
  const int g = grid_for(n);
  switch (dtype) {
    case kF64: fwd_point_kernel<double><<<g, kThreads, 0, st>>>(a); break;
    case kF32: fwd_point_kernel<float><<<g, kThreads, 0, st>>>(a); break;
    case kF16S: fwd_point_kernel<__half><<<g, kThreads, 0, st>>>(a); break;
    case kF64FF: fwd_point_kernel<f64ff><<<g, kThreads, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_adj_point(int dtype, const AdjArgs& a, cudaStream_t st) {
  const size_t n = (size_t)a.s.nx * a.s.ny * a.s.nz;
  const int g = grid_for(n);
  switch (dtype) {
    case kF64: adj_point_kernel<double><<<g, kThreads, 0, st>>>(a); break;
    case kF32: adj_point_kernel<float><<<g, kThreads, 0, st>>>(a); break;
    case kF64FF: adj_point_kernel<f64ff><<<g, kThreads, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace advect
