/*
 * advect.h -- C ABI of the GB300 (sm_103a) Piacsek-Williams momentum-advection
 * library.
 *
 * The operation is MONC's PW advection of the three wind components (Brown,
 * "Exploring the acceleration of the Met Office NERC Cloud model using FPGAs",
 * Sec. 2.1, Listing 1): for every grid point it forms the source terms
 * su, sv, sw from the winds u, v, w using the +-1 neighbours in x, y and z,
 * the horizontal coefficients tcx, tcy and the per-level vertical
 * coefficients tzc1/tzc2 (u and v) and tzd1/tzd2 (w).  All arithmetic in the
 * paper is double precision (Sec. 2.1).
 *
 * Data layout (all calls).  A field is a contiguous array [nx][ny][nz] with z
 * contiguous: element (i, j, k) (0-based) is at (i*ny + j)*nz + k, which is
 * the Fortran u(k,j,i) order of Listing 1 and the column-contiguous copies of
 * Listing 3.  The lateral directions are periodic.  Level k (0-based) is the
 * paper's level k+1.  su and sv are computed for k = 1..nz-1 with the upper
 * vertical flux dropped at k = nz-1 (Listing 1's else branch); sw for
 * k = 1..nz-2; every other level of an output is written as zero, so outputs
 * are fully overwritten.
 *
 * Element types (advect_dtype): ADVECT_F64 stores and computes in binary64;
 * ADVECT_F32 stores and computes in binary32 (coefficient tables kept in
 * binary64; optionally the vertical terms of the lowest levels in binary64 --
 * see advect_set_f64_levels); ADVECT_F16S stores binary16 values x/s with a
 * power-of-two scale s per field and computes in binary32 (the paper's
 * future-work precision trade-off, Sec. 6).  ADVECT_F64_FF stores binary64
 * (same buffers as ADVECT_F64) but computes each value as an unevaluated sum
 * of two binary32 numbers on the binary32 pipes, which on GB300 run 74x the
 * binary64 rate; results agree with binary64 to about 1e-14 normwise (never
 * worse than 1e-12 in the tests) for magnitudes in [2^-80, 2^126]; single
 * grids only (forward, integration step, adjoint, host path, no-allocation
 * call).
 *
 * Memory ownership.  Every buffer pointer is owned by the caller.  Device
 * pointers must be device memory of the current CUDA device, 16-byte aligned
 * for the fast paths (any alignment of the element size is accepted).  The
 * library copies coefficient tables at create time and keeps no pointer to
 * caller memory after a call returns.  Inputs must not overlap outputs or
 * outputs each other; inputs may share memory (they are only read).
 *
 * Streams and errors.  Device calls are asynchronous on the given stream
 * (NULL = legacy default stream).  Every call returns an advect_status;
 * nothing aborts and no C++ exception crosses the ABI.  On failure
 * advect_last_error() returns a message for the calling thread.  Kernels
 * report internal timeouts (bounded spin-waits) through a device flag that
 * the next call on the same context, or advect_sync(), turns into
 * ADVECT_ETIMEOUT.
 */
#ifndef ADVECT_H
#define ADVECT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;                       /* == cudaStream_t */
typedef struct CUstream_st *advect_stream;

typedef struct advect_ctx advect_ctx;      /* opaque, owned by the library */

typedef enum {
    ADVECT_OK = 0,
    ADVECT_EINVAL = 1,        /* bad argument: sizes, NULL, alias, alignment */
    ADVECT_ENOMEM = 2,        /* host or device allocation failed            */
    ADVECT_ECUDA = 3,         /* a CUDA runtime call failed                  */
    ADVECT_EUNSUPPORTED = 4,  /* valid request the library does not offer  */
    ADVECT_ETIMEOUT = 5       /* a kernel gave up a bounded wait             */
} advect_status;

typedef enum {
    ADVECT_F64 = 0,           /* binary64 storage and arithmetic             */
    ADVECT_F32 = 1,           /* binary32 storage and arithmetic             */
    ADVECT_F16S = 2,          /* binary16 storage with power-of-two scales   */
    ADVECT_F64_FF = 3         /* binary64 storage, double-float arithmetic    */
} advect_dtype;

/*
 * Vertical grid of one column set (host arrays of length nz, 0-based levels):
 *   z    heights of the w levels (cell tops), z[k] > z[k-1]
 *   zn   heights of the u/v levels, zn[k] between z[k-1] and z[k] for k >= 1
 *   rho  reference density on w levels, rhon on u/v levels (both > 0)
 *   dx, dy  horizontal spacing (> 0).
 */
typedef struct {
    int nz;
    double dx, dy;
    const double *z, *zn, *rho, *rhon;
} advect_grid;

/*
 * Advection coefficients (host arrays of length nz, level k at [k], entries a
 * formula never reads are ignored).  Listing 1 uses tcx, tcy, tzc1(k),
 * tzc2(k) (Sec. 2.1); tzd1(k), tzd2(k) are their w-cell analogues.
 */
typedef struct {
    double tcx, tcy;
    const double *tzc1, *tzc2, *tzd1, *tzd2;
} advect_coeffs;

/*
 * Coefficient setup (the paper uses but does not define them, Listing 1; the
 * definitions are those of the skew-symmetric PW form on the staggered grid):
 *   tcx = 1/(4 dx), tcy = 1/(4 dy),
 *   tzc1[k] = rho[k-1] / (4 dz_k rhon[k]),   tzc2[k] = rho[k] / (4 dz_k rhon[k]),   k = 1..nz-1
 *   tzd1[k] = rhon[k] / (4 dzn_k rho[k]),    tzd2[k] = rhon[k+1] / (4 dzn_k rho[k]), k = 1..nz-2
 * with dz_k = z[k] - z[k-1] and dzn_k = zn[k+1] - zn[k]; other entries are 0.
 * Outputs are caller-owned host arrays of length g->nz.  EINVAL if nz < 3,
 * a spacing or density is not positive, or the levels are not increasing.
 */
advect_status advect_coeffs_from_grid(const advect_grid *g, double *tcx, double *tcy,
                                      double *tzc1, double *tzc2, double *tzd1, double *tzd2);

/*
 * Create a context for one grid shape nx x ny x nz (nx, ny >= 1, nz >= 3) and
 * element type.  Copies the coefficient tables to the device, allocates the
 * context's small device state, and picks kernel tiles (from the tuning cache
 * when present).  *out receives the context; release it with advect_destroy.
 */
advect_status advect_create(int nx, int ny, int nz, const advect_coeffs *c, advect_dtype dtype,
                            advect_ctx **out);

/*
 * Forward pass (Sec. 2.1, Listing 1 and its v/w analogues): su, sv, sw from
 * u, v, w.  Device pointers, layout as above, element type of the context.
 * scales: ADVECT_F16S only, host array of 6 floats -- input scales of u, v, w
 * then output scales of su, sv, sw (stored value = true value / scale; use
 * advect_f16s_output_scales for a safe choice); every scale must be a
 * positive, finite power of two (EINVAL otherwise); NULL for other types.
 */
advect_status advect_forward(advect_ctx *ctx, const void *u, const void *v, const void *w,
                             void *su, void *sv, void *sw, const float *scales,
                             advect_stream stream);

/*
 * Forward pass fused with the step that integrates the source terms into the
 * flow fields (Sec. 2.1: later in the timestep the source terms are added to
 * the prognostic fields; the paper does not fix the time scheme):
 *   u_out = u_base + dt * su(u,v,w),  v_out = v_base + dt * sv,  w_out = w_base + dt * sw
 * at every point (so out = base on the levels where the source term is zero).
 * u_base, v_base, w_base: all NULL for the winds themselves (one explicit
 * step), or all three given (e.g. the previous time level with 2 dt for a
 * leapfrog step).  The source terms are never written to memory: the kernel
 * reads the three winds and writes the three results (plus reads the bases
 * when given).  Same layout, element type and tile configuration as
 * advect_forward; never runs the tuner.  In place: each base may be its own
 * output (u_out == u_base), since every base element is read only by the
 * thread that then writes that output element; a base must not otherwise
 * overlap an output, and the outputs must not overlap u, v, w or each other
 * (EINVAL).  dt must be finite (EINVAL).  scales (ADVECT_F16S only): 6 floats
 * (u, v, w, then u_out, v_out, w_out) without bases, 9 with them (then
 * u_base, v_base, w_base).  ADVECT_F64_FF: the base passes through the
 * double-float type, so it is carried to a 47-bit significand (relative
 * 2^-47) rather than returned bit for bit where the source term is zero.
 * Asynchronous on stream.
 */
advect_status advect_forward_integrate(advect_ctx *ctx, const void *u, const void *v, const void *w,
                                       const void *u_base, const void *v_base, const void *w_base,
                                       double dt, void *u_out, void *v_out, void *w_out,
                                       const float *scales, advect_stream stream);

/*
 * Adjoint (vector-Jacobian product) of the forward pass with respect to all
 * of (u, v, w): (du, dv, dw) = J(u,v,w)^T (dsu, dsv, dsw).  Computed as a
 * gather (each output point sums the terms that read it; no atomics).
 * Cotangents on levels the forward does not compute are ignored.  F64 and F32
 * contexts only (EUNSUPPORTED for F16S).
 */
advect_status advect_adjoint(advect_ctx *ctx, const void *u, const void *v, const void *w,
                             const void *dsu, const void *dsv, const void *dsw,
                             void *du, void *dv, void *dw, advect_stream stream);

/*
 * End-to-end forward from HOST buffers (the offload setting of Sec. 4-5:
 * fields in, source terms out).  u, v, w, su, sv, sw are host arrays of
 * nx*ny*nz elements of the context's type (pinned memory gives full copy
 * bandwidth; pageable memory works).  The x range is cut into chunks whose
 * host-to-device copy, kernel and device-to-host copy overlap on internal
 * streams (the chunked transfer proposed in Sec. 6); 32 chunks, or
 * $ADVECT_HOST_CHUNKS (1..64) read when the context is created.  Device
 * staging buffers are allocated on the first call and kept by the context.
 * Returns after the results are in su, sv, sw.
 */
advect_status advect_forward_host(advect_ctx *ctx, const void *u, const void *v, const void *w,
                                  void *su, void *sv, void *sw, const float *scales);

/*
 * F16S helper: output scales (powers of two) from input scales, using the a
 * priori bound |su| <= 4 tcx Mu^2 + 4 tcy Mu Mv + 2 max(tzc1 + tzc2) Mu Mw
 * (and its sv, sw analogues) with M the input scales.  in, out: host arrays
 * of 3 floats.
 */
advect_status advect_f16s_output_scales(const advect_ctx *ctx, const float *in, float *out);

/*
 * ADVECT_F32 / ADVECT_F16S: number of levels k = 1..n whose vertical terms
 * are evaluated in binary64 with the binary64 tables (near-surface levels,
 * where dz is smallest and the vertical fluxes largest).  0 (the default)
 * disables: on GB300 binary64 runs at 1/74 of the binary32 rate, so even two
 * such levels more than double the kernel time.  EINVAL if n < 0.
 */
advect_status advect_set_f64_levels(advect_ctx *ctx, int n);

/*
 * Ensemble: n independent grids of uneven shape (nx[m], ny[m], nz[m]) with
 * their own coefficients c[m], one element type.  Forward and adjoint run
 * every member in one persistent kernel launch (replayed from a CUDA graph
 * when the pointers repeat).  Pointer arguments are host arrays of n device
 * pointers, one per member.
 */
advect_status advect_ensemble_create(int n, const int *nx, const int *ny, const int *nz,
                                     const advect_coeffs *c, advect_dtype dtype, advect_ctx **out);
advect_status advect_ensemble_forward(advect_ctx *ctx, const void *const *u, const void *const *v,
                                      const void *const *w, void *const *su, void *const *sv,
                                      void *const *sw, advect_stream stream);
advect_status advect_ensemble_adjoint(advect_ctx *ctx, const void *const *u, const void *const *v,
                                      const void *const *w, const void *const *dsu,
                                      const void *const *dsv, const void *const *dsw,
                                      void *const *du, void *const *dv, void *const *dw,
                                      advect_stream stream);

/*
 * Autotuning (ensembles: tile length in x, ring depth and register cap;
 * single grids: the same plus the point kernel).  enable != 0: the next
 * forward and the next adjoint call on this context time every candidate on
 * that call's own buffers (CUDA events on the call's stream; the call
 * synchronises with its stream), keep the fastest, write it to the tuning
 * cache ($ADVECT_TUNE_CACHE, else ~/.cache/advect_gb300/tune.json) and finish
 * with it, so the outputs are those of the chosen kernel.  Contexts created
 * later for the same shapes, type and SM count start from the cached choice.
 * ADVECT_TUNE=1 in the environment enables this for every new context.  The
 * tiling never changes the arithmetic of a point.
 */
advect_status advect_autotune(advect_ctx *ctx, int enable);

/* The tile configuration in use for forward (0) or adjoint (1), as text. */
const char *advect_tuned_config(const advect_ctx *ctx, int adjoint);

/*
 * Forward pass that allocates no device memory (the paper has no counterpart;
 * this exists for callers, not for the method).  Some callers may not call
 * cudaMalloc: code inside a framework whose memory pool owns every device
 * allocation, latency-critical loops where an allocation can block or
 * synchronise the device, or programs that must keep their device footprint
 * fixed after start-up.  advect_create allocates (tables, error flag); this
 * call needs no context.
 *
 * Arguments are those of advect_create plus advect_forward: shape, host
 * coefficient tables, element type, device fields (u, v, w in; su, sv, sw
 * out; owned by the caller), F16S scales, stream.  Results equal
 * advect_forward's for the same inputs bit for bit (the same kernels run,
 * with the tile a new context of that type starts from).
 *
 * Scratch: the coefficient tables and the kernels' error flag live in one
 * fixed library array in device memory (ADVECT_NOALLOC_MAX_NZ levels,
 * about 24 KB), which every GPU that loads the library holds until the
 * process exits.  Each call rewrites the tables and clears the flag on its
 * stream before the forward kernel runs.  All calls on a device share that
 * one array: calls whose work can overlap on the GPU (different streams, or
 * several host threads) race -- order them on one stream or serialise them.
 * A kernel-side timeout (a bounded wait giving up, not expected in normal
 * operation) is cleared by the next call without being reported; use the
 * context API where those reports matter.
 *
 * The first call made on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it with the device's current driver
 * context; make that first call before any stream capture on that device.
 * After cudaDeviceReset, or under another context, the next call looks the
 * address up again (make it, too, outside a capture).
 *
 * EINVAL if nz > ADVECT_NOALLOC_MAX_NZ, or for the argument errors of
 * advect_create / advect_forward.
 */
#define ADVECT_NOALLOC_MAX_NZ 512
advect_status advect_forward_noalloc(int nx, int ny, int nz, const advect_coeffs *c, advect_dtype dtype,
                                     const void *u, const void *v, const void *w, void *su, void *sv,
                                     void *sw, const float *scales, advect_stream stream);

/* Wait for the context's work on `stream` and report any device-side timeout. */
advect_status advect_sync(advect_ctx *ctx, advect_stream stream);

/* Name of the kernel variant the context uses for forward / adjoint. */
const char *advect_kernel_name(const advect_ctx *ctx, int adjoint);

/* Release a context and its device state (NULL is a no-op). */
void advect_destroy(advect_ctx *ctx);

/* Message of the calling thread's most recent failure ("" if none). */
const char *advect_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ADVECT_H */
