/*
 * advect_oracle.c -- plain, slow, FP64 CPU oracle for the Piacsek-Williams (PW)
 * momentum-advection source terms of MONC (Brown, "Exploring the acceleration
 * of the Met Office NERC Cloud model using FPGAs", Sec. 2.1, Listing 1).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this file: only the tests, the smoke check and the benchmark's CPU
 * baseline use it.  It shares no code with the CUDA library.
 *
 * Compile with -O2 -ffp-contract=off so that every operation below is one
 * IEEE-754 binary64 operation in round-to-nearest-even, in the order written.
 *
 * Layout.  Arrays are [nx][ny][nz] with z contiguous, i.e. the Fortran
 * u(k,j,i) of Listing 1; element (i,j,k) sits at (i*ny + j)*nz + k.  Indices
 * here are 0-based: the paper's level k (1-based) is stored at k-1.  The
 * lateral directions are periodic (the halo of Sec. 2.1 is the periodic
 * image), so i-1, i+1, j-1, j+1 wrap modulo nx and ny.
 *
 * What is computed (Sec. 2.1, Listing 1; 0-based k):
 *   su  for k = 1 .. nz-1 exactly as Listing 1: x term, y term, then the
 *       vertical pair; at the top level (k = nz-1) the upper vertical flux
 *       (the tzc2 term) is omitted, as in Listing 1's else-branch.
 *   sv  the paper states that v and w are advected in the same loop with
 *       "very similar" expressions that it omits (Sec. 2.1).  The reading
 *       used: Listing 1's pattern on the same Arakawa-C staggering with the
 *       roles of x/u and y/v exchanged; same k range and top branch.
 *   sw  the same pattern for the w cell centred on a w level, k = 1 .. nz-2,
 *       with vertical coefficients tzd1/tzd2.
 *   Levels the loops never write (su, sv at k = 0; sw at k = 0 and nz-1) are
 *   set to zero.
 * Evaluation order for every field: ((x term + y term) + lower vertical)
 * - upper vertical, each term as coefficient * A * (B + C) left to right,
 * which is Listing 1's statement order.
 *
 * Coefficients (the paper uses tcx, tcy, tzc1, tzc2 without defining them;
 * the reading is the skew-symmetric PW form on the staggered grid):
 *   tcx = 1/(4 dx), tcy = 1/(4 dy)
 *   tzc1(k) = rho_w(k-1) / (4 dz(k) rho_n(k)),  tzc2(k) = rho_w(k) / (4 dz(k) rho_n(k))
 *   tzd1(k) = rho_n(k) / (4 dzn(k+1) rho_w(k)), tzd2(k) = rho_n(k+1) / (4 dzn(k+1) rho_w(k))
 *   with dz(k) = z(k) - z(k-1), dzn(k) = zn(k) - zn(k-1).
 *
 * Adjoint: the transpose of the Jacobian of (u,v,w) -> (su,sv,sw) applied to
 * cotangents (dsu,dsv,dsw), accumulated as a scatter with the product rule
 * on each term c*A*(B+C): dA += c*l*(B+C), dB += c*l*A, dC += c*l*A.
 */
#include <stddef.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define AT(i, j, k) ((((size_t)(i)) * (size_t)ny + (size_t)(j)) * (size_t)nz + (size_t)(k))

/* ---- coefficient setup -------------------------------------------------- */
int oracle_coefficients(int nz, double dx, double dy, const double *z, const double *zn,
                        const double *rho, const double *rhon, double *tcxy,
                        double *tzc1, double *tzc2, double *tzd1, double *tzd2)
{
    if (nz < 3 || !(dx > 0.0) || !(dy > 0.0))
        return 1;
    tcxy[0] = 1.0 / (4.0 * dx);
    tcxy[1] = 1.0 / (4.0 * dy);
    for (int k = 0; k < nz; ++k) {
        tzc1[k] = 0.0;
        tzc2[k] = 0.0;
        tzd1[k] = 0.0;
        tzd2[k] = 0.0;
    }
    for (int k = 1; k < nz; ++k) {
        double dzk = z[k] - z[k - 1];
        tzc1[k] = rho[k - 1] / (4.0 * dzk * rhon[k]);
        tzc2[k] = rho[k] / (4.0 * dzk * rhon[k]);
    }
    for (int k = 1; k < nz - 1; ++k) {
        double dznk1 = zn[k + 1] - zn[k];
        tzd1[k] = rhon[k] / (4.0 * dznk1 * rho[k]);
        tzd2[k] = rhon[k + 1] / (4.0 * dznk1 * rho[k]);
    }
    return 0;
}

/* ---- forward: one grid point --------------------------------------------- */
static void point(int nx, int ny, int nz, double tcx, double tcy,
                  const double *tzc1, const double *tzc2, const double *tzd1, const double *tzd2,
                  const double *u, const double *v, const double *w,
                  int i, int j, int k, double *out_su, double *out_sv, double *out_sw)
{
    int im = (i + nx - 1) % nx, ip = (i + 1) % nx;
    int jm = (j + ny - 1) % ny, jp = (j + 1) % ny;
    double su = 0.0, sv = 0.0, sw = 0.0;

    if (k >= 1) {
        /* su: Listing 1 */
        su = tcx * (u[AT(im, j, k)] * (u[AT(i, j, k)] + u[AT(im, j, k)])
                  - u[AT(ip, j, k)] * (u[AT(i, j, k)] + u[AT(ip, j, k)]));
        su = su + tcy * (u[AT(i, jm, k)] * (v[AT(i, jm, k)] + v[AT(ip, jm, k)])
                       - u[AT(i, jp, k)] * (v[AT(i, j, k)] + v[AT(ip, j, k)]));
        if (k < nz - 1) {
            su = su + tzc1[k] * u[AT(i, j, k - 1)] * (w[AT(i, j, k - 1)] + w[AT(ip, j, k - 1)])
                    - tzc2[k] * u[AT(i, j, k + 1)] * (w[AT(i, j, k)] + w[AT(ip, j, k)]);
        } else {
            su = su + tzc1[k] * u[AT(i, j, k - 1)] * (w[AT(i, j, k - 1)] + w[AT(ip, j, k - 1)]);
        }

        /* sv: Listing 1's pattern with x<->y, u<->v exchanged */
        sv = tcx * (v[AT(im, j, k)] * (u[AT(im, j, k)] + u[AT(im, jp, k)])
                  - v[AT(ip, j, k)] * (u[AT(i, j, k)] + u[AT(i, jp, k)]));
        sv = sv + tcy * (v[AT(i, jm, k)] * (v[AT(i, j, k)] + v[AT(i, jm, k)])
                       - v[AT(i, jp, k)] * (v[AT(i, j, k)] + v[AT(i, jp, k)]));
        if (k < nz - 1) {
            sv = sv + tzc1[k] * v[AT(i, j, k - 1)] * (w[AT(i, j, k - 1)] + w[AT(i, jp, k - 1)])
                    - tzc2[k] * v[AT(i, j, k + 1)] * (w[AT(i, j, k)] + w[AT(i, jp, k)]);
        } else {
            sv = sv + tzc1[k] * v[AT(i, j, k - 1)] * (w[AT(i, j, k - 1)] + w[AT(i, jp, k - 1)]);
        }

        /* sw: the same pattern on the w cell, interior w levels only */
        if (k < nz - 1) {
            sw = tcx * (w[AT(im, j, k)] * (u[AT(im, j, k)] + u[AT(im, j, k + 1)])
                      - w[AT(ip, j, k)] * (u[AT(i, j, k)] + u[AT(i, j, k + 1)]));
            sw = sw + tcy * (w[AT(i, jm, k)] * (v[AT(i, jm, k)] + v[AT(i, jm, k + 1)])
                           - w[AT(i, jp, k)] * (v[AT(i, j, k)] + v[AT(i, j, k + 1)]));
            sw = sw + tzd1[k] * w[AT(i, j, k - 1)] * (w[AT(i, j, k)] + w[AT(i, j, k - 1)])
                    - tzd2[k] * w[AT(i, j, k + 1)] * (w[AT(i, j, k)] + w[AT(i, j, k + 1)]);
        }
    }
    *out_su = su;
    *out_sv = sv;
    *out_sw = sw;
}

/* Forward over the x-planes i in [i_begin, i_end); other planes untouched.
 * Every point is computed on its own from the inputs, so the x-planes may be
 * shared out among threads: built with -fopenmp the loop over i runs on all
 * host cores and gives the same bits as the single-threaded build. */
int oracle_forward(int nx, int ny, int nz, double tcx, double tcy,
                   const double *tzc1, const double *tzc2, const double *tzd1, const double *tzd2,
                   const double *u, const double *v, const double *w,
                   double *su, double *sv, double *sw, int i_begin, int i_end)
{
    if (nx < 1 || ny < 1 || nz < 3 || i_begin < 0 || i_end > nx || i_begin > i_end)
        return 1;
#pragma omp parallel for schedule(static)
    for (int i = i_begin; i < i_end; ++i)
        for (int j = 0; j < ny; ++j)
            for (int k = 0; k < nz; ++k)
                point(nx, ny, nz, tcx, tcy, tzc1, tzc2, tzd1, tzd2, u, v, w, i, j, k,
                      &su[AT(i, j, k)], &sv[AT(i, j, k)], &sw[AT(i, j, k)]);
    return 0;
}

/* Threads oracle_forward uses: 1 unless built with -fopenmp. */
int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---- adjoint (scatter) ---------------------------------------------------- */
/* One term c*A*(B+C) of output q, with cotangent l: product rule. */
static void term(double c, double l, const double *fa, size_t a, const double *fb, size_t b,
                 const double *fc, size_t cc, double *ga, double *gb, double *gc)
{
    double s = c * l;
    ga[a] += s * (fb[b] + fc[cc]);
    gb[b] += s * fa[a];
    gc[cc] += s * fa[a];
}

int oracle_adjoint(int nx, int ny, int nz, double tcx, double tcy,
                   const double *tzc1, const double *tzc2, const double *tzd1, const double *tzd2,
                   const double *u, const double *v, const double *w,
                   const double *dsu, const double *dsv, const double *dsw,
                   double *du, double *dv, double *dw)
{
    if (nx < 1 || ny < 1 || nz < 3)
        return 1;
    size_t n = (size_t)nx * ny * nz;
    memset(du, 0, n * sizeof(double));
    memset(dv, 0, n * sizeof(double));
    memset(dw, 0, n * sizeof(double));
    for (int i = 0; i < nx; ++i) {
        int im = (i + nx - 1) % nx, ip = (i + 1) % nx;
        for (int j = 0; j < ny; ++j) {
            int jm = (j + ny - 1) % ny, jp = (j + 1) % ny;
            for (int k = 1; k < nz; ++k) {
                size_t q = AT(i, j, k);
                int top = (k == nz - 1);
                double l;

                l = dsu[q]; /* su terms */
                term(tcx, l, u, AT(im, j, k), u, AT(i, j, k), u, AT(im, j, k), du, du, du);
                term(-tcx, l, u, AT(ip, j, k), u, AT(i, j, k), u, AT(ip, j, k), du, du, du);
                term(tcy, l, u, AT(i, jm, k), v, AT(i, jm, k), v, AT(ip, jm, k), du, dv, dv);
                term(-tcy, l, u, AT(i, jp, k), v, AT(i, j, k), v, AT(ip, j, k), du, dv, dv);
                term(tzc1[k], l, u, AT(i, j, k - 1), w, AT(i, j, k - 1), w, AT(ip, j, k - 1), du, dw, dw);
                if (!top)
                    term(-tzc2[k], l, u, AT(i, j, k + 1), w, AT(i, j, k), w, AT(ip, j, k), du, dw, dw);

                l = dsv[q]; /* sv terms */
                term(tcx, l, v, AT(im, j, k), u, AT(im, j, k), u, AT(im, jp, k), dv, du, du);
                term(-tcx, l, v, AT(ip, j, k), u, AT(i, j, k), u, AT(i, jp, k), dv, du, du);
                term(tcy, l, v, AT(i, jm, k), v, AT(i, j, k), v, AT(i, jm, k), dv, dv, dv);
                term(-tcy, l, v, AT(i, jp, k), v, AT(i, j, k), v, AT(i, jp, k), dv, dv, dv);
                term(tzc1[k], l, v, AT(i, j, k - 1), w, AT(i, j, k - 1), w, AT(i, jp, k - 1), dv, dw, dw);
                if (!top)
                    term(-tzc2[k], l, v, AT(i, j, k + 1), w, AT(i, j, k), w, AT(i, jp, k), dv, dw, dw);

                if (top)
                    continue;
                l = dsw[q]; /* sw terms, interior w levels */
                term(tcx, l, w, AT(im, j, k), u, AT(im, j, k), u, AT(im, j, k + 1), dw, du, du);
                term(-tcx, l, w, AT(ip, j, k), u, AT(i, j, k), u, AT(i, j, k + 1), dw, du, du);
                term(tcy, l, w, AT(i, jm, k), v, AT(i, jm, k), v, AT(i, jm, k + 1), dw, dv, dv);
                term(-tcy, l, w, AT(i, jp, k), v, AT(i, j, k), v, AT(i, j, k + 1), dw, dv, dv);
                term(tzd1[k], l, w, AT(i, j, k - 1), w, AT(i, j, k), w, AT(i, j, k - 1), dw, dw, dw);
                term(-tzd2[k], l, w, AT(i, j, k + 1), w, AT(i, j, k), w, AT(i, j, k + 1), dw, dw, dw);
            }
        }
    }
    return 0;
}
