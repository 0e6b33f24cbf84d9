/*
 * A plain C99 user of the library's C ABI (include/advect.h): builds the
 * coefficients of a uniform vertical grid, fills u, v, w with a fixed
 * pattern, runs the forward pass from host buffers and writes su, sv, sw to a
 * binary file.  Usage: forward_host NX NY NZ OUT_FILE.  Exit status 0 on
 * success; on failure prints the library's error message.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "advect.h"

static int fail(const char *what, advect_status s) {
    fprintf(stderr, "%s failed (status %d): %s\n", what, (int)s, advect_last_error());
    return 1;
}

/* the input pattern (the test reproduces it) */
static double pattern(int f, int i, int j, int k) {
    return 8.0 * sin(0.37 * i + 0.23 * j + 0.11 * k + 1.3 * f) + 0.5 * f;
}

int main(int argc, char **argv) {
    if (argc != 5) {
        fprintf(stderr, "usage: %s NX NY NZ OUT_FILE\n", argv[0]);
        return 2;
    }
    const int nx = atoi(argv[1]), ny = atoi(argv[2]), nz = atoi(argv[3]);
    const size_t n = (size_t)nx * ny * nz;
    double *z = malloc(nz * sizeof *z), *zn = malloc(nz * sizeof *zn);
    double *rho = malloc(nz * sizeof *rho), *rhon = malloc(nz * sizeof *rhon);
    double *tab = malloc(4 * (size_t)nz * sizeof *tab);
    double *fld = malloc(6 * n * sizeof *fld);
    if (!z || !zn || !rho || !rhon || !tab || !fld) return 3;
    for (int k = 0; k < nz; ++k) {
        z[k] = 10.0 * k;
        zn[k] = 10.0 * k - 5.0;
        rho[k] = rhon[k] = 1.0;
    }
    advect_grid g = {nz, 50.0, 50.0, z, zn, rho, rhon};
    advect_coeffs c;
    advect_status s = advect_coeffs_from_grid(&g, &c.tcx, &c.tcy, tab, tab + nz, tab + 2 * nz, tab + 3 * nz);
    if (s != ADVECT_OK) return fail("advect_coeffs_from_grid", s);
    c.tzc1 = tab;
    c.tzc2 = tab + nz;
    c.tzd1 = tab + 2 * nz;
    c.tzd2 = tab + 3 * nz;
    for (int f = 0; f < 3; ++f)
        for (int i = 0; i < nx; ++i)
            for (int j = 0; j < ny; ++j)
                for (int k = 0; k < nz; ++k) fld[f * n + ((size_t)i * ny + j) * nz + k] = pattern(f, i, j, k);
    advect_ctx *ctx = NULL;
    s = advect_create(nx, ny, nz, &c, ADVECT_F64, &ctx);
    if (s != ADVECT_OK) return fail("advect_create", s);
    s = advect_forward_host(ctx, fld, fld + n, fld + 2 * n, fld + 3 * n, fld + 4 * n, fld + 5 * n, NULL);
    if (s != ADVECT_OK) return fail("advect_forward_host", s);
    advect_destroy(ctx);
    FILE *out = fopen(argv[4], "wb");
    if (!out || fwrite(fld + 3 * n, sizeof *fld, 3 * n, out) != 3 * n) return 4;
    fclose(out);
    free(z);
    free(zn);
    free(rho);
    free(rhon);
    free(tab);
    free(fld);
    return 0;
}
