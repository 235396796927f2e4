/* A plain C11 client of the library's GRAPE-6 calling sequence (Sect. 2.1,
 * 2.5): reads n particles (mass, x[3], v[3] per line) from argv[1], stores
 * them as j-particles, computes the force on all of them at t = 0 with
 * softening eps2 = argv[3] and neighbour radius^2 h2 = argv[4], and writes
 * one line per particle to argv[2]: acc[3] jerk[3] pot nnb nblen.  Exit
 * status 0 on success, else the library's error code (negated). */
#include <stdio.h>
#include <stdlib.h>

#include "g6gb.h"

int main(int argc, char **argv)
{
    if (argc != 5)
        return 2;
    FILE *in = fopen(argv[1], "r");
    if (!in)
        return 3;
    int n = 0;
    if (fscanf(in, "%d", &n) != 1 || n < 1)
        return 4;
    double *m = malloc(sizeof(double) * n);
    double(*x)[3] = malloc(sizeof(double[3]) * n);
    double(*v)[3] = malloc(sizeof(double[3]) * n);
    double(*acc)[3] = malloc(sizeof(double[3]) * n);
    double(*jerk)[3] = malloc(sizeof(double[3]) * n);
    double *pot = malloc(sizeof(double) * n), *h2 = malloc(sizeof(double) * n);
    int *idx = malloc(sizeof(int) * n), *nnb = malloc(sizeof(int) * n);
    int *nbl = malloc(sizeof(int) * G6_MAXNB);
    for (int k = 0; k < n; ++k) {
        if (fscanf(in, "%lf %lf %lf %lf %lf %lf %lf", &m[k], &x[k][0], &x[k][1], &x[k][2],
                   &v[k][0], &v[k][1], &v[k][2]) != 7)
            return 5;
        idx[k] = k;
    }
    fclose(in);
    const double eps2 = atof(argv[3]), radius2 = atof(argv[4]);
    const double zero[3] = {0.0, 0.0, 0.0};
    int rc = g6x_open_ex(0, n, n);
    for (int k = 0; !rc && k < n; ++k)
        rc = g6_set_j_particle(0, k, k, 0.0, 0.0, m[k], zero, zero, zero, v[k], x[k]);
    if (!rc)
        rc = g6_set_ti(0, 0.0);
    for (int k = 0; k < n; ++k)
        h2[k] = radius2;
    if (!rc) {
        g6calc_firsthalf(0, n, n, idx, (const double(*)[3])x, (const double(*)[3])v, NULL,
                         NULL, NULL, eps2, h2);
        rc = g6calc_lasthalf2(0, n, n, idx, (const double(*)[3])x, (const double(*)[3])v, eps2,
                              h2, acc, jerk, pot, nnb);
    }
    if (!rc) {
        const int lr = g6_read_neighbour_list(0);
        rc = lr < 0 ? lr : 0;
    }
    FILE *out = rc ? NULL : fopen(argv[2], "w");
    for (int k = 0; out && k < n; ++k) {
        int len = 0;
        const int r = g6_get_neighbour_list(0, k, G6_MAXNB, &len, nbl);
        if (r < 0) {
            rc = r;
            break;
        }
        fprintf(out, "%.17g %.17g %.17g %.17g %.17g %.17g %.17g %d %d\n", acc[k][0], acc[k][1],
                acc[k][2], jerk[k][0], jerk[k][1], jerk[k][2], pot[k], nnb[k], len);
    }
    if (out)
        fclose(out);
    g6_close(0);
    free(m);
    free(x);
    free(v);
    free(acc);
    free(jerk);
    free(pot);
    free(h2);
    free(idx);
    free(nnb);
    free(nbl);
    return rc ? (rc < 0 ? -rc : rc) : 0;
}
