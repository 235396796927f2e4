/* Per-call cost of one block step through the GRAPE calling sequence
 * (Sect. 2.1, 2.5): for block sizes m = 1 .. 4096 against n j-particles,
 * each repetition updates the m j-records (g6x_set_j_particles), sets a new
 * block time (g6_set_ti, so the j-particles are predicted again), starts
 * the force (g6calc_firsthalf) and waits for it (g6calc_lasthalf2).  Prints
 * one JSON line per m: the host wall time of each call (microseconds, mean
 * over the repetitions after 20 warm-up ones), then, from a second pass of
 * the same repetitions with the library's CUDA-event timing on (which also
 * launches every kernel on its own, without programmatic dependent launch),
 * the device time of each phase, and the launch configuration.
 * Arguments: n, repetitions, and "tune" to run the autotuner first.
 * Particles are uniform in a unit cube (the cost does not depend on their
 * positions); eps2 = 1e-4. */
#define _POSIX_C_SOURCE 199309L
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#include "g6gb.h"

static double now_us(void)
{
    struct timespec t;
    clock_gettime(CLOCK_MONOTONIC, &t);
    return t.tv_sec * 1e6 + t.tv_nsec * 1e-3;
}

static double urand(unsigned *s)
{
    *s = *s * 1664525u + 1013904223u;
    return (*s >> 8) * (1.0 / 16777216.0);
}

int main(int argc, char **argv)
{
    const int n = argc > 1 ? atoi(argv[1]) : 32768;
    const int reps = argc > 2 ? atoi(argv[2]) : 300;
    const int tune = argc > 3 && strcmp(argv[3], "tune") == 0;
    if (n < 8192 || reps < 1)
        return 2;
    double *m = malloc(sizeof(double) * n), *tj = malloc(sizeof(double) * n);
    double(*x)[3] = malloc(sizeof(double[3]) * n), (*v)[3] = malloc(sizeof(double[3]) * n);
    double(*z)[3] = calloc(n, sizeof(double[3]));
    double(*acc)[3] = malloc(sizeof(double[3]) * n), (*jerk)[3] = malloc(sizeof(double[3]) * n);
    double *pot = malloc(sizeof(double) * n);
    int *idx = malloc(sizeof(int) * n), *nnb = malloc(sizeof(int) * n);
    if (!m || !tj || !x || !v || !z || !acc || !jerk || !pot || !idx || !nnb)
        return 3;
    unsigned s = 12345;
    for (int k = 0; k < n; ++k) {
        m[k] = 1.0 / n;
        tj[k] = 0.0;
        idx[k] = k;
        for (int d = 0; d < 3; ++d) {
            x[k][d] = urand(&s) - 0.5;
            v[k][d] = 0.1 * (urand(&s) - 0.5);
        }
    }
    int rc = g6x_open_ex(0, n, 4096);
    if (!rc)
        rc = g6x_set_j_particles(0, n, idx, idx, tj, m, (const double(*)[3])z,
                                 (const double(*)[3])z, (const double(*)[3])v,
                                 (const double(*)[3])x);
    if (!rc && tune)
        rc = g6x_autotune(0, n, 4096, NULL) < 0;
    if (rc) {
        fprintf(stderr, "setup failed: %d\n", rc);
        return 1;
    }
    const int ms[] = {1, 16, 64, 256, 1024, 4096};
    double t = 0.0;
    for (int mi = 0; mi < 6; ++mi) {
        const int mm = ms[mi];
        double tset = 0, tti = 0, tfh = 0, tlh = 0;
        int off = 0;
        for (int r = 0; r < 2 * reps + 20; ++r) {
            if (r == reps + 20)
                g6x_set_timing(0, 1);
            t += 1.0 / 1048576.0;
            for (int k = 0; k < mm; ++k)
                tj[off + k] = t;
            const double t0 = now_us();
            rc = g6x_set_j_particles(0, mm, idx + off, idx + off, tj + off, m + off,
                                     (const double(*)[3])z, (const double(*)[3])z,
                                     (const double(*)[3])(v + off),
                                     (const double(*)[3])(x + off));
            const double t1 = now_us();
            rc |= g6_set_ti(0, t);
            const double t2 = now_us();
            g6calc_firsthalf(0, n, mm, idx + off, (const double(*)[3])(x + off),
                             (const double(*)[3])(v + off), NULL, NULL, NULL, 1e-4, NULL);
            const double t3 = now_us();
            rc |= g6calc_lasthalf2(0, n, mm, idx + off, (const double(*)[3])(x + off),
                                   (const double(*)[3])(v + off), 1e-4, NULL, acc, jerk, pot,
                                   nnb);
            const double t4 = now_us();
            if (rc) {
                fprintf(stderr, "m = %d: error %d\n", mm, rc);
                return 1;
            }
            if (r >= 20 && r < reps + 20) {
                tset += t1 - t0;
                tti += t2 - t1;
                tfh += t3 - t2;
                tlh += t4 - t3;
            }
            off = (off + mm) % (n - mm);
        }
        double gms[4];
        long long cnt[4];
        int var, ti, tjj, nip, grid, jtl;
        g6x_get_timing(0, gms, cnt);
        g6x_set_timing(0, 0);
        g6x_last_config(0, &var, &ti, &tjj, &nip, &grid, &jtl);
        printf("{\"n\": %d, \"m\": %d, \"tuned\": %s, \"host_us\": {\"set_j\": %.2f, "
               "\"set_ti\": %.2f, \"firsthalf\": %.2f, \"lasthalf\": %.2f, \"total\": %.2f}, "
               "\"device_us\": {\"store_predict\": %.2f, \"force\": %.2f, \"reduce\": %.2f}, "
               "\"launches_per_call\": %.2f, \"config\": {\"variant\": %d, \"shape\": \"%dx%dx%d\", "
               "\"grid\": %d, \"jtiles\": %d}}\n",
               n, mm, tune ? "true" : "false", tset / reps, tti / reps, tfh / reps, tlh / reps,
               (tset + tti + tfh + tlh) / reps, 1e3 * (gms[0] + gms[1]) / reps,
               1e3 * gms[2] / reps, 1e3 * gms[3] / reps,
               (double)(cnt[0] + cnt[1] + cnt[2] + cnt[3]) / reps, var, ti, tjj, nip, grid, jtl);
        fflush(stdout);
    }
    g6_close(0);
    return 0;
}
