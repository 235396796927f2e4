/*
 * oracle.c -- plain FP64 CPU oracle for the direct-summation Hermite hot path
 * of arXiv:0902.4463 ("SAPPORO").
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * Every function is the textbook definition in double precision, in the order
 * the paper (or the work it cites for the integrator) states it.  The only
 * parallelism is an OpenMP loop over independent i-particles.
 *
 * Readings of points the paper leaves open (the paper prints neither the force
 * nor the corrector formulas; it cites Makino & Aarseth 1992 and Aarseth 1985):
 *   - pair force and jerk: standard Plummer-softened Hermite forms;
 *   - potential: negative physical potential, -sum m_j / sqrt(r^2 + eps^2);
 *   - self-interaction: skipped when the i and j indices match;
 *   - nearest neighbour: smallest unsoftened |r|^2, ties to the lower j
 *     position, -1 if no other particle exists;
 *   - neighbour list: strict |r|^2 < h2_i, ascending j, truncated at maxnb.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- predictor */

/* Eq. 1 and Eq. 2 (Sect. 2.2). */
void orc_predict(long n, const double *x0, const double *v0, const double *a0,
                 const double *j0, const double *tj, double t,
                 double *xp, double *vp)
{
    for (long k = 0; k < n; ++k) {
        double dt = t - tj[k];
        for (int c = 0; c < 3; ++c) {
            double x = x0[3 * k + c], v = v0[3 * k + c];
            double a = a0[3 * k + c], j = j0[3 * k + c];
            xp[3 * k + c] = x + v * dt + a * dt * dt / 2.0 + j * dt * dt * dt / 6.0;
            vp[3 * k + c] = v + a * dt + j * dt * dt / 2.0;
        }
    }
}

/* ------------------------------------------------------------- pair forces */

/* Sect. 2.3 (calculation step) and Sect. 2.5 (softening per i-block, nearest
 * neighbour).  Plain double loop, j in ascending order. */
void orc_force(long ni, const double *xi, const double *vi, const int *idx_i,
               long nj, const double *xj, const double *vj, const double *mj,
               const int *idx_j, double eps2,
               double *acc, double *jerk, double *pot, int *nnb, double *nnr2)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (long i = 0; i < ni; ++i) {
        double ax = 0, ay = 0, az = 0, jx = 0, jy = 0, jz = 0, phi = 0;
        double best = HUGE_VAL;
        int bestj = -1;
        for (long j = 0; j < nj; ++j) {
            if (idx_j[j] == idx_i[i])
                continue;                               /* self-interaction */
            double rx = xj[3 * j + 0] - xi[3 * i + 0];
            double ry = xj[3 * j + 1] - xi[3 * i + 1];
            double rz = xj[3 * j + 2] - xi[3 * i + 2];
            double ux = vj[3 * j + 0] - vi[3 * i + 0];
            double uy = vj[3 * j + 1] - vi[3 * i + 1];
            double uz = vj[3 * j + 2] - vi[3 * i + 2];
            double r2 = rx * rx + ry * ry + rz * rz;
            double s2 = r2 + eps2;
            double s = sqrt(s2);
            double s3 = s2 * s;
            double s5 = s3 * s2;
            double rv = rx * ux + ry * uy + rz * uz;
            double m = mj[j];
            ax += m * rx / s3;
            ay += m * ry / s3;
            az += m * rz / s3;
            jx += m * (ux / s3 - 3.0 * rv * rx / s5);
            jy += m * (uy / s3 - 3.0 * rv * ry / s5);
            jz += m * (uz / s3 - 3.0 * rv * rz / s5);
            phi -= m / s;
            if (r2 < best) {
                best = r2;
                bestj = (int)j;
            }
        }
        if (acc) { acc[3 * i] = ax; acc[3 * i + 1] = ay; acc[3 * i + 2] = az; }
        if (jerk) { jerk[3 * i] = jx; jerk[3 * i + 1] = jy; jerk[3 * i + 2] = jz; }
        if (pot) pot[i] = phi;
        if (nnb) nnb[i] = bestj;
        if (nnr2) nnr2[i] = best;
    }
}

/* Sect. 4: neighbour lists with a compile-time style maximum length. */
long orc_neighbours(long ni, const double *xi, const int *idx_i, long nj,
                    const double *xj, const int *idx_j, const double *h2,
                    int maxnb, int *nblen, int *nbl)
{
    long overflowed = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : overflowed)
    for (long i = 0; i < ni; ++i) {
        int cnt = 0;
        for (long j = 0; j < nj; ++j) {
            if (idx_j[j] == idx_i[i])
                continue;
            double rx = xj[3 * j + 0] - xi[3 * i + 0];
            double ry = xj[3 * j + 1] - xi[3 * i + 1];
            double rz = xj[3 * j + 2] - xi[3 * i + 2];
            double r2 = rx * rx + ry * ry + rz * rz;
            if (r2 < h2[i]) {
                if (cnt < maxnb)
                    nbl[(long)maxnb * i + cnt] = (int)j;
                ++cnt;
            }
        }
        nblen[i] = cnt;
        if (cnt > maxnb)
            ++overflowed;
    }
    return overflowed;
}

/* ------------------------------------------------------------- integrator */

/* Makino & Aarseth (1992) Hermite corrector (the scheme named in Sect. 2):
 * the cubic Hermite interpolant of a(t) through (a0, j0) and (a1, j1) gives
 * the second and third derivatives at t0, which add the dt^4 and dt^5 terms
 * missing from the prediction. */
void orc_hermite_correct(double dt, const double xp[3], const double vp[3],
                         const double a0[3], const double j0[3],
                         const double a1[3], const double j1[3],
                         double x1[3], double v1[3], double a2[3], double a3[3])
{
    double dt2 = dt * dt, dt3 = dt2 * dt, dt4 = dt3 * dt, dt5 = dt4 * dt;
    for (int c = 0; c < 3; ++c) {
        double d2 = (-6.0 * (a0[c] - a1[c]) - dt * (4.0 * j0[c] + 2.0 * j1[c])) / dt2;
        double d3 = (12.0 * (a0[c] - a1[c]) + 6.0 * dt * (j0[c] + j1[c])) / dt3;
        x1[c] = xp[c] + d2 * dt4 / 24.0 + d3 * dt5 / 120.0;
        v1[c] = vp[c] + d2 * dt3 / 6.0 + d3 * dt4 / 24.0;
        a2[c] = d2;
        a3[c] = d3;
    }
}

static double norm3(const double *a)
{
    return sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
}

/* Aarseth (1985) criterion, cited in Sect. 3.1 and 3.2. */
double orc_aarseth_dt(const double a[3], const double j[3], const double a2[3],
                      const double a3[3], double eta)
{
    double na = norm3(a), nj = norm3(j), n2 = norm3(a2), n3 = norm3(a3);
    return sqrt(eta * (na * n2 + nj * nj) / (nj * n3 + n2 * n2));
}

/* Power-of-two block time steps (Sect. 2, Sect. 2.1). */
double orc_block_dt(double dt_old, double dt_req, double t, double dt_max,
                    double dt_min)
{
    double dt = dt_old;
    if (dt_req < dt) {
        while (dt > dt_req)
            dt *= 0.5;
    } else if (dt_req >= 2.0 * dt && 2.0 * dt <= dt_max
               && fmod(t, 2.0 * dt) == 0.0) {
        dt *= 2.0;
    }
    if (dt < dt_min)
        return -1.0;
    return dt;
}

/* Sect. 3.2: total energy as an explicit pair loop. */
double orc_energy(long n, const double *m, const double *x, const double *v,
                  double eps2)
{
    double kin = 0.0, pot = 0.0;
    for (long i = 0; i < n; ++i)
        kin += 0.5 * m[i] * (v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1]
                             + v[3 * i + 2] * v[3 * i + 2]);
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : pot)
    for (long i = 0; i < n; ++i) {
        double w = 0.0;
        for (long j = i + 1; j < n; ++j) {
            double rx = x[3 * j] - x[3 * i];
            double ry = x[3 * j + 1] - x[3 * i + 1];
            double rz = x[3 * j + 2] - x[3 * i + 2];
            w -= m[i] * m[j] / sqrt(rx * rx + ry * ry + rz * rz + eps2);
        }
        pot += w;
    }
    return kin + pot;
}

int orc_hermite_run(long n, const double *m, double *x, double *v,
                    double eps2, double eta, double eta_s, double dt_max,
                    double dt_min, double t_end, double *acc, double *jerk,
                    long *hist, orc_run_stats *st)
{
    orc_run_stats local = {0, 0, 0.0, 0};
    if (!st)
        st = &local;
    *st = local;
    if (n < 1 || !(dt_max > 0) || !(t_end >= 0) || fmod(t_end, dt_max) != 0.0) {
        st->err = -2;
        return -2;
    }
    double *a = malloc(sizeof(double) * 3 * n);
    double *jk = malloc(sizeof(double) * 3 * n);
    double *xp = malloc(sizeof(double) * 3 * n);
    double *vp = malloc(sizeof(double) * 3 * n);
    double *t = malloc(sizeof(double) * n);
    double *dt = malloc(sizeof(double) * n);
    int *idx = malloc(sizeof(int) * n);
    long *act = malloc(sizeof(long) * n);
    double *xa = malloc(sizeof(double) * 3 * n);
    double *va = malloc(sizeof(double) * 3 * n);
    int *ia = malloc(sizeof(int) * n);
    double *a1 = malloc(sizeof(double) * 3 * n);
    double *j1 = malloc(sizeof(double) * 3 * n);
    int rc = 0;

    for (long k = 0; k < n; ++k) {
        idx[k] = (int)k;
        t[k] = 0.0;
    }
    /* Initial force at t = 0 on every particle. */
    orc_force(n, x, v, idx, n, x, v, m, idx, eps2, a, jk, NULL, NULL, NULL);
    for (long k = 0; k < n; ++k) {
        double req = eta_s * norm3(&a[3 * k]) / norm3(&jk[3 * k]);
        double d = dt_max;
        while (d > req)
            d *= 0.5;
        if (d < dt_min) {
            rc = -1;
            goto done;
        }
        dt[k] = d;
    }

    for (;;) {
        /* Block scheduler: the earliest next time and the particles due. */
        double tb = HUGE_VAL;
        for (long k = 0; k < n; ++k)
            if (t[k] + dt[k] < tb)
                tb = t[k] + dt[k];
        if (tb > t_end)
            break;
        long na = 0;
        for (long k = 0; k < n; ++k)
            if (t[k] + dt[k] == tb)
                act[na++] = k;

        /* Predict every particle to tb (Eq. 1, Eq. 2). */
        orc_predict(n, x, v, a, jk, t, tb, xp, vp);

        /* Force on the active block from all particles (Sect. 2.3). */
        for (long q = 0; q < na; ++q) {
            long k = act[q];
            memcpy(&xa[3 * q], &xp[3 * k], 3 * sizeof(double));
            memcpy(&va[3 * q], &vp[3 * k], 3 * sizeof(double));
            ia[q] = idx[k];
        }
        orc_force(na, xa, va, ia, n, xp, vp, m, idx, eps2, a1, j1, NULL, NULL, NULL);

        /* Correct the active block and pick its next time step. */
        for (long q = 0; q < na; ++q) {
            long k = act[q];
            double h = tb - t[k];
            double x1[3], v1[3], d2[3], d3[3], d2e[3];
            orc_hermite_correct(h, &xp[3 * k], &vp[3 * k], &a[3 * k], &jk[3 * k],
                                &a1[3 * q], &j1[3 * q], x1, v1, d2, d3);
            for (int c = 0; c < 3; ++c)
                d2e[c] = d2[c] + h * d3[c];       /* a^(2) at the end of the step */
            double req = orc_aarseth_dt(&a1[3 * q], &j1[3 * q], d2e, d3, eta);
            double nd = orc_block_dt(dt[k], req, tb, dt_max, dt_min);
            if (nd < 0) {
                rc = -1;
                goto done;
            }
            memcpy(&x[3 * k], x1, sizeof x1);
            memcpy(&v[3 * k], v1, sizeof v1);
            memcpy(&a[3 * k], &a1[3 * q], 3 * sizeof(double));
            memcpy(&jk[3 * k], &j1[3 * q], 3 * sizeof(double));
            t[k] = tb;
            dt[k] = nd;
        }
        st->nblocks += 1;
        st->nactive += na;
        st->t = tb;
        if (hist) {
            int b = 0;
            while ((2L << b) <= na && b < 63)
                ++b;
            hist[b] += 1;
        }
    }
    if (acc)
        memcpy(acc, a, sizeof(double) * 3 * n);
    if (jerk)
        memcpy(jerk, jk, sizeof(double) * 3 * n);

done:
    st->err = rc;
    free(a); free(jk); free(xp); free(vp); free(t); free(dt); free(idx);
    free(act); free(xa); free(va); free(ia); free(a1); free(j1);
    return rc;
}
