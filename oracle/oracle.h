/*
 * oracle.h -- plain FP64 CPU oracle for the direct-summation Hermite hot path
 * of Gaburov, Harfst & Portegies Zwart, "SAPPORO: A way to turn your graphics
 * cards into a GRAPE-6" (arXiv:0902.4463).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link,
 * load or call this code: only the tests, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code with the CUDA library.
 *
 * Everything is double precision, written as the plain definition with no
 * blocking or reordering.  Arrays of 3-vectors are row-major n x 3.  Units:
 * G = 1; the potential is the (negative) physical potential.
 */
#ifndef G6_ORACLE_H
#define G6_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Eq. 1 and Eq. 2 (Sect. 2.2): Taylor prediction of position and velocity.
 * dt = t - tj[k] for each particle k; a0 and j0 are the acceleration and jerk
 * themselves (not pre-scaled). */
void orc_predict(long n, const double *x0, const double *v0, const double *a0,
                 const double *j0, const double *tj, double t,
                 double *xp, double *vp);

/* Sect. 2.3 and Sect. 2.5: softened acceleration, jerk and potential on ni
 * i-particles from nj j-particles, plus the nearest neighbour.
 *   r = x_j - x_i, v = v_j - v_i, s2 = |r|^2 + eps2
 *   acc_i  =  sum_j m_j r / s^3
 *   jerk_i =  sum_j m_j [ v / s^3 - 3 (r.v) r / s^5 ]
 *   pot_i  = -sum_j m_j / s
 * The pair with idx_j == idx_i is skipped (self-interaction).  nnb[i] is the
 * j position (0..nj-1) with the smallest unsoftened |r|^2, ties to the smaller
 * position, or -1 when no other j exists; nnr2[i] is that |r|^2.  Any of the
 * output pointers may be NULL. */
void orc_force(long ni, const double *xi, const double *vi, const int *idx_i,
               long nj, const double *xj, const double *vj, const double *mj,
               const int *idx_j, double eps2,
               double *acc, double *jerk, double *pot, int *nnb, double *nnr2);

/* Sect. 4: neighbour lists.  For each i: the j positions (ascending) with
 * idx_j != idx_i and unsoftened |r|^2 < h2[i], at most maxnb of them.
 * nblen[i] receives the untruncated count; nbl is ni x maxnb.  Returns the
 * number of i whose list overflowed (count > maxnb). */
long orc_neighbours(long ni, const double *xi, const int *idx_i, long nj,
                    const double *xj, const int *idx_j, const double *h2,
                    int maxnb, int *nblen, int *nbl);

/* Hermite corrector (Makino & Aarseth 1992, the scheme named in Sect. 2).
 * In place for one particle: xp, vp are the predicted state at t0 + dt,
 * (a0, j0) the force at t0, (a1, j1) at t0 + dt.  Writes the corrected
 * x1, v1 and the second and third acceleration derivatives at t0
 * (a2 = a^(2), a3 = a^(3)). */
void orc_hermite_correct(double dt, const double xp[3], const double vp[3],
                         const double a0[3], const double j0[3],
                         const double a1[3], const double j1[3],
                         double x1[3], double v1[3], double a2[3], double a3[3]);

/* Aarseth (1985) time-step criterion, cited in Sect. 3.1 and 3.2:
 * dt = sqrt(eta (|a||a2| + |j|^2) / (|j||a3| + |a2|^2)). */
double orc_aarseth_dt(const double a[3], const double j[3], const double a2[3],
                      const double a3[3], double eta);

/* Block time step (Sect. 2, Sect. 2.1): the largest power of two <= dt_req,
 * starting from dt_old.  It may halve as often as needed, may double at most
 * once, and only if t is a multiple of 2 dt_old and 2 dt_old <= dt_max.
 * Returns -1 if the result would fall below dt_min. */
double orc_block_dt(double dt_old, double dt_req, double t, double dt_max,
                    double dt_min);

/* Total energy E = sum 1/2 m v^2 - sum_{i<j} m_i m_j / sqrt(|r|^2 + eps2),
 * evaluated as an explicit pair loop (Sect. 3.2, dE/E = (E1 - E0)/E0). */
double orc_energy(long n, const double *m, const double *x, const double *v,
                  double eps2);

typedef struct {
    long nblocks;      /* block steps taken                                 */
    long nactive;      /* sum of active-block sizes (i-force evaluations)   */
    double t;          /* time all particles were advanced to               */
    int err;           /* 0 ok, -1 time step underflow, -2 bad argument     */
} orc_run_stats;

/* Complete 4th-order Hermite block-time-step integration (Sect. 2): every
 * particle starts at t = 0 with the given x, v; a and j at t = 0 come from a
 * full sweep; initial dt = eta_s |a|/|j| quantised to a power of two.  Each
 * block step predicts every particle to t_blk, evaluates the force on the
 * active set, corrects it and picks its next step.  Runs until every particle
 * has reached t_end (t_end must be a multiple of dt_max).  x, v are updated in
 * place; acc, jerk (may be NULL) receive the final a and j.  hist (may be
 * NULL) is a 64-bin histogram of floor(log2(block size)). */
int orc_hermite_run(long n, const double *m, double *x, double *v,
                    double eps2, double eta, double eta_s, double dt_max,
                    double dt_min, double t_end, double *acc, double *jerk,
                    long *hist, orc_run_stats *st);

#ifdef __cplusplus
}
#endif
#endif
