// g6gb_hermite.cpp -- host 4th-order Hermite block-time-step driver on top
// of the g6_* calls (arXiv:0902.4463, Sect. 2 and 2.1: the host predicts the
// i-particles, runs the corrector and picks the time steps; the library
// predicts the j-particles and computes the forces).  Plain C++, FP64.
//
// Scheme: Makino & Aarseth (1992) predictor-corrector, as named in Sect. 2;
// time steps from the Aarseth (1985) criterion cited in Sect. 3.1-3.2,
// quantised to powers of two (block time steps).
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "g6gb.h"

struct g6h_sim {
    int cid = 0, n = 0;
    double eps2 = 0, eta = 0, eta_s = 0, dt_max = 0, dt_min = 0;
    std::vector<double> m, x, v, a, j, t, dt;   // x, v, a, j are n x 3
    std::vector<int> idx;
    long long nblocks = 0, nactive = 0;
    long long hist[64] = {};
    // work arrays for one block
    std::vector<int> act, aidx;
    std::vector<double> xp, vp, a1, j1, pot;
    double t_now = 0;
    // wall-clock seconds spent in the scheduler, the force calls and the
    // host correction (including sending corrected particles)
    double sec_sched = 0, sec_force = 0, sec_correct = 0;
    // block scheduler: particles keyed by their next time t + dt (block
    // times are dyadic, so equal times compare exactly)
    std::map<double, std::vector<int>> due;
};

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

double norm3(const double *p) { return std::sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]); }

// Send particle k's current state to j-memory slot k.
int send_j(g6h_sim &s, int k)
{
    double a2[3], j6[3], k18[3] = {0, 0, 0};
    for (int d = 0; d < 3; ++d) {
        a2[d] = 0.5 * s.a[3 * k + d];
        j6[d] = s.j[3 * k + d] / 6.0;
    }
    return g6_set_j_particle(s.cid, k, k, s.t[k], s.dt[k], s.m[k], k18, j6, a2,
                             &s.v[3 * k], &s.x[3 * k]);
}

// Force on ni i-particles (positions xi, velocities vi, ids ii) from all n
// j-particles predicted to t_blk.
int force(g6h_sim &s, int ni, const double *xi, const double *vi, const int *ii,
          double *acc, double *jerk, double *pot)
{
    g6calc_firsthalf(s.cid, s.n, ni, ii, (const double(*)[3])xi, (const double(*)[3])vi,
                     nullptr, nullptr, nullptr, s.eps2, nullptr);
    return g6calc_lasthalf(s.cid, s.n, ni, ii, (const double(*)[3])xi,
                           (const double(*)[3])vi, s.eps2, nullptr, (double(*)[3])acc,
                           (double(*)[3])jerk, pot);
}

// Makino & Aarseth (1992) corrector for one particle: from the force (a0, j0)
// at the start and (a1, j1) at the end of a step h, the Hermite interpolant
// gives a'' and a''' at the start; they add the h^4 and h^5 terms.
void correct(double h, const double *a0, const double *j0, const double *a1,
             const double *j1, double *xp, double *vp, double *d2, double *d3)
{
    const double ih = 1.0 / h, ih2 = ih * ih, ih3 = ih2 * ih;
    const double h2 = h * h, h3 = h2 * h, h4 = h2 * h2;
    for (int d = 0; d < 3; ++d) {
        const double da = a0[d] - a1[d];
        d2[d] = (-6.0 * da - h * (4.0 * j0[d] + 2.0 * j1[d])) * ih2;
        d3[d] = (12.0 * da + 6.0 * h * (j0[d] + j1[d])) * ih3;
        xp[d] += h4 * (d2[d] * (1.0 / 24.0) + h * d3[d] * (1.0 / 120.0));
        vp[d] += h3 * (d2[d] * (1.0 / 6.0) + h * d3[d] * (1.0 / 24.0));
    }
}

double dot3(const double *p, const double *q) { return p[0] * q[0] + p[1] * q[1] + p[2] * q[2]; }

// Aarseth (1985): sqrt(eta (|a||a''| + |j|^2) / (|j||a'''| + |a''|^2)),
// with |a||a''| = sqrt(|a|^2 |a''|^2) to save square roots.
double aarseth(const double *a, const double *j, const double *d2, const double *d3,
               double eta)
{
    const double a_2 = dot3(a, a), j_2 = dot3(j, j), d2_2 = dot3(d2, d2), d3_2 = dot3(d3, d3);
    return std::sqrt(eta * (std::sqrt(a_2 * d2_2) + j_2) / (std::sqrt(j_2 * d3_2) + d2_2));
}

// Is t an integer multiple of the power of two p?  t * (1/p) is exact.
bool multiple_of(double t, double p)
{
    const double q = t * (1.0 / p);
    return q == std::floor(q);
}

// Power-of-two step: halve until it fits the request; double at most once
// and only when the current time is a multiple of the doubled step.
double quantise(double dt, double req, double t, double dt_max)
{
    if (req < dt) {
        while (dt > req)
            dt *= 0.5;
    } else if (req >= 2.0 * dt && 2.0 * dt <= dt_max && multiple_of(t, 2.0 * dt)) {
        dt *= 2.0;
    }
    return dt;
}

}  // namespace

extern "C" {

int g6h_correct_block(int n, double t_blk, const double *t0, const double *dt, double eta,
                      double dt_max, double dt_min, double *xp, double *vp, const double *a0,
                      const double *j0, const double *a1, const double *j1, double *dt_new)
{
    if (n < 0 || (n > 0 && (!t0 || !dt || !xp || !vp || !a0 || !j0 || !a1 || !j1 || !dt_new)))
        return G6_EINVAL;
    int small = 0;
    for (int k = 0; k < n; ++k) {
        const double h = t_blk - t0[k];
        double d2[3], d3[3], d2e[3];
        correct(h, &a0[3 * k], &j0[3 * k], &a1[3 * k], &j1[3 * k], &xp[3 * k], &vp[3 * k], d2,
                d3);
        for (int d = 0; d < 3; ++d)
            d2e[d] = d2[d] + h * d3[d];
        const double req = aarseth(&a1[3 * k], &j1[3 * k], d2e, d3, eta);
        double nd = quantise(dt[k], req, t_blk, dt_max);
        if (!(nd >= dt_min)) {
            nd = -1.0;
            ++small;
        }
        dt_new[k] = nd;
    }
    return small;
}

g6h_sim *g6h_create(int cid, int n, const double *m, const double *x, const double *v,
                    double eps2, double eta, double eta_s, double dt_max, double dt_min,
                    int *err)
{
    int rc = 0;
    if (err)
        *err = 0;
    if (n < 1 || !m || !x || !v || !(eta > 0) || !(dt_max > 0) || !(dt_min > 0)
        || !(eps2 >= 0)) {
        if (err)
            *err = G6_EINVAL;
        return nullptr;
    }
    g6h_sim *s = new (std::nothrow) g6h_sim();
    if (!s) {
        if (err)
            *err = G6_ENOMEM;
        return nullptr;
    }
    s->cid = cid;
    s->n = n;
    s->eps2 = eps2;
    s->eta = eta;
    s->eta_s = eta_s > 0 ? eta_s : eta / 10.0;
    s->dt_max = dt_max;
    s->dt_min = dt_min;
    try {
        s->m.assign(m, m + n);
        s->x.assign(x, x + 3 * (size_t)n);
        s->v.assign(v, v + 3 * (size_t)n);
        s->a.assign(3 * (size_t)n, 0.0);
        s->j.assign(3 * (size_t)n, 0.0);
        s->t.assign(n, 0.0);
        s->dt.assign(n, dt_max);
        s->idx.resize(n);
        s->act.reserve(n);
        s->aidx.resize(n);
        s->xp.resize(3 * (size_t)n);
        s->vp.resize(3 * (size_t)n);
        s->a1.resize(3 * (size_t)n);
        s->j1.resize(3 * (size_t)n);
        s->pot.resize(n);
    } catch (...) {
        delete s;
        if (err)
            *err = G6_ENOMEM;
        return nullptr;
    }
    for (int k = 0; k < n; ++k)
        s->idx[k] = k;
    rc = g6x_set_ni_max(cid, n);
    for (int k = 0; !rc && k < n; ++k)
        rc = send_j(*s, k);
    if (!rc)
        rc = g6_set_ti(cid, 0.0);
    if (!rc)
        rc = force(*s, n, s->x.data(), s->v.data(), s->idx.data(), s->a.data(), s->j.data(),
                   s->pot.data());
    for (int k = 0; !rc && k < n; ++k) {
        double req = s->eta_s * norm3(&s->a[3 * k]) / norm3(&s->j[3 * k]);
        double d = dt_max;
        while (d > req)
            d *= 0.5;
        if (d < dt_min)
            rc = G6_EINVAL;
        s->dt[k] = d;
    }
    for (int k = 0; !rc && k < n; ++k)
        rc = send_j(*s, k);
    if (!rc) {
        try {
            for (int k = 0; k < n; ++k)
                s->due[s->t[k] + s->dt[k]].push_back(k);
        } catch (...) {
            rc = G6_ENOMEM;
        }
    }
    if (rc) {
        delete s;
        if (err)
            *err = rc;
        return nullptr;
    }
    return s;
}

int g6h_run(g6h_sim *s, double t_end)
{
    if (!s || !(t_end >= 0) || std::fmod(t_end, s->dt_max) != 0.0)
        return G6_EINVAL;
    for (;;) {
        double w0 = now_s();
        // block scheduler: the earliest next time and the particles due then
        if (s->due.empty())
            break;
        auto first = s->due.begin();
        const double tb = first->first;
        if (tb > t_end)
            break;
        s->act.swap(first->second);
        s->due.erase(first);
        const int na = (int)s->act.size();
        std::vector<int> *last_bucket = nullptr;
        double last_time = 0.0;
        // host prediction of the active i-particles (Eq. 1, Eq. 2)
        for (int q = 0; q < na; ++q) {
            const int k = s->act[q];
            const double h = tb - s->t[k];
            for (int d = 0; d < 3; ++d) {
                const double xa = s->a[3 * k + d], xj = s->j[3 * k + d];
                s->xp[3 * q + d] = s->x[3 * k + d]
                                   + h * (s->v[3 * k + d] + h * (xa / 2.0 + h * xj / 6.0));
                s->vp[3 * q + d] = s->v[3 * k + d] + h * (xa + h * xj / 2.0);
            }
            s->aidx[q] = k;
        }
        double w1 = now_s();
        int rc = g6_set_ti(s->cid, tb);
        if (!rc)
            rc = force(*s, na, s->xp.data(), s->vp.data(), s->aidx.data(), s->a1.data(),
                       s->j1.data(), s->pot.data());
        if (rc)
            return rc;
        double w2 = now_s();
        for (int q = 0; q < na; ++q) {
            const int k = s->act[q];
            const double h = tb - s->t[k];
            double d2[3], d3[3], d2e[3];
            correct(h, &s->a[3 * k], &s->j[3 * k], &s->a1[3 * q], &s->j1[3 * q],
                    &s->xp[3 * q], &s->vp[3 * q], d2, d3);
            for (int d = 0; d < 3; ++d)
                d2e[d] = d2[d] + h * d3[d];
            const double req = aarseth(&s->a1[3 * q], &s->j1[3 * q], d2e, d3, s->eta);
            const double nd = quantise(s->dt[k], req, tb, s->dt_max);
            if (!(nd >= s->dt_min))
                return G6_EINVAL;
            std::memcpy(&s->x[3 * k], &s->xp[3 * q], 3 * sizeof(double));
            std::memcpy(&s->v[3 * k], &s->vp[3 * q], 3 * sizeof(double));
            std::memcpy(&s->a[3 * k], &s->a1[3 * q], 3 * sizeof(double));
            std::memcpy(&s->j[3 * k], &s->j1[3 * q], 3 * sizeof(double));
            s->t[k] = tb;
            s->dt[k] = nd;
            rc = send_j(*s, k);
            if (rc)
                return rc;
            // most of a block moves to one or two new times: reuse the bucket
            const double tn = tb + nd;
            if (!last_bucket || tn != last_time) {
                last_bucket = &s->due[tn];
                last_time = tn;
            }
            last_bucket->push_back(k);
        }
        s->act.clear();
        double w3 = now_s();
        s->sec_sched += w1 - w0;
        s->sec_force += w2 - w1;
        s->sec_correct += w3 - w2;
        s->nblocks += 1;
        s->nactive += na;
        int b = 0;
        while (b < 63 && (2LL << b) <= na)
            ++b;
        s->hist[b] += 1;
        s->t_now = tb;
    }
    return 0;
}

int g6h_get_state(const g6h_sim *s, double *x, double *v, double *acc, double *jerk,
                  double *t, double *dt)
{
    if (!s)
        return G6_EINVAL;
    const size_t n3 = 3 * (size_t)s->n * sizeof(double), n1 = (size_t)s->n * sizeof(double);
    if (x)
        std::memcpy(x, s->x.data(), n3);
    if (v)
        std::memcpy(v, s->v.data(), n3);
    if (acc)
        std::memcpy(acc, s->a.data(), n3);
    if (jerk)
        std::memcpy(jerk, s->j.data(), n3);
    if (t)
        std::memcpy(t, s->t.data(), n1);
    if (dt)
        std::memcpy(dt, s->dt.data(), n1);
    return 0;
}

int g6h_energy(g6h_sim *s, double *e_kin, double *e_pot)
{
    if (!s)
        return G6_EINVAL;
    const int n = s->n;
    for (int k = 1; k < n; ++k)
        if (s->t[k] != s->t[0])
            return G6_EINVAL;            // not synchronised
    std::vector<double> acc(3 * (size_t)n), jerk(3 * (size_t)n), pot(n);
    int rc = g6_set_ti(s->cid, s->t[0]);
    if (!rc)
        rc = force(*s, n, s->x.data(), s->v.data(), s->idx.data(), acc.data(), jerk.data(),
                   pot.data());
    if (rc)
        return rc;
    double ek = 0, ep = 0;
    for (int k = 0; k < n; ++k) {
        const double *w = &s->v[3 * k];
        ek += 0.5 * s->m[k] * (w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
        ep += 0.5 * s->m[k] * pot[k];
    }
    if (e_kin)
        *e_kin = ek;
    if (e_pot)
        *e_pot = ep;
    return 0;
}

int g6h_stats(const g6h_sim *s, long long *nblocks, long long *nactive, long long *hist)
{
    if (!s)
        return G6_EINVAL;
    if (nblocks)
        *nblocks = s->nblocks;
    if (nactive)
        *nactive = s->nactive;
    if (hist)
        std::memcpy(hist, s->hist, sizeof(s->hist));
    return 0;
}

int g6h_profile(const g6h_sim *s, double *sec_sched, double *sec_force, double *sec_correct)
{
    if (!s)
        return G6_EINVAL;
    if (sec_sched)
        *sec_sched = s->sec_sched;
    if (sec_force)
        *sec_force = s->sec_force;
    if (sec_correct)
        *sec_correct = s->sec_correct;
    return 0;
}

void g6h_destroy(g6h_sim *s) { delete s; }

}  // extern "C"
