// g6gb_hermite.cpp -- host 4th-order Hermite block-time-step driver on top
// of the g6_* calls (arXiv:0902.4463, Sect. 2 and 2.1: the host predicts the
// i-particles, runs the corrector and picks the time steps; the library
// predicts the j-particles and computes the forces).  Plain C++, FP64.
//
// Scheme: Makino & Aarseth (1992) predictor-corrector, as named in Sect. 2;
// time steps from the Aarseth (1985) criterion cited in Sect. 3.1-3.2,
// quantised to powers of two (block time steps).
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include <atomic>
#include <memory>
#include <mutex>

#include "g6gb.h"
#include "g6gb_pool.h"

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
    // neighbour lists (Sect. 4): requested with radius^2 h2 on every block
    // step when h2 > 0, read back and counted
    double h2 = 0;
    std::vector<double> h2v;
    // relative force error allowed for in the time-step choice (0: none)
    double noise = 0;
    std::vector<int> nbl;
    long long nb_lists = 0, nb_entries = 0, nb_overflowed = 0;
    // host threads for the per-particle work of a block, and the block's
    // j-records for one bulk update (tj, mass, a/2, j/6 per active particle)
    std::vector<double> tjb, mb, a2b, j6b;
    std::vector<int> crc;
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
// j-particles predicted to t_blk; with lists, also every i's neighbour list
// (read back and counted).
int force(g6h_sim &s, int ni, const double *xi, const double *vi, const int *ii,
          double *acc, double *jerk, double *pot, bool lists = false)
{
    const double *h2 = nullptr;
    if (lists && s.h2 > 0) {
        std::fill(s.h2v.begin(), s.h2v.begin() + ni, s.h2);
        h2 = s.h2v.data();
    }
    g6calc_firsthalf(s.cid, s.n, ni, ii, (const double(*)[3])xi, (const double(*)[3])vi,
                     nullptr, nullptr, nullptr, s.eps2, h2);
    int rc = g6calc_lasthalf(s.cid, s.n, ni, ii, (const double(*)[3])xi,
                             (const double(*)[3])vi, s.eps2, h2, (double(*)[3])acc,
                             (double(*)[3])jerk, pot);
    if (rc || !h2)
        return rc;
    rc = g6_read_neighbour_list(s.cid);
    if (rc < 0)
        return rc;
    const int maxnb = g6x_max_neighbours(s.cid);
    if (maxnb < 0)
        return maxnb;
    try {
        if ((int)s.nbl.size() < maxnb)
            s.nbl.resize(maxnb);
    } catch (...) {
        return G6_ENOMEM;
    }
    for (int q = 0; q < ni; ++q) {
        int len = 0;
        const int r = g6_get_neighbour_list(s.cid, q, maxnb, &len, s.nbl.data());
        if (r < 0)
            return r;
        s.nb_entries += std::min(len, maxnb);
        s.nb_overflowed += r == G6_EOVERFLOW;
    }
    s.nb_lists += ni;
    return 0;
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

// Aarseth's request from the end-of-step derivatives.  With noise > 0 (the
// relative error of the force evaluation) the magnitudes of a'' and a''' are
// first reduced by what force errors of that size alone can put into them:
// a''' = (12 (a0 - a1) + 6 h (j0 + j1)) / h^3 and a''(t1) = a'' + h a''' take
// differences of nearly equal forces, so errors of na = noise |a| and
// nj = noise |j| in each force give up to (24 na + 12 h nj) / h^3 in a''' and
// (36 na + 18 h nj) / h^2 in a''(t1).  Without this, force noise read as
// structure shrinks the steps, which makes the noise larger still.  The
// allowance only ever lengthens a step: with a near-zero jerk, a reduced a''
// of 0 would leave sqrt(eta |j| / |a'''|) and collapse the request, so the
// larger of the plain and the reduced request is taken (a 0/0 of the reduced
// one, no measurable derivative at all, also gives the plain one).
double step_request(const double *a1, const double *j1, const double *d2e, const double *d3,
                    double h, double eta, double noise)
{
    const double plain = aarseth(a1, j1, d2e, d3, eta);
    if (!(noise > 0))
        return plain;
    const double am = norm3(a1), jm = norm3(j1);
    const double na = noise * am, nj = noise * jm;
    const double e3 = (24.0 * na + 12.0 * h * nj) / (h * h * h);
    const double e2 = (36.0 * na + 18.0 * h * nj) / (h * h);
    const double m3 = std::max(norm3(d3) - e3, 0.0), m2 = std::max(norm3(d2e) - e2, 0.0);
    const double reduced = std::sqrt(eta * (am * m2 + jm * jm) / (jm * m3 + m2 * m2));
    return plain < reduced ? reduced : plain;
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

// Particles per host work item of a block.
constexpr int CHUNK = 64;

// Per-block work arrays of a driver of n particles.
int alloc_block_work(g6h_sim &s)
{
    try {
        const size_t n = (size_t)s.n;
        s.tjb.resize(n);
        s.mb.resize(n);
        s.a2b.resize(3 * n);
        s.j6b.resize(3 * n);
        s.crc.resize((n + CHUNK - 1) / CHUNK);
    } catch (...) {
        return G6_ENOMEM;
    }
    return 0;
}

}  // namespace

extern "C" {

int g6h_correct_block(int n, double t_blk, const double *t0, const double *dt, double eta,
                      double dt_max, double dt_min, double *xp, double *vp, const double *a0,
                      const double *j0, const double *a1, const double *j1, double *dt_new)
{
    return g6h_correct_block_ex(n, t_blk, t0, dt, eta, dt_max, dt_min, xp, vp, a0, j0, a1, j1,
                                dt_new, 0.0);
}

int g6h_correct_block_ex(int n, double t_blk, const double *t0, const double *dt, double eta,
                         double dt_max, double dt_min, double *xp, double *vp, const double *a0,
                         const double *j0, const double *a1, const double *j1, double *dt_new,
                         double force_noise)
{
    if (!(force_noise >= 0))
        return G6_EINVAL;
    if (n < 0 || (n > 0 && (!t0 || !dt || !xp || !vp || !a0 || !j0 || !a1 || !j1 || !dt_new)))
        return G6_EINVAL;
    auto block = [=](int k0, int k1) -> int {
        int small = 0;
        for (int k = k0; k < k1; ++k) {
            const double h = t_blk - t0[k];
            double d2[3], d3[3], d2e[3];
            correct(h, &a0[3 * k], &j0[3 * k], &a1[3 * k], &j1[3 * k], &xp[3 * k], &vp[3 * k],
                    d2, d3);
            for (int d = 0; d < 3; ++d)
                d2e[d] = d2[d] + h * d3[d];
            const double req = step_request(&a1[3 * k], &j1[3 * k], d2e, d3, h, eta,
                                            force_noise);
            double nd = quantise(dt[k], req, t_blk, dt_max);
            if (!(nd >= dt_min)) {
                nd = -1.0;
                ++small;
            }
            dt_new[k] = nd;
        }
        return small;
    };
    // large blocks on the process-wide host threads
    constexpr int BIG = 8192, PART = 4096;
    if (n < BIG)
        return block(0, n);
    const int nch = (n + PART - 1) / PART;
    std::atomic<int> small{0};
    g6::parallel_run(nch, [&](int i) { small += block(i * PART, std::min(n, (i + 1) * PART)); });
    return small.load();
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
    rc = alloc_block_work(*s);
    if (!rc)
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

long long g6h_run_blocks(g6h_sim *s, double t_end, long long max_blocks)
{
    if (!s || !(t_end >= 0) || std::fmod(t_end, s->dt_max) != 0.0 || max_blocks < 0)
        return G6_EINVAL;
    long long done = 0;
    while (done < max_blocks) {
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
        const int nch = (na + CHUNK - 1) / CHUNK;
        // host prediction of the active i-particles (Eq. 1, Eq. 2)
        g6::parallel_run(nch, [s, tb, na](int c) {
            for (int q = c * CHUNK, qe = std::min(na, q + CHUNK); q < qe; ++q) {
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
        });
        double w1 = now_s();
        int rc = g6_set_ti(s->cid, tb);
        if (!rc)
            rc = force(*s, na, s->xp.data(), s->vp.data(), s->aidx.data(), s->a1.data(),
                       s->j1.data(), s->pot.data(), true);
        if (rc)
            return rc;
        double w2 = now_s();
        // correct, choose the next steps and fill the block's j-records
        g6::parallel_run(nch, [s, tb, na](int c) {
            int small = 0;
            for (int q = c * CHUNK, qe = std::min(na, q + CHUNK); q < qe; ++q) {
                const int k = s->act[q];
                const double h = tb - s->t[k];
                double d2[3], d3[3], d2e[3];
                correct(h, &s->a[3 * k], &s->j[3 * k], &s->a1[3 * q], &s->j1[3 * q],
                        &s->xp[3 * q], &s->vp[3 * q], d2, d3);
                for (int d = 0; d < 3; ++d)
                    d2e[d] = d2[d] + h * d3[d];
                const double req = step_request(&s->a1[3 * q], &s->j1[3 * q], d2e, d3, h,
                                                s->eta, s->noise);
                const double nd = quantise(s->dt[k], req, tb, s->dt_max);
                small += !(nd >= s->dt_min);
                for (int d = 0; d < 3; ++d) {
                    s->x[3 * k + d] = s->xp[3 * q + d];
                    s->v[3 * k + d] = s->vp[3 * q + d];
                    s->a[3 * k + d] = s->a1[3 * q + d];
                    s->j[3 * k + d] = s->j1[3 * q + d];
                    s->a2b[3 * q + d] = 0.5 * s->a1[3 * q + d];
                    s->j6b[3 * q + d] = s->j1[3 * q + d] / 6.0;
                }
                s->t[k] = tb;
                s->dt[k] = nd;
                s->tjb[q] = tb;
                s->mb[q] = s->m[k];
            }
            s->crc[c] = small;
        });
        for (int c = 0; c < nch; ++c)
            if (s->crc[c])
                return G6_EINVAL;
        rc = g6x_set_j_particles(s->cid, na, s->aidx.data(), s->aidx.data(), s->tjb.data(),
                                 s->mb.data(), (const double(*)[3])s->j6b.data(),
                                 (const double(*)[3])s->a2b.data(),
                                 (const double(*)[3])s->vp.data(),
                                 (const double(*)[3])s->xp.data());
        if (rc)
            return rc;
        // most of a block moves to one or two new times: reuse the bucket
        std::vector<int> *last_bucket = nullptr;
        double last_time = 0.0;
        try {
            for (int q = 0; q < na; ++q) {
                const int k = s->act[q];
                const double tn = tb + s->dt[k];
                if (!last_bucket || tn != last_time) {
                    last_bucket = &s->due[tn];
                    last_time = tn;
                }
                last_bucket->push_back(k);
            }
        } catch (...) {
            return G6_ENOMEM;
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
        ++done;
    }
    return done;
}

int g6h_run(g6h_sim *s, double t_end)
{
    const long long r = g6h_run_blocks(s, t_end, LLONG_MAX);
    return r < 0 ? (int)r : 0;
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

int g6h_set_neighbour_radius(g6h_sim *s, double h2)
{
    if (!s || !(h2 >= 0) || !std::isfinite(h2))
        return G6_EINVAL;
    if (h2 > 0) {
        try {
            s->h2v.resize(s->n);
        } catch (...) {
            return G6_ENOMEM;
        }
    }
    s->h2 = h2;
    return 0;
}

int g6h_set_force_noise(g6h_sim *s, double rel)
{
    if (!s || !(rel >= 0) || !(rel < 1))
        return G6_EINVAL;
    s->noise = rel;
    return 0;
}

int g6h_neighbour_stats(const g6h_sim *s, long long *lists, long long *entries,
                        long long *overflowed)
{
    if (!s)
        return G6_EINVAL;
    if (lists)
        *lists = s->nb_lists;
    if (entries)
        *entries = s->nb_entries;
    if (overflowed)
        *overflowed = s->nb_overflowed;
    return 0;
}

void g6h_destroy(g6h_sim *s) { delete s; }

}  // extern "C"

// ------------------------------------------------------ checkpoint/resume
//
// File layout (host byte order, little-endian on every supported host):
//   char    magic[8] = "G6HCKPT1"
//   int64   n, nbuckets, nblocks, nactive, hist[64]
//   double  eps2, eta, eta_s, dt_max, dt_min, t_now
//   double  m[n], x[n][3], v[n][3], a[n][3], j[n][3], t[n], dt[n]
//   per scheduler bucket, in time order: double time, int64 count,
//           int32 particle[count] (in the bucket's order, which fixes the
//           order of the block's i-particles and so the force sums' grouping)
//   uint64  FNV-1a hash of every byte above

namespace {

const char kMagic[8] = {'G', '6', 'H', 'C', 'K', 'P', 'T', '1'};

struct Hasher {
    uint64_t h = 1469598103934665603ull;
    void add(const void *p, size_t n)
    {
        const unsigned char *c = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < n; ++i) {
            h ^= c[i];
            h *= 1099511628211ull;
        }
    }
};

struct Writer {
    FILE *f;
    Hasher hs;
    bool ok = true;
    void put(const void *p, size_t n)
    {
        if (ok && n && std::fwrite(p, 1, n, f) != n)
            ok = false;
        hs.add(p, n);
    }
};

struct Reader {
    const std::vector<unsigned char> &buf;
    size_t pos = 0;
    Hasher hs;
    bool get(void *p, size_t n)
    {
        if (n > buf.size() - pos)
            return false;
        std::memcpy(p, buf.data() + pos, n);
        hs.add(buf.data() + pos, n);
        pos += n;
        return true;
    }
};

}  // namespace

extern "C" {

int g6h_checkpoint(const g6h_sim *s, const char *path)
{
    if (!s || !path)
        return G6_EINVAL;
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "wb");
    if (!f)
        return G6_EIO;
    Writer w{f};
    const size_t n = (size_t)s->n;
    const int64_t hdr[4] = {s->n, (int64_t)s->due.size(), s->nblocks, s->nactive};
    const double par[6] = {s->eps2, s->eta, s->eta_s, s->dt_max, s->dt_min, s->t_now};
    w.put(kMagic, sizeof kMagic);
    w.put(hdr, sizeof hdr);
    w.put(s->hist, sizeof s->hist);
    w.put(par, sizeof par);
    w.put(s->m.data(), n * sizeof(double));
    w.put(s->x.data(), 3 * n * sizeof(double));
    w.put(s->v.data(), 3 * n * sizeof(double));
    w.put(s->a.data(), 3 * n * sizeof(double));
    w.put(s->j.data(), 3 * n * sizeof(double));
    w.put(s->t.data(), n * sizeof(double));
    w.put(s->dt.data(), n * sizeof(double));
    for (const auto &b : s->due) {
        const double tb = b.first;
        const int64_t cnt = (int64_t)b.second.size();
        w.put(&tb, sizeof tb);
        w.put(&cnt, sizeof cnt);
        w.put(b.second.data(), b.second.size() * sizeof(int));
    }
    const uint64_t hash = w.hs.h;
    const bool ok = w.ok && std::fwrite(&hash, sizeof hash, 1, f) == 1;
    if (std::fclose(f) != 0 || !ok || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return G6_EIO;
    }
    return 0;
}

g6h_sim *g6h_restore(int cid, const char *path, int *err)
{
    auto fail = [&](int code) -> g6h_sim * {
        if (err)
            *err = code;
        return nullptr;
    };
    if (err)
        *err = 0;
    if (!path)
        return fail(G6_EINVAL);
    std::vector<unsigned char> buf;
    {
        FILE *f = std::fopen(path, "rb");
        if (!f)
            return fail(G6_EIO);
        unsigned char chunk[1 << 16];
        size_t got;
        bool bad = false;
        try {
            while ((got = std::fread(chunk, 1, sizeof chunk, f)) > 0)
                buf.insert(buf.end(), chunk, chunk + got);
        } catch (...) {
            bad = true;
        }
        const bool rerr = std::ferror(f) != 0;
        std::fclose(f);
        if (bad)
            return fail(G6_ENOMEM);
        if (rerr)
            return fail(G6_EIO);
    }
    // everything below checks the content before any state is built
    Reader r{buf};
    char magic[8];
    int64_t hdr[4];
    double par[6];
    g6h_sim *s = new (std::nothrow) g6h_sim();
    if (!s)
        return fail(G6_ENOMEM);
    auto bad = [&](int code) -> g6h_sim * {
        delete s;
        return fail(code);
    };
    if (!r.get(magic, 8) || std::memcmp(magic, kMagic, 8) != 0 || !r.get(hdr, sizeof hdr)
        || !r.get(s->hist, sizeof s->hist) || !r.get(par, sizeof par))
        return bad(G6_EINVAL);
    const int64_t n = hdr[0], nb = hdr[1];
    if (n < 1 || n > (1 << 28) || nb < 0 || nb > n || hdr[2] < 0 || hdr[3] < 0)
        return bad(G6_EINVAL);
    // the arrays and the scheduler's entries must fit in the file
    if ((size_t)n * (15 * sizeof(double) + sizeof(int)) > buf.size())
        return bad(G6_EINVAL);
    s->cid = cid;
    s->n = (int)n;
    s->nblocks = hdr[2];
    s->nactive = hdr[3];
    s->eps2 = par[0];
    s->eta = par[1];
    s->eta_s = par[2];
    s->dt_max = par[3];
    s->dt_min = par[4];
    s->t_now = par[5];
    if (!(s->eps2 >= 0) || !(s->eta > 0) || !(s->eta_s > 0) || !(s->dt_max > 0)
        || !(s->dt_min > 0) || !std::isfinite(s->t_now))
        return bad(G6_EINVAL);
    const size_t un = (size_t)n;
    try {
        s->m.resize(un);
        s->x.resize(3 * un);
        s->v.resize(3 * un);
        s->a.resize(3 * un);
        s->j.resize(3 * un);
        s->t.resize(un);
        s->dt.resize(un);
        s->idx.resize(un);
        s->act.reserve(un);
        s->aidx.resize(un);
        s->xp.resize(3 * un);
        s->vp.resize(3 * un);
        s->a1.resize(3 * un);
        s->j1.resize(3 * un);
        s->pot.resize(un);
    } catch (...) {
        return bad(G6_ENOMEM);
    }
    if (!r.get(s->m.data(), un * sizeof(double)) || !r.get(s->x.data(), 3 * un * sizeof(double))
        || !r.get(s->v.data(), 3 * un * sizeof(double))
        || !r.get(s->a.data(), 3 * un * sizeof(double))
        || !r.get(s->j.data(), 3 * un * sizeof(double))
        || !r.get(s->t.data(), un * sizeof(double)) || !r.get(s->dt.data(), un * sizeof(double)))
        return bad(G6_EINVAL);
    std::vector<char> seen(un, 0);
    int64_t filed = 0;
    try {
        for (int64_t b = 0; b < nb; ++b) {
            double tb;
            int64_t cnt;
            if (!r.get(&tb, sizeof tb) || !r.get(&cnt, sizeof cnt) || cnt < 1 || cnt > n - filed)
                return bad(G6_EINVAL);
            std::vector<int> &v = s->due[tb];
            if (!v.empty())
                return bad(G6_EINVAL);                 // times must be distinct
            v.resize((size_t)cnt);
            if (!r.get(v.data(), (size_t)cnt * sizeof(int)))
                return bad(G6_EINVAL);
            for (int k : v) {
                if (k < 0 || k >= n || seen[k] || !(s->dt[k] > 0) || s->t[k] + s->dt[k] != tb)
                    return bad(G6_EINVAL);
                seen[k] = 1;
            }
            filed += cnt;
        }
    } catch (...) {
        return bad(G6_ENOMEM);
    }
    uint64_t want = r.hs.h, hash = 0;
    if (filed != n || !r.get(&hash, sizeof hash) || hash != want || r.pos != buf.size())
        return bad(G6_EINVAL);
    for (int64_t k = 0; k < n; ++k)
        s->idx[k] = (int)k;
    // j-memory: every particle's last corrected state, as the original run
    // left it
    int rc = alloc_block_work(*s);
    if (!rc)
        rc = g6x_set_ni_max(cid, s->n);
    for (int k = 0; !rc && k < s->n; ++k)
        rc = send_j(*s, k);
    if (rc)
        return bad(rc);
    return s;
}

}  // extern "C"
