// g6gb_api.cu -- C ABI of the GRAPE-6-style force library (arXiv:0902.4463,
// Sect. 2.5: the library keeps the GRAPE-6 calling sequence so that N-body
// codes only relink).  Host side of the hot path: contexts, j-memory staging,
// the prediction bookkeeping of Sect. 2.1-2.2 (j-particles are predicted once
// per block time), launches and the copy back.  All arithmetic of the method
// runs in the kernels of g6gb_kernels.cu; this file only moves data.
#include "g6gb_internal.h"
#include "g6gb_pool.h"

#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <fstream>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <utility>
#include <array>
#include <vector>

namespace {

using g6::ForceConfig;
using g6::JT;
using g6::Partial;

g6x_alloc_fn g_alloc = nullptr;
g6x_free_fn g_free = nullptr;
void *g_alloc_user = nullptr;

void *dev_alloc(size_t bytes)
{
    if (bytes == 0)
        bytes = 16;
    if (g_alloc)
        return g_alloc(bytes, g_alloc_user);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(void *p)
{
    if (!p)
        return;
    if (g_free)
        g_free(p, g_alloc_user);
    else
        cudaFree(p);
}

void *host_alloc(size_t bytes)
{
    void *p = nullptr;
    if (cudaHostAlloc(&p, bytes ? bytes : 16, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

// Pinned host memory that kernels read and write directly (zero-copy): the
// GRAPE path's staging, i-records, results and error word live here, so a
// calculation needs no separate host<->device copies.  *dev receives the
// device-side address.
void *host_alloc_mapped(size_t bytes, void **dev)
{
    void *p = nullptr;
    if (cudaHostAlloc(&p, bytes ? bytes : 16, cudaHostAllocMapped) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (cudaHostGetDevicePointer(dev, p, 0) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeHost(p);
        return nullptr;
    }
    return p;
}

void host_free(void *p)
{
    if (p)
        cudaFreeHost(p);
}

int env_int(const char *name, int dflt)
{
    const char *s = std::getenv(name);
    if (!s || !*s)
        return dflt;
    long v = std::strtol(s, nullptr, 10);
    return v > 0 ? (int)v : dflt;
}

int round_up(int n, int k) { return (n + k - 1) / k * k; }

struct Ctx {
    bool open = false;
    int dev = 0, sm_count = 0;
    cudaStream_t own = nullptr;
    cudaStream_t stream = nullptr;
    int cap = 0, ni_max = 0, prec = G6X_PREC_DS;   // force arithmetic
    int pmode = G6X_PREC_DS;                           // G6X_PREC_* as selected
    g6::JStore js{};
    g6::Pred pred{};
    // j-memory updates staged on the host, uploaded by the next calculation
    g6x_jrec *h_jst = nullptr, *d_jst = nullptr;
    int n_jst = 0, jst_cap = 0;
    std::vector<int> slot_of;
    cudaEvent_t ev_jst = nullptr;
    bool jst_inflight = false;
    // the staged records sorted by tile for the fused update + predict launch
    g6x_jrec *h_jsort = nullptr, *d_jsort = nullptr;
    int jsort_cap = 0;
    int *h_toff = nullptr, *d_toff = nullptr;
    int toff_cap = 0;
    std::vector<int> tcur;
    cudaEvent_t ev_jsort = nullptr;
    bool jsort_inflight = false;
    // i-data and results of the GRAPE path
    g6x_irec *h_irec = nullptr, *d_irec = nullptr;
    g6x_out *h_out = nullptr, *d_out = nullptr;
    int io_cap = 0;
    // partial results and the per-i-tile counters of the fused reduction
    Partial *d_part = nullptr;
    size_t part_cap = 0;
    unsigned *d_tcnt = nullptr;
    size_t tcnt_cap = 0;
    bool tcnt_dirty = false;          // a launch may have stopped mid-count
    int *d_nbl_part = nullptr, *d_nbc_part = nullptr;
    size_t nbp_cap = 0;               // list counts of d_nbc_part
    size_t nbl_ints = 0;              // ints of d_nbl_part
    int nbp_seg = 0;                  // entries per list partial of d_nbl_part
    int *d_nbl = nullptr, *d_nblen = nullptr, *h_nbl = nullptr, *h_nblen = nullptr;
    size_t nbo_cap = 0;
    int nbo_maxnb = 0;                // list length of d_nbl / h_nbl
    // neighbour lists (Sect. 4): entries kept per i-particle, room per list
    // partial (grown when a launch needed more), and the largest count a
    // launch saw (mapped)
    int maxnb = G6_MAXNB;
    int nbseg = 16;
    int *h_nbmax = nullptr, *d_nbmax = nullptr;
    long long list_reruns = 0;
    int *d_err = nullptr, *h_err = nullptr;
    // prediction bookkeeping per precision mode
    double t_set = 0.0;
    double t_pred[3] = {NAN, NAN, NAN};
    int nj_pred[3] = {-1, -1, -1};
    long long ver = 0, ver_pred[3] = {-1, -1, -1};
    // calculation in flight
    bool pending = false;
    int latched = 0;
    int calc_ni = 0, calc_nj = 0;
    bool lists_ready = false, lists_host = false;
    int list_ni = 0;
    // what the last list launch computed, to compute its lists again with
    // more room per partial: its launch, inputs, block time and j-memory version
    ForceConfig list_cfg{};
    int list_nj = 0;
    const g6x_irec *list_irec = nullptr;
    g6x_out *list_out = nullptr;
    double list_eps2 = 0.0, list_t = 0.0;
    long long list_ver = -1;
    cudaEvent_t ev_done = nullptr;
    ForceConfig last_cfg{};
    long long launches = 0;
    int force_variant = -1, force_grid = 0;
    // optional per-phase event timing
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending[4];
    double t_ms[4] = {0, 0, 0, 0};
    long long t_cnt[4] = {0, 0, 0, 0};
    // per-call marks that detect an address given twice to one bulk call,
    // staging indices, and per-chunk tile counts of the parallel sort
    std::vector<unsigned> stamp;
    unsigned stamp_now = 0;
    std::vector<int> sidx;
    std::vector<int> cnt;                 // per worker chunk x tile counts
};

Ctx g_ctx[G6_MAX_CLUSTERS];

// Host loops over at least this many particles run on the host threads, in
// chunks of PAR_CHUNK (a fork and join of the pool costs a few microseconds,
// a chunk's copies about as much); the staging sort, whose parallel form
// keeps and sums per-chunk tile counts, only from PAR_MIN_SORT records and
// twice as many records as tiles on.
constexpr int PAR_MIN = 1024;
constexpr int PAR_CHUNK = 512;
constexpr int PAR_MIN_SORT = 2048;

// f(k0, k1) over [0, n): serially for small n, else in chunks on the host threads.
template <class F>
void par_for(Ctx &, int n, const F &f)
{
    if (n < PAR_MIN) {
        f(0, n);
        return;
    }
    const int nch = (n + PAR_CHUNK - 1) / PAR_CHUNK;
    g6::parallel_run(nch, [&](int i) { f(i * PAR_CHUNK, std::min(n, (i + 1) * PAR_CHUNK)); });
}

}  // namespace

namespace g6 {
void *dev_alloc_hooked(size_t bytes) { return dev_alloc(bytes); }
void dev_free_hooked(void *p) { dev_free(p); }
void *host_alloc_zero_copy(size_t bytes, void **dev) { return host_alloc_mapped(bytes, dev); }
void host_free_pinned(void *p) { host_free(p); }
}  // namespace g6

namespace {

enum Phase { PH_SCATTER = 0, PH_PREDICT = 1, PH_FORCE = 2, PH_REDUCE = 3 };

cudaEvent_t pool_event(Ctx &c)
{
    if (!c.ev_pool.empty()) {
        cudaEvent_t e = c.ev_pool.back();
        c.ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Bracket one launch with events when timing is on.
// One phase of a calculation: an NVTX range on the host (visible to
// profilers that collect NVTX; near free otherwise) and, with timing on, a
// pair of CUDA events on the context's stream.
const char *const kPhaseName[4] = {"g6gb j-update", "g6gb predict", "g6gb force",
                                   "g6gb reduce"};

struct PhaseTimer {
    Ctx &c;
    int ph;
    cudaEvent_t e0 = nullptr;
    PhaseTimer(Ctx &cc, int p) : c(cc), ph(p)
    {
        nvtxRangePushA(kPhaseName[p]);
        if (c.timing && (e0 = pool_event(c)) != nullptr)
            cudaEventRecord(e0, c.stream);
    }
    ~PhaseTimer()
    {
        nvtxRangePop();
        if (!e0)
            return;
        cudaEvent_t e1 = pool_event(c);
        if (!e1) {
            c.ev_pool.push_back(e0);
            return;
        }
        cudaEventRecord(e1, c.stream);
        c.ev_pending[ph].push_back({e0, e1});
    }
};

void resolve_timing(Ctx &c)
{
    for (int p = 0; p < 4; ++p) {
        for (auto &pr : c.ev_pending[p]) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) {
                c.t_ms[p] += ms;
                c.t_cnt[p] += 1;
            } else {
                cudaGetLastError();
            }
            c.ev_pool.push_back(pr.first);
            c.ev_pool.push_back(pr.second);
        }
        c.ev_pending[p].clear();
    }
}

Ctx *get(int cid, int *err)
{
    if (cid < 0 || cid >= G6_MAX_CLUSTERS) {
        *err = G6_EINVAL;
        return nullptr;
    }
    if (!g_ctx[cid].open) {
        *err = G6_ENOTOPEN;
        return nullptr;
    }
    *err = 0;
    return &g_ctx[cid];
}

int cuda_err(cudaError_t e)
{
    if (e == cudaSuccess)
        return 0;
    cudaGetLastError();
    if (e == cudaErrorMemoryAllocation)
        return G6_ENOMEM;
    if (e == cudaErrorNoKernelImageForDevice || e == cudaErrorNoDevice
        || e == cudaErrorInsufficientDriver)
        return G6_ENODEV;
    return G6_EIO;
}

void free_ctx(Ctx &c)
{
    if (c.stream)
        cudaStreamSynchronize(c.stream);
    g6::JStore &js = c.js;
    // d_jst, d_irec, d_out, d_nbl, d_nblen and d_err are device aliases of
    // mapped host buffers, freed with them below
    void *dptrs[] = {js.x0, js.raw, js.v64, js.a264, js.j664, js.idx, c.pred.pt, c.pred.trange, c.pred.p64, c.pred.v64,
                     c.d_part, c.d_tcnt, c.d_nbl_part, c.d_nbc_part};
    for (void *p : dptrs)
        dev_free(p);
    void *hptrs[] = {c.h_jst, c.h_jsort, c.h_toff, c.h_irec, c.h_out, c.h_nbl, c.h_nblen,
                     c.h_err, c.h_nbmax};
    for (void *p : hptrs)
        host_free(p);
    for (int p = 0; p < 4; ++p)
        for (auto &pr : c.ev_pending[p]) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
    for (cudaEvent_t e : c.ev_pool)
        cudaEventDestroy(e);
    if (c.ev_jst)
        cudaEventDestroy(c.ev_jst);
    if (c.ev_jsort)
        cudaEventDestroy(c.ev_jsort);
    if (c.ev_done)
        cudaEventDestroy(c.ev_done);
    if (c.own)
        cudaStreamDestroy(c.own);
    c = Ctx();
}

// Grow a device buffer to at least `need` elements (contents not kept).
template <class T>
int grow_dev(T *&p, size_t &cap, size_t need)
{
    if (need <= cap && p)
        return 0;
    size_t n = need + need / 4 + 64;
    T *q = (T *)dev_alloc(n * sizeof(T));
    if (!q)
        return G6_ENOMEM;
    dev_free(p);
    p = q;
    cap = n;
    return 0;
}

int ensure_io(Ctx &c, int n)
{
    if (n <= c.io_cap && c.h_irec)
        return 0;
    int cap = n < 16 ? 16 : n;
    void *di = nullptr, *dout = nullptr;
    g6x_irec *hi = (g6x_irec *)host_alloc_mapped(sizeof(g6x_irec) * cap, &di);
    g6x_out *ho = (g6x_out *)host_alloc_mapped(sizeof(g6x_out) * cap, &dout);
    if (!hi || !ho) {
        host_free(hi);
        host_free(ho);
        return G6_ENOMEM;
    }
    host_free(c.h_irec);
    host_free(c.h_out);
    c.h_irec = hi;
    c.h_out = ho;
    c.d_irec = (g6x_irec *)di;
    c.d_out = (g6x_out *)dout;
    c.io_cap = cap;
    return 0;
}

int ensure_jstage(Ctx &c, int need)
{
    if (need <= c.jst_cap)
        return 0;
    int cap = c.jst_cap ? c.jst_cap : 1024;
    while (cap < need)
        cap *= 2;
    if (cap > c.cap)
        cap = c.cap;
    void *d = nullptr;
    g6x_jrec *h = (g6x_jrec *)host_alloc_mapped(sizeof(g6x_jrec) * cap, &d);
    if (!h)
        return G6_ENOMEM;
    if (c.jst_inflight) {
        cudaEventSynchronize(c.ev_jst);
        c.jst_inflight = false;
    }
    if (c.n_jst)
        std::memcpy(h, c.h_jst, sizeof(g6x_jrec) * c.n_jst);
    host_free(c.h_jst);
    c.h_jst = h;
    c.d_jst = (g6x_jrec *)d;
    c.jst_cap = cap;
    return 0;
}

// Upload staged j updates and scatter them into j-memory (K0).
int flush_jstage(Ctx &c)
{
    if (c.n_jst == 0)
        return 0;
    cudaError_t e;
    {
        PhaseTimer pt(c, PH_SCATTER);
        e = g6::launch_scatter(c.d_jst, c.n_jst, c.js, c.stream);   // reads the mapped staging
    }
    if (e == cudaSuccess)
        e = cudaEventRecord(c.ev_jst, c.stream);
    if (e != cudaSuccess)
        return cuda_err(e);
    c.launches += 1;
    c.jst_inflight = true;
    for (int k = 0; k < c.n_jst; ++k)
        c.slot_of[c.h_jst[k].address] = -1;
    c.n_jst = 0;
    c.ver += 1;
    return 0;
}

// Predict j-slots 0 .. nj-1 to t_set unless this mode already holds exactly
// that prediction (Sect. 2.1: the O(n) predictor runs once per block time).
int predict_if_stale(Ctx &c, int nj)
{
    // kind of prediction: the two DS predictors share one output buffer
    const int m = c.pmode == G6X_PREC_FP64 ? g6::PRED_FP64
                  : c.pmode == G6X_PREC_DS_X64 ? g6::PRED_DS_X64 : g6::PRED_DS;
    if (c.t_pred[m] == c.t_set && c.nj_pred[m] == nj && c.ver_pred[m] == c.ver)
        return 0;
    int nj_pad = round_up(nj > 0 ? nj : 1, JT);
    cudaError_t e;
    {
        PhaseTimer pt(c, PH_PREDICT);
        e = g6::launch_predict(m, c.js, c.pred, nj, nj_pad, c.t_set, c.sm_count, c.stream);
    }
    if (e != cudaSuccess)
        return cuda_err(e);
    c.launches += 1;
    c.t_pred[m] = c.t_set;
    c.nj_pred[m] = nj;
    c.ver_pred[m] = c.ver;
    if (m != g6::PRED_FP64) {
        const int other = m == g6::PRED_DS ? g6::PRED_DS_X64 : g6::PRED_DS;
        c.ver_pred[other] = -1;
    }
    return 0;
}

// The GRAPE path's j-store update and prediction in one launch: the staged
// records are counting-sorted by tile on the host into mapped memory, and
// each predictor CTA stores its tile's records before predicting the tile.
// Counting sort of the staged records by j-tile into the mapped buffer,
// with the per-tile ranges in h_toff; large batches in parallel chunks
// (per-chunk counts, one prefix pass, per-chunk scatter -- the same order
// within a tile as the serial sort).  False if out of memory.
bool sort_by_tile(Ctx &c, int ntiles)
{
    const int n = c.n_jst;
    g6::HostPool *pool = n < std::max(PAR_MIN_SORT, 2 * ntiles) ? nullptr : g6::shared_pool();
    if (!pool) {
        try {
            c.tcur.assign(ntiles + 1, 0);
        } catch (...) {
            return false;
        }
        for (int k = 0; k < n; ++k)
            ++c.tcur[c.h_jst[k].address / JT + 1];
        for (int tl = 0; tl < ntiles; ++tl)
            c.tcur[tl + 1] += c.tcur[tl];
        std::memcpy(c.h_toff, c.tcur.data(), sizeof(int) * (ntiles + 1));
        for (int k = 0; k < n; ++k)
            c.h_jsort[c.tcur[c.h_jst[k].address / JT]++] = c.h_jst[k];
        return true;
    }
    const int nch = std::min(2 * pool->size(), (n + PAR_CHUNK - 1) / PAR_CHUNK);
    const int per = (n + nch - 1) / nch;
    try {
        c.cnt.assign((size_t)nch * ntiles, 0);
    } catch (...) {
        return false;
    }
    int *cnt = c.cnt.data();
    g6::parallel_run(nch, [&](int i) {
        int *ci = cnt + (size_t)i * ntiles;
        for (int k = i * per, ke = std::min(n, (i + 1) * per); k < ke; ++k)
            ++ci[c.h_jst[k].address / JT];
    });
    int run = 0;
    for (int tl = 0; tl < ntiles; ++tl) {
        c.h_toff[tl] = run;
        for (int i = 0; i < nch; ++i) {
            const int v = cnt[(size_t)i * ntiles + tl];
            cnt[(size_t)i * ntiles + tl] = run;
            run += v;
        }
    }
    c.h_toff[ntiles] = run;
    g6::parallel_run(nch, [&](int i) {
        int *ci = cnt + (size_t)i * ntiles;
        for (int k = i * per, ke = std::min(n, (i + 1) * per); k < ke; ++k)
            c.h_jsort[ci[c.h_jst[k].address / JT]++] = c.h_jst[k];
    });
    return true;
}

// predict = false: only store the staged records (for a force kernel that
// predicts the j-tiles itself); every cached prediction is then stale.
// fold_jtiles > 0 (with predict = false): when every staged record lies in
// the first fold_jtiles tiles, only sort them; the force kernel stores them
// (one i-tile: each j-tile read by one CTA) and *folded is set -- the caller
// then records ev_jsort after that launch.
int update_and_predict(Ctx &c, int nj, bool predict = true, int fold_jtiles = 0,
                       bool *folded = nullptr)
{
    if (folded)
        *folded = false;
    if (c.n_jst == 0)
        return predict ? predict_if_stale(c, nj) : 0;
    const int nj_pad = predict ? round_up(nj > 0 ? nj : 1, JT) : 0;
    int max_tile = 0;
    for (int k = 0; k < c.n_jst; ++k) {
        const int tl = c.h_jst[k].address / JT;
        if (tl > max_tile)
            max_tile = tl;
    }
    const bool fold = !predict && folded && fold_jtiles > 0 && max_tile + 1 <= fold_jtiles;
    const int ntiles_all = fold ? fold_jtiles
                           : nj_pad / JT > max_tile + 1 ? nj_pad / JT : max_tile + 1;
    if (c.jsort_inflight) {                 // the previous sorted batch is still read
        if (cudaEventQuery(c.ev_jsort) != cudaSuccess)
            cudaEventSynchronize(c.ev_jsort);
        cudaGetLastError();
        c.jsort_inflight = false;
    }
    if (c.n_jst > c.jsort_cap) {
        int cap = c.jsort_cap ? c.jsort_cap : 1024;
        while (cap < c.n_jst)
            cap *= 2;
        void *d = nullptr;
        g6x_jrec *h = (g6x_jrec *)host_alloc_mapped(sizeof(g6x_jrec) * cap, &d);
        if (!h)
            return G6_ENOMEM;
        host_free(c.h_jsort);
        c.h_jsort = h;
        c.d_jsort = (g6x_jrec *)d;
        c.jsort_cap = cap;
    }
    if (ntiles_all + 1 > c.toff_cap) {
        int cap = ntiles_all + 1 + 64;
        void *d = nullptr;
        int *h = (int *)host_alloc_mapped(sizeof(int) * cap, &d);
        if (!h)
            return G6_ENOMEM;
        host_free(c.h_toff);
        c.h_toff = h;
        c.d_toff = (int *)d;
        c.toff_cap = cap;
    }
    if (!sort_by_tile(c, ntiles_all))
        return G6_ENOMEM;
    const int kind = c.pmode == G6X_PREC_FP64 ? g6::PRED_FP64
                     : c.pmode == G6X_PREC_DS_X64 ? g6::PRED_DS_X64 : g6::PRED_DS;
    if (fold) {
        *folded = true;
    } else {
        cudaError_t e;
        {
            PhaseTimer pt(c, PH_PREDICT);
            e = g6::launch_update_predict(kind, c.js, c.pred, nj, nj_pad, c.t_set, c.d_jsort,
                                          c.d_toff, ntiles_all, c.sm_count, c.stream);
        }
        if (e == cudaSuccess)
            e = cudaEventRecord(c.ev_jsort, c.stream);
        if (e != cudaSuccess)
            return cuda_err(e);
        c.launches += 1;
        c.jsort_inflight = true;
    }
    par_for(c, c.n_jst, [&](int k0, int k1) {
        for (int k = k0; k < k1; ++k)
            c.slot_of[c.h_jst[k].address] = -1;
    });
    c.n_jst = 0;
    c.ver += 1;
    if (!predict)
        return 0;                  // c.ver moved on: every cached prediction is stale
    c.t_pred[kind] = c.t_set;
    c.nj_pred[kind] = nj;
    c.ver_pred[kind] = c.ver;
    if (kind != g6::PRED_FP64) {
        const int other = kind == g6::PRED_DS ? g6::PRED_DS_X64 : g6::PRED_DS;
        c.ver_pred[other] = -1;
    }
    if (kind != g6::PRED_FP64)
        c.ver_pred[g6::PRED_FP64] = -1;
    else
        c.ver_pred[g6::PRED_DS] = c.ver_pred[g6::PRED_DS_X64] = -1;
    return 0;
}

// Output neighbour lists for ni i-particles, in mapped host memory: the
// reduction writes each list's entries and its length there directly, so a
// read moves only the entries found, not ni x maxnb slots.
int grow_nb_out(Ctx &c, int ni)
{
    if ((size_t)ni <= c.nbo_cap && c.d_nbl && c.nbo_maxnb == c.maxnb)
        return 0;
    size_t n = (size_t)(ni > 16 ? ni : 16);
    void *dl = nullptr, *dn = nullptr;
    int *hl = (int *)host_alloc_mapped(n * c.maxnb * sizeof(int), &dl);
    int *hn = (int *)host_alloc_mapped(n * sizeof(int), &dn);
    if (!hl || !hn) {
        host_free(hl);
        host_free(hn);
        return G6_ENOMEM;
    }
    host_free(c.h_nbl);
    host_free(c.h_nblen);
    c.d_nbl = (int *)dl;
    c.d_nblen = (int *)dn;
    c.h_nbl = hl;
    c.h_nblen = hn;
    c.nbo_cap = n;
    c.nbo_maxnb = c.maxnb;
    return 0;
}

// Force + reduction on ni i records already on the device.
// The launch for ni i-particles against nj j-particles; a fused-prediction
// shape only with the DS + SP predictor and no lists.
ForceConfig pick_config(const Ctx &c, int nj, int ni, bool list)
{
    const int nj_pad = round_up(nj > 0 ? nj : 1, JT);
    return g6::choose_config(c.prec, ni, nj_pad, list ? 1 : 0, c.sm_count, c.force_variant,
                             c.force_grid, c.pmode == G6X_PREC_DS && !list);
}

// j-store update, prediction (unless the force kernel predicts itself),
// force and reduction.
int run_force(Ctx &c, const ForceConfig &cfg, int nj, int ni, const g6x_irec *d_irec,
              double eps2, g6x_out *d_out, bool folded);

int predict_and_force(Ctx &c, int nj, int ni, const g6x_irec *d_irec, double eps2, bool list,
                      g6x_out *d_out)
{
    const ForceConfig cfg = pick_config(c, nj, ni, list);
    const bool fp = g6::variant_info(cfg.variant).fpred != 0 && ni > 0;
    // a small block is one launch: the fused-prediction kernel also stores
    // the staged records of its tiles
    bool folded = false;
    int rc = update_and_predict(c, nj, !fp, fp && cfg.n_itile == 1 ? cfg.jtiles : 0, &folded);
    if (!rc && ni > 0)
        rc = run_force(c, cfg, nj, ni, d_irec, eps2, d_out, folded);
    if (folded) {
        if (rc) {
            // no kernel stored the sorted records: store them now
            const int kind = c.pmode == G6X_PREC_DS_X64 ? g6::PRED_DS_X64 : g6::PRED_DS;
            if (g6::launch_update_predict(kind, c.js, c.pred, nj, 0, c.t_set, c.d_jsort, c.d_toff,
                                          cfg.jtiles, c.sm_count, c.stream) == cudaSuccess)
                c.launches += 1;
            else
                cudaGetLastError();
        }
        if (cudaEventRecord(c.ev_jsort, c.stream) != cudaSuccess)
            cudaGetLastError();
        c.jsort_inflight = true;
    }
    return rc;
}

// At least n zeroed arrival counters for the reductions inside the force
// launch (zeroed again after a launch that may have stopped mid-count).
int ensure_counters(Ctx &c, size_t n)
{
    if (n > c.tcnt_cap) {
        size_t cap = n + n / 4 + 64;
        unsigned *q = (unsigned *)dev_alloc(cap * sizeof(*q));
        if (!q)
            return G6_ENOMEM;
        dev_free(c.d_tcnt);
        c.d_tcnt = q;
        c.tcnt_cap = cap;
        c.tcnt_dirty = true;
    }
    if (c.tcnt_dirty) {
        if (cudaMemsetAsync(c.d_tcnt, 0, c.tcnt_cap * sizeof(unsigned), c.stream) != cudaSuccess)
            return cuda_err(cudaGetLastError());
        c.tcnt_dirty = false;
    }
    return 0;
}

int run_force(Ctx &c, const ForceConfig &cfg, int nj, int ni, const g6x_irec *d_irec,
              double eps2, g6x_out *d_out, bool folded)
{
    // fused-prediction shapes read the j-store itself (the predicted tiles
    // and their cache entry are left as they are); folded: they also store
    // the staged records first
    g6::FusedPred fpa{c.js, c.t_set, nj};
    if (folded) {
        fpa.rec = c.d_jsort;
        fpa.toff = c.d_toff;
    }
    const g6::FusedPred *fpp = g6::variant_info(cfg.variant).fpred ? &fpa : nullptr;
    size_t slots = g6::partial_slots(cfg);
    int rc = grow_dev(c.d_part, c.part_cap, slots);
    if (rc)
        return rc;
    g6::ListArgs la{c.maxnb, c.nbseg < c.maxnb ? c.nbseg : c.maxnb, c.d_nbmax};
    if (cfg.list) {
        // each list partial (one CTA's segment of one i-particle) has room
        // for la.nbseg entries, not for a whole list: the partials take
        // slots x nbseg ints instead of slots x maxnb (the split-j shapes
        // also keep one run per j-group)
        rc = grow_dev(c.d_nbc_part, c.nbp_cap, slots);
        if (rc)
            return rc;
        rc = grow_dev(c.d_nbl_part, c.nbl_ints, g6::list_part_ints(cfg, la.nbseg));
        if (rc)
            return rc;
        c.nbp_seg = la.nbseg;
        rc = grow_nb_out(c, ni);
        if (rc)
            return rc;
        if (cudaMemsetAsync(c.d_nbmax, 0, sizeof(int), c.stream) != cudaSuccess)
            return cuda_err(cudaGetLastError());
    }
    cudaError_t e;
    // Programmatic dependent launch of the force kernel and the reduction
    // (each starts behind its predecessor and waits for it on the device),
    // except under per-phase event timing, whose events must bracket whole
    // kernels, and on the all-FP64 path, whose block steps it made about 2x
    // slower.
    const bool pdl = !c.timing && cfg.prec != G6X_PREC_FP64;
    const long long seg_per_tile = (long long)cfg.grid / cfg.n_itile + 1;
    if (cfg.ws) {
        // small block: store, prediction, force and reduction in one launch
        rc = ensure_counters(c, g6::counter_slots(cfg));
        if (rc)
            return rc;
        PhaseTimer pt(c, PH_FORCE);
        e = g6::launch_force_ws(cfg, d_irec, ni, eps2, nj, c.d_part, c.d_tcnt, d_out, c.js.idx,
                                c.d_err, fpa, c.stream, pdl);
        c.launches += 1;
    } else if (cfg.prec == G6X_PREC_DS && seg_per_tile <= g6::FUSED_MAX_SEGS) {
        // one launch: the last CTA of each i-tile reduces it (K3 fused into
        // K2), lists included, when every tile has only a few partials
        // (large blocks); with many partials per tile that serial tail
        // costs more than the separate K3, which spreads the sums over many
        // CTAs
        rc = ensure_counters(c, g6::counter_slots(cfg));
        if (rc)
            return rc;
        la.nbl_part = c.d_nbl_part;
        la.nbc_part = c.d_nbc_part;
        la.nbl_out = c.d_nbl;
        la.nblen_out = c.d_nblen;
        PhaseTimer pt(c, PH_FORCE);
        e = g6::launch_force_fused(cfg, c.pred, d_irec, ni, eps2, c.d_part, c.d_err, d_out,
                                   c.js.idx, c.d_tcnt, c.stream, fpp, pdl, &la);
        c.launches += 1;
    } else {
        {
            PhaseTimer pt(c, PH_FORCE);
            e = g6::launch_force(cfg, c.pred, d_irec, ni, eps2, c.d_part, c.d_nbl_part,
                                 c.d_nbc_part, c.d_err, c.stream, fpp, pdl, &la);
        }
        if (e == cudaSuccess) {
            PhaseTimer pt(c, PH_REDUCE);
            e = g6::launch_reduce(cfg, c.d_part, c.d_nbl_part, c.d_nbc_part, c.js.idx, ni,
                                  d_out, c.d_nbl, c.d_nblen, c.stream, pdl, &la);
        }
        c.launches += 2;
    }
    if (e != cudaSuccess)
        return cuda_err(e);
    c.last_cfg = cfg;
    c.lists_ready = cfg.list != 0;
    c.lists_host = false;
    c.list_ni = ni;
    if (cfg.list) {
        c.list_cfg = cfg;
        c.list_nj = nj;
        c.list_irec = d_irec;
        c.list_out = d_out;
        c.list_eps2 = eps2;
        c.list_t = c.t_set;
        c.list_ver = c.ver;
    }
    return 0;
}

int check_eps2(double eps2)
{
    return (eps2 >= 0.0 && std::isfinite(eps2)) ? 0 : G6_EINVAL;
}

}  // namespace

extern "C" {

int g6_npipes(void) { return env_int("G6GB_NPIPES", G6_NPIPES_DEFAULT); }

int g6_set_tunit(int) { return 0; }
int g6_set_xunit(int) { return 0; }

int g6x_set_allocator(g6x_alloc_fn alloc, g6x_free_fn release, void *user)
{
    if ((alloc == nullptr) != (release == nullptr))
        return G6_EINVAL;
    for (auto &c : g_ctx)
        if (c.open)
            return G6_EBUSY;
    g_alloc = alloc;
    g_free = release;
    g_alloc_user = user;
    return 0;
}

int g6x_open_ex(int cid, int nj_max, int ni_max)
{
    if (cid < 0 || cid >= G6_MAX_CLUSTERS || nj_max < 1 || ni_max < 1)
        return G6_EINVAL;
    Ctx &c = g_ctx[cid];
    if (c.open)
        return G6_EBUSY;
    c = Ctx();
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return G6_ENODEV;
    }
    if (cudaGetDevice(&c.dev) != cudaSuccess)
        return G6_ENODEV;
    cudaDeviceGetAttribute(&c.sm_count, cudaDevAttrMultiProcessorCount, c.dev);
    if (c.sm_count < 1)
        return G6_ENODEV;
    if (g6::variant_occupancy(0) < 1) {      // kernels not loadable on this GPU
        cudaGetLastError();
        return G6_ENODEV;
    }
    c.open = true;                         // so that free_ctx releases partial work
    int rc = 0;
    if (cudaStreamCreateWithFlags(&c.own, cudaStreamNonBlocking) != cudaSuccess
        || cudaEventCreateWithFlags(&c.ev_jst, cudaEventDisableTiming) != cudaSuccess
        || cudaEventCreateWithFlags(&c.ev_jsort, cudaEventDisableTiming) != cudaSuccess
        || cudaEventCreateWithFlags(&c.ev_done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        free_ctx(c);
        return G6_EIO;
    }
    c.stream = c.own;
    c.cap = round_up(nj_max, JT);
    c.ni_max = ni_max;
    size_t n = (size_t)c.cap;
    g6::JStore &js = c.js;
    js.cap = c.cap;
    js.x0 = (double *)dev_alloc(3 * n * sizeof(double));
    js.raw = (unsigned char *)dev_alloc((n / JT) * g6::RAW_TILE_BYTES);
    js.v64 = (double4_32a *)dev_alloc(n * sizeof(double4_32a));
    js.a264 = (double4_32a *)dev_alloc(n * sizeof(double4_32a));
    js.j664 = (double4_32a *)dev_alloc(n * sizeof(double4_32a));
    js.idx = (int *)dev_alloc(n * sizeof(int));
    c.pred.pt = (float *)dev_alloc(n * g6::JW * sizeof(float));
    c.pred.trange = (int2 *)dev_alloc((n / JT) * sizeof(int2));
    c.pred.p64 = (double4_32a *)dev_alloc(n * sizeof(double4_32a));
    c.pred.v64 = (double4_32a *)dev_alloc(n * sizeof(double4_32a));
    {
        void *de = nullptr;
        c.h_err = (int *)host_alloc_mapped(sizeof(int), &de);
        c.d_err = (int *)de;
        void *dm = nullptr;
        c.h_nbmax = (int *)host_alloc_mapped(sizeof(int), &dm);
        c.d_nbmax = (int *)dm;
    }
    if (!js.x0 || !js.raw || !js.v64 || !js.a264
        || !js.j664 || !js.idx || !c.pred.pt || !c.pred.trange || !c.pred.p64
        || !c.pred.v64 || !c.d_err || !c.h_err || !c.h_nbmax)
        rc = G6_ENOMEM;
    if (!rc)
        rc = ensure_io(c, ni_max < 4096 ? ni_max : 4096);
    if (!rc)
        rc = ensure_jstage(c, 1024 < c.cap ? 1024 : c.cap);
    if (!rc) {
        try {
            c.slot_of.assign(n, -1);
        } catch (...) {
            rc = G6_ENOMEM;
        }
    }
    if (!rc) {
        *c.h_err = 0;
        cudaError_t e = g6::launch_init_store(js, c.stream);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(c.stream);
        rc = cuda_err(e);
        c.launches += 1;
    }
    if (rc) {
        free_ctx(c);
        return rc;
    }
    return 0;
}

int g6_open(int cid)
{
    static bool tuning_loaded = false;
    const char *tf = std::getenv("G6GB_TUNE_FILE");
    if (!tuning_loaded && tf && *tf) {
        tuning_loaded = true;
        g6x_load_tuning(tf);
    }
    return g6x_open_ex(cid, env_int("G6GB_NJ", G6_NJ_DEFAULT), g6_npipes());
}

int g6_close(int cid)
{
    int err;
    Ctx *c = get(cid, &err);
    if (!c)
        return err;
    free_ctx(*c);
    return 0;
}

int g6x_set_precision(int cid, int mode)
{
    int err;
    Ctx *c = get(cid, &err);
    if (!c)
        return err;
    if (mode != G6X_PREC_DS && mode != G6X_PREC_FP64 && mode != G6X_PREC_DS_X64
        && mode != G6X_PREC_DS_DSSUB)
        return G6_EINVAL;
    c->pmode = mode;
    c->prec = mode == G6X_PREC_FP64 || mode == G6X_PREC_DS_DSSUB ? mode : G6X_PREC_DS;
    return 0;
}

int g6x_set_ni_max(int cid, int ni_max)
{
    int err;
    Ctx *c = get(cid, &err);
    if (!c)
        return err;
    if (ni_max < 1 || c->pending)
        return G6_EINVAL;
    c->ni_max = ni_max;
    return 0;
}

int g6x_set_stream(int cid, void *stream)
{
    int err;
    Ctx *c = get(cid, &err);
    if (!c)
        return err;
    if (c->pending)
        return G6_EBUSY;
    cudaStreamSynchronize(c->stream);
    c->stream = stream ? (cudaStream_t)stream : c->own;
    return 0;
}

int g6x_set_variant(int cid, int variant, int grid)
{
    int err;
    Ctx *c = get(cid, &err);
    if (!c)
        return err;
    if (variant >= g6::variant_count())
        return G6_EINVAL;
    c->force_variant = variant;
    c->force_grid = grid > 0 ? grid : 0;
    return 0;
}

int g6_set_ti(int cid, double ti)
{
    int err;
    Ctx *c = get(cid, &err);
    if (!c)
        return err;
    if (!std::isfinite(ti))
        return G6_EINVAL;
    c->t_set = ti;
    return 0;
}

int g6_set_j_particle(int cid, int address, int index, double tj, double dtj,
                      double mass, const double k18[3], const double j6[3],
                      const double a2[3], const double v[3], const double x[3])
{
    (void)dtj;
    (void)k18;
    int err;
    Ctx *c = get(cid, &err);
    if (!c)
        return err;
    if (address < 0 || address >= c->cap || index < 0 || !j6 || !a2 || !v || !x)
        return G6_EINVAL;
    if (c->jst_inflight) {             // staging may still be read by the GPU
        if (cudaEventQuery(c->ev_jst) != cudaSuccess)
            cudaEventSynchronize(c->ev_jst);
        cudaGetLastError();
        c->jst_inflight = false;
    }
    int slot = c->slot_of[address];
    if (slot < 0) {
        int rc = ensure_jstage(*c, c->n_jst + 1);
        if (rc)
            return rc;
        slot = c->n_jst++;
        c->slot_of[address] = slot;
    }
    g6x_jrec &r = c->h_jst[slot];
    for (int d = 0; d < 3; ++d) {
        r.x[d] = x[d];
        r.v[d] = v[d];
        r.a2[d] = a2[d];
        r.j6[d] = j6[d];
    }
    r.mass = mass;
    r.tj = tj;
    r.address = address;
    r.index = index;
    return 0;
}

void g6calc_firsthalf(int cid, int nj, int ni, const int index[],
                      const double xi[][3], const double vi[][3],
                      const double aold[][3], const double j6old[][3],
                      const double phiold[], double eps2, const double h2[])
{
    (void)aold;
    (void)j6old;
    (void)phiold;
    int err;
    Ctx *c = get(cid, &err);
    if (!c)
        return;
    if (c->pending) {                  // previous calculation never collected
        cudaEventSynchronize(c->ev_done);
        c->pending = false;
    }
    c->latched = 0;
    c->calc_ni = ni;
    c->calc_nj = nj;
    if (nj < 0 || nj > c->cap || ni < 0 || ni > c->ni_max || check_eps2(eps2)
        || (ni > 0 && (!index || !xi || !vi))) {
        c->latched = G6_EINVAL;
        c->pending = true;
        return;
    }
    int rc = ensure_io(*c, ni);
    std::atomic<int> bad{0}, any_list{0};
    if (!rc)
        par_for(*c, ni, [&](int k0, int k1) {
            int b = 0, l = 0;
            for (int k = k0; k < k1; ++k) {
                g6x_irec &r = c->h_irec[k];
                for (int d = 0; d < 3; ++d) {
                    r.x[d] = xi[k][d];
                    r.v[d] = vi[k][d];
                }
                r.h2 = h2 ? h2[k] : 0.0;
                r.index = index[k];
                r.pad = 0;
                b |= index[k] < 0;
                l |= h2 && h2[k] > 0.0;
            }
            if (b)
                bad.store(1);
            if (l)
                any_list.store(1);
        });
    if (!rc && bad.load())
        rc = G6_EINVAL;
    const bool list = any_list.load() != 0;
    // the kernels read the i-records from, and write results to, the mapped
    // host buffers: no separate copies
    if (!rc)
        rc = predict_and_force(*c, nj, ni, c->d_irec, eps2, list, c->d_out);
    if (!rc && ni > 0) {
        if (!rc && h2 && !list) {
            // every radius is <= 0: no list can have entries; skip the list
            // kernel; the read publishes empty lists
            rc = grow_nb_out(*c, ni);
            if (!rc) {
                c->lists_ready = true;
                c->list_ni = ni;
                c->list_cfg = ForceConfig{};      // nothing to compute again
            }
        }
    }
    if (!rc)
        rc = cuda_err(cudaEventRecord(c->ev_done, c->stream));
    c->latched = rc;
    c->pending = true;
}

static int lasthalf_common(int cid, int nj, int ni, double acc[][3], double jerk[][3],
                           double pot[], int nnb[])
{
    int err;
    Ctx *c = get(cid, &err);
    if (!c)
        return err;
    if (!c->pending)
        return G6_EBUSY;
    c->pending = false;
    if (c->latched)
        return c->latched;
    if (ni != c->calc_ni || nj != c->calc_nj)
        return G6_EINVAL;
    cudaError_t e = cudaEventSynchronize(c->ev_done);
    if (e != cudaSuccess)
        return cuda_err(e);
    if (*(volatile int *)c->h_err) {
        int code = *c->h_err;
        *(volatile int *)c->h_err = 0;
        c->tcnt_dirty = true;
        return code < 0 ? code : G6_EIO;
    }
    par_for(*c, ni, [&](int k0, int k1) {
        for (int k = k0; k < k1; ++k) {
            const g6x_out &o = c->h_out[k];
            for (int d = 0; d < 3; ++d) {
                if (acc)
                    acc[k][d] = o.acc[d];
                if (jerk)
                    jerk[k][d] = o.jerk[d];
            }
            if (pot)
                pot[k] = o.pot;
            if (nnb)
                nnb[k] = o.nnb;
        }
    });
    return 0;
}

int g6calc_lasthalf(int cid, int nj, int ni, const int index[], const double xi[][3],
                    const double vi[][3], double eps2, const double h2[],
                    double acc[][3], double jerk[][3], double pot[])
{
    (void)index;
    (void)xi;
    (void)vi;
    (void)eps2;
    (void)h2;
    return lasthalf_common(cid, nj, ni, acc, jerk, pot, nullptr);
}

int g6calc_lasthalf2(int cid, int nj, int ni, const int index[], const double xi[][3],
                     const double vi[][3], double eps2, const double h2[],
                     double acc[][3], double jerk[][3], double pot[], int nnbindex[])
{
    (void)index;
    (void)xi;
    (void)vi;
    (void)eps2;
    (void)h2;
    return lasthalf_common(cid, nj, ni, acc, jerk, pot, nnbindex);
}

int g6_read_neighbour_list(int cid)
{
    int err;
    Ctx *c = get(cid, &err);
    if (!c)
        return err;
    if (c->pending || !c->lists_ready)
        return G6_EINVAL;
    int n = c->list_ni;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess)
        return cuda_err(e);
    if (c->list_cfg.list && *(volatile int *)c->h_nbmax > c->nbp_seg) {
        // a list partial found more entries than it had room for: compute
        // the lists of that calculation again with enough room per partial
        // (the same launch on the same inputs, so the forces it writes
        // again are identical)
        if (c->ver != c->list_ver || c->n_jst != 0)
            return G6_EBUSY;              // j-memory has changed since
        int need = *(volatile int *)c->h_nbmax;
        int seg = c->nbseg;
        while (seg < need)
            seg *= 2;
        c->nbseg = seg < c->maxnb ? seg : c->maxnb;
        const double t_keep = c->t_set;
        c->t_set = c->list_t;
        int rc = predict_if_stale(*c, c->list_nj);
        if (!rc)
            rc = run_force(*c, c->list_cfg, c->list_nj, n, c->list_irec, c->list_eps2,
                           c->list_out, false);
        c->t_set = t_keep;
        if (rc)
            return rc;
        c->list_reruns += 1;
        e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess)
            return cuda_err(e);
        if (*(volatile int *)c->h_err) {
            int code = *c->h_err;
            *(volatile int *)c->h_err = 0;
            c->tcnt_dirty = true;
            return code < 0 ? code : G6_EIO;
        }
    }
    // the reduction wrote the lists into mapped host memory; a calculation
    // whose radii were all <= 0 ran no list kernel and has empty lists
    if (!c->list_cfg.list)
        std::memset(c->h_nblen, 0, sizeof(int) * n);
    c->lists_host = true;
    for (int k = 0; k < n; ++k)
        if (c->h_nblen[k] > c->maxnb)
            return G6_EOVERFLOW;
    return 0;
}

int g6_get_neighbour_list(int cid, int ipipe, int maxlength, int *nblen, int nbl[])
{
    int err;
    Ctx *c = get(cid, &err);
    if (!c)
        return err;
    if (!c->lists_host || ipipe < 0 || ipipe >= c->list_ni || maxlength < 0 || !nblen)
        return G6_EINVAL;
    int len = c->h_nblen[ipipe];
    *nblen = len;
    int keep = len < c->maxnb ? len : c->maxnb;
    if (keep > maxlength)
        keep = maxlength;
    if (keep > 0 && !nbl)
        return G6_EINVAL;
    for (int k = 0; k < keep; ++k)
        nbl[k] = c->h_nbl[(size_t)ipipe * c->maxnb + k];
    return (len > c->maxnb || len > maxlength) ? G6_EOVERFLOW : 0;
}

int g6x_set_max_neighbours(int cid, int maxnb)
{
    int err;
    Ctx *c = get(cid, &err);
    if (!c)
        return err;
    if (c->pending || maxnb < 1 || maxnb > G6X_MAXNB_LIMIT)
        return G6_EINVAL;
    if (maxnb != c->maxnb) {
        c->maxnb = maxnb;
        c->lists_ready = false;
        c->lists_host = false;
    }
    return 0;
}

int g6x_max_neighbours(int cid)
{
    int err;
    Ctx *c = get(cid, &err);
    return c ? c->maxnb : err;
}

long long g6x_list_reruns(int cid)
{
    int err;
    Ctx *c = get(cid, &err);
    return c ? c->list_reruns : (long long)err;
}

int g6x_set_j_particles(int cid, int n, const int address[], const int index[],
                        const double tj[], const double mass[], const double j6[][3],
                        const double a2[][3], const double v[][3], const double x[][3])
{
    if (n < 0 || (n > 0 && (!address || !index || !tj || !mass || !j6 || !a2 || !v || !x)))
        return G6_EINVAL;
    int err;
    Ctx *c = get(cid, &err);
    if (!c)
        return err;
    if (c->n_jst + n > c->jst_cap) {
        int rc = ensure_jstage(*c, c->n_jst + n < c->cap ? c->n_jst + n : c->cap);
        if (rc)
            return rc;
    }
    if (n < PAR_MIN) {
        for (int k = 0; k < n; ++k) {
            int rc = g6_set_j_particle(cid, address[k], index[k], tj[k], 0.0, mass[k], nullptr,
                                       j6[k], a2[k], v[k], x[k]);
            if (rc)
                return rc;
        }
        return 0;
    }
    // large calls: check everything, give every address its staging record
    // (in order, so an address given twice keeps its last values), then fill
    // the records on the pool
    for (int k = 0; k < n; ++k)
        if (address[k] < 0 || address[k] >= c->cap || index[k] < 0)
            return G6_EINVAL;
    if (c->jst_inflight) {             // staging may still be read by the GPU
        if (cudaEventQuery(c->ev_jst) != cudaSuccess)
            cudaEventSynchronize(c->ev_jst);
        cudaGetLastError();
        c->jst_inflight = false;
    }
    try {
        c->sidx.resize(n);
        if (c->stamp.size() < (size_t)c->jst_cap)
            c->stamp.resize(c->jst_cap, 0);
    } catch (...) {
        return G6_ENOMEM;
    }
    if (++c->stamp_now == 0) {
        std::fill(c->stamp.begin(), c->stamp.end(), 0u);
        c->stamp_now = 1;
    }
    bool twice = false;
    for (int k = 0; k < n; ++k) {
        int slot = c->slot_of[address[k]];
        if (slot < 0) {
            if (c->n_jst + 1 > c->jst_cap) {
                int rc = ensure_jstage(*c, c->n_jst + 1);
                if (rc)
                    return rc;
                if (c->stamp.size() < (size_t)c->jst_cap)
                    c->stamp.resize(c->jst_cap, 0);
            }
            slot = c->n_jst++;
            c->slot_of[address[k]] = slot;
        }
        twice |= c->stamp[slot] == c->stamp_now;
        c->stamp[slot] = c->stamp_now;
        c->sidx[k] = slot;
    }
    auto fill = [&](int k0, int k1) {
        for (int k = k0; k < k1; ++k) {
            g6x_jrec &r = c->h_jst[c->sidx[k]];
            for (int d = 0; d < 3; ++d) {
                r.x[d] = x[k][d];
                r.v[d] = v[k][d];
                r.a2[d] = a2[k][d];
                r.j6[d] = j6[k][d];
            }
            r.mass = mass[k];
            r.tj = tj[k];
            r.address = address[k];
            r.index = index[k];
        }
    };
    if (twice)
        fill(0, n);                    // in order: the last values win
    else
        par_for(*c, n, fill);
    return 0;
}

int g6x_set_j_dev(int cid, int n, const g6x_jrec *d_rec)
{
    int err;
    Ctx *c = get(cid, &err);
    if (!c)
        return err;
    if (n < 0 || (n > 0 && !d_rec) || c->pending)
        return G6_EINVAL;
    int rc = flush_jstage(*c);
    if (rc)
        return rc;
    if (n == 0)
        return 0;
    cudaError_t e;
    {
        PhaseTimer pt(*c, PH_SCATTER);
        e = g6::launch_scatter(d_rec, n, c->js, c->stream);
    }
    if (e != cudaSuccess)
        return cuda_err(e);
    c->launches += 1;
    c->ver += 1;
    return 0;
}

int g6x_calc_dev(int cid, double ti, int nj, int ni, const g6x_irec *d_irec, double eps2,
                 int nl, g6x_out *d_out)
{
    int err;
    Ctx *c = get(cid, &err);
    if (!c)
        return err;
    if (c->pending || nj < 0 || nj > c->cap || ni < 0 || check_eps2(eps2)
        || !std::isfinite(ti) || (ni > 0 && (!d_irec || !d_out)))
        return G6_EINVAL;
    c->t_set = ti;
    return predict_and_force(*c, nj, ni, d_irec, eps2, nl != 0, d_out);
}

// ------------------------------------------------ allocation-free variant
//
// g6x_calc_dev_noalloc keeps the partial sums between the force kernel and
// the reduction in the file-scope device array below instead of in context
// memory that grows on demand, so the call itself never allocates.  The
// array is G6X_NOALLOC_SCRATCH_BYTES on every GPU that loads this library,
// held until the process exits.  In host code its name only stands in for
// the device object; kernels get its device address from
// cudaGetSymbolAddress, looked up once per device by the first call there.
static __device__ __align__(256) unsigned char g6x_noalloc_scratch[G6X_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr size_t kNoallocSlots = G6X_NOALLOC_SCRATCH_BYTES / sizeof(g6::Partial);
// the header states the array as 147456 records of 72 bytes
static_assert(sizeof(g6::Partial) == 72, "partial slot size the header documents");
static_assert(kNoallocSlots == 147456, "partial slot count the header documents");
static_assert(G6X_NOALLOC_SCRATCH_BYTES % sizeof(g6::Partial) == 0,
              "scratch holds a whole number of partial records");
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices];

// Device address of the scratch array on the context's device `dev`, which
// must be the caller's current device (the kernels go to the context's
// stream on that device).
int noalloc_scratch(int dev, void **out)
{
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess)
        return cuda_err(e);
    if (cur != dev)
        return G6_EINVAL;
    if (dev < 0 || dev >= kMaxDevices)
        return G6_ENODEV;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g6x_noalloc_scratch);
        if (e != cudaSuccess)
            return cuda_err(e);
        if (!p)
            return G6_EIO;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return 0;
}

}  // namespace

extern "C" int g6x_calc_dev_noalloc(int cid, double ti, int nj, int ni,
                                    const g6x_irec *d_irec, double eps2, g6x_out *d_out)
{
    int err;
    Ctx *c = get(cid, &err);
    if (!c)
        return err;
    if (c->pending || nj < 0 || nj > c->cap || ni < 0 || ni > G6X_NOALLOC_NI_MAX
        || check_eps2(eps2) || !std::isfinite(ti) || (ni > 0 && (!d_irec || !d_out)))
        return G6_EINVAL;
    // Choose the launch before any work, shrinking the grid if the partial
    // records would not fit the array; reject what still does not fit.
    const int nj_pad = round_up(nj > 0 ? nj : 1, JT);
    ForceConfig cfg = g6::choose_config(c->prec, ni, nj_pad, 0, c->sm_count,
                                        c->force_variant, c->force_grid);
    if (cfg.list)
        return G6_EINVAL;
    if (g6::partial_slots(cfg) > kNoallocSlots) {
        long long g = (long long)(kNoallocSlots / cfg.itile) - cfg.n_itile;
        if (g < 1)
            return G6_EINVAL;
        cfg = g6::choose_config(c->prec, ni, nj_pad, 0, c->sm_count, cfg.variant, (int)g);
        if (g6::partial_slots(cfg) > kNoallocSlots)
            return G6_EINVAL;
    }
    void *scratch = nullptr;
    int rc = noalloc_scratch(c->dev, &scratch);
    if (rc)
        return rc;
    c->t_set = ti;
    rc = flush_jstage(*c);
    if (!rc)
        rc = predict_if_stale(*c, nj);
    if (rc || ni == 0)
        return rc;
    // Every record the reduction reads is written by the force kernel of
    // this same call, so nothing left by an earlier call needs clearing.
    g6::Partial *part = static_cast<g6::Partial *>(scratch);
    cudaError_t e;
    {
        PhaseTimer pt(*c, PH_FORCE);
        e = g6::launch_force(cfg, c->pred, d_irec, ni, eps2, part, nullptr, nullptr, c->d_err,
                             c->stream);
    }
    if (e == cudaSuccess) {
        PhaseTimer pt(*c, PH_REDUCE);
        e = g6::launch_reduce(cfg, part, nullptr, nullptr, c->js.idx, ni, d_out, nullptr,
                              nullptr, c->stream);
    }
    if (e != cudaSuccess)
        return cuda_err(e);
    c->launches += 2;
    c->last_cfg = cfg;
    c->lists_ready = false;
    return 0;
}

// ------------------------------------------------------------ autotuner
//
// For each power-of-two block size the tuner times every force-kernel
// variant of the current precision whose i-tile suits the block, on grids of
// one and two times the resident CTAs, with i-particles taken from the first
// m j-slots, and keeps the fastest in the process-wide table that
// choose_config consults.  Sizes above 2^17 reuse the 2^17 choice.

namespace {

int write_tuning(const char *path)
{
    std::ofstream f(path);
    if (!f)
        return G6_EINVAL;
    f << "# g6gb force-kernel tuning table: precision log2(m) variant grid_multiplier\n";
    int n = 0;
    for (int prec = 0; prec < 2; ++prec)
        for (int b = 0; b < g6::TUNE_BUCKETS; ++b) {
            int v, g;
            if (g6::tune_exact(prec, b, &v, &g)) {
                f << prec << " " << b << " " << v << " " << g << "\n";
                ++n;
            }
        }
    return f ? n : G6_EIO;
}

}  // namespace

extern "C" int g6x_autotune(int cid, int nj, int m_max, const char *path)
{
    int err;
    Ctx *c = get(cid, &err);
    if (!c)
        return err;
    if (c->pending || nj < 1 || nj > c->cap || m_max < 16 || c->prec > G6X_PREC_FP64)
        return G6_EINVAL;
    if (m_max > nj)
        m_max = nj;
    int rc = flush_jstage(*c);
    if (!rc)
        rc = predict_if_stale(*c, nj);
    if (rc)
        return rc;
    const int nj_pad = round_up(nj, JT);
    const int m_cap = m_max < (1 << 17) ? m_max : (1 << 17);
    g6x_irec *d_i = (g6x_irec *)dev_alloc(sizeof(g6x_irec) * m_cap);
    g6x_out *d_o = (g6x_out *)dev_alloc(sizeof(g6x_out) * m_cap);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!d_i || !d_o || cudaEventCreate(&e0) != cudaSuccess
        || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        dev_free(d_i);
        dev_free(d_o);
        if (e0)
            cudaEventDestroy(e0);
        return G6_ENOMEM;
    }
    cudaError_t e = g6::launch_irec_from_store(c->js, d_i, m_cap, c->stream);
    c->launches += 1;
    const int pkind = c->pmode == G6X_PREC_FP64 ? g6::PRED_FP64
                      : c->pmode == G6X_PREC_DS_X64 ? g6::PRED_DS_X64 : g6::PRED_DS;
    int tuned = 0;
    bool lost_work = false;
    for (int m = 16; e == cudaSuccess && m <= m_cap; m *= 2) {
        float best = 1e30f;
        int bv = -1, bg = 1;
        for (int v = 0; v < g6::variant_count() && e == cudaSuccess; ++v) {
            const g6::VariantInfo vi = g6::variant_info(v);
            if (vi.prec != c->prec || vi.list || vi.ti * vi.nper > 16 * m
                || (vi.fpred && c->pmode != G6X_PREC_DS) || (vi.ws && vi.ti * vi.nper < m))
                continue;
            int occ = g6::variant_occupancy(v);
            if (occ < 1)
                continue;
            int last_grid = -1;
            for (int gm = 1; gm <= 8 && e == cudaSuccess; gm *= 2) {
                // more than two waves only for the widest tiles on long work lines
                if (gm > 2 && (vi.ti * vi.nper < 256 || m < 16384))
                    break;
                ForceConfig cfg = g6::choose_config(c->prec, m, nj_pad, 0, c->sm_count, v,
                                                    c->sm_count * occ * gm, true);
                if (cfg.grid == last_grid)
                    continue;
                last_grid = cfg.grid;
                if (grow_dev(c->d_part, c->part_cap, g6::partial_slots(cfg))
                    || (vi.ws && ensure_counters(*c, g6::counter_slots(cfg)))) {
                    lost_work = true;
                    continue;
                }
                float t_best = 1e30f;
                // a step: the prediction (inside the kernel for fused
                // shapes) + force + reduction; the tiles predicted by either
                // route at the same time are identical, so the cached
                // prediction stays valid
                const g6::FusedPred fpa{c->js, c->t_set, nj};
                for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
                    e = cudaEventRecord(e0, c->stream);
                    if (e == cudaSuccess && !vi.fpred)
                        e = g6::launch_predict(pkind, c->js, c->pred, nj, nj_pad, c->t_set,
                                               c->sm_count, c->stream);
                    if (e == cudaSuccess && vi.ws) {
                        e = g6::launch_force_ws(cfg, d_i, m, 1e-6, nj, c->d_part, c->d_tcnt, d_o,
                                                c->js.idx, c->d_err, fpa, c->stream, false);
                    } else {
                        if (e == cudaSuccess)
                            e = g6::launch_force(cfg, c->pred, d_i, m, 1e-6, c->d_part, nullptr,
                                                 nullptr, c->d_err, c->stream,
                                                 vi.fpred ? &fpa : nullptr);
                        if (e == cudaSuccess)
                            e = g6::launch_reduce(cfg, c->d_part, nullptr, nullptr, c->js.idx,
                                                  m, d_o, nullptr, nullptr, c->stream);
                    }
                    if (e == cudaSuccess)
                        e = cudaEventRecord(e1, c->stream);
                    if (e == cudaSuccess)
                        e = cudaEventSynchronize(e1);
                    float ms = 0.f;
                    if (e == cudaSuccess)
                        e = cudaEventElapsedTime(&ms, e0, e1);
                    c->launches += 2;
                    if (r > 0 && ms < t_best)
                        t_best = ms;
                }
                if (t_best < best) {
                    best = t_best;
                    bv = v;
                    bg = gm;
                }
            }
        }
        if (bv >= 0) {
            g6::tune_set(c->prec, g6::tune_bucket(m), bv, bg);
            ++tuned;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dev_free(d_i);
    dev_free(d_o);
    if (e != cudaSuccess)
        return cuda_err(e);
    if (lost_work && tuned == 0)
        return G6_ENOMEM;
    if (path) {
        int w = write_tuning(path);
        if (w < 0)
            return w;
    }
    return tuned;
}

extern "C" int g6x_load_tuning(const char *path)
{
    if (!path)
        return G6_EINVAL;
    std::ifstream f(path);
    if (!f)
        return G6_EINVAL;
    // the whole file is checked before any entry takes effect
    std::string line;
    std::vector<std::array<int, 4>> rows;
    while (std::getline(f, line)) {
        if (line.empty() || line[0] == '#')
            continue;
        std::istringstream is(line);
        int prec, b, v, g;
        if (!(is >> prec >> b >> v >> g))
            return G6_EINVAL;
        if (prec < 0 || prec > 1 || b < 0 || b >= g6::TUNE_BUCKETS || v < 0
            || v >= g6::variant_count() || g < 1 || g > 8
            || g6::variant_info(v).prec != prec || g6::variant_info(v).list)
            return G6_EINVAL;
        rows.push_back({prec, b, v, g});
    }
    for (const auto &r : rows)
        g6::tune_set(r[0], r[1], r[2], r[3]);
    return (int)rows.size();
}

extern "C" int g6x_clear_tuning(void)
{
    g6::tune_clear();
    return 0;
}

int g6x_sync(int cid)
{
    int err;
    Ctx *c = get(cid, &err);
    if (!c)
        return err;
    if (c->pending)
        return G6_EBUSY;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess)
        return cuda_err(e);
    if (*(volatile int *)c->h_err) {
        int code = *c->h_err;
        *(volatile int *)c->h_err = 0;
        c->tcnt_dirty = true;
        return code < 0 ? code : G6_EIO;
    }
    return 0;
}

int g6x_set_wait_limit(double seconds)
{
    const double max_s = 1e-9 * (double)g6::max_wait_limit_ns();
    if (!(seconds >= 1e-6) || !(seconds <= max_s))
        return G6_EINVAL;
    g6::set_wait_limit_ns((unsigned long long)(seconds * 1e9));
    return 0;
}

int g6x_probe_wait_timeout(int cid)
{
    int err;
    Ctx *c = get(cid, &err);
    if (!c)
        return err;
    if (c->pending)
        return G6_EBUSY;
    cudaError_t e = g6::launch_wait_probe(c->d_err, c->stream);
    if (e != cudaSuccess)
        return cuda_err(e);
    return g6x_sync(cid);
}

int g6x_get_predicted(int cid, int nj, float *hi, float *lo, float *vel, double *x64,
                      double *v64)
{
    int err;
    Ctx *c = get(cid, &err);
    if (!c)
        return err;
    if (c->pending || nj < 0 || nj > c->cap)
        return G6_EINVAL;
    int rc = flush_jstage(*c);
    if (!rc)
        rc = predict_if_stale(*c, nj);
    if (rc)
        return rc;
    cudaError_t e = cudaSuccess;
    size_t d4 = sizeof(double4_32a) * (size_t)nj;
    if (c->prec != G6X_PREC_FP64) {
        // copy the tiled layout back and unpack it into (x, y, z, w) rows
        const int ntile = (nj + JT - 1) / JT;
        std::vector<float> t((size_t)ntile * JT * g6::JW);
        e = cudaMemcpyAsync(t.data(), c->pred.pt, t.size() * sizeof(float),
                            cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(c->stream);
        if (e == cudaSuccess) {
            for (int k = 0; k < nj; ++k) {
                const float *b = t.data() + (size_t)(k / JT) * JT * g6::JW + k % JT;
                auto w = [&](int comp) { return b[comp * JT]; };
                if (hi) {
                    hi[4 * k + 0] = w(g6::W_XH);
                    hi[4 * k + 1] = w(g6::W_YH);
                    hi[4 * k + 2] = w(g6::W_ZH);
                    hi[4 * k + 3] = w(g6::W_M);
                }
                if (lo) {
                    lo[4 * k + 0] = w(g6::W_XL);
                    lo[4 * k + 1] = w(g6::W_YL);
                    lo[4 * k + 2] = w(g6::W_ZL);
                    lo[4 * k + 3] = 0.f;
                }
                if (vel) {
                    vel[4 * k + 0] = w(g6::W_VX);
                    vel[4 * k + 1] = w(g6::W_VY);
                    vel[4 * k + 2] = w(g6::W_VZ);
                    vel[4 * k + 3] = w(g6::W_ID);
                }
            }
        }
    } else {
        if (x64 && e == cudaSuccess)
            e = cudaMemcpyAsync(x64, c->pred.p64, d4, cudaMemcpyDeviceToHost, c->stream);
        if (v64 && e == cudaSuccess)
            e = cudaMemcpyAsync(v64, c->pred.v64, d4, cudaMemcpyDeviceToHost, c->stream);
    }
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(c->stream);
    return cuda_err(e);
}

int g6x_set_timing(int cid, int enable)
{
    int err;
    Ctx *c = get(cid, &err);
    if (!c)
        return err;
    cudaStreamSynchronize(c->stream);
    resolve_timing(*c);
    for (int p = 0; p < 4; ++p) {
        c->t_ms[p] = 0.0;
        c->t_cnt[p] = 0;
    }
    c->timing = enable != 0;
    return 0;
}

int g6x_get_timing(int cid, double ms[4], long long count[4])
{
    int err;
    Ctx *c = get(cid, &err);
    if (!c)
        return err;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess)
        return cuda_err(e);
    resolve_timing(*c);
    for (int p = 0; p < 4; ++p) {
        if (ms)
            ms[p] = c->t_ms[p];
        if (count)
            count[p] = c->t_cnt[p];
    }
    return 0;
}

int g6x_plan_launch(int mode, int nj, int ni, int list, int sm_count, int out[6])
{
    if ((mode != G6X_PREC_DS && mode != G6X_PREC_FP64 && mode != G6X_PREC_DS_X64
         && mode != G6X_PREC_DS_DSSUB)
        || nj < 1 || nj > (1 << 30) || ni < 1 || ni > (1 << 30) || sm_count < 1
        || sm_count > 4096 || !out || (list && mode == G6X_PREC_DS_DSSUB))
        return G6_EINVAL;
    const int prec = mode == G6X_PREC_FP64 || mode == G6X_PREC_DS_DSSUB ? mode : G6X_PREC_DS;
    const int nj_pad = round_up(nj, JT);
    const ForceConfig f = g6::choose_config(prec, ni, nj_pad, list ? 1 : 0, sm_count, -1, 0,
                                            mode == G6X_PREC_DS && !list);
    // without a device the occupancy query fails: clear its error
    cudaGetLastError();
    out[0] = f.variant;
    out[1] = f.ti;
    out[2] = f.tj;
    out[3] = f.nper;
    out[4] = f.grid;
    out[5] = f.jtiles;
    return 0;
}

int g6x_variant_info(int variant, int out[8])
{
    const int n = g6::variant_count();
    if (variant == -1 && !out)
        return n;
    if (variant < 0 || variant >= n || !out)
        return G6_EINVAL;
    const g6::VariantInfo v = g6::variant_info(variant);
    out[0] = v.ti;
    out[1] = v.tj;
    out[2] = v.nper;
    out[3] = v.list;
    out[4] = v.prec;
    out[5] = v.fpred;
    out[6] = v.twin;
    out[7] = v.ws;
    return n;
}

int g6x_last_config(int cid, int *variant, int *ti, int *tj, int *ni_per, int *grid,
                    int *jtiles)
{
    int err;
    Ctx *c = get(cid, &err);
    if (!c)
        return err;
    const ForceConfig &f = c->last_cfg;
    if (variant)
        *variant = f.variant;
    if (ti)
        *ti = f.ti;
    if (tj)
        *tj = f.tj;
    if (ni_per)
        *ni_per = f.nper;
    if (grid)
        *grid = f.grid;
    if (jtiles)
        *jtiles = f.jtiles;
    return 0;
}

long long g6x_launch_count(int cid)
{
    int err;
    Ctx *c = get(cid, &err);
    return c ? c->launches : (long long)err;
}

const char *g6x_strerror(int code)
{
    switch (code) {
    case G6_OK: return "ok";
    case G6_EINVAL: return "invalid argument";
    case G6_ENOTOPEN: return "cluster id not open";
    case G6_EBUSY: return "cluster id busy or call out of order";
    case G6_ENOMEM: return "out of device or pinned host memory";
    case G6_EIO: return "CUDA runtime error";
    case G6_ETIMEDOUT: return "device-side bounded wait timed out";
    case G6_ENODEV: return "no usable CUDA device for this library";
    case G6_EOVERFLOW: return "neighbour list overflow";
    default: return "unknown error";
    }
}

}  // extern "C"
