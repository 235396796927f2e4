// g6gb_batch.cu -- many independent clusters in one launch sequence.
//
// A batch holds the j-memory of every cluster (each cluster at a JT-aligned
// range of slots).  One batch calculation gives every cluster its own block
// time and active set (Sect. 2, Sect. 2.1: block time steps, O(nm) force per
// block) and computes all of them with three launches -- the j-store update
// fused into the per-cluster prediction (Eq. 1, Eq. 2), one force kernel over
// a single work line that concatenates every cluster's (i-tile, j-tile) pairs
// and is cut evenly over a fixed grid, and the reduction -- all of which read
// their per-step geometry from mapped memory, so the sequence is captured
// once in a CUDA graph and replayed every step.  For comparison the same
// kernels can run as one launch sequence per cluster.
//
// The C++ batch driver (g6hb_*) runs a Hermite block-time-step integration in
// every cluster with its own block scheduler, advancing each cluster by one
// of its own block steps per batch step.
#include "g6gb_internal.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <vector>

using g6::JT;

struct g6x_batch {
    int ncl = 0, pmode = G6X_PREC_DS, sms = 0;
    cudaStream_t stream = nullptr;
    std::vector<int> nj, jtile, ntile, ioff;
    int total_tiles = 0, total_slots = 0, total_i = 0;
    g6::JStore js{};
    g6::Pred pred{};
    int *d_tile_cluster = nullptr, *d_cl_jtile = nullptr, *d_cl_nj = nullptr;
    // per-step tables in mapped memory (host pointer h_*, device alias d_*)
    long long *h_hdr = nullptr, *d_hdr = nullptr;           // [2]
    long long *h_gts = nullptr, *d_gts = nullptr;           // [gt_cap + 1]
    int *h_gtc = nullptr, *d_gtc = nullptr, *h_gti = nullptr, *d_gti = nullptr;
    int *h_ioff = nullptr, *d_ioff = nullptr, *h_ni = nullptr, *d_ni = nullptr;
    double *h_eps2 = nullptr, *d_eps2 = nullptr, *h_t = nullptr, *d_t = nullptr;
    long long *h_hdr_each = nullptr, *d_hdr_each = nullptr; // [ncl][2]
    long long *h_gts_each = nullptr, *d_gts_each = nullptr; // per-cluster work starts
    std::vector<int> gts_each_off;                          // ncl + 1
    std::vector<int> gt_first;                              // first global i-tile per cluster
    g6x_irec *h_irec = nullptr, *d_irec = nullptr;
    g6x_out *h_out = nullptr, *d_out = nullptr;
    // j staging: one record per global slot, sorted by tile at launch
    std::vector<g6x_jrec> stage;
    std::vector<int> slot_of;
    g6x_jrec *h_jsort = nullptr, *d_jsort = nullptr;
    int jsort_cap = 0;
    int *h_toff = nullptr, *d_toff = nullptr;
    std::vector<int> tcur;
    void *d_part = nullptr;
    int *h_err = nullptr, *d_err = nullptr;
    int variant = 0, grid = 0, itile = 16, gt_cap = 0, k3_blocks = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    long long launches = 0;
};

namespace {

template <class T>
T *dalloc(size_t n)
{
    return static_cast<T *>(g6::dev_alloc_hooked(n * sizeof(T)));
}

template <class T>
T *halloc(size_t n, T **dev)
{
    void *d = nullptr;
    T *h = static_cast<T *>(g6::host_alloc_zero_copy(n * sizeof(T), &d));
    *dev = static_cast<T *>(d);
    return h;
}

int cuda_code(cudaError_t e)
{
    if (e == cudaSuccess)
        return 0;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? G6_ENOMEM : G6_EIO;
}

void free_batch(g6x_batch *b)
{
    if (b->stream)
        cudaStreamSynchronize(b->stream);
    if (b->gexec)
        cudaGraphExecDestroy(b->gexec);
    if (b->graph)
        cudaGraphDestroy(b->graph);
    g6::JStore &js = b->js;
    void *dp[] = {js.x0, js.xds, js.xds2, js.t0, js.v0m, js.a2f, js.j6f, js.v64, js.a264,
                  js.j664, js.idx, b->pred.pt, b->pred.trange, b->pred.p64, b->pred.v64,
                  b->d_tile_cluster, b->d_cl_jtile, b->d_cl_nj, b->d_part};
    for (void *p : dp)
        g6::dev_free_hooked(p);
    void *hp[] = {b->h_hdr, b->h_gts, b->h_gtc, b->h_gti, b->h_ioff, b->h_ni, b->h_eps2, b->h_t,
                  b->h_hdr_each, b->h_gts_each, b->h_irec, b->h_out, b->h_jsort, b->h_toff,
                  b->h_err};
    for (void *p : hp)
        g6::host_free_pinned(p);
    if (b->stream)
        cudaStreamDestroy(b->stream);
    delete b;
}

// Sort the staged records by tile into the mapped buffer; toff gets the
// per-tile ranges (all equal when nothing is staged).
int stage_sorted(g6x_batch *b)
{
    // at most one staged record per slot, and the buffer holds one per
    // particle, so the captured graph's pointer never changes
    if ((int)b->stage.size() > b->jsort_cap)
        return G6_EINVAL;
    b->tcur.assign(b->total_tiles + 1, 0);
    for (const g6x_jrec &r : b->stage)
        ++b->tcur[r.address / JT + 1];
    for (int t = 0; t < b->total_tiles; ++t)
        b->tcur[t + 1] += b->tcur[t];
    std::memcpy(b->h_toff, b->tcur.data(), sizeof(int) * (b->total_tiles + 1));
    for (const g6x_jrec &r : b->stage)
        b->h_jsort[b->tcur[r.address / JT]++] = r;
    for (const g6x_jrec &r : b->stage)
        b->slot_of[r.address] = -1;
    b->stage.clear();
    return 0;
}

int pred_kind(const g6x_batch *b)
{
    return b->pmode == G6X_PREC_DS_X64 ? g6::PRED_DS_X64 : g6::PRED_DS;
}

g6::BatchPredTables pred_tables(const g6x_batch *b)
{
    g6::BatchPredTables bp;
    bp.tile_cluster = b->d_tile_cluster;
    bp.cl_jtile = b->d_cl_jtile;
    bp.cl_nj = b->d_cl_nj;
    bp.cl_ni = b->d_ni;
    bp.cl_t = b->d_t;
    return bp;
}

g6::BatchTables force_tables(const g6x_batch *b, const long long *hdr, const long long *gts,
                             const int *gtc, const int *gti)
{
    g6::BatchTables bt;
    bt.hdr = hdr;
    bt.gt_start = gts;
    bt.gt_cluster = gtc;
    bt.gt_itile = gti;
    bt.cl_jtile = b->d_cl_jtile;
    bt.cl_ioff = b->d_ioff;
    bt.cl_ni = b->d_ni;
    bt.cl_eps2 = b->d_eps2;
    return bt;
}

// The three launches over every cluster.
cudaError_t enqueue_all(g6x_batch *b)
{
    cudaError_t e = g6::launch_predict_batch(pred_kind(b), b->js, b->pred, pred_tables(b),
                                             b->d_jsort, b->d_toff, 0, b->total_tiles, b->sms,
                                             b->stream);
    const g6::BatchTables bt = force_tables(b, b->d_hdr, b->d_gts, b->d_gtc, b->d_gti);
    if (e == cudaSuccess)
        e = g6::launch_force_batch(b->variant, b->grid, b->pred, b->d_irec, b->d_part, b->d_err,
                                   bt, b->stream);
    if (e == cudaSuccess)
        e = g6::launch_reduce_batch(b->variant, b->grid, b->d_part, b->js.idx, b->d_out, bt,
                                    b->k3_blocks, b->stream);
    return e;
}

}  // namespace

extern "C" {

g6x_batch *g6x_batch_create(int ncl, const int nj[], int precision, int variant, int grid_mul,
                            int *err)
{
    if (err)
        *err = 0;
    if (ncl < 1 || !nj || (precision != G6X_PREC_DS && precision != G6X_PREC_DS_X64)
        || variant < -1 || variant >= g6::batch_variant_count() || grid_mul < 0) {
        if (err)
            *err = G6_EINVAL;
        return nullptr;
    }
    g6x_batch *b = new (std::nothrow) g6x_batch();
    if (!b) {
        if (err)
            *err = G6_ENOMEM;
        return nullptr;
    }
    int rc = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    b->ncl = ncl;
    b->pmode = precision;
    b->variant = variant >= 0 ? variant : 0;
    b->itile = g6::batch_variant_info(b->variant).ti * g6::batch_variant_info(b->variant).nper;
    const int occ = g6::batch_variant_occupancy(b->variant);
    if (b->sms < 1 || occ < 1) {
        if (err)
            *err = G6_ENODEV;
        delete b;
        cudaGetLastError();
        return nullptr;
    }
    b->grid = b->sms * occ * (grid_mul > 0 ? grid_mul : 1);
    try {
        b->nj.assign(nj, nj + ncl);
        b->jtile.resize(ncl);
        b->ntile.resize(ncl);
        b->ioff.resize(ncl);
        b->gts_each_off.resize(ncl + 1);
        b->gt_first.resize(ncl);
    } catch (...) {
        delete b;
        if (err)
            *err = G6_ENOMEM;
        return nullptr;
    }
    int tiles = 0, slots_i = 0, gts_each = 0;
    for (int k = 0; k < ncl; ++k) {
        if (nj[k] < 1) {
            delete b;
            if (err)
                *err = G6_EINVAL;
            return nullptr;
        }
        b->jtile[k] = tiles;
        b->ntile[k] = (nj[k] + JT - 1) / JT;
        tiles += b->ntile[k];
        b->ioff[k] = slots_i;
        slots_i += nj[k];
        b->gts_each_off[k] = gts_each;
        gts_each += (nj[k] + b->itile - 1) / b->itile + 1;
        b->gt_cap += (nj[k] + b->itile - 1) / b->itile;
    }
    b->gts_each_off[ncl] = gts_each;
    b->total_tiles = tiles;
    b->total_slots = tiles * JT;
    b->total_i = slots_i;
    const size_t n = (size_t)b->total_slots;
    g6::JStore &js = b->js;
    js.cap = b->total_slots;
    js.x0 = dalloc<double>(3 * n);
    js.xds = dalloc<float4>(n);
    js.xds2 = dalloc<float2>(n);
    js.t0 = dalloc<double>(n);
    js.v0m = dalloc<float4>(n);
    js.a2f = dalloc<float4>(n);
    js.j6f = dalloc<float4>(n);
    js.v64 = dalloc<double4_32a>(n);
    js.a264 = dalloc<double4_32a>(n);
    js.j664 = dalloc<double4_32a>(n);
    js.idx = dalloc<int>(n);
    b->pred.pt = dalloc<float>(n * g6::JW);
    b->pred.trange = dalloc<int2>(tiles);
    b->d_tile_cluster = dalloc<int>(tiles);
    b->d_cl_jtile = dalloc<int>(ncl);
    b->d_cl_nj = dalloc<int>(ncl);
    b->d_part = g6::dev_alloc_hooked((size_t)(b->grid + b->gt_cap) * b->itile * g6::PARTIAL_BYTES);
    b->h_hdr = halloc<long long>(2, &b->d_hdr);
    b->h_gts = halloc<long long>(b->gt_cap + 1, &b->d_gts);
    b->h_gtc = halloc<int>(b->gt_cap + 1, &b->d_gtc);
    b->h_gti = halloc<int>(b->gt_cap + 1, &b->d_gti);
    b->h_ioff = halloc<int>(ncl, &b->d_ioff);
    b->h_ni = halloc<int>(ncl, &b->d_ni);
    b->h_eps2 = halloc<double>(ncl, &b->d_eps2);
    b->h_t = halloc<double>(ncl, &b->d_t);
    b->h_hdr_each = halloc<long long>(2 * (size_t)ncl, &b->d_hdr_each);
    b->h_gts_each = halloc<long long>(gts_each, &b->d_gts_each);
    b->h_irec = halloc<g6x_irec>(slots_i, &b->d_irec);
    b->h_out = halloc<g6x_out>(slots_i, &b->d_out);
    b->h_toff = halloc<int>(tiles + 1, &b->d_toff);
    b->h_jsort = halloc<g6x_jrec>(slots_i, &b->d_jsort);
    b->jsort_cap = slots_i;
    b->h_err = halloc<int>(1, &b->d_err);
    if (!js.x0 || !js.xds || !js.xds2 || !js.t0 || !js.v0m || !js.a2f || !js.j6f || !js.v64
        || !js.a264 || !js.j664 || !js.idx || !b->pred.pt || !b->pred.trange
        || !b->d_tile_cluster || !b->d_cl_jtile || !b->d_cl_nj || !b->d_part || !b->h_hdr
        || !b->h_gts || !b->h_gtc || !b->h_gti || !b->h_ioff || !b->h_ni || !b->h_eps2
        || !b->h_t || !b->h_hdr_each || !b->h_gts_each || !b->h_irec || !b->h_out
        || !b->h_toff || !b->h_jsort || !b->h_err)
        rc = G6_ENOMEM;
    if (!rc) {
        try {
            b->slot_of.assign(n, -1);
            b->stage.reserve(1024);
        } catch (...) {
            rc = G6_ENOMEM;
        }
    }
    if (!rc && cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
        rc = G6_EIO;
    if (!rc) {
        std::vector<int> tc(tiles);
        for (int k = 0; k < ncl; ++k)
            for (int t = 0; t < b->ntile[k]; ++t)
                tc[b->jtile[k] + t] = k;
        *b->h_err = 0;
        for (int k = 0; k < ncl; ++k) {
            b->h_ioff[k] = b->ioff[k];
            b->h_ni[k] = 0;
            b->h_eps2[k] = 0.0;
            b->h_t[k] = 0.0;
        }
        for (int t = 0; t <= tiles; ++t)
            b->h_toff[t] = 0;
        b->h_hdr[0] = b->h_hdr[1] = 0;
        cudaError_t e = cudaMemcpyAsync(b->d_tile_cluster, tc.data(), sizeof(int) * tiles,
                                        cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_cl_jtile, b->jtile.data(), sizeof(int) * ncl,
                                cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_cl_nj, b->nj.data(), sizeof(int) * ncl,
                                cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess)
            e = g6::launch_init_store(js, b->stream);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(b->stream);
        rc = cuda_code(e);
        b->k3_blocks = std::max(1, std::min(b->sms * 16, (b->gt_cap * b->itile * 32 + 255) / 256));
    }
    if (rc) {
        free_batch(b);
        if (err)
            *err = rc;
        return nullptr;
    }
    return b;
}

int g6x_batch_destroy(g6x_batch *b)
{
    if (!b)
        return G6_EINVAL;
    free_batch(b);
    return 0;
}

g6x_irec *g6x_batch_irecs(g6x_batch *b, int cl)
{
    if (!b || cl < 0 || cl >= b->ncl)
        return nullptr;
    return b->h_irec + b->ioff[cl];
}

const g6x_out *g6x_batch_results(const g6x_batch *b, int cl)
{
    if (!b || cl < 0 || cl >= b->ncl)
        return nullptr;
    return b->h_out + b->ioff[cl];
}

int g6x_batch_set_j(g6x_batch *b, int cl, int address, int index, double tj, double mass,
                    const double j6[3], const double a2[3], const double v[3],
                    const double x[3])
{
    if (!b || cl < 0 || cl >= b->ncl || address < 0 || address >= b->nj[cl] || index < 0
        || !j6 || !a2 || !v || !x)
        return G6_EINVAL;
    const int slot = b->jtile[cl] * JT + address;
    int s = b->slot_of[slot];
    if (s < 0) {
        try {
            b->stage.emplace_back();
        } catch (...) {
            return G6_ENOMEM;
        }
        s = (int)b->stage.size() - 1;
        b->slot_of[slot] = s;
    }
    g6x_jrec &r = b->stage[s];
    for (int d = 0; d < 3; ++d) {
        r.x[d] = x[d];
        r.v[d] = v[d];
        r.a2[d] = a2[d];
        r.j6[d] = j6[d];
    }
    r.mass = mass;
    r.tj = tj;
    r.address = slot;
    r.index = index;
    return 0;
}

int g6x_batch_set_j_many(g6x_batch *b, int cl, int n, const int address[], const int index[],
                         const double tj[], const double mass[], const double j6[],
                         const double a2[], const double v[], const double x[])
{
    if (!b || cl < 0 || cl >= b->ncl || n < 0
        || (n > 0 && (!address || !index || !tj || !mass || !j6 || !a2 || !v || !x)))
        return G6_EINVAL;
    for (int q = 0; q < n; ++q)
        if (address[q] < 0 || address[q] >= b->nj[cl] || index[q] < 0)
            return G6_EINVAL;
    for (int q = 0; q < n; ++q) {
        const int rc = g6x_batch_set_j(b, cl, address[q], index[q], tj[q], mass[q], &j6[3 * q],
                                       &a2[3 * q], &v[3 * q], &x[3 * q]);
        if (rc)
            return rc;
    }
    return 0;
}

int g6x_batch_calc(g6x_batch *b, const double t_blk[], const double eps2[], const int ni[],
                   int mode)
{
    if (!b || !t_blk || !eps2 || !ni || mode < 0 || mode > 2)
        return G6_EINVAL;
    for (int k = 0; k < b->ncl; ++k)
        if (ni[k] < 0 || ni[k] > b->nj[k] || !(eps2[k] >= 0) || !std::isfinite(t_blk[k]))
            return G6_EINVAL;
    int rc = stage_sorted(b);
    if (rc)
        return rc;
    // per-step tables: one global work line over the active clusters
    long long W = 0;
    int g = 0;
    for (int k = 0; k < b->ncl; ++k) {
        b->h_ni[k] = ni[k];
        b->h_eps2[k] = eps2[k];
        b->h_t[k] = t_blk[k];
        b->gt_first[k] = g;
        const int nit = (ni[k] + b->itile - 1) / b->itile;
        long long Wk = 0;
        long long *ge = b->h_gts_each + b->gts_each_off[k];
        for (int t = 0; t < nit; ++t, ++g) {
            b->h_gts[g] = W;
            b->h_gtc[g] = k;
            b->h_gti[g] = t;
            ge[t] = Wk;
            W += b->ntile[k];
            Wk += b->ntile[k];
        }
        ge[nit] = Wk;
        b->h_hdr_each[2 * k] = Wk;
        b->h_hdr_each[2 * k + 1] = nit;
    }
    b->h_gts[g] = W;
    b->h_hdr[0] = W;
    b->h_hdr[1] = g;
    cudaError_t e = cudaSuccess;
    if (mode == 0) {
        if (!b->gexec) {
            cudaGraph_t gr = nullptr;
            e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t e2 = enqueue_all(b);
                e = cudaStreamEndCapture(b->stream, &gr);
                if (e2 != cudaSuccess)
                    e = e2;
            }
            if (e == cudaSuccess)
                e = cudaGraphInstantiate(&b->gexec, gr, 0);
            if (e == cudaSuccess)
                b->graph = gr;
            else if (gr)
                cudaGraphDestroy(gr);
        }
        if (e == cudaSuccess)
            e = cudaGraphLaunch(b->gexec, b->stream);
        b->launches += 3;
    } else if (mode == 1) {
        e = enqueue_all(b);
        b->launches += 3;
    } else {
        // one launch sequence per active cluster
        for (int k = 0; k < b->ncl && e == cudaSuccess; ++k) {
            if (ni[k] == 0)
                continue;
            e = g6::launch_predict_batch(pred_kind(b), b->js, b->pred, pred_tables(b), b->d_jsort,
                                         b->d_toff, b->jtile[k], b->ntile[k], b->sms, b->stream);
            const int g0 = b->gt_first[k];
            const g6::BatchTables bt =
                force_tables(b, b->d_hdr_each + 2 * k, b->d_gts_each + b->gts_each_off[k],
                             b->d_gtc + g0, b->d_gti + g0);
            const int nit = (ni[k] + b->itile - 1) / b->itile;
            const int grid = (int)std::min<long long>(b->grid, (long long)nit * b->ntile[k]);
            if (e == cudaSuccess)
                e = g6::launch_force_batch(b->variant, grid, b->pred, b->d_irec, b->d_part,
                                           b->d_err, bt, b->stream);
            if (e == cudaSuccess)
                e = g6::launch_reduce_batch(b->variant, grid, b->d_part, b->js.idx, b->d_out, bt,
                                            std::max(1, (nit * b->itile * 32 + 255) / 256),
                                            b->stream);
            b->launches += 3;
        }
        // records of idle clusters still have to reach j-memory
        if (e == cudaSuccess)
            for (int k = 0; k < b->ncl && e == cudaSuccess; ++k)
                if (ni[k] == 0 && b->h_toff[b->jtile[k] + b->ntile[k]] > b->h_toff[b->jtile[k]])
                    e = g6::launch_predict_batch(pred_kind(b), b->js, b->pred, pred_tables(b),
                                                 b->d_jsort, b->d_toff, b->jtile[k],
                                                 b->ntile[k], b->sms, b->stream);
    }
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess)
        return cuda_code(e);
    // the staged records were consumed: clear the per-tile ranges
    for (int t = 0; t <= b->total_tiles; ++t)
        b->h_toff[t] = 0;
    if (*(volatile int *)b->h_err) {
        const int code = *b->h_err;
        *(volatile int *)b->h_err = 0;
        return code < 0 ? code : G6_EIO;
    }
    return 0;
}

long long g6x_batch_launch_count(const g6x_batch *b) { return b ? b->launches : 0; }

}  // extern "C"

// ------------------------------------------------------------ batch driver

struct g6hb_sim {
    g6x_batch *b = nullptr;
    int ncl = 0, mode = 0;
    double eta = 0, eta_s = 0, dt_max = 0, dt_min = 0;
    std::vector<int> n, off;                 // particles per cluster, offset into arrays
    std::vector<double> eps2;
    std::vector<double> m, x, v, a, j, t, dt;
    std::vector<std::map<double, std::vector<int>>> due;
    std::vector<std::vector<int>> act;
    std::vector<double> tblk;
    std::vector<int> ni;
    std::vector<double> xp, vp;               // predicted i (per particle slot)
    long long nsteps = 0, nactive = 0, interactions = 0;
    double sec_gpu = 0, sec_host = 0;
};

namespace {

double nrm(const double *p) { return std::sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]); }

int hb_send(g6hb_sim &s, int k, int q)
{
    const int p = s.off[k] + q;
    double a2[3], j6[3];
    for (int d = 0; d < 3; ++d) {
        a2[d] = 0.5 * s.a[3 * p + d];
        j6[d] = s.j[3 * p + d] / 6.0;
    }
    return g6x_batch_set_j(s.b, k, q, q, s.t[p], s.m[p], j6, a2, &s.v[3 * p], &s.x[3 * p]);
}

}  // namespace

extern "C" {

g6hb_sim *g6hb_create(int ncl, const int n[], const double *m, const double *x,
                      const double *v, const double eps2[], double eta, double eta_s,
                      double dt_max, double dt_min, int variant, int grid_mul, int mode,
                      int *err)
{
    if (err)
        *err = 0;
    if (ncl < 1 || !n || !m || !x || !v || !eps2 || !(eta > 0) || !(dt_max > 0)
        || !(dt_min > 0) || mode < 0 || mode > 2) {
        if (err)
            *err = G6_EINVAL;
        return nullptr;
    }
    g6hb_sim *s = new (std::nothrow) g6hb_sim();
    if (!s) {
        if (err)
            *err = G6_ENOMEM;
        return nullptr;
    }
    int rc = 0;
    s->b = g6x_batch_create(ncl, n, G6X_PREC_DS, variant, grid_mul, &rc);
    if (!s->b) {
        delete s;
        if (err)
            *err = rc;
        return nullptr;
    }
    s->ncl = ncl;
    s->mode = mode;
    s->eta = eta;
    s->eta_s = eta_s > 0 ? eta_s : eta / 10.0;
    s->dt_max = dt_max;
    s->dt_min = dt_min;
    int tot = 0;
    try {
        s->n.assign(n, n + ncl);
        s->off.resize(ncl);
        for (int k = 0; k < ncl; ++k) {
            s->off[k] = tot;
            tot += n[k];
        }
        s->eps2.assign(eps2, eps2 + ncl);
        s->m.assign(m, m + tot);
        s->x.assign(x, x + 3 * (size_t)tot);
        s->v.assign(v, v + 3 * (size_t)tot);
        s->a.assign(3 * (size_t)tot, 0.0);
        s->j.assign(3 * (size_t)tot, 0.0);
        s->t.assign(tot, 0.0);
        s->dt.assign(tot, dt_max);
        s->due.resize(ncl);
        s->act.resize(ncl);
        s->tblk.assign(ncl, 0.0);
        s->ni.assign(ncl, 0);
        s->xp.resize(3 * (size_t)tot);
        s->vp.resize(3 * (size_t)tot);
    } catch (...) {
        g6x_batch_destroy(s->b);
        delete s;
        if (err)
            *err = G6_ENOMEM;
        return nullptr;
    }
    // initial force: every particle of every cluster active at t = 0
    for (int k = 0; !rc && k < ncl; ++k)
        for (int q = 0; !rc && q < n[k]; ++q)
            rc = hb_send(*s, k, q);
    for (int k = 0; !rc && k < ncl; ++k) {
        g6x_irec *ir = g6x_batch_irecs(s->b, k);
        for (int q = 0; q < n[k]; ++q) {
            const int p = s->off[k] + q;
            for (int d = 0; d < 3; ++d) {
                ir[q].x[d] = s->x[3 * p + d];
                ir[q].v[d] = s->v[3 * p + d];
            }
            ir[q].h2 = 0.0;
            ir[q].index = q;
            ir[q].pad = 0;
        }
        s->ni[k] = n[k];
    }
    if (!rc)
        rc = g6x_batch_calc(s->b, s->tblk.data(), s->eps2.data(), s->ni.data(), mode);
    for (int k = 0; !rc && k < ncl; ++k) {
        const g6x_out *o = g6x_batch_results(s->b, k);
        for (int q = 0; q < n[k]; ++q) {
            const int p = s->off[k] + q;
            for (int d = 0; d < 3; ++d) {
                s->a[3 * p + d] = o[q].acc[d];
                s->j[3 * p + d] = o[q].jerk[d];
            }
            const double req = s->eta_s * nrm(&s->a[3 * p]) / nrm(&s->j[3 * p]);
            double d = dt_max;
            while (d > req)
                d *= 0.5;
            if (d < s->dt_min)
                rc = G6_EINVAL;
            s->dt[p] = d;
            s->due[k][d].push_back(q);
        }
    }
    for (int k = 0; !rc && k < ncl; ++k)
        for (int q = 0; !rc && q < n[k]; ++q)
            rc = hb_send(*s, k, q);
    if (rc) {
        g6x_batch_destroy(s->b);
        delete s;
        if (err)
            *err = rc;
        return nullptr;
    }
    return s;
}

// One batch step: every cluster that has not reached t_end takes its next
// block step.  Returns the number of clusters that stepped (0: all done).
int g6hb_step(g6hb_sim *s, double t_end)
{
    if (!s)
        return G6_EINVAL;
    auto w0 = std::chrono::steady_clock::now();
    int stepping = 0;
    for (int k = 0; k < s->ncl; ++k) {
        s->ni[k] = 0;
        if (s->due[k].empty())
            continue;
        auto first = s->due[k].begin();
        if (first->first > t_end)
            continue;
        const double tb = first->first;
        s->tblk[k] = tb;
        s->act[k].swap(first->second);
        s->due[k].erase(first);
        g6x_irec *ir = g6x_batch_irecs(s->b, k);
        const int na = (int)s->act[k].size();
        for (int i = 0; i < na; ++i) {
            const int q = s->act[k][i];
            const int p = s->off[k] + q;
            const double h = tb - s->t[p];
            for (int d = 0; d < 3; ++d) {
                const double aa = s->a[3 * p + d], jj = s->j[3 * p + d];
                s->xp[3 * p + d] = s->x[3 * p + d]
                                   + h * (s->v[3 * p + d] + h * (aa / 2.0 + h * jj / 6.0));
                s->vp[3 * p + d] = s->v[3 * p + d] + h * (aa + h * jj / 2.0);
                ir[i].x[d] = s->xp[3 * p + d];
                ir[i].v[d] = s->vp[3 * p + d];
            }
            ir[i].h2 = 0.0;
            ir[i].index = q;
            ir[i].pad = 0;
        }
        s->ni[k] = na;
        s->interactions += (long long)na * s->n[k];
        s->nactive += na;
        ++stepping;
    }
    if (stepping == 0)
        return 0;
    auto w1 = std::chrono::steady_clock::now();
    int rc = g6x_batch_calc(s->b, s->tblk.data(), s->eps2.data(), s->ni.data(), s->mode);
    if (rc)
        return rc;
    auto w2 = std::chrono::steady_clock::now();
    for (int k = 0; k < s->ncl; ++k) {
        if (s->ni[k] == 0)
            continue;
        const g6x_out *o = g6x_batch_results(s->b, k);
        const double tb = s->tblk[k];
        std::vector<int> *last = nullptr;
        double last_t = 0.0;
        for (int i = 0; i < s->ni[k]; ++i) {
            const int q = s->act[k][i];
            const int p = s->off[k] + q;
            double t0[1] = {s->t[p]}, dtv[1] = {s->dt[p]}, dn[1];
            rc = g6h_correct_block(1, tb, t0, dtv, s->eta, s->dt_max, s->dt_min, &s->xp[3 * p],
                                   &s->vp[3 * p], &s->a[3 * p], &s->j[3 * p], o[i].acc,
                                   o[i].jerk, dn);
            if (rc != 0)
                return rc < 0 ? rc : G6_EINVAL;
            for (int d = 0; d < 3; ++d) {
                s->x[3 * p + d] = s->xp[3 * p + d];
                s->v[3 * p + d] = s->vp[3 * p + d];
                s->a[3 * p + d] = o[i].acc[d];
                s->j[3 * p + d] = o[i].jerk[d];
            }
            s->t[p] = tb;
            s->dt[p] = dn[0];
            rc = hb_send(*s, k, q);
            if (rc)
                return rc;
            const double tn = tb + dn[0];
            if (!last || tn != last_t) {
                last = &s->due[k][tn];
                last_t = tn;
            }
            last->push_back(q);
        }
        s->act[k].clear();
    }
    auto w3 = std::chrono::steady_clock::now();
    s->sec_host += std::chrono::duration<double>(w1 - w0).count()
                   + std::chrono::duration<double>(w3 - w2).count();
    s->sec_gpu += std::chrono::duration<double>(w2 - w1).count();
    ++s->nsteps;
    return stepping;
}

int g6hb_run(g6hb_sim *s, double t_end)
{
    if (!s || !(t_end >= 0) || std::fmod(t_end, s->dt_max) != 0.0)
        return G6_EINVAL;
    for (;;) {
        const int r = g6hb_step(s, t_end);
        if (r < 0)
            return r;
        if (r == 0)
            return 0;
    }
}

int g6hb_stats(const g6hb_sim *s, long long *nsteps, long long *nactive,
               long long *interactions, double *sec_gpu, double *sec_host)
{
    if (!s)
        return G6_EINVAL;
    if (nsteps)
        *nsteps = s->nsteps;
    if (nactive)
        *nactive = s->nactive;
    if (interactions)
        *interactions = s->interactions;
    if (sec_gpu)
        *sec_gpu = s->sec_gpu;
    if (sec_host)
        *sec_host = s->sec_host;
    return 0;
}

int g6hb_get_state(const g6hb_sim *s, double *x, double *v, double *t)
{
    if (!s)
        return G6_EINVAL;
    const size_t tot = s->m.size();
    if (x)
        std::memcpy(x, s->x.data(), 3 * tot * sizeof(double));
    if (v)
        std::memcpy(v, s->v.data(), 3 * tot * sizeof(double));
    if (t)
        std::memcpy(t, s->t.data(), tot * sizeof(double));
    return 0;
}

int g6hb_set_mode(g6hb_sim *s, int mode)
{
    if (!s || mode < 0 || mode > 2)
        return G6_EINVAL;
    s->mode = mode;
    return 0;
}

void g6hb_destroy(g6hb_sim *s)
{
    if (!s)
        return;
    g6x_batch_destroy(s->b);
    delete s;
}

}  // extern "C"
