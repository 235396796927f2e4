// g6gb_batch.cu -- many independent clusters in one launch sequence.
//
// A batch holds the j-memory of every cluster (each cluster at a JT-aligned
// range of slots).  One batch calculation gives every cluster its own block
// time and active set (Sect. 2, Sect. 2.1: block time steps, O(nm) force per
// block) and computes all of them in one launch sequence -- one copy of the
// step's geometry tables to the device, the j-store update fused into the
// per-cluster prediction (Eq. 1, Eq. 2), the force kernels, and the
// reductions (an i-tile whose work spans a few CTAs is reduced by the last of
// them inside the force launch, the others by the reduction kernel, which
// skips the former).  The kernels read the geometry from device memory, so the
// sequence is captured once in a CUDA graph and replayed every step (only
// the size of the table copy is updated before a replay).  For comparison
// the same kernels can run as plain launches or as one launch sequence per
// cluster.
//
// Schedule.  The i-particles of a cluster are cut into i-tiles of the force
// kernel's width, and every (i-tile, j-tile) pair of every cluster is one
// unit of one work line cut evenly over a fixed grid.  Clusters whose active
// set is small waste most of a wide i-tile, so a schedule may have two work
// classes: active sets of at most `threshold` particles go to a narrow
// kernel, the rest to a wide one; the two force kernels run concurrently
// (forked streams inside the graph).  g6x_batch_autotune times candidate
// schedules on given active-set patterns and keeps the fastest.
//
// The C++ batch driver (g6hb_*) runs a Hermite block-time-step integration in
// every cluster with its own block scheduler, advancing each cluster by one
// of its own block steps per batch step; the per-cluster host work (i
// prediction, correction, staging) runs on the library's host threads.
#include "g6gb_internal.h"
#include "g6gb_pool.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <cmath>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

using g6::BatchGT;
using g6::JT;

namespace {

// A staged j-record whose default construction leaves it uninitialised: a
// block's records are reserved in one resize and every field is written
// right after, so the reservation costs no zeroing.
struct StagedRec : g6x_jrec {
    StagedRec() {}
};

// One work class of a schedule: its force kernel, grid and partial sums.
struct WorkClass {
    int variant = -1, grid_mul = 1, grid = 0, itile = 0, gt_cap = 0, k3_blocks = 1;
    void *d_part = nullptr;
    unsigned *d_cnt = nullptr;     // per entry of the line: arrivals (inside d_part's block)
};

constexpr size_t HDR_WORDS = 4;     // per work line: W, entries, first entry, unused

}  // namespace

struct g6x_batch {
    int ncl = 0, pmode = G6X_PREC_DS, sms = 0;
    cudaStream_t stream = nullptr, stream2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
    std::vector<int> nj, jtile, ntile, ioff;
    int total_tiles = 0, total_slots = 0, total_i = 0;
    g6::JStore js{};
    g6::Pred pred{};
    int *d_tile_cluster = nullptr, *d_cl_jtile = nullptr, *d_cl_nj = nullptr;
    // Per-step geometry: one pinned host block, copied (used prefix) to its
    // device mirror at the head of every step.  Layout: ni[ncl] ioff[ncl]
    // eps2[ncl] t[ncl] toff[tiles + 1] | hdr[hdr_cap][4] | gt[gt_cap_all].
    unsigned char *h_tab = nullptr, *d_tab = nullptr;
    size_t tab_bytes = 0, tab_used = 0;
    int hdr_cap = 0, gt_cap_all = 0;
    int *h_ni = nullptr, *h_ioff = nullptr, *h_toff = nullptr;
    double *h_eps2 = nullptr, *h_t = nullptr;
    long long *h_hdr = nullptr;
    BatchGT *h_gt = nullptr;
    int *d_ni = nullptr, *d_ioff = nullptr, *d_toff = nullptr;
    double *d_eps2 = nullptr, *d_t = nullptr;
    long long *d_hdr = nullptr;
    BatchGT *d_gt = nullptr;
    // schedule
    WorkClass wc[2];
    int nclass = 1, threshold = INT_MAX;
    g6x_irec *h_irec = nullptr, *d_irec = nullptr;
    g6x_out *h_out = nullptr, *d_out = nullptr;
    // j staging: per cluster, at most one record per slot; sorted by tile
    // into the mapped buffer at launch
    std::vector<std::vector<StagedRec>> stage;
    std::vector<int> slot_of;
    std::vector<int> base;
    g6x_jrec *h_jsort = nullptr, *d_jsort = nullptr;
    int *h_err = nullptr, *d_err = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaGraphNode_t copy_node = nullptr;
    long long launches = 0;
    bool timing = false;
    double gpu_ms = 0.0;
    long long timed = 0;
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

void drop_graph(g6x_batch *b)
{
    if (b->gexec)
        cudaGraphExecDestroy(b->gexec);
    if (b->graph)
        cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
    b->copy_node = nullptr;
}

void free_class(WorkClass &w)
{
    g6::dev_free_hooked(w.d_part);
    w = WorkClass();
}

void free_tables(g6x_batch *b)
{
    g6::host_free_pinned(b->h_tab);
    g6::dev_free_hooked(b->d_tab);
    b->h_tab = b->d_tab = nullptr;
    b->tab_bytes = 0;
}

void free_batch(g6x_batch *b)
{
    if (b->stream)
        cudaStreamSynchronize(b->stream);
    if (b->stream2)
        cudaStreamSynchronize(b->stream2);
    drop_graph(b);
    g6::JStore &js = b->js;
    void *dp[] = {js.x0, js.raw, js.v64, js.a264,
                  js.j664, js.idx, b->pred.pt, b->pred.trange, b->pred.p64, b->pred.v64,
                  b->d_tile_cluster, b->d_cl_jtile, b->d_cl_nj};
    for (void *p : dp)
        g6::dev_free_hooked(p);
    for (WorkClass &w : b->wc)
        free_class(w);
    free_tables(b);
    void *hp[] = {b->h_irec, b->h_out, b->h_jsort, b->h_err};
    for (void *p : hp)
        g6::host_free_pinned(p);
    cudaEvent_t ev[] = {b->ev_fork, b->ev_join, b->ev_t0, b->ev_t1};
    for (cudaEvent_t e : ev)
        if (e)
            cudaEventDestroy(e);
    if (b->stream)
        cudaStreamDestroy(b->stream);
    if (b->stream2)
        cudaStreamDestroy(b->stream2);
    delete b;
}

bool valid_variant(int v) { return v >= 0 && v < g6::batch_variant_count(); }

// (Re)build work class c for batch variant v and grid multiplier gm.
int setup_class(g6x_batch *b, int c, int v, int gm)
{
    WorkClass &w = b->wc[c];
    free_class(w);
    const g6::VariantInfo vi = g6::batch_variant_info(v);
    const int occ = g6::batch_variant_occupancy(v);
    if (occ < 1)
        return G6_ENODEV;
    w.variant = v;
    w.grid_mul = gm;
    w.itile = vi.ti * vi.nper;
    w.grid = b->sms * occ * gm;
    w.gt_cap = 0;
    for (int k = 0; k < b->ncl; ++k)
        w.gt_cap += (b->nj[k] + w.itile - 1) / w.itile;
    w.k3_blocks = std::max(1, std::min(b->sms * 16, (w.gt_cap * w.itile * 32 + 255) / 256));
    // the partial records, then one arrival counter per entry (zero between
    // launches: the CTA that completes a count resets it)
    const size_t pbytes = (size_t)(w.grid + w.gt_cap) * w.itile * g6::PARTIAL_BYTES;
    w.d_part = g6::dev_alloc_hooked(pbytes + (size_t)w.gt_cap * sizeof(unsigned));
    if (!w.d_part) {
        free_class(w);
        return G6_ENOMEM;
    }
    w.d_cnt = reinterpret_cast<unsigned *>(static_cast<char *>(w.d_part) + pbytes);
    if (cudaMemset(w.d_cnt, 0, (size_t)w.gt_cap * sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        free_class(w);
        return G6_EIO;
    }
    return 0;
}

size_t align8(size_t n) { return (n + 7) & ~(size_t)7; }

// (Re)allocate the geometry block for the current schedule: entries for
// both class lines (plus sentinels) or for one line per cluster.
int setup_tables(g6x_batch *b)
{
    free_tables(b);
    int it_min = b->wc[0].itile;
    if (b->nclass == 2)
        it_min = std::min(it_min, b->wc[1].itile);
    long long per_cluster = 0;
    for (int k = 0; k < b->ncl; ++k)
        per_cluster += (b->nj[k] + it_min - 1) / it_min + 1;
    const long long classes = (long long)b->wc[0].gt_cap + 1
                              + (b->nclass == 2 ? b->wc[1].gt_cap + 1 : 0);
    b->gt_cap_all = (int)std::max(per_cluster, classes);
    b->hdr_cap = std::max(2, b->ncl);
    const size_t n = (size_t)b->ncl;
    size_t o = 0;
    const size_t o_ni = o;
    o = align8(o + n * sizeof(int));
    const size_t o_ioff = o;
    o = align8(o + n * sizeof(int));
    const size_t o_eps2 = o;
    o += n * sizeof(double);
    const size_t o_t = o;
    o += n * sizeof(double);
    const size_t o_toff = o;
    o = align8(o + (b->total_tiles + 1) * sizeof(int));
    const size_t o_hdr = o;
    o += (size_t)b->hdr_cap * HDR_WORDS * sizeof(long long);
    const size_t o_gt = o;
    o += (size_t)b->gt_cap_all * sizeof(BatchGT);
    b->tab_bytes = o;
    void *dev_alias = nullptr;
    b->h_tab = static_cast<unsigned char *>(g6::host_alloc_zero_copy(o, &dev_alias));
    b->d_tab = static_cast<unsigned char *>(g6::dev_alloc_hooked(o));
    if (!b->h_tab || !b->d_tab) {
        free_tables(b);
        return G6_ENOMEM;
    }
    std::memset(b->h_tab, 0, o);
    unsigned char *h = b->h_tab, *d = b->d_tab;
    b->h_ni = reinterpret_cast<int *>(h + o_ni);
    b->d_ni = reinterpret_cast<int *>(d + o_ni);
    b->h_ioff = reinterpret_cast<int *>(h + o_ioff);
    b->d_ioff = reinterpret_cast<int *>(d + o_ioff);
    b->h_eps2 = reinterpret_cast<double *>(h + o_eps2);
    b->d_eps2 = reinterpret_cast<double *>(d + o_eps2);
    b->h_t = reinterpret_cast<double *>(h + o_t);
    b->d_t = reinterpret_cast<double *>(d + o_t);
    b->h_toff = reinterpret_cast<int *>(h + o_toff);
    b->d_toff = reinterpret_cast<int *>(d + o_toff);
    b->h_hdr = reinterpret_cast<long long *>(h + o_hdr);
    b->d_hdr = reinterpret_cast<long long *>(d + o_hdr);
    b->h_gt = reinterpret_cast<BatchGT *>(h + o_gt);
    b->d_gt = reinterpret_cast<BatchGT *>(d + o_gt);
    for (int k = 0; k < b->ncl; ++k)
        b->h_ioff[k] = b->ioff[k];
    b->tab_used = o_gt;
    return 0;
}

int set_schedule(g6x_batch *b, int v0, int gm0, int threshold, int v1, int gm1)
{
    if (!valid_variant(v0) || gm0 < 1 || gm0 > 16
        || (v1 >= 0 && (!valid_variant(v1) || gm1 < 1 || gm1 > 16 || threshold < 1)))
        return G6_EINVAL;
    cudaStreamSynchronize(b->stream);
    cudaStreamSynchronize(b->stream2);
    drop_graph(b);
    int rc = setup_class(b, 0, v0, gm0);
    if (!rc && v1 >= 0) {
        rc = setup_class(b, 1, v1, gm1);
        b->nclass = 2;
        b->threshold = threshold;
    } else {
        free_class(b->wc[1]);
        b->nclass = 1;
        b->threshold = INT_MAX;
    }
    if (!rc)
        rc = setup_tables(b);
    return rc;
}

// Sort the staged records by tile into the mapped buffer; toff gets the
// per-tile ranges (all equal when nothing is staged).
void stage_sorted(g6x_batch *b)
{
    int total = 0;
    for (int k = 0; k < b->ncl; ++k) {
        b->base[k] = total;
        total += (int)b->stage[k].size();
    }
    g6::parallel_run(b->ncl, [b](int k) {
        const int t0 = b->jtile[k], nt = b->ntile[k];
        int *off = b->h_toff + t0;
        std::vector<StagedRec> &st = b->stage[k];
        if (st.empty()) {
            for (int t = 0; t < nt; ++t)
                off[t] = b->base[k];
            return;
        }
        // counting sort by tile within the cluster's tile range (one count
        // buffer per host thread, kept between calls)
        thread_local std::vector<int> cnt;
        cnt.assign(nt + 1, 0);
        for (const g6x_jrec &r : st)
            ++cnt[r.address / JT - t0 + 1];
        int acc = b->base[k];
        for (int t = 0; t < nt; ++t) {
            off[t] = acc;
            acc += cnt[t + 1];
            cnt[t + 1] = off[t];
        }
        for (const g6x_jrec &r : st) {
            b->h_jsort[cnt[r.address / JT - t0 + 1]++] = r;
            b->slot_of[r.address] = -1;
        }
        st.clear();
    });
    b->h_toff[b->total_tiles] = total;
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

// Tables of work line `line` (header index).
g6::BatchTables line_tables(const g6x_batch *b, int line)
{
    g6::BatchTables bt;
    bt.hdr = b->d_hdr + (size_t)line * HDR_WORDS;
    bt.gt = b->d_gt;
    bt.cl_jtile = b->d_cl_jtile;
    bt.cl_ioff = b->d_ioff;
    bt.cl_ni = b->d_ni;
    bt.cl_eps2 = b->d_eps2;
    return bt;
}

cudaError_t enqueue_class(g6x_batch *b, int c, cudaStream_t s)
{
    const WorkClass &w = b->wc[c];
    const g6::BatchTables bt = line_tables(b, c);
    cudaError_t e = g6::launch_force_batch(w.variant, w.grid, b->pred, b->d_irec, w.d_part,
                                           b->d_err, bt, s, w.d_cnt, b->d_out, b->js.idx);
    if (e == cudaSuccess)
        e = g6::launch_reduce_batch(w.variant, w.grid, w.d_part, b->js.idx, b->d_out, bt,
                                    w.k3_blocks, s, true);
    return e;
}

cudaError_t enqueue_copy(g6x_batch *b)
{
    return cudaMemcpyAsync(b->d_tab, b->h_tab, b->tab_used, cudaMemcpyHostToDevice, b->stream);
}

// The whole step over every cluster: tables, update + predict, then the work
// classes (the second on a forked stream), joined back on the main stream.
cudaError_t enqueue_all(g6x_batch *b)
{
    cudaError_t e = enqueue_copy(b);
    if (e == cudaSuccess)
        e = g6::launch_predict_batch(pred_kind(b), b->js, b->pred, pred_tables(b), b->d_jsort,
                                     b->d_toff, 0, b->total_tiles, b->sms, b->stream);
    if (e == cudaSuccess && b->nclass == 2) {
        e = cudaEventRecord(b->ev_fork, b->stream);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(b->stream2, b->ev_fork, 0);
        if (e == cudaSuccess)
            e = enqueue_class(b, 1, b->stream2);
        if (e == cudaSuccess)
            e = cudaEventRecord(b->ev_join, b->stream2);
    }
    if (e == cudaSuccess)
        e = enqueue_class(b, 0, b->stream);
    if (e == cudaSuccess && b->nclass == 2)
        e = cudaStreamWaitEvent(b->stream, b->ev_join, 0);
    return e;
}

int class_of(const g6x_batch *b, int ni) { return b->nclass == 2 && ni > b->threshold ? 1 : 0; }

// Append the entries of cluster k's active i-tiles to a line whose work so
// far is W; returns the new entry count.
int append_cluster(g6x_batch *b, int k, int nit, int g, long long &W)
{
    for (int t = 0; t < nit; ++t, ++g) {
        b->h_gt[g].start = W;
        b->h_gt[g].cluster = k;
        b->h_gt[g].itile = t;
        W += b->ntile[k];
    }
    return g;
}

void close_line(g6x_batch *b, int line, int first, int g, long long W)
{
    b->h_gt[g].start = W;                           // sentinel
    b->h_gt[g].cluster = 0;
    b->h_gt[g].itile = 0;
    long long *h = b->h_hdr + (size_t)line * HDR_WORDS;
    h[0] = W;
    h[1] = g - first;
    h[2] = first;
    h[3] = 0;
}

// Per-step work lines: one per class (graph and plain modes).
void build_class_lines(g6x_batch *b, const int ni[])
{
    int g = 0;
    for (int c = 0; c < b->nclass; ++c) {
        const int first = g;
        const int it = b->wc[c].itile;
        long long W = 0;
        for (int k = 0; k < b->ncl; ++k)
            if (ni[k] > 0 && class_of(b, ni[k]) == c)
                g = append_cluster(b, k, (ni[k] + it - 1) / it, g, W);
        close_line(b, c, first, g, W);
        ++g;
    }
    b->tab_used = (size_t)((unsigned char *)(b->h_gt + g) - b->h_tab);
}

// Per-step work lines: one per active cluster (per-cluster mode).
void build_cluster_lines(g6x_batch *b, const int ni[])
{
    int g = 0;
    for (int k = 0; k < b->ncl; ++k) {
        if (ni[k] == 0)
            continue;
        const int first = g;
        const int it = b->wc[class_of(b, ni[k])].itile;
        long long W = 0;
        g = append_cluster(b, k, (ni[k] + it - 1) / it, g, W);
        close_line(b, k, first, g, W);
        ++g;
    }
    b->tab_used = (size_t)((unsigned char *)(b->h_gt + g) - b->h_tab);
}

// Find the table copy among the nodes of the captured graph.
cudaError_t find_copy_node(g6x_batch *b)
{
    size_t n = 0;
    cudaError_t e = cudaGraphGetNodes(b->graph, nullptr, &n);
    if (e != cudaSuccess)
        return e;
    std::vector<cudaGraphNode_t> nodes(n);
    e = cudaGraphGetNodes(b->graph, nodes.data(), &n);
    for (size_t i = 0; e == cudaSuccess && i < n; ++i) {
        cudaGraphNodeType ty;
        e = cudaGraphNodeGetType(nodes[i], &ty);
        if (e == cudaSuccess && ty == cudaGraphNodeTypeMemcpy) {
            b->copy_node = nodes[i];
            return cudaSuccess;
        }
    }
    return e == cudaSuccess ? cudaErrorInvalidValue : e;
}

int run_graph(g6x_batch *b)
{
    cudaError_t e = cudaSuccess;
    if (!b->gexec) {
        cudaGraph_t gr = nullptr;
        e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t e2 = enqueue_all(b);
            e = cudaStreamEndCapture(b->stream, &gr);
            if (e2 != cudaSuccess)
                e = e2;
        }
        if (e == cudaSuccess)
            e = cudaGraphInstantiate(&b->gexec, gr, 0);
        if (e == cudaSuccess) {
            b->graph = gr;
            e = find_copy_node(b);
            if (e != cudaSuccess)
                drop_graph(b);
        } else if (gr) {
            cudaGraphDestroy(gr);
        }
    }
    // the copy moves only this step's part of the table block
    if (e == cudaSuccess)
        e = cudaGraphExecMemcpyNodeSetParams1D(b->gexec, b->copy_node, b->d_tab, b->h_tab,
                                               b->tab_used, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaGraphLaunch(b->gexec, b->stream);
    b->launches += 1 + 2 * b->nclass;
    return cuda_code(e);
}

int run_per_cluster(g6x_batch *b, const int ni[])
{
    cudaError_t e = enqueue_copy(b);
    for (int k = 0; k < b->ncl && e == cudaSuccess; ++k) {
        const bool staged = b->h_toff[b->jtile[k] + b->ntile[k]] > b->h_toff[b->jtile[k]];
        if (ni[k] == 0) {
            // records of an idle cluster still have to reach j-memory
            if (staged) {
                e = g6::launch_predict_batch(pred_kind(b), b->js, b->pred, pred_tables(b),
                                             b->d_jsort, b->d_toff, b->jtile[k], b->ntile[k],
                                             b->sms, b->stream);
                ++b->launches;
            }
            continue;
        }
        const WorkClass &w = b->wc[class_of(b, ni[k])];
        e = g6::launch_predict_batch(pred_kind(b), b->js, b->pred, pred_tables(b), b->d_jsort,
                                     b->d_toff, b->jtile[k], b->ntile[k], b->sms, b->stream);
        const int nit = (ni[k] + w.itile - 1) / w.itile;
        const g6::BatchTables bt = line_tables(b, k);
        const int grid = (int)std::min<long long>(w.grid, (long long)nit * b->ntile[k]);
        if (e == cudaSuccess)
            e = g6::launch_force_batch(w.variant, grid, b->pred, b->d_irec, w.d_part, b->d_err,
                                       bt, b->stream, w.d_cnt, b->d_out, b->js.idx);
        if (e == cudaSuccess)
            e = g6::launch_reduce_batch(w.variant, grid, w.d_part, b->js.idx, b->d_out, bt,
                                        std::max(1, (nit * w.itile * 32 + 255) / 256),
                                        b->stream, true);
        b->launches += 3;
    }
    return cuda_code(e);
}

}  // namespace

extern "C" {

g6x_batch *g6x_batch_create(int ncl, const int nj[], int precision, int variant, int grid_mul,
                            int *err)
{
    if (err)
        *err = 0;
    if (ncl < 1 || !nj || (precision != G6X_PREC_DS && precision != G6X_PREC_DS_X64)
        || variant < -1 || variant >= g6::batch_variant_count() || grid_mul < 0
        || grid_mul > 16) {
        if (err)
            *err = G6_EINVAL;
        return nullptr;
    }
    for (int k = 0; k < ncl; ++k)
        if (nj[k] < 1) {
            if (err)
                *err = G6_EINVAL;
            return nullptr;
        }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess
        || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess
        || sms < 1 || g6::batch_variant_occupancy(0) < 1) {
        cudaGetLastError();
        if (err)
            *err = G6_ENODEV;
        return nullptr;
    }
    g6x_batch *b = new (std::nothrow) g6x_batch();
    if (!b) {
        if (err)
            *err = G6_ENOMEM;
        return nullptr;
    }
    int rc = 0;
    b->sms = sms;
    b->ncl = ncl;
    b->pmode = precision;
    try {
        b->nj.assign(nj, nj + ncl);
        b->jtile.resize(ncl);
        b->ntile.resize(ncl);
        b->ioff.resize(ncl);
        b->base.resize(ncl);
        b->stage.resize(ncl);
    } catch (...) {
        free_batch(b);
        if (err)
            *err = G6_ENOMEM;
        return nullptr;
    }
    int tiles = 0, slots_i = 0;
    for (int k = 0; k < ncl; ++k) {
        b->jtile[k] = tiles;
        b->ntile[k] = (nj[k] + JT - 1) / JT;
        tiles += b->ntile[k];
        b->ioff[k] = slots_i;
        slots_i += nj[k];
    }
    b->total_tiles = tiles;
    b->total_slots = tiles * JT;
    b->total_i = slots_i;
    const size_t n = (size_t)b->total_slots;
    g6::JStore &js = b->js;
    js.cap = b->total_slots;
    js.x0 = dalloc<double>(3 * n);
    js.raw = dalloc<unsigned char>((n / JT) * g6::RAW_TILE_BYTES);
    js.v64 = dalloc<double4_32a>(n);
    js.a264 = dalloc<double4_32a>(n);
    js.j664 = dalloc<double4_32a>(n);
    js.idx = dalloc<int>(n);
    b->pred.pt = dalloc<float>(n * g6::JW);
    b->pred.trange = dalloc<int2>(tiles);
    b->d_tile_cluster = dalloc<int>(tiles);
    b->d_cl_jtile = dalloc<int>(ncl);
    b->d_cl_nj = dalloc<int>(ncl);
    b->h_irec = halloc<g6x_irec>(slots_i, &b->d_irec);
    b->h_out = halloc<g6x_out>(slots_i, &b->d_out);
    b->h_jsort = halloc<g6x_jrec>(slots_i, &b->d_jsort);
    b->h_err = halloc<int>(1, &b->d_err);
    if (!js.x0 || !js.raw || !js.v64
        || !js.a264 || !js.j664 || !js.idx || !b->pred.pt || !b->pred.trange
        || !b->d_tile_cluster || !b->d_cl_jtile || !b->d_cl_nj || !b->h_irec || !b->h_out
        || !b->h_jsort || !b->h_err)
        rc = G6_ENOMEM;
    if (!rc) {
        try {
            b->slot_of.assign(n, -1);
        } catch (...) {
            rc = G6_ENOMEM;
        }
    }
    if (!rc && (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess
                || cudaStreamCreateWithFlags(&b->stream2, cudaStreamNonBlocking) != cudaSuccess
                || cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess
                || cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) != cudaSuccess
                || cudaEventCreate(&b->ev_t0) != cudaSuccess
                || cudaEventCreate(&b->ev_t1) != cudaSuccess))
        rc = G6_EIO;
    if (!rc) {
        // default schedule: one class of the given variant, or a narrow
        // kernel for active sets of up to 32 and a wide one above
        if (variant >= 0)
            rc = set_schedule(b, variant, grid_mul > 0 ? grid_mul : 1, 0, -1, 0);
        else
            rc = set_schedule(b, 0, 1, 32, 3, grid_mul > 0 ? grid_mul : 2);
    }
    if (!rc) {
        std::vector<int> tc(tiles);
        for (int k = 0; k < ncl; ++k)
            for (int t = 0; t < b->ntile[k]; ++t)
                tc[b->jtile[k] + t] = k;
        *b->h_err = 0;
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

int g6x_batch_set_schedule(g6x_batch *b, int small_variant, int small_grid_mul, int threshold,
                           int large_variant, int large_grid_mul)
{
    if (!b)
        return G6_EINVAL;
    return set_schedule(b, small_variant, small_grid_mul, threshold, large_variant,
                        large_grid_mul);
}

int g6x_batch_get_schedule(const g6x_batch *b, int sched[5])
{
    if (!b || !sched)
        return G6_EINVAL;
    sched[0] = b->wc[0].variant;
    sched[1] = b->wc[0].grid_mul;
    sched[2] = b->nclass == 2 ? b->threshold : 0;
    sched[3] = b->nclass == 2 ? b->wc[1].variant : -1;
    sched[4] = b->nclass == 2 ? b->wc[1].grid_mul : 0;
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
    std::vector<StagedRec> &st = b->stage[cl];
    int s = b->slot_of[slot];
    if (s < 0) {
        try {
            st.emplace_back();
        } catch (...) {
            return G6_ENOMEM;
        }
        s = (int)st.size() - 1;
        b->slot_of[slot] = s;
    }
    g6x_jrec &r = st[s];
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
    stage_sorted(b);
    for (int k = 0; k < b->ncl; ++k) {
        b->h_ni[k] = ni[k];
        b->h_eps2[k] = eps2[k];
        b->h_t[k] = t_blk[k];
    }
    if (mode == 2)
        build_cluster_lines(b, ni);
    else
        build_class_lines(b, ni);
    int rc = 0;
    if (b->timing)
        rc = cuda_code(cudaEventRecord(b->ev_t0, b->stream));
    if (!rc) {
        if (mode == 0) {
            rc = run_graph(b);
        } else if (mode == 1) {
            rc = cuda_code(enqueue_all(b));
            b->launches += 1 + 2 * b->nclass;
        } else {
            rc = run_per_cluster(b, ni);
        }
    }
    if (!rc && b->timing)
        rc = cuda_code(cudaEventRecord(b->ev_t1, b->stream));
    if (!rc)
        rc = cuda_code(cudaStreamSynchronize(b->stream));
    if (rc)
        return rc;
    if (b->timing) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, b->ev_t0, b->ev_t1) == cudaSuccess) {
            b->gpu_ms += ms;
            ++b->timed;
        }
    }
    if (*(volatile int *)b->h_err) {
        const int code = *b->h_err;
        *(volatile int *)b->h_err = 0;
        // a launch that gave up may have left arrival counts behind
        for (int c = 0; c < b->nclass; ++c)
            if (b->wc[c].d_cnt
                && cudaMemset(b->wc[c].d_cnt, 0, (size_t)b->wc[c].gt_cap * sizeof(unsigned))
                       != cudaSuccess)
                cudaGetLastError();
        return code < 0 ? code : G6_EIO;
    }
    return 0;
}

int g6x_batch_set_timing(g6x_batch *b, int enable)
{
    if (!b)
        return G6_EINVAL;
    b->timing = enable != 0;
    b->gpu_ms = 0.0;
    b->timed = 0;
    return 0;
}

int g6x_batch_get_timing(const g6x_batch *b, double *gpu_ms, long long *calls)
{
    if (!b)
        return G6_EINVAL;
    if (gpu_ms)
        *gpu_ms = b->gpu_ms;
    if (calls)
        *calls = b->timed;
    return 0;
}

int g6x_batch_autotune(g6x_batch *b, int npat, const int ni[], const double eps2[],
                       const double t_blk[], int reps, int sched[5], double *best_ms)
{
    if (!b || npat < 1 || !ni || !eps2 || !t_blk || reps < 1)
        return G6_EINVAL;
    for (int p = 0; p < npat; ++p)
        for (int k = 0; k < b->ncl; ++k)
            if (ni[(size_t)p * b->ncl + k] < 0 || ni[(size_t)p * b->ncl + k] > b->nj[k])
                return G6_EINVAL;
    struct Cand {
        int v0, g0, th, v1, g1;
    };
    std::vector<Cand> cands;
    const int nv = g6::batch_variant_count();
    for (int v = 0; v < nv; ++v)
        for (int gm = 1; gm <= 2; ++gm)
            cands.push_back({v, gm, 0, -1, 0});
    const int ths[] = {8, 16, 32, 64, 128};
    for (int vs = 0; vs < nv; ++vs)
        for (int vl = 0; vl < nv; ++vl) {
            const g6::VariantInfo is = g6::batch_variant_info(vs), il = g6::batch_variant_info(vl);
            if (is.ti * is.nper >= il.ti * il.nper)
                continue;
            for (int th : ths)
                if (th >= is.ti * is.nper && th < il.ti * il.nper * 2)
                    cands.push_back({vs, 1, th, vl, 2});
        }
    int keep[5];
    g6x_batch_get_schedule(b, keep);
    double best = 1e300;
    Cand bc = {keep[0], keep[1], keep[2], keep[3], keep[4]};
    for (const Cand &c : cands) {
        int rc = set_schedule(b, c.v0, c.g0, c.th, c.v1, c.g1);
        if (rc == G6_ENODEV)
            continue;
        if (rc)
            return rc;
        rc = g6x_batch_calc(b, t_blk, eps2, ni, 0);           // capture + warm-up
        if (rc)
            return rc;
        const auto w0 = std::chrono::steady_clock::now();
        for (int r = 0; r < reps && !rc; ++r)
            for (int p = 0; p < npat && !rc; ++p)
                rc = g6x_batch_calc(b, t_blk, eps2, ni + (size_t)p * b->ncl, 0);
        if (rc)
            return rc;
        const double ms = 1e3
                          * std::chrono::duration<double>(std::chrono::steady_clock::now() - w0)
                                .count()
                          / (reps * npat);
        if (ms < best) {
            best = ms;
            bc = c;
        }
    }
    const int rc = set_schedule(b, bc.v0, bc.g0, bc.th, bc.v1, bc.g1);
    if (rc)
        return rc;
    if (sched)
        g6x_batch_get_schedule(b, sched);
    if (best_ms)
        *best_ms = best;
    return 0;
}

long long g6x_batch_launch_count(const g6x_batch *b) { return b ? b->launches : 0; }

}  // extern "C"

// ------------------------------------------------------------ batch driver

struct g6hb_sim {
    g6x_batch *b = nullptr;
    int ncl = 0, mode = 0;
    double eta = 0, eta_s = 0, dt_max = 0, dt_min = 0;
    double noise = 0;                        // relative force error for the time steps
    std::vector<int> n, off;                 // particles per cluster, offset into arrays
    std::vector<double> eps2;
    // One particle's state in one record: the host phases visit the active
    // particles of many clusters in scattered order, and a record costs them
    // three cache lines where separate arrays cost eight.
    struct Part {
        double x[3], v[3], a[3], j[3];       // at its time t
        double xp[3], vp[3];                 // predicted to its block time
        double t, dt;
    };
    std::vector<double> m;
    std::vector<Part> ps;
    std::vector<std::map<double, std::vector<int>>> due;
    std::vector<std::vector<int>> act;
    std::vector<double> tblk;
    std::vector<int> ni, rc;
    std::vector<int> hist;                    // recent ni patterns [HIST][ncl]
    int hist_n = 0, hist_pos = 0;
    // host work items: particles [i0, i1) of cluster k's active block
    struct Chunk {
        int k, i0, i1;
    };
    std::vector<Chunk> chunks;
    std::vector<int> crc;                     // per chunk status
    std::vector<size_t> sbase;                // per cluster: first reserved staging record
    long long nsteps = 0, nactive = 0, interactions = 0;
    double sec_gpu = 0, sec_host = 0;
};

namespace {

constexpr int HIST = 64;

double nrm(const double *p) { return std::sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]); }

int hb_send(g6hb_sim &s, int k, int q)
{
    const int p = s.off[k] + q;
    const g6hb_sim::Part &P = s.ps[p];
    double a2[3], j6[3];
    for (int d = 0; d < 3; ++d) {
        a2[d] = 0.5 * P.a[d];
        j6[d] = P.j[d] / 6.0;
    }
    return g6x_batch_set_j(s.b, k, q, q, P.t, s.m[p], j6, a2, P.v, P.x);
}

// Cluster k's next block: its earliest due time, if not past t_end.
void hb_pop(g6hb_sim &s, int k, double t_end)
{
    s.ni[k] = 0;
    if (s.due[k].empty())
        return;
    auto first = s.due[k].begin();
    if (first->first > t_end)
        return;
    s.tblk[k] = first->first;
    s.act[k].swap(first->second);
    s.due[k].erase(first);
    s.ni[k] = (int)s.act[k].size();
}

// Host prediction (Eq. 1, Eq. 2) of the active particles [i0, i1) of
// cluster k into its i-records.
void hb_predict(g6hb_sim &s, const g6hb_sim::Chunk &c)
{
    const int k = c.k;
    const double tb = s.tblk[k];
    g6x_irec *ir = g6x_batch_irecs(s.b, k);
    for (int i = c.i0; i < c.i1; ++i) {
        const int q = s.act[k][i];
        g6hb_sim::Part &P = s.ps[s.off[k] + q];
        const double h = tb - P.t;
        for (int d = 0; d < 3; ++d) {
            const double aa = P.a[d], jj = P.j[d];
            P.xp[d] = P.x[d] + h * (P.v[d] + h * (aa / 2.0 + h * jj / 6.0));
            P.vp[d] = P.v[d] + h * (aa + h * jj / 2.0);
            ir[i].x[d] = P.xp[d];
            ir[i].v[d] = P.vp[d];
        }
        ir[i].h2 = 0.0;
        ir[i].index = q;
        ir[i].pad = 0;
    }
}

// Correct the particles [i0, i1) of cluster k's block, choose their next
// steps and write their j-records into the staging records reserved for
// the block (each active particle is staged exactly once per step, and only
// here, so every slot is free).
int hb_correct(g6hb_sim &s, const g6hb_sim::Chunk &c)
{
    const int k = c.k;
    const g6x_out *o = g6x_batch_results(s.b, k);
    const double tb = s.tblk[k];
    g6x_batch *b = s.b;
    for (int i = c.i0; i < c.i1; ++i) {
        const int q = s.act[k][i];
        const int p = s.off[k] + q;
        g6hb_sim::Part &P = s.ps[p];
        double t0[1] = {P.t}, dtv[1] = {P.dt}, dn[1];
        const int rc = g6h_correct_block_ex(1, tb, t0, dtv, s.eta, s.dt_max, s.dt_min, P.xp, P.vp,
                                            P.a, P.j, o[i].acc, o[i].jerk, dn, s.noise);
        if (rc != 0)
            return rc < 0 ? rc : G6_EINVAL;
        const size_t si = s.sbase[k] + i;
        g6x_jrec &r = b->stage[k][si];
        for (int d = 0; d < 3; ++d) {
            P.x[d] = P.xp[d];
            P.v[d] = P.vp[d];
            P.a[d] = o[i].acc[d];
            P.j[d] = o[i].jerk[d];
            r.x[d] = P.x[d];
            r.v[d] = P.v[d];
            r.a2[d] = 0.5 * P.a[d];
            r.j6[d] = P.j[d] / 6.0;
        }
        P.t = tb;
        P.dt = dn[0];
        const int slot = b->jtile[k] * JT + q;
        r.mass = s.m[p];
        r.tj = tb;
        r.address = slot;
        r.index = q;
        b->slot_of[slot] = (int)si;
    }
    return 0;
}

// File cluster k's corrected particles under their next block times.
int hb_file(g6hb_sim &s, int k)
{
    if (s.ni[k] == 0)
        return 0;
    std::vector<int> *last = nullptr;
    double last_t = 0.0;
    try {
        for (int q : s.act[k]) {
            const int p = s.off[k] + q;
            const double tn = s.ps[p].t + s.ps[p].dt;
            if (!last || tn != last_t) {
                last = &s.due[k][tn];
                last_t = tn;
            }
            last->push_back(q);
        }
    } catch (...) {
        return G6_ENOMEM;
    }
    s.act[k].clear();
    return 0;
}

// Drop the staging records reserved for a block that failed to correct.
void hb_unstage(g6hb_sim &s)
{
    g6x_batch *b = s.b;
    for (int k = 0; k < s.ncl; ++k) {
        std::vector<StagedRec> &st = b->stage[k];
        for (size_t i = s.sbase[k]; i < st.size(); ++i) {
            const int slot = b->jtile[k] * JT + s.act[k][i - s.sbase[k]];
            if (b->slot_of[slot] == (int)i)
                b->slot_of[slot] = -1;
        }
        st.resize(s.sbase[k]);
    }
}

constexpr int CHUNK = 96;

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
        s->ps.assign(tot, g6hb_sim::Part{});
        for (int p = 0; p < tot; ++p) {
            g6hb_sim::Part &P = s->ps[p];
            for (int d = 0; d < 3; ++d) {
                P.x[d] = x[3 * (size_t)p + d];
                P.v[d] = v[3 * (size_t)p + d];
            }
            P.t = 0.0;
            P.dt = dt_max;
        }
        s->due.resize(ncl);
        s->act.resize(ncl);
        s->tblk.assign(ncl, 0.0);
        s->ni.assign(ncl, 0);
        s->rc.assign(ncl, 0);
        s->hist.assign((size_t)HIST * ncl, 0);
        s->sbase.assign(ncl, 0);
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
            const g6hb_sim::Part &P = s->ps[s->off[k] + q];
            for (int d = 0; d < 3; ++d) {
                ir[q].x[d] = P.x[d];
                ir[q].v[d] = P.v[d];
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
            g6hb_sim::Part &P = s->ps[s->off[k] + q];
            for (int d = 0; d < 3; ++d) {
                P.a[d] = o[q].acc[d];
                P.j[d] = o[q].jerk[d];
            }
            const double req = s->eta_s * nrm(P.a) / nrm(P.j);
            double d = dt_max;
            while (d > req)
                d *= 0.5;
            if (d < dt_min)
                rc = G6_EINVAL;
            P.dt = d;
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
    g6::parallel_run(s->ncl, [s, t_end](int k) { hb_pop(*s, k, t_end); });
    int stepping = 0;
    s->chunks.clear();
    for (int k = 0; k < s->ncl; ++k)
        if (s->ni[k]) {
            ++stepping;
            s->nactive += s->ni[k];
            s->interactions += (long long)s->ni[k] * s->n[k];
            for (int i0 = 0; i0 < s->ni[k]; i0 += CHUNK)
                s->chunks.push_back({k, i0, std::min(s->ni[k], i0 + CHUNK)});
        }
    if (stepping == 0)
        return 0;
    const int nch = (int)s->chunks.size();
    g6::parallel_run(nch, [s](int c) { hb_predict(*s, s->chunks[c]); });
    std::memcpy(&s->hist[(size_t)s->hist_pos * s->ncl], s->ni.data(), sizeof(int) * s->ncl);
    s->hist_pos = (s->hist_pos + 1) % HIST;
    s->hist_n = std::min(s->hist_n + 1, HIST);
    auto w1 = std::chrono::steady_clock::now();
    int rc = g6x_batch_calc(s->b, s->tblk.data(), s->eps2.data(), s->ni.data(), s->mode);
    if (rc)
        return rc;
    auto w2 = std::chrono::steady_clock::now();
    // reserve the block's staging records, correct in chunks, then file the
    // particles under their next times
    try {
        for (int k = 0; k < s->ncl; ++k) {
            s->sbase[k] = s->b->stage[k].size();
            if (s->ni[k])
                s->b->stage[k].resize(s->sbase[k] + s->ni[k]);
        }
        s->crc.assign(nch, 0);
    } catch (...) {
        return G6_ENOMEM;
    }
    g6::parallel_run(nch, [s](int c) { s->crc[c] = hb_correct(*s, s->chunks[c]); });
    for (int c = 0; c < nch; ++c)
        if (s->crc[c]) {
            hb_unstage(*s);
            return s->crc[c];
        }
    g6::parallel_run(s->ncl, [s](int k) { s->rc[k] = hb_file(*s, k); });
    for (int k = 0; k < s->ncl; ++k)
        if (s->rc[k])
            return s->rc[k];
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

int g6hb_autotune(g6hb_sim *s, int reps, int sched[5], double *best_ms)
{
    if (!s || reps < 1)
        return G6_EINVAL;
    if (s->hist_n == 0)
        return G6_EBUSY;
    // the tuning calls overwrite the results and predicted j, both of which
    // the next step recomputes; staged records are applied by the first call
    return g6x_batch_autotune(s->b, s->hist_n, s->hist.data(), s->eps2.data(), s->tblk.data(),
                              reps, sched, best_ms);
}

int g6hb_set_schedule(g6hb_sim *s, int small_variant, int small_grid_mul, int threshold,
                      int large_variant, int large_grid_mul)
{
    if (!s)
        return G6_EINVAL;
    return g6x_batch_set_schedule(s->b, small_variant, small_grid_mul, threshold,
                                  large_variant, large_grid_mul);
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
    for (size_t p = 0; p < tot; ++p) {
        const g6hb_sim::Part &P = s->ps[p];
        for (int d = 0; d < 3; ++d) {
            if (x)
                x[3 * p + d] = P.x[d];
            if (v)
                v[3 * p + d] = P.v[d];
        }
        if (t)
            t[p] = P.t;
    }
    return 0;
}

int g6hb_get_state_ex(const g6hb_sim *s, double *x, double *v, double *acc, double *jerk,
                      double *t, double *dt)
{
    int rc = g6hb_get_state(s, x, v, t);
    if (rc)
        return rc;
    const size_t tot = s->m.size();
    for (size_t p = 0; p < tot; ++p) {
        const g6hb_sim::Part &P = s->ps[p];
        for (int d = 0; d < 3; ++d) {
            if (acc)
                acc[3 * p + d] = P.a[d];
            if (jerk)
                jerk[3 * p + d] = P.j[d];
        }
        if (dt)
            dt[p] = P.dt;
    }
    return 0;
}

int g6hb_set_force_noise(g6hb_sim *s, double rel)
{
    if (!s || !(rel >= 0) || !(rel < 1))
        return G6_EINVAL;
    s->noise = rel;
    return 0;
}

int g6hb_set_mode(g6hb_sim *s, int mode)
{
    if (!s || mode < 0 || mode > 2)
        return G6_EINVAL;
    s->mode = mode;
    return 0;
}

g6x_batch *g6hb_batch(g6hb_sim *s) { return s ? s->b : nullptr; }

void g6hb_destroy(g6hb_sim *s)
{
    if (!s)
        return;
    g6x_batch_destroy(s->b);
    delete s;
}

}  // extern "C"
